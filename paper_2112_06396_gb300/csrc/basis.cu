// basis.cu -- fast basis conversion, the NewLimb step of ModUp (Algorithm 6)
// and of ModDown / Rescale (table "CKKS Subroutines"); slot-wise access
// pattern (table "Data dependencies and access pattern").
//
// For every coefficient n, with source limbs x_i (coefficient form):
//   y_i = [(x_i + add_i) * mul_i]_{q_i}          (Shoup, constant mul_i)
//   z_t = (sum_i y_i * mat[t][i]  mod t) - sub_t (128-bit exact sum, one reduction)
// A thread owns two adjacent coefficients (16-byte loads and stores), keeps its
// y_i in registers and produces every target limb of its chunk, so each source
// word is read once per chunk and each target word is written once.
#include "batch.cuh"
#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

#include <algorithm>

namespace ckks {

template <int NS>
__global__ void __launch_bounds__(256) bconv_kernel(BConvLaunch L, const PrimeInfo *__restrict__ pinfo, int logN) {
    const int grp = blockIdx.y / L.chunks;
    const int chunk = blockIdx.y % L.chunks;
    const BConvGroup G = L.g[grp];
    const BConvPlan *__restrict__ plan = G.plan;
    const size_t N = size_t(1) << logN;
    const size_t n0 = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int n_src = plan->n_src;
    const int t0 = chunk * L.chunk;
    int t1 = t0 + L.chunk;
    if (t1 > plan->n_dst) t1 = plan->n_dst;

    u64 y0[NS], y1[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) {
        if (i < n_src) {
            const u64 p = pinfo[plan->src_prime[i]].p;
            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(G.src + size_t(i) * N + n0);
            const u64 ad = plan->src_add[i], m = plan->src_mul[i], ms = plan->src_mul_s[i];
            y0[i] = shoup_mul(add_mod(x.x, ad, p), m, ms, p);
            y1[i] = shoup_mul(add_mod(x.y, ad, p), m, ms, p);
        } else {
            y0[i] = 0;
            y1[i] = 0;
        }
    }
    for (int t = t0; t < t1; t++) {
        const PrimeInfo P = pinfo[plan->dst_prime[t]];
        const u64 *__restrict__ row = plan->mat[t];
        u64 lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
        for (int i = 0; i < NS; i++) {
            if (i < n_src) {
                const u64 c = row[i];
                mac128(lo0, hi0, y0[i], c);
                mac128(lo1, hi1, y1[i], c);
            }
        }
        const u64 sub = plan->dst_sub[t];
        ulonglong2 z;
        z.x = sub_mod(reduce128(lo0, hi0, P), sub, P.p);
        z.y = sub_mod(reduce128(lo1, hi1, P), sub, P.p);
        *reinterpret_cast<ulonglong2 *>(G.dst + size_t(plan->dst_pos[t]) * N + n0) = z;
    }
}

// Split variant (primes below 2^57).  y_i and the constants are cut into
// W-bit halves (W = ceil(bits(max prime)/2)).  With C = mat[t][i] = Ch*2^W + Cl
// and D = [C * 2^W]_t = Dh*2^W + Dl,
//   y_i * C == 2^W * (yh*Dh + yl*Ch) + (yh*Dl + yl*Cl)   (mod t),
// so every term is four 32x32->64 multiply-adds into two 64-bit accumulators
// A and B (no 64-bit high products, no carries), and each output needs one
// Shoup fold of A by [2^W]_t and one final reduction.  A CTA converts all
// targets of its group for 256 coefficients; the constants of the group sit
// in shared memory and every source word is read and scaled exactly once.
template <int NS, class GMAP>
__global__ void __launch_bounds__(128, 7) bconv_split_kernel(const __grid_constant__ GMAP gm, int chunks, int chunk,
                                                          const PrimeInfo *__restrict__ pinfo, int logN, int W) {
    extern __shared__ uint4 smat[];  // [n_dst][NS] then the per-target constants
    const BConvGroup G = gm.get(blockIdx.y / chunks);
    const BConvPlan *__restrict__ plan = G.plan;
    const size_t N = size_t(1) << logN;
    const int n_src = plan->n_src;
    const int t0 = (blockIdx.y % chunks) * chunk;  // this CTA's targets: t0 .. t0+n_dst-1
    const int n_dst = min(plan->n_dst - t0, chunk);
    if (n_dst <= 0) return;
    struct Dst {
        u64 p, one_s, rw, rw_s, sub, pos;
    };
    Dst *sdst = reinterpret_cast<Dst *>(smat + n_dst * NS);
    for (int e = threadIdx.x; e < n_dst * NS; e += blockDim.x) {
        const int t = e / NS, i = e % NS;
        smat[e] = i < n_src ? plan->matw[t0 + t][i] : make_uint4(0, 0, 0, 0);
    }
    for (int t = threadIdx.x; t < n_dst; t += blockDim.x) {
        const int tt = t0 + t;
        const PrimeInfo &P = pinfo[plan->dst_prime[tt]];
        sdst[t] = Dst{P.p, P.one_s, plan->dst_rw[tt], plan->dst_rw_s[tt], plan->dst_sub[tt], plan->dst_pos[tt]};
    }
    const size_t n0 = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) * 2;
    const u64 mask = (u64(1) << W) - 1;
    uint32_t yh0[NS], yl0[NS], yh1[NS], yl1[NS];
#pragma unroll
    for (int i = 0; i < NS; i++) {
        // y must be the reduced residue [(x + add) * mul]_q: the conversion's
        // integer result (and its multiple-of-Q error term) depends on the
        // representative, so a lazy y would change the bits of the output.
        u64 y0 = 0, y1 = 0;
        if (i < n_src) {
            const u64 q = pinfo[plan->src_prime[i]].p, nq = u64(0) - q;
            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(G.src + size_t(i) * N + n0);
            const u64 ad = plan->src_add[i], m = plan->src_mul[i], ms = plan->src_mul_s[i];
            y0 = csub(csub(shoup_approx(x.x + ad, m, ms, nq), 2 * q), q);
            y1 = csub(csub(shoup_approx(x.y + ad, m, ms, nq), 2 * q), q);
        }
        yh0[i] = uint32_t(y0 >> W);
        yl0[i] = uint32_t(y0 & mask);
        yh1[i] = uint32_t(y1 >> W);
        yl1[i] = uint32_t(y1 & mask);
    }
    __syncthreads();
#pragma unroll 2
    for (int t = 0; t < n_dst; t++) {
        // two accumulators per sum (hi-word and lo-word products) keep the
        // multiply-add chains short
        u64 A0 = 0, B0 = 0, A1 = 0, B1 = 0, C0 = 0, D0 = 0, C1 = 0, D1 = 0;
#pragma unroll
        for (int i = 0; i < NS; i++) {
            const uint4 m = smat[t * NS + i];
            mad_wide(A0, yh0[i], m.x);
            mad_wide(C0, yl0[i], m.y);
            mad_wide(B0, yh0[i], m.z);
            mad_wide(D0, yl0[i], m.w);
            mad_wide(A1, yh1[i], m.x);
            mad_wide(C1, yl1[i], m.y);
            mad_wide(B1, yh1[i], m.z);
            mad_wide(D1, yl1[i], m.w);
        }
        A0 += C0;
        B0 += D0;
        A1 += C1;
        B1 += D1;
        const Dst d = sdst[t];
        const u64 np = u64(0) - d.p;
        // A, B < 2^(2W+8) <= 2^62 and the folded A < 3t: the sum stays below
        // 2^64.  The output is left in [0, 4t): z + (t - sub) with z in [0, 3t).
        // Its only consumer is the lazy forward NTT, whose bound allows inputs
        // below 4t (see ntt.cu).
        u64 v0 = B0 + shoup_approx(A0, d.rw, d.rw_s, np);
        u64 v1 = B1 + shoup_approx(A1, d.rw, d.rw_s, np);
        const u64 off = d.p - d.sub;
        v0 = shoup_one(v0, d.one_s, np) + off;
        v1 = shoup_one(v1, d.one_s, np) + off;
        *reinterpret_cast<ulonglong2 *>(G.dst + size_t(d.pos) * N + n0) = make_ulonglong2(v0, v1);
    }
}

// Tensor-core variant (tcgen05).  The conversion of 128 coefficients to a
// chunk of targets is a matrix product over the integers: with the reduced
// y_i cut into bytes y_ij (j = 0..6, y < 2^56) and M_tij = [2^(8j) C_ti]_t cut
// into bytes m_tijc,
//   sum_i y_i C_ti == sum_c 2^(8c) S_tc  (mod t),  S_tc = sum_ij y_ij m_tijc,
// and every S_tc (at most 16 sources: below 112 * 255^2 < 2^23) is an exact
// integer in f16 x f16 -> f32 arithmetic.  A (128 coefficients x 8 KG bytes,
// f16) is built in shared memory from the sources; B (targets x 8 rows c, same
// K) is the plan's precomputed image; the f32 sums land in tensor memory,
// column 8t + c of the coefficient's lane.  A constant column (2048 in A, 4096
// in B) adds 2^23 to every sum, so the bits of the f32 result read as the
// integer 0x4B000000 + S_tc with no conversion; the epilogue combines the
// seven columns of a target with wide multiply-adds into lo + hi * 2^32,
// folds hi by [2^32]_t, adds the plan's dst_off (which removes the biases and
// sub_t) and reduces once: the output is in [0, 3t) for the lazy forward NTT.
constexpr uint32_t kTcWaitPolls = 1u << 24;  // about a second of 64 ns sleeps

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
// bytes 2k, 2k+1 of w as two f16 values: (0x6400 | byte) is the f16 1024 + byte,
// and subtracting 1024 is exact
__device__ __forceinline__ uint32_t byte_pair_f16(uint32_t w, uint32_t sel) {
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(prmt(w, 0x64646464u, sel)), "r"(0x64006400u));
    return d;
}

template <int KG, class GMAP>
__global__ void __launch_bounds__(256, 2) bconv_tc_kernel(const __grid_constant__ GMAP gm, int chunks, int chunk,
                                                         const PrimeInfo *__restrict__ pinfo, int logN,
                                                         int *__restrict__ status) {
    extern __shared__ __align__(1024) uint4 tsm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    struct Dst {
        u64 p, one_s, r32, r32_s, off;
        uint32_t pos, pad;
    };
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BConvGroup G = gm.get(blockIdx.y / chunks);
    const BConvPlan *__restrict__ plan = G.plan;
    const uint32_t N = 1u << logN;
    const int t0 = (blockIdx.y % chunks) * chunk;
    const int nd = min(plan->n_dst - t0, chunk);
    if (nd <= 0) return;
    const int ntp = (nd + 1) & ~1;  // N of the MMA = 8 * ntp, a multiple of 16
    const int n_src = plan->n_src;
    uint4 *As = tsm;                                        // [16 row groups][KG][8 rows]
    uint4 *Bs = tsm + 128 * KG;                             // [ntp][KG][8 rows]
    Dst *sd = reinterpret_cast<Dst *>(Bs + size_t(ntp) * KG * 8);  // [chunk]

    if (warp == 0) tc::tmem_alloc(&tslot, 256);
    if (tid == 32) tc::mbar_init(&mbar, 1);
    const uint4 *__restrict__ img = plan->tc_img + size_t(t0) * KG * 8;
    for (int i = tid; i < ntp * KG * 8; i += blockDim.x) Bs[i] = img[i];
    for (int t = tid; t < nd; t += blockDim.x) {
        const int tt = t0 + t;
        const PrimeInfo &P = pinfo[plan->dst_prime[tt]];
        sd[t] = Dst{P.p, P.one_s, plan->dst_r32[tt], plan->dst_r32_s[tt], plan->dst_off[tt], plan->dst_pos[tt], 0};
    }
    // A: row m is coefficient n0 + m; group g < n_src holds the bytes of the
    // reduced y_g (see bconv_split_kernel: the representative matters), group
    // KG-1 the bias entry, the rest zeros
    const uint32_t n0 = blockIdx.x * 128u;
    {
        const int m = tid & 127;
        uint4 *row = As + (m >> 3) * (KG * 8) + (m & 7);
        for (int g = tid >> 7; g < KG; g += 2) {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (g < n_src) {
                const u64 q = pinfo[plan->src_prime[g]].p, nq = u64(0) - q;
                const u64 x = G.src[size_t(g) * N + n0 + m];
                const u64 y =
                    csub(csub(shoup_approx(x + plan->src_add[g], plan->src_mul[g], plan->src_mul_s[g], nq), 2 * q), q);
                const uint32_t w0 = uint32_t(y), w1 = uint32_t(y >> 32);
                v = make_uint4(byte_pair_f16(w0, 0x4140u), byte_pair_f16(w0, 0x4342u), byte_pair_f16(w1, 0x4140u),
                               byte_pair_f16(w1, 0x4342u));
            } else if (g == KG - 1) {
                v.x = 0x6800u;  // f16 2048
            }
            row[g * 8] = v;
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    if (tid == 0) {
        const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs);
        const uint32_t idesc = tc::idesc_f16_f32(128, 8 * ntp);
#pragma unroll
        for (int s = 0; s < KG / 2; ++s)
            tc::mma_f16(taddr, tc::desc_kmajor(a0 + 256u * s, 128u, 128u * KG),
                        tc::desc_kmajor(b0 + 256u * s, 128u, 128u * KG), idesc, s > 0);
        tc::mma_commit(&mbar);
    }
    bool ok = tc::mbar_wait(&mbar, 0, kTcWaitPolls);
    tc::fence_after_sync();
    if (ok) {
        // warp w reads lanes 32*(w % 4) .. +31 (its coefficients) for half the targets
        const int quarter = warp & 3, half = warp >> 2;
        const int h0 = (nd + 1) >> 1;
        const int tb = half ? h0 : 0, te = half ? nd : h0;
        const uint32_t laddr = taddr + (uint32_t(quarter * 32) << 16);
        const uint32_t n = n0 + uint32_t(quarter * 32 + lane);
        for (int t = tb; t < te; t += 2) {
            uint32_t r[16];
            tc::tmem_ld16(laddr + uint32_t(t * 8), r);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (t + j >= te) break;
                const Dst &d = sd[t + j];
                const uint32_t *b = r + 8 * j;
                u64 lo = b[0], hi = b[4];
                mad_wide(lo, b[1], 1u << 8);
                mad_wide(lo, b[2], 1u << 16);
                mad_wide(lo, b[3], 1u << 24);
                mad_wide(hi, b[5], 1u << 8);
                mad_wide(hi, b[6], 1u << 16);
                const u64 np = u64(0) - d.p;
                const u64 v = shoup_one(lo + shoup_approx(hi, d.r32, d.r32_s, np) + d.off, d.one_s, np);
                G.dst[size_t(d.pos) * N + n] = v;
            }
        }
    } else {
        if (lane == 0) atomicOr(status, 1);
        // the multiplies may still be running: wait once more before freeing their memory
        tc::mbar_wait(&mbar, 0, kTcWaitPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 256);
}

template <int KG, class GMAP>
static void launch_tc_kg(const ckks_ctx *ctx, const GMAP &gm, int ngroups, int chunks, int chunk, cudaStream_t st) {
    const int ntp = (chunk + 1) & ~1;
    // at least 80 KiB: no more than two CTAs share an SM, as many as fit their
    // 256 tensor-memory columns (a third would wait inside tcgen05.alloc)
    const size_t need = (size_t(128) * KG + size_t(ntp) * KG * 8) * sizeof(uint4) + size_t(chunk) * 48;
    const size_t smem = std::max<size_t>(need, 80 * 1024);
    auto kern = bconv_tc_kernel<KG, GMAP>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    dim3 grid(unsigned(ctx->N / 128), unsigned(ngroups * chunks));
    kern<<<grid, 256, smem, st>>>(gm, chunks, chunk, ctx->d_pinfo, ctx->logN, ctx->d_status);
}

// Tensor-core conversion over `ngroups` groups of up to n_all targets each,
// in chunks of at most 32 targets (256 tensor-memory columns).
template <class GMAP>
static cudaError_t launch_tc(const ckks_ctx *ctx, const GMAP &gm, int ngroups, int n_all, cudaStream_t st) {
    const int chunks = (n_all + 31) / 32;
    const int chunk = (n_all + chunks - 1) / chunks;
    ProfScope ps(ctx, K_BCONV, double(ngroups) * n_all, st);
    switch (ctx->tc_kg) {
    case 4: launch_tc_kg<4>(ctx, gm, ngroups, chunks, chunk, st); break;
    case 6: launch_tc_kg<6>(ctx, gm, ngroups, chunks, chunk, st); break;
    case 8: launch_tc_kg<8>(ctx, gm, ngroups, chunks, chunk, st); break;
    case 10: launch_tc_kg<10>(ctx, gm, ngroups, chunks, chunk, st); break;
    case 12: launch_tc_kg<12>(ctx, gm, ngroups, chunks, chunk, st); break;
    case 14: launch_tc_kg<14>(ctx, gm, ngroups, chunks, chunk, st); break;
    case 16: launch_tc_kg<16>(ctx, gm, ngroups, chunks, chunk, st); break;
    case 18: launch_tc_kg<18>(ctx, gm, ngroups, chunks, chunk, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Split conversion over `ngroups` groups of up to n_all targets each: targets
// in chunks of at most 12 per CTA row (enough CTAs to fill the SMs while each
// source word is still scaled once per 12 targets).
template <class GMAP>
static cudaError_t launch_split(const ckks_ctx *ctx, const GMAP &gm, int ngroups, int n_all, int max_src,
                                cudaStream_t st) {
    if (ctx->tc_kg && ctx->tc_on) return launch_tc(ctx, gm, ngroups, n_all, st);
    const int chunks = (n_all + 11) / 12;
    const int chunk = (n_all + chunks - 1) / chunks;
    const int tpb = 128;
    dim3 grid(unsigned((ctx->N / 2 + tpb - 1) / tpb), unsigned(ngroups * chunks));
    ProfScope ps(ctx, K_BCONV, double(ngroups) * n_all, st);
    const int W = ctx->split_bits;
    auto smem = [&](int ns) { return size_t(chunk) * ns * sizeof(uint4) + size_t(chunk) * 48; };
#define CKKS_BCONV_SPLIT(NSV)                                                                                      \
    do {                                                                                                           \
        auto kern = bconv_split_kernel<NSV, GMAP>;                                                                 \
        if (smem(NSV) > 48 * 1024)                                                                                 \
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem(NSV)));               \
        kern<<<grid, tpb, smem(NSV), st>>>(gm, chunks, chunk, ctx->d_pinfo, ctx->logN, W);                         \
    } while (0)
    if (max_src <= 1) CKKS_BCONV_SPLIT(1);
    else if (max_src <= 2) CKKS_BCONV_SPLIT(2);
    else if (max_src <= 3) CKKS_BCONV_SPLIT(3);
    else if (max_src <= 4) CKKS_BCONV_SPLIT(4);
    else if (max_src <= 6) CKKS_BCONV_SPLIT(6);
    else if (max_src <= 8) CKKS_BCONV_SPLIT(8);
    else if (max_src <= 12) CKKS_BCONV_SPLIT(12);
    else if (max_src <= 16) CKKS_BCONV_SPLIT(16);
    else if (max_src <= 24) CKKS_BCONV_SPLIT(24);
    else CKKS_BCONV_SPLIT(32);
#undef CKKS_BCONV_SPLIT
    return cudaGetLastError();
}

// The basis conversions of one batched phase: ModUp digits (GM_MODUP), the
// ModDown of both polynomials (GM_MODDOWN) or the Rescale of both polynomials
// of the Mult entries (GM_RESCALE).  Needs the split conversion.
cudaError_t launch_bconv_batch(const ckks_ctx *ctx, const KsBatchDesc &d, int down, cudaStream_t st) {
    GroupMapBatch gm;
    gm.d = d;
    gm.down = down;
    gm.modup = ctx->d_modup;
    gm.moddown = ctx->d_moddown;
    gm.rescale = ctx->d_rescale;
    gm.merged = ctx->d_mdmerged;
    int groups = 0, n_all = 0, max_src = 1;
    for (int c = 0; c < d.n; ++c) {
        const CtDesc &x = d.ct[c];
        const int ell = x.ell, beta = (ell + d.alpha - 1) / d.alpha;
        gm.d.pre[c] = groups;
        if (down == GM_MODUP) {
            groups += beta;
            n_all = std::max(n_all, ell + d.k - std::min(d.alpha, ell - (beta - 1) * d.alpha));
            max_src = std::max(max_src, d.alpha);
        } else if (down == GM_MODDOWN) {
            groups += 2;
            n_all = std::max(n_all, ell - x.merged);
            max_src = std::max(max_src, d.k + x.merged);
        } else if (x.ra != nullptr) {
            groups += 2;
            n_all = std::max(n_all, ell - 1);
        }
    }
    gm.d.pre[d.n] = groups;
    if (groups == 0 || n_all == 0) return cudaSuccess;
    return launch_split(ctx, gm, groups, n_all, max_src, st);
}

cudaError_t launch_bconv(const ckks_ctx *ctx, const BConvLaunch &l, int max_src, cudaStream_t st) {
    if (l.ngroups == 0) return cudaSuccess;
    const int threads = 256;
    if (ctx->split_bits && max_src <= kMaxSrc) {
        GroupMapList gm;
        gm.l = l;
        return launch_split(ctx, gm, l.ngroups, l.chunk * l.chunks, max_src, st);
    }
    dim3 grid(unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(l.ngroups * l.chunks));
    ProfScope ps(ctx, K_BCONV, double(l.ngroups) * l.chunk, st);
    if (max_src <= 1) bconv_kernel<1><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 2) bconv_kernel<2><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 3) bconv_kernel<3><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 4) bconv_kernel<4><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 6) bconv_kernel<6><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 8) bconv_kernel<8><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 12) bconv_kernel<12><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 16) bconv_kernel<16><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else if (max_src <= 24) bconv_kernel<24><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    else bconv_kernel<32><<<grid, threads, 0, st>>>(l, ctx->d_pinfo, ctx->logN);
    return cudaGetLastError();
}

}  // namespace ckks
