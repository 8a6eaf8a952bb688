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
#include "launch_policy.h"
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
// integer 0x4B000000 + S_tc with no conversion; the epilogue recombines the
// seven columns of a target (the arithmetic is spelled out before the kernel).
constexpr uint64_t kTcWaitNs = 1000000000ull;  // give up after a second (ns)

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

// Persistent, warp-specialised: a CTA owns one group and one target chunk
// (its B image is loaded once) and walks over tiles of 128 coefficients
// blockIdx.x, blockIdx.x + gridDim.x, ...  Lane 0 of warp 21 copies the B
// image once and streams the source words of the coming tiles (1 KiB per
// source limb) into a ring of kTcXStages shared-memory stages with bulk
// copies; warps 12-19 turn a staged tile into the A operand (one of two
// stages; two threads per row, alternate sources); lane 0 of warp 20 issues the
// MMAs of a tile into one of two tensor-memory accumulators (columns 0 and
// 256) and commits them to the stage's "A empty" and "D full" mbarriers;
// warps 0-11 read a finished accumulator (warp w: lanes 32*(w % 4), every
// third group of four targets), reduce and store, then free it.  Every wait is
// bounded; a role that gives up raises the CTA's abort flag and the context's
// status word.
//
// Epilogue arithmetic, with b_c = 0x4B000000 + S_c the f32 bits of column c:
//   lo = sum_{c<5} 2^(8c) S_c  (< 2^55 for 16 sources),  hi = S_5 + 2^8 S_6 (< 2^32),
//   out = lo + hi * [2^40]_t (an exact 32-bit Shoup product, < 2t) + [-sub]_t,
// below 8t for the lazy forward NTT when the context's primes are large
// enough (tc_lazy), else reduced once more to [0, 3t).
constexpr int kTcEpiWarps = 12, kTcProdWarps = 8, kTcThreads = (kTcEpiWarps + kTcProdWarps + 2) * 32;
constexpr int kTcXStages = 4;

template <int KG, class GMAP>
__global__ void __launch_bounds__(kTcThreads, 1)
    bconv_tc_kernel(const __grid_constant__ GMAP gm, int chunks, int chunk, const PrimeInfo *__restrict__ pinfo,
                    int logN, int lazy, int *__restrict__ status) {
    extern __shared__ __align__(1024) uint4 tsm[];
    __shared__ uint64_t a_full[2], a_empty[2], d_full[2], d_empty[2], x_full[kTcXStages], x_empty[kTcXStages], b_full;
    __shared__ uint32_t tslot;
    __shared__ volatile int abort_flag;
    struct Src {
        u64 q, add, mul, mul_s;
    };
    __shared__ Src ssrc[KG];
    struct Dst {
        u64 r40, r40_s, off, np, one_s;
        u64 *out;
    };
    constexpr int kMmaWarp = kTcEpiWarps + kTcProdWarps, kLoadWarp = kMmaWarp + 1;
    // f32 bits of 2^23 + S (the MMA's bias), and the bias of the low word lo
    constexpr uint32_t kBias = 0x4B000000u;
    constexpr u64 kLoBias = u64(kBias) * (1ull + (1ull << 8) + (1ull << 16) + (1ull << 24) + (1ull << 32));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const BConvGroup G = gm.get(blockIdx.y / chunks);
    const BConvPlan *__restrict__ plan = G.plan;
    const uint32_t N = 1u << logN;
    const int t0 = (blockIdx.y % chunks) * chunk;
    const int nd = min(plan->n_dst - t0, chunk);
    if (nd <= 0) return;
    const int ntp = (nd + 3) & ~3;  // N of the MMA = 8 * ntp: whole groups of four targets
    const int n_src = plan->n_src;
    const int ntiles = int(N >> 7);
    uint4 *As = tsm;                                               // [2][16 row groups][KG][8 rows]
    u64 *Xs = reinterpret_cast<u64 *>(tsm + 2 * 128 * KG);         // [kTcXStages][KG - 1][128]
    uint4 *Bs = tsm + 2 * 128 * KG + kTcXStages * (KG - 1) * 64;   // [ntp][KG][8 rows]
    Dst *sd = reinterpret_cast<Dst *>(Bs + size_t(ntp) * KG * 8);  // [chunk]

    if (warp == kMmaWarp) tc::tmem_alloc(&tslot, 512);
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&a_full[s], kTcProdWarps * 32);
            tc::mbar_init(&a_empty[s], 1);
            tc::mbar_init(&d_full[s], 1);
            tc::mbar_init(&d_empty[s], kTcEpiWarps);
        }
        for (int s = 0; s < kTcXStages; ++s) {
            tc::mbar_init(&x_full[s], 1);
            tc::mbar_init(&x_empty[s], kTcProdWarps * 32);
        }
        tc::mbar_init(&b_full, 1);
        abort_flag = 0;
    }
    for (int t = tid; t < nd; t += kTcThreads) {
        const int tt = t0 + t;
        const PrimeInfo &P = pinfo[plan->dst_prime[tt]];
        sd[t] = Dst{plan->dst_r40[tt], plan->dst_r40_s[tt], plan->dst_off[tt] - kLoBias, u64(0) - P.p, P.one_s,
                    G.dst + size_t(plan->dst_pos[tt]) * N};
    }
    if (tid < n_src)
        ssrc[tid] = Src{pinfo[plan->src_prime[tid]].p, plan->src_add[tid], plan->src_mul[tid], plan->src_mul_s[tid]};
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    auto give_up = [&]() {
        abort_flag = 1;
        atomicOr(status, 1);
    };

    if (warp == kLoadWarp) {
        // ---- loader: the B image, then the n_src source slices (1 KiB each) of every tile
        if (lane == 0) {
            const uint32_t bbytes = uint32_t(ntp) * KG * 128u;
            tc::mbar_arrive_expect_tx(&b_full, bbytes);
            tc::bulk_g2s(Bs, plan->tc_img + size_t(t0) * KG * 8, bbytes, &b_full);
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const int xs = it % kTcXStages;
                if (it >= kTcXStages &&
                    !tc::mbar_wait(&x_empty[xs], ((it / kTcXStages) - 1) & 1, kTcWaitNs, &abort_flag)) {
                    give_up();
                    break;
                }
                // order the producers' reads of the stage (generic proxy), seen
                // through x_empty, before the bulk copies that overwrite it
                tc::fence_async_smem();
                tc::mbar_arrive_expect_tx(&x_full[xs], uint32_t(n_src) * 1024u);
                for (int g = 0; g < n_src; ++g)
                    tc::bulk_g2s(Xs + (size_t(xs) * (KG - 1) + g) * 128, G.src + size_t(g) * N + size_t(tile) * 128,
                                 1024u, &x_full[xs]);
            }
            // no copy may still be in flight when the CTA ends (they all have
            // landed unless another role gave up)
            for (int j = it - 1; j >= 0 && j >= it - kTcXStages; --j)
                tc::mbar_wait(&x_full[j % kTcXStages], (j / kTcXStages) & 1, kTcWaitNs);
            tc::mbar_wait(&b_full, 0, kTcWaitNs);
        }
        __syncwarp();
    } else if (warp >= kTcEpiWarps && warp < kMmaWarp) {
        // ---- producers: thread = row m of the A tile (coefficient n0 + m);
        // group g < n_src holds the bytes of the reduced y_g (see
        // bconv_split_kernel: the representative matters), group KG-1 the
        // bias entry 2048, the rest zeros
        const int pt = tid - kTcEpiWarps * 32;
        // row m; the groups g = 2i + par of kPars parities starting at par0
        constexpr int kPars = 256 / (kTcProdWarps * 32);
        const int m = pt & 127, par0 = (pt >> 7) * kPars;
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it & 1, xs = it % kTcXStages;
            if ((it >= 2 && !tc::mbar_wait(&a_empty[s], ((it >> 1) & 1) ^ 1, kTcWaitNs, &abort_flag)) ||
                !tc::mbar_wait(&x_full[xs], (it / kTcXStages) & 1, kTcWaitNs, &abort_flag)) {
                give_up();
                break;
            }
            const u64 *xrow = Xs + size_t(xs) * (KG - 1) * 128 + m;
            uint4 *row = As + s * (128 * KG) + (m >> 3) * (KG * 8) + (m & 7);
#pragma unroll
            for (int pr = 0; pr < kPars; ++pr) {
            const int par = par0 + pr;
            u64 x[KG / 2];
#pragma unroll
            for (int i = 0; i < KG / 2; ++i) {
                const int g = 2 * i + par;
                x[i] = g < n_src ? xrow[g * 128] : 0;
            }
#pragma unroll
            for (int i = 0; i < KG / 2; ++i) {
                const int g = 2 * i + par;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (g < n_src) {
                    const Src c = ssrc[g];
                    const u64 y = csub(csub(shoup_approx(x[i] + c.add, c.mul, c.mul_s, u64(0) - c.q), 2 * c.q), c.q);
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
            // the source stage is handed back only now, after every value read
            // from it has been used: releasing it right after the loads let the
            // next bulk copy into the stage land before some of them completed
            // when the SM was shared with other kernels (wrong sums, no error)
            tc::mbar_arrive(&x_empty[xs]);
            tc::mbar_arrive(&a_full[s]);
        }
    } else if (warp == kMmaWarp) {
        // ---- one thread issues the MMAs of every tile
        if (lane == 0) {
            const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs);
            const uint32_t idesc = tc::idesc_f16_f32(128, 8 * ntp);
            int it = 0;
            const bool have_b = tc::mbar_wait(&b_full, 0, kTcWaitNs, &abort_flag);
            if (!have_b) give_up();
            for (int tile = blockIdx.x; have_b && tile < ntiles; tile += gridDim.x, ++it) {
                const int s = it & 1;
                const uint32_t ph = (it >> 1) & 1;
                if (!tc::mbar_wait(&a_full[s], ph, kTcWaitNs, &abort_flag) ||
                    (it >= 2 && !tc::mbar_wait(&d_empty[s], ph ^ 1, kTcWaitNs, &abort_flag))) {
                    give_up();
                    break;
                }
                tc::fence_after_sync();
                const uint32_t as = a0 + uint32_t(s) * (128u * KG * 16u);
#pragma unroll
                for (int k = 0; k < KG / 2; ++k)
                    tc::mma_f16(taddr + uint32_t(s) * 256u, tc::desc_kmajor(as + 256u * k, 128u, 128u * KG),
                                tc::desc_kmajor(b0 + 256u * k, 128u, 128u * KG), idesc, k > 0);
                tc::mma_commit(&a_empty[s]);
                tc::mma_commit(&d_full[s]);
            }
            // whatever happened, no MMA may still run when the memory is freed
            if (it > 0) tc::mbar_wait(&d_full[(it - 1) & 1], ((it - 1) >> 1) & 1, kTcWaitNs);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w reads lanes 32*(w % 4) .. +31, groups of four
        // targets part, part + 3, ... (part = w / 4)
        constexpr int kParts = kTcEpiWarps / 4;
        const int quarter = warp & 3, part = warp >> 2;
        const int ngroups4 = ntp >> 2;
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int s = it & 1;
            if (!tc::mbar_wait(&d_full[s], (it >> 1) & 1, kTcWaitNs, &abort_flag)) {
                give_up();
                break;
            }
            tc::fence_after_sync();
            const uint32_t laddr = taddr + uint32_t(s) * 256u + (uint32_t(quarter * 32) << 16);
            const uint32_t n = uint32_t(tile) * 128u + uint32_t(quarter * 32 + lane);
            for (int q4 = part; q4 < ngroups4; q4 += kParts) {
                uint32_t r[32];
                tc::tmem_ld32(laddr + uint32_t(q4 * 32), r);
                tc::tmem_wait_ld();
                tc::tmem_hold(r);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int t = q4 * 4 + j;
                    if (t >= nd) break;
                    const Dst &d = sd[t];
                    const uint32_t *b = r + 8 * j;
                    u64 lo = b[0];
                    mad_wide(lo, b[1], 1u << 8);
                    mad_wide(lo, b[2], 1u << 16);
                    mad_wide(lo, b[3], 1u << 24);
                    lo += u64(b[4]) << 32;
                    const uint32_t hi = b[5] + (b[6] << 8) - kBias * 257u;  // exact: the true value is < 2^32
                    // d.off = [-sub]_t - kLoBias (mod 2^64) removes the biases of lo
                    // in the same add: the true sum is >= 0 and < 2^64
                    u64 v = lo + shoup_u32(hi, d.r40, d.r40_s, d.np) + d.off;
                    if (!lazy) v = shoup_one(v, d.one_s, d.np);
                    d.out[n] = v;
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&d_empty[s]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(taddr, 512);
    }
}

template <int KG, class GMAP>
static void launch_tc_kg(const ckks_ctx *ctx, const GMAP &gm, int ngroups, int chunks, int chunk, cudaStream_t st,
                         int *status) {
    // 512 tensor-memory columns: one CTA of this kernel per SM (the shared
    // memory is sized so that a second cannot be placed beside it and wait in
    // tcgen05.alloc; CTAs of other kernels still fit); as many CTAs per
    // (group, chunk) as share the SMs, each walking over tiles
    const size_t need = (size_t(2 * 128) * KG + size_t(kTcXStages) * (KG - 1) * 64 + size_t(chunk) * KG * 8) *
                            sizeof(uint4) +
                        size_t(chunk) * 48;
    const size_t smem = std::max<size_t>(need, 116 * 1024);
    auto kern = bconv_tc_kernel<KG, GMAP>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    const int tiles = ctx->N / 128;
    const int rows = ngroups * chunks;
    // CTAs per (group, chunk): each SM runs one CTA at a time and a CTA its tiles
    // one after the other, so the launch takes about waves * ceil(tiles / per)
    // tile times plus a fixed cost (B image, tensor memory, pipeline fill: about
    // two tiles) per wave; pick the count that minimises it (a batch has more
    // (group, chunk) rows than SMs, a single operation a few).  The waves are
    // counted on the launch's share of the SMs: all of them for an operation
    // alone, 1/n of them when the caller runs n operations at once
    // (ckks_concurrency_hint), where fewer, longer CTAs pay the fixed cost less
    // often and the other operations fill the SMs.
    const int per = policy::tc_ctas_per_row(tiles, rows, policy::sm_share(ctx->sms, ctx->concurrency));
    const dim3 grid(static_cast<unsigned>(per), static_cast<unsigned>(rows));
    kern<<<grid, kTcThreads, smem, st>>>(gm, chunks, chunk, ctx->d_pinfo, ctx->logN, ctx->tc_lazy ? 1 : 0, status);
}

// Tensor-core conversion over `ngroups` groups of up to n_all targets each,
// in chunks of at most 32 targets (256 tensor-memory columns), each a
// multiple of four targets.  A wait that runs out is recorded in *status.
template <class GMAP>
static cudaError_t launch_tc(const ckks_ctx *ctx, const GMAP &gm, int ngroups, int n_all, cudaStream_t st,
                             int *status) {
    const int chunks = (n_all + 31) / 32;
    const int chunk = ((n_all + chunks - 1) / chunks + 3) & ~3;
    ProfScope ps(ctx, K_BCONV, double(ngroups) * n_all, st);
    switch (ctx->tc_kg) {
    case 4: launch_tc_kg<4>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    case 6: launch_tc_kg<6>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    case 8: launch_tc_kg<8>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    case 10: launch_tc_kg<10>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    case 12: launch_tc_kg<12>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    case 14: launch_tc_kg<14>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    case 16: launch_tc_kg<16>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    case 18: launch_tc_kg<18>(ctx, gm, ngroups, chunks, chunk, st, status); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Split conversion over `ngroups` groups of up to n_all targets each: targets
// in chunks of at most 12 per CTA row (enough CTAs to fill the SMs while each
// source word is still scaled once per 12 targets).
template <class GMAP>
static cudaError_t launch_split(const ckks_ctx *ctx, const GMAP &gm, int ngroups, int n_all, int max_src,
                                cudaStream_t st, int *status) {
    if (ctx->tc_kg && ctx->tc_on) return launch_tc(ctx, gm, ngroups, n_all, st, status);
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

// Self-test of the bounded wait: one CTA waits on an mbarrier that expects an
// arrival no thread makes; the wait gives up after limit_ns and the kernel
// records the timeout in the status word exactly as bconv_tc_kernel does.
__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, int *__restrict__ status) {
    __shared__ uint64_t never;
    if (threadIdx.x == 0) tc::mbar_init(&never, 1);
    __syncthreads();
    if (!tc::mbar_wait(&never, 0, limit_ns) && threadIdx.x == 0) atomicOr(status, 1);
}

cudaError_t launch_bounded_wait_selftest(const ckks_ctx *ctx, uint64_t limit_ns, cudaStream_t st, int *status) {
    bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, status != nullptr ? status : ctx->d_status);
    return cudaGetLastError();
}

// The basis conversions of one batched phase: ModUp digits (GM_MODUP), the
// ModDown of both polynomials (GM_MODDOWN) or the Rescale of both polynomials
// of the Mult entries (GM_RESCALE).  Needs the split conversion.  A bounded
// wait that runs out is recorded in *status (the context's word when null).
cudaError_t launch_bconv_batch(const ckks_ctx *ctx, const KsBatchDesc &d, int down, cudaStream_t st, int *status) {
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
    return launch_split(ctx, gm, groups, n_all, max_src, st, status != nullptr ? status : ctx->d_status);
}

cudaError_t launch_bconv(const ckks_ctx *ctx, const BConvLaunch &l, int max_src, cudaStream_t st) {
    if (l.ngroups == 0) return cudaSuccess;
    const int threads = 256;
    if (ctx->split_bits && max_src <= kMaxSrc) {
        GroupMapList gm;
        gm.l = l;
        return launch_split(ctx, gm, l.ngroups, l.chunk * l.chunks, max_src, st, ctx->d_status);
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
