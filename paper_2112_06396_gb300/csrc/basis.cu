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

// Split conversion over `ngroups` groups of up to n_all targets each: targets
// in chunks of at most 12 per CTA row (enough CTAs to fill the SMs while each
// source word is still scaled once per 12 targets).
template <class GMAP>
static cudaError_t launch_split(const ckks_ctx *ctx, const GMAP &gm, int ngroups, int n_all, int max_src,
                                cudaStream_t st) {
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
