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
#include "common.cuh"
#include "internal.h"

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

cudaError_t launch_bconv(const ckks_ctx *ctx, const BConvLaunch &l, int max_src, cudaStream_t st) {
    if (l.ngroups == 0) return cudaSuccess;
    const int threads = 256;
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
