// ntt.cu -- negacyclic NTT / iNTT over batches of limbs (Sec. 2.3,
// "Polynomial Representation"; limb-wise access pattern of the table
// "Data dependencies and access pattern").
//
// Transform: a_hat[j] = sum_i a_i psi^((2 brv(j)+1) i) mod q, computed as the
// merged-twist Cooley-Tukey network (stage s, block i uses psi^brv(2^s + i));
// the inverse is the Gentleman-Sande network with psi^-brv(2^s + i) and the
// factor N^-1 folded into its last stage.
//
// GB300 layout: a limb (N words) is viewed as a 2^L1 x 2^L2 matrix (L1 =
// ceil(logN/2)).  Pass S runs the first L1 stages down the columns (rows are
// 2^L2 words apart), pass C the last L2 stages inside each contiguous block
// of 2^L2 words.  One CTA owns C columns (pass S) or C blocks (pass C); each
// thread holds E = 2^A words in registers, runs A stages there, the tile is
// transposed once through shared memory, and the remaining B = LOGR - A
// stages run in registers again.  Global loads and stores are coalesced (the
// contiguous-pass output is re-staged through shared memory).  Values stay in
// [0, 4p) between stages (Harvey's lazy butterflies) and are fully reduced
// only when the transform ends.
#include "common.cuh"
#include "internal.h"

namespace ckks {

// Cooley-Tukey butterfly, X, Y in [0, 4p) -> [0, 4p)
__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 p, u64 two_p) {
    X = csub(X, two_p);
    u64 T = shoup_lazy(Y, w.x, w.y, p);
    Y = X + two_p - T;
    X = X + T;
}
// Gentleman-Sande butterfly, X, Y in [0, 2p) -> [0, 2p)
__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 p, u64 two_p) {
    u64 T = X + two_p - Y;
    X = csub(X + Y, two_p);
    Y = shoup_lazy(T, w.x, w.y, p);
}

template <int LOGR, int A, int C, bool INV, bool CONTIG, bool EPI>
__global__ void __launch_bounds__((1 << (LOGR - A)) * C)
ntt_pass_kernel(NttBatch batch, const PrimeInfo *__restrict__ pinfo, const ulonglong2 *__restrict__ tw_all,
                int logN, Epi epi) {
    constexpr int B = LOGR - A;
    constexpr int TPC = 1 << B;   // threads per column
    constexpr int E = 1 << A;     // words per thread
    constexpr int R = 1 << LOGR;  // rows per column
    constexpr int RS = R + TPC;   // pass-C smem row stride (one pad word per E rows)
    extern __shared__ u64 sm[];

    const int L2 = logN >> 1;
    const int L1 = logN - L2;
    const size_t N = size_t(1) << logN;
    const int limb = blockIdx.y;
    const int prime = batch.prime[limb];
    const u64 *__restrict__ src = batch.src[limb];
    u64 *dst = batch.dst[limb];
    const ulonglong2 *__restrict__ tw = tw_all + size_t(prime) * N;
    const u64 p = pinfo[prime].p;
    const u64 two_p = 2 * p;

    const int tid = threadIdx.x;
    const int g = CONTIG ? (tid % TPC) : (tid / C);
    const int cl = CONTIG ? (tid / TPC) : (tid % C);
    const int col = blockIdx.x * C + cl;
    const int s0 = CONTIG ? L1 : 0;
    const u64 prefix = CONTIG ? u64(col) : 0;

    auto gidx = [&](int r) -> size_t {
        return CONTIG ? ((size_t(col) << L2) + r) : ((size_t(r) << L2) + col);
    };
    auto sidx = [&](int r) -> int { return CONTIG ? (cl * RS + r + (r >> A)) : (r * C + cl); };
    auto twi = [&](int sigma, int r) -> size_t {
        return (size_t(1) << (s0 + sigma)) + (prefix << sigma) + (size_t(r) >> (LOGR - sigma));
    };

    u64 x[E];
    if (!INV) {
        // ---- load in strided layout: word k is row g + k*TPC
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = src[gidx(g + (k << B))];
        // ---- stages 0..A-1 (pairs E/2 .. 1 words apart in this layout)
#pragma unroll
        for (int sg = 0; sg < A; sg++) {
            const int half = 1 << (A - 1 - sg);
#pragma unroll
            for (int k = 0; k < E; k++) {
                if (k & half) continue;
                ulonglong2 w = __ldg(&tw[twi(sg, g + (k << B))]);
                ct_bfly(x[k], x[k + half], w, p, two_p);
            }
        }
#pragma unroll
        for (int k = 0; k < E; k++) sm[sidx(g + (k << B))] = x[k];
        __syncthreads();
        // ---- contiguous layout: word e is row g*E + e
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = sm[sidx((g << A) + e)];
#pragma unroll
        for (int sg = A; sg < LOGR; sg++) {
            const int half = 1 << (LOGR - 1 - sg);
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & half) continue;
                ulonglong2 w = __ldg(&tw[twi(sg, (g << A) + e)]);
                ct_bfly(x[e], x[e + half], w, p, two_p);
            }
        }
        if (!CONTIG) {
            // pass S: store contiguous layout (lanes run over columns: coalesced)
#pragma unroll
            for (int e = 0; e < E; e++) dst[gidx((g << A) + e)] = x[e];
        } else {
            // pass C (last pass): restage to strided layout for coalesced stores
#pragma unroll
            for (int e = 0; e < E; e++) sm[sidx((g << A) + e)] = x[e];
            __syncthreads();
#pragma unroll
            for (int k = 0; k < E; k++) x[k] = sm[sidx(g + (k << B))];
#pragma unroll
            for (int k = 0; k < E; k++) {
                const size_t i = gidx(g + (k << B));
                u64 v = csub(csub(x[k], two_p), p);
                if (!EPI || epi.mode == EPI_STORE) {
                    dst[i] = v;
                } else {
                    const int poly = limb / epi.nper;
                    const size_t base = size_t(limb % epi.nper) * N;
                    const ulonglong2 c = epi.cmul[prime];
                    u64 r = shoup_mul(sub_mod(epi.x[poly][base + i], v, p), c.x, c.y, p);
                    if (epi.add[poly] != nullptr) {
                        const uint32_t si = epi.galois == 1 ? uint32_t(i) : automorph_src(uint32_t(i), epi.galois, logN);
                        r = add_mod(r, epi.add[poly][base + si], p);
                    }
                    if (epi.accumulate) r = add_mod(r, epi.out[poly][base + i], p);
                    epi.out[poly][base + i] = r;
                }
            }
        }
    } else {
        if (CONTIG) {
            // pass C (first inverse pass): coalesced strided load, restage to contiguous
#pragma unroll
            for (int k = 0; k < E; k++) x[k] = src[gidx(g + (k << B))];
#pragma unroll
            for (int k = 0; k < E; k++) sm[sidx(g + (k << B))] = x[k];
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; e++) x[e] = sm[sidx((g << A) + e)];
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) x[e] = src[gidx((g << A) + e)];
        }
        // ---- stages LOGR-1 .. A in contiguous layout
#pragma unroll
        for (int sg = LOGR - 1; sg >= A; sg--) {
            const int half = 1 << (LOGR - 1 - sg);
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & half) continue;
                ulonglong2 w = __ldg(&tw[twi(sg, (g << A) + e)]);
                gs_bfly(x[e], x[e + half], w, p, two_p);
            }
        }
#pragma unroll
        for (int e = 0; e < E; e++) sm[sidx((g << A) + e)] = x[e];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < E; k++) x[k] = sm[sidx(g + (k << B))];
        // ---- stages A-1 .. 0 in strided layout
#pragma unroll
        for (int sg = A - 1; sg >= 0; sg--) {
            const int half = 1 << (A - 1 - sg);
            if (!CONTIG && sg == 0) {
                // global stage 0: fold N^-1 into both outputs
                const PrimeInfo &P = pinfo[prime];
#pragma unroll
                for (int k = 0; k < E; k++) {
                    if (k & half) continue;
                    u64 X = x[k], Y = x[k + half];
                    u64 T = X + two_p - Y;
                    x[k] = shoup_lazy(X + Y, P.ninv, P.ninv_s, p);
                    x[k + half] = shoup_lazy(T, P.ninv_w, P.ninv_w_s, p);
                }
            } else {
#pragma unroll
                for (int k = 0; k < E; k++) {
                    if (k & half) continue;
                    ulonglong2 w = __ldg(&tw[twi(sg, g + (k << B))]);
                    gs_bfly(x[k], x[k + half], w, p, two_p);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < E; k++) {
            u64 v = x[k];
            if (!CONTIG) v = csub(v, p);  // last pass: fully reduce
            dst[gidx(g + (k << B))] = v;
        }
    }
}

// ------------------------------------------------------------------ host side
namespace {

template <int LOGR, int C, bool INV, bool CONTIG, bool EPI>
cudaError_t launch_one(const NttBatch &b, const ckks_ctx *ctx, const Epi &epi, int tiles, cudaStream_t st,
                       bool set_attr) {
    constexpr int A = (LOGR + 1) / 2;
    constexpr int B = LOGR - A;
    constexpr int TPC = 1 << B;
    constexpr int R = 1 << LOGR;
    const size_t smem = CONTIG ? size_t(C) * (R + TPC) * 8 : size_t(R) * C * 8;
    auto kern = ntt_pass_kernel<LOGR, A, C, INV, CONTIG, EPI>;
    if (set_attr) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    dim3 grid(tiles, b.count);
    kern<<<grid, TPC * C, smem, st>>>(b, ctx->d_pinfo, INV ? ctx->d_tw_inv : ctx->d_tw_fwd, ctx->logN, epi);
    return cudaGetLastError();
}

// C = columns (pass S) or blocks (pass C) per CTA: 256 threads, clamped to the
// number of columns/blocks of the matrix view.
template <bool INV, bool CONTIG, bool EPI>
cudaError_t dispatch(int LOGR, int other, const NttBatch &b, const ckks_ctx *ctx, const Epi &epi, cudaStream_t st,
                     bool set_attr) {
    const int ncols = 1 << other;
    switch (LOGR) {
    case 5:
        if (ncols >= 64) return launch_one<5, 64, INV, CONTIG, EPI>(b, ctx, epi, ncols / 64, st, set_attr);
        return launch_one<5, 32, INV, CONTIG, EPI>(b, ctx, epi, ncols / 32, st, set_attr);
    case 6: return launch_one<6, 32, INV, CONTIG, EPI>(b, ctx, epi, ncols / 32, st, set_attr);
    case 7: return launch_one<7, 32, INV, CONTIG, EPI>(b, ctx, epi, ncols / 32, st, set_attr);
    case 8: return launch_one<8, 16, INV, CONTIG, EPI>(b, ctx, epi, ncols / 16, st, set_attr);
    case 9: return launch_one<9, 16, INV, CONTIG, EPI>(b, ctx, epi, ncols / 16, st, set_attr);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t ntt_set_attributes(const ckks_ctx *ctx) {
    const int L2 = ctx->logN >> 1, L1 = ctx->logN - L2;
    NttBatch b{};
    Epi e{};
    cudaError_t err;
    if ((err = dispatch<false, false, false>(L1, L2, b, ctx, e, nullptr, true)) != cudaSuccess) return err;
    if ((err = dispatch<false, true, false>(L2, L1, b, ctx, e, nullptr, true)) != cudaSuccess) return err;
    if ((err = dispatch<false, true, true>(L2, L1, b, ctx, e, nullptr, true)) != cudaSuccess) return err;
    if ((err = dispatch<true, true, false>(L2, L1, b, ctx, e, nullptr, true)) != cudaSuccess) return err;
    if ((err = dispatch<true, false, false>(L1, L2, b, ctx, e, nullptr, true)) != cudaSuccess) return err;
    return cudaSuccess;
}

// Forward transform of a batch (src -> dst, then in place); the optional
// epilogue replaces the store of the last pass.
cudaError_t launch_ntt_fwd(const ckks_ctx *ctx, const NttBatch &b, const Epi *epi, cudaStream_t st) {
    if (b.count == 0) return cudaSuccess;
    const int L2 = ctx->logN >> 1, L1 = ctx->logN - L2;
    Epi none{};
    none.mode = EPI_STORE;
    cudaError_t err;
    {
        ProfScope ps(ctx, K_NTT_FWD, b.count, st);
        err = dispatch<false, false, false>(L1, L2, b, ctx, none, st, false);
    }
    if (err != cudaSuccess) return err;
    NttBatch b2 = b;
    for (int l = 0; l < b.count; l++) b2.src[l] = b.dst[l];
    ProfScope ps(ctx, K_NTT_FWD, b.count, st);
    if (epi != nullptr && epi->mode != EPI_STORE) return dispatch<false, true, true>(L2, L1, b2, ctx, *epi, st, false);
    return dispatch<false, true, false>(L2, L1, b2, ctx, none, st, false);
}

cudaError_t launch_ntt_inv(const ckks_ctx *ctx, const NttBatch &b, cudaStream_t st) {
    if (b.count == 0) return cudaSuccess;
    const int L2 = ctx->logN >> 1, L1 = ctx->logN - L2;
    Epi none{};
    cudaError_t err;
    {
        ProfScope ps(ctx, K_NTT_INV, b.count, st);
        err = dispatch<true, true, false>(L2, L1, b, ctx, none, st, false);
    }
    if (err != cudaSuccess) return err;
    NttBatch b2 = b;
    for (int l = 0; l < b.count; l++) b2.src[l] = b.dst[l];
    ProfScope ps(ctx, K_NTT_INV, b.count, st);
    return dispatch<true, false, false>(L1, L2, b2, ctx, none, st, false);
}

}  // namespace ckks
