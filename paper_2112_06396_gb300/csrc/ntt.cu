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
#include "batch.cuh"
#include "common.cuh"
#include "internal.h"

namespace ckks {

// Butterflies.  SMALLP (every prime < 2^57) uses the approximate-quotient
// Shoup product (result in [0, 3p)):
//  * forward (Cooley-Tukey): X' = X + T, Y' = X + 4p - T with T = W*Y in
//    [0, 3p), no conditional subtraction: a value below M*p before a stage is
//    below (M+4)*p after it.  Inputs may be lazy up to 8p (the basis
//    conversions leave their outputs below 4p on the integer units and
//    below 8p on the tensor cores), so after all logN <= 17 stages every
//    value is below (8 + 68)p < 2^64 and one reduction at the very end
//    suffices (the ModDown/Rescale epilogue folds it into its product);
//  * inverse (Gentleman-Sande): X' = (X + Y) mod' 4p, Y' = W*(X - Y + 4p),
//    keeping every value in [0, 4p).
// Otherwise (primes up to 2^60) Harvey's exact-quotient butterflies keep
// [0, 4p) forward and [0, 2p) inverse.
template <bool SMALLP>
__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 p, u64 np) {
    if (SMALLP) {
        const u64 T = shoup_approx(Y, w.x, w.y, np);
        Y = X + 4 * p - T;
        X = X + T;
    } else {
        X = csub(X, 2 * p);
        const u64 T = shoup_lazy(Y, w.x, w.y, p);
        Y = X + 2 * p - T;
        X = X + T;
    }
}
template <bool SMALLP>
__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, ulonglong2 w, u64 p, u64 np) {
    if (SMALLP) {
        const u64 T = X + 4 * p - Y;
        X = csub(X + Y, 4 * p);
        Y = shoup_approx(T, w.x, w.y, np);
    } else {
        const u64 T = X + 2 * p - Y;
        X = csub(X + Y, 2 * p);
        Y = shoup_lazy(T, w.x, w.y, p);
    }
}

template <int LOGN, int LOGR, int A, int C, bool INV, bool CONTIG, bool EPI, bool SMALLP, class MAP>
__global__ void __launch_bounds__((1 << (LOGR - A)) * C, (A <= 4 ? 1024 : 512) / ((1 << (LOGR - A)) * C))
ntt_pass_kernel(const __grid_constant__ MAP map, const PrimeInfo *__restrict__ pinfo,
                const ulonglong2 *__restrict__ tw_all) {
    constexpr int B = LOGR - A;
    constexpr int TPC = 1 << B;   // threads per column
    constexpr int E = 1 << A;     // words per thread
    constexpr int R = 1 << LOGR;  // rows per column
    constexpr int RS = R + TPC;   // pass-C smem row stride (one pad word per E rows)
    constexpr int NT = TPC * C;
    constexpr int TILE = CONTIG ? C * RS : R * C;
    extern __shared__ u64 sm[];

    // every shift is a compile-time constant and every index fits 32 bits
    constexpr int L2 = LOGN >> 1;
    constexpr int L1 = LOGN - L2;
    constexpr uint32_t N = 1u << LOGN;
    constexpr int logN = LOGN;
    // limbs sharing a prime are adjacent: co-resident CTAs reuse twiddles
    // The limb's pointers are derived twice (here for the source and the L2
    // prefetch, again before the stores): nothing but the source and the prime
    // stays live across the butterflies.
    const LimbIO io0 = map.get(blockIdx.x, N);
    const int prime = io0.prime;
    const u64 *__restrict__ src = io0.src;
    const ulonglong2 *__restrict__ tw = tw_all + size_t(prime) * N;
    const u64 p = pinfo[prime].p;
    const u64 np = u64(0) - p;

    const int tid = threadIdx.x;
    const int g = CONTIG ? (tid % TPC) : (tid / C);
    const int cl = CONTIG ? (tid / TPC) : (tid % C);
    const uint32_t col = blockIdx.y * C + cl;
    constexpr int s0 = CONTIG ? L1 : 0;
    const uint32_t prefix = CONTIG ? col : 0;

    auto gidx = [&](int r) -> uint32_t { return CONTIG ? ((col << L2) + r) : ((uint32_t(r) << L2) + col); };
    auto sidx = [&](int r) -> int { return CONTIG ? (cl * RS + r + (r >> A)) : (r * C + cl); };
    auto twi = [&](int sigma, int r) -> uint32_t {
        return (1u << (s0 + sigma)) + (prefix << sigma) + (uint32_t(r) >> (LOGR - sigma));
    };
    // Pass S uses only the twiddles 1 .. R-1 of this prime: stage them in shared memory.
    ulonglong2 *stw = reinterpret_cast<ulonglong2 *>(sm + TILE);
    if (!CONTIG) {
        for (int i = tid; i < R; i += NT) stw[i] = ld_keep(&tw[i]);
        __syncthreads();
    }
    auto TW = [&](int sigma, int r) -> ulonglong2 {
        const size_t i = twi(sigma, r);
        return CONTIG ? ld_keep(&tw[i]) : stw[i];
    };
    // Pass C: one thread asks the TMA unit to pull this CTA's twiddle ranges
    // (stage sigma uses C * 2^sigma consecutive entries) and, for the ModDown
    // epilogue, the x and add tiles into L2 while the data loads run.
    if (CONTIG && tid == 0) {
        const size_t col0 = size_t(blockIdx.y) * C;
#pragma unroll
        for (int sg = 0; sg < LOGR; sg++) {
            const ulonglong2 *t0 = tw + (size_t(1) << (s0 + sg)) + (col0 << sg);
            l2_prefetch(t0, uint32_t(C * sizeof(ulonglong2)) << sg);
        }
        if (EPI) {
            l2_prefetch(io0.ex + (col0 << L2), uint32_t(C * sizeof(u64)) << L2);
            if (io0.accumulate) l2_prefetch(io0.eout + (col0 << L2), uint32_t(C * sizeof(u64)) << L2);
            if (io0.eadd != nullptr) {
                for (int b = 0; b < C; b++) {
                    const uint32_t first = uint32_t((col0 + b) << L2);
                    const uint32_t sblk = (io0.galois == 1 ? first : automorph_src(first, io0.galois, logN)) >> L2;
                    l2_prefetch(io0.eadd + (size_t(sblk) << L2), uint32_t(sizeof(u64)) << L2);
                }
            }
        }
    }

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
                ct_bfly<SMALLP>(x[k], x[k + half], TW(sg, g + (k << B)), p, np);
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
                ct_bfly<SMALLP>(x[e], x[e + half], TW(sg, (g << A) + e), p, np);
            }
        }
        const LimbIO io = map.get(blockIdx.x, N);
        u64 *dst = io.dst;
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
            // the ModDown/Rescale tail, and a lazy store, take the lazy values
            // (below 76p) as they are
            if (!(SMALLP && (EPI || io.lazy))) {
                const u64 one_s = pinfo[prime].one_s;
#pragma unroll
                for (int k = 0; k < E; k++) {
                    u64 v = SMALLP ? shoup_one(x[k], one_s, np) : x[k];
                    x[k] = csub(csub(v, 2 * p), p);
                }
            }
            if (!EPI) {
#pragma unroll
                for (int k = 0; k < E; k++) dst[gidx(g + (k << B))] = x[k];
            } else {
                // Epilogue operands are read-only for this launch: load a group of
                // them through the non-coherent path before any store, so the
                // loads overlap instead of waiting behind each store.
                const ulonglong2 c = io.cmul[prime];
                const u64 *__restrict__ xp = io.ex;
                const u64 *__restrict__ ap = io.eadd;
                u64 *op = io.eout;
                constexpr int GRP = E < 4 ? E : 4;
#pragma unroll
                for (int k0 = 0; k0 < E; k0 += GRP) {
                    u64 xv[GRP], av[GRP], ov[GRP];
#pragma unroll
                    for (int k = 0; k < GRP; k++) {
                        const uint32_t i = uint32_t(gidx(g + ((k0 + k) << B)));
                        xv[k] = __ldg(xp + i);
                        av[k] = 0;
                        ov[k] = 0;
                        if (ap != nullptr)
                            av[k] = __ldg(ap + (io.galois == 1 ? i : automorph_src(i, io.galois, logN)));
                        if (io.accumulate) ov[k] = op[i];
                    }
#pragma unroll
                    for (int k = 0; k < GRP; k++) {
                        const uint32_t i = uint32_t(gidx(g + ((k0 + k) << B)));
                        u64 r;
                        if (SMALLP) {
                            // x lazy below 76p (at most 17 stages from inputs below
                            // 8p), xv < p: xv + 80p - x is below 81p < 2^64 and
                            // congruent to xv - x; the product is in [0, 3p), the
                            // two reduced addends bring it below 5p
                            r = shoup_approx(xv[k] + 80 * p - x[k0 + k], c.x, c.y, np) + av[k] + ov[k];
                            r = csub(csub(csub(r, 4 * p), 2 * p), p);
                        } else {
                            r = shoup_mul(sub_mod(xv[k], x[k0 + k], p), c.x, c.y, p);
                            r = add_mod(r, av[k], p);
                            r = add_mod(r, ov[k], p);
                        }
                        op[i] = r;
                    }
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
                gs_bfly<SMALLP>(x[e], x[e + half], TW(sg, (g << A) + e), p, np);
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
                    const u64 X = x[k], Y = x[k + half];
                    if (SMALLP) {
                        const u64 T = X + 4 * p - Y;
                        x[k] = shoup_approx(X + Y, P.ninv, P.ninv_s, np);
                        x[k + half] = shoup_approx(T, P.ninv_w, P.ninv_w_s, np);
                    } else {
                        const u64 T = X + 2 * p - Y;
                        x[k] = shoup_lazy(X + Y, P.ninv, P.ninv_s, p);
                        x[k + half] = shoup_lazy(T, P.ninv_w, P.ninv_w_s, p);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < E; k++) {
                    if (k & half) continue;
                    gs_bfly<SMALLP>(x[k], x[k + half], TW(sg, g + (k << B)), p, np);
                }
            }
        }
        u64 *dst = map.get(blockIdx.x, N).dst;
#pragma unroll
        for (int k = 0; k < E; k++) {
            u64 v = x[k];
            if (!CONTIG) v = SMALLP ? csub(csub(v, 2 * p), p) : csub(v, p);  // last pass: fully reduce
            dst[gidx(g + (k << B))] = v;
        }
    }
}

// ------------------------------------------------------------------ host side
namespace {

// CSEL picks the CTA width (the tile shape): 0 = the default below, 1 = half
// of it, 2 = twice it.  The autotuner (ntt_autotune) chooses per pass and per
// batch size; widths other than the default exist for logN >= 14 with small
// primes (the key-switching shapes), elsewhere every CSEL maps to 0.
template <int LOGN, bool INV, bool CONTIG, bool EPI, bool SMALLP, int CSEL, class MAP>
cudaError_t launch_one_p(const MAP &m, int count, const ckks_ctx *ctx, cudaStream_t st, bool set_attr) {
    // pass S transforms columns of 2^L1 rows, pass C blocks of 2^L2 words
    constexpr int L2 = LOGN >> 1, L1 = LOGN - L2;
    constexpr int LOGR = CONTIG ? L2 : L1;
    constexpr int OTHER = CONTIG ? L1 : L2;
    constexpr int A = (LOGR + 1) / 2;
    constexpr int B = LOGR - A;
    constexpr int TPC = 1 << B;
    constexpr int R = 1 << LOGR;
    // C = columns (pass S) or blocks (pass C) per CTA: small CTAs (128 threads
    // for pass S, 64 for pass C, measured best at N=2^16) keep barriers local and
    // let many independent CTAs hide the load latency; clamped to the number of
    // columns / blocks of the matrix view
    constexpr int BASE = (CONTIG ? 64 : 128) * (CSEL == 2 ? 2 : 1) / (CSEL == 1 ? 2 : 1);
    constexpr int WANT = BASE / TPC > 0 ? BASE / TPC : 1;
    constexpr int C = WANT < (1 << OTHER) ? WANT : (1 << OTHER);
    const size_t smem = CONTIG ? size_t(C) * (R + TPC) * 8 : size_t(R) * C * 8 + size_t(R) * 16;
    auto kern = ntt_pass_kernel<LOGN, LOGR, A, C, INV, CONTIG, EPI, SMALLP, MAP>;
    if (set_attr) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    dim3 grid(count, (1 << OTHER) / C);
    kern<<<grid, TPC * C, smem, st>>>(m, ctx->d_pinfo, INV ? ctx->d_tw_inv : ctx->d_tw_fwd);
    return cudaGetLastError();
}

template <int LOGN, bool INV, bool CONTIG, bool EPI, class MAP>
cudaError_t launch_one(const MAP &m, int count, const ckks_ctx *ctx, cudaStream_t st, bool set_attr, int csel) {
    constexpr bool TUNED = LOGN >= 14;
    if (set_attr) {
        cudaError_t e = launch_one_p<LOGN, INV, CONTIG, EPI, false, 0>(m, count, ctx, st, true);
        if (e == cudaSuccess) e = launch_one_p<LOGN, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, true);
        if (TUNED && e == cudaSuccess) e = launch_one_p<LOGN, INV, CONTIG, EPI, true, TUNED ? 1 : 0>(m, count, ctx, st, true);
        if (TUNED && e == cudaSuccess) e = launch_one_p<LOGN, INV, CONTIG, EPI, true, TUNED ? 2 : 0>(m, count, ctx, st, true);
        return e;
    }
    if (!ctx->small_primes) return launch_one_p<LOGN, INV, CONTIG, EPI, false, 0>(m, count, ctx, st, false);
    if (TUNED && csel == 1) return launch_one_p<LOGN, INV, CONTIG, EPI, true, TUNED ? 1 : 0>(m, count, ctx, st, false);
    if (TUNED && csel == 2) return launch_one_p<LOGN, INV, CONTIG, EPI, true, TUNED ? 2 : 0>(m, count, ctx, st, false);
    return launch_one_p<LOGN, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, false);
}

// The tuned width of a pass for a launch of `count` limbs (-1: use the table).
inline int csel_for(const ckks_ctx *ctx, bool contig, int count, int force) {
    if (force >= 0) return force;
    return ctx->ntt_csel[contig ? 1 : 0][count > kTuneSmallBatch ? 1 : 0];
}

template <bool INV, bool CONTIG, bool EPI, class MAP>
cudaError_t dispatch(const MAP &m, int count, const ckks_ctx *ctx, cudaStream_t st, bool set_attr, int force = -1) {
    const int cs = csel_for(ctx, CONTIG, count, force);
    switch (ctx->logN) {
    case 10: return launch_one<10, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    case 11: return launch_one<11, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    case 12: return launch_one<12, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    case 13: return launch_one<13, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    case 14: return launch_one<14, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    case 15: return launch_one<15, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    case 16: return launch_one<16, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    case 17: return launch_one<17, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs);
    default: return cudaErrorInvalidValue;
    }
}

template <class MAP>
cudaError_t set_attributes_for(const ckks_ctx *ctx) {
    MAP m{};
    cudaError_t err;
    if ((err = dispatch<false, false, false>(m, 0, ctx, nullptr, true)) != cudaSuccess) return err;
    if ((err = dispatch<false, true, false>(m, 0, ctx, nullptr, true)) != cudaSuccess) return err;
    if ((err = dispatch<false, true, true>(m, 0, ctx, nullptr, true)) != cudaSuccess) return err;
    if ((err = dispatch<true, true, false>(m, 0, ctx, nullptr, true)) != cudaSuccess) return err;
    return dispatch<true, false, false>(m, 0, ctx, nullptr, true);
}

// Two passes of one transform: the second runs in place on the first's output.
template <class MAP>
cudaError_t run_fwd(MAP m, int count, bool epi, const ckks_ctx *ctx, cudaStream_t st) {
    cudaError_t err;
    m.second = 0;
    {
        ProfScope ps(ctx, K_NTT_FWD, count, st);
        err = dispatch<false, false, false>(m, count, ctx, st, false);
    }
    if (err != cudaSuccess) return err;
    m.second = 1;
    ProfScope ps(ctx, K_NTT_FWD, count, st);
    if (epi) return dispatch<false, true, true>(m, count, ctx, st, false);
    return dispatch<false, true, false>(m, count, ctx, st, false);
}

template <class MAP>
cudaError_t run_inv(MAP m, int count, const ckks_ctx *ctx, cudaStream_t st) {
    cudaError_t err;
    m.second = 0;
    {
        ProfScope ps(ctx, K_NTT_INV, count, st);
        err = dispatch<true, true, false>(m, count, ctx, st, false);
    }
    if (err != cudaSuccess) return err;
    m.second = 1;
    ProfScope ps(ctx, K_NTT_INV, count, st);
    return dispatch<true, false, false>(m, count, ctx, st, false);
}

}  // namespace

cudaError_t ntt_set_attributes(const ckks_ctx *ctx) {
    cudaError_t err = set_attributes_for<MapList>(ctx);
    if (err != cudaSuccess) return err;
    return set_attributes_for<MapBatch>(ctx);
}

// Forward transform of a limb list (src -> dst, then in place); the optional
// ModDown/Rescale epilogue replaces the store of the last pass.
cudaError_t launch_ntt_fwd(const ckks_ctx *ctx, const NttBatch &b, const Epi *epi, cudaStream_t st) {
    if (b.count == 0) return cudaSuccess;
    MapList m;
    m.b = b;
    const bool scale = epi != nullptr && epi->mode == EPI_SCALE;
    if (scale) m.e = *epi;
    else {
        m.e = Epi{};
        m.e.mode = epi != nullptr && epi->mode == EPI_LAZY ? EPI_LAZY : EPI_STORE;
    }
    return run_fwd(m, b.count, scale, ctx, st);
}

cudaError_t launch_ntt_inv(const ckks_ctx *ctx, const NttBatch &b, cudaStream_t st) {
    if (b.count == 0) return cudaSuccess;
    MapList m;
    m.b = b;
    m.e = Epi{};
    m.e.mode = EPI_STORE;
    return run_inv(m, b.count, ctx, st);
}

// One phase of batched key switching over every ciphertext of the batch.
cudaError_t launch_ntt_batch(const ckks_ctx *ctx, const KsBatchDesc &d, int phase, cudaStream_t st) {
    MapBatch m;
    m.d = d;
    m.phase = phase;
    m.cm = ctx->d_Pinv;
    m.qlinv = ctx->d_qlinv;
    m.dinv = ctx->d_Dinv;
    int count = 0;
    for (int c = 0; c < d.n; ++c) {
        m.d.pre[c] = count;
        count += phase_count(d, d.ct[c], phase);
    }
    m.d.pre[d.n] = count;
    if (count == 0) return cudaSuccess;
    if (phase == PH_INTT_A || phase == PH_INTT_P || phase == PH_RS_INTT) return run_inv(m, count, ctx, st);
    return run_fwd(m, count, phase == PH_NTT_DOWN || phase == PH_RS_NTT, ctx, st);
}

// ------------------------------------------------------------------ autotuner
// Times every CTA width of the column pass (S) and the block pass (C), forward
// and inverse together, on `small` and `large` limbs of scratch data (in
// place, values are transformed and transformed back), and keeps the fastest
// per pass and batch-size class in the context.  scratch: at least
// large * N words.  Returns the chosen widths through ctx->ntt_csel.
cudaError_t ntt_autotune(ckks_ctx *ctx, u64 *scratch, int small, int large, cudaStream_t st, float *times_out) {
    if (ctx->logN < 14 || !ctx->small_primes) return cudaSuccess;  // one width only
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    if ((err = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    const bool prof = ctx->prof_on;
    ctx->prof_on = false;
    err = cudaMemsetAsync(scratch, 0, size_t(large) * ctx->N * sizeof(u64), st);
    const int counts[2] = {small, large};
    for (int bucket = 0; bucket < 2 && err == cudaSuccess; ++bucket) {
        const int count = counts[bucket];
        MapList m{};
        m.b.count = count;
        for (int l = 0; l < count; ++l) {
            m.b.src[l] = scratch + size_t(l) * ctx->N;
            m.b.dst[l] = scratch + size_t(l) * ctx->N;
            m.b.prime[l] = uint16_t(l % (ctx->L + ctx->k));
        }
        m.e.mode = EPI_STORE;
        for (int contig = 0; contig < 2 && err == cudaSuccess; ++contig) {
            float best = 1e30f;
            int pick = 0;
            for (int cs = 0; cs < 3 && err == cudaSuccess; ++cs) {
                auto run = [&]() {
                    m.second = 1;
                    cudaError_t e2 = contig ? dispatch<false, true, false>(m, count, ctx, st, false, cs)
                                            : dispatch<false, false, false>(m, count, ctx, st, false, cs);
                    if (e2 == cudaSuccess)
                        e2 = contig ? dispatch<true, true, false>(m, count, ctx, st, false, cs)
                                    : dispatch<true, false, false>(m, count, ctx, st, false, cs);
                    return e2;
                };
                err = run();  // warm-up
                if (err != cudaSuccess) break;
                cudaEventRecord(e0, st);
                for (int r = 0; r < 5 && err == cudaSuccess; ++r) err = run();
                cudaEventRecord(e1, st);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                if (times_out) times_out[(contig * 2 + bucket) * 3 + cs] = ms / 5;
                if (ms < best) {
                    best = ms;
                    pick = cs;
                }
            }
            ctx->ntt_csel[contig][bucket] = pick;
        }
    }
    ctx->prof_on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

}  // namespace ckks
