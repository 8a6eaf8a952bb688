// ntt.cu -- negacyclic NTT / iNTT over batches of limbs (Sec. 2.3,
// "Polynomial Representation"; limb-wise access pattern of the table
// "Data dependencies and access pattern").
//
// Transform: a_hat[j] = sum_i a_i psi^((2 brv(j)+1) i) mod q, computed as the
// merged-twist Cooley-Tukey network (stage s, block i uses psi^brv(2^s + i));
// the inverse is the Gentleman-Sande network with psi^-brv(2^s + i) and the
// factor N^-1 folded into its last stage.
//
// GB300 layout: a limb (N words) is viewed as a 2^L1 x 2^L2 matrix (by
// default L1 = ceil(logN/2); the autotuner may move one stage from one pass
// to the other, the radix split).  Pass S runs the first L1 stages down the
// columns (rows are 2^L2 words apart), pass C the last L2 stages inside each
// contiguous block of 2^L2 words.  One CTA owns C columns (pass S) or C blocks
// (pass C); each thread holds E = 2^A words in registers, runs A stages there,
// the tile is transposed once through shared memory, and the remaining
// B = LOGR - A stages run in registers again.  Global loads and stores are coalesced (the
// contiguous-pass output is re-staged through shared memory).  Values stay in
// [0, 4p) between stages (Harvey's lazy butterflies) and are fully reduced
// only when the transform ends.
#include "batch.cuh"
#include "common.cuh"
#include "internal.h"
#include "launch_policy.h"
#include "prng.cuh"
#include "tc.cuh"

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

template <int LOGN, int L2, int LOGR, int A, int C, bool INV, bool CONTIG, bool EPI, bool SMALLP, class MAP>
__global__ void __launch_bounds__((1 << (LOGR - A)) * C, (A <= 4 ? 1024 : 512) / ((1 << (LOGR - A)) * C))
ntt_pass_kernel(const __grid_constant__ MAP map, const PrimeInfo *__restrict__ pinfo,
                const ulonglong2 *__restrict__ tw_all) {
    constexpr int B = LOGR - A;
    constexpr int TPC = 1 << B;   // threads per column
    constexpr int E = 1 << A;     // words per thread
    constexpr int R = 1 << LOGR;  // rows per column
    constexpr int RS = R + TPC;   // pass-C smem row stride (one pad word per E rows)
    extern __shared__ u64 sm[];

    // every shift is a compile-time constant and every index fits 32 bits
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
    // Twiddles come through L1 (the prime's table stays in L2): pass S reads only
    // entries 1 .. R-1, which every CTA of the prime on this SM shares.  (Staging
    // them in shared memory cost 4 KB per CTA, which other kernels of a
    // concurrent step need on the same SM.)
    auto TW = [&](int sigma, int r) -> ulonglong2 {
        const size_t i = twi(sigma, r);
        return ld_keep(&tw[i]);
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

// ------------------------------------------------------------------ fused ModUp tail + KSKInnerProd
// The last forward pass of ModUp's NTT (pass C) fused with KSKInnerProd and,
// on the special positions, with the first pass of ModDown's inverse NTT (the
// beta-limb caching of Sec. 4.2 and the re-ordering of Sec. 4.4).  A CTA owns
// one extended position t and C consecutive output blocks of 2^L2 slots, with
// one group of 64 threads per digit (four groups; a group whose digit does not
// exist or holds t, on a chain position, has no pass to run):
//  0. One thread asks the TMA unit to pull the CTA's key rows (2 beta tiles of
//     C * 2^L2 contiguous words, or beta with a compressed key) and, on a
//     chain position, the C source blocks of the digit's own limb into L2:
//     the key stream overlaps step 1 and step 2 reads it from L2.
//  1. Each group runs pass C of its digit's limb at t, written by pass S of
//     ModUp's NTT, on the C source blocks that the output blocks read through
//     Automorph_g (an aligned block of slots maps onto one aligned block, a
//     slot pair onto an aligned pair), leaving the lazy values in shared
//     memory; the groups share the prime's twiddles through L1.
//  2. The threads form u = sum_j d_j a_j and v = sum_j d_j b_j slot pair by
//     slot pair: digits from shared memory through the permutation, exact
//     128-bit sums (digits below 76p), one reduction.
//  3. Chain positions store u and v.  Special positions, which ModDown only
//     reads in coefficient form, run pass C of the inverse NTT on u and v and
//     store the result in place of u and v, where ModDown's inverse pass S
//     continues.
// The new ModUp limbs never reach HBM in evaluation form, nor the special
// limbs of u and v in evaluation form.
template <int LOGN, bool COMP>
__global__ void __launch_bounds__(256, 4)
modup_ip_kernel(const __grid_constant__ FusedIpArgs F, const PrimeInfo *__restrict__ pinfo,
                const ulonglong2 *__restrict__ twf_all, const ulonglong2 *__restrict__ twi_all, int L, int k,
                int alpha, int t_base) {
    constexpr int L2 = LOGN >> 1, L1 = LOGN - L2, LOGR = L2;
    constexpr int A = (LOGR + 1) / 2, B = LOGR - A, TPC = 1 << B, E = 1 << A, R = 1 << LOGR, RS = R + TPC;
    constexpr int C = 64 / TPC;                   // blocks per CTA: 64 threads of E words cover them
    constexpr int CR = C * R;                     // slots of the CTA
    constexpr uint32_t N = 1u << LOGN;
    constexpr int logN = LOGN;
    extern __shared__ __align__(16) u64 sm[];
    constexpr int PAIRS = CR / 2 / 256;           // slot pairs per thread in step 2
    u64 *const dig = sm;                          // [4][C * RS]: transformed digits (padded rows)
    u64 *const uvs = sm + 4 * C * RS;             // [2][C * RS]: u, v of a special position
    const int tid = threadIdx.x, grp = tid >> 6, lt = tid & 63;
    const int g = lt % TPC, cl = lt / TPC;
    const int t = t_base + int(blockIdx.y);
    const int ell = F.ell, ext = ell + k, LK = L + k;
    const int prime = t < ell ? t : L + (t - ell);
    const int beta = (ell + alpha - 1) / alpha;
    const int own_j = t < ell ? t / alpha : -1;
    const uint32_t c0 = blockIdx.x * C;
    const uint32_t gal = F.galois;
    const u64 p = pinfo[prime].p, np = u64(0) - p;
    auto sidx = [&](int b, int r) -> int { return b * RS + r + (r >> A); };
    auto group_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(1 + grp) : "memory"); };
    auto src_block = [&](uint32_t oblk) -> uint32_t {
        return gal == 1 ? oblk : (automorph_src(oblk << L2, gal, logN) >> L2);
    };
    // shared-memory buffer of digit j (the digits with a pass, in order)
    auto buf = [&](int j) -> int { return (own_j >= 0 && j > own_j) ? j - 1 : j; };

    // ---- 0. the key rows and the own limb's blocks into L2
    if (tid == 0) {
        const uint32_t rowb = uint32_t(CR) * sizeof(u64);
        for (int j = 0; j < beta; j++) {
            for (int ab = COMP ? 1 : 0; ab < 2; ab++) {
                const u64 *src = COMP ? F.key + (size_t(j) * LK + prime) * N
                                      : F.key + ((size_t(j) * 2 + ab) * LK + prime) * N;
                l2_prefetch(src + (size_t(c0) << L2), rowb);
            }
        }
        if (own_j >= 0)
            for (int b = 0; b < C; b++)
                l2_prefetch(F.own + size_t(t) * N + (size_t(src_block(c0 + b)) << L2), uint32_t(R) * sizeof(u64));
    }

    // ---- 1. pass C of the digits' new limbs (group grp: the grp-th digit with a pass)
    const int jd = (own_j >= 0 && grp >= own_j) ? grp + 1 : grp;
    if (jd < beta) {
        u64 *gs = dig + grp * (C * RS);
        const uint32_t sblk = src_block(c0 + cl);
        const u64 *__restrict__ src = F.ext + (size_t(jd) * ext + t) * N + (size_t(sblk) << L2);
        const ulonglong2 *__restrict__ tw = twf_all + size_t(prime) * N;
        auto TW = [&](int sigma, int r) -> ulonglong2 {
            return ld_keep(&tw[(1u << (L1 + sigma)) + (sblk << sigma) + (uint32_t(r) >> (LOGR - sigma))]);
        };
        u64 x[E];
#pragma unroll
        for (int q = 0; q < E; q++) x[q] = src[g + (q << B)];
#pragma unroll
        for (int sg = 0; sg < A; sg++) {
            const int half = 1 << (A - 1 - sg);
#pragma unroll
            for (int q = 0; q < E; q++) {
                if (q & half) continue;
                ct_bfly<true>(x[q], x[q + half], TW(sg, g + (q << B)), p, np);
            }
        }
#pragma unroll
        for (int q = 0; q < E; q++) gs[sidx(cl, g + (q << B))] = x[q];
        group_sync();
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = gs[sidx(cl, (g << A) + e)];
#pragma unroll
        for (int sg = A; sg < LOGR; sg++) {
            const int half = 1 << (LOGR - 1 - sg);
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & half) continue;
                ct_bfly<true>(x[e], x[e + half], TW(sg, (g << A) + e), p, np);
            }
        }
#pragma unroll
        for (int e = 0; e < E; e++) gs[sidx(cl, (g << A) + e)] = x[e];  // the slots this thread read
    }
    __syncthreads();

    // ---- 2. the inner product, PAIRS slot pairs per thread
    const PrimeInfo P = pinfo[prime];
    const int shift = __clzll(p);
#pragma unroll
    for (int q = 0; q < PAIRS; q++) {
        const int pi = tid + q * 256;
        const int b = pi / (R / 2), r = (pi % (R / 2)) * 2;
        const uint32_t n0 = ((c0 + uint32_t(b)) << L2) + uint32_t(r);
        const uint32_t s = gal == 1 ? n0 : automorph_src(n0, gal, logN);
        const int rs = int(s & uint32_t(R - 1)) & ~1;
        const bool swap = s & 1u;
        u64 ul0 = 0, uh0 = 0, ul1 = 0, uh1 = 0, vl0 = 0, vh0 = 0, vl1 = 0, vh1 = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (j < beta) {
                ulonglong2 dv;
                if (j == own_j) {
                    const u64 *o = F.own + size_t(t) * N + (size_t(s >> L2) << L2);
                    dv = *reinterpret_cast<const ulonglong2 *>(o + rs);
                } else {
                    const u64 *gs = dig + buf(j) * (C * RS);
                    dv = make_ulonglong2(gs[sidx(b, rs)], gs[sidx(b, rs + 1)]);
                }
                if (swap) {
                    const u64 tmp = dv.x;
                    dv.x = dv.y;
                    dv.y = tmp;
                }
                ulonglong2 ka, kb;
                if (COMP) {
                    kb = __ldcs(reinterpret_cast<const ulonglong2 *>(F.key + (size_t(j) * LK + prime) * N + n0));
                    const u64 e0 = (u64(j) * LK + prime) * N + n0;
                    ka = make_ulonglong2(key_a_element(F.seed, e0, p, shift), key_a_element(F.seed, e0 + 1, p, shift));
                } else {
                    ka = __ldcs(reinterpret_cast<const ulonglong2 *>(F.key + ((size_t(j) * 2 + 0) * LK + prime) * N + n0));
                    kb = __ldcs(reinterpret_cast<const ulonglong2 *>(F.key + ((size_t(j) * 2 + 1) * LK + prime) * N + n0));
                }
                mac128(ul0, uh0, dv.x, ka.x);
                mac128(ul1, uh1, dv.y, ka.y);
                mac128(vl0, vh0, dv.x, kb.x);
                mac128(vl1, vh1, dv.y, kb.y);
            }
        }
        const ulonglong2 uo = make_ulonglong2(reduce128(ul0, uh0, P), reduce128(ul1, uh1, P));
        const ulonglong2 vo = make_ulonglong2(reduce128(vl0, vh0, P), reduce128(vl1, vh1, P));
        if (t < ell) {
            const size_t o = size_t(t) * N + n0;
            *reinterpret_cast<ulonglong2 *>(F.u + o) = uo;
            *reinterpret_cast<ulonglong2 *>(F.v + o) = vo;
        } else {
            uvs[sidx(b, r)] = uo.x;
            uvs[sidx(b, r + 1)] = uo.y;
            uvs[C * RS + sidx(b, r)] = vo.x;
            uvs[C * RS + sidx(b, r + 1)] = vo.y;
        }
    }
    if (t < ell) return;  // uniform: t is the CTA's

    // ---- 3. special positions: pass C of the inverse NTT on u (group 0) and v (group 1)
    __syncthreads();
    if (grp < 2) {
        const int poly = grp;
        u64 *gs = uvs + poly * (C * RS);
        const uint32_t oblk = c0 + cl;
        const ulonglong2 *__restrict__ tw = twi_all + size_t(prime) * N;
        auto TW = [&](int sigma, int r) -> ulonglong2 {
            return ld_keep(&tw[(1u << (L1 + sigma)) + (oblk << sigma) + (uint32_t(r) >> (LOGR - sigma))]);
        };
        u64 x[E];
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = gs[sidx(cl, (g << A) + e)];
#pragma unroll
        for (int sg = LOGR - 1; sg >= A; sg--) {
            const int half = 1 << (LOGR - 1 - sg);
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & half) continue;
                gs_bfly<true>(x[e], x[e + half], TW(sg, (g << A) + e), p, np);
            }
        }
#pragma unroll
        for (int e = 0; e < E; e++) gs[sidx(cl, (g << A) + e)] = x[e];
        group_sync();
#pragma unroll
        for (int q = 0; q < E; q++) x[q] = gs[sidx(cl, g + (q << B))];
#pragma unroll
        for (int sg = A - 1; sg >= 0; sg--) {
            const int half = 1 << (A - 1 - sg);
#pragma unroll
            for (int q = 0; q < E; q++) {
                if (q & half) continue;
                gs_bfly<true>(x[q], x[q + half], TW(sg, g + (q << B)), p, np);
            }
        }
        u64 *dst = (poly == 0 ? F.u : F.v) + size_t(t) * N + (size_t(oblk) << L2);
#pragma unroll
        for (int q = 0; q < E; q++) dst[g + (q << B)] = x[q];
    }
}

// ------------------------------------------------------------------ host side
namespace {

// CSEL picks the CTA width (the tile shape): 0 = the default below, 1 = half
// of it, 2 = twice it.  SPL moves the radix split: L2 = floor(logN/2) + SPL
// stages in pass C, the rest in pass S.  The autotuner (ntt_autotune) chooses
// the width per pass and batch size, and the split per direction and batch
// size (both passes of a transform share it); shapes other than the default
// exist for logN >= 14 with small primes (the key-switching shapes), and a
// split other than 0 only with the default width.
template <int LOGN, int SPL, bool INV, bool CONTIG, bool EPI, bool SMALLP, int CSEL, class MAP>
cudaError_t launch_one_p(const MAP &m, int count, const ckks_ctx *ctx, cudaStream_t st, bool set_attr) {
    // pass S transforms columns of 2^L1 rows, pass C blocks of 2^L2 words
    constexpr int L2 = (LOGN >> 1) + SPL, L1 = LOGN - L2;
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
    const size_t smem = CONTIG ? size_t(C) * (R + TPC) * 8 : size_t(R) * C * 8;
    auto kern = ntt_pass_kernel<LOGN, L2, LOGR, A, C, INV, CONTIG, EPI, SMALLP, MAP>;
    if (set_attr) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    dim3 grid(count, (1 << OTHER) / C);
    kern<<<grid, TPC * C, smem, st>>>(m, ctx->d_pinfo, INV ? ctx->d_tw_inv : ctx->d_tw_fwd);
    return cudaGetLastError();
}

template <int LOGN, bool INV, bool CONTIG, bool EPI, class MAP>
cudaError_t launch_one(const MAP &m, int count, const ckks_ctx *ctx, cudaStream_t st, bool set_attr, int csel,
                       int split) {
    constexpr bool TUNED = LOGN >= 14;
    constexpr int SM1 = TUNED ? -1 : 0, SP1 = TUNED ? 1 : 0;
    if (set_attr) {
        cudaError_t e = launch_one_p<LOGN, 0, INV, CONTIG, EPI, false, 0>(m, count, ctx, st, true);
        if (e == cudaSuccess) e = launch_one_p<LOGN, 0, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, true);
        if (TUNED && e == cudaSuccess) e = launch_one_p<LOGN, 0, INV, CONTIG, EPI, true, TUNED ? 1 : 0>(m, count, ctx, st, true);
        if (TUNED && e == cudaSuccess) e = launch_one_p<LOGN, 0, INV, CONTIG, EPI, true, TUNED ? 2 : 0>(m, count, ctx, st, true);
        if (TUNED && e == cudaSuccess) e = launch_one_p<LOGN, SM1, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, true);
        if (TUNED && e == cudaSuccess) e = launch_one_p<LOGN, SP1, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, true);
        return e;
    }
    if (!ctx->small_primes) return launch_one_p<LOGN, 0, INV, CONTIG, EPI, false, 0>(m, count, ctx, st, false);
    if (TUNED && split < 0) return launch_one_p<LOGN, SM1, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, false);
    if (TUNED && split > 0) return launch_one_p<LOGN, SP1, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, false);
    if (TUNED && csel == 1) return launch_one_p<LOGN, 0, INV, CONTIG, EPI, true, TUNED ? 1 : 0>(m, count, ctx, st, false);
    if (TUNED && csel == 2) return launch_one_p<LOGN, 0, INV, CONTIG, EPI, true, TUNED ? 2 : 0>(m, count, ctx, st, false);
    return launch_one_p<LOGN, 0, INV, CONTIG, EPI, true, 0>(m, count, ctx, st, false);
}

// The tuned width of a pass for a launch of `count` limbs (-1: use the table).
inline int csel_for(const ckks_ctx *ctx, bool contig, int count, int force) {
    if (force >= 0) return force;
    return ctx->ntt_csel[contig ? 1 : 0][count > kTuneSmallBatch ? 1 : 0];
}

// The tuned radix split of a transform of `count` limbs (both passes).
inline int split_for(const ckks_ctx *ctx, bool inv, int count) {
    return ctx->ntt_split[inv ? 1 : 0][count > kTuneSmallBatch ? 1 : 0];
}

// split: the radix split both passes of this transform use (split_for, or 0
// where another kernel runs the other pass with the default split).
template <bool INV, bool CONTIG, bool EPI, class MAP>
cudaError_t dispatch(const MAP &m, int count, const ckks_ctx *ctx, cudaStream_t st, bool set_attr, int split,
                     int force = -1) {
    const int cs = csel_for(ctx, CONTIG, count, force);
    switch (ctx->logN) {
    case 10: return launch_one<10, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    case 11: return launch_one<11, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    case 12: return launch_one<12, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    case 13: return launch_one<13, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    case 14: return launch_one<14, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    case 15: return launch_one<15, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    case 16: return launch_one<16, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    case 17: return launch_one<17, INV, CONTIG, EPI>(m, count, ctx, st, set_attr, cs, split);
    default: return cudaErrorInvalidValue;
    }
}

template <class MAP>
cudaError_t set_attributes_for(const ckks_ctx *ctx) {
    MAP m{};
    cudaError_t err;
    if ((err = dispatch<false, false, false>(m, 0, ctx, nullptr, true, 0)) != cudaSuccess) return err;
    if ((err = dispatch<false, true, false>(m, 0, ctx, nullptr, true, 0)) != cudaSuccess) return err;
    if ((err = dispatch<false, true, true>(m, 0, ctx, nullptr, true, 0)) != cudaSuccess) return err;
    if ((err = dispatch<true, true, false>(m, 0, ctx, nullptr, true, 0)) != cudaSuccess) return err;
    return dispatch<true, false, false>(m, 0, ctx, nullptr, true, 0);
}

// Two passes of one transform: the second runs in place on the first's output.
template <class MAP>
cudaError_t run_fwd(MAP m, int count, bool epi, const ckks_ctx *ctx, cudaStream_t st) {
    cudaError_t err;
    const int split = split_for(ctx, false, count);
    m.second = 0;
    {
        ProfScope ps(ctx, K_NTT_FWD, count, st);
        err = dispatch<false, false, false>(m, count, ctx, st, false, split);
    }
    if (err != cudaSuccess) return err;
    m.second = 1;
    ProfScope ps(ctx, K_NTT_FWD, count, st);
    if (epi) return dispatch<false, true, true>(m, count, ctx, st, false, split);
    return dispatch<false, true, false>(m, count, ctx, st, false, split);
}

template <class MAP>
cudaError_t run_inv(MAP m, int count, const ckks_ctx *ctx, cudaStream_t st) {
    cudaError_t err;
    const int split = split_for(ctx, true, count);
    m.second = 0;
    {
        ProfScope ps(ctx, K_NTT_INV, count, st);
        err = dispatch<true, true, false>(m, count, ctx, st, false, split);
    }
    if (err != cudaSuccess) return err;
    m.second = 1;
    ProfScope ps(ctx, K_NTT_INV, count, st);
    return dispatch<true, false, false>(m, count, ctx, st, false, split);
}

}  // namespace

static cudaError_t modup_ip_dispatch(const ckks_ctx *ctx, const FusedIpArgs &f, cudaStream_t st, bool set_attr);

cudaError_t ntt_set_attributes(const ckks_ctx *ctx) {
    cudaError_t err = set_attributes_for<MapList>(ctx);
    if (err != cudaSuccess) return err;
    err = set_attributes_for<MapBatch>(ctx);
    if (err != cudaSuccess || ctx->logN < 10 || ctx->logN > 17) return err;
    return modup_ip_dispatch(ctx, FusedIpArgs{}, nullptr, true);
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

// ------------------------------------------------------------------ fused ModUp tail launchers
template <int LOGN>
static size_t modup_ip_smem(int groups) {
    constexpr int L2 = LOGN >> 1, A = (L2 + 1) / 2, B = L2 - A, TPC = 1 << B;
    constexpr int C = 64 / TPC, RS = (1 << L2) + TPC;
    return size_t(groups + 2) * C * RS * sizeof(u64);
}

// One launch over every extended position, 256 threads.  Two variants were
// measured slower at N=2^16, ell=24, dnum=3: beta groups only (192 threads,
// one launch) and separate launches for the chain positions (beta - 1 busy
// groups) and the special positions (whose few CTAs then run as a tail).
template <int LOGN>
static cudaError_t launch_modup_ip_n(const ckks_ctx *ctx, const FusedIpArgs &f, cudaStream_t st, bool set_attr) {
    constexpr int L2 = LOGN >> 1, L1 = LOGN - L2, A = (L2 + 1) / 2, B = L2 - A, TPC = 1 << B;
    constexpr int C = 64 / TPC;
    if (set_attr) {
        const int smax = int(modup_ip_smem<LOGN>(4));
        cudaError_t e = cudaFuncSetAttribute(modup_ip_kernel<LOGN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(modup_ip_kernel<LOGN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        return e;
    }
    const int beta = beta_of(ctx, f.ell);  // at most 4 (modup_ip_supported)
    const struct {
        int t0, count, groups;
    } parts[1] = {{0, f.ell + ctx->k, 4}};
    (void)beta;
    for (const auto &pt : parts) {
        const dim3 grid(unsigned((1 << L1) / C), unsigned(pt.count));
        const size_t smem = modup_ip_smem<LOGN>(pt.groups);
        if (f.compressed)
            modup_ip_kernel<LOGN, true><<<grid, 64 * pt.groups, smem, st>>>(f, ctx->d_pinfo, ctx->d_tw_fwd, ctx->d_tw_inv,
                                                                           ctx->L, ctx->k, ctx->alpha, pt.t0);
        else
            modup_ip_kernel<LOGN, false><<<grid, 64 * pt.groups, smem, st>>>(f, ctx->d_pinfo, ctx->d_tw_fwd,
                                                                            ctx->d_tw_inv, ctx->L, ctx->k, ctx->alpha,
                                                                            pt.t0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t modup_ip_dispatch(const ckks_ctx *ctx, const FusedIpArgs &f, cudaStream_t st, bool set_attr) {
    switch (ctx->logN) {
    case 10: return launch_modup_ip_n<10>(ctx, f, st, set_attr);
    case 11: return launch_modup_ip_n<11>(ctx, f, st, set_attr);
    case 12: return launch_modup_ip_n<12>(ctx, f, st, set_attr);
    case 13: return launch_modup_ip_n<13>(ctx, f, st, set_attr);
    case 14: return launch_modup_ip_n<14>(ctx, f, st, set_attr);
    case 15: return launch_modup_ip_n<15>(ctx, f, st, set_attr);
    case 16: return launch_modup_ip_n<16>(ctx, f, st, set_attr);
    case 17: return launch_modup_ip_n<17>(ctx, f, st, set_attr);
    default: return cudaErrorInvalidValue;
    }
}

bool modup_ip_supported(const ckks_ctx *ctx, int ell) {
    return ctx->small_primes && beta_of(ctx, ell) <= 4 && ctx->logN >= 10 && ctx->logN <= 17;
}

cudaError_t launch_modup_ip(const ckks_ctx *ctx, const FusedIpArgs &f, cudaStream_t st) {
    ProfScope ps(ctx, K_FUSED, f.ell + ctx->k, st);
    return modup_ip_dispatch(ctx, f, st, false);
}

// Pass S alone of the forward transform (src -> dst, lazy values), with the
// default radix split: the fused ModUp tail runs pass C.
cudaError_t launch_ntt_fwd_colpass(const ckks_ctx *ctx, const NttBatch &b, cudaStream_t st) {
    if (b.count == 0) return cudaSuccess;
    MapList m;
    m.b = b;
    m.e = Epi{};
    m.e.mode = EPI_STORE;
    m.second = 0;
    ProfScope ps(ctx, K_NTT_FWD, b.count, st);
    return dispatch<false, false, false>(m, b.count, ctx, st, false, 0);
}

// Pass S alone of the inverse transform, in place on dst, with the default
// radix split (pass C ran in the fused ModUp tail).
cudaError_t launch_ntt_inv_colpass(const ckks_ctx *ctx, const NttBatch &b, cudaStream_t st) {
    if (b.count == 0) return cudaSuccess;
    MapList m;
    m.b = b;
    m.e = Epi{};
    m.e.mode = EPI_STORE;
    m.second = 1;
    ProfScope ps(ctx, K_NTT_INV, b.count, st);
    return dispatch<true, false, false>(m, b.count, ctx, st, false, 0);
}

// ------------------------------------------------------------------ butterfly ceiling
// Register-only throughput of the forward butterfly of the transforms (the
// measured ceiling of their ALU roofline): every thread keeps 16 words in
// registers and runs rounds of 4 lazy Cooley-Tukey stages (8 butterflies per
// stage, one twiddle per stage held in registers), with no memory access
// inside the loop.  The instruction stream is that of ct_bfly<true>; the values
// wrap and mean nothing, so one word per thread is stored only to keep the
// work.  Launched at the transforms' occupancy (32 warps per SM).
__global__ void __launch_bounds__(256) bfly_peak_kernel(int rounds, const PrimeInfo *__restrict__ pinfo,
                                                        const ulonglong2 *__restrict__ tw, u64 *__restrict__ sink) {
    const u64 p = pinfo[0].p, np = u64(0) - p;
    ulonglong2 w[4];
#pragma unroll
    for (int sg = 0; sg < 4; sg++) w[sg] = tw[1 + sg + (threadIdx.x & 7)];
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = (u64(blockIdx.x * blockDim.x + threadIdx.x) << 20) + u64(k) * 977u;
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int sg = 0; sg < 4; sg++) {
            const int half = 8 >> sg;
#pragma unroll
            for (int k = 0; k < 16; k++) {
                if (k & half) continue;
                ct_bfly<true>(x[k], x[k + half], w[sg], p, np);
            }
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) acc ^= x[k];
    sink[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = acc;
}

cudaError_t launch_bfly_peak(const ckks_ctx *ctx, int rounds, u64 *sink, cudaStream_t st, double *butterflies) {
    const int threads = 256, blocks = ctx->sms * 4;  // 32 warps per SM
    bfly_peak_kernel<<<blocks, threads, 0, st>>>(rounds, ctx->d_pinfo, ctx->d_tw_fwd, sink);
    *butterflies = double(blocks) * threads * rounds * 32.0;
    return cudaGetLastError();
}

size_t bfly_peak_sink_words(const ckks_ctx *ctx) { return size_t(ctx->sms) * 4 * 256; }

// ------------------------------------------------------------------ autotuner
// Times every CTA width of the column pass (S) and the block pass (C), forward
// and inverse together, on `small` and `large` limbs of scratch data (in
// place, values are transformed and transformed back), and keeps the fastest
// per pass and batch-size class; then, with those widths, times whole forward
// and whole inverse transforms at each radix split (0, -1, +1: pass C gets
// floor(logN/2) + split stages) and keeps the fastest per direction and class.
// The default shape is kept unless another is faster by a margin (0.5% for a
// width, 3% for a split; policy::tune_choose): closer timings are within the
// run-to-run spread of launches timed alone, and inside a step of concurrent
// calls an unbalanced split measured up to 12% slower.  scratch: at least
// large * N words.  The choices go to ctx->ntt_csel and ctx->ntt_split;
// times_out (24 floats, ms per run) gets the widths' times at
// [(pass * 2 + class) * 3 + width] and the splits' at
// 12 + [(direction * 2 + class) * 3 + split + 1].
cudaError_t ntt_autotune(ckks_ctx *ctx, u64 *scratch, int small, int large, cudaStream_t st, float *times_out) {
    if (ctx->logN < 14 || !ctx->small_primes) return cudaSuccess;  // one shape only
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
    // ms per run of `run` (two warm-up runs, then 10 timed runs)
    constexpr int kReps = 10;
    auto timed = [&](auto run, float *ms) {
        cudaError_t e2 = run();
        if (e2 == cudaSuccess) e2 = run();
        if (e2 != cudaSuccess) return e2;
        cudaEventRecord(e0, st);
        for (int r = 0; r < kReps && e2 == cudaSuccess; ++r) e2 = run();
        cudaEventRecord(e1, st);
        if (e2 == cudaSuccess) e2 = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e2 == cudaSuccess) e2 = cudaEventElapsedTime(&t, e0, e1);
        *ms = t / kReps;
        return e2;
    };
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
        m.second = 1;
        for (int contig = 0; contig < 2 && err == cudaSuccess; ++contig) {
            float t[3] = {0.f, 0.f, 0.f};
            for (int cs = 0; cs < 3 && err == cudaSuccess; ++cs) {
                auto run = [&]() {
                    cudaError_t e2 = contig ? dispatch<false, true, false>(m, count, ctx, st, false, 0, cs)
                                            : dispatch<false, false, false>(m, count, ctx, st, false, 0, cs);
                    if (e2 == cudaSuccess)
                        e2 = contig ? dispatch<true, true, false>(m, count, ctx, st, false, 0, cs)
                                    : dispatch<true, false, false>(m, count, ctx, st, false, 0, cs);
                    return e2;
                };
                err = timed(run, &t[cs]);
                if (err != cudaSuccess) break;
                if (times_out) times_out[(contig * 2 + bucket) * 3 + cs] = t[cs];
            }
            if (err == cudaSuccess) ctx->ntt_csel[contig][bucket] = policy::tune_choose(t, 0.005f);
        }
        for (int inv = 0; inv < 2 && err == cudaSuccess; ++inv) {
            float t[3] = {0.f, 0.f, 0.f};  // splits 0, -1, +1
            for (int o = 0; o < 3 && err == cudaSuccess; ++o) {
                const int sp = o == 0 ? 0 : (o == 1 ? -1 : 1);
                auto run = [&]() {
                    cudaError_t e2 = inv ? dispatch<true, true, false>(m, count, ctx, st, false, sp)
                                         : dispatch<false, false, false>(m, count, ctx, st, false, sp);
                    if (e2 == cudaSuccess)
                        e2 = inv ? dispatch<true, false, false>(m, count, ctx, st, false, sp)
                                 : dispatch<false, true, false>(m, count, ctx, st, false, sp);
                    return e2;
                };
                err = timed(run, &t[o]);
                if (err != cudaSuccess) break;
                if (times_out) times_out[12 + (inv * 2 + bucket) * 3 + sp + 1] = t[o];
            }
            if (err == cudaSuccess) {
                const int o = policy::tune_choose(t, 0.03f);
                ctx->ntt_split[inv][bucket] = o == 0 ? 0 : (o == 1 ? -1 : 1);
            }
        }
    }
    ctx->prof_on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

}  // namespace ckks
