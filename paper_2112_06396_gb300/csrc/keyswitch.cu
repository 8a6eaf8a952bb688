// keyswitch.cu -- KSKInnerProd, Automorph, PModUp, the fused inner loop of
// PtMatVecMult (Algorithm 8) and the element-wise steps of key generation.
//
// Automorph in bit-reversed evaluation order maps every aligned block of 2^m
// slots onto an aligned block of 2^m slots (the low bits of a slot index only
// reach the high bits of its evaluation exponent), so a thread that owns the
// slot pair (2n, 2n+1) reads one aligned source pair, swapped when the image
// of 2n is odd.  Gathers therefore stay 16-byte vector loads and every warp
// touches whole 256-byte segments.
#include "batch.cuh"
#include "common.cuh"
#include "internal.h"
#include "launch_policy.h"
#include "prng.cuh"

#include <algorithm>

namespace ckks {

__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *reinterpret_cast<const ulonglong2 *>(p); }
__device__ __forceinline__ void st2(u64 *p, ulonglong2 v) { *reinterpret_cast<ulonglong2 *>(p) = v; }
// Key-switching keys are read once per operation: stream them past L1 and L2.
__device__ __forceinline__ ulonglong2 ld2_stream(const u64 *p) { return __ldcs(reinterpret_cast<const ulonglong2 *>(p)); }

// Load the automorphed pair (out slots n0, n0+1) of one limb.
__device__ __forceinline__ ulonglong2 ld2_perm(const u64 *limb, uint32_t n0, uint32_t g, int logN) {
    if (g == 1) return ld2(limb + n0);
    const uint32_t s = automorph_src(n0, g, logN);
    ulonglong2 v = ld2(limb + (s & ~1u));
    if (s & 1u) {
        const u64 t = v.x;
        v.x = v.y;
        v.y = t;
    }
    return v;
}

// ------------------------------------------------------------------ KSKInnerProd
// u_t = sum_{j<beta} d_j[t] * key[j][0][t'], v_t = sum_j d_j[t] * key[j][1][t']
// (t' = key row of position t), with d_j read through Automorph_g.  The
// digit's own limbs come from `own` when given (ModUp copies them unchanged).
// With padd set (NewMult), P*padd[0] and P*padd[1] join the sums on the chain
// positions (PModUp is 0 on the P positions), before the one reduction.
__device__ __forceinline__ void add_pmodup(const InnerArgs &A, int t, uint32_t n0, size_t N, ulonglong2 pm, u64 &ul0,
                                           u64 &uh0, u64 &ul1, u64 &uh1, u64 &vl0, u64 &vh0, u64 &vl1, u64 &vh1) {
    if (A.padd[0] == nullptr || t >= A.ell) return;
    const ulonglong2 b = ld2(A.padd[0] + size_t(t) * N + n0), c = ld2(A.padd[1] + size_t(t) * N + n0);
    mac128(ul0, uh0, b.x, pm.x);
    mac128(ul1, uh1, b.y, pm.x);
    mac128(vl0, vh0, c.x, pm.x);
    mac128(vl1, vh1, c.y, pm.x);
}

// COMP: the key is compressed (rows b_j only); a_j is drawn from A.seed while
// the loads are in flight.
template <int BETA, bool COMP>
__global__ void __launch_bounds__(256) inner_prod_kernel(InnerArgs A, const PrimeInfo *__restrict__ pinfo, int logN,
                                                         int L, int k, int alpha, const ulonglong2 *__restrict__ Pmod) {
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int t = blockIdx.y;
    const int ell = A.ell, ext = ell + k, LK = L + k;
    const int prime = t < ell ? t : L + (t - ell);
    // all 3*BETA loads are issued before the first multiply
    ulonglong2 dv[BETA], ka[BETA], kb[BETA];
#pragma unroll
    for (int j = 0; j < BETA; j++) {
        const bool own = (A.own != nullptr) && t < ell && (t / alpha) == j;
        const u64 *d = own ? A.own + size_t(t) * N : A.ext + (size_t(j) * ext + t) * N;
        dv[j] = ld2_perm(d, n0, A.galois, logN);
        if (COMP) {
            kb[j] = ld2_stream(A.key + (size_t(j) * LK + prime) * N + n0);
        } else {
            ka[j] = ld2_stream(A.key + ((size_t(j) * 2 + 0) * LK + prime) * N + n0);
            kb[j] = ld2_stream(A.key + ((size_t(j) * 2 + 1) * LK + prime) * N + n0);
        }
    }
    const PrimeInfo P = pinfo[prime];
    if (COMP) {
        const int shift = __clzll(P.p);
#pragma unroll
        for (int j = 0; j < BETA; j++) {
            const u64 e = (u64(j) * LK + prime) * N + n0;
            ka[j] = make_ulonglong2(key_a_element(A.seed, e, P.p, shift), key_a_element(A.seed, e + 1, P.p, shift));
        }
    }
    u64 ul0 = 0, uh0 = 0, ul1 = 0, uh1 = 0, vl0 = 0, vh0 = 0, vl1 = 0, vh1 = 0;
#pragma unroll
    for (int j = 0; j < BETA; j++) {
        mac128(ul0, uh0, dv[j].x, ka[j].x);
        mac128(ul1, uh1, dv[j].y, ka[j].y);
        mac128(vl0, vh0, dv[j].x, kb[j].x);
        mac128(vl1, vh1, dv[j].y, kb[j].y);
    }
    add_pmodup(A, t, n0, N, Pmod[prime], ul0, uh0, ul1, uh1, vl0, vh0, vl1, vh1);
    st2(A.u + size_t(t) * N + n0, make_ulonglong2(reduce128(ul0, uh0, P), reduce128(ul1, uh1, P)));
    st2(A.v + size_t(t) * N + n0, make_ulonglong2(reduce128(vl0, vh0, P), reduce128(vl1, vh1, P)));
}

// beta > 4: loop over digits
template <bool COMP>
__global__ void __launch_bounds__(256) inner_prod_kernel_any(InnerArgs A, const PrimeInfo *__restrict__ pinfo, int logN,
                                                             int L, int k, int alpha,
                                                             const ulonglong2 *__restrict__ Pmod) {
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int t = blockIdx.y;
    const int ell = A.ell, ext = ell + k, LK = L + k;
    const int beta = (ell + alpha - 1) / alpha;
    const int prime = t < ell ? t : L + (t - ell);
    const PrimeInfo P = pinfo[prime];
    u64 ul0 = 0, uh0 = 0, ul1 = 0, uh1 = 0, vl0 = 0, vh0 = 0, vl1 = 0, vh1 = 0;
    for (int j = 0; j < beta; j++) {
        const bool own = (A.own != nullptr) && t < ell && (t / alpha) == j;
        const u64 *d = own ? A.own + size_t(t) * N : A.ext + (size_t(j) * ext + t) * N;
        const ulonglong2 dv = ld2_perm(d, n0, A.galois, logN);
        ulonglong2 ka, kb;
        if (COMP) {
            const u64 e = (u64(j) * LK + prime) * N + n0;
            const int shift = __clzll(P.p);
            ka = make_ulonglong2(key_a_element(A.seed, e, P.p, shift), key_a_element(A.seed, e + 1, P.p, shift));
            kb = ld2_stream(A.key + (size_t(j) * LK + prime) * N + n0);
        } else {
            ka = ld2_stream(A.key + ((size_t(j) * 2 + 0) * LK + prime) * N + n0);
            kb = ld2_stream(A.key + ((size_t(j) * 2 + 1) * LK + prime) * N + n0);
        }
        mac128(ul0, uh0, dv.x, ka.x);
        mac128(ul1, uh1, dv.y, ka.y);
        mac128(vl0, vh0, dv.x, kb.x);
        mac128(vl1, vh1, dv.y, kb.y);
    }
    add_pmodup(A, t, n0, N, Pmod[prime], ul0, uh0, ul1, uh1, vl0, vh0, vl1, vh1);
    st2(A.u + size_t(t) * N + n0, make_ulonglong2(reduce128(ul0, uh0, P), reduce128(ul1, uh1, P)));
    st2(A.v + size_t(t) * N + n0, make_ulonglong2(reduce128(vl0, vh0, P), reduce128(vl1, vh1, P)));
}

cudaError_t launch_inner_prod(const ckks_ctx *ctx, const InnerArgs &a, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(a.ell + ctx->k));
    ProfScope ps(ctx, K_INNER, a.ell + ctx->k, st);
    const int beta = beta_of(ctx, a.ell);
#define CKKS_IP(B, CMP)                                                                                            \
    inner_prod_kernel<B, CMP><<<grid, threads, 0, st>>>(a, ctx->d_pinfo, ctx->logN, ctx->L, ctx->k, ctx->alpha,    \
                                                        ctx->d_Pmod)
#define CKKS_IP_BETA(CMP)                                                                                          \
    switch (beta) {                                                                                                \
    case 1: CKKS_IP(1, CMP); break;                                                                                \
    case 2: CKKS_IP(2, CMP); break;                                                                                \
    case 3: CKKS_IP(3, CMP); break;                                                                                \
    case 4: CKKS_IP(4, CMP); break;                                                                                \
    default:                                                                                                       \
        inner_prod_kernel_any<CMP><<<grid, threads, 0, st>>>(a, ctx->d_pinfo, ctx->logN, ctx->L, ctx->k,           \
                                                             ctx->alpha, ctx->d_Pmod);                             \
    }
    if (a.compressed) {
        CKKS_IP_BETA(true)
    } else {
        CKKS_IP_BETA(false)
    }
#undef CKKS_IP_BETA
#undef CKKS_IP
    return cudaGetLastError();
}

// Batched KSKInnerProd.  The grid is (entry, coefficient tile, prime of the
// extended basis) with the entry index fastest, so the CTAs of every entry at
// one (tile, prime) are scheduled back to back: a key shared by several
// entries is fetched from DRAM by the first of them and served from L2 to the
// rest (cached loads, unlike the single-ciphertext kernel, whose key is used
// once and streamed).  A chain prime q_i belongs to the entries with ell > i
// (position i), a special prime p_m to every entry (position ell + m); CTAs of
// entries below a chain prime exit at once.  Each entry reads its own digits
// through its own Galois element and writes its u, v into its workspace.
// Full keys only (a batch with a compressed key goes to the grouped kernel).
template <int BMAX>
__global__ void __launch_bounds__(256) inner_prod_batch_kernel(const __grid_constant__ KsBatchDesc d,
                                                               const PrimeInfo *__restrict__ pinfo,
                                                               const ulonglong2 *__restrict__ Pmod) {
    const CtDesc &ct = d.ct[blockIdx.x];
    const int ell = ct.ell;
    const int pi = blockIdx.z;
    if (pi < d.L && pi >= ell) return;
    const int logN = d.logN;
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.y * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int LK = d.L + d.k, alpha = d.alpha;
    const int t = pi < d.L ? pi : ell + (pi - d.L);
    const CtLayout lo = ct_layout(d, ct);
    const int beta = lo.beta;
    const uint32_t g = ct.galois;
    const u64 *key = ct.key;
    u64 ul0 = 0, uh0 = 0, ul1 = 0, uh1 = 0, vl0 = 0, vh0 = 0, vl1 = 0, vh1 = 0;
    if constexpr (BMAX > 0) {
        ulonglong2 dv[BMAX], ka[BMAX], kb[BMAX];
#pragma unroll
        for (int j = 0; j < BMAX; j++) {
            if (j < beta) {
                const bool own = t < ell && (t / alpha) == j;
                const u64 *src = own ? ct.a + size_t(t) * N : lo.extp + (size_t(j) * lo.ext + t) * N;
                dv[j] = ld2_perm(src, n0, g, logN);
                ka[j] = ld2(key + ((size_t(j) * 2 + 0) * LK + pi) * N + n0);
                kb[j] = ld2(key + ((size_t(j) * 2 + 1) * LK + pi) * N + n0);
            }
        }
#pragma unroll
        for (int j = 0; j < BMAX; j++) {
            if (j < beta) {
                mac128(ul0, uh0, dv[j].x, ka[j].x);
                mac128(ul1, uh1, dv[j].y, ka[j].y);
                mac128(vl0, vh0, dv[j].x, kb[j].x);
                mac128(vl1, vh1, dv[j].y, kb[j].y);
            }
        }
    } else {
        for (int j = 0; j < beta; j++) {
            const bool own = t < ell && (t / alpha) == j;
            const u64 *src = own ? ct.a + size_t(t) * N : lo.extp + (size_t(j) * lo.ext + t) * N;
            const ulonglong2 dv = ld2_perm(src, n0, g, logN);
            const ulonglong2 a2 = ld2(key + ((size_t(j) * 2 + 0) * LK + pi) * N + n0);
            const ulonglong2 b2 = ld2(key + ((size_t(j) * 2 + 1) * LK + pi) * N + n0);
            mac128(ul0, uh0, dv.x, a2.x);
            mac128(ul1, uh1, dv.y, a2.y);
            mac128(vl0, vh0, dv.x, b2.x);
            mac128(vl1, vh1, dv.y, b2.y);
        }
    }
    if (ct.merged && t < ell) {
        // NewMult: PModUp(b3), PModUp(c3) join the sums before the one reduction
        const u64 pm = Pmod[pi].x;
        const ulonglong2 b = ld2(ct.add[0] + size_t(t) * N + n0), c = ld2(ct.add[1] + size_t(t) * N + n0);
        mac128(ul0, uh0, b.x, pm);
        mac128(ul1, uh1, b.y, pm);
        mac128(vl0, vh0, c.x, pm);
        mac128(vl1, vh1, c.y, pm);
    }
    const PrimeInfo P = pinfo[pi];
    st2(lo.uv + size_t(t) * N + n0, make_ulonglong2(reduce128(ul0, uh0, P), reduce128(ul1, uh1, P)));
    st2(lo.uv + (size_t(lo.ext) + t) * N + n0, make_ulonglong2(reduce128(vl0, vh0, P), reduce128(vl1, vh1, P)));
}

// Batched KSKInnerProd for batches that hold a compressed key.  Consecutive
// entries that use the same key (same rows, same compression and seed) form
// groups (sized by the launcher); the grid is (group, coefficient tile, prime
// of the extended basis).  A CTA regenerates (or loads) the key rows of its tile
// once and serves every entry of its group with them, so a compressed key
// shared across a batch is generated once per group instead of once per entry.
// (With full keys the per-entry kernel above is faster: a shared key row comes
// from L2 after the first entry, and holding the rows across entries costs
// registers, hence resident warps.)  A chain prime q_i belongs to the entries
// with ell > i (position i), a special prime p_m to every entry (position
// ell + m); the key rows are those of the deepest digit among the group's
// entries at this prime.  Each entry reads its own digits through its own
// Galois element and writes its u, v into its workspace; the next entry's
// digits are fetched while the current one is accumulated.
template <int BMAX>
__global__ void __launch_bounds__(256, 4) inner_prod_group_kernel(const __grid_constant__ KsBatchDesc d,
                                                               const __grid_constant__ IpGroups G,
                                                               const PrimeInfo *__restrict__ pinfo,
                                                               const ulonglong2 *__restrict__ Pmod) {
    const int c0 = G.start[blockIdx.x], c1 = G.start[blockIdx.x + 1];
    const int pi = blockIdx.z;
    const int logN = d.logN;
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.y * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int LK = d.L + d.k, alpha = d.alpha;
    // entries of the group that own this prime, and the deepest digit among them
    int bmax = 0;
    for (int c = c0; c < c1; ++c) {
        const int ell = d.ct[c].ell;
        if (pi >= d.L || pi < ell) bmax = max(bmax, (ell + alpha - 1) / alpha);
    }
    if (bmax == 0) return;
    const CtDesc &first = d.ct[c0];
    const u64 *key = first.key;
    const bool comp = first.compressed;  // this group's key
    const PrimeInfo P = pinfo[pi];
    constexpr int KB = BMAX > 0 ? BMAX : 1;
    if constexpr (BMAX > 0) {
        ulonglong2 ka[KB], kb[KB], dv[KB], nx[KB] = {};  // slots the next entry lacks stay 0
#pragma unroll
        for (int j = 0; j < KB; j++) {
            if (j < bmax) {
                if (comp) {
                    kb[j] = ld2(key + (size_t(j) * LK + pi) * N + n0);
                } else {
                    ka[j] = ld2(key + ((size_t(j) * 2 + 0) * LK + pi) * N + n0);
                    kb[j] = ld2(key + ((size_t(j) * 2 + 1) * LK + pi) * N + n0);
                }
            }
        }
        // the first owning entry's digits, in flight with the key rows
        int c = c0;
        while (c < c1 && !(pi >= d.L || pi < d.ct[c].ell)) ++c;
        // entry e's digits at this prime into out[0 .. beta-1]
        auto fetch = [&](int e, ulonglong2 *out) {
            const CtDesc &ct = d.ct[e];
            const int ell = ct.ell, t = pi < d.L ? pi : ell + (pi - d.L);
            const CtLayout lo = ct_layout(d, ct);
#pragma unroll
            for (int j = 0; j < KB; j++) {
                if (j < lo.beta) {
                    const bool own = t < ell && (t / alpha) == j;
                    const u64 *src = own ? ct.a + size_t(t) * N : lo.extp + (size_t(j) * lo.ext + t) * N;
                    out[j] = ld2_perm(src, n0, ct.galois, logN);
                }
            }
        };
        fetch(c, dv);
        if (comp) {
            // the key's uniform half, regenerated while the loads are in flight
            const int shift = __clzll(P.p);
#pragma unroll
            for (int j = 0; j < KB; j++) {
                if (j < bmax) {
                    const u64 e = (u64(j) * LK + pi) * N + n0;
                    ka[j] = make_ulonglong2(key_a_element(first.seed, e, P.p, shift),
                                            key_a_element(first.seed, e + 1, P.p, shift));
                }
            }
        }
        while (c < c1) {
            int next = c + 1;
            while (next < c1 && !(pi >= d.L || pi < d.ct[next].ell)) ++next;
            if (next < c1) fetch(next, nx);
            const CtDesc &ct = d.ct[c];
            const int ell = ct.ell, t = pi < d.L ? pi : ell + (pi - d.L);
            const CtLayout lo = ct_layout(d, ct);
            u64 ul0 = 0, uh0 = 0, ul1 = 0, uh1 = 0, vl0 = 0, vh0 = 0, vl1 = 0, vh1 = 0;
#pragma unroll
            for (int j = 0; j < KB; j++) {
                if (j < lo.beta) {
                    mac128(ul0, uh0, dv[j].x, ka[j].x);
                    mac128(ul1, uh1, dv[j].y, ka[j].y);
                    mac128(vl0, vh0, dv[j].x, kb[j].x);
                    mac128(vl1, vh1, dv[j].y, kb[j].y);
                }
            }
            if (ct.merged && t < ell) {
                // NewMult: PModUp(b3), PModUp(c3) join the sums before the one reduction
                const u64 pm = Pmod[pi].x;
                const ulonglong2 b = ld2(ct.add[0] + size_t(t) * N + n0), cc = ld2(ct.add[1] + size_t(t) * N + n0);
                mac128(ul0, uh0, b.x, pm);
                mac128(ul1, uh1, b.y, pm);
                mac128(vl0, vh0, cc.x, pm);
                mac128(vl1, vh1, cc.y, pm);
            }
            st2(lo.uv + size_t(t) * N + n0, make_ulonglong2(reduce128(ul0, uh0, P), reduce128(ul1, uh1, P)));
            st2(lo.uv + (size_t(lo.ext) + t) * N + n0,
                make_ulonglong2(reduce128(vl0, vh0, P), reduce128(vl1, vh1, P)));
#pragma unroll
            for (int j = 0; j < KB; j++) dv[j] = nx[j];
            c = next;
        }
    } else {
        // dnum > 4: key rows re-read per entry (from L2 after the first), digits looped
        const int shift = __clzll(P.p);
        for (int c = c0; c < c1; ++c) {
            const CtDesc &ct = d.ct[c];
            const int ell = ct.ell;
            if (pi < d.L && pi >= ell) continue;
            const int t = pi < d.L ? pi : ell + (pi - d.L);
            const CtLayout lo = ct_layout(d, ct);
            u64 ul0 = 0, uh0 = 0, ul1 = 0, uh1 = 0, vl0 = 0, vh0 = 0, vl1 = 0, vh1 = 0;
            for (int j = 0; j < lo.beta; j++) {
                const bool own = t < ell && (t / alpha) == j;
                const u64 *src = own ? ct.a + size_t(t) * N : lo.extp + (size_t(j) * lo.ext + t) * N;
                const ulonglong2 dv = ld2_perm(src, n0, ct.galois, logN);
                ulonglong2 a2, b2;
                if (comp) {
                    const u64 e = (u64(j) * LK + pi) * N + n0;
                    a2 = make_ulonglong2(key_a_element(first.seed, e, P.p, shift),
                                         key_a_element(first.seed, e + 1, P.p, shift));
                    b2 = ld2(key + (size_t(j) * LK + pi) * N + n0);
                } else {
                    a2 = ld2(key + ((size_t(j) * 2 + 0) * LK + pi) * N + n0);
                    b2 = ld2(key + ((size_t(j) * 2 + 1) * LK + pi) * N + n0);
                }
                mac128(ul0, uh0, dv.x, a2.x);
                mac128(ul1, uh1, dv.y, a2.y);
                mac128(vl0, vh0, dv.x, b2.x);
                mac128(vl1, vh1, dv.y, b2.y);
            }
            if (ct.merged && t < ell) {
                const u64 pm = Pmod[pi].x;
                const ulonglong2 b = ld2(ct.add[0] + size_t(t) * N + n0), cc = ld2(ct.add[1] + size_t(t) * N + n0);
                mac128(ul0, uh0, b.x, pm);
                mac128(ul1, uh1, b.y, pm);
                mac128(vl0, vh0, cc.x, pm);
                mac128(vl1, vh1, cc.y, pm);
            }
            st2(lo.uv + size_t(t) * N + n0, make_ulonglong2(reduce128(ul0, uh0, P), reduce128(ul1, uh1, P)));
            st2(lo.uv + (size_t(lo.ext) + t) * N + n0,
                make_ulonglong2(reduce128(vl0, vh0, P), reduce128(vl1, vh1, P)));
        }
    }
}

cudaError_t launch_inner_prod_batch(const ckks_ctx *ctx, const KsBatchDesc &d, cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    int units = 0;
    for (int c = 0; c < d.n; ++c) units += d.ct[c].ell + d.k;
    const int threads = 256;
    const unsigned tiles = unsigned((ctx->N / 2 + threads - 1) / threads);
    ProfScope ps(ctx, K_INNER, units, st);
    bool comp = false;
    for (int c = 0; c < d.n; ++c) comp = comp || d.ct[c].compressed;
    if (!comp) {
        dim3 grid(unsigned(d.n), tiles, unsigned(ctx->L + ctx->k));
#define CKKS_IPB(B) inner_prod_batch_kernel<B><<<grid, threads, 0, st>>>(d, ctx->d_pinfo, ctx->d_Pmod)
        switch (ctx->dnum) {
        case 1: CKKS_IPB(1); break;
        case 2: CKKS_IPB(2); break;
        case 3: CKKS_IPB(3); break;
        case 4: CKKS_IPB(4); break;
        default: CKKS_IPB(0);
        }
#undef CKKS_IPB
        return cudaGetLastError();
    }
    // groups of consecutive entries with one key (rows, compression, seed), as
    // large as the launch allows while it keeps at least 8 CTAs per SM (fewer
    // key generations, enough CTAs to fill the GPU at small N); with more than
    // 4 digits the rows are not held in registers, so groups of one
    const int cap = policy::ip_group_cap(long(tiles) * (ctx->L + ctx->k), d.n, ctx->sms, ctx->dnum, kIpGroup);
    IpGroups G{};
    G.n = policy::ip_groups(d.n, cap, [&](int a, int c) {
        const CtDesc &x = d.ct[a], &y = d.ct[c];
        return y.key == x.key && y.compressed == x.compressed && (!x.compressed || y.seed == x.seed);
    }, G.start);
    dim3 grid(unsigned(G.n), tiles, unsigned(ctx->L + ctx->k));
#define CKKS_IPG(B) inner_prod_group_kernel<B><<<grid, threads, 0, st>>>(d, G, ctx->d_pinfo, ctx->d_Pmod)
    switch (ctx->dnum) {
    case 1: CKKS_IPG(1); break;
    case 2: CKKS_IPG(2); break;
    case 3: CKKS_IPG(3); break;
    case 4: CKKS_IPG(4); break;
    default: CKKS_IPG(0);
    }
#undef CKKS_IPG
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Mult tensor step
// (a3, b3, c3) = (a1 a2, a1 b2 + a2 b1, b1 b2) slot-wise (Algorithm 2), for
// every Mult entry of a batch.  Grid (entry, coefficient tile, limb).
__global__ void __launch_bounds__(256) tensor_kernel(const __grid_constant__ TensorBatch T,
                                                     const PrimeInfo *__restrict__ pinfo) {
    const TensorEntry &e = T.e[blockIdx.x];
    const int i = blockIdx.z;
    if (i >= e.ell) return;
    const size_t N = size_t(1) << T.logN;
    const uint32_t n0 = (blockIdx.y * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const size_t o = size_t(i) * N + n0;
    const ulonglong2 a1 = ld2(e.a1 + o), b1 = ld2(e.b1 + o), a2 = ld2(e.a2 + o), b2 = ld2(e.b2 + o);
    const PrimeInfo P = pinfo[i];
    st2(e.a3 + o, make_ulonglong2(mul_mod(a1.x, a2.x, P), mul_mod(a1.y, a2.y, P)));
    u64 l0 = 0, h0 = 0, l1 = 0, h1 = 0;
    mac128(l0, h0, a1.x, b2.x);
    mac128(l0, h0, a2.x, b1.x);
    mac128(l1, h1, a1.y, b2.y);
    mac128(l1, h1, a2.y, b1.y);
    st2(e.b3 + o, make_ulonglong2(reduce128(l0, h0, P), reduce128(l1, h1, P)));
    st2(e.c3 + o, make_ulonglong2(mul_mod(b1.x, b2.x, P), mul_mod(b1.y, b2.y, P)));
}

cudaError_t launch_tensor(const ckks_ctx *ctx, const TensorBatch &T, cudaStream_t st) {
    if (T.n == 0) return cudaSuccess;
    int maxell = 0, units = 0;
    for (int c = 0; c < T.n; ++c) {
        maxell = std::max(maxell, T.e[c].ell);
        units += T.e[c].ell;
    }
    const int threads = 256;
    dim3 grid(unsigned(T.n), unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(maxell));
    ProfScope ps(ctx, K_ELEMWISE, units, st);
    tensor_kernel<<<grid, threads, 0, st>>>(T, ctx->d_pinfo);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ hoisted inner product
// The lifted (u, v) of every entry of a batch summed into entry 0's, slot-wise
// mod each prime of the extended basis (all entries at one level).  Grid
// (coefficient tile, position of the 2(ell+k) limbs of u and v).
__global__ void __launch_bounds__(256) sum_uv_kernel(const __grid_constant__ KsBatchDesc d,
                                                     const PrimeInfo *__restrict__ pinfo) {
    const size_t N = size_t(1) << d.logN;
    const size_t n0 = (size_t(blockIdx.x) * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int ell = d.ct[0].ell, ext = ell + d.k;
    const int y = blockIdx.y;  // poly * ext + t
    const int t = y % ext;
    const PrimeInfo P = pinfo[t < ell ? t : d.L + (t - ell)];
    u64 s0 = 0, s1 = 0;  // n < 2^9 values below 2^55 each: no overflow
    for (int c = 0; c < d.n; ++c) {
        const CtLayout lo = ct_layout(d, d.ct[c]);
        const ulonglong2 v = ld2(lo.uv + size_t(y) * N + n0);
        s0 += v.x;
        s1 += v.y;
    }
    const CtLayout l0 = ct_layout(d, d.ct[0]);
    st2(l0.uv + size_t(y) * N + n0, make_ulonglong2(reduce128(s0, 0, P), reduce128(s1, 0, P)));
}

cudaError_t launch_sum_uv(const ckks_ctx *ctx, const KsBatchDesc &d, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(2 * (d.ct[0].ell + ctx->k)));
    ProfScope ps(ctx, K_ELEMWISE, 2.0 * (d.ct[0].ell + ctx->k) * d.n, st);
    sum_uv_kernel<<<grid, threads, 0, st>>>(d, ctx->d_pinfo);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ compressed keys
// a[(j*(L+k) + l)*N + n] for digits j0 .. j0+gridDim.z-1, written at
// dst + ((j - j0)*(L+k) + l)*N + n: the key half regenerated from the seed.
__global__ void __launch_bounds__(256) key_a_fill_kernel(u64 seed, int j0, u64 *__restrict__ dst,
                                                         const PrimeInfo *__restrict__ pinfo, int logN, int LK) {
    const size_t N = size_t(1) << logN;
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y, j = j0 + int(blockIdx.z);
    const u64 q = pinfo[l].p;
    dst[(size_t(blockIdx.z) * LK + l) * N + n] = key_a_element(seed, (u64(j) * LK + l) * N + n, q, __clzll(q));
}

cudaError_t launch_key_a_fill(const ckks_ctx *ctx, u64 seed, int j0, int ndig, u64 *dst, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N + threads - 1) / threads), unsigned(ctx->L + ctx->k), unsigned(ndig));
    ProfScope ps(ctx, K_ELEMWISE, double(ctx->L + ctx->k) * ndig, st);
    key_a_fill_kernel<<<grid, threads, 0, st>>>(seed, j0, dst, ctx->d_pinfo, ctx->logN, ctx->L + ctx->k);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ PtMatVecMult inner loop
// One giant step of Algorithm 8: for every extended position t and slot n,
//   acc_a = sum_i M_i * u_i,   acc_b = sum_i M_i * (v_i + [P*b_rot,i]),
// where (u_i, v_i) is the inner product of the hoisted digits automorphed by
// g_i with key_i, and baby step i = 0 (no key) contributes M_0 * (P*a, P*b).
// u_i and v_i never leave registers (the beta-limb caching of Sec. 4.2).
template <bool COMP>
__global__ void __launch_bounds__(256) pmv_accum_kernel(PmvArgs A, const PrimeInfo *__restrict__ pinfo,
                                                        const ulonglong2 *__restrict__ Pmod, int logN, int L, int k,
                                                        int alpha) {
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int t = blockIdx.y;
    const int ell = A.ell, ext = ell + k, LK = L + k;
    const int beta = (ell + alpha - 1) / alpha;
    const int prime = t < ell ? t : L + (t - ell);
    const PrimeInfo P = pinfo[prime];
    const ulonglong2 pm = Pmod[prime];
    u64 al0 = 0, ah0 = 0, al1 = 0, ah1 = 0, bl0 = 0, bh0 = 0, bl1 = 0, bh1 = 0;
    for (int i = 0; i < A.nb; i++) {
        const ulonglong2 M = ld2(A.diag[i] + size_t(t) * N + n0);
        u64 u0, u1, w0, w1;
        if (A.key[i] == nullptr) {
            if (t < ell) {
                const ulonglong2 av = ld2(A.a + size_t(t) * N + n0);
                const ulonglong2 bv = ld2(A.b + size_t(t) * N + n0);
                u0 = shoup_mul(av.x, pm.x, pm.y, P.p);
                u1 = shoup_mul(av.y, pm.x, pm.y, P.p);
                w0 = shoup_mul(bv.x, pm.x, pm.y, P.p);
                w1 = shoup_mul(bv.y, pm.x, pm.y, P.p);
            } else {
                u0 = u1 = w0 = w1 = 0;
            }
        } else {
            const uint32_t g = A.galois[i];
            const u64 *key = A.key[i];
            u64 ul0 = 0, uh0 = 0, ul1 = 0, uh1 = 0, vl0 = 0, vh0 = 0, vl1 = 0, vh1 = 0;
            for (int j = 0; j < beta; j++) {
                const bool own = t < ell && (t / alpha) == j;
                const u64 *d = own ? A.a + size_t(t) * N : A.ext + (size_t(j) * ext + t) * N;
                const ulonglong2 dv = ld2_perm(d, n0, g, logN);
                ulonglong2 ka, kb;
                if (COMP && A.compressed[i]) {
                    const u64 e = (u64(j) * LK + prime) * N + n0;
                    const int shift = __clzll(P.p);
                    kb = ld2_stream(key + (size_t(j) * LK + prime) * N + n0);
                    ka = make_ulonglong2(key_a_element(A.seed[i], e, P.p, shift),
                                         key_a_element(A.seed[i], e + 1, P.p, shift));
                } else {
                    ka = ld2_stream(key + ((size_t(j) * 2 + 0) * LK + prime) * N + n0);
                    kb = ld2_stream(key + ((size_t(j) * 2 + 1) * LK + prime) * N + n0);
                }
                mac128(ul0, uh0, dv.x, ka.x);
                mac128(ul1, uh1, dv.y, ka.y);
                mac128(vl0, vh0, dv.x, kb.x);
                mac128(vl1, vh1, dv.y, kb.y);
            }
            u0 = reduce128(ul0, uh0, P);
            u1 = reduce128(ul1, uh1, P);
            w0 = reduce128(vl0, vh0, P);
            w1 = reduce128(vl1, vh1, P);
            if (t < ell) {
                const ulonglong2 bv = ld2_perm(A.b + size_t(t) * N, n0, g, logN);
                w0 = add_mod(w0, shoup_mul(bv.x, pm.x, pm.y, P.p), P.p);
                w1 = add_mod(w1, shoup_mul(bv.y, pm.x, pm.y, P.p), P.p);
            }
        }
        mac128(al0, ah0, M.x, u0);
        mac128(al1, ah1, M.y, u1);
        mac128(bl0, bh0, M.x, w0);
        mac128(bl1, bh1, M.y, w1);
    }
    st2(A.acc_a + size_t(t) * N + n0, make_ulonglong2(reduce128(al0, ah0, P), reduce128(al1, ah1, P)));
    st2(A.acc_b + size_t(t) * N + n0, make_ulonglong2(reduce128(bl0, bh0, P), reduce128(bl1, bh1, P)));
}

cudaError_t launch_pmv_accum(const ckks_ctx *ctx, const PmvArgs &a, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(a.ell + ctx->k));
    ProfScope ps(ctx, K_PMV, double(a.ell + ctx->k) * a.nb, st);
    bool comp = false;
    for (int i = 0; i < a.nb; ++i) comp = comp || a.compressed[i];
    if (comp)
        pmv_accum_kernel<true><<<grid, threads, 0, st>>>(a, ctx->d_pinfo, ctx->d_Pmod, ctx->logN, ctx->L, ctx->k,
                                                          ctx->alpha);
    else
        pmv_accum_kernel<false><<<grid, threads, 0, st>>>(a, ctx->d_pinfo, ctx->d_Pmod, ctx->logN, ctx->L, ctx->k,
                                                           ctx->alpha);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ PtMatVecMult, every giant step at once
// The same sums as pmv_accum_kernel, for all giant steps t < NG in one pass:
// baby step i's (u_i, v_i + [P*b_rot,i]) is formed once per slot and added,
// times M_{t,i}, into every giant step's accumulator.  Each baby-step key is
// therefore read once per call instead of once per giant step (the key stream
// dominates the bytes of Algorithm 8 with BSGS, Sec. 5.2), and every diagonal
// once.  One slot per thread (8-byte loads, coalesced by the warp; the
// Automorph gather stays inside aligned 32-slot blocks): the NG x 2 128-bit
// accumulators live in registers.  Grid (slot tile, extended position).
template <int BETA, int NG, bool COMP>
__global__ void __launch_bounds__(256, 3) pmv_all_kernel(const __grid_constant__ PmvAllArgs A,
                                                      const PrimeInfo *__restrict__ pinfo,
                                                      const ulonglong2 *__restrict__ Pmod, int logN, int L, int k,
                                                      int alpha) {
    const size_t N = size_t(1) << logN;
    const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int t = blockIdx.y;
    const int ell = A.ell, ext = ell + k, LK = L + k;
    const int prime = t < ell ? t : L + (t - ell);
    const PrimeInfo P = pinfo[prime];
    const ulonglong2 pm = Pmod[prime];
    const size_t to = size_t(t) * N;
    u64 al[NG], ah[NG], bl[NG], bh[NG];
#pragma unroll
    for (int g = 0; g < NG; g++) al[g] = ah[g] = bl[g] = bh[g] = 0;
#pragma unroll 1
    for (int i = 0; i < A.nb; i++) {
        u64 M[NG];
#pragma unroll
        for (int g = 0; g < NG; g++) M[g] = g < A.ng ? __ldcs(A.diag[g * A.nb + i] + to + n) : 0;
        u64 u, w;
        if (A.key[i] == nullptr) {
            // baby step 0 (no rotation): (P*a, P*b) on the chain, 0 on the special primes
            u = w = 0;
            if (t < ell) {
                u = shoup_mul(A.a[to + n], pm.x, pm.y, P.p);
                w = shoup_mul(A.b[to + n], pm.x, pm.y, P.p);
            }
        } else {
            const uint32_t g = A.galois[i];
            const uint32_t src = g == 1 ? n : automorph_src(n, g, logN);
            const u64 *key = A.key[i];
            u64 dv[BETA], ka[BETA], kb[BETA];
#pragma unroll
            for (int j = 0; j < BETA; j++) {
                const bool own = t < ell && (t / alpha) == j;
                const u64 *d = own ? A.a + to : A.ext + (size_t(j) * ext + t) * N;
                dv[j] = d[src];
                if (COMP && A.compressed[i]) {
                    kb[j] = __ldcs(key + (size_t(j) * LK + prime) * N + n);
                } else {
                    ka[j] = __ldcs(key + ((size_t(j) * 2 + 0) * LK + prime) * N + n);
                    kb[j] = __ldcs(key + ((size_t(j) * 2 + 1) * LK + prime) * N + n);
                }
            }
            const u64 bsrc = t < ell ? A.b[to + src] : 0;
            if (COMP && A.compressed[i]) {
                const int shift = __clzll(P.p);
#pragma unroll
                for (int j = 0; j < BETA; j++)
                    ka[j] = key_a_element(A.seed[i], (u64(j) * LK + prime) * N + n, P.p, shift);
            }
            u64 ul = 0, uh = 0, vl = 0, vh = 0;
#pragma unroll
            for (int j = 0; j < BETA; j++) {
                mac128(ul, uh, dv[j], ka[j]);
                mac128(vl, vh, dv[j], kb[j]);
            }
            u = reduce128(ul, uh, P);
            w = reduce128(vl, vh, P);
            if (t < ell) w = add_mod(w, shoup_mul(bsrc, pm.x, pm.y, P.p), P.p);
        }
#pragma unroll
        for (int g = 0; g < NG; g++) {
            mac128(al[g], ah[g], M[g], u);
            mac128(bl[g], bh[g], M[g], w);
        }
    }
#pragma unroll
    for (int g = 0; g < NG; g++) {
        if (g < A.ng) {
            A.acc_a[g][to + n] = reduce128(al[g], ah[g], P);
            A.acc_b[g][to + n] = reduce128(bl[g], bh[g], P);
        }
    }
}

bool pmv_all_supported(const ckks_ctx *ctx, int ell, int nb, int ng) {
    return beta_of(ctx, ell) <= 4 && ng >= 1 && ng <= kMaxGiant && nb * ng <= kMaxRot;
}

cudaError_t launch_pmv_all(const ckks_ctx *ctx, const PmvAllArgs &a, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N + threads - 1) / threads), unsigned(a.ell + ctx->k));
    ProfScope ps(ctx, K_PMV, double(a.ell + ctx->k) * a.nb * a.ng, st);
    bool comp = false;
    for (int i = 0; i < a.nb; ++i) comp = comp || a.compressed[i];
    const int beta = beta_of(ctx, a.ell);
#define CKKS_PMV(B, G, C)                                                                                          \
    pmv_all_kernel<B, G, C><<<grid, threads, 0, st>>>(a, ctx->d_pinfo, ctx->d_Pmod, ctx->logN, ctx->L, ctx->k,    \
                                                      ctx->alpha)
#define CKKS_PMV_G(B, C)                                                                                           \
    switch (a.ng) {                                                                                                \
    case 1: CKKS_PMV(B, 1, C); break;                                                                              \
    case 2: CKKS_PMV(B, 2, C); break;                                                                              \
    case 3: CKKS_PMV(B, 3, C); break;                                                                              \
    case 4: CKKS_PMV(B, 4, C); break;                                                                              \
    default: CKKS_PMV(B, 8, C);                                                                                    \
    }
#define CKKS_PMV_B(C)                                                                                              \
    switch (beta) {                                                                                                \
    case 1: CKKS_PMV_G(1, C) break;                                                                                \
    case 2: CKKS_PMV_G(2, C) break;                                                                                \
    case 3: CKKS_PMV_G(3, C) break;                                                                                \
    default: CKKS_PMV_G(4, C) break;                                                                               \
    }
    if (comp) {
        CKKS_PMV_B(true)
    } else {
        CKKS_PMV_B(false)
    }
#undef CKKS_PMV_B
#undef CKKS_PMV_G
#undef CKKS_PMV
    return cudaGetLastError();
}

// ------------------------------------------------------------------ sum of polynomials
// acc[i] = (acc[i] + sum_j in_j[i]) mod q_i over the first ell primes, for two
// polynomials at once (the giant steps of PtMatVecMult computed apart).
__global__ void __launch_bounds__(256) poly_sum_kernel(const __grid_constant__ PolySum S,
                                                       const PrimeInfo *__restrict__ pinfo, int logN) {
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int i = blockIdx.y, poly = blockIdx.z;
    const u64 p = pinfo[i].p;
    const size_t o = size_t(i) * N + n0;
    ulonglong2 a = ld2(S.acc[poly] + o);
    for (int j = 0; j < S.n; j++) {
        const ulonglong2 x = ld2(S.in[poly][j] + o);
        a.x = add_mod(a.x, x.x, p);
        a.y = add_mod(a.y, x.y, p);
    }
    st2(S.acc[poly] + o, a);
}

cudaError_t launch_poly_sum(const ckks_ctx *ctx, const PolySum &S, int ell, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    const int threads = 256;
    dim3 grid(unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(ell), 2u);
    ProfScope ps(ctx, K_ELEMWISE, 2.0 * ell * (S.n + 1), st);
    poly_sum_kernel<<<grid, threads, 0, st>>>(S, ctx->d_pinfo, ctx->logN);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Automorph
__global__ void __launch_bounds__(256) automorph_kernel(const u64 *__restrict__ in, u64 *__restrict__ out, uint32_t g,
                                                        int logN) {
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const size_t base = size_t(blockIdx.y) * N;
    st2(out + base + n0, ld2_perm(in + base, n0, g, logN));
}

cudaError_t launch_automorph(const ckks_ctx *ctx, const u64 *in, u64 *out, int nlimbs, uint32_t g, cudaStream_t st) {
    if (nlimbs == 0) return cudaSuccess;
    const int threads = 256;
    dim3 grid(unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(nlimbs));
    ProfScope ps(ctx, K_ELEMWISE, nlimbs, st);
    automorph_kernel<<<grid, threads, 0, st>>>(in, out, g, ctx->logN);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ PModUp (Sec. 5.1)
__global__ void __launch_bounds__(256) pmodup_kernel(const u64 *__restrict__ in, u64 *__restrict__ out, int ell,
                                                     const PrimeInfo *__restrict__ pinfo,
                                                     const ulonglong2 *__restrict__ Pmod, int logN) {
    const size_t N = size_t(1) << logN;
    const uint32_t n0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (n0 >= N) return;
    const int t = blockIdx.y;
    ulonglong2 r = make_ulonglong2(0, 0);
    if (t < ell) {
        const u64 p = pinfo[t].p;
        const ulonglong2 c = Pmod[t];
        const ulonglong2 x = ld2(in + size_t(t) * N + n0);
        r.x = shoup_mul(x.x, c.x, c.y, p);
        r.y = shoup_mul(x.y, c.x, c.y, p);
    }
    st2(out + size_t(t) * N + n0, r);
}

cudaError_t launch_pmodup(const ckks_ctx *ctx, const u64 *in, u64 *out, int ell, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N / 2 + threads - 1) / threads), unsigned(ell + ctx->k));
    ProfScope ps(ctx, K_ELEMWISE, ell + ctx->k, st);
    pmodup_kernel<<<grid, threads, 0, st>>>(in, out, ell, ctx->d_pinfo, ctx->d_Pmod, ctx->logN);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ key generation
// Signed coefficients -> residues over all L+k primes (limb l uses prime l).
__global__ void signed_to_res_kernel(const int64_t *__restrict__ c, u64 *__restrict__ out,
                                     const PrimeInfo *__restrict__ pinfo, int logN) {
    const size_t N = size_t(1) << logN;
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y;
    const u64 p = pinfo[l].p;
    const int64_t x = c[n];
    u64 r;
    if (x >= 0) {
        r = u64(x) % p;
    } else {
        r = u64(-(x + 1)) % p;  // |x| - 1, safe for INT64_MIN
        r = p - 1 - r;
    }
    out[size_t(l) * N + n] = r;
}

cudaError_t launch_signed_to_res(const ckks_ctx *ctx, const int64_t *c, u64 *out, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N + threads - 1) / threads), unsigned(ctx->L + ctx->k));
    ProfScope ps(ctx, K_ELEMWISE, ctx->L + ctx->k, st);
    signed_to_res_kernel<<<grid, threads, 0, st>>>(c, out, ctx->d_pinfo, ctx->logN);
    return cudaGetLastError();
}

__global__ void square_kernel(const u64 *__restrict__ in, u64 *__restrict__ out, const PrimeInfo *__restrict__ pinfo,
                              int logN) {
    const size_t N = size_t(1) << logN;
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y;
    const PrimeInfo P = pinfo[l];
    const u64 x = in[size_t(l) * N + n];
    out[size_t(l) * N + n] = mul_mod(x, x, P);
}

cudaError_t launch_square(const ckks_ctx *ctx, const u64 *in, u64 *out, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N + threads - 1) / threads), unsigned(ctx->L + ctx->k));
    ProfScope ps(ctx, K_ELEMWISE, ctx->L + ctx->k, st);
    square_kernel<<<grid, threads, 0, st>>>(in, out, ctx->d_pinfo, ctx->logN);
    return cudaGetLastError();
}

// b_j = e_j - a_j * s + g_j * s', g_j = [P]_{q_i} on digit j's chain limbs (Eq. kskShape)
__global__ void keygen_row_kernel(const u64 *__restrict__ a, const u64 *__restrict__ s, const u64 *__restrict__ sp,
                                  const u64 *__restrict__ e, int j, u64 *__restrict__ row0, u64 *__restrict__ row1,
                                  const PrimeInfo *__restrict__ pinfo, const ulonglong2 *__restrict__ Pmod, int logN,
                                  int L, int alpha) {
    const size_t N = size_t(1) << logN;
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int l = blockIdx.y;
    const PrimeInfo P = pinfo[l];
    const size_t o = size_t(l) * N + n;
    const u64 av = a[o];
    u64 b = sub_mod(e[o], mul_mod(av, s[o], P), P.p);
    if (l < L && l / alpha == j) {
        const ulonglong2 c = Pmod[l];
        b = add_mod(b, shoup_mul(sp[o], c.x, c.y, P.p), P.p);
    }
    if (row0 != nullptr) row0[o] = av;  // null: compressed key, only b is kept
    row1[o] = b;
}

cudaError_t launch_keygen_row(const ckks_ctx *ctx, const u64 *a, const u64 *s, const u64 *sp, const u64 *e, int j,
                              u64 *row0, u64 *row1, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(unsigned((ctx->N + threads - 1) / threads), unsigned(ctx->L + ctx->k));
    ProfScope ps(ctx, K_ELEMWISE, ctx->L + ctx->k, st);
    keygen_row_kernel<<<grid, threads, 0, st>>>(a, s, sp, e, j, row0, row1, ctx->d_pinfo, ctx->d_Pmod, ctx->logN,
                                                ctx->L, ctx->alpha);
    return cudaGetLastError();
}

}  // namespace ckks
