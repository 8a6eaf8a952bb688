// batch.cuh -- where each limb (NTT launches), group (basis conversions) and
// position (inner products) of a launch reads and writes.
//
// Single operations describe their limbs with explicit pointer lists in the
// launch parameters (MapList).  Batched key switching (many ciphertexts at
// their own levels, each with its own key and Galois element, in one launch
// per phase) describes only the ciphertexts (KsBatchDesc) and every kernel
// derives its limb's pointers on the device from a prefix sum over the
// per-ciphertext counts of its phase.
#pragma once

#include "common.cuh"

namespace ckks {

// One limb of an NTT launch.  The epilogue operands are used by launches with
// the ModDown/Rescale epilogue: out = (x - ntt) * cmul[prime] [+ add at the
// Automorph_galois slot] [+ out].
struct LimbIO {
    const u64 *src;
    u64 *dst;
    int prime;
    const u64 *ex;
    u64 *eout;
    const u64 *eadd;
    const ulonglong2 *cmul;  // scale table (indexed by prime) of the epilogue
    uint32_t galois;
    int accumulate;
    int lazy;  // store the forward transform without its final reduction (EPI_LAZY)
};

// Explicit limb list (single operations).
struct MapList {
    NttBatch b;
    Epi e;
    int second;  // second pass of a transform: read the first pass's output in place
    __device__ __forceinline__ LimbIO get(int l, uint32_t N) const {
        LimbIO io;
        io.src = second ? b.dst[l] : b.src[l];
        io.dst = b.dst[l];
        io.prime = b.prime[l];
        io.ex = nullptr;
        io.eout = nullptr;
        io.eadd = nullptr;
        io.cmul = e.cmul;
        io.galois = 1;
        io.accumulate = 0;
        io.lazy = e.mode == EPI_LAZY;
        if (e.mode == EPI_SCALE) {
            const int poly = l % e.npolys;
            const size_t base = size_t(l / e.npolys) * N;
            io.ex = e.x[poly] + base;
            io.eout = e.out[poly] + base;
            io.eadd = e.add[poly] == nullptr ? nullptr : e.add[poly] + base;
            io.galois = e.galois;
            io.accumulate = e.accumulate;
        }
        return io;
    }
};

// ---------------------------------------------------------------- batched key switching
constexpr int kMaxCts = 64;

// One entry of a batch: a key switch of a (evaluation form, [ell][N]) whose
// ModDown epilogue adds add[p] read through Automorph_galois to output p:
//   KeySwitch:                 add = {0, 0}, galois = 1, outputs (u, v);
//   HRotate, one rotation:     add = {0, b}, digits read through galois
//                              (Algorithm 4): (u, v + Automorph_g(b));
//   Mult (Algorithm 2):        a = a1*a2, add = {a1 b2 + a2 b1, b1 b2},
//                              galois = 1, then ra/rb = Rescale(oa/ob);
//   NewMult (Algorithm 7):     merged = 1: the inner product adds
//                              PModUp(add[p]) on the chain positions and one
//                              ModDown by D = P*q_{ell-1} (sources: the k
//                              P-limbs and q_{ell-1}) writes oa/ob [ell-1][N].
// ws: this entry's workspace, laid out for its level:
//   ext [beta][ell+k][N] | uv [2][ell+k][N] | tmp (acoeff [ell][N], later
//   pcoeff [2][k(+1)][N] and w [2][ell(-1)][N]).  After the key switch the
//   Rescale of a Mult entry reuses ext: c [2][N] | w [2][ell-1][N].
struct CtDesc {
    const u64 *a, *key;
    const u64 *add[2];
    u64 *oa, *ob, *ws;
    u64 *ra, *rb;  // Rescale outputs [ell-1][N] (Mult entries), else null
    int ell;
    uint32_t galois;
    int merged;      // NewMult entry
    int compressed;  // key holds only the b rows [dnum][L+k][N]; a is regenerated from seed
    u64 seed;
    u64 *ext_shared; // hoisted rotations: the ModUp digits of another entry of the same
                     // ciphertext; ws then holds only uv | tmp
};

struct KsBatchDesc {
    int n;
    int L, k, alpha, dnum, logN;
    CtDesc ct[kMaxCts];
    int pre[kMaxCts + 1];  // prefix sums of this launch's per-ciphertext counts
};

struct CtLayout {
    int beta, ext;
    u64 *extp, *uv, *acoeff, *pcoeff, *w;
};

__host__ __device__ __forceinline__ CtLayout ct_layout(const KsBatchDesc &d, const CtDesc &c) {
    CtLayout o;
    const size_t N = size_t(1) << d.logN;
    o.beta = (c.ell + d.alpha - 1) / d.alpha;
    o.ext = c.ell + d.k;
    o.extp = c.ext_shared != nullptr ? c.ext_shared : c.ws;
    o.uv = c.ext_shared != nullptr ? c.ws : c.ws + size_t(o.beta) * o.ext * N;
    o.acoeff = o.uv + size_t(2) * o.ext * N;
    o.pcoeff = o.acoeff;
    o.w = o.pcoeff + size_t(2) * (d.k + c.merged) * N;
    return o;
}

// index l of a phase -> (ciphertext, index within it)
__device__ __forceinline__ int batch_find(const KsBatchDesc &d, int l, int &i) {
    int lo = 0, hi = d.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d.pre[mid] <= l) lo = mid;
        else hi = mid - 1;
    }
    i = l - d.pre[lo];
    return lo;
}

// Per-entry limb counts of the batched phases (Rescale phases: Mult entries only).
enum { PH_INTT_A = 0, PH_NTT_UP = 1, PH_INTT_P = 2, PH_NTT_DOWN = 3, PH_RS_INTT = 4, PH_RS_NTT = 5 };
__host__ __device__ __forceinline__ int phase_count(const KsBatchDesc &d, const CtDesc &c, int phase) {
    const int ell = c.ell;
    const int beta = (ell + d.alpha - 1) / d.alpha;
    switch (phase) {
    case PH_INTT_A: return ell;
    case PH_NTT_UP: return beta * (ell + d.k) - ell;
    case PH_INTT_P: return 2 * (d.k + c.merged);
    case PH_NTT_DOWN: return 2 * (ell - c.merged);
    case PH_RS_INTT: return c.ra != nullptr ? 2 : 0;
    default: return c.ra != nullptr ? 2 * (ell - 1) : 0;
    }
}

struct MapBatch {
    KsBatchDesc d;
    int phase;
    int second;               // second pass: in place on the first pass's output
    const ulonglong2 *cm;     // [P^-1]_q per prime (ModDown epilogue)
    const ulonglong2 *qlinv;  // [q_{ell-1}^-1]_{q_i} at ell*(L+k) + i (Rescale epilogue)
    const ulonglong2 *dinv;   // [(P q_{ell-1})^-1]_{q_i} at ell*(L+k) + i (merged ModDown epilogue)
    __device__ __forceinline__ LimbIO get(int l, uint32_t N) const {
        int i;
        const int c = batch_find(d, l, i);
        const CtDesc &ct = d.ct[c];
        const CtLayout lo = ct_layout(d, ct);
        const int ell = ct.ell;
        LimbIO io;
        io.ex = nullptr;
        io.eout = nullptr;
        io.eadd = nullptr;
        io.cmul = cm;
        io.galois = 1;
        io.accumulate = 0;
        io.lazy = phase == PH_NTT_UP;  // the ModUp digits go to the inner product only
        if (phase == PH_INTT_A) {
            io.src = ct.a + size_t(i) * N;
            io.dst = lo.acoeff + size_t(i) * N;
            io.prime = i;
        } else if (phase == PH_NTT_UP) {
            // new ModUp limbs in position-major order: a chain position t < ell
            // appears for the beta-1 digits that do not hold it, a special
            // position for every digit
            int t, j;
            const int bm1 = lo.beta - 1;
            if (i < ell * bm1) {
                t = i / bm1;
                const int r = i % bm1;
                j = r < t / d.alpha ? r : r + 1;
            } else {
                const int i2 = i - ell * bm1;
                t = ell + i2 / lo.beta;
                j = i2 % lo.beta;
            }
            u64 *p = lo.extp + (size_t(j) * lo.ext + t) * N;
            io.src = p;
            io.dst = p;
            io.prime = t < ell ? t : d.L + (t - ell);
        } else if (phase == PH_INTT_P) {
            // the k P-limbs (and for NewMult q_{ell-1} as source k) of both polynomials
            const int m = i >> 1, poly = i & 1;
            const int pos = m < d.k ? ell + m : ell - 1;
            io.src = lo.uv + (size_t(poly) * lo.ext + pos) * N;
            io.dst = lo.pcoeff + (size_t(poly) * (d.k + ct.merged) + m) * N;
            io.prime = m < d.k ? d.L + m : ell - 1;
        } else if (phase == PH_NTT_DOWN) {
            const int t = i >> 1, poly = i & 1;
            const int nout = ell - ct.merged;
            u64 *p = lo.w + (size_t(poly) * nout + t) * N;
            io.src = p;
            io.dst = p;
            io.prime = t;
            io.ex = lo.uv + (size_t(poly) * lo.ext + t) * N;
            io.eout = (poly ? ct.ob : ct.oa) + size_t(t) * N;
            io.eadd = (!ct.merged && ct.add[poly] != nullptr) ? ct.add[poly] + size_t(t) * N : nullptr;
            io.galois = ct.galois;
            if (ct.merged) io.cmul = dinv + size_t(ell) * (d.L + d.k);
        } else if (phase == PH_RS_INTT) {
            // last limb of the key switch's output p -> c[p]
            io.src = (i ? ct.ob : ct.oa) + size_t(ell - 1) * N;
            io.dst = ct.ws + size_t(i) * N;
            io.prime = ell - 1;
        } else {
            const int t = i >> 1, poly = i & 1;
            u64 *p = ct.ws + (size_t(2) + size_t(poly) * (ell - 1) + t) * N;
            io.src = p;
            io.dst = p;
            io.prime = t;
            io.ex = (poly ? ct.ob : ct.oa) + size_t(t) * N;
            io.eout = (poly ? ct.rb : ct.ra) + size_t(t) * N;
            io.cmul = qlinv + size_t(ell) * (d.L + d.k);
        }
        if (second) io.src = io.dst;
        return io;
    }
};

// Tensor step of the Mult entries of a batch.
struct TensorEntry {
    const u64 *a1, *b1, *a2, *b2;
    u64 *a3, *b3, *c3;
    int ell;
};
struct TensorBatch {
    int n, logN;
    TensorEntry e[kMaxCts];
};

// Basis-conversion groups.
struct GroupMapList {
    BConvLaunch l;
    __device__ __forceinline__ BConvGroup get(int gi) const { return l.g[gi]; }
};

enum { GM_MODUP = 0, GM_MODDOWN = 1, GM_RESCALE = 2 };
struct GroupMapBatch {
    KsBatchDesc d;
    int down;                   // GM_MODUP: digits; GM_MODDOWN / GM_RESCALE: 2 polynomials
    const BConvPlan *modup;     // [(L+1)*dnum]
    const BConvPlan *moddown;   // [L+1]
    const BConvPlan *rescale;   // [L+1]
    const BConvPlan *merged;    // [L+1]: D = P*q_{ell-1} -> q_0..q_{ell-2}
    __device__ __forceinline__ BConvGroup get(int gi) const {
        int i;
        const int c = batch_find(d, gi, i);
        const CtDesc &ct = d.ct[c];
        const CtLayout lo = ct_layout(d, ct);
        const size_t N = size_t(1) << d.logN;
        BConvGroup g;
        if (down == GM_MODUP) {
            g.plan = modup + size_t(ct.ell) * d.dnum + i;
            g.src = lo.acoeff + size_t(i) * d.alpha * N;
            g.dst = lo.extp + size_t(i) * lo.ext * N;
        } else if (down == GM_MODDOWN) {
            g.plan = (ct.merged ? merged : moddown) + ct.ell;
            g.src = lo.pcoeff + size_t(i) * (d.k + ct.merged) * N;
            g.dst = lo.w + size_t(i) * (ct.ell - ct.merged) * N;
        } else {
            g.plan = rescale + ct.ell;
            g.src = ct.ws + size_t(i) * N;
            g.dst = ct.ws + (size_t(2) + size_t(i) * (ct.ell - 1)) * N;
        }
        return g;
    }
};

}  // namespace ckks
