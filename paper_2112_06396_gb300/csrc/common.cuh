// common.cuh -- shared device/host definitions of the CKKS key-switching
// library: per-prime constants, modular arithmetic, launch descriptors.
//
// Modular arithmetic (Sec. 2.2, "Scalar Modular Arithmetic"):
//  * Shoup constant multiplication [Shoup, NTL]: for a constant w < p with
//    w' = floor(w * 2^64 / p), x*w - umulhi(x, w')*p lies in [0, 2p) for every
//    64-bit x.  Used for every twiddle and every precomputed constant.
//  * Lazy reduction: NTT values travel in [0, 4p) (Harvey, "Faster arithmetic
//    for number-theoretic transforms", J. Symb. Comp. 2014), which needs
//    4p < 2^64; this library requires p < 2^60.
//  * Sums of products are accumulated exactly in 128 bits and reduced once at
//    the end (the paper's "reduce once at the end of a sum").
//  * The 128-bit reduction writes hi*2^64 + lo = hi*[2^64]_p + lo and reduces
//    both words with Shoup multiplications (by [2^64]_p and by 1).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

typedef uint64_t u64;

namespace ckks {

constexpr int kMaxLimbs = 96;      // L + k
constexpr int kMaxSrc = 32;        // limbs per basis-conversion source (alpha, k)
constexpr int kMaxDst = 96;        // limbs per basis-conversion target set
constexpr int kMaxBatch = 128;     // limbs per NTT launch
constexpr int kMaxRot = 64;        // rotations per fused inner-product launch

// Constants of one prime modulus.
struct PrimeInfo {
    u64 p;
    u64 r64, r64_s;        // [2^64]_p and its Shoup companion
    u64 one_s;             // floor(2^64 / p): Shoup companion of 1
    u64 ninv, ninv_s;      // [N^-1]_p
    u64 ninv_w, ninv_w_s;  // [N^-1 * psi^-brv(1)]_p (last inverse stage)
};

// ------------------------------------------------------------------ device
__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 ws, u64 p) {
    u64 q = __umul64hi(x, ws);
    return x * w - q * p;
}
__device__ __forceinline__ u64 csub(u64 x, u64 m) { return x >= m ? x - m : x; }

// Shoup multiplication with an approximate quotient.  With x = x1*2^32 + x0,
// w' = s1*2^32 + s0, T = x1*s0 and U = x0*s1 + lo(T) (< 2^64, no overflow):
//   x*w' = (x1*s1 + hi(T) + hi(U)) * 2^64 + lo(U)*2^32 + x0*s0,
// and the last two terms sum to less than 2^65, so q_hat = x1*s1 + hi(T) +
// hi(U) is in [q - 1, q] for q = floor(x*w'/2^64), and x*w - q_hat*p lies in
// [0, 3p) (within [0, 4p)) for every 64-bit x.  np = 2^64 - p; the low words
// of x*w and q_hat*np are accumulated on 32-bit halves.  Only full-rate
// 32-bit multiply-adds (no high-half multiply) and two adds, against a full
// 64x64 high product plus two 64-bit low products.
__device__ __forceinline__ u64 shoup_approx(u64 x, u64 w, u64 ws, u64 np) {
    u64 r;
    asm("{\n\t"
        ".reg .u32 x0, x1, w0, w1, s0, s1, n0, n1, h1, h2, q0, q1, r0, r1, m1, m2;\n\t"
        ".reg .u64 q, acc, t;\n\t"
        "mov.b64 {x0, x1}, %1;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {s0, s1}, %3;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        // T = x1*s0; U = x0*s1 + lo(T) (middle word, exact carry);
        // q_hat = x1*s1 + hi(T) + hi(U): three wide multiply-adds and one add
        // (mul.hi.u32 issues at half the rate of mad.wide.u32)
        "mul.wide.u32 t, x1, s0;\n\t"
        "mov.b64 {h1, h2}, t;\n\t"
        "cvt.u64.u32 acc, h1;\n\t"
        "mad.wide.u32 acc, x0, s1, acc;\n\t"
        "cvt.u64.u32 t, h2;\n\t"
        "mad.wide.u32 q, x1, s1, t;\n\t"
        "mov.b64 {h1, h2}, acc;\n\t"
        "cvt.u64.u32 t, h2;\n\t"
        "add.u64 q, q, t;\n\t"
        // low word of x*w, independent of the quotient
        "mul.wide.u32 acc, x0, w0;\n\t"
        "mul.lo.u32 m1, x0, w1;\n\t"
        "mad.lo.u32 m1, x1, w0, m1;\n\t"
        "mov.b64 {q0, q1}, q;\n\t"
        // + q * (2^64 - p), low word
        "mad.wide.u32 acc, q0, n0, acc;\n\t"
        "mad.lo.u32 m2, q0, n1, m1;\n\t"
        "mad.lo.u32 m2, q1, n0, m2;\n\t"
        "mov.b64 {r0, r1}, acc;\n\t"
        "add.u32 r1, r1, m2;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "l"(x), "l"(w), "l"(ws), "l"(np));
    return r;
}
__device__ __forceinline__ u64 shoup_mul(u64 x, u64 w, u64 ws, u64 p) { return csub(shoup_lazy(x, w, ws, p), p); }
// shoup_approx with w = 1 (a reduction of any 64-bit x to [0, 3p) with
// ones = floor(2^64 / p)): the same quotient, and x - q_hat*p = x + q_hat*np
// needs one wide multiply-add with x as the addend and two low products.
__device__ __forceinline__ u64 shoup_one(u64 x, u64 ones, u64 np) {
    u64 r;
    asm("{\n\t"
        ".reg .u32 x0, x1, s0, s1, n0, n1, h1, h2, q0, q1, m, r0, r1;\n\t"
        ".reg .u64 q, acc, t;\n\t"
        "mov.b64 {x0, x1}, %1;\n\t"
        "mov.b64 {s0, s1}, %2;\n\t"
        "mov.b64 {n0, n1}, %3;\n\t"
        "mul.wide.u32 t, x1, s0;\n\t"
        "mov.b64 {h1, h2}, t;\n\t"
        "cvt.u64.u32 acc, h1;\n\t"
        "mad.wide.u32 acc, x0, s1, acc;\n\t"
        "cvt.u64.u32 t, h2;\n\t"
        "mad.wide.u32 q, x1, s1, t;\n\t"
        "mov.b64 {h1, h2}, acc;\n\t"
        "cvt.u64.u32 t, h2;\n\t"
        "add.u64 q, q, t;\n\t"
        "mov.b64 {q0, q1}, q;\n\t"
        // x + q * (2^64 - p), low word
        "mad.wide.u32 acc, q0, n0, %1;\n\t"
        "mul.lo.u32 m, q0, n1;\n\t"
        "mad.lo.u32 m, q1, n0, m;\n\t"
        "mov.b64 {r0, r1}, acc;\n\t"
        "add.u32 r1, r1, m;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "l"(x), "l"(ones), "l"(np));
    return r;
}

// Shoup product of a 32-bit x by the constant w (companion ws = floor(w 2^64 / p)):
// with T = x*s0 and U = x*s1 + hi(T) (no overflow), floor(x*ws / 2^64) is
// exactly hi(U), so x*w - q*p is in [0, 2p).  Six 32-bit multiply-adds.
__device__ __forceinline__ u64 shoup_u32(uint32_t x, u64 w, u64 ws, u64 np) {
    u64 r;
    asm("{\n\t"
        ".reg .u32 w0, w1, s0, s1, n0, n1, t0, t1, u0, q, m, r0, r1;\n\t"
        ".reg .u64 t, u, acc;\n\t"
        "mov.b64 {w0, w1}, %2;\n\t"
        "mov.b64 {s0, s1}, %3;\n\t"
        "mov.b64 {n0, n1}, %4;\n\t"
        "mul.wide.u32 t, %1, s0;\n\t"
        "mov.b64 {t0, t1}, t;\n\t"
        "cvt.u64.u32 u, t1;\n\t"
        "mad.wide.u32 u, %1, s1, u;\n\t"
        "mov.b64 {u0, q}, u;\n\t"
        // x*w + q*(2^64 - p), low word
        "mul.wide.u32 acc, %1, w0;\n\t"
        "mad.wide.u32 acc, q, n0, acc;\n\t"
        "mul.lo.u32 m, %1, w1;\n\t"
        "mad.lo.u32 m, q, n1, m;\n\t"
        "mov.b64 {r0, r1}, acc;\n\t"
        "add.u32 r1, r1, m;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "r"(x), "l"(w), "l"(ws), "l"(np));
    return r;
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 p) { return csub(a + b, p); }
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 p) { return a >= b ? a - b : a + p - b; }

// acc += a*b for 32-bit a, b: one wide multiply-add with the 64-bit addend
__device__ __forceinline__ void mad_wide(u64 &acc, uint32_t a, uint32_t b) {
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// (hi:lo) += a*b, exact
__device__ __forceinline__ void mac128(u64 &lo, u64 &hi, u64 a, u64 b) {
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
}

// (hi:lo) mod p for hi < 2^64 (any value below 2^128)
__device__ __forceinline__ u64 reduce128(u64 lo, u64 hi, const PrimeInfo &P) {
    u64 t = shoup_lazy(hi, P.r64, P.r64_s, P.p) + shoup_lazy(lo, 1, P.one_s, P.p);  // < 4p
    t = csub(t, 2 * P.p);
    return csub(t, P.p);
}

__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeInfo &P) {
    u64 lo = 0, hi = 0;
    mac128(lo, hi, a, b);
    return reduce128(lo, hi, P);
}

// 16-byte load that asks L2 to keep the line (twiddle tables, reused by every
// limb of the same prime) ahead of streamed data such as key-switching keys.
__device__ __forceinline__ ulonglong2 ld_keep(const ulonglong2 *p) {
    ulonglong2 v;
    asm("{\n\t"
        ".reg .b64 pol;\n\t"
        "createpolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
        "ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], pol;\n\t"
        "}"
        : "=l"(v.x), "=l"(v.y)
        : "l"(p));
    return v;
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2 by the
// TMA unit; no register or shared-memory destination, nothing to wait for.
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Slot permutation of Automorph in bit-reversed evaluation order: output
// slot j reads input slot brv(((2 brv(j) + 1) * g mod 2N - 1) / 2).
__device__ __forceinline__ uint32_t automorph_src(uint32_t j, uint32_t g, int logN) {
    uint32_t rj = __brev(j) >> (32 - logN);
    uint32_t e = (uint32_t)(((2ull * rj + 1ull) * g) & ((2ull << logN) - 1ull));
    return __brev((e - 1) >> 1) >> (32 - logN);
}

// ------------------------------------------------------------------ descriptors
// A batch of limbs for one NTT launch: limb l reads src[l], writes dst[l]
// (equal for in-place work) and uses prime table entry prime[l].
struct NttBatch {
    int count;
    const u64 *src[kMaxBatch];
    u64 *dst[kMaxBatch];
    uint16_t prime[kMaxBatch];
};

// Epilogue of the last forward pass.  EPI_STORE writes the transform.
// EPI_LAZY writes it without the final reduction (small primes: values below
// 76p < 2^64), for consumers that only multiply-accumulate it exactly in 128
// bits and reduce once (the inner products after ModUp).
// EPI_SCALE treats batch limb l as limb (l / npolys) of polynomial (l % npolys)
// (the polynomials' limbs of one prime are adjacent in the batch):
//   out = (x - ntt) * c  [+ add[perm_g(n)]]  [+ out if accumulate]
// with c = cmul[prime] (value, Shoup companion).  This is the last step of
// ModDown (c = P^-1) and Rescale (c = q_{ell-1}^-1).
enum { EPI_STORE = 0, EPI_SCALE = 1, EPI_LAZY = 2 };
struct Epi {
    int mode;
    int npolys;
    const u64 *x[2];
    u64 *out[2];
    const u64 *add[2];
    uint32_t galois;
    int accumulate;
    const ulonglong2 *cmul;
};

// Basis conversion (the NewLimb step of ModUp/ModDown, Algorithm 6 and the
// table "CKKS Subroutines"): from n_src coefficient-form limbs x_i to n_dst
// limbs z_t = (sum_i [(x_i + add_i) * mul_i]_{q_i} * mat[t][i] - sub_t) mod t.
struct BConvPlan {
    int n_src, n_dst;
    uint16_t src_prime[kMaxSrc];
    u64 src_add[kMaxSrc];
    u64 src_mul[kMaxSrc], src_mul_s[kMaxSrc];
    uint16_t dst_pos[kMaxDst];
    uint16_t dst_prime[kMaxDst];
    u64 dst_sub[kMaxDst];
    u64 mat[kMaxDst][kMaxSrc];
    // Split form for the 32-bit multiply-add path (primes below 2^57), with
    // W = ceil(bits(max prime) / 2), C = mat = Ch*2^W + Cl, D = [C*2^W]_t =
    // Dh*2^W + Dl: matw = (Dh, Ch, Dl, Cl).
    uint4 matw[kMaxDst][kMaxSrc];
    u64 dst_rw[kMaxDst], dst_rw_s[kMaxDst];  // [2^W]_t, Shoup companion
    // Tensor-core form (primes below 2^56, at most 16 sources): tc_img holds,
    // per target t (n_dst rounded up to a multiple of 4), KG groups of an 8 x 8
    // f16 core matrix, row c and column j of group i < n_src being byte c of
    // [2^(8j) * mat[t][i]]_t, group KG-1 holding 4096 in column 0 of every row
    // (with the 2048 in the A operand: the bias 2^23 of every sum).  The
    // epilogue folds the sums of rows 5 and 6 with dst_r40 = [2^40]_t and adds
    // dst_off = [-sub_t]_t.
    const uint4 *tc_img;
    u64 dst_r40[kMaxDst], dst_r40_s[kMaxDst], dst_off[kMaxDst];
};

struct BConvGroup {
    const BConvPlan *plan;  // device pointer
    const u64 *src;         // [n_src][N] contiguous
    u64 *dst;               // limb t written at dst + dst_pos[t]*N
};
constexpr int kMaxGroups = 8;
struct BConvLaunch {
    int ngroups;
    int chunks;             // target chunks per group (grid.y = ngroups*chunks)
    int chunk;              // targets per chunk
    BConvGroup g[kMaxGroups];
};

}  // namespace ckks
