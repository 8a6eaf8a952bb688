/*
 * ckks_oracle.c -- plain, slow, single-threaded CPU oracle for the CKKS
 * key-switching path of "Does Fully Homomorphic Encryption Need Compute
 * Acceleration?" (arXiv 2112.06396).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it exists so the tests, the smoke check and the benchmark's CPU-baseline
 * leg have an independent answer to compare the CUDA path against.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Style: every modular operation is written with unsigned __int128 and the
 * C '%' operator.  No Shoup, no Barrett, no lazy reduction, no blocking or
 * fusion: each function follows the paper's definition or algorithm in the
 * paper's order so it can be read against the paper.
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *  - L and ell count limbs; alpha = ceil(L/dnum); beta = ceil(ell/alpha).
 *  - primes[0..L-1] are the chain q_0..q_{L-1}; primes[L..L+k-1] the special
 *    primes p_0..p_{k-1}.  At level ell the extended basis is ordered
 *    q_0..q_{ell-1}, p_0..p_{k-1}.
 *  - Evaluation form: a_hat[j] = sum_i a_i * psi^((2*brv(j)+1)*i) mod q, with
 *    psi the smallest primitive 2N-th root of unity mod q (bit-reversed order).
 *  - A key-switching key is [dnum][2][L+k][N]; row 0 holds a_j, row 1 holds
 *    b_j = -a_j*s + e_j + g_j*s', g_j = [P]_{q_i} on digit-j limbs, else 0
 *    (the Han-Ki hybrid key of Eq. (kskShape), Sec. 2.4).
 *  - A ciphertext (a, b) decrypts as a*s + b.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;
typedef __int128 i128;

typedef struct {
    int logN;
    int L;      /* chain limbs */
    int k;      /* special primes */
    int dnum;   /* key-switching digits */
    const u64 *primes; /* L + k primes: chain then special */
} or_params;

/* ------------------------------------------------------------------ */
/* Scalar modular arithmetic (Sec. 2.2, plain definitions)             */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
static u64 addmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a + b) % m); }
static u64 submod(u64 a, u64 b, u64 m) { return (u64)(((u128)a + m - (b % m)) % m); }

static u64 powmod(u64 a, u64 e, u64 m) {
    u64 r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}

/* Modular inverse by the extended Euclidean algorithm. */
static u64 invmod(u64 a, u64 m) {
    i128 t = 0, newt = 1, r = m, newr = a % m;
    while (newr != 0) {
        i128 q = r / newr, tmp;
        tmp = t - q * newt; t = newt; newt = tmp;
        tmp = r - q * newr; r = newr; newr = tmp;
    }
    if (t < 0) t += m;
    return (u64)t;
}

/* Deterministic Miller-Rabin for n < 2^64 (bases 2..37). */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* NTT-friendly primes q = 1 + m*2N < 2^bits, largest first (the configs ask
 * for the largest such primes below 2^bits).  Returns 0 on success. */
int or_gen_primes(int bits, int logN, int count, u64 *out) {
    if (bits < 2 || bits > 62) return -1;
    u64 twoN = (u64)2 << logN;
    u64 m = (((u64)1 << bits) - 2) / twoN;
    int got = 0;
    while (got < count && m > 0) {
        u64 q = 1 + m * twoN;
        if (or_is_prime(q)) out[got++] = q;
        m--;
    }
    return got == count ? 0 : -2;
}

/* Smallest primitive 2N-th root of unity mod q (Sec. 2.3 uses the NTT;
 * the root is a convention of this build). */
u64 or_min_psi(u64 q, int logN) {
    u64 N = (u64)1 << logN, twoN = 2 * N;
    u64 g = 0;
    for (u64 x = 2; x < q; x++) {
        u64 c = powmod(x, (q - 1) / twoN, q);
        if (powmod(c, N, q) == q - 1) { g = c; break; }
    }
    /* all primitive 2N-th roots are g^(odd) */
    u64 best = g, cur = g, g2 = mulmod(g, g, q);
    for (u64 i = 1; i < N; i++) {
        cur = mulmod(cur, g2, q);
        if (cur < best) best = cur;
    }
    return best;
}

static u64 brv(u64 x, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* ------------------------------------------------------------------ */
/* NTT / iNTT (Sec. 2.3 "Polynomial Representation")                   */
/* ------------------------------------------------------------------ */

/* The definition, O(N^2): out[j] = sum_i a_i psi^((2 brv(j)+1) i). */
void or_ntt_naive(const u64 *a, u64 *out, int logN, u64 q) {
    u64 N = (u64)1 << logN;
    u64 psi = or_min_psi(q, logN);
    for (u64 j = 0; j < N; j++) {
        u64 x = powmod(psi, 2 * brv(j, logN) + 1, q);
        u64 acc = 0, xp = 1;
        for (u64 i = 0; i < N; i++) {
            acc = addmod(acc, mulmod(a[i], xp, q), q);
            xp = mulmod(xp, x, q);
        }
        out[j] = acc;
    }
}

/* Fast forward transform, textbook form: twist by psi^i (negacyclic ->
 * cyclic), then the radix-2 decimation-in-frequency cyclic DFT with
 * omega = psi^2, whose output is in bit-reversed order. */
void or_ntt(u64 *a, int logN, u64 q) {
    u64 N = (u64)1 << logN;
    u64 psi = or_min_psi(q, logN);
    u64 omega = mulmod(psi, psi, q);
    u64 pw = 1;
    for (u64 i = 0; i < N; i++) { a[i] = mulmod(a[i], pw, q); pw = mulmod(pw, psi, q); }
    for (u64 len = N; len >= 2; len >>= 1) {
        u64 half = len / 2;
        u64 wlen = powmod(omega, N / len, q);
        for (u64 s = 0; s < N; s += len) {
            u64 w = 1;
            for (u64 t = 0; t < half; t++) {
                u64 u = a[s + t], v = a[s + t + half];
                a[s + t] = addmod(u, v, q);
                a[s + t + half] = mulmod(submod(u, v, q), w, q);
                w = mulmod(w, wlen, q);
            }
        }
    }
}

/* Exact inverse of or_ntt: undo each DIF stage in reverse order with
 * omega^-1, scale by N^-1, untwist by psi^-i. */
void or_intt(u64 *a, int logN, u64 q) {
    u64 N = (u64)1 << logN;
    u64 psi = or_min_psi(q, logN);
    u64 omega_inv = invmod(mulmod(psi, psi, q), q);
    for (u64 len = 2; len <= N; len <<= 1) {
        u64 half = len / 2;
        u64 wlen = powmod(omega_inv, N / len, q);
        for (u64 s = 0; s < N; s += len) {
            u64 w = 1;
            for (u64 t = 0; t < half; t++) {
                u64 x = a[s + t], y = mulmod(a[s + t + half], w, q);
                a[s + t] = addmod(x, y, q);
                a[s + t + half] = submod(x, y, q);
                w = mulmod(w, wlen, q);
            }
        }
    }
    u64 ninv = invmod(N % q, q), psi_inv = invmod(psi, q);
    u64 pw = ninv;
    for (u64 i = 0; i < N; i++) { a[i] = mulmod(a[i], pw, q); pw = mulmod(pw, psi_inv, q); }
}

/* ------------------------------------------------------------------ */
/* Automorph (Table "CKKS Subroutines"): X -> X^g                      */
/* ------------------------------------------------------------------ */

/* Coefficient form: a_i X^i -> a_i X^(i g mod 2N), negated past N. */
void or_automorph_coeff(const u64 *in, u64 *out, int logN, u64 g, u64 q) {
    u64 N = (u64)1 << logN, twoN = 2 * N;
    for (u64 i = 0; i < N; i++) {
        u64 e = (u64)(((u128)i * g) % twoN);
        if (e < N) out[e] = in[i] % q;
        else out[e - N] = submod(0, in[i], q);
    }
}

/* Evaluation form: slot j holds a(psi^(2 brv(j)+1)); sigma_g(a) there is
 * a(psi^((2 brv(j)+1) g)), which is stored at slot brv(((2brv(j)+1)g mod 2N - 1)/2). */
void or_automorph_eval(const u64 *in, u64 *out, int logN, u64 g) {
    u64 N = (u64)1 << logN, twoN = 2 * N;
    for (u64 j = 0; j < N; j++) {
        u64 e = (u64)(((u128)(2 * brv(j, logN) + 1) * g) % twoN);
        out[j] = in[brv((e - 1) / 2, logN)];
    }
}

/* ------------------------------------------------------------------ */
/* Parameter helpers                                                   */
/* ------------------------------------------------------------------ */
static int p_alpha(const or_params *P) { return (P->L + P->dnum - 1) / P->dnum; }
static int p_beta(const or_params *P, int ell) { int a = p_alpha(P); return (ell + a - 1) / a; }
static u64 prime_at(const or_params *P, int ell, int pos) {
    return pos < ell ? P->primes[pos] : P->primes[P->L + (pos - ell)];
}
static int key_index(const or_params *P, int ell, int pos) {
    return pos < ell ? pos : P->L + (pos - ell);
}
static size_t N_of(const or_params *P) { return (size_t)1 << P->logN; }

int or_alpha(const or_params *P) { return p_alpha(P); }
int or_beta(const or_params *P, int ell) { return p_beta(P, ell); }

/* ------------------------------------------------------------------ */
/* ModUp (Algorithm 6, "NewLimb" basis conversion)                     */
/* ------------------------------------------------------------------ */

/* Extend digit j of a (evaluation form, [ell][N]) to the basis
 * C_ell U P.  out is [ell+k][N]: digit limbs copied, every other limb is
 * iNTT -> y_i = x_i [(Q_j/q_i)^-1]_{q_i} -> z_t = sum_i y_i [Q_j/q_i]_t -> NTT. */
int or_modup(const or_params *P, int ell, int j, const u64 *a_eval, u64 *out) {
    size_t N = N_of(P);
    int alpha = p_alpha(P), k = P->k;
    int lo = j * alpha, hi = lo + alpha;
    if (hi > ell) hi = ell;
    if (lo >= ell) return -1;
    int na = hi - lo;
    /* step 1: iNTT of the digit limbs (limb-wise) */
    u64 *x = (u64 *)malloc(sizeof(u64) * na * N);
    for (int i = 0; i < na; i++) {
        memcpy(x + i * N, a_eval + (size_t)(lo + i) * N, sizeof(u64) * N);
        or_intt(x + i * N, P->logN, P->primes[lo + i]);
    }
    /* step 2: y_i = x_i * [(Q_j/q_i)^-1]_{q_i} */
    for (int i = 0; i < na; i++) {
        u64 qi = P->primes[lo + i];
        u64 qhat = 1;
        for (int i2 = 0; i2 < na; i2++)
            if (i2 != i) qhat = mulmod(qhat, P->primes[lo + i2] % qi, qi);
        u64 c = invmod(qhat, qi);
        for (size_t n = 0; n < N; n++) x[i * N + n] = mulmod(x[i * N + n], c, qi);
    }
    /* steps 3-4: new limbs (slot-wise), then NTT (limb-wise) */
    for (int t = 0; t < ell + k; t++) {
        u64 *dst = out + (size_t)t * N;
        if (t >= lo && t < hi) { memcpy(dst, a_eval + (size_t)t * N, sizeof(u64) * N); continue; }
        u64 pt = prime_at(P, ell, t);
        u64 *cst = (u64 *)malloc(sizeof(u64) * na);
        for (int i = 0; i < na; i++) {
            u64 qhat = 1;
            for (int i2 = 0; i2 < na; i2++)
                if (i2 != i) qhat = mulmod(qhat, P->primes[lo + i2] % pt, pt);
            cst[i] = qhat;
        }
        for (size_t n = 0; n < N; n++) {
            u64 acc = 0;
            for (int i = 0; i < na; i++) acc = addmod(acc, mulmod(x[i * N + n] % pt, cst[i], pt), pt);
            dst[n] = acc;
        }
        free(cst);
        or_ntt(dst, P->logN, pt);
    }
    free(x);
    return 0;
}

/* ------------------------------------------------------------------ */
/* KSKInnerProd (Table "CKKS Subroutines")                             */
/* ------------------------------------------------------------------ */

/* u = <row 0 of ksk, digits>, v = <row 1 of ksk, digits> over C_ell U P.
 * digits: [beta][ell+k][N]; key: [dnum][2][L+k][N]; u, v: [ell+k][N]. */
int or_ksk_inner_prod(const or_params *P, int ell, const u64 *digits, const u64 *key, u64 *u, u64 *v) {
    size_t N = N_of(P);
    int beta = p_beta(P, ell), ext = ell + P->k, LK = P->L + P->k;
    for (int t = 0; t < ext; t++) {
        u64 pt = prime_at(P, ell, t);
        int kt = key_index(P, ell, t);
        for (size_t n = 0; n < N; n++) {
            u64 au = 0, av = 0;
            for (int j = 0; j < beta; j++) {
                u64 d = digits[((size_t)j * ext + t) * N + n];
                u64 ka = key[(((size_t)j * 2 + 0) * LK + kt) * N + n];
                u64 kb = key[(((size_t)j * 2 + 1) * LK + kt) * N + n];
                au = addmod(au, mulmod(d, ka, pt), pt);
                av = addmod(av, mulmod(d, kb, pt), pt);
            }
            u[(size_t)t * N + n] = au;
            v[(size_t)t * N + n] = av;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* ModDown by P (Table "CKKS Subroutines"; rounding per Sec. 2.4)      */
/* ------------------------------------------------------------------ */

/* [floor(P/2)]_m for odd P = prod p: (P - 1)/2 mod m. */
static u64 halfP_mod(const or_params *P, u64 m) {
    u64 Pm = 1 % m;
    for (int i = 0; i < P->k; i++) Pm = mulmod(Pm, P->primes[P->L + i] % m, m);
    return mulmod(submod(Pm, 1, m), invmod(2 % m, m), m);
}
static u64 P_mod(const or_params *P, u64 m) {
    u64 Pm = 1 % m;
    for (int i = 0; i < P->k; i++) Pm = mulmod(Pm, P->primes[P->L + i] % m, m);
    return Pm;
}

/* in: [ell+k][N] evaluation form over C_ell U P; out: [ell][N] evaluation
 * form, out ~= round(in / P) (up to the fast-base-conversion error). */
int or_moddown(const or_params *P, int ell, const u64 *in, u64 *out) {
    size_t N = N_of(P);
    int k = P->k;
    u64 *x = (u64 *)malloc(sizeof(u64) * k * N);
    /* (1) iNTT the P limbs; (2) add floor(P/2); (3) times [(P/p_m)^-1]_{p_m} */
    for (int m = 0; m < k; m++) {
        u64 pm = P->primes[P->L + m];
        memcpy(x + m * N, in + (size_t)(ell + m) * N, sizeof(u64) * N);
        or_intt(x + m * N, P->logN, pm);
        u64 H = halfP_mod(P, pm);
        u64 phat = 1;
        for (int m2 = 0; m2 < k; m2++)
            if (m2 != m) phat = mulmod(phat, P->primes[P->L + m2] % pm, pm);
        u64 c = invmod(phat, pm);
        for (size_t n = 0; n < N; n++) x[m * N + n] = mulmod(addmod(x[m * N + n], H, pm), c, pm);
    }
    u64 *w = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < ell; i++) {
        u64 qi = P->primes[i];
        u64 *cst = (u64 *)malloc(sizeof(u64) * k);
        for (int m = 0; m < k; m++) {
            u64 phat = 1;
            for (int m2 = 0; m2 < k; m2++)
                if (m2 != m) phat = mulmod(phat, P->primes[P->L + m2] % qi, qi);
            cst[m] = phat;
        }
        u64 H = halfP_mod(P, qi);
        /* (4) z_i = sum_m y_m [P/p_m]_{q_i}; w_i = z_i - floor(P/2) (coefficient form) */
        for (size_t n = 0; n < N; n++) {
            u64 acc = 0;
            for (int m = 0; m < k; m++) acc = addmod(acc, mulmod(x[m * N + n] % qi, cst[m], qi), qi);
            w[n] = submod(acc, H, qi);
        }
        free(cst);
        /* (5) NTT; (6) out_i = (in_i - w_hat_i) * [P^-1]_{q_i} */
        or_ntt(w, P->logN, qi);
        u64 Pinv = invmod(P_mod(P, qi), qi);
        for (size_t n = 0; n < N; n++)
            out[(size_t)i * N + n] = mulmod(submod(in[(size_t)i * N + n], w[n], qi), Pinv, qi);
    }
    free(w);
    free(x);
    return 0;
}

/* ------------------------------------------------------------------ */
/* ModDown and Rescale merged (Sec. 5.1, NewMult): one fast basis       */
/* conversion dividing by D = P * q_{ell-1}                             */
/* ------------------------------------------------------------------ */

/* The dropped basis D: p_0..p_{k-1}, then q_{ell-1}. */
static u64 D_prime(const or_params *P, int ell, int m) { return m < P->k ? P->primes[P->L + m] : P->primes[ell - 1]; }
static u64 D_mod(const or_params *P, int ell, u64 m) {
    u64 r = 1 % m;
    for (int i = 0; i <= P->k; i++) r = mulmod(r, D_prime(P, ell, i) % m, m);
    return r;
}
/* [floor(D/2)]_m = (D - 1)/2 mod m (D is odd). */
static u64 halfD_mod(const or_params *P, int ell, u64 m) {
    return mulmod(submod(D_mod(P, ell, m), 1, m), invmod(2 % m, m), m);
}

/* in: [ell+k][N] evaluation form over C_ell U P; out: [ell-1][N] evaluation
 * form over C_{ell-1}, out ~= round(in / (P q_{ell-1})) up to the fast
 * conversion error.  Steps: (1) iNTT the k+1 limbs of D; (2) add
 * [floor(D/2)]; (3) times [(D/d_m)^-1]_{d_m}; (4) z_i = sum_m y_m [D/d_m]_{q_i}
 * - [floor(D/2)]_{q_i} for i < ell-1 (coefficient form); (5) NTT;
 * (6) out_i = (in_i - z_hat_i) [D^-1]_{q_i}.  Needs ell >= 2. */
int or_moddown_merged(const or_params *P, int ell, const u64 *in, u64 *out) {
    if (ell < 2) return -1;
    size_t N = N_of(P);
    int nd = P->k + 1;
    u64 *x = (u64 *)malloc(sizeof(u64) * nd * N);
    for (int m = 0; m < nd; m++) {
        u64 dm = D_prime(P, ell, m);
        const u64 *src = in + (size_t)(m < P->k ? ell + m : ell - 1) * N;
        memcpy(x + m * N, src, sizeof(u64) * N);
        or_intt(x + m * N, P->logN, dm);
        u64 H = halfD_mod(P, ell, dm);
        u64 dhat = 1;
        for (int m2 = 0; m2 < nd; m2++)
            if (m2 != m) dhat = mulmod(dhat, D_prime(P, ell, m2) % dm, dm);
        u64 c = invmod(dhat, dm);
        for (size_t n = 0; n < N; n++) x[m * N + n] = mulmod(addmod(x[m * N + n], H, dm), c, dm);
    }
    u64 *w = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < ell - 1; i++) {
        u64 qi = P->primes[i];
        u64 *cst = (u64 *)malloc(sizeof(u64) * nd);
        for (int m = 0; m < nd; m++) {
            u64 dhat = 1;
            for (int m2 = 0; m2 < nd; m2++)
                if (m2 != m) dhat = mulmod(dhat, D_prime(P, ell, m2) % qi, qi);
            cst[m] = dhat;
        }
        u64 H = halfD_mod(P, ell, qi);
        for (size_t n = 0; n < N; n++) {
            u64 acc = 0;
            for (int m = 0; m < nd; m++) acc = addmod(acc, mulmod(x[m * N + n] % qi, cst[m], qi), qi);
            w[n] = submod(acc, H, qi);
        }
        free(cst);
        or_ntt(w, P->logN, qi);
        u64 Dinv = invmod(D_mod(P, ell, qi), qi);
        for (size_t n = 0; n < N; n++)
            out[(size_t)i * N + n] = mulmod(submod(in[(size_t)i * N + n], w[n], qi), Dinv, qi);
    }
    free(w);
    free(x);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Rescale = ModDown_{B,1} (Algorithm 1): exact rounded division by     */
/* the last limb q_{ell-1}                                             */
/* ------------------------------------------------------------------ */
int or_rescale(const or_params *P, int ell, const u64 *in, u64 *out) {
    if (ell < 2) return -1;
    size_t N = N_of(P);
    u64 ql = P->primes[ell - 1];
    u64 h = ql / 2;
    u64 *c = (u64 *)malloc(sizeof(u64) * N);
    u64 *w = (u64 *)malloc(sizeof(u64) * N);
    memcpy(c, in + (size_t)(ell - 1) * N, sizeof(u64) * N);
    or_intt(c, P->logN, ql);
    for (size_t n = 0; n < N; n++) c[n] = addmod(c[n], h, ql);
    for (int i = 0; i < ell - 1; i++) {
        u64 qi = P->primes[i];
        for (size_t n = 0; n < N; n++) w[n] = submod(c[n] % qi, h % qi, qi);
        or_ntt(w, P->logN, qi);
        u64 inv = invmod(ql % qi, qi);
        for (size_t n = 0; n < N; n++)
            out[(size_t)i * N + n] = mulmod(submod(in[(size_t)i * N + n], w[n], qi), inv, qi);
    }
    free(c);
    free(w);
    return 0;
}

/* PModUp (Sec. 5.1): multiply by P mod Q, read the result modulo PQ. */
int or_pmodup(const or_params *P, int ell, const u64 *in, u64 *out) {
    size_t N = N_of(P);
    for (int t = 0; t < ell + P->k; t++) {
        if (t < ell) {
            u64 qi = P->primes[t], Pm = P_mod(P, qi);
            for (size_t n = 0; n < N; n++) out[(size_t)t * N + n] = mulmod(in[(size_t)t * N + n], Pm, qi);
        } else {
            memset(out + (size_t)t * N, 0, sizeof(u64) * N);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* KeySwitch, Rotate (Alg. 3), HRotate (Alg. 4)                         */
/* ------------------------------------------------------------------ */

/* Decomp -> ModUp every digit -> KSKInnerProd -> ModDown(u), ModDown(v). */
int or_keyswitch(const or_params *P, int ell, const u64 *a, const u64 *key, u64 *u, u64 *v) {
    size_t N = N_of(P);
    int beta = p_beta(P, ell), ext = ell + P->k;
    u64 *digits = (u64 *)malloc(sizeof(u64) * beta * ext * N);
    for (int j = 0; j < beta; j++) or_modup(P, ell, j, a, digits + (size_t)j * ext * N);
    u64 *uh = (u64 *)malloc(sizeof(u64) * ext * N), *vh = (u64 *)malloc(sizeof(u64) * ext * N);
    or_ksk_inner_prod(P, ell, digits, key, uh, vh);
    or_moddown(P, ell, uh, u);
    or_moddown(P, ell, vh, v);
    free(uh); free(vh); free(digits);
    return 0;
}

/* Algorithm 2: Mult with relinearisation and Rescale.  Slot-wise (evaluation
 * form) products (a3, b3, c3) = (a1*a2, a1*b2 + a2*b1, b1*b2); KeySwitch of a3
 * with the key for s^2 gives (u, v); (a', b') = (b3 + u, c3 + v); the result
 * is (Rescale(a'), Rescale(b')) at level ell-1.  Needs ell >= 2. */
int or_mult(const or_params *P, int ell, const u64 *a1, const u64 *b1, const u64 *a2, const u64 *b2,
            const u64 *key, u64 *oa, u64 *ob) {
    if (ell < 2) return -1;
    size_t N = N_of(P), sz = (size_t)ell * N;
    u64 *a3 = (u64 *)malloc(sizeof(u64) * sz), *b3 = (u64 *)malloc(sizeof(u64) * sz);
    u64 *c3 = (u64 *)malloc(sizeof(u64) * sz);
    for (int i = 0; i < ell; i++) {
        u64 q = P->primes[i];
        for (size_t n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            a3[o] = mulmod(a1[o], a2[o], q);
            b3[o] = addmod(mulmod(a1[o], b2[o], q), mulmod(a2[o], b1[o], q), q);
            c3[o] = mulmod(b1[o], b2[o], q);
        }
    }
    u64 *u = (u64 *)malloc(sizeof(u64) * sz), *v = (u64 *)malloc(sizeof(u64) * sz);
    or_keyswitch(P, ell, a3, key, u, v);
    for (int i = 0; i < ell; i++) {
        u64 q = P->primes[i];
        for (size_t n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            u[o] = addmod(b3[o], u[o], q);
            v[o] = addmod(c3[o], v[o], q);
        }
    }
    or_rescale(P, ell, u, oa);
    or_rescale(P, ell, v, ob);
    free(a3); free(b3); free(c3); free(u); free(v);
    return 0;
}

/* Algorithm 7 (NewMult, Sec. 5.1): the tensor step of Algorithm 2; ModUp of
 * the digits of a3 and KSKInnerProd with the key for s^2 give (u_hat, v_hat)
 * over C_ell U P; PModUp lifts b3 and c3 to the same basis and they are added
 * before any ModDown, so the ModDown by P and the Rescale by q_{ell-1} of
 * Algorithm 2 become one merged ModDown per polynomial.  Outputs at level
 * ell-1.  Needs ell >= 2. */
int or_newmult(const or_params *P, int ell, const u64 *a1, const u64 *b1, const u64 *a2, const u64 *b2,
               const u64 *key, u64 *oa, u64 *ob) {
    if (ell < 2) return -1;
    size_t N = N_of(P), sz = (size_t)ell * N;
    int beta = p_beta(P, ell), ext = ell + P->k;
    u64 *a3 = (u64 *)malloc(sizeof(u64) * sz), *b3 = (u64 *)malloc(sizeof(u64) * sz);
    u64 *c3 = (u64 *)malloc(sizeof(u64) * sz);
    for (int i = 0; i < ell; i++) {
        u64 q = P->primes[i];
        for (size_t n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            a3[o] = mulmod(a1[o], a2[o], q);
            b3[o] = addmod(mulmod(a1[o], b2[o], q), mulmod(a2[o], b1[o], q), q);
            c3[o] = mulmod(b1[o], b2[o], q);
        }
    }
    u64 *digits = (u64 *)malloc(sizeof(u64) * beta * ext * N);
    for (int j = 0; j < beta; j++) or_modup(P, ell, j, a3, digits + (size_t)j * ext * N);
    u64 *uh = (u64 *)malloc(sizeof(u64) * ext * N), *vh = (u64 *)malloc(sizeof(u64) * ext * N);
    or_ksk_inner_prod(P, ell, digits, key, uh, vh);
    u64 *bh = (u64 *)malloc(sizeof(u64) * ext * N), *ch = (u64 *)malloc(sizeof(u64) * ext * N);
    or_pmodup(P, ell, b3, bh);
    or_pmodup(P, ell, c3, ch);
    for (int t = 0; t < ext; t++) {
        u64 pt = prime_at(P, ell, t);
        for (size_t n = 0; n < N; n++) {
            size_t o = (size_t)t * N + n;
            uh[o] = addmod(uh[o], bh[o], pt);
            vh[o] = addmod(vh[o], ch[o], pt);
        }
    }
    or_moddown_merged(P, ell, uh, oa);
    or_moddown_merged(P, ell, vh, ob);
    free(a3); free(b3); free(c3); free(digits); free(uh); free(vh); free(bh); free(ch);
    return 0;
}

/* Encrypted inner product with the ModDown hoisted (Sec. 5.1, the consequence
 * of Algorithm 7): sum over i < n of NewMult(ct1_i, ct2_i).  Each pair's lifted
 * (u_hat_i + PModUp(b3_i), v_hat_i + PModUp(c3_i)) over C_ell U P is summed
 * first, and one merged ModDown by P*q_{ell-1} per polynomial ends the sum.
 * a1s..b2s: n pointers to [ell][N]; outputs [ell-1][N].  Needs ell >= 2. */
int or_newmult_sum(const or_params *P, int ell, int n, const u64 *const *a1s, const u64 *const *b1s,
                   const u64 *const *a2s, const u64 *const *b2s, const u64 *key, u64 *oa, u64 *ob) {
    if (ell < 2 || n < 1) return -1;
    size_t N = N_of(P), sz = (size_t)ell * N;
    int beta = p_beta(P, ell), ext = ell + P->k;
    u64 *su = (u64 *)calloc((size_t)ext * N, sizeof(u64)), *sv = (u64 *)calloc((size_t)ext * N, sizeof(u64));
    u64 *a3 = (u64 *)malloc(sizeof(u64) * sz), *b3 = (u64 *)malloc(sizeof(u64) * sz);
    u64 *c3 = (u64 *)malloc(sizeof(u64) * sz);
    u64 *digits = (u64 *)malloc(sizeof(u64) * beta * ext * N);
    u64 *uh = (u64 *)malloc(sizeof(u64) * ext * N), *vh = (u64 *)malloc(sizeof(u64) * ext * N);
    u64 *bh = (u64 *)malloc(sizeof(u64) * ext * N), *ch = (u64 *)malloc(sizeof(u64) * ext * N);
    for (int p = 0; p < n; p++) {
        for (int i = 0; i < ell; i++) {
            u64 q = P->primes[i];
            for (size_t m = 0; m < N; m++) {
                size_t o = (size_t)i * N + m;
                a3[o] = mulmod(a1s[p][o], a2s[p][o], q);
                b3[o] = addmod(mulmod(a1s[p][o], b2s[p][o], q), mulmod(a2s[p][o], b1s[p][o], q), q);
                c3[o] = mulmod(b1s[p][o], b2s[p][o], q);
            }
        }
        for (int j = 0; j < beta; j++) or_modup(P, ell, j, a3, digits + (size_t)j * ext * N);
        or_ksk_inner_prod(P, ell, digits, key, uh, vh);
        or_pmodup(P, ell, b3, bh);
        or_pmodup(P, ell, c3, ch);
        for (int t = 0; t < ext; t++) {
            u64 pt = prime_at(P, ell, t);
            for (size_t m = 0; m < N; m++) {
                size_t o = (size_t)t * N + m;
                su[o] = addmod(su[o], addmod(uh[o], bh[o], pt), pt);
                sv[o] = addmod(sv[o], addmod(vh[o], ch[o], pt), pt);
            }
        }
    }
    or_moddown_merged(P, ell, su, oa);
    or_moddown_merged(P, ell, sv, ob);
    free(su); free(sv); free(a3); free(b3); free(c3); free(digits); free(uh); free(vh); free(bh); free(ch);
    return 0;
}

/* Algorithm 3: automorph (a, b) first, key-switch a_rot, return (u, v + b_rot). */
int or_rotate(const or_params *P, int ell, const u64 *a, const u64 *b, u64 g, const u64 *key, u64 *oa, u64 *ob) {
    size_t N = N_of(P);
    u64 *ar = (u64 *)malloc(sizeof(u64) * ell * N), *br = (u64 *)malloc(sizeof(u64) * ell * N);
    for (int i = 0; i < ell; i++) {
        or_automorph_eval(a + (size_t)i * N, ar + (size_t)i * N, P->logN, g);
        or_automorph_eval(b + (size_t)i * N, br + (size_t)i * N, P->logN, g);
    }
    u64 *v = (u64 *)malloc(sizeof(u64) * ell * N);
    or_keyswitch(P, ell, ar, key, oa, v);
    for (int i = 0; i < ell; i++) {
        u64 qi = P->primes[i];
        for (size_t n = 0; n < N; n++)
            ob[(size_t)i * N + n] = addmod(v[(size_t)i * N + n], br[(size_t)i * N + n], qi);
    }
    free(ar); free(br); free(v);
    return 0;
}

/* Algorithm 4: Decomp and ModUp once; per rotation automorph the extended
 * digits, inner product with that rotation's key, ModDown, add b_rot. */
int or_hrotate(const or_params *P, int ell, const u64 *a, const u64 *b, int r, const u64 *gs,
               const u64 *const *keys, u64 *const *oa, u64 *const *ob) {
    size_t N = N_of(P);
    int beta = p_beta(P, ell), ext = ell + P->k;
    u64 *digits = (u64 *)malloc(sizeof(u64) * beta * ext * N);
    u64 *rot = (u64 *)malloc(sizeof(u64) * beta * ext * N);
    for (int j = 0; j < beta; j++) or_modup(P, ell, j, a, digits + (size_t)j * ext * N);
    u64 *uh = (u64 *)malloc(sizeof(u64) * ext * N), *vh = (u64 *)malloc(sizeof(u64) * ext * N);
    u64 *v = (u64 *)malloc(sizeof(u64) * ell * N), *br = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < r; i++) {
        for (int l = 0; l < beta * ext; l++)
            or_automorph_eval(digits + (size_t)l * N, rot + (size_t)l * N, P->logN, gs[i]);
        or_ksk_inner_prod(P, ell, rot, keys[i], uh, vh);
        or_moddown(P, ell, uh, oa[i]);
        or_moddown(P, ell, vh, v);
        for (int t = 0; t < ell; t++) {
            u64 qt = P->primes[t];
            or_automorph_eval(b + (size_t)t * N, br, P->logN, gs[i]);
            for (size_t n = 0; n < N; n++)
                ob[i][(size_t)t * N + n] = addmod(v[(size_t)t * N + n], br[n], qt);
        }
    }
    free(digits); free(rot); free(uh); free(vh); free(v); free(br);
    return 0;
}

/* ------------------------------------------------------------------ */
/* PtMatVecMult with hoisted ModUp and ModDown (Algorithm 8), arranged  */
/* as baby steps x giant steps (Sec. 5.2)                               */
/* ------------------------------------------------------------------ */

/* Diagonal (t, i) is diag[t*nb + i], an [ell+k][N] evaluation-form
 * polynomial over C_ell U P.  Baby step i > 0 rotates by g_baby[i] with
 * key_baby[i]; baby step 0 is the identity (no key).  Giant step t > 0
 * rotates the ModDown'ed partial sum by g_giant[t] (Algorithm 3) with
 * key_giant[t].  With rescale != 0 the sum is rescaled by q_{ell-1}. */
int or_ptmatvec(const or_params *P, int ell, const u64 *a, const u64 *b, int nb, int ng,
                const u64 *g_baby, const u64 *g_giant, const u64 *const *key_baby,
                const u64 *const *key_giant, const u64 *const *diag, int rescale, u64 *oa, u64 *ob) {
    size_t N = N_of(P);
    int beta = p_beta(P, ell), ext = ell + P->k;
    u64 *digits = (u64 *)malloc(sizeof(u64) * beta * ext * N);
    u64 *rot = (u64 *)malloc(sizeof(u64) * beta * ext * N);
    for (int j = 0; j < beta; j++) or_modup(P, ell, j, a, digits + (size_t)j * ext * N);
    u64 *uh = (u64 *)malloc(sizeof(u64) * ext * N), *vh = (u64 *)malloc(sizeof(u64) * ext * N);
    u64 *bh = (u64 *)malloc(sizeof(u64) * ext * N), *br = (u64 *)malloc(sizeof(u64) * ell * N);
    u64 *acc_a = (u64 *)malloc(sizeof(u64) * ext * N), *acc_b = (u64 *)malloc(sizeof(u64) * ext * N);
    u64 *ca = (u64 *)malloc(sizeof(u64) * ell * N), *cb = (u64 *)malloc(sizeof(u64) * ell * N);
    u64 *ra = (u64 *)calloc((size_t)ell * N, sizeof(u64)), *rb = (u64 *)calloc((size_t)ell * N, sizeof(u64));
    u64 *ta = (u64 *)malloc(sizeof(u64) * ell * N), *tb = (u64 *)malloc(sizeof(u64) * ell * N);
    for (int t = 0; t < ng; t++) {
        memset(acc_a, 0, sizeof(u64) * ext * N);
        memset(acc_b, 0, sizeof(u64) * ext * N);
        for (int i = 0; i < nb; i++) {
            const u64 *M = diag[(size_t)t * nb + i];
            if (i == 0) {
                or_pmodup(P, ell, a, uh);          /* (u_hat, v_hat + P b) = (P a, P b) */
                or_pmodup(P, ell, b, bh);
                memset(vh, 0, sizeof(u64) * ext * N);
            } else {
                for (int l = 0; l < beta * ext; l++)
                    or_automorph_eval(digits + (size_t)l * N, rot + (size_t)l * N, P->logN, g_baby[i]);
                or_ksk_inner_prod(P, ell, rot, key_baby[i], uh, vh);
                for (int l = 0; l < ell; l++)
                    or_automorph_eval(b + (size_t)l * N, br + (size_t)l * N, P->logN, g_baby[i]);
                or_pmodup(P, ell, br, bh);
            }
            for (int l = 0; l < ext; l++) {
                u64 pl = prime_at(P, ell, l);
                for (size_t n = 0; n < N; n++) {
                    size_t o = (size_t)l * N + n;
                    acc_a[o] = addmod(acc_a[o], mulmod(M[o], uh[o], pl), pl);
                    acc_b[o] = addmod(acc_b[o], mulmod(M[o], addmod(vh[o], bh[o], pl), pl), pl);
                }
            }
        }
        or_moddown(P, ell, acc_a, ca);
        or_moddown(P, ell, acc_b, cb);
        if (t > 0) {
            or_rotate(P, ell, ca, cb, g_giant[t], key_giant[t], ta, tb);
            memcpy(ca, ta, sizeof(u64) * ell * N);
            memcpy(cb, tb, sizeof(u64) * ell * N);
        }
        for (int l = 0; l < ell; l++) {
            u64 ql = P->primes[l];
            for (size_t n = 0; n < N; n++) {
                size_t o = (size_t)l * N + n;
                ra[o] = addmod(ra[o], ca[o], ql);
                rb[o] = addmod(rb[o], cb[o], ql);
            }
        }
    }
    if (rescale) {
        or_rescale(P, ell, ra, oa);
        or_rescale(P, ell, rb, ob);
    } else {
        memcpy(oa, ra, sizeof(u64) * ell * N);
        memcpy(ob, rb, sizeof(u64) * ell * N);
    }
    free(digits); free(rot); free(uh); free(vh); free(bh); free(br);
    free(acc_a); free(acc_b); free(ca); free(cb); free(ra); free(rb); free(ta); free(tb);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Key generation, encryption, decryption (test data; Eq. kskShape)     */
/* ------------------------------------------------------------------ */

/* Signed small coefficients -> evaluation form over primes[first..first+n). */
static void small_to_eval(const or_params *P, const int64_t *c, const u64 *primes, int n, u64 *out) {
    size_t N = N_of(P);
    for (int l = 0; l < n; l++) {
        u64 q = primes[l];
        for (size_t i = 0; i < N; i++) {
            int64_t x = c[i];
            out[(size_t)l * N + i] = x >= 0 ? ((u64)x) % q : submod(0, ((u64)(-x)) % q, q);
        }
        or_ntt(out + (size_t)l * N, P->logN, q);
    }
}

/* Evaluation form of a signed polynomial over all L+k primes. */
int or_signed_to_eval(const or_params *P, const int64_t *c, u64 *out) {
    small_to_eval(P, c, P->primes, P->L + P->k, out);
    return 0;
}

/* Key switching s' -> s: a [dnum][L+k][N] uniform (evaluation form),
 * s ternary coefficients, sp = s' in evaluation form [L+k][N],
 * e [dnum][N] error coefficients; key out [dnum][2][L+k][N]. */
int or_keygen(const or_params *P, const u64 *a, const int64_t *s, const u64 *sp, const int64_t *e, u64 *key) {
    size_t N = N_of(P);
    int LK = P->L + P->k, alpha = p_alpha(P);
    u64 *sh = (u64 *)malloc(sizeof(u64) * LK * N), *eh = (u64 *)malloc(sizeof(u64) * LK * N);
    small_to_eval(P, s, P->primes, LK, sh);
    for (int j = 0; j < P->dnum; j++) {
        small_to_eval(P, e + (size_t)j * N, P->primes, LK, eh);
        for (int l = 0; l < LK; l++) {
            u64 q = P->primes[l];
            int in_digit = (l < P->L) && (l / alpha == j);
            u64 gj = in_digit ? P_mod(P, q) : 0;
            for (size_t n = 0; n < N; n++) {
                size_t o = (size_t)l * N + n;
                u64 aj = a[(size_t)j * LK * N + o];
                u64 bj = addmod(submod(eh[o], mulmod(aj, sh[o], q), q), mulmod(gj, sp[o], q), q);
                key[(((size_t)j * 2 + 0) * LK + l) * N + n] = aj;
                key[(((size_t)j * 2 + 1) * LK + l) * N + n] = bj;
            }
        }
    }
    free(sh); free(eh);
    return 0;
}

/* Key compression (Sec. 5.3): the uniform half a_j of a key-switching key is
 * regenerated from a 64-bit seed instead of being stored.  The generator is
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): draw c of seed s is mix(s + (c + 1) * gamma) with
 * gamma = 0x9E3779B97F4A7C15 and mix(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
 * z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.  Element (j, l, n) of a
 * (digit j, key limb l of the L+k, coefficient n; evaluation form) takes the
 * draws 16e .. 16e+15 with e = (j*(L+k) + l)*N + n and keeps the first whose
 * top b bits (b = bit length of the limb's prime q) are below q; if none is,
 * the last draw's top bits mod q. */
static u64 sm_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static int bitlen(u64 x) {
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}
u64 or_prng_key_a(const or_params *P, u64 seed, int j, int l, u64 n) {
    u64 q = P->primes[l];
    int b = bitlen(q);
    u64 e = ((u64)j * (u64)(P->L + P->k) + (u64)l) * (u64)N_of(P) + n;
    u64 v = 0;
    for (int r = 0; r < 16; r++) {
        v = sm_mix(seed + (16 * e + (u64)r + 1) * 0x9E3779B97F4A7C15ull) >> (64 - b);
        if (v < q) return v;
    }
    return v % q;
}
/* a: [dnum][L+k][N], the whole uniform half of the key for this seed. */
int or_prng_key_a_fill(const or_params *P, u64 seed, u64 *a) {
    size_t N = N_of(P);
    int LK = P->L + P->k;
    for (int j = 0; j < P->dnum; j++)
        for (int l = 0; l < LK; l++)
            for (size_t n = 0; n < N; n++) a[((size_t)j * LK + l) * N + n] = or_prng_key_a(P, seed, j, l, n);
    return 0;
}

/* s' for a rotation key: sigma_g(s), evaluation form over all L+k primes. */
int or_rot_secret(const or_params *P, const int64_t *s, u64 g, u64 *out) {
    size_t N = N_of(P);
    int LK = P->L + P->k;
    u64 *tmp = (u64 *)malloc(sizeof(u64) * LK * N);
    small_to_eval(P, s, P->primes, LK, tmp);
    for (int l = 0; l < LK; l++) or_automorph_eval(tmp + (size_t)l * N, out + (size_t)l * N, P->logN, g);
    free(tmp);
    return 0;
}

/* s' for a relinearisation key: s^2, evaluation form over all L+k primes. */
int or_sq_secret(const or_params *P, const int64_t *s, u64 *out) {
    size_t N = N_of(P);
    int LK = P->L + P->k;
    small_to_eval(P, s, P->primes, LK, out);
    for (int l = 0; l < LK; l++) {
        u64 q = P->primes[l];
        for (size_t n = 0; n < N; n++) out[(size_t)l * N + n] = mulmod(out[(size_t)l * N + n], out[(size_t)l * N + n], q);
    }
    return 0;
}

/* b = -a*s + m + e at level ell (a given uniform in evaluation form). */
int or_encrypt(const or_params *P, int ell, const int64_t *s, const int64_t *m_plus_e, const u64 *a, u64 *b) {
    size_t N = N_of(P);
    u64 *sh = (u64 *)malloc(sizeof(u64) * ell * N), *mh = (u64 *)malloc(sizeof(u64) * ell * N);
    small_to_eval(P, s, P->primes, ell, sh);
    small_to_eval(P, m_plus_e, P->primes, ell, mh);
    for (int l = 0; l < ell; l++) {
        u64 q = P->primes[l];
        for (size_t n = 0; n < N; n++) {
            size_t o = (size_t)l * N + n;
            b[o] = submod(mh[o], mulmod(a[o], sh[o], q), q);
        }
    }
    free(sh); free(mh);
    return 0;
}

/* Coefficient-form residues of a*s + b at level ell. */
int or_decrypt(const or_params *P, int ell, const int64_t *s, const u64 *a, const u64 *b, u64 *out) {
    size_t N = N_of(P);
    u64 *sh = (u64 *)malloc(sizeof(u64) * ell * N);
    small_to_eval(P, s, P->primes, ell, sh);
    for (int l = 0; l < ell; l++) {
        u64 q = P->primes[l];
        for (size_t n = 0; n < N; n++) {
            size_t o = (size_t)l * N + n;
            out[o] = addmod(mulmod(a[o], sh[o], q), b[o], q);
        }
        or_intt(out + (size_t)l * N, P->logN, q);
    }
    free(sh);
    return 0;
}

/* Per-limb forward / inverse transforms over the level-ell extended basis,
 * for tests that need coefficient views of oracle outputs. */
int or_ntt_limbs(const or_params *P, int ell, u64 *x, int first, int count, int inverse) {
    size_t N = N_of(P);
    for (int t = first; t < first + count; t++) {
        u64 q = prime_at(P, ell, t);
        if (inverse) or_intt(x + (size_t)t * N, P->logN, q);
        else or_ntt(x + (size_t)t * N, P->logN, q);
    }
    return 0;
}
