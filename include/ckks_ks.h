/*
 * ckks_ks.h -- C ABI of the GB300 (sm_103a) CKKS key-switching library.
 *
 * The calls follow the operations of "Does Fully Homomorphic Encryption Need
 * Compute Acceleration?" (arXiv 2112.06396): the table "CKKS Subroutines"
 * (ModDown, ModUp, Decomp, KSKInnerProd, Automorph), Algorithms 1, 3, 4, 6
 * and 8, and Sec. 5.1 (PModUp).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Ring Z_Q[X]/(X^N+1), N = 2^logN.  A polynomial is limb-major
 *    uint64_t[nlimbs][N], contiguous, device memory, 16-byte aligned, every
 *    residue fully reduced in [0, q).
 *  - ell ("level") counts the limbs of a ciphertext, 1 <= ell <= L.  The
 *    extended basis at level ell is ordered q_0..q_{ell-1}, p_0..p_{k-1};
 *    "position t" of an extended polynomial [ell+k][N] is the t-th modulus of
 *    that list.
 *  - alpha = ceil(L/dnum) limbs per digit; beta = ceil(ell/alpha) digits at
 *    level ell; digit j covers chain limbs [j*alpha, min((j+1)*alpha, ell))
 *    (Decomp, table "CKKS Subroutines"; Table 1 with ell and L counting limbs).
 *  - Evaluation (NTT) form is the default.  Slot j of the evaluation form of
 *    a holds a(psi^(2*brv(j)+1)), brv the logN-bit reversal and psi the
 *    smallest primitive 2N-th root of unity mod q (Sec. 2.3).
 *  - A key-switching key is uint64_t[dnum][2][L+k][N] in evaluation form:
 *    [j][0] is a_j (uniform), [j][1] is b_j = -a_j*s + e_j + g_j*s' with
 *    g_j = [P]_{q_i} on the limbs of digit j and 0 elsewhere (the 2 x dnum key
 *    of Eq. (kskShape), Sec. 2.4).  Keys are always stored at full level L;
 *    a call at level ell reads the limbs q_0..q_{ell-1}, p_0..p_{k-1}.
 *  - A ciphertext is two polynomials (a, b) that decrypt as a*s + b.
 *  - Ownership: the caller owns every device buffer (inputs, outputs, keys,
 *    workspace).  The library owns only its context (constant tables).
 *  - Streams: every device call enqueues work on `stream` and returns without
 *    synchronising.  Inputs must stay valid until that work completes.
 *    Outputs must not alias inputs unless a call says so.
 *  - Workspace: calls taking `ws` need ckks_workspace_bytes() bytes of device
 *    memory, 16-byte aligned, not shared with concurrently running calls.
 *  - Host threads: compute calls only read the context (apart from recording
 *    the last CUDA error), so several host threads may issue them at once on
 *    different streams with separate workspaces while the measurement hook is
 *    off.  The calls that change the context (ckks_key_register_seed,
 *    ckks_key_unregister, ckks_bconv_select, ckks_tune_set, ckks_autotune,
 *    ckks_profile_*, ckks_ctx_destroy) must not overlap any other call on it.
 *  - Errors: CKKS_EINVAL for bad arguments (checked on the host before any
 *    launch), CKKS_ECUDA when a launch fails (ckks_last_cuda_error() gives the
 *    cudaError_t), CKKS_EUNSUPPORTED for parameters a call cannot serve, and
 *    CKKS_ETIMEOUT from ckks_poll_status when a bounded device-side wait gave up
 *    (see there).  No call allocates device memory after ckks_ctx_create() except
 *    ckks_server_create().
 */
#ifndef CKKS_KS_H
#define CKKS_KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ckks_stream_t; /* the same type as cudaStream_t */
typedef struct ckks_ctx ckks_ctx;

enum {
    CKKS_OK = 0,
    CKKS_EINVAL = 1,
    CKKS_ENOMEM = 2,
    CKKS_ECUDA = 3,
    CKKS_EUNSUPPORTED = 4,
    CKKS_ETIMEOUT = 5
};

/* Operation ids for ckks_workspace_bytes(). */
enum {
    CKKS_OP_MODUP = 1,
    CKKS_OP_MODDOWN = 2,
    CKKS_OP_KEYSWITCH = 3,
    CKKS_OP_ROTATE = 4,
    CKKS_OP_HROTATE = 5,
    CKKS_OP_RESCALE = 6,
    CKKS_OP_PTMATVEC = 7,
    CKKS_OP_KEYGEN = 8,
    CKKS_OP_MULT = 9,
    CKKS_OP_NEWMULT = 10,
    CKKS_OP_KEYGEN_SEEDED = 11
};

typedef struct {
    int logN;          /* 10 <= logN <= 17 */
    int L;             /* chain limbs q_0..q_{L-1}, 1 <= L <= 64 */
    int k;             /* special primes p_0..p_{k-1}, 1 <= k <= 32 */
    int dnum;          /* key-switching digits, 1 <= dnum <= L */
    const uint64_t *q; /* host array [L]: distinct primes, q = 1 mod 2N, q < 2^60 */
    const uint64_t *p; /* host array [k]: distinct primes, p = 1 mod 2N, p < 2^60 */
} ckks_params;

/* Text for a status code (static storage). */
const char *ckks_strerror(int status);

/* Host only.  The `count` largest primes q = 1 + m*2N below 2^bits, largest
 * first, written to the host array out[count].  Chain primes are the first L
 * of this list and special primes the next k (a reading: the paper fixes no
 * prime order).  Returns CKKS_EINVAL if bits is outside [20, 60] or too few
 * primes exist. */
int ckks_gen_primes(int bits, int logN, int count, uint64_t *out);

/* Create a context on CUDA device `device`: validates the parameters, builds
 * the twiddle, Shoup and basis-conversion tables on the host and uploads them
 * (the only device allocation the library makes).  *out receives the handle. */
int ckks_ctx_create(const ckks_params *params, int device, ckks_ctx **out);
/* Frees the context's device tables; the caller must have synchronised every
 * stream that used it. */
int ckks_ctx_destroy(ckks_ctx *ctx);
/* cudaError_t of the last failed CUDA call made through this context. */
int ckks_last_cuda_error(const ckks_ctx *ctx);
/* Device bytes of the context's constant tables. */
size_t ckks_ctx_table_bytes(const ckks_ctx *ctx);

/* Workspace bytes the call `op` needs at level ell (r = rotation count for
 * CKKS_OP_HROTATE, giant-step count for CKKS_OP_PTMATVEC, else ignored). */
int ckks_workspace_bytes(const ckks_ctx *ctx, int op, int level, int r, size_t *bytes);

/* NTT (Sec. 2.3): in place, coefficient -> evaluation form, on positions
 * [first, first+count) of an extended polynomial at level ell.  d_poly points
 * to position 0.  Negacyclic, output in bit-reversed order (see above). */
int ckks_ntt(ckks_ctx *ctx, uint64_t *d_poly, int level, int first, int count, ckks_stream_t stream);
/* iNTT: the exact inverse of ckks_ntt (includes the factor N^-1). */
int ckks_intt(ckks_ctx *ctx, uint64_t *d_poly, int level, int first, int count, ckks_stream_t stream);

/* Automorph (table "CKKS Subroutines"): out = psi_g(in), X -> X^g, on nlimbs
 * evaluation-form limbs.  g odd, 0 < g < 2N (g = 5^r mod 2N rotates by r
 * slots, g = 2N-1 conjugates).  d_out must not alias d_in. */
int ckks_automorph(ckks_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int nlimbs, uint32_t galois,
                   ckks_stream_t stream);

/* ModUp of digit `digit` (Algorithm 6): d_a is [ell][N] evaluation form;
 * d_out receives [ell+k][N] over q_0..q_{ell-1}, p_0..p_{k-1}: the digit's own
 * limbs copied, every other limb = NTT(sum_i [x_i (Q_j/q_i)^-1]_{q_i} [Q_j/q_i]_t)
 * with x = iNTT(digit limbs).  Workspace CKKS_OP_MODUP. */
int ckks_modup(ckks_ctx *ctx, const uint64_t *d_a, int level, int digit, uint64_t *d_out, void *ws,
               ckks_stream_t stream);

/* KSKInnerProd (table "CKKS Subroutines"): d_digits is [beta][ell+k][N] (the
 * beta ModUp outputs); u = sum_j digit_j * key[j][0], v = sum_j digit_j *
 * key[j][1], both [ell+k][N]. */
int ckks_ksk_inner_prod(ckks_ctx *ctx, const uint64_t *d_digits, int level, const uint64_t *d_key,
                        uint64_t *d_u, uint64_t *d_v, ckks_stream_t stream);

/* ModDown by P (table "CKKS Subroutines", rounding as in Sec. 2.4): d_in is
 * [ell+k][N]; d_out [ell][N] = round(in / P) up to the fast base conversion
 * error eps in [0, k).  Workspace CKKS_OP_MODDOWN. */
int ckks_moddown(ckks_ctx *ctx, const uint64_t *d_in, int level, uint64_t *d_out, void *ws,
                 ckks_stream_t stream);

/* PModUp (Sec. 5.1): d_out [ell+k][N] = P * d_in on q limbs, 0 on p limbs. */
int ckks_pmodup(ckks_ctx *ctx, const uint64_t *d_in, int level, uint64_t *d_out, ckks_stream_t stream);

/* Rescale = ModDown_{B,1} (Algorithm 1): d_out [ell-1][N] = round(in / q_{ell-1})
 * exactly, for ell >= 2.  Workspace CKKS_OP_RESCALE. */
int ckks_rescale(ckks_ctx *ctx, const uint64_t *d_in, int level, uint64_t *d_out, void *ws,
                 ckks_stream_t stream);

/* KeySwitch (the core of Algorithms 2-4): Decomp -> ModUp every digit ->
 * KSKInnerProd -> ModDown(u), ModDown(v).  d_a [ell][N]; d_u, d_v [ell][N] with
 * u*s + v ~= a*s'.  Workspace CKKS_OP_KEYSWITCH. */
int ckks_keyswitch(ckks_ctx *ctx, const uint64_t *d_a, int level, const uint64_t *d_key, uint64_t *d_u,
                   uint64_t *d_v, void *ws, ckks_stream_t stream);

/* Rotate (Algorithm 3): automorph (a, b) by g, key-switch a_rot with the key
 * for psi_g(s) -> s, return (u, v + b_rot).  Workspace CKKS_OP_ROTATE. */
int ckks_rotate(ckks_ctx *ctx, const uint64_t *d_a, const uint64_t *d_b, int level, uint32_t galois,
                const uint64_t *d_key, uint64_t *d_oa, uint64_t *d_ob, void *ws, ckks_stream_t stream);

/* HRotate (Algorithm 4): Decomp and ModUp once, then for i < r: automorph the
 * extended digits by galois[i], KSKInnerProd with d_keys[i], ModDown, add the
 * automorphed b.  galois, d_keys, d_oa, d_ob are host arrays of length r
 * (d_keys/d_oa/d_ob hold device pointers).  Workspace CKKS_OP_HROTATE(r). */
int ckks_hrotate(ckks_ctx *ctx, const uint64_t *d_a, const uint64_t *d_b, int level, int r,
                 const uint32_t *galois, const uint64_t *const *d_keys, uint64_t *const *d_oa,
                 uint64_t *const *d_ob, void *ws, ckks_stream_t stream);

/* Batched key switching: n independent ciphertexts, each at its own level
 * levels[i] (1..L) and with its own key, processed together so that every
 * step of the pipeline is one kernel launch over the whole batch (iNTT of the
 * inputs, ModUp's basis conversion, NTT of the new limbs, KSKInnerProd, iNTT
 * of the P-limbs, ModDown's basis conversion, NTT + scale), in batches of 64.
 * The arithmetic per ciphertext is that of the single-ciphertext calls, and
 * so are the bits of every result:
 *   d_b == NULL or d_b[i] == NULL: KeySwitch of d_a[i] with d_keys[i]
 *     (as ckks_keyswitch; galois[i] is ignored, galois may be NULL);
 *   otherwise: HRotate of (d_a[i], d_b[i]) by the one Galois element
 *     galois[i] with its rotation key d_keys[i] (Algorithm 4 with r = 1, as
 *     ckks_hrotate).
 * Every array is a host array of length n; the pointers in it are device
 * pointers.  Inputs are [levels[i]][N] (evaluation form); d_oa[i], d_ob[i]
 * receive [levels[i]][N] and must not overlap any input or each other.  Keys
 * are [dnum][2][L+k][N] and may be shared between entries.  The workspace
 * holds every ciphertext's intermediates at once: its size comes from
 * ckks_batch_workspace_bytes with the same levels.  Contexts whose primes are
 * too wide for the split basis conversion run the entries one after another.
 * Returns CKKS_EINVAL for n < 0, a level out of range, a null or misaligned
 * pointer, or an invalid Galois element of a rotation entry. */
int ckks_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, size_t *bytes);
int ckks_keyswitch_batch(ckks_ctx *ctx, int n, const uint64_t *const *d_a, const uint64_t *const *d_b,
                         const int *levels, const uint32_t *galois, const uint64_t *const *d_keys,
                         uint64_t *const *d_oa, uint64_t *const *d_ob, void *ws, ckks_stream_t stream);

/* Batched HRotate with hoisted rotations (Algorithm 4 over many ciphertexts):
 * ciphertext c (d_a[c], d_b[c] at levels[c]) is rotated by nrot[c] >= 1 Galois
 * elements; the rotations are listed ciphertext by ciphertext in galois,
 * d_keys, d_oa, d_ob (sum of nrot entries; d_oa/d_ob [levels[c]][N]).  The
 * ModUp of every ciphertext runs once (one launch per step for all of them),
 * then the inner product and ModDown of every rotation (one launch per step
 * for all rotations, 64 per launch).  Bits: those of ckks_hrotate with the
 * same rotations.  Workspace: ckks_hrotate_batch_workspace_bytes. */
int ckks_hrotate_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, const int *nrot,
                                       size_t *bytes);
int ckks_hrotate_batch(ckks_ctx *ctx, int n, const uint64_t *const *d_a, const uint64_t *const *d_b,
                       const int *levels, const int *nrot, const uint32_t *galois, const uint64_t *const *d_keys,
                       uint64_t *const *d_oa, uint64_t *const *d_ob, void *ws, ckks_stream_t stream);

/* Mult with relinearisation and Rescale (Algorithm 2): for ciphertexts
 * (d_a1, d_b1), (d_a2, d_b2) at level ell >= 2 (evaluation form, [ell][N]):
 * (a3, b3, c3) = (a1 a2, a1 b2 + a2 b1, b1 b2) slot-wise, (u, v) = KeySwitch
 * of a3 with the relinearisation key d_key (s^2 -> s), and the outputs
 * d_oa, d_ob ([ell-1][N]) are Rescale(b3 + u), Rescale(c3 + v).  Workspace
 * CKKS_OP_MULT.  The batched form runs n such products (each at its own level,
 * with its own key) with one launch per pipeline step, with the same bits per
 * entry; its workspace comes from ckks_mult_batch_workspace_bytes.  Outputs
 * must not overlap inputs.  CKKS_EINVAL for a level < 2 or > L, or a null or
 * misaligned pointer. */
int ckks_mult(ckks_ctx *ctx, const uint64_t *d_a1, const uint64_t *d_b1, const uint64_t *d_a2,
              const uint64_t *d_b2, int level, const uint64_t *d_key, uint64_t *d_oa, uint64_t *d_ob, void *ws,
              ckks_stream_t stream);
int ckks_mult_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, size_t *bytes);
int ckks_mult_batch(ckks_ctx *ctx, int n, const uint64_t *const *d_a1, const uint64_t *const *d_b1,
                    const uint64_t *const *d_a2, const uint64_t *const *d_b2, const int *levels,
                    const uint64_t *const *d_keys, uint64_t *const *d_oa, uint64_t *const *d_ob, void *ws,
                    ckks_stream_t stream);

/* NewMult (Algorithm 7, Sec. 5.1): the product of ckks_mult with its two
 * ModDowns merged.  The tensor step and the ModUp / KSKInnerProd of a3 are
 * those of Algorithm 2; PModUp(b3) and PModUp(c3) (P times the polynomial on
 * the chain limbs, 0 on the P-limbs) are added to (u_hat, v_hat) inside the
 * inner product, and one ModDown by D = P*q_{ell-1} per polynomial (fast basis
 * conversion from the k P-limbs and q_{ell-1} to q_0..q_{ell-2}, rounding by
 * adding floor(D/2), then (x - conv) * D^-1) gives the outputs at level
 * ell-1.  Same message as ckks_mult within the error bounds, different bits.
 * Workspace CKKS_OP_NEWMULT; batched form as ckks_mult_batch.  Needs
 * k + 1 <= 32 (CKKS_EUNSUPPORTED otherwise). */
int ckks_newmult(ckks_ctx *ctx, const uint64_t *d_a1, const uint64_t *d_b1, const uint64_t *d_a2,
                 const uint64_t *d_b2, int level, const uint64_t *d_key, uint64_t *d_oa, uint64_t *d_ob, void *ws,
                 ckks_stream_t stream);
int ckks_newmult_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, size_t *bytes);
int ckks_newmult_batch(ckks_ctx *ctx, int n, const uint64_t *const *d_a1, const uint64_t *const *d_b1,
                       const uint64_t *const *d_a2, const uint64_t *const *d_b2, const int *levels,
                       const uint64_t *const *d_keys, uint64_t *const *d_oa, uint64_t *const *d_ob, void *ws,
                       ckks_stream_t stream);

/* Encrypted inner product with the ModDown hoisted (Sec. 5.1, a consequence of
 * Algorithm 7): out = sum over i < n of NewMult((a1[i], b1[i]), (a2[i], b2[i]))
 * computed with one merged ModDown for the whole sum: each pair's tensor step,
 * ModUp and KSKInnerProd with PModUp(b3), PModUp(c3) added run as one batch,
 * the n lifted (u, v) are summed over the extended basis, and one ModDown by
 * P*q_{ell-1} per polynomial gives d_oa, d_ob [ell-1][N].  All pairs at
 * `level` (>= 2) with one relinearisation key; 1 <= n <= 64.  For n = 1 the
 * bits are those of ckks_newmult.  Workspace: ckks_newmult_batch_workspace_bytes
 * with n copies of the level.  CKKS_EUNSUPPORTED for contexts without the split
 * basis conversion or with k + 1 > 32. */
int ckks_newmult_sum(ckks_ctx *ctx, int n, const uint64_t *const *d_a1, const uint64_t *const *d_b1,
                     const uint64_t *const *d_a2, const uint64_t *const *d_b2, int level, const uint64_t *d_key,
                     uint64_t *d_oa, uint64_t *d_ob, void *ws, ckks_stream_t stream);

/* PtMatVecMult with hoisted ModUp and ModDown (Algorithm 8) in baby-step /
 * giant-step form (Sec. 5.2): nb baby steps, ng giant steps, diagonal (t, i) =
 * d_diag[t*nb + i], an [ell+k][N] evaluation-form plaintext over the extended
 * basis.  Baby step 0 and giant step 0 are the identity: g_baby[0],
 * key_baby[0], g_giant[0], key_giant[0] are ignored.  For each giant step t:
 * acc = sum_i diag(t,i) * (u_i, v_i + PModUp(psi_{g_i}(b))) over the extended
 * basis, (c_a, c_b) = ModDown(acc), rotated by g_giant[t] (Algorithm 3) when
 * t > 0; the sum over t is rescaled by q_{ell-1} when rescale != 0.  Output
 * [ell'][N] with ell' = ell-1 if rescale else ell.  All arrays are host
 * arrays of device pointers / values.  Workspace CKKS_OP_PTMATVEC(ng).
 * With at most 8 giant steps, 64 diagonals and 4 digits, one kernel forms
 * every giant step's accumulator (each baby-step key and diagonal read once)
 * and the giant steps t >= 1 run on the context's streams (as for
 * ckks_batch_streams: forked from and joined back to `stream` by events, or on
 * `stream` itself when another call holds them). */
int ckks_ptmatvecmult(ckks_ctx *ctx, const uint64_t *d_a, const uint64_t *d_b, int level, int nb, int ng,
                      const uint32_t *g_baby, const uint32_t *g_giant, const uint64_t *const *key_baby,
                      const uint64_t *const *key_giant, const uint64_t *const *d_diag, int rescale,
                      uint64_t *d_oa, uint64_t *d_ob, void *ws, ckks_stream_t stream);

/* Key generation (Eq. (kskShape), Sec. 2.4): writes d_key [dnum][2][L+k][N].
 * d_s: int64 [N] secret coefficients; d_e: int64 [dnum][N] error
 * coefficients; d_a: [dnum][L+k][N] uniform evaluation-form residues.
 * galois = 0 makes a relinearisation key (s' = s^2); otherwise s' = psi_g(s),
 * a rotation key for Rotate/HRotate with that g.  Workspace CKKS_OP_KEYGEN. */
int ckks_keygen_ksk(ckks_ctx *ctx, const int64_t *d_s, const int64_t *d_e, const uint64_t *d_a, uint32_t galois,
                    uint64_t *d_key, void *ws, ckks_stream_t stream);

/* Compressed keys (Sec. 5.3): the rows a_j of a key are uniformly random, so
 * they are regenerated from a 64-bit seed where they are used instead of being
 * stored and read; a compressed key is the rows b_j only, [dnum][L+k][N]
 * (half the bytes of a full key).  Element (j, l, n) of a_j is drawn from
 * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) seeded with `seed`: draws
 * 16e .. 16e+15 with e = (j*(L+k) + l)*N + n, the first whose top b bits
 * (b = bit length of the limb's prime q_l) are below q_l, else the last
 * one's top bits mod q_l.
 * ckks_keygen_ksk_seeded: as ckks_keygen_ksk with a_j from the seed; writes
 *   key_b [dnum][L+k][N].  Workspace CKKS_OP_KEYGEN_SEEDED.
 * ckks_ksk_expand: the full key [dnum][2][L+k][N] of a compressed key.
 * ckks_keyswitch_batch_seeded: ckks_keyswitch_batch with compressed keys
 *   keys_b[i] and seeds[i]; same bits as the full keys (ckks_ksk_expand). */
int ckks_keygen_ksk_seeded(ckks_ctx *ctx, const int64_t *d_s, const int64_t *d_e, uint64_t seed, uint32_t galois,
                           uint64_t *d_key_b, void *ws, ckks_stream_t stream);
int ckks_ksk_expand(ckks_ctx *ctx, const uint64_t *d_key_b, uint64_t seed, uint64_t *d_key, ckks_stream_t stream);
/* ckks_key_register_seed records in the context that d_key_b is a compressed
 * key with this seed; from then on every call of the context that takes a key
 * (ckks_keyswitch, ckks_rotate, ckks_hrotate, ckks_ksk_inner_prod,
 * ckks_ptmatvecmult, the batched calls, ckks_mult / ckks_newmult /
 * ckks_newmult_sum, ckks_server_add_key) treats that pointer as a compressed key
 * and regenerates its rows a_j on chip.  ckks_key_unregister forgets it.
 * Host-side only (no device work); not thread-safe against concurrent calls on
 * the same context.  The registry is keyed by address: memory freed while
 * registered and reused for another key would make that key read as
 * compressed, so unregister before freeing (the Python binding keeps a
 * registered tensor referenced until it is unregistered). */
int ckks_key_register_seed(ckks_ctx *ctx, const uint64_t *d_key_b, uint64_t seed);
int ckks_key_unregister(ckks_ctx *ctx, const uint64_t *d_key_b);
int ckks_keyswitch_batch_seeded(ckks_ctx *ctx, int n, const uint64_t *const *d_a, const uint64_t *const *d_b,
                                const int *levels, const uint32_t *galois, const uint64_t *const *d_keys_b,
                                const uint64_t *seeds, uint64_t *const *d_oa, uint64_t *const *d_ob, void *ws,
                                ckks_stream_t stream);

/* NTT autotuner (no counterpart in the paper).  Each NTT pass (the column
 * pass and the block pass of the two-pass transform) exists in three tile
 * shapes (CTA widths: the default, half, double), and each transform in three
 * radix splits (the block pass runs floor(logN/2) + split stages, the column
 * pass the rest; split -1, 0 or +1, the other shapes at split 0 only), for
 * logN >= 14 with primes below 2^57.  ckks_autotune times every width,
 * forward and inverse, on 24 limbs and on min(128, ws_bytes / (8N)) limbs of
 * the workspace (zeroed, then transformed in place); then, with the widths
 * chosen, every split of a whole forward and of a whole inverse transform.
 * It synchronises the stream and keeps the fastest width per pass and launch
 * size (<= 48 limbs, larger) and the fastest split per direction and launch
 * size in the context; the default width (split) is kept unless another is
 * faster by 0.5% (3%), since closer timings are within the spread of launches
 * timed alone.
 * choice (optional, 8 ints): [column pass small, column pass large, block pass
 * small, block pass large] with 0 = default, 1 = half width, 2 = double width,
 * then [forward small, forward large, inverse small, inverse large] splits in
 * {-1, 0, 1}.  times (optional, 24 floats): ms per forward+inverse pass for
 * [(pass * 2 + size class) * 3 + width], then ms per transform for
 * 12 + [(direction * 2 + size class) * 3 + split + 1].  ckks_tune_set applies
 * a saved choice (8 ints; EINVAL for a value out of range).  Results are
 * identical for every shape and split; only the speed changes.  Contexts
 * outside the tuned range keep the default (choice all 0). */
int ckks_autotune(ckks_ctx *ctx, void *ws, size_t ws_bytes, ckks_stream_t stream, int *choice, float *times);
int ckks_tune_set(ckks_ctx *ctx, const int *choice);

/* Fast basis conversion path (Algorithm 6 and the table "CKKS Subroutines"):
 * with every prime below 2^56 and at most 16 source limbs (max(alpha, k + 1)),
 * the conversions of ModUp, ModDown and Rescale run on the tensor cores
 * (tcgen05 f16 MMA on 8-bit pieces of the residues, exact f32 sums, one
 * modular reduction per output); otherwise, or after tensor_cores = 0, on the
 * integer units (32-bit split multiply-adds).  Both give the same residues
 * bit for bit.  *available (optional) = 1 when the tensor-core form exists
 * for this context.  Takes effect for later calls. */
int ckks_bconv_select(ckks_ctx *ctx, int tensor_cores, int *available);

/* The fused key-switching dataflow (Sec. 4.2 beta-limb caching with the
 * Sec. 4.4 re-ordering of ModDown): with on = 1, ckks_keyswitch, ckks_rotate
 * and a one-rotation ckks_hrotate run the last forward NTT pass of ModUp, the
 * KSKInnerProd (digits read through Automorph, keys streamed once per digit)
 * and the first inverse NTT pass of ModDown's special limbs in one kernel, so
 * the new ModUp limbs and the special limbs of (u, v) never reach HBM in
 * evaluation form (9 launches per HRotate instead of 11).  Same residues bit
 * for bit.  Off by default: on one GB300 the unfused kernels give more
 * throughput when many calls overlap on several streams, the fused one lower
 * latency for a call alone.  *available (optional) = 1 when the context's
 * primes and digit count allow it (every prime < 2^57, at most 4 digits at the
 * full level, N from 2^10 to 2^17); elsewhere the calls stay unfused.  Takes
 * effect for later calls. */
int ckks_fuse_select(ckks_ctx *ctx, int on, int *available);

/* Concurrency hint (no counterpart in the paper): the number of operations
 * the caller keeps running at once on this context (calls on that many
 * streams, say).  The tensor-core basis conversion sizes its grid for a 1/n
 * share of the SMs: fewer, longer CTAs per (group, chunk), which pay their
 * fixed cost (tensor-memory allocation, B image, pipeline fill) less often
 * while the other operations fill the SMs.  n = 1 (the default) sizes every
 * launch for the GPU alone, the lowest latency for one call; on one GB300 the
 * 8-stream HRotate step at N=2^16, ell=24 runs about 3% faster with n = 8
 * and a call alone about 20% slower.  Same residues bit for bit.  n: 1 .. 64,
 * CKKS_EINVAL outside.  Takes effect for later calls. */
int ckks_concurrency_hint(ckks_ctx *ctx, int n);

/* Streams of a batched call (no counterpart in the paper): the batched calls
 * (ckks_keyswitch_batch, ckks_mult_batch, ckks_newmult_batch, the serving
 * loop's batches) cut a batch of at least 4 * nstreams entries into nstreams
 * parts of about equal limb counts (ckks_hrotate_batch: its ciphertexts, each
 * with all its rotations, into parts of about equal rotation counts, at least
 * four rotations per part) and run them on the caller's stream and
 * nstreams - 1 streams of the
 * context, forked from and joined back to the caller's stream with events, so
 * that the parts' pipeline steps overlap (a transform of one part beside the
 * inner product of another).  The call stays asynchronous on the caller's
 * stream and can be captured in a CUDA graph.  nstreams: 1 .. 4 (default 2).
 * When another call holds the context's streams the batch runs unsplit.
 * Same residues bit for bit.  CKKS_EINVAL outside the range. */
int ckks_batch_streams(ckks_ctx *ctx, int nstreams);

/* ------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper; it serves the paper's operations).
 * A server owns one device arena for request workspace and nstreams CUDA
 * streams.  Requests (HRotate with one rotation, KeySwitch, or Mult with
 * relinearisation and Rescale) of any of the server's contexts (ring degrees)
 * and any level are queued by ckks_server_submit; their ciphertexts are
 * device buffers owned by the caller, which must keep them unchanged (inputs)
 * and unread (outputs) until the request is reported finished.
 * ckks_server_step retires finished batches and, for every free stream, forms
 * a batch at once (continuous batching): the oldest pending request picks the
 * context, then pending requests of that context join in arrival order, up to
 * max_batch, while device memory admits them:
 *   resident keys + sum over admitted requests (ciphertext bytes in and out +
 *   workspace) <= mem_budget,
 * where a key counts once, from ckks_server_add_key on.  A batch runs as one
 * launch per pipeline step (the batched calls above), so the bits of every
 * result are those of the single-ciphertext call.  ckks_server_poll returns
 * finished requests with latency = device completion time - arrival_ms (the
 * arrival time on the server's clock, ckks_server_now_ms; a negative
 * arrival_ms means "at submission").  Nothing blocks; the caller calls step
 * and poll in a loop.  Single-threaded: one thread at a time per server.
 * ckks_server_create allocates the arena (mem_budget bytes), one status word
 * per stream and its pinned host copy; it is the only call of this library
 * besides ckks_ctx_create that allocates device memory.
 * Errors: CKKS_EINVAL for bad arguments, CKKS_ENOMEM when a key or a request
 * can never fit the budget; after CKKS_ECUDA the server must be destroyed.
 * ------------------------------------------------------------------------ */
typedef struct ckks_server ckks_server;
enum { CKKS_REQ_HROTATE = 1, CKKS_REQ_MULT = 2, CKKS_REQ_KEYSWITCH = 3, CKKS_REQ_NEWMULT = 4 };
typedef struct {
    int op;                    /* CKKS_REQ_* */
    int ctx;                   /* index into the server's contexts */
    int level;                 /* ell of the inputs (>= 2 for Mult / NewMult) */
    const uint64_t *a, *b;     /* HRotate: (a, b); KeySwitch: a; (New)Mult: first ciphertext */
    const uint64_t *a2, *b2;   /* (New)Mult: second ciphertext */
    uint32_t galois;           /* HRotate: Galois element, odd, < 2N */
    int key;                   /* handle from ckks_server_add_key (same context) */
    uint64_t *oa, *ob;         /* outputs: [ell][N], (New)Mult [ell-1][N] */
    double arrival_ms;         /* on the server's clock; < 0: now */
} ckks_request;
typedef struct {
    int pending, in_flight, finished_unpolled, lanes_busy;
    size_t mem_budget, mem_keys, mem_in_flight;
    long long batches, requests_launched;
    int last_cuda_error;
} ckks_server_stats_t;
int ckks_server_create(ckks_ctx *const *ctxs, int nctx, size_t mem_budget, int max_batch, int nstreams,
                       ckks_server **out);
int ckks_server_destroy(ckks_server *srv);
int ckks_server_add_key(ckks_server *srv, int ctx, const uint64_t *d_key, int *handle);
/* A compressed key (rows b_j only, a_j from seed) counts half the bytes. */
int ckks_server_add_key_seeded(ckks_server *srv, int ctx, const uint64_t *d_key_b, uint64_t seed, int *handle);
double ckks_server_now_ms(const ckks_server *srv);
int ckks_server_submit(ckks_server *srv, const ckks_request *req, uint64_t *id);
int ckks_server_step(ckks_server *srv, int *n_launched);
/* Up to max finished requests: ids[i], latency_ms[i], done_ms[i] (device
 * completion time on the server's clock) and status[i]; any of the last three
 * arrays may be NULL; *n = count.  status[i] is CKKS_OK, or CKKS_ETIMEOUT when
 * a bounded device-side wait (see ckks_poll_status) ran out in the batch that
 * carried the request: its outputs are then not valid and it should be
 * resubmitted.  Each stream of the server has its own status word, so such a
 * failure is charged only to the requests of the batch that had it. */
int ckks_server_poll(ckks_server *srv, int max, uint64_t *ids, double *latency_ms, double *done_ms, int *status,
                     int *n);
/* Test hook (no counterpart in the paper): the next batch the server launches
 * first runs the bounded-wait self-test (ckks_selftest_bounded_wait, limit_us
 * 1 .. 2000000, else CKKS_EINVAL) on its stream, recording into that stream's
 * status word, so that every request of that batch is reported with
 * CKKS_ETIMEOUT.  Nothing faults; later batches run normally. */
int ckks_server_selftest_timeout(ckks_server *srv, uint32_t limit_us);
int ckks_server_stats(const ckks_server *srv, ckks_server_stats_t *stats);

/* Asynchronous errors: every call returns after enqueueing its kernels, so a
 * failure during execution (a CUDA error of an earlier launch) surfaces on a
 * later call or here.  ckks_poll_status does not block: it returns CKKS_OK
 * while the stream's work is pending or finished without error (*done, when
 * given, is 1 once everything enqueued on the stream has finished) and
 * CKKS_ECUDA with the CUDA error in ckks_last_cuda_error otherwise.  The one
 * device-side wait of this library, the tensor-core basis conversion waiting
 * for its own matrix multiplies (an mbarrier), gives up after a bounded number
 * of polls (about a second), skips its outputs and records the fact in the
 * context: once the stream's work has finished, ckks_poll_status returns
 * CKKS_ETIMEOUT for it (once; the record is cleared) and the outputs of that
 * work are not valid.  The record is one word per context, shared by its
 * streams: a timeout in work on another stream is reported by whichever poll
 * reads it first, and one raised between this call's read and its clear is
 * lost, so poll once more after synchronising every stream that uses the
 * context when a complete account is needed. */
int ckks_poll_status(ckks_ctx *ctx, ckks_stream_t stream, int *done);

/* Self-test of that bounded wait (no counterpart in the paper): launches one
 * CTA that waits on an mbarrier no thread arrives on.  The wait gives up after
 * limit_us microseconds (1 .. 2000000, else CKKS_EINVAL) and records the
 * timeout like the conversion does, so that the next ckks_poll_status on the
 * stream, once it has finished, returns CKKS_ETIMEOUT.  Nothing else in the
 * context is touched; later calls run normally. */
int ckks_selftest_bounded_wait(ckks_ctx *ctx, uint32_t limit_us, ckks_stream_t stream);

/* ------------------------------------------------------------------------
 * Measurement hook (no counterpart in the paper).  While enabled, every
 * kernel the context launches is bracketed by a pair of CUDA events recorded
 * on the launch stream, grouped by kernel class; ckks_profile_read()
 * synchronises those events and reports, per class, the summed device time,
 * the number of launches and the number of limbs (or limb-sized units) they
 * processed.  Enabling adds two event records per launch; disabled (the
 * default) it costs nothing.  Returns CKKS_EINVAL for an unknown class.
 * ------------------------------------------------------------------------ */
enum {
    CKKS_K_NTT_FWD = 0,   /* forward NTT passes (incl. the ModDown/Rescale epilogue) */
    CKKS_K_NTT_INV = 1,   /* inverse NTT passes */
    CKKS_K_BCONV = 2,     /* basis conversions of ModUp / ModDown / Rescale */
    CKKS_K_INNER = 3,     /* KSKInnerProd (with Automorph of the digits) */
    CKKS_K_PMV = 4,       /* PtMatVecMult inner loop */
    CKKS_K_ELEMWISE = 5,  /* Automorph, PModUp, key-generation element-wise kernels */
    CKKS_K_FUSED = 6,     /* fused ModUp tail: last forward NTT pass + KSKInnerProd (+ ModDown's first
                             inverse pass on the special positions) */
    CKKS_K_COUNT = 7
};
int ckks_profile_enable(ckks_ctx *ctx, int on);
int ckks_profile_reset(ckks_ctx *ctx);
int ckks_profile_read(ckks_ctx *ctx, int kclass, double *total_ms, long long *launches, double *units);

/* Measured ceiling of the transforms' butterfly rate (no counterpart in the
 * paper; the measurement behind the NTT's ALU roofline, Sec. 2.3's butterfly
 * with the Shoup product of Sec. 2.2).  Runs the forward lazy butterfly of
 * the transforms from registers only (16 words per thread, 4 stages per round,
 * no memory access in the loop) over every SM at the transforms' occupancy
 * (32 warps per SM) for `rounds` rounds (1 .. 2^24), timed with CUDA events on
 * `stream`; blocks until done.  *ms = the kernel's time, *butterflies = the
 * butterflies it ran.  sink: a device buffer of at least
 * ckks_butterfly_peak_sink_bytes bytes (16-byte aligned) that receives
 * meaningless words.  CKKS_EINVAL on bad arguments, CKKS_ECUDA on a CUDA error. */
int ckks_butterfly_peak_sink_bytes(const ckks_ctx *ctx, size_t *bytes);
int ckks_butterfly_peak(ckks_ctx *ctx, int rounds, void *sink, ckks_stream_t stream, float *ms, double *butterflies);

/* ------------------------------------------------------------------------
 * ModDown without a caller-supplied workspace (the paper has no counterpart;
 * this is a convenience of this library).
 *
 * ckks_moddown needs (k + ell) * N words of device workspace from the caller.
 * Some callers cannot provide it: code that runs inside a host framework which
 * owns all device memory and gives its plugins no allocator, services that
 * forbid device allocations after start-up, or callers that simply have no
 * cudaMalloc in reach.  This entry point computes exactly what ckks_moddown
 * computes (same arguments minus `ws`, bit-identical output) but takes its
 * scratch from a fixed array compiled into the library, so it allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *
 *  - Limit: the array holds 2^21 words (16 MiB), i.e. (k + ell) * N <= 2^21;
 *    N = 2^16 with ell + k <= 32 fits (e.g. ell = 24, k = 8).  Larger
 *    requests return CKKS_EUNSUPPORTED before anything is launched.
 *  - Every GPU that loads the library holds the 16 MiB array until the
 *    process exits.
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and caches it; make that first call before any
 *    stream capture.
 *  - All calls share the one array and it keeps the last call's contents.
 *    Every word a call reads there it has written first in the same call, so
 *    nothing needs clearing, but calls whose GPU work overlaps (different
 *    streams, or different host threads) race on the array and corrupt each
 *    other: order them on one stream or synchronise between them.
 * ------------------------------------------------------------------------ */
int ckks_moddown_noalloc(ckks_ctx *ctx, const uint64_t *d_in, int level, uint64_t *d_out, ckks_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CKKS_KS_H */
