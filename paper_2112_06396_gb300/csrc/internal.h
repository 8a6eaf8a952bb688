// internal.h -- the library context and the kernel launchers shared by the
// translation units (not part of the public C ABI).
#pragma once

#include <cstddef>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "common.cuh"

struct ckks_ctx {
    int device;
    int sms;                          // streaming multiprocessors of the device
    int logN, N, L, k, dnum, alpha;
    bool small_primes;                // every prime < 2^57: lazy NTT without conditional subtractions
    int split_bits;                   // W of the split basis conversion, 0 if primes are too large for it
    int tc_kg;                        // K groups of the tensor-core basis conversion, 0 if not available
    bool tc_on = true;                // use it when available (ckks_bconv_select can switch it off)
    bool tc_lazy;                     // its outputs stay below 8t without a final reduction
    bool fuse_on = false;             // single KeySwitch / one-rotation HRotate through modup_ip_kernel
    int concurrency = 1;              // operations the caller runs at once (ckks_concurrency_hint)
                                      // (ckks_fuse_select)
    // Batched calls split over `batch_split` streams: the caller's and
    // batch_split - 1 of these, forked and joined by events.  One call at a
    // time holds them (aux_mu); a call that finds them taken runs unsplit.
    static constexpr int kAux = 3;
    int batch_split = 2;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kAux] = {};
    std::mutex aux_mu;
    std::vector<u64> primes;          // L + k: q_0..q_{L-1}, p_0..p_{k-1}
    // device tables (one allocation)
    void *d_block;
    size_t table_bytes;
    ckks::PrimeInfo *d_pinfo;         // [L+k]
    ulonglong2 *d_tw_fwd;             // [L+k][N]: psi^brv(i) and Shoup companion
    ulonglong2 *d_tw_inv;             // [L+k][N]: psi^-brv(i) and Shoup companion
    ckks::BConvPlan *d_modup;         // [(L+1)*dnum]: plan (ell, digit j) at ell*dnum + j
    ckks::BConvPlan *d_moddown;       // [L+1]: P -> q_0..q_{ell-1} with rounding
    ckks::BConvPlan *d_rescale;       // [L+1]: q_{ell-1} -> q_0..q_{ell-2} with rounding
    ckks::BConvPlan *d_mdmerged;      // [L+1]: P*q_{ell-1} -> q_0..q_{ell-2} with rounding (NewMult)
    ulonglong2 *d_Pinv;               // [L+k]: [P^-1]_{q} (chain entries used)
    ulonglong2 *d_Pmod;               // [L+k]: [P]_{q}
    ulonglong2 *d_qlinv;              // [(L+1)*(L+k)]: [q_{ell-1}^-1]_{q_i} at ell*(L+k) + i
    ulonglong2 *d_Dinv;               // [(L+1)*(L+k)]: [(P q_{ell-1})^-1]_{q_i} at ell*(L+k) + i
    int last_cuda_error;
    int *d_status;                    // device word: bit 0 set when a kernel's bounded wait ran out
    uint4 *d_tc_img;                  // tensor-core operand images of every plan
    // NTT tile shape per pass (0 column, 1 block) and batch class (count <=
    // kTuneSmallBatch, larger): 0 default width, 1 half, 2 double (ntt_autotune)
    int ntt_csel[2][2] = {{0, 0}, {0, 0}};
    // NTT radix split per direction (0 forward, 1 inverse) and batch class:
    // pass C runs floor(logN/2) + split stages, split in {-1, 0, 1} (ntt_autotune)
    int ntt_split[2][2] = {{0, 0}, {0, 0}};
    // compressed keys registered with ckks_key_register_seed: device pointer of
    // the rows b_j -> seed of the rows a_j
    std::unordered_map<const u64 *, u64> comp_keys;
    // measurement hook (ckks_profile_*): event pairs around every launch
    struct ProfRec {
        cudaEvent_t a, b;
        int kclass;
        double units;
    };
    mutable bool prof_on = false;
    mutable std::vector<ProfRec> prof_pending;
    mutable std::vector<cudaEvent_t> prof_pool;
    mutable double prof_ms[8] = {};
    mutable long long prof_n[8] = {};
    mutable double prof_units[8] = {};  // indexed by kernel class (K_*, at most 8)
};

namespace ckks {

enum { K_NTT_FWD = 0, K_NTT_INV = 1, K_BCONV = 2, K_INNER = 3, K_PMV = 4, K_ELEMWISE = 5, K_FUSED = 6 };

// Brackets one launch with CUDA events when the context's measurement hook is on.
class ProfScope {
  public:
    ProfScope(const ckks_ctx *c, int kclass, double units, cudaStream_t st) : c_(c), st_(st) {
        if (!c_->prof_on) return;
        rec_.kclass = kclass;
        rec_.units = units;
        rec_.a = take();
        cudaEventRecord(rec_.a, st_);
    }
    ~ProfScope() {
        if (!c_->prof_on) return;
        rec_.b = take();
        cudaEventRecord(rec_.b, st_);
        c_->prof_pending.push_back(rec_);
    }

  private:
    cudaEvent_t take() {
        if (!c_->prof_pool.empty()) {
            cudaEvent_t e = c_->prof_pool.back();
            c_->prof_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    const ckks_ctx *c_;
    cudaStream_t st_;
    ckks_ctx::ProfRec rec_{};
};

inline int ext_prime(const ckks_ctx *c, int ell, int pos) { return pos < ell ? pos : c->L + (pos - ell); }
inline int beta_of(const ckks_ctx *c, int ell) { return (ell + c->alpha - 1) / c->alpha; }

cudaError_t ntt_set_attributes(const ckks_ctx *ctx);
cudaError_t launch_bounded_wait_selftest(const ckks_ctx *ctx, uint64_t limit_ns, cudaStream_t st,
                                         int *status = nullptr);
cudaError_t launch_ntt_fwd(const ckks_ctx *ctx, const NttBatch &b, const Epi *epi, cudaStream_t st);
cudaError_t launch_ntt_inv(const ckks_ctx *ctx, const NttBatch &b, cudaStream_t st);
cudaError_t launch_ntt_batch(const ckks_ctx *ctx, const KsBatchDesc &d, int phase, cudaStream_t st);
constexpr int kTuneSmallBatch = 48;
// Fused ModUp tail + KSKInnerProd (+ ModDown's first inverse pass on the
// special positions), modup_ip_kernel.
struct FusedIpArgs {
    const u64 *ext;   // [beta][ell+k][N]: the new ModUp limbs after pass S of the forward NTT
    const u64 *own;   // [ell][N] evaluation-form input: the digits' own limbs
    const u64 *key;   // [dnum][2][L+k][N], or the rows b_j only [dnum][L+k][N] when compressed
    u64 *u, *v;       // [ell+k][N]: chain positions in evaluation form; special positions after
                      // the first pass of the inverse NTT
    int ell;
    uint32_t galois;  // digits read through Automorph_galois (1: none)
    int compressed;
    u64 seed;
};
bool modup_ip_supported(const ckks_ctx *ctx, int ell);
cudaError_t launch_modup_ip(const ckks_ctx *ctx, const FusedIpArgs &f, cudaStream_t st);
cudaError_t launch_ntt_fwd_colpass(const ckks_ctx *ctx, const NttBatch &b, cudaStream_t st);
cudaError_t launch_ntt_inv_colpass(const ckks_ctx *ctx, const NttBatch &b, cudaStream_t st);
cudaError_t launch_bfly_peak(const ckks_ctx *ctx, int rounds, u64 *sink, cudaStream_t st, double *butterflies);
size_t bfly_peak_sink_words(const ckks_ctx *ctx);
cudaError_t ntt_autotune(ckks_ctx *ctx, u64 *scratch, int small, int large, cudaStream_t st, float *times_out);
cudaError_t launch_bconv(const ckks_ctx *ctx, const BConvLaunch &l, int max_src, cudaStream_t st);
cudaError_t launch_bconv_batch(const ckks_ctx *ctx, const KsBatchDesc &d, int down, cudaStream_t st,
                               int *status = nullptr);

// keyswitch.cu
struct InnerArgs {
    const u64 *ext;      // [beta][ell+k][N] ModUp outputs
    const u64 *own;      // [ell][N] evaluation-form input whose digit limbs stand in for ext (or null)
    const u64 *key;      // [dnum][2][L+k][N]
    u64 *u, *v;          // [ell+k][N]
    int ell;
    uint32_t galois;     // 1 = no automorphism
    const u64 *padd[2] = {nullptr, nullptr};  // optional [ell][N]: u += P*padd[0], v += P*padd[1] on the
                                               // chain positions (NewMult)
    int compressed = 0;  // key = rows b_j only [dnum][L+k][N]; a_j regenerated from seed
    u64 seed = 0;
};
cudaError_t launch_inner_prod(const ckks_ctx *ctx, const InnerArgs &a, cudaStream_t st);
// Batched KSKInnerProd with a compressed key: consecutive entries with one key,
// at most kIpGroup of them, share a CTA (entries start[g] .. start[g+1]-1 form
// group g).
constexpr int kIpGroup = kMaxCts;
struct IpGroups {
    int n;
    uint8_t start[kMaxCts + 1];
};
cudaError_t launch_inner_prod_batch(const ckks_ctx *ctx, const KsBatchDesc &d, cudaStream_t st);
cudaError_t launch_tensor(const ckks_ctx *ctx, const TensorBatch &T, cudaStream_t st);
cudaError_t launch_key_a_fill(const ckks_ctx *ctx, u64 seed, int j0, int ndig, u64 *dst, cudaStream_t st);
cudaError_t launch_sum_uv(const ckks_ctx *ctx, const KsBatchDesc &d, cudaStream_t st);

// ---- batch executor (abi.cu), shared with the serving loop (serve.cu)
enum { BE_KEYSWITCH = 0, BE_HROTATE = 1, BE_MULT = 2, BE_NEWMULT = 3 };
struct BatchEntry {
    int kind;
    const u64 *a, *b;    // KeySwitch: a; HRotate: (a, b); Mult: first ciphertext (a1, b1)
    const u64 *a2, *b2;  // Mult: second ciphertext
    const u64 *key;
    u64 *oa, *ob;        // outputs: [ell][N], Mult [ell-1][N]
    int ell;
    uint32_t galois;     // HRotate
    u64 *ws;             // this entry's workspace (entry_ws_words), or null: packed
    int compressed;      // key = b rows only [dnum][L+k][N], a regenerated from seed
    u64 seed;
};
size_t entry_ws_words(const ckks_ctx *c, int kind, int ell);
// status: the word a bounded device wait that runs out sets (the context's when null)
int run_batch(ckks_ctx *ctx, int n, const BatchEntry *e, u64 *w, cudaStream_t st, int *status = nullptr);

struct PmvArgs {
    const u64 *ext;      // hoisted ModUp outputs [beta][ell+k][N]
    const u64 *a, *b;    // input ciphertext [ell][N]
    u64 *acc_a, *acc_b;  // [ell+k][N]
    int ell, nb;
    uint32_t galois[kMaxRot];
    const u64 *key[kMaxRot];
    const u64 *diag[kMaxRot];
    u64 seed[kMaxRot];            // compressed keys: seed of the rows a_j
    uint8_t compressed[kMaxRot];  // key[i] holds the rows b_j only
};
cudaError_t launch_pmv_accum(const ckks_ctx *ctx, const PmvArgs &a, cudaStream_t st);

// Every giant step of Algorithm 8 in one launch (pmv_all_kernel): ng <= 8
// giant steps, nb * ng <= kMaxRot diagonals, beta <= 4.
constexpr int kMaxGiant = 8;
struct PmvAllArgs {
    const u64 *ext;               // hoisted ModUp outputs [beta][ell+k][N]
    const u64 *a, *b;             // input ciphertext [ell][N]
    u64 *acc_a[kMaxGiant], *acc_b[kMaxGiant];  // per giant step [ell+k][N]
    int ell, nb, ng;
    uint32_t galois[kMaxRot];
    const u64 *key[kMaxRot];
    const u64 *diag[kMaxRot];     // diagonal (t, i) at t*nb + i
    u64 seed[kMaxRot];
    uint8_t compressed[kMaxRot];
};
bool pmv_all_supported(const ckks_ctx *ctx, int ell, int nb, int ng);
// acc[p] += sum_j in[p][j] (mod each prime) over ell limbs, p = 0, 1
struct PolySum {
    u64 *acc[2];
    const u64 *in[2][kMaxGiant];
    int n;
};
cudaError_t launch_poly_sum(const ckks_ctx *ctx, const PolySum &S, int ell, cudaStream_t st);
cudaError_t launch_pmv_all(const ckks_ctx *ctx, const PmvAllArgs &a, cudaStream_t st);

cudaError_t launch_automorph(const ckks_ctx *ctx, const u64 *in, u64 *out, int nlimbs, uint32_t g, cudaStream_t st);
cudaError_t launch_pmodup(const ckks_ctx *ctx, const u64 *in, u64 *out, int ell, cudaStream_t st);
cudaError_t launch_signed_to_res(const ckks_ctx *ctx, const int64_t *c, u64 *out, cudaStream_t st);
cudaError_t launch_square(const ckks_ctx *ctx, const u64 *in, u64 *out, cudaStream_t st);
cudaError_t launch_keygen_row(const ckks_ctx *ctx, const u64 *a, const u64 *s, const u64 *sp, const u64 *e, int j,
                              u64 *row0, u64 *row1, cudaStream_t st);

}  // namespace ckks
