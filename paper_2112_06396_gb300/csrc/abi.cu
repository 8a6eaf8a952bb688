// abi.cu -- the C ABI (include/ckks_ks.h): context construction (host-side
// constant tables, uploaded once) and the orchestration of the key-switching
// operations as sequences of kernel launches on the caller's stream.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/ckks_ks.h"
#include "common.cuh"
#include "internal.h"

#include <nvtx3/nvToolsExt.h>

using namespace ckks;

typedef unsigned __int128 u128;

// ------------------------------------------------------------------ host arithmetic
static u64 hmul(u64 a, u64 b, u64 m) { return u64((u128)a * b % m); }
static u64 hpow(u64 a, u64 e, u64 m) {
    u64 r = 1 % m;
    a %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = hmul(r, a, m);
        a = hmul(a, a, m);
    }
    return r;
}
static u64 hinv(u64 a, u64 p) { return hpow(a % p, p - 2, p); }  // p prime (Fermat)
static u64 shoup_of(u64 w, u64 p) { return u64(((u128)w << 64) / p); }

// Miller-Rabin with the seven bases of Sinclair (deterministic below 2^64).
static bool strong_probable_prime(u64 n, u64 a) {
    a %= n;
    if (a == 0) return true;
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++s;
    }
    u64 x = hpow(a, d, n);
    if (x == 1 || x == n - 1) return true;
    for (int r = 1; r < s; ++r) {
        x = hmul(x, x, n);
        if (x == n - 1) return true;
    }
    return false;
}
static bool is_prime_u64(u64 n) {
    if (n < 2) return false;
    for (u64 sp : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull}) {
        if (n % sp == 0) return n == sp;
    }
    for (u64 a : {2ull, 325ull, 9375ull, 28178ull, 450775ull, 9780504ull, 1795265022ull})
        if (!strong_probable_prime(n, a)) return false;
    return true;
}

// Smallest primitive 2N-th root of unity mod q.
static u64 min_root(u64 q, int logN) {
    const u64 N = u64(1) << logN;
    u64 g = 0;
    for (u64 x = 2;; ++x) {
        u64 c = hpow(x, (q - 1) >> (logN + 1), q);
        if (hpow(c, N, q) == q - 1) {
            g = c;
            break;
        }
    }
    u64 best = g, cur = g;
    const u64 g2 = hmul(g, g, q);
    for (u64 i = 1; i < N; ++i) {
        cur = hmul(cur, g2, q);
        best = std::min(best, cur);
    }
    return best;
}

static uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

extern "C" const char *ckks_strerror(int s) {
    switch (s) {
    case CKKS_OK: return "ok";
    case CKKS_EINVAL: return "invalid argument";
    case CKKS_ENOMEM: return "out of device memory";
    case CKKS_ECUDA: return "CUDA error (see ckks_last_cuda_error)";
    case CKKS_EUNSUPPORTED: return "unsupported parameters";
    case CKKS_ETIMEOUT: return "a bounded device-side wait ran out";
    default: return "unknown status";
    }
}

extern "C" int ckks_gen_primes(int bits, int logN, int count, uint64_t *out) {
    if (bits < 20 || bits > 60 || logN < 1 || logN > 20 || count < 0 || (count > 0 && out == nullptr))
        return CKKS_EINVAL;
    const u64 step = u64(2) << logN;
    u64 q = ((u64(1) << bits) - 2) / step * step + 1;  // largest 1 + m*2N below 2^bits
    int got = 0;
    for (; got < count && q > step; q -= step)
        if (is_prime_u64(q)) out[got++] = q;
    return got == count ? CKKS_OK : CKKS_EINVAL;
}

// ------------------------------------------------------------------ context
static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

static void fill_plan(BConvPlan &pl) { std::memset(&pl, 0, sizeof(pl)); }

extern "C" int ckks_ctx_create(const ckks_params *prm, int device, ckks_ctx **out) {
    if (prm == nullptr || out == nullptr || prm->q == nullptr || prm->p == nullptr) return CKKS_EINVAL;
    const int logN = prm->logN, L = prm->L, k = prm->k, dnum = prm->dnum;
    if (logN < 10 || logN > 17 || L < 1 || L > 64 || k < 1 || k > kMaxSrc || L + k > kMaxLimbs || dnum < 1 ||
        dnum > L)
        return CKKS_EINVAL;
    const int alpha = (L + dnum - 1) / dnum;
    if (alpha > kMaxSrc) return CKKS_EUNSUPPORTED;
    const u64 N = u64(1) << logN;
    std::vector<u64> primes(prm->q, prm->q + L);
    primes.insert(primes.end(), prm->p, prm->p + k);
    for (size_t i = 0; i < primes.size(); ++i) {
        const u64 q = primes[i];
        if (q >= (u64(1) << 60) || q % (2 * N) != 1 || !is_prime_u64(q)) return CKKS_EINVAL;
        for (size_t j = 0; j < i; ++j)
            if (primes[j] == q) return CKKS_EINVAL;
    }
    ckks_ctx *c = new (std::nothrow) ckks_ctx();
    if (!c) return CKKS_ENOMEM;
    c->device = device;
    c->logN = logN;
    c->N = int(N);
    c->L = L;
    c->k = k;
    c->dnum = dnum;
    c->alpha = alpha;
    c->primes = primes;
    c->last_cuda_error = 0;
    c->small_primes = *std::max_element(primes.begin(), primes.end()) < (u64(1) << 57);
    {
        int maxbits = 0;
        for (u64 q : primes) maxbits = std::max(maxbits, 64 - __builtin_clzll(q));
        const int W = (maxbits + 1) / 2;
        // sources in [0, 3q) split at W bits give products below 2^(2W+2); 2*kMaxSrc
        // of them must sum below 2^62, so W <= 27 (primes of at most 54 bits)
        c->split_bits = W <= 27 ? W : 0;
    }
    const int LK = L + k;

    // ---- host tables
    std::vector<PrimeInfo> pinfo(LK);
    std::vector<ulonglong2> twf(size_t(LK) * N), twi(size_t(LK) * N);
    for (int e = 0; e < LK; ++e) {
        const u64 q = primes[e];
        const u64 psi = min_root(q, logN), ipsi = hinv(psi, q);
        std::vector<u64> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (u64 i = 1; i < N; ++i) {
            pw[i] = hmul(pw[i - 1], psi, q);
            ipw[i] = hmul(ipw[i - 1], ipsi, q);
        }
        for (u64 i = 0; i < N; ++i) {
            const u64 w = pw[bitrev(uint32_t(i), logN)], iw = ipw[bitrev(uint32_t(i), logN)];
            twf[size_t(e) * N + i] = make_ulonglong2(w, shoup_of(w, q));
            twi[size_t(e) * N + i] = make_ulonglong2(iw, shoup_of(iw, q));
        }
        PrimeInfo &P = pinfo[e];
        P.p = q;
        P.r64 = u64(((u128)1 << 64) % q);
        P.r64_s = shoup_of(P.r64, q);
        P.one_s = shoup_of(1, q);
        P.ninv = hinv(N % q, q);
        P.ninv_s = shoup_of(P.ninv, q);
        P.ninv_w = hmul(P.ninv, twi[size_t(e) * N + 1].x, q);
        P.ninv_w_s = shoup_of(P.ninv_w, q);
    }
    auto prod_mod = [&](int lo, int hi, int skip, u64 m) {
        u64 r = 1 % m;
        for (int i = lo; i < hi; ++i)
            if (i != skip) r = hmul(r, primes[i] % m, m);
        return r;
    };
    auto ext_p = [&](int ell, int t) { return t < ell ? t : L + (t - ell); };

    // ModUp plans (ell, j)
    std::vector<BConvPlan> modup(size_t(L + 1) * dnum);
    for (auto &pl : modup) fill_plan(pl);
    for (int ell = 1; ell <= L; ++ell) {
        const int beta = (ell + alpha - 1) / alpha;
        for (int j = 0; j < beta; ++j) {
            BConvPlan &pl = modup[size_t(ell) * dnum + j];
            const int lo = j * alpha, hi = std::min(lo + alpha, ell);
            pl.n_src = hi - lo;
            for (int i = 0; i < pl.n_src; ++i) {
                const u64 qi = primes[lo + i];
                pl.src_prime[i] = uint16_t(lo + i);
                pl.src_add[i] = 0;
                pl.src_mul[i] = hinv(prod_mod(lo, hi, lo + i, qi), qi);
                pl.src_mul_s[i] = shoup_of(pl.src_mul[i], qi);
            }
            int d = 0;
            for (int t = 0; t < ell + k; ++t) {
                if (t >= lo && t < hi) continue;
                const int pe = ext_p(ell, t);
                pl.dst_pos[d] = uint16_t(t);
                pl.dst_prime[d] = uint16_t(pe);
                pl.dst_sub[d] = 0;
                for (int i = 0; i < pl.n_src; ++i) pl.mat[d][i] = prod_mod(lo, hi, lo + i, primes[pe]);
                ++d;
            }
            pl.n_dst = d;
        }
    }
    // ModDown plans: P -> q_0..q_{ell-1}, with the rounding constant H = floor(P/2) = (P-1)/2
    auto halfP = [&](u64 m) { return hmul((prod_mod(L, L + k, -1, m) + m - 1) % m, hinv(2, m), m); };
    std::vector<BConvPlan> mdown(L + 1), resc(L + 1);
    for (auto &pl : mdown) fill_plan(pl);
    for (auto &pl : resc) fill_plan(pl);
    for (int ell = 1; ell <= L; ++ell) {
        BConvPlan &pl = mdown[ell];
        pl.n_src = k;
        for (int m = 0; m < k; ++m) {
            const u64 pm = primes[L + m];
            pl.src_prime[m] = uint16_t(L + m);
            pl.src_add[m] = halfP(pm);
            pl.src_mul[m] = hinv(prod_mod(L, L + k, L + m, pm), pm);
            pl.src_mul_s[m] = shoup_of(pl.src_mul[m], pm);
        }
        pl.n_dst = ell;
        for (int t = 0; t < ell; ++t) {
            pl.dst_pos[t] = uint16_t(t);
            pl.dst_prime[t] = uint16_t(t);
            pl.dst_sub[t] = halfP(primes[t]);
            for (int m = 0; m < k; ++m) pl.mat[t][m] = prod_mod(L, L + k, L + m, primes[t]);
        }
        if (ell >= 2) {
            BConvPlan &rs = resc[ell];
            const u64 ql = primes[ell - 1], h = ql / 2;
            rs.n_src = 1;
            rs.src_prime[0] = uint16_t(ell - 1);
            rs.src_add[0] = h;
            rs.src_mul[0] = 1;
            rs.src_mul_s[0] = shoup_of(1, ql);
            rs.n_dst = ell - 1;
            for (int t = 0; t < ell - 1; ++t) {
                rs.dst_pos[t] = uint16_t(t);
                rs.dst_prime[t] = uint16_t(t);
                rs.dst_sub[t] = h % primes[t];
                rs.mat[t][0] = 1;
            }
        }
    }
    // merged ModDown of NewMult: D = P * q_{ell-1} (sources p_0..p_{k-1} and
    // q_{ell-1}) -> q_0..q_{ell-2}, rounding constant floor(D/2) = (D-1)/2
    std::vector<BConvPlan> mdrs(L + 1);
    for (auto &pl : mdrs) fill_plan(pl);
    auto D_mod = [&](int ell, u64 m) { return hmul(prod_mod(L, L + k, -1, m), primes[ell - 1] % m, m); };
    auto halfD = [&](int ell, u64 m) { return hmul((D_mod(ell, m) + m - 1) % m, hinv(2, m), m); };
    auto Dhat_mod = [&](int ell, int src, u64 m) {  // (D / d_src) mod m; src k is q_{ell-1}
        if (src == k) return prod_mod(L, L + k, -1, m);
        return hmul(prod_mod(L, L + k, L + src, m), primes[ell - 1] % m, m);
    };
    if (k + 1 <= kMaxSrc) {
        for (int ell = 2; ell <= L; ++ell) {
            BConvPlan &pl = mdrs[ell];
            pl.n_src = k + 1;
            for (int m = 0; m <= k; ++m) {
                const int pe = m < k ? L + m : ell - 1;
                const u64 dm = primes[pe];
                pl.src_prime[m] = uint16_t(pe);
                pl.src_add[m] = halfD(ell, dm);
                pl.src_mul[m] = hinv(Dhat_mod(ell, m, dm), dm);
                pl.src_mul_s[m] = shoup_of(pl.src_mul[m], dm);
            }
            pl.n_dst = ell - 1;
            for (int t = 0; t < ell - 1; ++t) {
                pl.dst_pos[t] = uint16_t(t);
                pl.dst_prime[t] = uint16_t(t);
                pl.dst_sub[t] = halfD(ell, primes[t]);
                for (int m = 0; m <= k; ++m) pl.mat[t][m] = Dhat_mod(ell, m, primes[t]);
            }
        }
    }
    // split form of every plan's matrix for the 32-bit multiply-add basis conversion
    if (c->split_bits) {
        const int W = c->split_bits;
        const u64 mask = (u64(1) << W) - 1;
        auto split = [&](BConvPlan &pl) {
            for (int d = 0; d < pl.n_dst; ++d) {
                const u64 t = primes[pl.dst_prime[d]];
                for (int i = 0; i < pl.n_src; ++i) {
                    const u64 C = pl.mat[d][i], D = hmul(C, u64((u128(1) << W) % t), t);
                    pl.matw[d][i] = make_uint4(uint32_t(D >> W), uint32_t(C >> W), uint32_t(D & mask), uint32_t(C & mask));
                }
                pl.dst_rw[d] = u64(((u128)1 << W) % t);
                pl.dst_rw_s[d] = shoup_of(pl.dst_rw[d], t);
            }
        };
        for (auto &pl : modup) split(pl);
        for (auto &pl : mdown) split(pl);
        for (auto &pl : resc) split(pl);
        for (auto &pl : mdrs) split(pl);
    }
    // tensor-core form of every plan (basis.cu, bconv_tc_kernel): 7-byte
    // residues (primes below 2^56) and at most 16 sources keep every f32 sum
    // of byte products below 2^23
    {
        const u64 maxp = *std::max_element(primes.begin(), primes.end());
        const int nsrc = std::max(alpha, k + 1);
        c->tc_kg = (c->split_bits && maxp < (u64(1) << 56) && nsrc <= 16) ? ((nsrc + 2) & ~1) : 0;
    }
    std::vector<uint16_t> tc_img;  // f16 bit patterns
    std::vector<size_t> tc_off[4];
    if (c->tc_kg) {
        const int KG = c->tc_kg;
        auto f16 = [](unsigned v) -> uint16_t {  // exact below 2048 and for powers of two up to 2^15
            if (v == 0) return 0;
            const int e = 31 - __builtin_clz(v);
            const unsigned mant = e <= 10 ? (v << (10 - e)) : (v >> (e - 10));
            return uint16_t(((e + 15) << 10) | (mant & 0x3FFu));
        };
        // the epilogue's sum lo = sum_{c<5} 2^(8c) S_c + fold (< 2t) + off (< t)
        // stays below 8t, the lazy forward NTT's input bound, when lo < 5t for
        // the smallest prime; otherwise the epilogue reduces once more
        {
            const u128 smax = u128(std::max(alpha, k + 1)) * 7 * 255 * 255;
            const u128 lo_max = smax * (u128(1) + (1u << 8) + (1u << 16) + (1u << 24) + (u128(1) << 32));
            const u64 tmin = *std::min_element(primes.begin(), primes.end());
            c->tc_lazy = lo_max < u128(5) * tmin;
        }
        auto prep = [&](BConvPlan &pl) -> size_t {
            const size_t off0 = tc_img.size() / 8;  // in 16-byte units
            const int ntp = (pl.n_dst + 3) & ~3;
            tc_img.resize(tc_img.size() + size_t(ntp) * KG * 64, 0);
            uint16_t *base = tc_img.data() + off0 * 8;
            for (int d = 0; d < ntp; ++d) {
                uint16_t *blk = base + size_t(d) * KG * 64;
                for (int r = 0; r < 8; ++r) blk[(KG - 1) * 64 + r * 8] = f16(4096);
                if (d >= pl.n_dst) continue;
                const u64 t = primes[pl.dst_prime[d]];
                for (int i = 0; i < pl.n_src; ++i)
                    for (int j = 0; j < 7; ++j) {
                        const u64 mj = hmul(pl.mat[d][i] % t, u64(((u128)1 << (8 * j)) % t), t);
                        for (int r = 0; r < 7; ++r) blk[i * 64 + r * 8 + j] = f16(unsigned(mj >> (8 * r)) & 0xFFu);
                    }
                pl.dst_r40[d] = u64(((u128)1 << 40) % t);
                pl.dst_r40_s[d] = shoup_of(pl.dst_r40[d], t);
                pl.dst_off[d] = (t - pl.dst_sub[d] % t) % t;
            }
            return off0;
        };
        std::vector<BConvPlan> *kinds[4] = {&modup, &mdown, &resc, &mdrs};
        for (int kd = 0; kd < 4; ++kd)
            for (auto &pl : *kinds[kd]) tc_off[kd].push_back(prep(pl));
    }
    std::vector<ulonglong2> Pinv(LK), Pmod(LK), qlinv(size_t(L + 1) * LK);
    for (int i = 0; i < LK; ++i) {
        const u64 q = primes[i];
        const u64 pm = prod_mod(L, L + k, -1, q);
        Pmod[i] = make_ulonglong2(pm, shoup_of(pm, q));
        const u64 pinv = pm == 0 ? 0 : hinv(pm, q);
        Pinv[i] = make_ulonglong2(pinv, shoup_of(pinv, q));
    }
    std::vector<ulonglong2> Dinv(size_t(L + 1) * LK);
    for (int ell = 2; ell <= L; ++ell)
        for (int i = 0; i < ell - 1; ++i) {
            const u64 q = primes[i], v = hinv(primes[ell - 1] % q, q);
            qlinv[size_t(ell) * LK + i] = make_ulonglong2(v, shoup_of(v, q));
            const u64 dv = hinv(D_mod(ell, q), q);
            Dinv[size_t(ell) * LK + i] = make_ulonglong2(dv, shoup_of(dv, q));
        }

    // ---- one device allocation
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t o_pinfo = take(sizeof(PrimeInfo) * LK);
    const size_t o_twf = take(sizeof(ulonglong2) * twf.size());
    const size_t o_twi = take(sizeof(ulonglong2) * twi.size());
    const size_t o_modup = take(sizeof(BConvPlan) * modup.size());
    const size_t o_mdown = take(sizeof(BConvPlan) * mdown.size());
    const size_t o_resc = take(sizeof(BConvPlan) * resc.size());
    const size_t o_pinv = take(sizeof(ulonglong2) * LK);
    const size_t o_pmod = take(sizeof(ulonglong2) * LK);
    const size_t o_qlinv = take(sizeof(ulonglong2) * qlinv.size());
    const size_t o_mdrs = take(sizeof(BConvPlan) * mdrs.size());
    const size_t o_dinv = take(sizeof(ulonglong2) * Dinv.size());
    const size_t o_tcimg = take(sizeof(uint16_t) * tc_img.size());
    const size_t o_status = take(sizeof(int));
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t err = cudaSetDevice(device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (err == cudaSuccess) err = cudaMalloc(&c->d_block, off);
    if (err != cudaSuccess) {
        cudaGetLastError();  // not sticky: leave no error behind for the caller
        const cudaError_t back = cudaSetDevice(prev);
        delete c;
        if (back != cudaSuccess) return CKKS_ECUDA;  // the caller's device could not be restored
        return err == cudaErrorMemoryAllocation ? CKKS_ENOMEM : CKKS_ECUDA;
    }
    char *base = static_cast<char *>(c->d_block);
    c->table_bytes = off;
    c->d_pinfo = reinterpret_cast<PrimeInfo *>(base + o_pinfo);
    c->d_tw_fwd = reinterpret_cast<ulonglong2 *>(base + o_twf);
    c->d_tw_inv = reinterpret_cast<ulonglong2 *>(base + o_twi);
    c->d_modup = reinterpret_cast<BConvPlan *>(base + o_modup);
    c->d_moddown = reinterpret_cast<BConvPlan *>(base + o_mdown);
    c->d_rescale = reinterpret_cast<BConvPlan *>(base + o_resc);
    c->d_Pinv = reinterpret_cast<ulonglong2 *>(base + o_pinv);
    c->d_Pmod = reinterpret_cast<ulonglong2 *>(base + o_pmod);
    c->d_qlinv = reinterpret_cast<ulonglong2 *>(base + o_qlinv);
    c->d_mdmerged = reinterpret_cast<BConvPlan *>(base + o_mdrs);
    c->d_Dinv = reinterpret_cast<ulonglong2 *>(base + o_dinv);
    c->d_tc_img = reinterpret_cast<uint4 *>(base + o_tcimg);
    c->d_status = reinterpret_cast<int *>(base + o_status);
    if (c->tc_kg) {
        std::vector<BConvPlan> *kinds[4] = {&modup, &mdown, &resc, &mdrs};
        for (int kd = 0; kd < 4; ++kd)
            for (size_t i = 0; i < kinds[kd]->size(); ++i) (*kinds[kd])[i].tc_img = c->d_tc_img + tc_off[kd][i];
    }
    struct Up {
        void *dst;
        const void *src;
        size_t n;
    } ups[] = {{c->d_pinfo, pinfo.data(), sizeof(PrimeInfo) * LK},
               {c->d_tw_fwd, twf.data(), sizeof(ulonglong2) * twf.size()},
               {c->d_tw_inv, twi.data(), sizeof(ulonglong2) * twi.size()},
               {c->d_modup, modup.data(), sizeof(BConvPlan) * modup.size()},
               {c->d_moddown, mdown.data(), sizeof(BConvPlan) * mdown.size()},
               {c->d_rescale, resc.data(), sizeof(BConvPlan) * resc.size()},
               {c->d_Pinv, Pinv.data(), sizeof(ulonglong2) * LK},
               {c->d_Pmod, Pmod.data(), sizeof(ulonglong2) * LK},
               {c->d_qlinv, qlinv.data(), sizeof(ulonglong2) * qlinv.size()},
               {c->d_mdmerged, mdrs.data(), sizeof(BConvPlan) * mdrs.size()},
               {c->d_Dinv, Dinv.data(), sizeof(ulonglong2) * Dinv.size()},
               {c->d_tc_img, tc_img.data(), sizeof(uint16_t) * tc_img.size()}};
    for (auto &u : ups)
        if (err == cudaSuccess && u.n) err = cudaMemcpy(u.dst, u.src, u.n, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(c->d_status, 0, sizeof(int));
    if (err == cudaSuccess) err = ntt_set_attributes(c);
    for (int i = 0; i < ckks_ctx::kAux && err == cudaSuccess; ++i) {
        err = cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming);
    }
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
    // the caller's current device is restored; a failure to do so fails the call
    const cudaError_t back = cudaSetDevice(prev);
    if (err == cudaSuccess) err = back;
    if (err != cudaSuccess) {
        for (int i = 0; i < ckks_ctx::kAux; ++i) {
            if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
            if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
        }
        if (c->fork_ev) cudaEventDestroy(c->fork_ev);
        cudaFree(c->d_block);
        delete c;
        return CKKS_ECUDA;
    }
    *out = c;
    return CKKS_OK;
}

extern "C" int ckks_ctx_destroy(ckks_ctx *c) {
    if (c == nullptr) return CKKS_EINVAL;
    int prev = 0;
    cudaError_t err = cudaGetDevice(&prev);
    if (err == cudaSuccess) err = cudaSetDevice(c->device);
    for (auto &r : c->prof_pending) {
        cudaEventSynchronize(r.b);
        c->prof_pool.push_back(r.a);
        c->prof_pool.push_back(r.b);
    }
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    for (int i = 0; i < ckks_ctx::kAux; ++i) {
        if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
        if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    cudaFree(c->d_block);  // a device pointer is freed whichever device is current
    const cudaError_t back = cudaSetDevice(prev);
    if (err == cudaSuccess) err = back;
    delete c;
    return err == cudaSuccess ? CKKS_OK : CKKS_ECUDA;
}

extern "C" int ckks_last_cuda_error(const ckks_ctx *c) { return c ? c->last_cuda_error : 0; }
extern "C" size_t ckks_ctx_table_bytes(const ckks_ctx *c) { return c ? c->table_bytes : 0; }

// ------------------------------------------------------------------ helpers
#define CK(call)                                                                                                  \
    do {                                                                                                          \
        cudaError_t e_ = (call);                                                                                  \
        if (e_ != cudaSuccess) {                                                                                  \
            ctx->last_cuda_error = int(e_);                                                                       \
            return CKKS_ECUDA;                                                                                    \
        }                                                                                                         \
    } while (0)
#define RC(call)                                                                                                  \
    do {                                                                                                          \
        int r_ = (call);                                                                                          \
        if (r_ != CKKS_OK) return r_;                                                                             \
    } while (0)

// An NVTX range per C-ABI operation (visible in Nsight timelines; a no-op when
// no tool is attached).
struct OpRange {
    explicit OpRange(const char *name) { nvtxRangePushA(name); }
    ~OpRange() { nvtxRangePop(); }
    OpRange(const OpRange &) = delete;
    OpRange &operator=(const OpRange &) = delete;
};

static bool al16(const void *p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
static bool level_ok(const ckks_ctx *c, int ell) { return c != nullptr && ell >= 1 && ell <= c->L; }
static bool galois_ok(const ckks_ctx *c, uint32_t g) { return (g & 1u) && g < uint32_t(2 * c->N); }
// A key pointer registered with ckks_key_register_seed is a compressed key.
static bool key_seed(const ckks_ctx *c, const u64 *key, u64 *seed) {
    const auto it = c->comp_keys.find(key);
    if (it == c->comp_keys.end()) return false;
    *seed = it->second;
    return true;
}

// Launch forward (or inverse) NTTs over a list of limbs, in chunks of kMaxBatch.
struct LimbList {
    std::vector<const u64 *> src;
    std::vector<u64 *> dst;
    std::vector<uint16_t> prime;
    void add(const u64 *s, u64 *d, int p) {
        src.push_back(s);
        dst.push_back(d);
        prime.push_back(uint16_t(p));
    }
};
// lazy: forward transforms stored without their final reduction (EPI_LAZY).
static int run_ntt(ckks_ctx *ctx, const LimbList &ll, bool inverse, cudaStream_t st, bool lazy = false) {
    const size_t n = ll.src.size();
    Epi lz{};
    lz.mode = EPI_LAZY;
    for (size_t b0 = 0; b0 < n; b0 += kMaxBatch) {
        NttBatch b;
        b.count = int(std::min(n - b0, size_t(kMaxBatch)));
        for (int l = 0; l < b.count; ++l) {
            b.src[l] = ll.src[b0 + l];
            b.dst[l] = ll.dst[b0 + l];
            b.prime[l] = ll.prime[b0 + l];
        }
        CK(inverse ? launch_ntt_inv(ctx, b, st) : launch_ntt_fwd(ctx, b, lazy ? &lz : nullptr, st));
    }
    return CKKS_OK;
}

static size_t words_modup_all(const ckks_ctx *c, int ell) {
    return size_t(beta_of(c, ell)) * (ell + c->k) + size_t(ell);
}
static size_t words_moddown2(const ckks_ctx *c, int ell) { return size_t(2) * c->k + size_t(2) * ell; }

// ModUp of every digit of a (Algorithm 6 per digit): iNTT -> BConv -> NTT.
// ext: [beta][ell+k][N] (digit limbs are not written); acoeff: [ell][N] scratch.
// The new limbs are left lazy (below 2^64, see EPI_LAZY): every caller feeds
// them only to inner products with exact 128-bit sums.
static int modup_all(ckks_ctx *ctx, const u64 *a, int ell, u64 *ext, u64 *acoeff, cudaStream_t st) {
    const size_t N = ctx->N;
    const int k = ctx->k, beta = beta_of(ctx, ell), ext_n = ell + k;
    LimbList inv;
    for (int i = 0; i < ell; ++i) inv.add(a + i * N, acoeff + i * N, i);
    RC(run_ntt(ctx, inv, true, st));
    for (int j0 = 0; j0 < beta; j0 += kMaxGroups) {
        BConvLaunch l{};
        l.ngroups = std::min(beta - j0, kMaxGroups);
        // targets per digit: every position outside the digit (the smallest,
        // last digit has the most)
        l.chunk = ext_n - std::min(ctx->alpha, ell - (beta - 1) * ctx->alpha);
        l.chunks = 1;
        for (int g = 0; g < l.ngroups; ++g) {
            const int j = j0 + g;
            l.g[g].plan = ctx->d_modup + size_t(ell) * ctx->dnum + j;
            l.g[g].src = acoeff + size_t(j) * ctx->alpha * N;
            l.g[g].dst = ext + size_t(j) * ext_n * N;
        }
        CK(launch_bconv(ctx, l, std::min(ctx->alpha, ell), st));
    }
    // position-major order: the new limbs of one prime (one per digit) are
    // adjacent, so the CTAs transforming them run together and share twiddles
    LimbList fw;
    for (int t = 0; t < ext_n; ++t)
        for (int j = 0; j < beta; ++j) {
            const int lo = j * ctx->alpha, hi = std::min(lo + ctx->alpha, ell);
            if (t >= lo && t < hi) continue;
            u64 *p = ext + (size_t(j) * ext_n + t) * N;
            fw.add(p, p, ext_prime(ctx, ell, t));
        }
    return run_ntt(ctx, fw, false, st, true);
}

// ModDown of npolys extended polynomials in[p] ([ell+k][N]) to out[p] ([ell][N]):
// iNTT of the k P-limbs -> BConv P -> q with rounding -> NTT with the
// (x - w) * P^-1 epilogue; add[p] (read through Automorph_g) and accumulation
// are folded into the epilogue.  Scratch: pcoeff [npolys*k][N], w [npolys*ell][N].
// p_half: the P-limbs of in[p] already went through the first pass of the
// inverse NTT (the fused ModUp tail wrote them so): the second pass runs in
// place on them, they are the conversion's sources, and pcoeff is not used.
static int moddown_polys(ckks_ctx *ctx, int ell, int npolys, const u64 *const in[2], u64 *const out[2],
                         const u64 *const add[2], uint32_t g, int accumulate, u64 *pcoeff, u64 *w, cudaStream_t st,
                         bool p_half = false) {
    const size_t N = ctx->N;
    const int k = ctx->k;
    const u64 *csrc[2] = {nullptr, nullptr};
    if (p_half) {
        NttBatch b;
        b.count = 0;
        for (int m = 0; m < k; ++m)
            for (int p = 0; p < npolys; ++p) {
                u64 *limb = const_cast<u64 *>(in[p]) + size_t(ell + m) * N;
                b.src[b.count] = limb;
                b.dst[b.count] = limb;
                b.prime[b.count++] = uint16_t(ctx->L + m);
            }
        CK(launch_ntt_inv_colpass(ctx, b, st));
        for (int p = 0; p < npolys; ++p) csrc[p] = in[p] + size_t(ell) * N;
    } else {
        LimbList inv;  // prime-major: both polynomials' limbs of one prime are adjacent
        for (int m = 0; m < k; ++m)
            for (int p = 0; p < npolys; ++p)
                inv.add(in[p] + size_t(ell + m) * N, pcoeff + size_t(p * k + m) * N, ctx->L + m);
        RC(run_ntt(ctx, inv, true, st));
        for (int p = 0; p < npolys; ++p) csrc[p] = pcoeff + size_t(p) * k * N;
    }
    BConvLaunch l{};
    l.ngroups = npolys;
    l.chunk = ell;
    l.chunks = 1;
    for (int p = 0; p < npolys; ++p) {
        l.g[p].plan = ctx->d_moddown + ell;
        l.g[p].src = csrc[p];
        l.g[p].dst = w + size_t(p) * ell * N;
    }
    CK(launch_bconv(ctx, l, k, st));
    NttBatch b;
    b.count = npolys * ell;
    for (int t = 0; t < ell; ++t)
        for (int p = 0; p < npolys; ++p) {
            u64 *q = w + (size_t(p) * ell + t) * N;
            b.src[t * npolys + p] = q;
            b.dst[t * npolys + p] = q;
            b.prime[t * npolys + p] = uint16_t(t);
        }
    Epi e{};
    e.mode = EPI_SCALE;
    e.npolys = npolys;
    for (int p = 0; p < 2; ++p) {
        e.x[p] = p < npolys ? in[p] : nullptr;
        e.out[p] = p < npolys ? out[p] : nullptr;
        e.add[p] = p < npolys ? add[p] : nullptr;
    }
    e.galois = g;
    e.accumulate = accumulate;
    e.cmul = ctx->d_Pinv;
    CK(launch_ntt_fwd(ctx, b, &e, st));
    return CKKS_OK;
}

// Rescale of npolys polynomials in[p] ([ell][N]) to out[p] ([ell-1][N]).
// Scratch: c [npolys][N], w [npolys*(ell-1)][N].
static int rescale_polys(ckks_ctx *ctx, int ell, int npolys, const u64 *const in[2], u64 *const out[2], u64 *c,
                         u64 *w, cudaStream_t st) {
    const size_t N = ctx->N;
    LimbList inv;
    for (int p = 0; p < npolys; ++p) inv.add(in[p] + size_t(ell - 1) * N, c + size_t(p) * N, ell - 1);
    RC(run_ntt(ctx, inv, true, st));
    BConvLaunch l{};
    l.ngroups = npolys;
    l.chunk = ell - 1;
    l.chunks = 1;
    for (int p = 0; p < npolys; ++p) {
        l.g[p].plan = ctx->d_rescale + ell;
        l.g[p].src = c + size_t(p) * N;
        l.g[p].dst = w + size_t(p) * (ell - 1) * N;
    }
    CK(launch_bconv(ctx, l, 1, st));
    NttBatch b;
    b.count = npolys * (ell - 1);
    for (int t = 0; t < ell - 1; ++t)
        for (int p = 0; p < npolys; ++p) {
            u64 *q = w + (size_t(p) * (ell - 1) + t) * N;
            b.src[t * npolys + p] = q;
            b.dst[t * npolys + p] = q;
            b.prime[t * npolys + p] = uint16_t(t);
        }
    Epi e{};
    e.mode = EPI_SCALE;
    e.npolys = npolys;
    for (int p = 0; p < 2; ++p) {
        e.x[p] = p < npolys ? in[p] : nullptr;
        e.out[p] = p < npolys ? out[p] : nullptr;
        e.add[p] = nullptr;
    }
    e.galois = 1;
    e.accumulate = 0;
    e.cmul = ctx->d_qlinv + size_t(ell) * (ctx->L + ctx->k);
    CK(launch_ntt_fwd(ctx, b, &e, st));
    return CKKS_OK;
}

// The merged ModDown of NewMult (Algorithm 7) over npolys extended polynomials
// in[p] ([ell+k][N]) to out[p] ([ell-1][N]): iNTT of the k P-limbs and of the
// q_{ell-1} limb -> basis conversion from D = P*q_{ell-1} to q_0..q_{ell-2}
// with rounding -> NTT with the (x - w) * D^-1 epilogue.
// Scratch: pcoeff [npolys*(k+1)][N], w [npolys*(ell-1)][N].
static int moddown_merged_polys(ckks_ctx *ctx, int ell, int npolys, const u64 *const in[2], u64 *const out[2],
                                u64 *pcoeff, u64 *w, cudaStream_t st) {
    const size_t N = ctx->N;
    const int k = ctx->k, ns = k + 1, nd = ell - 1;
    LimbList inv;  // prime-major: both polynomials' limbs of one prime are adjacent
    for (int m = 0; m < ns; ++m)
        for (int p = 0; p < npolys; ++p) {
            const int pos = m < k ? ell + m : ell - 1;
            inv.add(in[p] + size_t(pos) * N, pcoeff + size_t(p * ns + m) * N, m < k ? ctx->L + m : ell - 1);
        }
    RC(run_ntt(ctx, inv, true, st));
    BConvLaunch l{};
    l.ngroups = npolys;
    l.chunk = nd;
    l.chunks = 1;
    for (int p = 0; p < npolys; ++p) {
        l.g[p].plan = ctx->d_mdmerged + ell;
        l.g[p].src = pcoeff + size_t(p) * ns * N;
        l.g[p].dst = w + size_t(p) * nd * N;
    }
    CK(launch_bconv(ctx, l, ns, st));
    NttBatch b;
    b.count = npolys * nd;
    for (int t = 0; t < nd; ++t)
        for (int p = 0; p < npolys; ++p) {
            u64 *q = w + (size_t(p) * nd + t) * N;
            b.src[t * npolys + p] = q;
            b.dst[t * npolys + p] = q;
            b.prime[t * npolys + p] = uint16_t(t);
        }
    Epi e{};
    e.mode = EPI_SCALE;
    e.npolys = npolys;
    for (int p = 0; p < 2; ++p) {
        e.x[p] = p < npolys ? in[p] : nullptr;
        e.out[p] = p < npolys ? out[p] : nullptr;
        e.add[p] = nullptr;
    }
    e.galois = 1;
    e.accumulate = 0;
    e.cmul = ctx->d_Dinv + size_t(ell) * (ctx->L + ctx->k);
    CK(launch_ntt_fwd(ctx, b, &e, st));
    return CKKS_OK;
}

// ---- workspace layouts (in words)
struct KsLayout {
    size_t uv, ext, acoeff, pcoeff, w, total;
};
static KsLayout ks_layout(const ckks_ctx *c, int ell) {
    const size_t N = c->N;
    KsLayout o;
    const size_t uvw = size_t(2) * (ell + c->k);
    const size_t r1 = std::max(words_modup_all(c, ell), words_moddown2(c, ell));
    o.uv = 0;
    o.ext = uvw * N;
    o.acoeff = o.ext + size_t(beta_of(c, ell)) * (ell + c->k) * N;
    o.pcoeff = o.ext;                        // aliases ext: used after the inner product
    o.w = o.pcoeff + size_t(2) * c->k * N;
    o.total = (uvw + r1) * N;
    return o;
}

// ModUp of every digit with the fused tail: iNTT -> conversion -> pass S of the
// new limbs' forward NTT -> modup_ip_kernel (pass C, KSKInnerProd with the
// digits read through Automorph_g, and the first inverse pass of ModDown on the
// special positions of u and v).  ext: [beta][ell+k][N] and acoeff: [ell][N]
// scratch; u, v: [ell+k][N] (special positions half inverse-transformed, for
// moddown_polys with p_half).
static int modup_ip_fused(ckks_ctx *ctx, const u64 *a, int ell, const u64 *key, uint32_t g, u64 *ext, u64 *acoeff,
                          u64 *u, u64 *v, cudaStream_t st) {
    const size_t N = ctx->N;
    const int k = ctx->k, beta = beta_of(ctx, ell), ext_n = ell + k;
    LimbList inv;
    for (int i = 0; i < ell; ++i) inv.add(a + i * N, acoeff + i * N, i);
    RC(run_ntt(ctx, inv, true, st));
    for (int j0 = 0; j0 < beta; j0 += kMaxGroups) {
        BConvLaunch l{};
        l.ngroups = std::min(beta - j0, kMaxGroups);
        l.chunk = ext_n - std::min(ctx->alpha, ell - (beta - 1) * ctx->alpha);
        l.chunks = 1;
        for (int gi = 0; gi < l.ngroups; ++gi) {
            const int j = j0 + gi;
            l.g[gi].plan = ctx->d_modup + size_t(ell) * ctx->dnum + j;
            l.g[gi].src = acoeff + size_t(j) * ctx->alpha * N;
            l.g[gi].dst = ext + size_t(j) * ext_n * N;
        }
        CK(launch_bconv(ctx, l, std::min(ctx->alpha, ell), st));
    }
    NttBatch b;
    b.count = 0;
    for (int t = 0; t < ext_n; ++t)
        for (int j = 0; j < beta; ++j) {
            const int lo = j * ctx->alpha, hi = std::min(lo + ctx->alpha, ell);
            if (t >= lo && t < hi) continue;
            if (b.count == kMaxBatch) {
                CK(launch_ntt_fwd_colpass(ctx, b, st));
                b.count = 0;
            }
            u64 *p = ext + (size_t(j) * ext_n + t) * N;
            b.src[b.count] = p;
            b.dst[b.count] = p;
            b.prime[b.count++] = uint16_t(ext_prime(ctx, ell, t));
        }
    CK(launch_ntt_fwd_colpass(ctx, b, st));
    FusedIpArgs f{ext, a, key, u, v, ell, g, 0, 0};
    f.compressed = key_seed(ctx, key, &f.seed);
    CK(launch_modup_ip(ctx, f, st));
    return CKKS_OK;
}

// KeySwitch core: ModUp(a), inner product (digits through Automorph_gin), ModDown.
static int keyswitch_core(ckks_ctx *ctx, const u64 *a, int ell, const u64 *key, uint32_t gin, u64 *out0, u64 *out1,
                          const u64 *add1, uint32_t gadd, int accumulate, u64 *ws, cudaStream_t st) {
    const size_t N = ctx->N;
    const KsLayout lo = ks_layout(ctx, ell);
    u64 *u = ws + lo.uv, *v = u + size_t(ell + ctx->k) * N;
    if (ctx->fuse_on && modup_ip_supported(ctx, ell)) {
        RC(modup_ip_fused(ctx, a, ell, key, gin, ws + lo.ext, ws + lo.acoeff, u, v, st));
        const u64 *in[2] = {u, v};
        u64 *out[2] = {out0, out1};
        const u64 *add[2] = {nullptr, add1};
        return moddown_polys(ctx, ell, 2, in, out, add, gadd, accumulate, ws + lo.pcoeff, ws + lo.w, st, true);
    }
    RC(modup_all(ctx, a, ell, ws + lo.ext, ws + lo.acoeff, st));
    InnerArgs ia{ws + lo.ext, a, key, u, v, ell, gin};
    ia.compressed = key_seed(ctx, key, &ia.seed);
    CK(launch_inner_prod(ctx, ia, st));
    const u64 *in[2] = {u, v};
    u64 *out[2] = {out0, out1};
    const u64 *add[2] = {nullptr, add1};
    return moddown_polys(ctx, ell, 2, in, out, add, gadd, accumulate, ws + lo.pcoeff, ws + lo.w, st);
}

static size_t words_rotate(const ckks_ctx *c, int ell) { return size_t(2) * ell * c->N + ks_layout(c, ell).total; }

// Algorithm 3 with the outputs optionally accumulated into (oa, ob).
static int rotate_core(ckks_ctx *ctx, const u64 *a, const u64 *b, int ell, uint32_t g, const u64 *key, u64 *oa,
                       u64 *ob, int accumulate, u64 *ws, cudaStream_t st) {
    const size_t N = ctx->N;
    u64 *ar = ws, *br = ws + size_t(ell) * N;
    CK(launch_automorph(ctx, a, ar, ell, g, st));
    CK(launch_automorph(ctx, b, br, ell, g, st));
    return keyswitch_core(ctx, ar, ell, key, 1, oa, ob, br, 1, accumulate, ws + size_t(2) * ell * N, st);
}

struct HrLayout {
    size_t ext, uv, tmp, total;
};
static HrLayout hr_layout(const ckks_ctx *c, int ell) {
    const size_t N = c->N;
    HrLayout o;
    o.ext = 0;
    o.uv = size_t(beta_of(c, ell)) * (ell + c->k) * N;
    o.tmp = o.uv + size_t(2) * (ell + c->k) * N;
    o.total = o.tmp + std::max(size_t(ell), words_moddown2(c, ell)) * N;
    return o;
}

struct PmvLayout {
    size_t ext, acc, tmp, ct, res, rot, chain, chain_words, total;
};
// acc holds one (a, b) accumulator pair per giant step when every giant step
// runs in one launch (pmv_all_kernel), else one pair reused per giant step.
static PmvLayout pmv_layout(const ckks_ctx *c, int ell, int ng) {
    const size_t N = c->N;
    PmvLayout o;
    o.ext = 0;
    o.acc = size_t(beta_of(c, ell)) * (ell + c->k) * N;
    const int nacc = ng >= 1 && ng <= kMaxGiant && beta_of(c, ell) <= 4 ? ng : 1;
    o.tmp = o.acc + size_t(2) * nacc * (ell + c->k) * N;
    o.ct = o.tmp + std::max(size_t(ell), words_moddown2(c, ell)) * N;
    o.res = o.ct + size_t(2) * ell * N;
    o.rot = o.res + size_t(2) * ell * N;
    o.total = o.rot + (ng > 1 ? words_rotate(c, ell) : 0);
    // every giant step t >= 1 of the one-launch path has its own ModDown scratch,
    // rotated input, rotated output and Rotate workspace, so the giant steps can
    // run on separate streams
    o.chain = o.total;
    o.chain_words = (std::max(size_t(ell), words_moddown2(c, ell)) + size_t(4) * ell) * N + words_rotate(c, ell);
    if (nacc > 1) o.total = o.chain + size_t(ng - 1) * o.chain_words;
    return o;
}

extern "C" int ckks_workspace_bytes(const ckks_ctx *c, int op, int ell, int r, size_t *bytes) {
    if (c == nullptr || bytes == nullptr || !level_ok(c, ell)) return CKKS_EINVAL;
    const size_t N = c->N;
    size_t w = 0;
    switch (op) {
    case CKKS_OP_MODUP: w = size_t(c->alpha) * N; break;
    case CKKS_OP_MODDOWN: w = size_t(c->k + ell) * N; break;
    case CKKS_OP_KEYSWITCH: w = ks_layout(c, ell).total; break;
    case CKKS_OP_ROTATE: w = words_rotate(c, ell); break;
    case CKKS_OP_HROTATE: w = hr_layout(c, ell).total; break;
    case CKKS_OP_RESCALE:
        if (ell < 2) return CKKS_EINVAL;
        w = size_t(ell) * N;
        break;
    case CKKS_OP_PTMATVEC:
        if (r < 1) return CKKS_EINVAL;
        w = pmv_layout(c, ell, r).total;
        break;
    case CKKS_OP_KEYGEN: w = size_t(3) * (c->L + c->k) * N; break;
    case CKKS_OP_MULT:
        if (ell < 2) return CKKS_EINVAL;
        w = hr_layout(c, ell).total + size_t(5) * ell * N;
        break;
    case CKKS_OP_NEWMULT:
        if (ell < 2) return CKKS_EINVAL;
        w = hr_layout(c, ell).total + size_t(3) * ell * N;
        break;
    case CKKS_OP_KEYGEN_SEEDED: w = size_t(4) * (c->L + c->k) * N; break;
    default: return CKKS_EINVAL;
    }
    *bytes = w * sizeof(u64);
    return CKKS_OK;
}

// ------------------------------------------------------------------ API
extern "C" int ckks_ntt(ckks_ctx *ctx, uint64_t *d, int ell, int first, int count, ckks_stream_t stream) {
    OpRange r_("ckks_ntt");
    if (!level_ok(ctx, ell) || !al16(d) || first < 0 || count < 0 || first + count > ell + ctx->k) return CKKS_EINVAL;
    LimbList ll;
    for (int t = first; t < first + count; ++t) ll.add(d + size_t(t) * ctx->N, d + size_t(t) * ctx->N, ext_prime(ctx, ell, t));
    return run_ntt(ctx, ll, false, (cudaStream_t)stream);
}

extern "C" int ckks_intt(ckks_ctx *ctx, uint64_t *d, int ell, int first, int count, ckks_stream_t stream) {
    OpRange r_("ckks_intt");
    if (!level_ok(ctx, ell) || !al16(d) || first < 0 || count < 0 || first + count > ell + ctx->k) return CKKS_EINVAL;
    LimbList ll;
    for (int t = first; t < first + count; ++t) ll.add(d + size_t(t) * ctx->N, d + size_t(t) * ctx->N, ext_prime(ctx, ell, t));
    return run_ntt(ctx, ll, true, (cudaStream_t)stream);
}

extern "C" int ckks_automorph(ckks_ctx *ctx, const uint64_t *in, uint64_t *out, int nlimbs, uint32_t g,
                              ckks_stream_t stream) {
    OpRange r_("ckks_automorph");
    if (ctx == nullptr || !al16(in) || !al16(out) || in == out || nlimbs < 0 || nlimbs > 65535 || !galois_ok(ctx, g))
        return CKKS_EINVAL;
    CK(launch_automorph(ctx, in, out, nlimbs, g, (cudaStream_t)stream));
    return CKKS_OK;
}

extern "C" int ckks_modup(ckks_ctx *ctx, const uint64_t *a, int ell, int digit, uint64_t *out, void *ws,
                          ckks_stream_t stream) {
    OpRange r_("ckks_modup");
    if (!level_ok(ctx, ell) || !al16(a) || !al16(out) || !al16(ws) || digit < 0 || digit >= beta_of(ctx, ell))
        return CKKS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = ctx->N;
    const int lo = digit * ctx->alpha, hi = std::min(lo + ctx->alpha, ell), ext_n = ell + ctx->k;
    u64 *acoeff = static_cast<u64 *>(ws);
    LimbList inv;
    for (int i = lo; i < hi; ++i) inv.add(a + i * N, acoeff + (i - lo) * N, i);
    RC(run_ntt(ctx, inv, true, st));
    BConvLaunch l{};
    l.ngroups = 1;
    l.chunk = ext_n - (hi - lo);
    l.chunks = 1;
    l.g[0].plan = ctx->d_modup + size_t(ell) * ctx->dnum + digit;
    l.g[0].src = acoeff;
    l.g[0].dst = out;
    CK(launch_bconv(ctx, l, hi - lo, st));
    LimbList fw;
    for (int t = 0; t < ext_n; ++t)
        if (t < lo || t >= hi) fw.add(out + t * N, out + t * N, ext_prime(ctx, ell, t));
    RC(run_ntt(ctx, fw, false, st));
    CK(cudaMemcpyAsync(out + lo * N, a + lo * N, size_t(hi - lo) * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    return CKKS_OK;
}

extern "C" int ckks_ksk_inner_prod(ckks_ctx *ctx, const uint64_t *digits, int ell, const uint64_t *key, uint64_t *u,
                                   uint64_t *v, ckks_stream_t stream) {
    OpRange r_("ckks_ksk_inner_prod");
    if (!level_ok(ctx, ell) || !al16(digits) || !al16(key) || !al16(u) || !al16(v)) return CKKS_EINVAL;
    InnerArgs ia{digits, nullptr, key, u, v, ell, 1};
    ia.compressed = key_seed(ctx, key, &ia.seed);
    CK(launch_inner_prod(ctx, ia, (cudaStream_t)stream));
    return CKKS_OK;
}

extern "C" int ckks_moddown(ckks_ctx *ctx, const uint64_t *in, int ell, uint64_t *out, void *ws,
                            ckks_stream_t stream) {
    OpRange r_("ckks_moddown");
    if (!level_ok(ctx, ell) || !al16(in) || !al16(out) || !al16(ws)) return CKKS_EINVAL;
    u64 *w = static_cast<u64 *>(ws);
    const u64 *ins[2] = {in, nullptr};
    u64 *outs[2] = {out, nullptr};
    const u64 *adds[2] = {nullptr, nullptr};
    return moddown_polys(ctx, ell, 1, ins, outs, adds, 1, 0, w, w + size_t(ctx->k) * ctx->N, (cudaStream_t)stream);
}

extern "C" int ckks_pmodup(ckks_ctx *ctx, const uint64_t *in, int ell, uint64_t *out, ckks_stream_t stream) {
    OpRange r_("ckks_pmodup");
    if (!level_ok(ctx, ell) || !al16(in) || !al16(out)) return CKKS_EINVAL;
    CK(launch_pmodup(ctx, in, out, ell, (cudaStream_t)stream));
    return CKKS_OK;
}

extern "C" int ckks_rescale(ckks_ctx *ctx, const uint64_t *in, int ell, uint64_t *out, void *ws,
                            ckks_stream_t stream) {
    OpRange r_("ckks_rescale");
    if (!level_ok(ctx, ell) || ell < 2 || !al16(in) || !al16(out) || !al16(ws)) return CKKS_EINVAL;
    u64 *w = static_cast<u64 *>(ws);
    const u64 *ins[2] = {in, nullptr};
    u64 *outs[2] = {out, nullptr};
    return rescale_polys(ctx, ell, 1, ins, outs, w, w + ctx->N, (cudaStream_t)stream);
}

extern "C" int ckks_keyswitch(ckks_ctx *ctx, const uint64_t *a, int ell, const uint64_t *key, uint64_t *u,
                              uint64_t *v, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_keyswitch");
    if (!level_ok(ctx, ell) || !al16(a) || !al16(key) || !al16(u) || !al16(v) || !al16(ws)) return CKKS_EINVAL;
    return keyswitch_core(ctx, a, ell, key, 1, u, v, nullptr, 1, 0, static_cast<u64 *>(ws), (cudaStream_t)stream);
}

extern "C" int ckks_rotate(ckks_ctx *ctx, const uint64_t *a, const uint64_t *b, int ell, uint32_t g,
                           const uint64_t *key, uint64_t *oa, uint64_t *ob, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_rotate");
    if (!level_ok(ctx, ell) || !al16(a) || !al16(b) || !al16(key) || !al16(oa) || !al16(ob) || !al16(ws) ||
        !galois_ok(ctx, g))
        return CKKS_EINVAL;
    return rotate_core(ctx, a, b, ell, g, key, oa, ob, 0, static_cast<u64 *>(ws), (cudaStream_t)stream);
}

extern "C" int ckks_hrotate(ckks_ctx *ctx, const uint64_t *a, const uint64_t *b, int ell, int r,
                            const uint32_t *galois, const uint64_t *const *keys, uint64_t *const *oa,
                            uint64_t *const *ob, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_hrotate");
    if (!level_ok(ctx, ell) || !al16(a) || !al16(b) || !al16(ws) || r < 0 || (r > 0 && (!galois || !keys || !oa || !ob)))
        return CKKS_EINVAL;
    for (int i = 0; i < r; ++i)
        if (!galois_ok(ctx, galois[i]) || !al16(keys[i]) || !al16(oa[i]) || !al16(ob[i])) return CKKS_EINVAL;
    if (r == 0) return CKKS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = ctx->N;
    u64 *w = static_cast<u64 *>(ws);
    const HrLayout lo = hr_layout(ctx, ell);
    u64 *u = w + lo.uv, *v = u + size_t(ell + ctx->k) * N;
    if (r == 1 && ctx->fuse_on && modup_ip_supported(ctx, ell)) {
        // one rotation: the ModUp tail, the inner product and ModDown's first
        // inverse pass in one kernel (several rotations share the transformed
        // digits instead)
        RC(modup_ip_fused(ctx, a, ell, keys[0], galois[0], w + lo.ext, w + lo.tmp, u, v, st));
        const u64 *in[2] = {u, v};
        u64 *out[2] = {oa[0], ob[0]};
        const u64 *add[2] = {nullptr, b};
        return moddown_polys(ctx, ell, 2, in, out, add, galois[0], 0, w + lo.tmp, w + lo.tmp + size_t(2) * ctx->k * N,
                             st, true);
    }
    RC(modup_all(ctx, a, ell, w + lo.ext, w + lo.tmp, st));
    for (int i = 0; i < r; ++i) {
        InnerArgs ia{w + lo.ext, a, keys[i], u, v, ell, galois[i]};
        ia.compressed = key_seed(ctx, keys[i], &ia.seed);
        CK(launch_inner_prod(ctx, ia, st));
        const u64 *in[2] = {u, v};
        u64 *out[2] = {oa[i], ob[i]};
        const u64 *add[2] = {nullptr, b};
        RC(moddown_polys(ctx, ell, 2, in, out, add, galois[i], 0, w + lo.tmp, w + lo.tmp + size_t(2) * ctx->k * N, st));
    }
    return CKKS_OK;
}

// ---- batched key switching and Mult
// Per-entry workspace: the HRotate layout of its level, then for Mult entries
// a3, b3, c3 and the key switch's outputs (a', b') before the Rescale.
size_t ckks::entry_ws_words(const ckks_ctx *c, int kind, int ell) {
    const size_t extra = kind == BE_MULT ? 5 : kind == BE_NEWMULT ? 3 : 0;
    return hr_layout(c, ell).total + extra * ell * c->N;
}

static size_t batch_ws_words(const ckks_ctx *c, int n, const int *levels, int kind) {
    size_t w = 0;
    for (int i = 0; i < n; ++i) w += entry_ws_words(c, kind, levels[i]);
    return w;
}

extern "C" int ckks_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, size_t *bytes) {
    if (ctx == nullptr || bytes == nullptr || n < 0 || (n > 0 && levels == nullptr)) return CKKS_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!level_ok(ctx, levels[i])) return CKKS_EINVAL;
    *bytes = batch_ws_words(ctx, n, levels, BE_HROTATE) * sizeof(u64);
    return CKKS_OK;
}

extern "C" int ckks_mult_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, size_t *bytes) {
    if (ctx == nullptr || bytes == nullptr || n < 0 || (n > 0 && levels == nullptr)) return CKKS_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!level_ok(ctx, levels[i]) || levels[i] < 2) return CKKS_EINVAL;
    *bytes = batch_ws_words(ctx, n, levels, BE_MULT) * sizeof(u64);
    return CKKS_OK;
}

// The device descriptor of one entry; ws is the entry's workspace.
static CtDesc entry_desc(const ckks_ctx *ctx, const BatchEntry &e, u64 *ws, TensorEntry *te) {
    const size_t N = ctx->N, lN = size_t(e.ell) * N;
    CtDesc x{};
    x.key = e.key;
    x.ws = ws;
    x.ell = e.ell;
    x.galois = 1;
    x.compressed = e.compressed;
    x.seed = e.seed;
    if (e.kind == BE_NEWMULT) {
        u64 *m = ws + hr_layout(ctx, e.ell).total;
        *te = TensorEntry{e.a, e.b, e.a2, e.b2, m, m + lN, m + 2 * lN, e.ell};
        x.a = m;
        x.add[0] = m + lN;
        x.add[1] = m + 2 * lN;
        x.oa = e.oa;
        x.ob = e.ob;
        x.merged = 1;
    } else if (e.kind == BE_MULT) {
        u64 *m = ws + hr_layout(ctx, e.ell).total;
        *te = TensorEntry{e.a, e.b, e.a2, e.b2, m, m + lN, m + 2 * lN, e.ell};
        x.a = m;
        x.add[0] = m + lN;
        x.add[1] = m + 2 * lN;
        x.oa = m + 3 * lN;
        x.ob = m + 4 * lN;
        x.ra = e.oa;
        x.rb = e.ob;
    } else {
        x.a = e.a;
        x.oa = e.oa;
        x.ob = e.ob;
        if (e.kind == BE_HROTATE) {
            x.add[1] = e.b;
            x.galois = e.galois;
        }
    }
    return x;
}

// One entry on its own, with the single-operation launches (contexts whose
// primes are too wide for the split basis conversion).
static int entry_one(ckks_ctx *ctx, const CtDesc &c, const TensorEntry *te, cudaStream_t st) {
    const size_t N = ctx->N;
    if (te != nullptr) {
        TensorBatch T;
        T.n = 1;
        T.logN = ctx->logN;
        T.e[0] = *te;
        CK(launch_tensor(ctx, T, st));
    }
    const HrLayout lo = hr_layout(ctx, c.ell);
    RC(modup_all(ctx, c.a, c.ell, c.ws + lo.ext, c.ws + lo.tmp, st));
    u64 *u = c.ws + lo.uv, *v = u + size_t(c.ell + ctx->k) * N;
    InnerArgs ia{c.ws + lo.ext, c.a, c.key, u, v, c.ell, c.galois, {nullptr, nullptr}, c.compressed, c.seed};
    if (c.merged) {
        ia.padd[0] = c.add[0];
        ia.padd[1] = c.add[1];
    }
    CK(launch_inner_prod(ctx, ia, st));
    if (c.merged) {
        const u64 *in[2] = {u, v};
        u64 *out[2] = {c.oa, c.ob};
        return moddown_merged_polys(ctx, c.ell, 2, in, out, c.ws + lo.tmp,
                                    c.ws + lo.tmp + size_t(2) * (ctx->k + 1) * N, st);
    }
    const u64 *in[2] = {u, v};
    u64 *out[2] = {c.oa, c.ob};
    const u64 *add[2] = {c.add[0], c.add[1]};
    RC(moddown_polys(ctx, c.ell, 2, in, out, add, c.galois, 0, c.ws + lo.tmp, c.ws + lo.tmp + size_t(2) * ctx->k * N,
                     st));
    if (c.ra != nullptr) {
        const u64 *rin[2] = {c.oa, c.ob};
        u64 *rout[2] = {c.ra, c.rb};
        RC(rescale_polys(ctx, c.ell, 2, rin, rout, c.ws, c.ws + 2 * N, st));
    }
    return CKKS_OK;
}

// The steps of a batch up to the inner product: tensor step of the Mult
// entries, iNTT of the inputs, ModUp conversion, NTT of the new limbs, KSKInnerProd.
static int batch_front(ckks_ctx *ctx, const KsBatchDesc &d, const TensorBatch &T, cudaStream_t st,
                       int *status = nullptr) {
    CK(launch_tensor(ctx, T, st));
    CK(launch_ntt_batch(ctx, d, PH_INTT_A, st));
    CK(launch_bconv_batch(ctx, d, GM_MODUP, st, status));
    CK(launch_ntt_batch(ctx, d, PH_NTT_UP, st));
    CK(launch_inner_prod_batch(ctx, d, st));
    return CKKS_OK;
}

// The ModDown steps (and the Rescale of Mult entries).
static int batch_back(ckks_ctx *ctx, const KsBatchDesc &d, bool rescale, cudaStream_t st, int *status = nullptr) {
    CK(launch_ntt_batch(ctx, d, PH_INTT_P, st));
    CK(launch_bconv_batch(ctx, d, GM_MODDOWN, st, status));
    CK(launch_ntt_batch(ctx, d, PH_NTT_DOWN, st));
    if (rescale) {
        CK(launch_ntt_batch(ctx, d, PH_RS_INTT, st));
        CK(launch_bconv_batch(ctx, d, GM_RESCALE, st, status));
        CK(launch_ntt_batch(ctx, d, PH_RS_NTT, st));
    }
    return CKKS_OK;
}

static int run_batch_on(ckks_ctx *ctx, int n, const BatchEntry *e, u64 *w, cudaStream_t st, int *status);

// Runs a batch.  An entry's workspace is its ws when set, else the next
// entry_ws_words region of w (batch order).  With ctx->batch_split > 1 and at
// least four entries per part, the entries are cut into that many parts of
// about equal limb counts, run as independent batches on the caller's stream
// and ctx->batch_split - 1 more, forked from and joined back to the caller's
// stream by events: the parts' steps overlap on the GPU (a transform of one
// part beside the inner product of another).  Same bits as unsplit.
int ckks::run_batch(ckks_ctx *ctx, int n, const BatchEntry *e, u64 *w, cudaStream_t st, int *status) {
    const int parts = std::min(ctx->batch_split, n / 4);
    std::unique_lock<std::mutex> lock(ctx->aux_mu, std::try_to_lock);
    if (parts < 2 || !lock.owns_lock()) return run_batch_on(ctx, n, e, w, st, status);
    // every entry's workspace fixed before the cut
    std::vector<BatchEntry> all(e, e + n);
    long long total = 0;
    for (int c = 0; c < n; ++c) {
        if (all[c].ws == nullptr) {
            all[c].ws = w;
            w += entry_ws_words(ctx, all[c].kind, all[c].ell);
        }
        total += all[c].ell;
    }
    CK(cudaEventRecord(ctx->fork_ev, st));
    for (int i = 1; i < parts; ++i) CK(cudaStreamWaitEvent(ctx->aux[i - 1], ctx->fork_ev, 0));
    int c0 = 0;
    long long done = 0;
    for (int i = 0; i < parts; ++i) {
        int c1 = c0;
        if (i == parts - 1) c1 = n;
        else
            while (c1 < n && (done + all[c1].ell) * parts <= total * (i + 1)) done += all[c1++].ell;
        if (c1 == c0 && c1 < n) done += all[c1++].ell;
        cudaStream_t s = i == 0 ? st : ctx->aux[i - 1];
        RC(run_batch_on(ctx, c1 - c0, all.data() + c0, nullptr, s, status));
        c0 = c1;
    }
    for (int i = 1; i < parts; ++i) {
        CK(cudaEventRecord(ctx->join_ev[i - 1], ctx->aux[i - 1]));
        CK(cudaStreamWaitEvent(st, ctx->join_ev[i - 1], 0));
    }
    return CKKS_OK;
}

// Runs a batch in groups of kMaxCts entries on one stream.
static int run_batch_on(ckks_ctx *ctx, int n, const BatchEntry *e, u64 *w, cudaStream_t st, int *status) {
    for (int c0 = 0; c0 < n; c0 += kMaxCts) {
        KsBatchDesc d{};
        d.n = std::min(n - c0, kMaxCts);
        d.L = ctx->L;
        d.k = ctx->k;
        d.alpha = ctx->alpha;
        d.dnum = ctx->dnum;
        d.logN = ctx->logN;
        TensorBatch T;
        T.n = 0;
        T.logN = ctx->logN;
        int te_of[kMaxCts];
        for (int c = 0; c < d.n; ++c) {
            const BatchEntry &x = e[c0 + c];
            te_of[c] = -1;
            TensorEntry te{};
            d.ct[c] = entry_desc(ctx, x, x.ws != nullptr ? x.ws : w, &te);
            if (x.kind == BE_MULT || x.kind == BE_NEWMULT) {
                te_of[c] = T.n;
                T.e[T.n++] = te;
            }
            if (x.ws == nullptr) w += entry_ws_words(ctx, x.kind, x.ell);
        }
        if (!ctx->split_bits) {
            for (int c = 0; c < d.n; ++c) RC(entry_one(ctx, d.ct[c], te_of[c] >= 0 ? &T.e[te_of[c]] : nullptr, st));
            continue;
        }
        // one launch per step over the whole batch
        RC(batch_front(ctx, d, T, st, status));
        RC(batch_back(ctx, d, T.n > 0, st, status));
    }
    return CKKS_OK;
}

static int keyswitch_batch_any(ckks_ctx *ctx, int n, const uint64_t *const *a, const uint64_t *const *b,
                               const int *levels, const uint32_t *galois, const uint64_t *const *keys,
                               const uint64_t *seeds, uint64_t *const *oa, uint64_t *const *ob, void *ws,
                               ckks_stream_t stream) {
    if (ctx == nullptr || n < 0) return CKKS_EINVAL;
    if (n == 0) return CKKS_OK;
    if (!a || !levels || !keys || !oa || !ob || !al16(ws)) return CKKS_EINVAL;
    std::vector<BatchEntry> e(n);
    for (int i = 0; i < n; ++i) {
        const bool rot = b != nullptr && b[i] != nullptr;
        if (!level_ok(ctx, levels[i]) || !al16(a[i]) || !al16(keys[i]) || !al16(oa[i]) || !al16(ob[i]))
            return CKKS_EINVAL;
        if (rot && (!al16(b[i]) || galois == nullptr || !galois_ok(ctx, galois[i]))) return CKKS_EINVAL;
        e[i] = BatchEntry{rot ? BE_HROTATE : BE_KEYSWITCH, a[i], rot ? b[i] : nullptr, nullptr, nullptr, keys[i],
                          oa[i], ob[i], levels[i], rot ? galois[i] : 1u, nullptr, seeds != nullptr,
                          seeds != nullptr ? seeds[i] : 0};
        if (seeds == nullptr) e[i].compressed = key_seed(ctx, keys[i], &e[i].seed);
    }
    return run_batch(ctx, n, e.data(), static_cast<u64 *>(ws), (cudaStream_t)stream);
}

extern "C" int ckks_keyswitch_batch(ckks_ctx *ctx, int n, const uint64_t *const *a, const uint64_t *const *b,
                                    const int *levels, const uint32_t *galois, const uint64_t *const *keys,
                                    uint64_t *const *oa, uint64_t *const *ob, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_keyswitch_batch");
    return keyswitch_batch_any(ctx, n, a, b, levels, galois, keys, nullptr, oa, ob, ws, stream);
}

// ---- batched HRotate with hoisted rotations (Algorithm 4 over many ciphertexts)
// Ciphertext c has nrot[c] rotations; its first rotation owns the full HRotate
// workspace (ModUp digits, uv, scratch), every further rotation only uv and
// scratch and reads the owner's digits.
static size_t rot_extra_words(const ckks_ctx *c, int ell) {
    const HrLayout lo = hr_layout(c, ell);
    return lo.total - lo.uv;  // uv | tmp
}

extern "C" int ckks_hrotate_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, const int *nrot,
                                                  size_t *bytes) {
    if (ctx == nullptr || bytes == nullptr || n < 0 || (n > 0 && (levels == nullptr || nrot == nullptr)))
        return CKKS_EINVAL;
    size_t w = 0;
    for (int i = 0; i < n; ++i) {
        if (!level_ok(ctx, levels[i]) || nrot[i] < 1) return CKKS_EINVAL;
        w += hr_layout(ctx, levels[i]).total + size_t(nrot[i] - 1) * rot_extra_words(ctx, levels[i]);
    }
    *bytes = w * sizeof(u64);
    return CKKS_OK;
}

extern "C" int ckks_hrotate_batch(ckks_ctx *ctx, int n, const uint64_t *const *a, const uint64_t *const *b,
                                  const int *levels, const int *nrot, const uint32_t *galois,
                                  const uint64_t *const *keys, uint64_t *const *oa, uint64_t *const *ob, void *ws,
                                  ckks_stream_t stream) {
    OpRange r_("ckks_hrotate_batch");
    if (ctx == nullptr || n < 0) return CKKS_EINVAL;
    if (n == 0) return CKKS_OK;
    if (!a || !b || !levels || !nrot || !galois || !keys || !oa || !ob || !al16(ws)) return CKKS_EINVAL;
    int m = 0;
    for (int c = 0; c < n; ++c) {
        if (!level_ok(ctx, levels[c]) || nrot[c] < 1 || !al16(a[c]) || !al16(b[c])) return CKKS_EINVAL;
        for (int r = 0; r < nrot[c]; ++r, ++m)
            if (!galois_ok(ctx, galois[m]) || !al16(keys[m]) || !al16(oa[m]) || !al16(ob[m])) return CKKS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    u64 *w = static_cast<u64 *>(ws);
    if (!ctx->split_bits) {
        // one ciphertext at a time: ModUp once, then every rotation (the single-call path)
        for (int c = 0, i = 0; c < n; i += nrot[c], ++c) {
            RC(ckks_hrotate(ctx, a[c], b[c], levels[c], nrot[c], galois + i, keys + i, oa + i, ob + i, w, stream));
            w += hr_layout(ctx, levels[c]).total + size_t(nrot[c] - 1) * rot_extra_words(ctx, levels[c]);
        }
        return CKKS_OK;
    }
    // descriptors of every rotation; the first of each ciphertext owns the digits
    std::vector<CtDesc> all(m), owners(n);
    for (int c = 0, i = 0; c < n; ++c) {
        u64 *own = w;
        for (int r = 0; r < nrot[c]; ++r, ++i) {
            BatchEntry e{BE_HROTATE, a[c], b[c], nullptr, nullptr, keys[i], oa[i], ob[i], levels[c], galois[i],
                         nullptr, 0, 0};
            e.compressed = key_seed(ctx, keys[i], &e.seed);
            TensorEntry te{};
            all[i] = entry_desc(ctx, e, w, &te);
            if (r == 0) {
                owners[c] = all[i];
                w += hr_layout(ctx, levels[c]).total;
            } else {
                all[i].ext_shared = own;
                w += rot_extra_words(ctx, levels[c]);
            }
        }
    }
    auto desc = [&](const CtDesc *v, int cnt) {
        KsBatchDesc d{};
        d.n = cnt;
        d.L = ctx->L;
        d.k = ctx->k;
        d.alpha = ctx->alpha;
        d.dnum = ctx->dnum;
        d.logN = ctx->logN;
        for (int i = 0; i < cnt; ++i) d.ct[i] = v[i];
        return d;
    };
    // ciphertexts [c0, c1) with their rotations [i0, i1): ModUp of each
    // ciphertext once, then every rotation's inner product and ModDown
    auto run_part = [&](int c0, int c1, int i0, int i1, cudaStream_t s2) -> int {
        for (int c = c0; c < c1; c += kMaxCts) {
            const KsBatchDesc d = desc(owners.data() + c, std::min(c1 - c, kMaxCts));
            CK(launch_ntt_batch(ctx, d, PH_INTT_A, s2));
            CK(launch_bconv_batch(ctx, d, GM_MODUP, s2));
            CK(launch_ntt_batch(ctx, d, PH_NTT_UP, s2));
        }
        for (int i = i0; i < i1; i += kMaxCts) {
            const KsBatchDesc d = desc(all.data() + i, std::min(i1 - i, kMaxCts));
            CK(launch_inner_prod_batch(ctx, d, s2));
            RC(batch_back(ctx, d, false, s2));
        }
        return CKKS_OK;
    };
    // as in run_batch: with ctx->batch_split > 1 and at least four rotations
    // per part, the ciphertexts (each with all its rotations) are cut into parts
    // of about equal rotation counts on the context's streams
    const int parts = std::min({ctx->batch_split, n, m / 4});
    std::unique_lock<std::mutex> lock(ctx->aux_mu, std::try_to_lock);
    if (parts < 2 || !lock.owns_lock()) return run_part(0, n, 0, m, st);
    CK(cudaEventRecord(ctx->fork_ev, st));
    for (int i = 1; i < parts; ++i) CK(cudaStreamWaitEvent(ctx->aux[i - 1], ctx->fork_ev, 0));
    int c0 = 0, i0 = 0;
    for (int pt = 0; pt < parts; ++pt) {
        int c1 = c0, i1 = i0;
        while (c1 < n && (c1 == c0 || pt == parts - 1 || (i1 + nrot[c1]) * parts <= m * (pt + 1))) i1 += nrot[c1++];
        RC(run_part(c0, c1, i0, i1, pt == 0 ? st : ctx->aux[pt - 1]));
        c0 = c1;
        i0 = i1;
    }
    for (int i = 1; i < parts; ++i) {
        CK(cudaEventRecord(ctx->join_ev[i - 1], ctx->aux[i - 1]));
        CK(cudaStreamWaitEvent(st, ctx->join_ev[i - 1], 0));
    }
    return CKKS_OK;
}

extern "C" int ckks_keyswitch_batch_seeded(ckks_ctx *ctx, int n, const uint64_t *const *a, const uint64_t *const *b,
                                           const int *levels, const uint32_t *galois,
                                           const uint64_t *const *keys_b, const uint64_t *seeds, uint64_t *const *oa,
                                           uint64_t *const *ob, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_keyswitch_batch_seeded");
    if (seeds == nullptr && n > 0) return CKKS_EINVAL;
    return keyswitch_batch_any(ctx, n, a, b, levels, galois, keys_b, seeds, oa, ob, ws, stream);
}

static int mult_like_batch(ckks_ctx *ctx, int kind, int n, const uint64_t *const *a1, const uint64_t *const *b1,
                           const uint64_t *const *a2, const uint64_t *const *b2, const int *levels,
                           const uint64_t *const *keys, uint64_t *const *oa, uint64_t *const *ob, void *ws,
                           ckks_stream_t stream) {
    if (ctx == nullptr || n < 0) return CKKS_EINVAL;
    if (n == 0) return CKKS_OK;
    if (!a1 || !b1 || !a2 || !b2 || !levels || !keys || !oa || !ob || !al16(ws)) return CKKS_EINVAL;
    if (kind == BE_NEWMULT && ctx->k + 1 > kMaxSrc) return CKKS_EUNSUPPORTED;
    std::vector<BatchEntry> e(n);
    for (int i = 0; i < n; ++i) {
        if (!level_ok(ctx, levels[i]) || levels[i] < 2 || !al16(a1[i]) || !al16(b1[i]) || !al16(a2[i]) ||
            !al16(b2[i]) || !al16(keys[i]) || !al16(oa[i]) || !al16(ob[i]))
            return CKKS_EINVAL;
        e[i] = BatchEntry{kind, a1[i], b1[i], a2[i], b2[i], keys[i], oa[i], ob[i], levels[i], 1u, nullptr, 0, 0};
        e[i].compressed = key_seed(ctx, keys[i], &e[i].seed);
    }
    return run_batch(ctx, n, e.data(), static_cast<u64 *>(ws), (cudaStream_t)stream);
}

extern "C" int ckks_mult_batch(ckks_ctx *ctx, int n, const uint64_t *const *a1, const uint64_t *const *b1,
                               const uint64_t *const *a2, const uint64_t *const *b2, const int *levels,
                               const uint64_t *const *keys, uint64_t *const *oa, uint64_t *const *ob, void *ws,
                               ckks_stream_t stream) {
    OpRange r_("ckks_mult_batch");
    return mult_like_batch(ctx, BE_MULT, n, a1, b1, a2, b2, levels, keys, oa, ob, ws, stream);
}

extern "C" int ckks_newmult_batch_workspace_bytes(const ckks_ctx *ctx, int n, const int *levels, size_t *bytes) {
    if (ctx == nullptr || bytes == nullptr || n < 0 || (n > 0 && levels == nullptr)) return CKKS_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!level_ok(ctx, levels[i]) || levels[i] < 2) return CKKS_EINVAL;
    *bytes = batch_ws_words(ctx, n, levels, BE_NEWMULT) * sizeof(u64);
    return CKKS_OK;
}

extern "C" int ckks_newmult_batch(ckks_ctx *ctx, int n, const uint64_t *const *a1, const uint64_t *const *b1,
                                  const uint64_t *const *a2, const uint64_t *const *b2, const int *levels,
                                  const uint64_t *const *keys, uint64_t *const *oa, uint64_t *const *ob, void *ws,
                                  ckks_stream_t stream) {
    OpRange r_("ckks_newmult_batch");
    return mult_like_batch(ctx, BE_NEWMULT, n, a1, b1, a2, b2, levels, keys, oa, ob, ws, stream);
}

extern "C" int ckks_newmult(ckks_ctx *ctx, const uint64_t *a1, const uint64_t *b1, const uint64_t *a2,
                            const uint64_t *b2, int level, const uint64_t *key, uint64_t *oa, uint64_t *ob, void *ws,
                            ckks_stream_t stream) {
    return ckks_newmult_batch(ctx, 1, &a1, &b1, &a2, &b2, &level, &key, &oa, &ob, ws, stream);
}

// Encrypted inner product with the ModDown hoisted (Sec. 5.1): the n NewMult
// products are lifted and summed over the extended basis, then one merged
// ModDown per polynomial.  All pairs at one level; workspace: n NewMult entries.
extern "C" int ckks_newmult_sum(ckks_ctx *ctx, int n, const uint64_t *const *a1, const uint64_t *const *b1,
                                const uint64_t *const *a2, const uint64_t *const *b2, int level,
                                const uint64_t *key, uint64_t *oa, uint64_t *ob, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_newmult_sum");
    if (ctx == nullptr || n < 1 || n > kMaxCts || !a1 || !b1 || !a2 || !b2 || !level_ok(ctx, level) || level < 2 ||
        !al16(key) || !al16(oa) || !al16(ob) || !al16(ws))
        return CKKS_EINVAL;
    if (ctx->k + 1 > kMaxSrc || !ctx->split_bits) return CKKS_EUNSUPPORTED;
    for (int i = 0; i < n; ++i)
        if (!al16(a1[i]) || !al16(b1[i]) || !al16(a2[i]) || !al16(b2[i])) return CKKS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    KsBatchDesc d{};
    d.n = n;
    d.L = ctx->L;
    d.k = ctx->k;
    d.alpha = ctx->alpha;
    d.dnum = ctx->dnum;
    d.logN = ctx->logN;
    TensorBatch T;
    T.n = 0;
    T.logN = ctx->logN;
    u64 *w = static_cast<u64 *>(ws);
    for (int i = 0; i < n; ++i) {
        BatchEntry e{BE_NEWMULT, a1[i], b1[i], a2[i], b2[i], key, oa, ob, level, 1u, nullptr, 0, 0};
        e.compressed = key_seed(ctx, key, &e.seed);
        TensorEntry te{};
        d.ct[i] = entry_desc(ctx, e, w, &te);
        T.e[T.n++] = te;
        w += entry_ws_words(ctx, BE_NEWMULT, level);
    }
    RC(batch_front(ctx, d, T, st));
    if (n > 1) CK(launch_sum_uv(ctx, d, st));
    KsBatchDesc d1 = d;
    d1.n = 1;
    return batch_back(ctx, d1, false, st);
}

extern "C" int ckks_mult(ckks_ctx *ctx, const uint64_t *a1, const uint64_t *b1, const uint64_t *a2,
                         const uint64_t *b2, int level, const uint64_t *key, uint64_t *oa, uint64_t *ob, void *ws,
                         ckks_stream_t stream) {
    return ckks_mult_batch(ctx, 1, &a1, &b1, &a2, &b2, &level, &key, &oa, &ob, ws, stream);
}

extern "C" int ckks_ptmatvecmult(ckks_ctx *ctx, const uint64_t *a, const uint64_t *b, int ell, int nb, int ng,
                                 const uint32_t *g_baby, const uint32_t *g_giant, const uint64_t *const *key_baby,
                                 const uint64_t *const *key_giant, const uint64_t *const *diag, int rescale,
                                 uint64_t *oa, uint64_t *ob, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_ptmatvecmult");
    if (!level_ok(ctx, ell) || !al16(a) || !al16(b) || !al16(oa) || !al16(ob) || !al16(ws) || nb < 1 ||
        nb > kMaxRot || ng < 1 || diag == nullptr || (rescale && ell < 2))
        return CKKS_EINVAL;
    if (nb > 1 && (g_baby == nullptr || key_baby == nullptr)) return CKKS_EINVAL;
    if (ng > 1 && (g_giant == nullptr || key_giant == nullptr)) return CKKS_EINVAL;
    for (int i = 1; i < nb; ++i)
        if (!galois_ok(ctx, g_baby[i]) || !al16(key_baby[i])) return CKKS_EINVAL;
    for (int t = 1; t < ng; ++t)
        if (!galois_ok(ctx, g_giant[t]) || !al16(key_giant[t])) return CKKS_EINVAL;
    for (int d = 0; d < nb * ng; ++d)
        if (!al16(diag[d])) return CKKS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = ctx->N;
    const int k = ctx->k;
    u64 *w = static_cast<u64 *>(ws);
    const PmvLayout lo = pmv_layout(ctx, ell, ng);
    RC(modup_all(ctx, a, ell, w + lo.ext, w + lo.tmp, st));
    u64 *acc_a = w + lo.acc, *acc_b = acc_a + size_t(ell + k) * N;
    u64 *res_a = rescale ? w + lo.res : oa, *res_b = rescale ? w + lo.res + size_t(ell) * N : ob;
    u64 *ct_a = w + lo.ct, *ct_b = ct_a + size_t(ell) * N;
    if (pmv_all_supported(ctx, ell, nb, ng)) {
        // every giant step's accumulator in one pass over the baby-step keys
        PmvAllArgs pa{};
        pa.ext = w + lo.ext;
        pa.a = a;
        pa.b = b;
        pa.ell = ell;
        pa.nb = nb;
        pa.ng = ng;
        for (int t = 0; t < ng; ++t) {
            pa.acc_a[t] = acc_a + size_t(2) * t * (ell + k) * N;
            pa.acc_b[t] = pa.acc_a[t] + size_t(ell + k) * N;
        }
        for (int i = 0; i < nb; ++i) {
            pa.galois[i] = i == 0 ? 1u : g_baby[i];
            pa.key[i] = i == 0 ? nullptr : key_baby[i];
            pa.compressed[i] = i == 0 ? 0 : uint8_t(key_seed(ctx, key_baby[i], &pa.seed[i]));
        }
        for (int d = 0; d < nb * ng; ++d) pa.diag[d] = diag[d];
        CK(launch_pmv_all(ctx, pa, st));
        // The giant steps are independent until they are summed: step 0 is
        // ModDown'ed into res on the caller's stream; step t >= 1 (ModDown, then
        // Rotate by its giant element into its own output) runs on a context
        // stream when the call holds them (forked and joined by events), else on
        // the caller's stream; then res += the rotated steps.
        const u64 *noadd[2] = {nullptr, nullptr};
        std::unique_lock<std::mutex> lock(ctx->aux_mu, std::try_to_lock);
        const bool split = lock.owns_lock() && ng > 1;
        if (split) {
            CK(cudaEventRecord(ctx->fork_ev, st));
            for (int i = 0; i < std::min(ng - 1, ckks_ctx::kAux); ++i)
                CK(cudaStreamWaitEvent(ctx->aux[i], ctx->fork_ev, 0));
        }
        PolySum sum{};
        sum.acc[0] = res_a;
        sum.acc[1] = res_b;
        for (int t = 0; t < ng; ++t) {
            const u64 *in[2] = {pa.acc_a[t], pa.acc_b[t]};
            if (t == 0) {
                u64 *out[2] = {res_a, res_b};
                RC(moddown_polys(ctx, ell, 2, in, out, noadd, 1, 0, w + lo.tmp, w + lo.tmp + size_t(2) * k * N, st));
                continue;
            }
            u64 *ch = w + lo.chain + size_t(t - 1) * lo.chain_words;
            u64 *tmp = ch, *cta = tmp + std::max(size_t(ell), words_moddown2(ctx, ell)) * N;
            u64 *ctb = cta + size_t(ell) * N, *oa_t = ctb + size_t(ell) * N, *ob_t = oa_t + size_t(ell) * N;
            u64 *rws = ob_t + size_t(ell) * N;
            cudaStream_t s2 = split ? ctx->aux[(t - 1) % ckks_ctx::kAux] : st;
            u64 *out[2] = {cta, ctb};
            RC(moddown_polys(ctx, ell, 2, in, out, noadd, 1, 0, tmp, tmp + size_t(2) * k * N, s2));
            RC(rotate_core(ctx, cta, ctb, ell, g_giant[t], key_giant[t], oa_t, ob_t, 0, rws, s2));
            sum.in[0][sum.n] = oa_t;
            sum.in[1][sum.n++] = ob_t;
        }
        if (split)
            for (int i = 0; i < std::min(ng - 1, ckks_ctx::kAux); ++i) {
                CK(cudaEventRecord(ctx->join_ev[i], ctx->aux[i]));
                CK(cudaStreamWaitEvent(st, ctx->join_ev[i], 0));
            }
        CK(launch_poly_sum(ctx, sum, ell, st));
    }
    for (int t = 0; t < ng && !pmv_all_supported(ctx, ell, nb, ng); ++t) {
        PmvArgs pa{};
        pa.ext = w + lo.ext;
        pa.a = a;
        pa.b = b;
        pa.acc_a = acc_a;
        pa.acc_b = acc_b;
        pa.ell = ell;
        pa.nb = nb;
        for (int i = 0; i < nb; ++i) {
            pa.galois[i] = i == 0 ? 1u : g_baby[i];
            pa.key[i] = i == 0 ? nullptr : key_baby[i];
            pa.compressed[i] = i == 0 ? 0 : uint8_t(key_seed(ctx, key_baby[i], &pa.seed[i]));
            pa.diag[i] = diag[size_t(t) * nb + i];
        }
        CK(launch_pmv_accum(ctx, pa, st));
        const u64 *in[2] = {acc_a, acc_b};
        const u64 *noadd[2] = {nullptr, nullptr};
        if (t == 0) {
            u64 *out[2] = {res_a, res_b};
            RC(moddown_polys(ctx, ell, 2, in, out, noadd, 1, 0, w + lo.tmp, w + lo.tmp + size_t(2) * k * N, st));
        } else {
            u64 *out[2] = {ct_a, ct_b};
            RC(moddown_polys(ctx, ell, 2, in, out, noadd, 1, 0, w + lo.tmp, w + lo.tmp + size_t(2) * k * N, st));
            RC(rotate_core(ctx, ct_a, ct_b, ell, g_giant[t], key_giant[t], res_a, res_b, 1, w + lo.rot, st));
        }
    }
    if (rescale) {
        const u64 *in[2] = {res_a, res_b};
        u64 *out[2] = {oa, ob};
        RC(rescale_polys(ctx, ell, 2, in, out, acc_a, acc_a + size_t(2) * N, st));
    }
    return CKKS_OK;
}

extern "C" int ckks_keygen_ksk(ckks_ctx *ctx, const int64_t *s, const int64_t *e, const uint64_t *a, uint32_t g,
                               uint64_t *key, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_keygen_ksk");
    if (ctx == nullptr || !al16(s) || !al16(e) || !al16(a) || !al16(key) || !al16(ws) || (g != 0 && !galois_ok(ctx, g)))
        return CKKS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = ctx->N;
    const int LK = ctx->L + ctx->k;
    u64 *sh = static_cast<u64 *>(ws), *sp = sh + size_t(LK) * N, *eh = sp + size_t(LK) * N;
    LimbList ls, le;
    for (int l = 0; l < LK; ++l) {
        ls.add(sh + l * N, sh + l * N, l);
        le.add(eh + l * N, eh + l * N, l);
    }
    CK(launch_signed_to_res(ctx, s, sh, st));  // element-wise kernels are timed in keyswitch.cu
    RC(run_ntt(ctx, ls, false, st));
    if (g != 0) CK(launch_automorph(ctx, sh, sp, LK, g, st));
    else CK(launch_square(ctx, sh, sp, st));
    for (int j = 0; j < ctx->dnum; ++j) {
        CK(launch_signed_to_res(ctx, e + size_t(j) * N, eh, st));
        RC(run_ntt(ctx, le, false, st));
        CK(launch_keygen_row(ctx, a + size_t(j) * LK * N, sh, sp, eh, j, key + size_t(2 * j) * LK * N,
                             key + size_t(2 * j + 1) * LK * N, st));
    }
    return CKKS_OK;
}

// Compressed keys (Sec. 5.3): only the rows b_j are stored; a_j comes from the seed.
extern "C" int ckks_keygen_ksk_seeded(ckks_ctx *ctx, const int64_t *s, const int64_t *e, uint64_t seed, uint32_t g,
                                      uint64_t *key_b, void *ws, ckks_stream_t stream) {
    OpRange r_("ckks_keygen_ksk_seeded");
    if (ctx == nullptr || !al16(s) || !al16(e) || !al16(key_b) || !al16(ws) || (g != 0 && !galois_ok(ctx, g)))
        return CKKS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = ctx->N;
    const int LK = ctx->L + ctx->k;
    u64 *sh = static_cast<u64 *>(ws), *sp = sh + size_t(LK) * N, *eh = sp + size_t(LK) * N, *aj = eh + size_t(LK) * N;
    LimbList ls, le;
    for (int l = 0; l < LK; ++l) {
        ls.add(sh + l * N, sh + l * N, l);
        le.add(eh + l * N, eh + l * N, l);
    }
    CK(launch_signed_to_res(ctx, s, sh, st));
    RC(run_ntt(ctx, ls, false, st));
    if (g != 0) CK(launch_automorph(ctx, sh, sp, LK, g, st));
    else CK(launch_square(ctx, sh, sp, st));
    for (int j = 0; j < ctx->dnum; ++j) {
        CK(launch_key_a_fill(ctx, seed, j, 1, aj, st));
        CK(launch_signed_to_res(ctx, e + size_t(j) * N, eh, st));
        RC(run_ntt(ctx, le, false, st));
        CK(launch_keygen_row(ctx, aj, sh, sp, eh, j, nullptr, key_b + size_t(j) * LK * N, st));
    }
    return CKKS_OK;
}

extern "C" int ckks_ksk_expand(ckks_ctx *ctx, const uint64_t *key_b, uint64_t seed, uint64_t *key,
                               ckks_stream_t stream) {
    OpRange r_("ckks_ksk_expand");
    if (ctx == nullptr || !al16(key_b) || !al16(key) || key_b == key) return CKKS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t row = size_t(ctx->L + ctx->k) * ctx->N;
    for (int j = 0; j < ctx->dnum; ++j) {
        CK(launch_key_a_fill(ctx, seed, j, 1, key + size_t(2 * j) * row, st));
        CK(cudaMemcpyAsync(key + size_t(2 * j + 1) * row, key_b + size_t(j) * row, row * sizeof(u64),
                           cudaMemcpyDeviceToDevice, st));
    }
    return CKKS_OK;
}

// ------------------------------------------------------------------ asynchronous errors
extern "C" int ckks_poll_status(ckks_ctx *ctx, ckks_stream_t stream, int *done) {
    if (ctx == nullptr) return CKKS_EINVAL;
    const cudaError_t q = cudaStreamQuery((cudaStream_t)stream);
    if (done) *done = q == cudaSuccess;
    if (q == cudaSuccess) {
        // a bounded wait that ran out in a finished kernel (read and cleared)
        int flag = 0;
        cudaError_t e = cudaMemcpy(&flag, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && flag != 0) e = cudaMemset(ctx->d_status, 0, sizeof(int));
        if (e != cudaSuccess) {
            ctx->last_cuda_error = int(e);
            return CKKS_ECUDA;
        }
        return flag ? CKKS_ETIMEOUT : CKKS_OK;
    }
    if (q == cudaErrorNotReady) return CKKS_OK;
    ctx->last_cuda_error = int(q);
    return CKKS_ECUDA;
}

// ------------------------------------------------------------------ compressed-key registry
extern "C" int ckks_key_register_seed(ckks_ctx *ctx, const uint64_t *key_b, uint64_t seed) {
    if (ctx == nullptr || !al16(key_b)) return CKKS_EINVAL;
    ctx->comp_keys[key_b] = seed;
    return CKKS_OK;
}

extern "C" int ckks_key_unregister(ckks_ctx *ctx, const uint64_t *key_b) {
    if (ctx == nullptr || key_b == nullptr) return CKKS_EINVAL;
    return ctx->comp_keys.erase(key_b) ? CKKS_OK : CKKS_EINVAL;
}

// ------------------------------------------------------------------ autotuner
extern "C" int ckks_autotune(ckks_ctx *ctx, void *ws, size_t ws_bytes, ckks_stream_t stream, int *choice,
                             float *times) {
    OpRange r_("ckks_autotune");
    if (ctx == nullptr || !al16(ws)) return CKKS_EINVAL;
    const size_t limb = size_t(ctx->N) * sizeof(u64);
    const int large = int(std::min<size_t>(kMaxBatch, ws_bytes / limb));
    const int small = 24;
    if (large < small) return CKKS_EINVAL;
    if (times)
        for (int i = 0; i < 24; ++i) times[i] = 0.f;
    CK(ntt_autotune(ctx, static_cast<u64 *>(ws), small, large, (cudaStream_t)stream, times));
    if (choice) {
        for (int i = 0; i < 4; ++i) choice[i] = ctx->ntt_csel[i / 2][i % 2];
        for (int i = 0; i < 4; ++i) choice[4 + i] = ctx->ntt_split[i / 2][i % 2];
    }
    return CKKS_OK;
}

extern "C" int ckks_tune_set(ckks_ctx *ctx, const int *choice) {
    if (ctx == nullptr || choice == nullptr) return CKKS_EINVAL;
    for (int i = 0; i < 4; ++i)
        if (choice[i] < 0 || choice[i] > 2 || choice[4 + i] < -1 || choice[4 + i] > 1) return CKKS_EINVAL;
    for (int i = 0; i < 4; ++i) ctx->ntt_csel[i / 2][i % 2] = choice[i];
    for (int i = 0; i < 4; ++i) ctx->ntt_split[i / 2][i % 2] = choice[4 + i];
    return CKKS_OK;
}

extern "C" int ckks_selftest_bounded_wait(ckks_ctx *ctx, uint32_t limit_us, ckks_stream_t stream) {
    if (ctx == nullptr || limit_us == 0 || limit_us > 2000000u) return CKKS_EINVAL;
    CK(launch_bounded_wait_selftest(ctx, uint64_t(limit_us) * 1000u, (cudaStream_t)stream));
    return CKKS_OK;
}

extern "C" int ckks_butterfly_peak_sink_bytes(const ckks_ctx *ctx, size_t *bytes) {
    if (ctx == nullptr || bytes == nullptr) return CKKS_EINVAL;
    *bytes = bfly_peak_sink_words(ctx) * sizeof(u64);
    return CKKS_OK;
}

extern "C" int ckks_butterfly_peak(ckks_ctx *ctx, int rounds, void *sink, ckks_stream_t stream, float *ms,
                                   double *butterflies) {
    OpRange r_("ckks_butterfly_peak");
    if (ctx == nullptr || rounds < 1 || rounds > (1 << 24) || !al16(sink) || ms == nullptr || butterflies == nullptr)
        return CKKS_EINVAL;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) err = launch_bfly_peak(ctx, rounds, static_cast<u64 *>(sink), st, butterflies);
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    CK(err);
    return CKKS_OK;
}

extern "C" int ckks_concurrency_hint(ckks_ctx *ctx, int n) {
    if (ctx == nullptr || n < 1 || n > 64) return CKKS_EINVAL;
    ctx->concurrency = n;
    return CKKS_OK;
}

extern "C" int ckks_batch_streams(ckks_ctx *ctx, int nstreams) {
    if (ctx == nullptr || nstreams < 1 || nstreams > ckks_ctx::kAux + 1) return CKKS_EINVAL;
    ctx->batch_split = nstreams;
    return CKKS_OK;
}

extern "C" int ckks_fuse_select(ckks_ctx *ctx, int on, int *available) {
    if (ctx == nullptr) return CKKS_EINVAL;
    if (available) *available = ctx->small_primes && ctx->logN >= 10 && ctx->logN <= 17 && ctx->alpha > 0 &&
                                beta_of(ctx, ctx->L) <= 4;
    ctx->fuse_on = on != 0;
    return CKKS_OK;
}

extern "C" int ckks_bconv_select(ckks_ctx *ctx, int tensor_cores, int *available) {
    if (ctx == nullptr) return CKKS_EINVAL;
    if (available) *available = ctx->tc_kg != 0;
    ctx->tc_on = tensor_cores != 0;
    return CKKS_OK;
}

// ------------------------------------------------------------------ measurement hook
extern "C" int ckks_profile_enable(ckks_ctx *ctx, int on) {
    if (ctx == nullptr) return CKKS_EINVAL;
    ctx->prof_on = on != 0;
    return CKKS_OK;
}

static int prof_drain(ckks_ctx *ctx) {
    for (auto &r : ctx->prof_pending) {
        float ms = 0.f;
        CK(cudaEventSynchronize(r.b));
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        ctx->prof_ms[r.kclass] += ms;
        ctx->prof_n[r.kclass] += 1;
        ctx->prof_units[r.kclass] += r.units;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    return CKKS_OK;
}

extern "C" int ckks_profile_reset(ckks_ctx *ctx) {
    if (ctx == nullptr) return CKKS_EINVAL;
    RC(prof_drain(ctx));
    for (int i = 0; i < 8; ++i) {
        ctx->prof_ms[i] = 0;
        ctx->prof_n[i] = 0;
        ctx->prof_units[i] = 0;
    }
    return CKKS_OK;
}

extern "C" int ckks_profile_read(ckks_ctx *ctx, int kclass, double *total_ms, long long *launches, double *units) {
    if (ctx == nullptr || kclass < 0 || kclass >= CKKS_K_COUNT) return CKKS_EINVAL;
    RC(prof_drain(ctx));
    if (total_ms) *total_ms = ctx->prof_ms[kclass];
    if (launches) *launches = ctx->prof_n[kclass];
    if (units) *units = ctx->prof_units[kclass];
    return CKKS_OK;
}

// ------------------------------------------------------------------ ModDown without a workspace
// For callers that cannot allocate device memory: the ModDown scratch (k P-limbs
// in coefficient form, then ell converted limbs) lives in this fixed array
// instead of a caller workspace.  2^21 words = 16 MiB, held by every GPU that
// loads the library until exit.  Calls share it; see the header for the races.
static constexpr size_t kNoallocWords = size_t(1) << 21;
static __device__ __align__(256) uint64_t g_moddown_scratch[kNoallocWords];

static std::mutex g_noalloc_mu;
static uint64_t *g_noalloc_ptr[256];  // device address of the array, per device ordinal

// Device address of the array on `device`, looked up once with that device current.
static cudaError_t noalloc_scratch(int device, uint64_t **out) {
    if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[device] == nullptr) {
        int prev = 0;
        cudaError_t err = cudaGetDevice(&prev);
        if (err != cudaSuccess) return err;
        if (prev != device && (err = cudaSetDevice(device)) != cudaSuccess) return err;
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_moddown_scratch);
        if (prev != device) {
            const cudaError_t back = cudaSetDevice(prev);
            if (err == cudaSuccess) err = back;
        }
        if (err != cudaSuccess) return err;
        g_noalloc_ptr[device] = static_cast<uint64_t *>(p);
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}

extern "C" int ckks_moddown_noalloc(ckks_ctx *ctx, const uint64_t *in, int ell, uint64_t *out, ckks_stream_t stream) {
    if (!level_ok(ctx, ell) || !al16(in) || !al16(out)) return CKKS_EINVAL;
    if (size_t(ctx->k + ell) * size_t(ctx->N) > kNoallocWords) return CKKS_EUNSUPPORTED;
    uint64_t *w = nullptr;
    CK(noalloc_scratch(ctx->device, &w));
    const u64 *ins[2] = {in, nullptr};
    u64 *outs[2] = {out, nullptr};
    const u64 *adds[2] = {nullptr, nullptr};
    return moddown_polys(ctx, ell, 1, ins, outs, adds, 1, 0, w, w + size_t(ctx->k) * ctx->N, (cudaStream_t)stream);
}
