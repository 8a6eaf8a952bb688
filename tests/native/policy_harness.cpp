// Host checks of launch_policy.h: the tensor-core conversion's CTAs per row,
// the grouping of batch entries that share a compressed key, and the NTT
// autotuner's choice.  Prints "ok <name>" per check; exits non-zero on the
// first failure.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "launch_policy.h"

using namespace ckks::policy;

#define CHECK(cond)                                                                  \
    do {                                                                             \
        if (!(cond)) {                                                               \
            std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #cond);              \
            std::exit(1);                                                            \
        }                                                                            \
    } while (0)

static void tc_grid() {
    const int sms = 152;
    // N = 2^16: 512 tiles of 128 coefficients.  A call alone (all SMs): one ModUp
    // of 3 digits and one ModDown of 2 polynomials, one chunk each.
    CHECK(sm_share(sms, 1) == 152);
    CHECK(tc_ctas_per_row(512, 3, sm_share(sms, 1)) == 50);
    CHECK(tc_ctas_per_row(512, 2, sm_share(sms, 1)) == 76);
    // 8 operations at once: 19 SMs each, 19 CTAs per row for both
    CHECK(sm_share(sms, 8) == 19);
    CHECK(tc_ctas_per_row(512, 3, 19) == 19);
    CHECK(tc_ctas_per_row(512, 2, 19) == 19);
    // a batched ModUp of 64 entries (192 rows): 7 CTAs per row
    CHECK(tc_ctas_per_row(512, 192, 152) == 7);
    // degenerate shares and small rings
    CHECK(sm_share(sms, 1000) == 1 && sm_share(sms, 0) == 152);
    CHECK(tc_ctas_per_row(8, 1, 152) == 8);  // at most one CTA per tile
    // the pick minimises the modelled cost, ties to more CTAs, within [1, min(tiles, 256)]
    std::mt19937 rng(7);
    for (int it = 0; it < 2000; ++it) {
        const int tiles = 1 + int(rng() % 1024), rows = 1 + int(rng() % 400), share = 1 + int(rng() % 200);
        const int per = tc_ctas_per_row(tiles, rows, share);
        CHECK(per >= 1 && per <= std::min(tiles, 256));
        const long best = tc_cost(tiles, rows, share, per);
        for (int c = 1; c <= std::min(tiles, 256); ++c) {
            const long cost = tc_cost(tiles, rows, share, c);
            CHECK(cost >= best);
            if (c > per) CHECK(cost > best);
        }
    }
    std::printf("ok tc_grid\n");
}

static void group_cap() {
    const int sms = 152;
    // N = 2^16, L + k = 32: 128 tiles x 32 primes per entry; a 32-entry half batch
    // fills the GPU many times over, so the cap is the maximum
    CHECK(ip_group_cap(128L * 32, 32, sms, 3, 64) == 64);
    // 4 entries: 16384 CTAs / 1216 = 13
    CHECK(ip_group_cap(128L * 32, 4, sms, 3, 64) == 13);
    // N = 2^11, L + k = 10: 4 tiles x 10 primes, 6 entries: groups of one
    CHECK(ip_group_cap(4L * 10, 6, sms, 3, 64) == 1);
    // more than 4 digits: groups of one whatever the size
    CHECK(ip_group_cap(128L * 32, 64, sms, 6, 64) == 1);
    std::printf("ok group_cap\n");
}

static void grouping() {
    // runs of keys, cut where the key changes or the group reaches the cap
    const std::vector<int> key = {7, 7, 7, 3, 3, 9, 9, 9, 9, 9, 7, 2};
    auto same = [&](int a, int c) { return key[a] == key[c]; };
    uint8_t start[65];
    int g = ip_groups(int(key.size()), 64, same, start);
    const std::vector<int> want = {0, 3, 5, 10, 11, 12};
    CHECK(g == int(want.size()) - 1);
    for (int i = 0; i <= g; ++i) CHECK(start[i] == want[i]);
    g = ip_groups(int(key.size()), 2, same, start);
    const std::vector<int> want2 = {0, 2, 3, 5, 7, 9, 10, 11, 12};
    CHECK(g == int(want2.size()) - 1);
    for (int i = 0; i <= g; ++i) CHECK(start[i] == want2[i]);
    // random batches: groups cover 0..n-1 in order, each at most cap long, each
    // of one key, and a cut between groups is forced (key change or cap)
    std::mt19937 rng(11);
    for (int it = 0; it < 5000; ++it) {
        const int n = 1 + int(rng() % 64), cap = 1 + int(rng() % 64);
        std::vector<int> k(n);
        for (int i = 0; i < n; ++i) k[i] = int(rng() % 3);
        auto eq = [&](int a, int c) { return k[a] == k[c]; };
        const int ng = ip_groups(n, cap, eq, start);
        CHECK(ng >= 1 && start[0] == 0 && start[ng] == n);
        for (int gi = 0; gi < ng; ++gi) {
            const int a = start[gi], b = start[gi + 1];
            CHECK(b > a && b - a <= cap);
            for (int c = a; c < b; ++c) CHECK(k[c] == k[a]);
            if (b < n) CHECK(b - a == cap || k[b] != k[a]);
        }
    }
    std::printf("ok grouping\n");
}

static void tuner() {
    // the fastest, unless within the margin of the default
    const float a[3] = {1.0f, 0.996f, 0.99f};
    CHECK(tune_choose(a, 0.005f) == 2);
    const float b[3] = {1.0f, 0.997f, 0.998f};
    CHECK(tune_choose(b, 0.005f) == 0);
    const float c[3] = {1.0f, 0.96f, 0.98f};
    CHECK(tune_choose(c, 0.03f) == 1);
    const float d[3] = {1.0f, 0.975f, 0.99f};
    CHECK(tune_choose(d, 0.03f) == 0);
    const float e[3] = {0.9f, 1.0f, 1.1f};
    CHECK(tune_choose(e, 0.005f) == 0);
    const float f[3] = {1.0f, 0.9f, 0.9f};  // equal times: the first of them
    CHECK(tune_choose(f, 0.005f) == 1);
    std::printf("ok tuner\n");
}

int main() {
    tc_grid();
    group_cap();
    grouping();
    tuner();
    return 0;
}
