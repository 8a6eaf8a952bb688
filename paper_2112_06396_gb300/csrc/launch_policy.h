// launch_policy.h -- host-side launch decisions of the kernels, free of CUDA so
// that they can be checked on the host: how many CTAs the tensor-core basis
// conversion runs per (group, chunk), how the batched inner product groups the
// entries that share a compressed key, and which of its timed shapes the NTT
// autotuner keeps.
#pragma once

#include <algorithm>
#include <cstdint>

namespace ckks {
namespace policy {

// The SMs a launch counts on when the caller runs `concurrency` operations at
// once: all of them for an operation alone, 1/n of them for n.
inline int sm_share(int sms, int concurrency) { return std::max(1, sms / std::max(1, concurrency)); }

// CTAs per (group, chunk) row of the tensor-core conversion.  Each SM runs one
// CTA of it at a time and a CTA its tiles one after the other, so a launch of
// `rows` rows takes about waves * (ceil(tiles / per) + 2) tile times, the 2
// being a CTA's fixed cost (tensor-memory allocation, B image, pipeline fill),
// with the waves counted on `share` SMs.  The count that minimises it, ties to
// more CTAs; at most 256 and at most one per tile.
inline long tc_cost(int tiles, int rows, int share, int per) {
    const long waves = (long(rows) * per + share - 1) / share;
    return waves * ((tiles + per - 1) / per + 2);
}
inline int tc_ctas_per_row(int tiles, int rows, int share) {
    int per = 1;
    long best = -1;
    for (int c = 1; c <= std::min(tiles, 256); ++c) {
        const long cost = tc_cost(tiles, rows, share, c);
        if (best < 0 || cost <= best) {
            best = cost;
            per = c;
        }
    }
    return per;
}

// Longest group of the batched inner product with a compressed key: as long as
// the launch keeps at least 8 CTAs per SM (ctas_per_entry CTAs per entry of an
// n-entry launch), at most cap_max; groups of one with more than 4 digits,
// whose key rows are not held in registers.
inline int ip_group_cap(long ctas_per_entry, int n, int sms, int dnum, int cap_max) {
    if (dnum > 4) return 1;
    const long fill = std::max(1L, ctas_per_entry * n / (8L * std::max(1, sms)));
    return int(std::min<long>(fill, cap_max));
}

// Cuts entries 0 .. n-1 into groups of consecutive entries for which
// same(first entry of the group, entry) holds, each at most `cap` long: group g
// is start[g] .. start[g+1]-1.  Returns the number of groups; start holds n+1
// slots at most.
template <class Same>
inline int ip_groups(int n, int cap, Same same, uint8_t *start) {
    int g = 0;
    start[0] = 0;
    for (int c = 1; c <= n; ++c) {
        if (c == n || c - start[g] >= cap || !same(int(start[g]), c)) start[++g] = uint8_t(c);
    }
    return g;
}

// The NTT autotuner's pick among three timed options, option 0 the default:
// the fastest, unless it beats the default by less than `margin` (a fraction),
// since closer timings are within the spread of launches timed alone.
inline int tune_choose(const float *t, float margin) {
    int f = 0;
    for (int o = 1; o < 3; ++o)
        if (t[o] < t[f]) f = o;
    return t[f] < t[0] * (1.f - margin) ? f : 0;
}

}  // namespace policy
}  // namespace ckks
