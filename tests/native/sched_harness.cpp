// Host-side checks of the serving loop's arena and batching policy (serve_policy.h).
// Built and run by tests/test_sched_host.py; prints "ok <name>" per check and
// exits non-zero at the first failure.
#include "serve_policy.h"

#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>

using namespace ckks;

#define CHECK(cond)                                                                     \
    do {                                                                                \
        if (!(cond)) {                                                                  \
            std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #cond);                 \
            std::exit(1);                                                               \
        }                                                                               \
    } while (0)

static void arena_basic() {
    Arena a(4096);
    size_t o1, o2, o3, o4;
    CHECK(a.alloc(100, &o1) && o1 == 0);
    CHECK(a.alloc(256, &o2) && o2 == 256);
    CHECK(a.alloc(1000, &o3) && o3 == 512);
    CHECK(a.in_use() == 256 + 256 + 1024);
    CHECK(!a.alloc(4096, &o4));
    CHECK(a.release(o2));
    CHECK(!a.release(o2));  // double free is refused
    CHECK(a.alloc(200, &o4) && o4 == 256);  // first fit reuses the hole
    CHECK(a.release(o1) && a.release(o4) && a.release(o3));
    CHECK(a.in_use() == 0 && a.free_blocks() == 1 && a.largest_free() == 4096);  // fully coalesced
    std::printf("ok arena_basic\n");
}

static void arena_random() {
    // random alloc/free never overlaps, stays aligned and coalesces back to one block
    Arena a(1 << 20);
    std::mt19937_64 rng(2112063960);
    std::vector<std::pair<size_t, size_t>> live;
    for (int it = 0; it < 20000; ++it) {
        if (live.empty() || (rng() % 3 != 0)) {
            const size_t b = 1 + rng() % 20000;
            size_t off;
            if (a.alloc(b, &off)) {
                CHECK(off % Arena::kAlign == 0 && off + b <= a.size());
                for (auto &l : live) CHECK(off + b <= l.first || l.first + l.second <= off);
                live.push_back({off, b});
            }
        } else {
            const size_t i = rng() % live.size();
            CHECK(a.release(live[i].first));
            live.erase(live.begin() + long(i));
        }
    }
    for (auto &l : live) CHECK(a.release(l.first));
    CHECK(a.in_use() == 0 && a.free_blocks() == 1);
    std::printf("ok arena_random\n");
}

static SchedReq R(uint64_t id, int ctx, size_t ws, size_t ct) { return SchedReq{id, ctx, ws, ct}; }

static void batching_policy() {
    // budget 10000: keys 2000; workspace arena 8192
    Scheduler s(10000, 8192, 3, 2);
    CHECK(s.add_resident(2000));
    CHECK(!s.add_resident(9000));
    for (uint64_t i = 1; i <= 5; ++i) s.submit(R(i, i == 2 ? 1 : 0, 1000, 500));
    std::vector<Admitted> b;
    // oldest (id 1, ctx 0) picks the context; ctx-0 requests join in order up to max_batch
    int lane = s.next_batch(&b);
    CHECK(lane == 0 && b.size() == 3 && b[0].r.id == 1 && b[1].r.id == 3 && b[2].r.id == 4);
    CHECK(s.charged() == 3 * (1024 + 500));
    // next lane: oldest is id 2 (ctx 1); id 5 (ctx 0) waits
    std::vector<Admitted> b2;
    lane = s.next_batch(&b2);
    CHECK(lane == 1 && b2.size() == 1 && b2[0].r.id == 2);
    // no free lane
    std::vector<Admitted> b3;
    CHECK(s.next_batch(&b3) == -1 && s.pending() == 1);
    s.complete(0, b);
    CHECK(s.next_batch(&b3) == 0 && b3.size() == 1 && b3[0].r.id == 5);
    s.complete(1, b2);
    s.complete(0, b3);
    CHECK(s.charged() == 0 && s.arena().in_use() == 0 && s.lanes_busy() == 0);
    std::printf("ok batching_policy\n");
}

static void memory_admission() {
    // budget allows two requests in flight at a time
    Scheduler s(5000, 8192, 8, 4);
    CHECK(s.add_resident(1000));
    for (uint64_t i = 1; i <= 4; ++i) s.submit(R(i, 0, 1500, 400));  // 1536 + 400 each
    std::vector<Admitted> b;
    CHECK(s.next_batch(&b) == 0 && b.size() == 2);  // 1000 + 2*1936 = 4872 <= 5000; a third would not fit
    std::vector<Admitted> b2;
    CHECK(s.next_batch(&b2) == -1);  // a free lane, but the oldest pending request does not fit
    s.complete(0, b);
    CHECK(s.next_batch(&b2) == 0 && b2.size() == 2 && b2[0].r.id == 3 && b2[1].r.id == 4);
    CHECK(!s.can_ever_fit(R(9, 0, 4000, 100)));
    CHECK(s.can_ever_fit(R(9, 0, 3000, 900)));
    std::printf("ok memory_admission\n");
}

static void fifo_within_context() {
    // a large request at the head of its context is not bypassed by later small ones
    Scheduler s(100000, 8192, 8, 2);
    s.submit(R(1, 0, 6000, 0));
    s.submit(R(2, 0, 6000, 0));  // does not fit beside 1 in the arena
    s.submit(R(3, 0, 100, 0));
    std::vector<Admitted> b;
    CHECK(s.next_batch(&b) == 0 && b.size() == 1 && b[0].r.id == 1);
    std::vector<Admitted> b2;
    CHECK(s.next_batch(&b2) == -1);  // 2 waits for memory and 3 stays behind it
    s.complete(0, b);
    CHECK(s.next_batch(&b2) == 0 && b2.size() == 2 && b2[0].r.id == 2 && b2[1].r.id == 3);
    std::printf("ok fifo_within_context\n");
}

static void random_load() {
    // every request is admitted exactly once; memory never exceeds the budget
    Scheduler s(200000, 150000, 16, 4);
    CHECK(s.add_resident(20000));
    std::mt19937_64 rng(7);
    std::set<uint64_t> seen;
    std::vector<std::pair<int, std::vector<Admitted>>> inflight;
    uint64_t next = 1, total = 3000;
    while (seen.size() < total) {
        for (int k = int(rng() % 4); k > 0 && next <= total; --k)
            s.submit(R(next++, int(rng() % 2), 1000 + rng() % 30000, rng() % 10000));
        std::vector<Admitted> b;
        int lane;
        while ((lane = s.next_batch(&b)) >= 0) {
            CHECK(s.resident() + s.charged() <= s.budget());
            for (auto &a : b) {
                CHECK(seen.insert(a.r.id).second);
                CHECK(a.r.ctx == b[0].r.ctx);
            }
            inflight.push_back({lane, b});
        }
        if (!inflight.empty() && (rng() % 2 == 0 || next > total)) {
            const size_t i = rng() % inflight.size();
            s.complete(inflight[i].first, inflight[i].second);
            inflight.erase(inflight.begin() + long(i));
        }
    }
    for (auto &f : inflight) s.complete(f.first, f.second);
    CHECK(s.charged() == 0 && s.pending() == 0 && s.arena().in_use() == 0);
    std::printf("ok random_load\n");
}

int main() {
    arena_basic();
    arena_random();
    batching_policy();
    memory_admission();
    fifo_within_context();
    random_load();
    return 0;
}
