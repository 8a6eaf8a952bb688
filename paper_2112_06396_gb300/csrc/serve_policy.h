// serve_policy.h -- host-side policy of the serving loop: a first-fit arena for the
// per-request device workspace, and continuous batching with admission by
// device memory.  Plain C++ without CUDA, so the policy is unit-tested on the
// host; serve.cu drives it with streams and events.
//
// Memory model: the budget covers the resident keys (counted once, when a key
// is registered) plus, for every admitted request, its ciphertexts (inputs and
// outputs, owned by the caller but counted here) and its workspace, which is
// carved out of one device arena owned by the server.
//
// Batching: the server has `lanes` CUDA streams and each runs one batch at a
// time.  Whenever a lane is free and requests are pending, a batch is formed at
// once (no waiting for it to fill): the oldest pending request picks the
// context (ring degree), then pending requests of that context join in arrival
// order while the batch has room and memory admits them.  The first request of
// that context that does not fit ends the batch, so a context's requests are
// admitted in arrival order and a large request is never starved by smaller
// later ones.  Requests of other contexts wait for the next free lane.
#pragma once

#include <cstddef>
#include <cstdint>
#include <deque>
#include <iterator>
#include <map>
#include <vector>

namespace ckks {

class Arena {
  public:
    static constexpr size_t kAlign = 256;
    explicit Arena(size_t size) : size_(size / kAlign * kAlign) {
        if (size_) free_[0] = size_;
    }
    // First fit; false when no free block is large enough.
    bool alloc(size_t bytes, size_t *off) {
        const size_t need = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            *off = it->first;
            const size_t rest = it->second - need;
            const size_t at = it->first + need;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used_[*off] = need;
            in_use_ += need;
            return true;
        }
        return false;
    }
    // Returns false for an offset that is not allocated.
    bool release(size_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        size_t start = off, len = u->second;
        in_use_ -= len;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && start + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
        return true;
    }
    size_t size() const { return size_; }
    size_t in_use() const { return in_use_; }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto &f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    size_t free_blocks() const { return free_.size(); }
    static size_t round(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

  private:
    size_t size_;
    size_t in_use_ = 0;
    std::map<size_t, size_t> free_;  // offset -> length, disjoint, never adjacent
    std::map<size_t, size_t> used_;  // offset -> length
};

struct SchedReq {
    uint64_t id;
    int ctx;
    size_t ws_bytes;  // workspace, taken from the arena
    size_t ct_bytes;  // ciphertexts in and out, counted against the budget
};

struct Admitted {
    SchedReq r;
    size_t ws_off;
};

class Scheduler {
  public:
    Scheduler(size_t budget, size_t arena_bytes, int max_batch, int lanes)
        : budget_(budget), arena_(arena_bytes), max_batch_(max_batch), busy_(size_t(lanes), false) {}

    // Keys are resident for the server's lifetime; false if they exceed the budget.
    bool add_resident(size_t bytes) {
        if (resident_ + bytes + charged_ > budget_) return false;
        resident_ += bytes;
        return true;
    }
    // Whether a request could ever be admitted (alone, with nothing in flight).
    bool can_ever_fit(const SchedReq &r) const {
        return resident_ + Arena::round(r.ws_bytes) + r.ct_bytes <= budget_ && Arena::round(r.ws_bytes) <= arena_.size();
    }
    void submit(const SchedReq &r) { pending_.push_back(r); }

    // Forms the next batch on a free lane.  Returns the lane index, or -1 when
    // no lane is free, nothing is pending, or the oldest request does not fit.
    int next_batch(std::vector<Admitted> *out) {
        out->clear();
        int lane = -1;
        for (size_t i = 0; i < busy_.size(); ++i)
            if (!busy_[i]) {
                lane = int(i);
                break;
            }
        if (lane < 0 || pending_.empty()) return -1;
        const int ctx = pending_.front().ctx;
        for (auto it = pending_.begin(); it != pending_.end() && int(out->size()) < max_batch_;) {
            if (it->ctx != ctx) {
                ++it;
                continue;
            }
            const size_t ws = Arena::round(it->ws_bytes);
            size_t off = 0;
            if (resident_ + charged_ + ws + it->ct_bytes > budget_ || !arena_.alloc(it->ws_bytes, &off)) break;
            charged_ += ws + it->ct_bytes;
            out->push_back(Admitted{*it, off});
            it = pending_.erase(it);
        }
        if (out->empty()) return -1;
        busy_[size_t(lane)] = true;
        return lane;
    }

    // The batch that ran on `lane` has finished: release its memory and the lane.
    void complete(int lane, const std::vector<Admitted> &batch) {
        for (const auto &a : batch) {
            arena_.release(a.ws_off);
            charged_ -= Arena::round(a.r.ws_bytes) + a.r.ct_bytes;
        }
        busy_[size_t(lane)] = false;
    }

    size_t pending() const { return pending_.size(); }
    size_t charged() const { return charged_; }
    size_t resident() const { return resident_; }
    size_t budget() const { return budget_; }
    const Arena &arena() const { return arena_; }
    int lanes_busy() const {
        int n = 0;
        for (bool b : busy_) n += b;
        return n;
    }

  private:
    size_t budget_;
    Arena arena_;
    int max_batch_;
    std::vector<bool> busy_;
    std::deque<SchedReq> pending_;
    size_t resident_ = 0;
    size_t charged_ = 0;
};

}  // namespace ckks
