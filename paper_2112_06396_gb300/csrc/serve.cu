// serve.cu -- the serving loop: continuous batching of HRotate, KeySwitch and
// Mult (with relinearisation and Rescale) requests of mixed ring degree and
// level, admitted by device memory, each batch run by the batch executor on
// one of several streams so that batches overlap on the GPU.
//
// The caller drives the loop: ckks_server_submit() queues a request (its
// ciphertexts already on the device), ckks_server_step() retires finished
// batches and launches new ones on free streams, ckks_server_poll() hands back
// the finished requests with their latency.  Nothing blocks: completion is
// read from CUDA events.  Latency = device completion time - arrival time, on
// one clock: at creation the server synchronises the device, records an origin
// event and reads the host clock, so event times and host times share t = 0.
// The admission and batching policy lives in serve_policy.h.
//
// Device-side failures of a batch: each lane (stream) has its own status word,
// cleared before the lane's batch and handed to every kernel of the batch that
// has a bounded wait (the tensor-core basis conversion); after the batch its
// value is copied to pinned host memory on the lane, before the lane's
// completion event.  When the event has completed the host reads the copy, and
// a set word marks every request of that batch as failed (CKKS_ETIMEOUT): its
// outputs are not valid.  Lanes never share a word, so a timeout is charged to
// the batch that had it.
#include "../../include/ckks_ks.h"
#include "internal.h"
#include "serve_policy.h"

#include <chrono>
#include <deque>
#include <unordered_map>
#include <vector>

using namespace ckks;

namespace {
struct Done {
    uint64_t id;
    double arrival_ms, done_ms;
    int status;  // CKKS_OK, or CKKS_ETIMEOUT when a bounded wait of its batch ran out
};
}  // namespace

struct ckks_server {
    int device = 0;
    std::vector<ckks_ctx *> ctxs;
    struct Key {
        int ctx;
        const u64 *ptr;
        int compressed;
        u64 seed;
    };
    std::vector<Key> keys;
    void *arena = nullptr;
    Scheduler *sched = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    std::vector<std::vector<Admitted>> lane_batch;
    std::unordered_map<uint64_t, ckks_request> reqs;
    std::deque<Done> finished;
    cudaEvent_t origin = nullptr;
    int *d_status = nullptr;  // [nstreams] device status words, one per lane
    int *h_status = nullptr;  // [nstreams] pinned host copies, valid once the lane's event completed
    uint32_t inject_wait_us = 0;  // test hook: the next batch also runs the bounded-wait self-test
    std::chrono::steady_clock::time_point t0;
    uint64_t next_id = 1;
    int last_cuda_error = 0;
    long long batches = 0, launched = 0;
};

static bool al16(const void *p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static double host_ms(const ckks_server *s) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s->t0).count();
}

#define SCK(call)                                                                                                 \
    do {                                                                                                          \
        cudaError_t e_ = (call);                                                                                  \
        if (e_ != cudaSuccess) {                                                                                  \
            s->last_cuda_error = int(e_);                                                                         \
            return CKKS_ECUDA;                                                                                    \
        }                                                                                                         \
    } while (0)

static void destroy(ckks_server *s) {
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto ev : s->done)
        if (ev) cudaEventDestroy(ev);
    if (s->origin) cudaEventDestroy(s->origin);
    if (s->arena) cudaFree(s->arena);
    if (s->d_status) cudaFree(s->d_status);
    if (s->h_status) cudaFreeHost(s->h_status);
    delete s->sched;
    delete s;
}

extern "C" int ckks_server_create(ckks_ctx *const *ctxs, int nctx, size_t mem_budget, int max_batch, int nstreams,
                                  ckks_server **out) {
    if (out == nullptr || ctxs == nullptr || nctx < 1 || max_batch < 1 || nstreams < 1 || nstreams > 64 ||
        mem_budget < Arena::kAlign)
        return CKKS_EINVAL;
    for (int i = 0; i < nctx; ++i)
        if (ctxs[i] == nullptr || ctxs[i]->device != ctxs[0]->device) return CKKS_EINVAL;
    ckks_server *s = new ckks_server;
    s->device = ctxs[0]->device;
    s->ctxs.assign(ctxs, ctxs + nctx);
    int prev = 0;
    cudaGetDevice(&prev);
    auto fail = [&](cudaError_t e) {
        cudaGetLastError();  // an allocation failure is not sticky: clear it for the caller
        cudaSetDevice(prev);
        destroy(s);
        return e == cudaErrorMemoryAllocation ? CKKS_ENOMEM : CKKS_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaSetDevice(s->device)) != cudaSuccess) return fail(e);
    // the workspace arena: one allocation, made here and nowhere else
    const size_t arena = mem_budget / Arena::kAlign * Arena::kAlign;
    if ((e = cudaMalloc(&s->arena, arena)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&s->d_status, size_t(nstreams) * sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(s->d_status, 0, size_t(nstreams) * sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_status), size_t(nstreams) * sizeof(int),
                           cudaHostAllocDefault)) != cudaSuccess)
        return fail(e);
    for (int i = 0; i < nstreams; ++i) s->h_status[i] = 0;
    s->sched = new Scheduler(mem_budget, arena, max_batch, nstreams);
    s->streams.assign(size_t(nstreams), nullptr);
    s->done.assign(size_t(nstreams), nullptr);
    s->lane_batch.resize(size_t(nstreams));
    for (int i = 0; i < nstreams; ++i) {
        if ((e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
        if ((e = cudaEventCreate(&s->done[i])) != cudaSuccess) return fail(e);
    }
    if ((e = cudaEventCreate(&s->origin)) != cudaSuccess) return fail(e);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
    if ((e = cudaEventRecord(s->origin, s->streams[0])) != cudaSuccess) return fail(e);
    if ((e = cudaEventSynchronize(s->origin)) != cudaSuccess) return fail(e);
    s->t0 = std::chrono::steady_clock::now();
    if ((e = cudaSetDevice(prev)) != cudaSuccess) return fail(e);
    *out = s;
    return CKKS_OK;
}

extern "C" int ckks_server_destroy(ckks_server *s) {
    if (s == nullptr) return CKKS_EINVAL;
    for (auto st : s->streams)
        if (st) cudaStreamSynchronize(st);
    destroy(s);
    return CKKS_OK;
}

static int add_key(ckks_server *s, int ctx, const uint64_t *d_key, int compressed, u64 seed, int *handle) {
    if (s == nullptr || handle == nullptr || ctx < 0 || ctx >= int(s->ctxs.size()) || !al16(d_key))
        return CKKS_EINVAL;
    const ckks_ctx *c = s->ctxs[size_t(ctx)];
    const size_t bytes = size_t(c->dnum) * (compressed ? 1 : 2) * (c->L + c->k) * c->N * sizeof(u64);
    if (!s->sched->add_resident(bytes)) return CKKS_ENOMEM;
    s->keys.push_back({ctx, d_key, compressed, seed});
    *handle = int(s->keys.size()) - 1;
    return CKKS_OK;
}

extern "C" int ckks_server_add_key(ckks_server *s, int ctx, const uint64_t *d_key, int *handle) {
    if (s != nullptr && ctx >= 0 && ctx < int(s->ctxs.size())) {
        // a key registered as compressed with its context
        const auto &m = s->ctxs[size_t(ctx)]->comp_keys;
        const auto it = m.find(d_key);
        if (it != m.end()) return add_key(s, ctx, d_key, 1, it->second, handle);
    }
    return add_key(s, ctx, d_key, 0, 0, handle);
}

extern "C" int ckks_server_add_key_seeded(ckks_server *s, int ctx, const uint64_t *d_key_b, uint64_t seed,
                                          int *handle) {
    return add_key(s, ctx, d_key_b, 1, seed, handle);
}

extern "C" double ckks_server_now_ms(const ckks_server *s) { return s ? host_ms(s) : 0.0; }

static size_t ct_bytes(const ckks_ctx *c, int op, int ell) {
    const size_t limb = size_t(c->N) * sizeof(u64);
    switch (op) {
    case CKKS_REQ_HROTATE: return size_t(4) * ell * limb;
    case CKKS_REQ_KEYSWITCH: return size_t(3) * ell * limb;
    default: return (size_t(4) * ell + size_t(2) * (ell - 1)) * limb;
    }
}
static int kind_of(int op) {
    switch (op) {
    case CKKS_REQ_HROTATE: return BE_HROTATE;
    case CKKS_REQ_MULT: return BE_MULT;
    case CKKS_REQ_NEWMULT: return BE_NEWMULT;
    default: return BE_KEYSWITCH;
    }
}

extern "C" int ckks_server_submit(ckks_server *s, const ckks_request *r, uint64_t *id) {
    if (s == nullptr || r == nullptr || id == nullptr) return CKKS_EINVAL;
    if (r->ctx < 0 || r->ctx >= int(s->ctxs.size())) return CKKS_EINVAL;
    if (r->op != CKKS_REQ_HROTATE && r->op != CKKS_REQ_MULT && r->op != CKKS_REQ_KEYSWITCH &&
        r->op != CKKS_REQ_NEWMULT)
        return CKKS_EINVAL;
    const ckks_ctx *c = s->ctxs[size_t(r->ctx)];
    const bool mult = r->op == CKKS_REQ_MULT || r->op == CKKS_REQ_NEWMULT;
    if (r->op == CKKS_REQ_NEWMULT && c->k + 1 > kMaxSrc) return CKKS_EUNSUPPORTED;
    const int min_level = mult ? 2 : 1;
    if (r->level < min_level || r->level > c->L) return CKKS_EINVAL;
    if (r->key < 0 || r->key >= int(s->keys.size()) || s->keys[size_t(r->key)].ctx != r->ctx) return CKKS_EINVAL;
    if (!al16(r->a) || !al16(r->oa) || !al16(r->ob)) return CKKS_EINVAL;
    if (r->op != CKKS_REQ_KEYSWITCH && !al16(r->b)) return CKKS_EINVAL;
    if (mult && (!al16(r->a2) || !al16(r->b2))) return CKKS_EINVAL;
    if (r->op == CKKS_REQ_HROTATE && (!(r->galois & 1u) || r->galois >= uint32_t(2 * c->N))) return CKKS_EINVAL;
    SchedReq q{s->next_id, r->ctx, entry_ws_words(c, kind_of(r->op), r->level) * sizeof(u64),
               ct_bytes(c, r->op, r->level)};
    if (!s->sched->can_ever_fit(q)) return CKKS_ENOMEM;
    ckks_request copy = *r;
    if (copy.arrival_ms < 0) copy.arrival_ms = host_ms(s);
    s->reqs[q.id] = copy;
    s->sched->submit(q);
    *id = s->next_id++;
    return CKKS_OK;
}

extern "C" int ckks_server_step(ckks_server *s, int *n_launched) {
    if (s == nullptr) return CKKS_EINVAL;
    int launched = 0;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != s->device) SCK(cudaSetDevice(s->device));
    int rc = CKKS_OK;
    // retire finished batches
    for (size_t lane = 0; lane < s->streams.size() && rc == CKKS_OK; ++lane) {
        auto &batch = s->lane_batch[lane];
        if (batch.empty()) continue;
        const cudaError_t q = cudaEventQuery(s->done[lane]);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            s->last_cuda_error = int(q);
            rc = CKKS_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->origin, s->done[lane]);
        const int status = s->h_status[lane] != 0 ? CKKS_ETIMEOUT : CKKS_OK;
        s->h_status[lane] = 0;
        for (const auto &a : batch) {
            auto it = s->reqs.find(a.r.id);
            s->finished.push_back({a.r.id, it->second.arrival_ms, double(ms), status});
            s->reqs.erase(it);
        }
        s->sched->complete(int(lane), batch);
        batch.clear();
    }
    // launch new batches on free lanes
    std::vector<Admitted> adm;
    std::vector<BatchEntry> ent;
    while (rc == CKKS_OK) {
        const int lane = s->sched->next_batch(&adm);
        if (lane < 0) break;
        ckks_ctx *c = s->ctxs[size_t(s->reqs[adm[0].r.id].ctx)];
        ent.clear();
        for (const auto &a : adm) {
            const ckks_request &r = s->reqs[a.r.id];
            BatchEntry be{};
            be.kind = kind_of(r.op);
            be.a = r.a;
            be.b = r.op == CKKS_REQ_KEYSWITCH ? nullptr : r.b;
            be.a2 = r.a2;
            be.b2 = r.b2;
            be.key = s->keys[size_t(r.key)].ptr;
            be.compressed = s->keys[size_t(r.key)].compressed;
            be.seed = s->keys[size_t(r.key)].seed;
            be.oa = r.oa;
            be.ob = r.ob;
            be.ell = r.level;
            be.galois = r.op == CKKS_REQ_HROTATE ? r.galois : 1u;
            be.ws = reinterpret_cast<u64 *>(static_cast<char *>(s->arena) + a.ws_off);
            ent.push_back(be);
        }
        cudaStream_t st = s->streams[size_t(lane)];
        int *lane_status = s->d_status + lane;
        cudaError_t e = cudaMemsetAsync(lane_status, 0, sizeof(int), st);
        if (e == cudaSuccess && s->inject_wait_us != 0) {
            e = launch_bounded_wait_selftest(c, uint64_t(s->inject_wait_us) * 1000u, st, lane_status);
            s->inject_wait_us = 0;
        }
        if (e != cudaSuccess) {
            s->last_cuda_error = int(e);
            rc = CKKS_ECUDA;
        } else {
            rc = run_batch(c, int(ent.size()), ent.data(), nullptr, st, lane_status);
            if (rc != CKKS_OK) s->last_cuda_error = c->last_cuda_error;
        }
        if (rc == CKKS_OK) {
            e = cudaMemcpyAsync(s->h_status + lane, lane_status, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(s->done[size_t(lane)], st);
            if (e != cudaSuccess) {
                s->last_cuda_error = int(e);
                rc = CKKS_ECUDA;
            }
        }
        s->lane_batch[size_t(lane)] = adm;
        s->batches += 1;
        launched += int(adm.size());
    }
    s->launched += launched;
    if (prev != s->device) {
        const cudaError_t e = cudaSetDevice(prev);
        if (e != cudaSuccess && rc == CKKS_OK) {
            s->last_cuda_error = int(e);
            rc = CKKS_ECUDA;
        }
    }
    if (n_launched) *n_launched = launched;
    return rc;
}

extern "C" int ckks_server_poll(ckks_server *s, int max, uint64_t *ids, double *latency_ms, double *done_ms,
                                int *status, int *n) {
    if (s == nullptr || n == nullptr || max < 0 || (max > 0 && ids == nullptr)) return CKKS_EINVAL;
    int k = 0;
    while (k < max && !s->finished.empty()) {
        const Done d = s->finished.front();
        s->finished.pop_front();
        ids[k] = d.id;
        if (latency_ms) latency_ms[k] = d.done_ms - d.arrival_ms;
        if (done_ms) done_ms[k] = d.done_ms;
        if (status) status[k] = d.status;
        ++k;
    }
    *n = k;
    return CKKS_OK;
}

extern "C" int ckks_server_selftest_timeout(ckks_server *s, uint32_t limit_us) {
    if (s == nullptr || limit_us == 0 || limit_us > 2000000u) return CKKS_EINVAL;
    s->inject_wait_us = limit_us;
    return CKKS_OK;
}

extern "C" int ckks_server_stats(const ckks_server *s, ckks_server_stats_t *st) {
    if (s == nullptr || st == nullptr) return CKKS_EINVAL;
    st->pending = int(s->sched->pending());
    int inflight = 0;
    for (const auto &b : s->lane_batch) inflight += int(b.size());
    st->in_flight = inflight;
    st->finished_unpolled = int(s->finished.size());
    st->lanes_busy = s->sched->lanes_busy();
    st->mem_budget = s->sched->budget();
    st->mem_keys = s->sched->resident();
    st->mem_in_flight = s->sched->charged();
    st->batches = s->batches;
    st->requests_launched = s->launched;
    st->last_cuda_error = s->last_cuda_error;
    return CKKS_OK;
}
