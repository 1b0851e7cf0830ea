// Continuous-batching solve server (rcpsp_server_*): requests that arrive
// while others run are admitted as launch slots and device memory free up,
// and their searches overlap on the GPU.
//
// A worker thread owns K library contexts, each with its own non-blocking
// stream; a context runs at most one batch (one rcpsp_tabu_search call).
// Submitting validates the instance on the caller's thread (the host
// preparation of rcpsp_load_instances) and queues it with its device
// footprint.  The worker loop
//   1. harvests every context whose batch finished: copies the results,
//      frees the batch's device memory, returns its footprint to the budget
//      and publishes one completion per request;
//   2. fills every free context with a batch: the launch class whose oldest
//      request is oldest, then its requests in arrival order with identical
//      search parameters, while the footprint fits the budget (a lone request
//      is admitted even if larger), up to a batch size that shrinks with the
//      instance size (256 / 96 / 32) and max_batch;
//   3. sleeps on a condition variable until a submission or the next poll
//      tick (no GPU spin: completion is an event query).
// With slice_iterations > 0 a request of more iterations runs in slices:
// each slice keeps the search state (rcpsp_params.checkpoint); at harvest an
// unfinished request takes its state to the host (rcpsp_get_state) and goes
// back to the end of its class queue, and its next batch restores the state
// (rcpsp_set_state) and resumes.  The slices add up to exactly the
// uninterrupted search.
// Searches are deterministic and independent per instance, so a request's
// result does not depend on what else is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rcpsp.h"
#include "host_prep.h"

#include "kernels.h"

namespace rcpsp {
int ctx_search_done(rcpsp_ctx *c);
int ctx_reserve(rcpsp_ctx *c, size_t staging_bytes, int plan_items);
}

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t tag = 0;
    int cls = 0;                 // launch class (footprint x size), as the search groups them
    rcpsp_params params{};
    int32_t n = 0, m = 0;
    std::vector<int32_t> dur, cap, req, succ_off, succ, key;
    bool has_key = false;
    int64_t bytes = 0;
    int64_t t_submit = 0;
    int32_t total_iters = 0;     // iterations asked for
    std::vector<char> state;     // kept search state between slices (empty: fresh)
    rcpsp_instance view() const {
        rcpsp_instance in;
        in.n = n;
        in.m = m;
        in.dur = dur.data();
        in.cap = cap.data();
        in.req = req.data();
        in.succ_off = succ_off.data();
        in.succ = succ.data();
        in.level_key = has_key ? key.data() : nullptr;
        return in;
    }
};

struct Completion {
    rcpsp_completion c{};
    std::vector<int32_t> W, S;
};

// Device memory of one slot: stream-ordered allocations on the slot's own
// stream from the server's pool.
struct SlotMem {
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
};

struct Slot {
    rcpsp_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    SlotMem mem;
    bool busy = false;
    std::vector<Request> reqs;
    std::vector<int32_t> ids;
    int64_t bytes = 0;
    int64_t t_launch = 0;
    int cls = -1;                // launch class of the batch in flight
};

bool same_params(const rcpsp_params &a, const rcpsp_params &b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

// Device memory of a slot: stream-ordered on the slot's own stream, from a
// pool that keeps up to the memory budget mapped between batches (no
// remapping on the request path), made ready before the upload that
// follows it.
void *slot_alloc(size_t bytes, void *, void *user) {
    const SlotMem *m = static_cast<const SlotMem *>(user);
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, m->pool, m->stream) != cudaSuccess) return nullptr;
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return nullptr;
    return p;
}

void slot_release(void *ptr, size_t, void *, void *user) {
    cudaFreeAsync(ptr, static_cast<const SlotMem *>(user)->stream);
}

}  // namespace

struct rcpsp_server {
    int device = 0;
    rcpsp_server_config cfg{};
    std::vector<Slot> slots;
    std::vector<rcpsp_allocator> allocs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending[rcpsp::kLaunchClasses];   // one FIFO per launch class
    std::deque<Completion> done;
    std::vector<Completion> handed;      // returned by the last poll, owned until the next one
    std::thread worker;
    cudaMemPool_t pool = nullptr;        // device memory of every slot
    std::atomic<bool> stop{false};
    int64_t inflight_bytes = 0;
    rcpsp_server_stats st{};
    std::string err;
    int fatal = RCPSP_OK;
};

namespace {

int64_t footprint(const rcpsp::PackedInstance &pk) {
    return static_cast<int64_t>(pk.h.record_words) * 4 + static_cast<int64_t>(rcpsp::align4(2 * pk.h.n + rcpsp::kOutStats)) * 4 +
           static_cast<int64_t>(sizeof(rcpsp::LaunchItem));
}

// Parameters of a request's next slice: `done` iterations are behind it.
void slice_params(const rcpsp_server *s, Request &r, int32_t done) {
    const int32_t left = r.total_iters - done;
    const int32_t sl = s->cfg.slice_iterations;
    r.params.iterations = sl > 0 ? std::min(left, sl) : left;
    r.params.checkpoint = sl > 0 && left > sl ? 1 : 0;
    r.params.resume = done > 0 ? 1 : 0;
}

void harvest(rcpsp_server *s, Slot &sl) {
    const int cnt = static_cast<int>(sl.ids.size());
    int total_n = 0;
    for (const Request &r : sl.reqs) total_n += r.n;
    std::vector<int32_t> W(total_n), S(total_n), cm(cnt);
    std::vector<rcpsp_stats> stats(cnt);
    const int rc = rcpsp_get_schedules(sl.ctx, sl.ids.data(), cnt, W.data(), S.data(), cm.data(), stats.data());
    const int64_t t = now_ns();
    std::vector<Completion> out;
    std::vector<Request> again;                  // unfinished slices, back to their queues
    out.reserve(cnt);
    int at = 0;
    for (int k = 0; k < cnt; ++k) {
        Request &r = sl.reqs[k];
        const bool stopped = r.params.stop_at_cp && cm[k] == stats[k].critical_path;
        if (rc == RCPSP_OK && stats[k].status == RCPSP_OK && r.params.checkpoint && !stopped &&
            stats[k].iterations < r.total_iters) {
            size_t bytes = 0;
            if (rcpsp_get_state(sl.ctx, sl.ids[k], nullptr, 0, &bytes) == RCPSP_OK) {
                r.state.resize(bytes);
                if (rcpsp_get_state(sl.ctx, sl.ids[k], r.state.data(), bytes, &bytes) == RCPSP_OK) {
                    slice_params(s, r, stats[k].iterations);
                    at += r.n;
                    again.push_back(std::move(r));
                    continue;
                }
            }
        }
        out.emplace_back();
        Completion &c = out.back();
        c.W.assign(W.begin() + at, W.begin() + at + r.n);
        c.S.assign(S.begin() + at, S.begin() + at + r.n);
        at += r.n;
        c.c.tag = r.tag;
        c.c.n = r.n;
        c.c.status = rc == RCPSP_OK ? stats[k].status : rc;
        c.c.best_cmax = cm[k];
        c.c.iterations = stats[k].iterations;
        c.c.eval_mode = stats[k].eval_mode;
        c.c.critical_path = stats[k].critical_path;
        c.c.evaluated = stats[k].evaluated;
        c.c.work = stats[k].work;
        c.c.t_submit_ns = r.t_submit;
        c.c.t_launch_ns = sl.t_launch;
        c.c.t_done_ns = t;
    }
    rcpsp_free_instances(sl.ctx, sl.ids.data(), cnt);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Completion &c : out) {
            s->st.completed++;
            s->st.evaluated += c.c.evaluated;
            s->done.push_back(std::move(c));
        }
        s->inflight_bytes -= sl.bytes;
        s->st.inflight_requests -= cnt;
        for (Request &r : again) {
            s->st.requeued++;
            s->pending[r.cls].push_back(std::move(r));
        }
    }
    s->cv_done.notify_all();
    sl.busy = false;
    sl.reqs.clear();
    sl.ids.clear();
    sl.bytes = 0;
}

// Launch class of a request: footprint (per-group scratch words up to 512,
// 2K, 8K, more) times size (N up to 64, 160, more), as rcpsp_tabu_search
// splits a call (rcpsp::launch_class).  Batches take one class, so small requests do not wait for the
// completion of large ones, and large requests come in small batches that
// can share clusters of CTAs.
int request_class(const rcpsp::PackedInstance &pk, const rcpsp_params &p) {
    const int mode = p.eval_mode == RCPSP_EVAL_AUTO ? pk.h.sel_mode : p.eval_mode;
    const int pw = rcpsp::profile_words(mode, pk.h.wps, pk.h.ub, pk.h.sum_cap);
    return rcpsp::launch_class(rcpsp::group_area_words(mode, pw, pk.h.n), pk.h.n);
}

int batch_limit(const rcpsp_server *s, int cls) {
    const int sz = cls % 3;
    return std::max(1, std::min(s->cfg.max_batch, sz == 0 ? 256 : (sz == 1 ? 96 : 32)));
}

// Takes a batch for a free slot: the class whose oldest request is oldest,
// then that class's requests in arrival order with the same parameters.
// Batches of the largest size class hold at most half of the slots, so that
// long searches cannot keep short ones waiting.  False when nothing can be
// admitted now.
bool admit(rcpsp_server *s, Slot &sl) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        int large_busy = 0;
        for (const Slot &o : s->slots) large_busy += o.busy && o.cls % 3 == 2;
        const bool large_ok = 2 * (large_busy + 1) <= static_cast<int>(s->slots.size()) || large_busy == 0;
        int cls = -1;
        for (int q = 0; q < rcpsp::kLaunchClasses; ++q)
            if (!s->pending[q].empty() && (large_ok || q % 3 != 2) &&
                (cls < 0 || s->pending[q].front().t_submit < s->pending[cls].front().t_submit))
                cls = q;
        if (cls < 0) return false;
        std::deque<Request> &pq = s->pending[cls];
        const rcpsp_params p0 = pq.front().params;
        const int lim = batch_limit(s, cls);
        while (!pq.empty() && static_cast<int>(sl.reqs.size()) < lim) {
            Request &r = pq.front();
            if (!same_params(r.params, p0)) break;
            const bool lone = s->inflight_bytes == 0 && sl.reqs.empty();
            if (!lone && s->inflight_bytes + r.bytes > s->cfg.memory_budget) break;
            s->inflight_bytes += r.bytes;
            sl.bytes += r.bytes;
            sl.reqs.push_back(std::move(r));
            pq.pop_front();
        }
        if (sl.reqs.empty()) return false;
        sl.cls = cls;
        s->st.admitted += static_cast<int64_t>(sl.reqs.size());
        s->st.inflight_requests += static_cast<int64_t>(sl.reqs.size());
        s->st.batches++;
        s->st.max_inflight_bytes = std::max(s->st.max_inflight_bytes, s->inflight_bytes);
    }
    std::vector<rcpsp_instance> views;
    for (const Request &r : sl.reqs) views.push_back(r.view());
    sl.ids.assign(views.size(), 0);
    int rc = rcpsp_load_instances(sl.ctx, views.data(), static_cast<int32_t>(views.size()), sl.ids.data());
    for (size_t k = 0; rc == RCPSP_OK && k < sl.reqs.size(); ++k)
        if (!sl.reqs[k].state.empty())
            rc = rcpsp_set_state(sl.ctx, sl.ids[k], sl.reqs[k].state.data(), sl.reqs[k].state.size());
    if (rc == RCPSP_OK) {
        sl.t_launch = now_ns();
        rc = rcpsp_tabu_search(sl.ctx, sl.ids.data(), static_cast<int32_t>(sl.ids.size()), &sl.reqs[0].params,
                               sl.stream);
    }
    if (rc != RCPSP_OK) {
        // report every request of the batch as failed
        const int64_t t = now_ns();
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Request &r : sl.reqs) {
            Completion c;
            c.c.tag = r.tag;
            c.c.n = r.n;
            c.c.status = rc;
            c.c.t_submit_ns = r.t_submit;
            c.c.t_done_ns = t;
            s->st.completed++;
            s->done.push_back(std::move(c));
        }
        s->inflight_bytes -= sl.bytes;
        s->st.inflight_requests -= static_cast<int64_t>(sl.reqs.size());
        s->err = rcpsp_last_error(sl.ctx);
        sl.reqs.clear();
        sl.bytes = 0;
        s->cv_done.notify_all();
        return false;
    }
    sl.busy = true;
    return true;
}

void run(rcpsp_server *s) {
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        bool progress = false;
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            const int d = rcpsp::ctx_search_done(sl.ctx);
            if (d != 0) {
                harvest(s, sl);                           // also reports device errors per request
                progress = true;
            }
        }
        for (Slot &sl : s->slots)
            if (!sl.busy && admit(s, sl)) progress = true;
        if (!progress) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait_for(lk, std::chrono::microseconds(s->cfg.poll_us), [&] {
                if (s->stop.load()) return true;
                for (const auto &q : s->pending)
                    if (!q.empty()) return true;
                return false;
            });
        }
    }
}

}  // namespace

extern "C" {

int rcpsp_server_create(rcpsp_server **out, int device, const rcpsp_server_config *cfg) {
    if (!out) return RCPSP_E_INVALID_ARG;
    *out = nullptr;
    rcpsp_server *s = new rcpsp_server();
    s->device = device;
    s->cfg.slots = 8;
    s->cfg.max_batch = 256;
    s->cfg.memory_budget = int64_t(1) << 30;
    s->cfg.poll_us = 100;
    if (cfg) {
        if (cfg->slots > 0) s->cfg.slots = std::min(cfg->slots, 16);
        if (cfg->max_batch > 0) s->cfg.max_batch = cfg->max_batch;
        if (cfg->memory_budget > 0) s->cfg.memory_budget = cfg->memory_budget;
        if (cfg->poll_us > 0) s->cfg.poll_us = cfg->poll_us;
        if (cfg->slice_iterations > 0) s->cfg.slice_iterations = cfg->slice_iterations;
        if (cfg->max_pending > 0) s->cfg.max_pending = cfg->max_pending;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        delete s;
        return RCPSP_E_CUDA;
    }
    {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        uint64_t keep = static_cast<uint64_t>(s->cfg.memory_budget);
        if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            rcpsp_server_destroy(s);
            return RCPSP_E_CUDA;
        }
    }
    s->slots.resize(s->cfg.slots);
    s->allocs.resize(s->cfg.slots);
    for (int k = 0; k < s->cfg.slots; ++k) {
        Slot &sl = s->slots[k];
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            rcpsp_server_destroy(s);
            return RCPSP_E_CUDA;
        }
        sl.mem.stream = sl.stream;
        sl.mem.pool = s->pool;
        s->allocs[k] = rcpsp_allocator{slot_alloc, slot_release, &sl.mem};
        int rc = rcpsp_create(&sl.ctx, device, &s->allocs[k]);
        // pinned staging and launch plan for a full batch of the largest
        // instances (N up to RCPSP_MAX_N, M up to 8: records of at most a few
        // tens of KB), so that admission never waits on cudaMallocHost
        if (rc == RCPSP_OK) rc = rcpsp::ctx_reserve(sl.ctx, size_t(8) << 20, std::min(s->cfg.max_batch, 256));
        if (rc != RCPSP_OK) {
            rcpsp_server_destroy(s);
            return rc;
        }
    }
    // map the memory budget in the pool once (it stays mapped: the release
    // threshold is the budget), and load the search kernels of every group
    // size with the device's shared-memory limit
    {
        cudaDeviceProp prop{};
        void *p = nullptr;
        cudaError_t e = cudaGetDeviceProperties(&prop, device);
        if (e == cudaSuccess)
            e = cudaMallocFromPoolAsync(&p, static_cast<size_t>(s->cfg.memory_budget), s->pool, s->slots[0].stream);
        if (e == cudaSuccess) e = cudaFreeAsync(p, s->slots[0].stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->slots[0].stream);
        const size_t smem_limit = prop.sharedMemPerBlockOptin > 1024 ? prop.sharedMemPerBlockOptin - 1024 : 0;
        for (int G = 1; G <= 32 && e == cudaSuccess; G *= 2) e = rcpsp::prepare_search(G, smem_limit);
        if (e != cudaSuccess) {
            rcpsp_server_destroy(s);
            return RCPSP_E_CUDA;
        }
    }
    s->worker = std::thread(run, s);
    *out = s;
    return RCPSP_OK;
}

int rcpsp_server_destroy(rcpsp_server *s) {
    if (!s) return RCPSP_E_INVALID_ARG;
    s->stop.store(true);
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot &sl : s->slots) {
        if (sl.ctx) rcpsp_destroy(sl.ctx);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return RCPSP_OK;
}

int rcpsp_server_submit(rcpsp_server *s, const rcpsp_instance *inst, const rcpsp_params *params, int64_t tag) {
    if (!s || !inst || !params) return RCPSP_E_INVALID_ARG;
    if (params->record_trace || params->use_graph || params->checkpoint || params->resume || params->iterations < 0)
        return RCPSP_E_INVALID_ARG;
    rcpsp::PackedInstance pk;
    std::string msg;
    const int rc = rcpsp::prepare_instance(*inst, pk, msg);
    if (rc != RCPSP_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.rejected++;
        s->err = msg;
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        int64_t waiting = 0;
        for (const auto &q : s->pending) waiting += static_cast<int64_t>(q.size());
        if (s->cfg.max_pending > 0 && waiting >= s->cfg.max_pending) {
            s->st.rejected++;
            s->err = "pending queue full";
            return RCPSP_E_TOO_LARGE;
        }
    }
    Request r;
    r.tag = tag;
    r.params = *params;
    r.n = inst->n;
    r.m = inst->m;
    r.dur.assign(inst->dur, inst->dur + inst->n);
    r.cap.assign(inst->cap, inst->cap + inst->m);
    r.req.assign(inst->req, inst->req + static_cast<size_t>(inst->n) * inst->m);
    r.succ_off.assign(inst->succ_off, inst->succ_off + inst->n + 1);
    r.succ.assign(inst->succ, inst->succ + inst->succ_off[inst->n]);
    if (inst->level_key) {
        r.key.assign(inst->level_key, inst->level_key + inst->n);
        r.has_key = true;
    }
    r.bytes = footprint(pk);
    r.cls = request_class(pk, *params);
    r.total_iters = params->iterations;
    slice_params(s, r, 0);
    r.t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.submitted++;
        s->pending[r.cls].push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return RCPSP_OK;
}

int rcpsp_server_poll(rcpsp_server *s, rcpsp_completion *out, int32_t capacity, int32_t *count, int32_t wait_ms) {
    if (!s || !count || capacity < 0 || (capacity > 0 && !out)) return RCPSP_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    s->handed.clear();
    int k = 0;
    while (k < capacity && !s->done.empty()) {
        s->handed.push_back(std::move(s->done.front()));
        s->done.pop_front();
        ++k;
    }
    for (int j = 0; j < k; ++j) {
        Completion &c = s->handed[j];
        c.c.order = c.W.empty() ? nullptr : c.W.data();
        c.c.start = c.S.empty() ? nullptr : c.S.data();
        out[j] = c.c;
    }
    *count = k;
    return RCPSP_OK;
}

int rcpsp_server_get_stats(rcpsp_server *s, rcpsp_server_stats *out) {
    if (!s || !out) return RCPSP_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->pending = 0;
    for (const auto &q : s->pending) out->pending += static_cast<int64_t>(q.size());
    out->inflight_bytes = s->inflight_bytes;
    return RCPSP_OK;
}

}  // extern "C"
