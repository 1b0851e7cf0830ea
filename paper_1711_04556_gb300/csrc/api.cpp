// C interface of the library (include/rcpsp.h): contexts, device memory,
// instance loading, launch planning (longest-first work queue, launch shape,
// CUDA-graph replay) and result retrieval.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "host_prep.h"
#include "kernels.h"
#include "rcpsp_internal.h"

using rcpsp::InstHeader;
using rcpsp::LaunchItem;

namespace {

struct Block {
    void *ptr = nullptr;
    size_t bytes = 0;
    size_t out_offset = 0;   // byte offset of the outputs of this block
    size_t out_bytes = 0;
    int live = 0;            // instances still loaded from this block
};

struct Inst {
    InstHeader h{};
    int block = -1;
    int32_t *record = nullptr;
    int32_t *out = nullptr;
    size_t out_word = 0;     // word offset of the outputs inside the block's output region
    int32_t *trace = nullptr;
    size_t trace_bytes = 0;
    int trace_iters = -1;    // iterations recorded by the last traced search, -1 = none
    bool alive = false;
    std::vector<int32_t> succ_off, succ;   // host copy of the arcs, to check caller lists
    std::vector<int32_t> w0;               // host copy of the initial list
    int feas_delta = -1, feas0 = 0;        // feasible swaps of w0 at that swap distance
    int32_t *ckpt = nullptr;               // kept search state (CkptLayout), device
    size_t ckpt_bytes = 0;
    bool ckpt_valid = false;               // holds a state for the parameters below
    int ckpt_delta = 0, ckpt_tl = 0, ckpt_mode = 0;
};

int out_words(int n) { return rcpsp::align4(2 * n + rcpsp::kOutStats); }

// A host phase as an NVTX range (shown by Nsight Systems; a no-op without a tool attached).
struct HostRange {
    explicit HostRange(const char *name) { nvtxRangePushA(name); }
    ~HostRange() { nvtxRangePop(); }
    HostRange(const HostRange &) = delete;
    HostRange &operator=(const HostRange &) = delete;
};

constexpr int kClasses = rcpsp::kLaunchClasses;   // launch classes of one call (see footprint_class)
constexpr int kMaxLaunches = 2 * kClasses;   // each class and its launch of clustered outliers
constexpr int kAuxStreams = kMaxLaunches - 1;
constexpr int kAutoSlices = 8;                  // slices per search when a class is sliced automatically

}  // namespace

struct rcpsp_ctx {
    int device = 0;
    rcpsp_allocator alloc{};
    bool has_alloc = false;
    cudaDeviceProp prop{};
    std::vector<Block> blocks;
    std::vector<Inst> insts;
    std::string err;
    LaunchItem *items_dev = nullptr;
    size_t items_cap = 0;
    LaunchItem *items_host = nullptr;   // pinned staging
    int *queue_dev = nullptr;
    cudaEvent_t done = nullptr;
    bool pending = false;
    // graph replay: the cached graph corresponds to the items now on the device
    cudaGraphExec_t gexec = nullptr;
    std::vector<LaunchItem> g_items;
    cudaStream_t g_stream = nullptr;
    long long h2d = 0, d2h = 0;   // bytes copied by the context
    long long kernels = 0;        // kernel launches issued (graph replays count their kernels)
    std::vector<LaunchItem> noalloc_plan;   // host copy of the last no-allocation plan
    // footprint classes beyond the first run on their own streams, forked
    // from and joined back to the caller's stream
    cudaStream_t aux[kAuxStreams] = {};
    cudaEvent_t fork = nullptr, join[kAuxStreams] = {};
    std::vector<long long> g_launch_sig;
    int32_t *snap_dev = nullptr;        // kept prefix states of the CTAs (prefix reuse)
    int32_t *slice_dev = nullptr;       // sync counters and slice states of sliced launches
    size_t slice_cap = 0;
    size_t snap_cap = 0;
    // co-operative searches: plan, initial lists, random words and working sets
    // instance upload: pinned staging and a stream of its own, so that a
    // load overlaps a search that is still running on the caller's stream
    cudaStream_t copy_stream = nullptr;
    char *load_host = nullptr;
    size_t load_host_cap = 0;
    void *coop_dev = nullptr;
    size_t coop_cap = 0;
    char *coop_host = nullptr;          // pinned staging of the uploaded part
    size_t coop_host_cap = 0;
    // measured launch shapes: workload signature -> (G, warps, CTAs per search)
    std::vector<std::pair<std::string, std::array<int, 3>>> tuned;
    std::vector<rcpsp_launch_info> last_launches;   // plan of the last search call
};

namespace {

int set_err(rcpsp_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_err(rcpsp_ctx *c, cudaError_t e, const char *what) {
    return set_err(c, RCPSP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void *dev_alloc(rcpsp_ctx *c, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    if (c->has_alloc) return c->alloc.alloc(bytes, st, c->alloc.user);
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

void dev_free(rcpsp_ctx *c, void *p, size_t bytes, cudaStream_t st) {
    if (!p) return;
    if (c->has_alloc) c->alloc.release(p, bytes, st, c->alloc.user);
    else cudaFree(p);
}

// Waits for the context's last search with a deadline (seconds from the
// environment variable RCPSP_WAIT_SECONDS, default 900).
int wait_done(rcpsp_ctx *c) {
    if (!c->pending) return RCPSP_OK;
    double limit = 900.0;
    if (const char *s = std::getenv("RCPSP_WAIT_SECONDS")) limit = std::atof(s);
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(c->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_err(c, e, "search");
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit) return set_err(c, RCPSP_E_TIMEOUT, "search did not finish within the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    c->pending = false;
    return RCPSP_OK;
}

// Default launch shape: G lanes per neighbour decode and warps per CTA.
void default_shape(const std::vector<LaunchItem> &items, int *G, int *warps) {
    double avg_d = 0, feas = 0;
    for (const LaunchItem &it : items) {
        avg_d += it.h.n > 2 ? static_cast<double>(it.h.ub) / (it.h.n - 2) : 1.0;
        feas += it.h.n > 3 ? 0.12 * (it.h.n - 3) * it.delta : 1.0;
    }
    avg_d /= std::max<size_t>(1, items.size());
    feas /= std::max<size_t>(1, items.size());
    int g = 1;
    while (g < 32 && g < avg_d) g *= 2;
    *G = g;
    const int groups_wanted = static_cast<int>(feas) + 1;
    int w = (groups_wanted * g + 31) / 32;
    *warps = std::max(1, std::min(rcpsp::kSearchMaxWarps, w));
}

// Entries of the move list of a launch: the largest number of potential
// moves (N-3)*delta of the batch, rounded up to a warp, at most
// kDefaultMoveCap (the list is filled over several filter passes and
// drained when the next pass might not fit; searches with more feasible
// moves take several such batches per iteration).
int launch_move_cap(const std::vector<LaunchItem> &items) {
    int m = 32;
    for (const LaunchItem &it : items) m = std::max(m, it.h.n > 3 ? (it.h.n - 3) * it.delta : 0);
    return std::min(rcpsp::kDefaultMoveCap, (m + 31) & ~31);
}

// Positions between the kept prefix states of an N-activity search: every 8
// positions, at most 32 states.
int prefix_k_for(int n) { return std::max(8, (n + 31) / 32); }

// Words of kept prefix states one CTA needs for a class (global scratch).
int prefix_words_max(const std::vector<LaunchItem> &items) {
    int words = 0;
    for (const LaunchItem &it : items) {
        const int pw = rcpsp::profile_words(it.mode, it.h.wps, it.h.ub, it.h.sum_cap);
        words = std::max(words, rcpsp::prefix_words(it.h.n, pw, prefix_k_for(it.h.n)));
    }
    return rcpsp::align4(words);
}

// Shared memory of a class at this shape.
size_t smem_bytes(const std::vector<LaunchItem> &items, int ngroups, int move_cap) {
    int words = 0;
    for (const LaunchItem &it : items) {
        const int pw = rcpsp::profile_words(it.mode, it.h.wps, it.h.ub, it.h.sum_cap);
        const rcpsp::StateLayout S =
            rcpsp::state_layout(it.h.inst_words, it.h.n, it.tabu_len, it.delta, move_cap, pw, ngroups, it.mode);
        words = std::max(words, S.total);
    }
    return static_cast<size_t>(words) * 4;
}

// Prefix reuse pays when an iteration takes several decode rounds: the
// kept states cost one decode of the current list per iteration.
bool prefix_pays(const std::vector<LaunchItem> &items, int ngroups, int csize) {
    double feas = 0;
    for (const LaunchItem &it : items) feas += it.h.n > 3 ? 0.12 * (it.h.n - 3) * it.delta : 0.0;
    feas /= std::max<size_t>(1, items.size());
    return feas >= 3.0 * ngroups * std::max(1, csize);
}

// Launch class of a search (rcpsp::launch_class).  Each class of a call gets
// its own launch shape, so that small instances are not run at the group
// count the largest one allows, and a few large searches can share clusters
// of CTAs while many small ones take one CTA each.
int footprint_class(const LaunchItem &it) {
    const int pw = rcpsp::profile_words(it.mode, it.h.wps, it.h.ub, it.h.sum_cap);
    return rcpsp::launch_class(rcpsp::group_area_words(it.mode, pw, it.h.n), it.h.n);
}

struct ClassLaunch {
    int offset = 0, count = 0, G = 0, threads = 0, blocks = 0, move_cap = 0, csize = 1;
    int nslices = 1;             // slices per search (SliceSched); 1: not sliced
    bool solo = false;           // one CTA per SM: the build that may take all its registers
    size_t slice_off = 0;        // first word of its sync counters and slice states in slice_dev
    bool prefix = false;         // prefix reuse (kernel variant, kept states in global scratch)
    int snap_words = 0;          // kept-state words per CTA
    size_t snap_off = 0;         // its first word in the context's scratch
    size_t smem = 0;
    int shape_source = 0;        // rcpsp_launch_info.shape_source
    double cost = 0;             // estimated work of the class
    bool outliers = false;       // the clustered outliers of a class (see split_outliers)
};

// Feasible swaps (u, v), 1 <= u < v <= N-2, v - u <= delta, of the list W:
// swap(u, v) keeps every arc pointing forward iff no successor of W[u] sits
// at a position up to v and no predecessor of W[v] at a position from u on
// (Eqs. 5-6), i.e. firstSucc(u) > v and lastPred(v) < u.
int feasible_swaps(const std::vector<int32_t> &succ_off, const std::vector<int32_t> &succ,
                   const std::vector<int32_t> &W, int delta) {
    const int n = static_cast<int>(W.size());
    std::vector<int> pos(n), fsp(n, n), lpp(n, -1);
    for (int p = 0; p < n; ++p) pos[W[p]] = p;
    for (int a = 0; a < n; ++a)
        for (int e = succ_off[a]; e < succ_off[a + 1]; ++e) {
            const int b = succ[e];
            fsp[pos[a]] = std::min(fsp[pos[a]], pos[b]);
            lpp[pos[b]] = std::max(lpp[pos[b]], pos[a]);
        }
    int cnt = 0;
    for (int u = 1; u <= n - 3; ++u)
        for (int v = u + 1; v <= std::min(u + delta, n - 2); ++v) cnt += fsp[u] > v && lpp[v] < u;
    return cnt;
}

// CTAs that share one search: 1 unless the class has few searches for the
// GPU and each has a large neighbourhood.
int default_cluster(const std::vector<LaunchItem> &items, int sms) {
    const int cnt = static_cast<int>(items.size());
    double feas = 0;
    for (const LaunchItem &it : items) feas += it.h.n > 3 ? 0.12 * (it.h.n - 3) * it.delta : 0.0;
    feas /= std::max(1, cnt);
    if (cnt * 4 > sms || feas < 128) return 1;
    int c = 1;
    while (c < 8 && cnt * c * 2 <= sms) c *= 2;
    return c;
}

// Workload signature of a launch plan for the shape table: largest N, time
// horizon in 64-step buckets, words per step, swap distance, evaluator mix,
// and the batch size in powers of two.
std::string shape_key(const std::vector<LaunchItem> &items) {
    int n = 0, ub = 0, wps = 0, dl = 0, cnt = static_cast<int>(items.size()), lg = 0;
    bool tm = false, cap = false;
    for (const LaunchItem &it : items) {
        n = std::max(n, it.h.n);
        ub = std::max(ub, it.h.ub);
        wps = std::max(wps, it.h.wps);
        dl = std::max(dl, it.delta);
        (it.mode == RCPSP_EVAL_CAPACITY ? cap : tm) = true;
    }
    while ((1 << lg) < cnt) ++lg;
    return "n" + std::to_string(n) + "_ub" + std::to_string((ub + 63) / 64) + "_w" + std::to_string(wps) + "_d" +
           std::to_string(dl) + (tm ? "_T" : "") + (cap ? "_C" : "") + "_b" + std::to_string(lg);
}

// Shape table on disk: the file named by RCPSP_TUNE_CACHE holds lines
// "<device name>\t<signature>\t<G> <warps> <CTAs per search>"; a context
// loads the lines of its own device and rcpsp_autotune writes them back.
std::string device_tag(const rcpsp_ctx *c) {
    std::string t = c->prop.name;
    for (char &ch : t)
        if (ch == '\t' || ch == '\n') ch = ' ';
    return t;
}

void load_tune_cache(rcpsp_ctx *c) {
    const char *path = std::getenv("RCPSP_TUNE_CACHE");
    if (!path || !*path) return;
    std::ifstream f(path);
    std::string line;
    const std::string dev = device_tag(c);
    while (std::getline(f, line)) {
        std::istringstream ls(line);
        std::string d, key;
        if (!std::getline(ls, d, '\t') || !std::getline(ls, key, '\t') || d != dev) continue;
        std::array<int, 3> v{};
        if (ls >> v[0] >> v[1] >> v[2]) c->tuned.push_back({key, v});
    }
}

void save_tune_cache(const rcpsp_ctx *c) {
    const char *path = std::getenv("RCPSP_TUNE_CACHE");
    if (!path || !*path) return;
    const std::string dev = device_tag(c);
    std::vector<std::string> keep;
    {
        std::ifstream f(path);
        std::string line;
        while (std::getline(f, line))
            if (line.compare(0, dev.size() + 1, dev + "\t") != 0) keep.push_back(line);   // other devices
    }
    std::ofstream o(std::string(path) + ".tmp");
    for (const std::string &l : keep) o << l << "\n";
    for (const auto &e : c->tuned) o << dev << "\t" << e.first << "\t" << e.second[0] << " " << e.second[1] << " " << e.second[2] << "\n";
    o.close();
    std::rename((std::string(path) + ".tmp").c_str(), path);
}

bool tuned_shape(const rcpsp_ctx *c, const std::string &key, int *G, int *warps, int *csize = nullptr) {
    for (const auto &e : c->tuned)
        if (e.first == key) {
            *G = e.second[0];
            *warps = e.second[1];
            if (csize) *csize = e.second[2];
            return true;
        }
    return false;
}

}  // namespace

namespace rcpsp {

// 1 when the context's last search has finished (or none is pending), 0 while
// it runs, a negative RCPSP_E_* code when the device reported an error.
// Sizes the context's pinned upload staging (bytes) and launch plan (items,
// pinned and device) ahead of use, so that later calls of up to that size
// allocate nothing there.
int ctx_reserve(rcpsp_ctx *c, size_t staging_bytes, int plan_items) {
    cudaSetDevice(c->device);
    if (c->load_host_cap < staging_bytes) {
        if (c->load_host) cudaFreeHost(c->load_host);
        c->load_host = nullptr;
        c->load_host_cap = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&c->load_host), staging_bytes) != cudaSuccess)
            return set_err(c, RCPSP_E_CUDA, "pinned staging");
        c->load_host_cap = staging_bytes;
    }
    const size_t ibytes = sizeof(LaunchItem) * static_cast<size_t>(std::max(1, plan_items));
    if (c->items_cap < ibytes) {
        dev_free(c, c->items_dev, c->items_cap, nullptr);
        if (c->items_host) cudaFreeHost(c->items_host);
        c->items_host = nullptr;
        c->items_dev = static_cast<LaunchItem *>(dev_alloc(c, ibytes, nullptr));
        c->items_cap = c->items_dev ? ibytes : 0;
        if (!c->items_dev) return set_err(c, RCPSP_E_CUDA, "plan allocation failed");
        if (cudaMallocHost(reinterpret_cast<void **>(&c->items_host), ibytes) != cudaSuccess)
            return set_err(c, RCPSP_E_CUDA, "pinned staging");
    }
    return RCPSP_OK;
}

int ctx_search_done(rcpsp_ctx *c) {
    if (!c->pending) return 1;
    const cudaError_t e = cudaEventQuery(c->done);
    if (e == cudaSuccess) {
        c->pending = false;
        return 1;
    }
    if (e == cudaErrorNotReady) return 0;
    return cuda_err(c, e, "search");
}

}  // namespace rcpsp

extern "C" {

int rcpsp_create(rcpsp_ctx **ctx, int device, const rcpsp_allocator *alloc) {
    if (!ctx) return RCPSP_E_INVALID_ARG;
    *ctx = nullptr;
    if (alloc && (!alloc->alloc || !alloc->release)) return RCPSP_E_INVALID_ARG;
    rcpsp_ctx *c = new (std::nothrow) rcpsp_ctx();
    if (!c) return RCPSP_E_INVALID_ARG;
    c->device = device;
    if (alloc) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&c->prop, device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    for (int q = 0; q < kAuxStreams && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&c->aux[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join[q], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return RCPSP_E_CUDA;
    }
    load_tune_cache(c);
    c->queue_dev = static_cast<int *>(dev_alloc(c, 4 * kMaxLaunches, nullptr));   // one counter per launch
    if (!c->queue_dev) {
        cudaEventDestroy(c->done);
        delete c;
        return RCPSP_E_CUDA;
    }
    *ctx = c;
    return RCPSP_OK;
}

int rcpsp_destroy(rcpsp_ctx *c) {
    if (!c) return RCPSP_E_INVALID_ARG;
    cudaSetDevice(c->device);
    wait_done(c);
    cudaDeviceSynchronize();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (Inst &in : c->insts) {
        dev_free(c, in.trace, in.trace_bytes, nullptr);
        dev_free(c, in.ckpt, in.ckpt_bytes, nullptr);
    }
    for (Block &b : c->blocks) dev_free(c, b.ptr, b.bytes, nullptr);
    dev_free(c, c->items_dev, c->items_cap, nullptr);
    dev_free(c, c->queue_dev, 4 * kMaxLaunches, nullptr);
    dev_free(c, c->coop_dev, c->coop_cap, nullptr);
    dev_free(c, c->slice_dev, c->slice_cap, nullptr);
    dev_free(c, c->snap_dev, c->snap_cap, nullptr);
    if (c->items_host) cudaFreeHost(c->items_host);
    if (c->coop_host) cudaFreeHost(c->coop_host);
    if (c->load_host) cudaFreeHost(c->load_host);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    cudaEventDestroy(c->done);
    cudaEventDestroy(c->fork);
    for (int q = 0; q < kAuxStreams; ++q) {
        if (c->aux[q]) cudaStreamDestroy(c->aux[q]);
        if (c->join[q]) cudaEventDestroy(c->join[q]);
    }
    delete c;
    return RCPSP_OK;
}

const char *rcpsp_last_error(const rcpsp_ctx *c) { return c ? c->err.c_str() : "null context"; }

int rcpsp_transfer_bytes(const rcpsp_ctx *c, int64_t *h2d, int64_t *d2h) {
    if (!c) return RCPSP_E_INVALID_ARG;
    if (h2d) *h2d = c->h2d;
    if (d2h) *d2h = c->d2h;
    return RCPSP_OK;
}

int rcpsp_multistart(rcpsp_ctx *c, const rcpsp_instance *inst, int32_t starts, const int32_t *level_keys,
                     const rcpsp_params *p, void *stream, int32_t *best_start, int32_t *order, int32_t *start,
                     int32_t *makespans, rcpsp_stats *stats) {
    HostRange range("rcpsp_multistart");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (!inst || !p || starts < 1) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    if (p->record_trace || p->checkpoint || p->resume)
        return set_err(c, RCPSP_E_INVALID_ARG, "a multi-start keeps no trace or state");
    const int n = inst->n;
    std::vector<rcpsp_instance> views(starts, *inst);
    for (int k = 0; k < starts; ++k) views[k].level_key = level_keys ? level_keys + static_cast<size_t>(k) * n : nullptr;
    std::vector<int32_t> ids(starts);
    int rc = rcpsp_load_instances(c, views.data(), starts, ids.data());
    if (rc != RCPSP_OK) return rc;
    rc = rcpsp_tabu_search(c, ids.data(), starts, p, stream);
    std::vector<int32_t> W, S, cm(starts);
    std::vector<rcpsp_stats> st(starts);
    if (rc == RCPSP_OK) {
        W.resize(static_cast<size_t>(starts) * n);
        S.resize(static_cast<size_t>(starts) * n);
        rc = rcpsp_get_schedules(c, ids.data(), starts, W.data(), S.data(), cm.data(), st.data());
    }
    const std::string msg = c->err;
    const int frc = rcpsp_free_instances(c, ids.data(), starts);
    if (rc != RCPSP_OK) return set_err(c, rc, msg);
    if (frc != RCPSP_OK) return frc;
    // the lowest best makespan, ties to the lowest start index
    int best = 0;
    for (int k = 1; k < starts; ++k)
        if (cm[k] < cm[best]) best = k;
    if (best_start) *best_start = best;
    if (order) std::memcpy(order, W.data() + static_cast<size_t>(best) * n, sizeof(int32_t) * n);
    if (start) std::memcpy(start, S.data() + static_cast<size_t>(best) * n, sizeof(int32_t) * n);
    if (makespans) std::memcpy(makespans, cm.data(), sizeof(int32_t) * starts);
    if (stats) *stats = st[best];
    return RCPSP_OK;
}

int rcpsp_last_launches(const rcpsp_ctx *c, rcpsp_launch_info *out, int32_t capacity, int32_t *count) {
    if (!c || !count || capacity < 0 || (capacity > 0 && !out)) return RCPSP_E_INVALID_ARG;
    const int n = static_cast<int>(c->last_launches.size());
    for (int k = 0; k < n && k < capacity; ++k) out[k] = c->last_launches[k];
    *count = n;
    return RCPSP_OK;
}

int rcpsp_kernel_launches(const rcpsp_ctx *c, int64_t *launches) {
    if (!c || !launches) return RCPSP_E_INVALID_ARG;
    *launches = c->kernels;
    return RCPSP_OK;
}

int rcpsp_prepare_instance(const rcpsp_instance *inst, int32_t *critical_path, int32_t *horizon,
                           int32_t *initial_order, int32_t *eval_mode, char *msg, int32_t msg_len) {
    if (!inst) return RCPSP_E_INVALID_ARG;
    rcpsp::PackedInstance pk;
    std::string err;
    const int rc = rcpsp::prepare_instance(*inst, pk, err);
    if (msg && msg_len > 0) {
        std::strncpy(msg, err.c_str(), static_cast<size_t>(msg_len) - 1);
        msg[msg_len - 1] = 0;
    }
    if (rc != RCPSP_OK) return rc;
    if (critical_path) *critical_path = pk.h.cp;
    if (horizon) *horizon = pk.h.ub;
    if (eval_mode) *eval_mode = pk.h.sel_mode;
    if (initial_order) std::memcpy(initial_order, pk.initial.data(), pk.initial.size() * 4);
    return RCPSP_OK;
}

int rcpsp_load_instances(rcpsp_ctx *c, const rcpsp_instance *inst, int32_t count, int32_t *out_ids) {
    HostRange range("rcpsp_load_instances");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (count < 0 || (count > 0 && (!inst || !out_ids))) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    if (count == 0) return RCPSP_OK;
    cudaSetDevice(c->device);
    // host preparation of every instance, spread over host threads
    std::vector<rcpsp::PackedInstance> packed(count);
    std::vector<int> codes(count, RCPSP_OK);
    std::vector<std::string> msgs(count);
    {
        const int hw = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
        const int nt = std::max(1, std::min({hw, 16, count / 32}));
        auto work = [&](int t) {
            for (int k = t; k < count; k += nt) codes[k] = rcpsp::prepare_instance(inst[k], packed[k], msgs[k]);
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < nt; ++t) pool.emplace_back(work, t);
        work(0);
        for (std::thread &th : pool) th.join();
    }
    size_t rec_words = 0, o_words = 0;
    for (int k = 0; k < count; ++k) {
        if (codes[k] != RCPSP_OK) return set_err(c, codes[k], "instance " + std::to_string(k) + ": " + msgs[k]);
        rec_words += packed[k].h.record_words;
        o_words += out_words(packed[k].h.n);
    }
    Block b;
    b.out_offset = rec_words * 4;
    b.out_bytes = o_words * 4;
    b.bytes = b.out_offset + b.out_bytes;
    b.ptr = dev_alloc(c, b.bytes, nullptr);
    if (!b.ptr) return set_err(c, RCPSP_E_CUDA, "device allocation failed");
    cudaError_t e = cudaSuccess;
    if (c->load_host_cap < rec_words * 4) {
        // grows geometrically: pinning memory is slow, and batch sizes vary
        const size_t cap = std::max(rec_words * 4, 2 * c->load_host_cap);
        if (c->load_host) cudaFreeHost(c->load_host);
        c->load_host = nullptr;
        c->load_host_cap = 0;
        e = cudaMallocHost(reinterpret_cast<void **>(&c->load_host), cap);
        if (e != cudaSuccess) {
            dev_free(c, b.ptr, b.bytes, nullptr);
            return cuda_err(c, e, "pinned staging");
        }
        c->load_host_cap = cap;
    }
    int32_t *host = reinterpret_cast<int32_t *>(c->load_host);
    size_t ro = 0;
    for (int k = 0; k < count; ++k) {
        std::memcpy(host + ro, packed[k].record.data(), packed[k].record.size() * 4);
        ro += packed[k].record.size();
    }
    e = cudaMemcpyAsync(b.ptr, host, rec_words * 4, cudaMemcpyHostToDevice, c->copy_stream);
    c->h2d += static_cast<long long>(rec_words) * 4;
    if (e == cudaSuccess)
        e = cudaMemsetAsync(static_cast<char *>(b.ptr) + b.out_offset, 0, b.out_bytes, c->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy_stream);   // staging free again, data in place
    if (e != cudaSuccess) {
        dev_free(c, b.ptr, b.bytes, nullptr);
        return cuda_err(c, e, "instance upload");
    }
    b.live = count;
    const int bid = static_cast<int>(c->blocks.size());
    c->blocks.push_back(b);
    ro = 0;
    size_t oo = 0;
    int32_t *base = static_cast<int32_t *>(b.ptr);
    for (int k = 0; k < count; ++k) {
        Inst in;
        in.h = packed[k].h;
        in.block = bid;
        in.record = base + ro;
        in.out_word = oo;
        in.out = base + rec_words + oo;
        in.alive = true;
        in.succ_off.assign(inst[k].succ_off, inst[k].succ_off + inst[k].n + 1);
        in.succ.assign(inst[k].succ, inst[k].succ + inst[k].succ_off[inst[k].n]);
        in.w0 = packed[k].initial;
        ro += packed[k].record.size();
        oo += out_words(in.h.n);
        out_ids[k] = static_cast<int32_t>(c->insts.size());
        c->insts.push_back(in);
    }
    return RCPSP_OK;
}

int rcpsp_free_instances(rcpsp_ctx *c, const int32_t *ids, int32_t count) {
    if (!c) return RCPSP_E_INVALID_ARG;
    if (count < 0 || (count > 0 && !ids)) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    for (int k = 0; k < count; ++k) {
        const int id = ids[k];
        if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
            return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
        Inst &in = c->insts[id];
        in.alive = false;
        std::vector<int32_t>().swap(in.succ_off);     // a long-lived context keeps no host copies
        std::vector<int32_t>().swap(in.succ);
        std::vector<int32_t>().swap(in.w0);
        dev_free(c, in.trace, in.trace_bytes, nullptr);
        in.trace = nullptr;
        in.trace_bytes = 0;
        dev_free(c, in.ckpt, in.ckpt_bytes, nullptr);
        in.ckpt = nullptr;
        in.ckpt_bytes = 0;
        in.ckpt_valid = false;
        Block &b = c->blocks[in.block];
        if (--b.live == 0) {
            dev_free(c, b.ptr, b.bytes, nullptr);
            b.ptr = nullptr;
        }
    }
    return RCPSP_OK;
}

int rcpsp_tabu_search(rcpsp_ctx *c, const int32_t *ids, int32_t count, const rcpsp_params *p, void *stream) {
    HostRange range("rcpsp_tabu_search");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (!p || count < 0 || (count > 0 && !ids)) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    if (p->iterations < 0 || p->max_swap_dist < 0 || p->tabu_len < 0 || p->tabu_len > RCPSP_MAX_TABU ||
        p->eval_mode < 0 || p->eval_mode > 2 || p->warps_per_cta < 0 ||
        p->warps_per_cta > rcpsp::kSearchMaxWarps || p->checkpoint < 0 || p->checkpoint > 1 || p->resume < 0 ||
        p->resume > 1 || p->slices < 0 || p->slices > rcpsp::kMaxSlices)
        return set_err(c, RCPSP_E_INVALID_ARG, "bad search parameters");
    const int gs = p->group_size;
    if (gs != 0 && gs != 1 && gs != 2 && gs != 4 && gs != 8 && gs != 16 && gs != 32)
        return set_err(c, RCPSP_E_INVALID_ARG, "group_size must be 0, 1, 2, 4, 8, 16 or 32");
    const int cs = p->cluster_size;
    if (cs != 0 && cs != 1 && cs != 2 && cs != 4 && cs != 8)
        return set_err(c, RCPSP_E_INVALID_ARG, "cluster_size must be 0, 1, 2, 4 or 8");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->use_graph && st == nullptr)
        return set_err(c, RCPSP_E_INVALID_ARG, "graph capture needs a non-default stream");
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    if (count == 0) return RCPSP_OK;
    std::vector<LaunchItem> items(count);
    std::vector<double> cost(count);
    for (int k = 0; k < count; ++k) {
        const int id = ids[k];
        if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
            return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
        Inst &in = c->insts[id];
        LaunchItem &it = items[k];
        std::memset(&it, 0, sizeof(it));
        it.h = in.h;
        it.record = in.record;
        it.out = in.out;
        it.mode = p->eval_mode == RCPSP_EVAL_AUTO ? in.h.sel_mode : p->eval_mode;
        int dd, tl;
        rcpsp::default_search_params(in.h.n, &dd, &tl);
        // v - u never exceeds N - 3, so a larger delta names the same moves
        it.delta = std::max(1, std::min(p->max_swap_dist ? p->max_swap_dist : dd, in.h.n - 3));
        it.tabu_len = p->tabu_len ? p->tabu_len : tl;
        it.iterations = p->iterations;
        it.stop_at_cp = p->stop_at_cp ? 1 : 0;
        if (p->checkpoint || p->resume) {
            if (p->resume && !(in.ckpt_valid && in.ckpt_delta == it.delta && in.ckpt_tl == it.tabu_len &&
                               in.ckpt_mode == it.mode))
                return set_err(c, RCPSP_E_INVALID_ARG,
                               "instance " + std::to_string(id) + " has no kept state for these parameters");
            const size_t need = static_cast<size_t>(rcpsp::ckpt_layout(in.h.n, it.tabu_len, it.delta).words) * 4;
            if (in.ckpt_bytes < need) {                   // (a kept state of these parameters has this size)
                dev_free(c, in.ckpt, in.ckpt_bytes, nullptr);
                in.ckpt = static_cast<int32_t *>(dev_alloc(c, need, nullptr));
                in.ckpt_bytes = in.ckpt ? need : 0;
                in.ckpt_valid = false;
                if (!in.ckpt) return set_err(c, RCPSP_E_CUDA, "state allocation failed");
            }
            it.state = in.ckpt;
            it.ckpt = (p->resume ? rcpsp::kCkptResume : 0) | (p->checkpoint ? rcpsp::kCkptSave : 0);
        }
        if (p->record_trace) {
            const size_t need = static_cast<size_t>(std::max(1, p->iterations)) * 3 * 4;
            if (in.trace_bytes < need) {
                dev_free(c, in.trace, in.trace_bytes, nullptr);
                in.trace = static_cast<int32_t *>(dev_alloc(c, need, nullptr));
                in.trace_bytes = in.trace ? need : 0;
                if (!in.trace) return set_err(c, RCPSP_E_CUDA, "trace allocation failed");
            }
            it.trace = in.trace;
            in.trace_iters = p->iterations;
        } else {
            in.trace_iters = -1;
        }
        cost[k] = rcpsp::estimate_cost(in.h, it.mode, it.iterations, it.delta, it.stop_at_cp != 0);
    }
    // footprint classes, each ordered longest first (LPT) on its own queue
    std::vector<LaunchItem> sorted;
    sorted.reserve(count);
    std::vector<ClassLaunch> launches;
    const size_t smem_limit = c->prop.sharedMemPerBlockOptin > 1024 ? c->prop.sharedMemPerBlockOptin - 1024 : 0;
    for (int q = 0; q < kClasses; ++q) {
        std::vector<int> idx;
        for (int k = 0; k < count; ++k)
            if (footprint_class(items[k]) == q) idx.push_back(k);
        if (idx.empty()) continue;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        std::vector<LaunchItem> part;
        for (int k : idx) part.push_back(items[k]);
        ClassLaunch L;
        L.offset = static_cast<int>(sorted.size());
        L.count = static_cast<int>(part.size());
        sorted.insert(sorted.end(), part.begin(), part.end());
        int G = gs, warps = p->warps_per_cta;
        int dG, dW, dC = default_cluster(part, c->prop.multiProcessorCount);
        default_shape(part, &dG, &dW);
        L.shape_source = gs || warps ? 2 : 0;
        if (!gs && !warps && tuned_shape(c, shape_key(part), &dG, &dW, &dC)) L.shape_source = 1;
        for (int k : idx) L.cost += cost[k];
        if (!G) G = dG;
        if (!warps) warps = std::max(dW, (G + 31) / 32);
        L.csize = cs ? cs : dC;
        L.move_cap = launch_move_cap(part);
        size_t smem = smem_bytes(part, warps * (32 / G), L.move_cap);
        while (smem > smem_limit && p->warps_per_cta == 0 && warps > 1) {
            --warps;
            smem = smem_bytes(part, warps * (32 / G), L.move_cap);
        }
        if (smem > smem_limit)
            return set_err(c, RCPSP_E_TOO_LARGE, "instance state does not fit in shared memory at this launch shape");
        if (prefix_pays(part, warps * (32 / G), L.csize)) {
            L.prefix = true;
            L.snap_words = prefix_words_max(part);
            for (int k = L.offset; k < L.offset + L.count; ++k) sorted[k].prefix_k = prefix_k_for(sorted[k].h.n);
        }
        L.G = G;
        L.threads = warps * 32;
        L.smem = smem;
        // the limit belongs to the kernel of this G, shared by every class that uses it
        cudaError_t e = rcpsp::prepare_search(G, smem_limit);
        if (e != cudaSuccess) return cuda_err(c, e, "kernel attributes");
        int units = 0;
        e = rcpsp::search_occupancy(G, L.threads, smem, L.csize, &units, L.prefix);
        if (e != cudaSuccess) return cuda_err(c, e, "occupancy");
        if (units < 1) return set_err(c, RCPSP_E_TOO_LARGE, "launch shape does not fit on the GPU");
        // shared memory that holds one CTA per SM anyway: the build whose
        // threads may use the registers of the whole SM
        int solo_units = 0;
        if (L.csize == 1 && units == 1 &&
            rcpsp::search_occupancy(G, L.threads, smem, 1, &solo_units, L.prefix, true) == cudaSuccess &&
            solo_units == 1)
            L.solo = true;
        L.blocks = L.csize == 1 ? std::max(1, std::min(L.count, units * c->prop.multiProcessorCount))
                                : L.csize * std::max(1, std::min(L.count, units));
        // Outliers: in a class whose searches take one CTA each and decode
        // their neighbourhood in about one round, a few searches whose
        // initial list has more feasible swaps than the CTA has decoding
        // groups need several rounds per iteration and would set the call's
        // length.  They get a launch of their own with clusters of 2-8 CTAs
        // that split their neighbourhoods (same results: the cluster search
        // follows the one-CTA trajectory), and it starts first.
        if (!cs && L.csize == 1 && !L.prefix && L.count >= 16) {
            const int ngroups = warps * (32 / G);
            std::vector<int> out;
            int worst = 0;
            for (int k = L.offset; k < L.offset + L.count; ++k) {
                Inst &in = c->insts[ids[idx[k - L.offset]]];
                if (in.feas_delta != sorted[k].delta) {
                    in.feas0 = feasible_swaps(in.succ_off, in.succ, in.w0, sorted[k].delta);
                    in.feas_delta = sorted[k].delta;
                }
                if (in.feas0 > ngroups) {
                    out.push_back(k);
                    worst = std::max(worst, in.feas0);
                }
            }
            int oc = 2;
            while (oc < 8 && oc * ngroups < worst) oc *= 2;
            int ounits = 0;
            if (!out.empty() && 16 * static_cast<int>(out.size()) <= L.count &&
                rcpsp::search_occupancy(G, L.threads, smem, oc, &ounits, false) == cudaSuccess && ounits >= 1) {
                // the outliers move to the end of the class's part of the plan
                std::vector<LaunchItem> keep, moved;
                std::vector<double> kc, mc;
                size_t o = 0;
                for (int k = L.offset; k < L.offset + L.count; ++k) {
                    if (o < out.size() && out[o] == k) {
                        moved.push_back(sorted[k]);
                        ++o;
                    } else {
                        keep.push_back(sorted[k]);
                    }
                }
                std::copy(keep.begin(), keep.end(), sorted.begin() + L.offset);
                std::copy(moved.begin(), moved.end(), sorted.begin() + L.offset + keep.size());
                ClassLaunch O = L;
                O.solo = false;
                O.offset = L.offset + static_cast<int>(keep.size());
                O.count = static_cast<int>(moved.size());
                O.csize = oc;
                O.outliers = true;
                O.blocks = oc * std::max(1, std::min(O.count, ounits));
                L.count = static_cast<int>(keep.size());
                L.blocks = std::max(1, std::min(L.count, units * c->prop.multiProcessorCount));
                launches.push_back(O);
            }
        }
        launches.push_back(L);
    }
    // Slices (rcpsp_params.slices): automatically when a class has at least
    // half as many searches again as the CTAs (or clusters) of its launch
    // hold at once.  With fewer, most of a class runs in one wave anyway and
    // the searches that start late are mostly short (they reach the
    // critical path early), while slicing would make long searches wait for
    // the CTAs of others.
    for (ClassLaunch &L : launches) {
        const int held = L.blocks / std::max(1, L.csize);
        L.nslices = p->slices ? p->slices : (2 * L.count >= 3 * held ? kAutoSlices : 1);
        if (p->iterations < 2) L.nslices = 1;
    }
    // launches of clustered outliers first, then classes of more work, so
    // that the long searches of a call are not queued behind short ones for SMs
    std::stable_sort(launches.begin(), launches.end(), [](const ClassLaunch &a, const ClassLaunch &b) {
        return a.outliers != b.outliers ? a.outliers : a.cost > b.cost;
    });
    // slice scratch: per sliced class, two sync words per search, then the
    // searches' slice states
    {
        size_t need = 0;
        for (ClassLaunch &L : launches) {
            if (L.nslices <= 1) continue;
            L.slice_off = need;
            size_t o = rcpsp::align4(2 * L.count);
            for (int k = L.offset; k < L.offset + L.count; ++k) {
                sorted[k].slice_off = static_cast<int32_t>(o);
                o += rcpsp::slice_state_words(sorted[k].h.n, sorted[k].tabu_len, sorted[k].delta);
            }
            need += o;
        }
        if (need * 4 > c->slice_cap) {
            dev_free(c, c->slice_dev, c->slice_cap, nullptr);
            c->slice_dev = static_cast<int32_t *>(dev_alloc(c, need * 4, nullptr));
            c->slice_cap = c->slice_dev ? need * 4 : 0;
            if (!c->slice_dev) return set_err(c, RCPSP_E_CUDA, "slice scratch allocation failed");
        }
    }
    // kept prefix states: one region per CTA of every class that uses them
    {
        size_t need = 0;
        for (ClassLaunch &L : launches)
            if (L.prefix) {
                L.snap_off = need;
                need += static_cast<size_t>(L.blocks) * L.snap_words;
            }
        if (need * 4 > c->snap_cap) {
            dev_free(c, c->snap_dev, c->snap_cap, nullptr);
            c->snap_dev = static_cast<int32_t *>(dev_alloc(c, need * 4, nullptr));
            c->snap_cap = c->snap_dev ? need * 4 : 0;
            if (!c->snap_dev) return set_err(c, RCPSP_E_CUDA, "prefix scratch allocation failed");
        }
    }
    std::vector<long long> sig;
    for (const ClassLaunch &L : launches)
        sig.insert(sig.end(), {L.offset, L.count, L.G, L.threads, L.blocks, L.move_cap, static_cast<long long>(L.smem),
                               L.csize, L.prefix ? 1 : 0, L.snap_words, static_cast<long long>(L.snap_off),
                               L.nslices, static_cast<long long>(L.slice_off), L.solo ? 1 : 0});
    sig.push_back(reinterpret_cast<long long>(c->snap_dev));
    sig.push_back(reinterpret_cast<long long>(c->slice_dev));
    // device copy of the plan
    cudaError_t e = cudaSuccess;
    const size_t ibytes = sizeof(LaunchItem) * count;
    const bool same_plan = c->gexec && c->g_stream == st && c->g_items.size() == sorted.size() &&
                           std::memcmp(c->g_items.data(), sorted.data(), ibytes) == 0 && c->g_launch_sig == sig;
    if (!(p->use_graph && same_plan)) {
        if (c->items_cap < ibytes) {
            const size_t cap = std::max(ibytes, 2 * c->items_cap);   // geometric growth
            cudaStreamSynchronize(st);
            dev_free(c, c->items_dev, c->items_cap, nullptr);
            if (c->items_host) cudaFreeHost(c->items_host);
            c->items_host = nullptr;
            c->items_dev = static_cast<LaunchItem *>(dev_alloc(c, cap, nullptr));
            c->items_cap = c->items_dev ? cap : 0;
            if (!c->items_dev) return set_err(c, RCPSP_E_CUDA, "plan allocation failed");
            e = cudaMallocHost(reinterpret_cast<void **>(&c->items_host), cap);
            if (e != cudaSuccess) return cuda_err(c, e, "pinned staging");
        } else {
            cudaStreamSynchronize(st);   // the staging buffer may still feed a copy
        }
        std::memcpy(c->items_host, sorted.data(), ibytes);
        e = cudaMemcpyAsync(c->items_dev, c->items_host, ibytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_err(c, e, "plan upload");
        c->h2d += static_cast<long long>(ibytes);
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
            c->g_items.clear();
        }
    }
    // queue reset, then one persistent launch per class; classes after the
    // first run on forked streams and join back before the done event
    auto launch_all = [&](cudaStream_t s0) -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(c->queue_dev, 0, sizeof(int) * kMaxLaunches, s0);
        if (r != cudaSuccess) return r;
        for (const ClassLaunch &L : launches)
            if (L.nslices > 1 &&
                (r = cudaMemsetAsync(c->slice_dev + L.slice_off, 0, sizeof(int) * 2 * L.count, s0)) != cudaSuccess)
                return r;
        if (launches.size() > 1 && (r = cudaEventRecord(c->fork, s0)) != cudaSuccess) return r;
        for (size_t q = 0; q < launches.size(); ++q) {
            const ClassLaunch &L = launches[q];
            cudaStream_t sq = q == 0 ? s0 : c->aux[q - 1];
            if (q > 0 && (r = cudaStreamWaitEvent(sq, c->fork, 0)) != cudaSuccess) return r;
            const rcpsp::SliceSched sl{L.nslices, L.nslices > 1 ? c->slice_dev + L.slice_off : nullptr,
                                       L.nslices > 1 ? c->slice_dev + L.slice_off : nullptr};
            r = rcpsp::launch_search(L.G, c->items_dev + L.offset, L.count, c->queue_dev + q, L.move_cap, L.blocks,
                                     L.threads, L.smem, sq, L.csize, L.prefix,
                                     L.prefix ? c->snap_dev + L.snap_off : nullptr, L.snap_words, sl, L.solo);
            if (r != cudaSuccess) return r;
            if (q > 0 && (r = cudaEventRecord(c->join[q - 1], sq)) != cudaSuccess) return r;
        }
        for (size_t q = 1; q < launches.size(); ++q)
            if ((r = cudaStreamWaitEvent(s0, c->join[q - 1], 0)) != cudaSuccess) return r;
        return cudaSuccess;
    };
    if (p->use_graph) {
        if (!c->gexec) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_err(c, e, "begin capture");
            const cudaError_t le = launch_all(st);
            e = cudaStreamEndCapture(st, &graph);
            if (le != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_err(c, le, "captured launch");
            }
            if (e != cudaSuccess) return cuda_err(c, e, "end capture");
            e = cudaGraphInstantiate(&c->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                c->gexec = nullptr;
                return cuda_err(c, e, "graph instantiate");
            }
            c->g_items = sorted;
            c->g_launch_sig = sig;
            c->g_stream = st;
        }
        e = cudaGraphLaunch(c->gexec, st);
        if (e != cudaSuccess) return cuda_err(c, e, "graph launch");
    } else {
        e = launch_all(st);
        if (e != cudaSuccess) return cuda_err(c, e, "search launch");
    }
    c->kernels += static_cast<long long>(launches.size());
    c->last_launches.clear();
    for (const ClassLaunch &L : launches)
        c->last_launches.push_back(rcpsp_launch_info{L.count, L.G, L.threads / 32, L.csize, L.blocks, L.prefix ? 1 : 0,
                                                     L.shape_source, L.nslices, static_cast<int64_t>(L.smem)});
    if (p->checkpoint)
        for (const LaunchItem &it : items) {
            // items[] holds the ids' searches in call order
            Inst &in = c->insts[ids[&it - items.data()]];
            in.ckpt_valid = true;
            in.ckpt_delta = it.delta;
            in.ckpt_tl = it.tabu_len;
            in.ckpt_mode = it.mode;
        }
    e = cudaEventRecord(c->done, st);
    if (e != cudaSuccess) return cuda_err(c, e, "event record");
    c->pending = true;
    return RCPSP_OK;
}

int rcpsp_get_state(rcpsp_ctx *c, int32_t id, void *buf, size_t capacity, size_t *bytes) {
    if (!c) return RCPSP_E_INVALID_ARG;
    if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
        return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
    const Inst &in = c->insts[id];
    if (!in.ckpt_valid) return set_err(c, RCPSP_E_INVALID_ARG, "instance has no kept state");
    const size_t need = static_cast<size_t>(rcpsp::ckpt_layout(in.h.n, in.ckpt_tl, in.ckpt_delta).words) * 4;
    if (bytes) *bytes = need;
    if (!buf) return RCPSP_OK;
    if (capacity < need) return set_err(c, RCPSP_E_TOO_LARGE, "state buffer too small");
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    const cudaError_t e = cudaMemcpy(buf, in.ckpt, need, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(c, e, "state copy");
    c->d2h += static_cast<long long>(need);
    return RCPSP_OK;
}

int rcpsp_set_state(rcpsp_ctx *c, int32_t id, const void *buf, size_t bytes) {
    if (!c) return RCPSP_E_INVALID_ARG;
    if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
        return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
    Inst &in = c->insts[id];
    const int32_t *m = static_cast<const int32_t *>(buf);
    if (!buf || bytes < static_cast<size_t>(rcpsp::kCkMeta) * 4 || m[rcpsp::kCkMagic] != rcpsp::kCkptMagic ||
        m[rcpsp::kCkN] != in.h.n)
        return set_err(c, RCPSP_E_INVALID_ARG, "not a kept state of this instance");
    const int delta = m[rcpsp::kCkDelta], tl = m[rcpsp::kCkTabu], mode = m[rcpsp::kCkMode];
    if (delta < 1 || delta > std::max(1, in.h.n - 3) || tl < 1 || tl > RCPSP_MAX_TABU ||
        (mode != RCPSP_EVAL_TIME && mode != RCPSP_EVAL_CAPACITY) ||
        bytes != static_cast<size_t>(rcpsp::ckpt_layout(in.h.n, tl, delta).words) * 4)
        return set_err(c, RCPSP_E_INVALID_ARG, "not a kept state of this instance");
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    if (in.ckpt_bytes < bytes) {
        dev_free(c, in.ckpt, in.ckpt_bytes, nullptr);
        in.ckpt = static_cast<int32_t *>(dev_alloc(c, bytes, nullptr));
        in.ckpt_bytes = in.ckpt ? bytes : 0;
        in.ckpt_valid = false;
        if (!in.ckpt) return set_err(c, RCPSP_E_CUDA, "state allocation failed");
    }
    const cudaError_t e = cudaMemcpy(in.ckpt, buf, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(c, e, "state copy");
    c->h2d += static_cast<long long>(bytes);
    in.ckpt_valid = true;
    in.ckpt_delta = delta;
    in.ckpt_tl = tl;
    in.ckpt_mode = mode;
    return RCPSP_OK;
}

int rcpsp_coop_search(rcpsp_ctx *c, const int32_t *ids, int32_t count, const rcpsp_params *p,
                      const rcpsp_coop_params *cp, const int32_t *slot_keys, const uint32_t *random_words,
                      void *stream) {
    HostRange range("rcpsp_coop_search");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (!p || !cp || count < 0 || (count > 0 && !ids)) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    if (p->iterations < 0 || p->max_swap_dist < 0 || p->tabu_len < 0 || p->tabu_len > RCPSP_MAX_TABU ||
        p->eval_mode < 0 || p->eval_mode > 2 || p->warps_per_cta < 0 || p->warps_per_cta > 16)
        return set_err(c, RCPSP_E_INVALID_ARG, "bad search parameters");
    const int gs = p->group_size;
    if (gs != 0 && gs != 1 && gs != 2 && gs != 4 && gs != 8 && gs != 16 && gs != 32)
        return set_err(c, RCPSP_E_INVALID_ARG, "group_size must be 0, 1, 2, 4, 8, 16 or 32");
    if (p->record_trace || p->use_graph || p->checkpoint || p->resume)
        return set_err(c, RCPSP_E_INVALID_ARG,
                       "co-operative searches keep no trace or state and capture no graph");
    const int B = cp->blocks, F = cp->working_set, P = cp->words_per_block;
    if (B < 1 || B > rcpsp::kMaxCoopBlocks || F < 1 || F > rcpsp::kMaxWorkingSet || cp->phi_max < 0 ||
        cp->phi_steps < 0 || cp->assign_fixed < 0 || P < 0 || cp->fbi_every < 0)
        return set_err(c, RCPSP_E_INVALID_ARG, "bad co-operation parameters");
    if (cp->phi_steps > 0 && (!random_words || P < 1))
        return set_err(c, RCPSP_E_INVALID_ARG, "diversification needs random words");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    if (count == 0) return RCPSP_OK;
    std::vector<LaunchItem> items(count);
    std::vector<double> cost(count);
    std::vector<size_t> key_off(count);
    size_t keys_total = 0;
    for (int k = 0; k < count; ++k) {
        const int id = ids[k];
        if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
            return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
        Inst &in = c->insts[id];
        LaunchItem &it = items[k];
        std::memset(&it, 0, sizeof(it));
        it.h = in.h;
        it.record = in.record;
        it.out = in.out;
        it.mode = p->eval_mode == RCPSP_EVAL_AUTO ? in.h.sel_mode : p->eval_mode;
        int dd, tl;
        rcpsp::default_search_params(in.h.n, &dd, &tl);
        it.delta = std::max(1, std::min(p->max_swap_dist ? p->max_swap_dist : dd, in.h.n - 3));
        it.tabu_len = p->tabu_len ? p->tabu_len : tl;
        it.iterations = p->iterations;
        it.stop_at_cp = p->stop_at_cp ? 1 : 0;
        in.trace_iters = -1;
        cost[k] = B * rcpsp::estimate_cost(in.h, it.mode, it.iterations, it.delta, it.stop_at_cp != 0);
        key_off[k] = keys_total;
        keys_total += static_cast<size_t>(F) * in.h.n;
    }
    // footprint classes as in rcpsp_tabu_search, each with its own shape
    // (every CTA of a cluster alike) and its own queue, longest first
    struct CoopLaunch {
        int offset = 0, count = 0, G = 0, warps = 0, move_cap = 0, nclusters = 0;
        size_t smem = 0;
        bool prefix = false;         // prefix reuse (kernel variant, kept states per CTA)
        int snap_words = 0;
        size_t snap_off = 0;
    };
    std::vector<int> order;
    order.reserve(count);
    std::vector<CoopLaunch> launches;
    const size_t static_smem = 3072;                       // the kernel's own bookkeeping
    const size_t smem_limit =
        c->prop.sharedMemPerBlockOptin > static_smem ? c->prop.sharedMemPerBlockOptin - static_smem : 0;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < kClasses; ++q) {
        std::vector<int> idx;
        for (int k = 0; k < count; ++k)
            if (footprint_class(items[k]) == q) idx.push_back(k);
        if (idx.empty()) continue;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        std::vector<LaunchItem> part;
        for (int k : idx) part.push_back(items[k]);
        CoopLaunch L;
        L.offset = static_cast<int>(order.size());
        L.count = static_cast<int>(idx.size());
        order.insert(order.end(), idx.begin(), idx.end());
        int G = gs, warps = p->warps_per_cta, dG, dW;
        default_shape(part, &dG, &dW);
        if (!gs && !warps) tuned_shape(c, shape_key(part), &dG, &dW);   // the search's tuned shape, if any
        if (!G) G = dG;
        if (!warps) warps = std::max(dW, (G + 31) / 32);
        L.move_cap = launch_move_cap(part);
        size_t smem = smem_bytes(part, warps * (32 / G), L.move_cap);
        while (smem > smem_limit && p->warps_per_cta == 0 && warps > 1) {
            --warps;
            smem = smem_bytes(part, warps * (32 / G), L.move_cap);
        }
        if (smem > smem_limit)
            return set_err(c, RCPSP_E_TOO_LARGE, "instance state does not fit in shared memory at this launch shape");
        // every CTA of a cluster evaluates the whole neighbourhood of its own
        // list, so prefix reuse pays as it does for a one-CTA search
        if (prefix_pays(part, warps * (32 / G), 1)) {
            L.prefix = true;
            L.snap_words = prefix_words_max(part);
            for (int k : idx) items[k].prefix_k = prefix_k_for(items[k].h.n);
        }
        int clusters = 0;
        e = rcpsp::coop_occupancy(G, warps * 32, smem, B, &clusters, L.prefix);
        if (e != cudaSuccess) return cuda_err(c, e, "co-operative occupancy");
        if (clusters < 1)
            return set_err(c, RCPSP_E_TOO_LARGE, "a cluster of this many CTAs does not fit at this shape");
        L.G = G;
        L.warps = warps;
        L.smem = smem;
        L.nclusters = std::max(1, std::min(L.count, clusters));
        launches.push_back(L);
    }
    // kept prefix states: one region per CTA of every launch that uses them
    {
        size_t need = 0;
        for (CoopLaunch &L : launches)
            if (L.prefix) {
                L.snap_off = need;
                need += static_cast<size_t>(L.nclusters) * B * L.snap_words;
            }
        if (need * 4 > c->snap_cap) {
            dev_free(c, c->snap_dev, c->snap_cap, nullptr);
            c->snap_dev = static_cast<int32_t *>(dev_alloc(c, need * 4, nullptr));
            c->snap_cap = c->snap_dev ? need * 4 : 0;
            if (!c->snap_dev) return set_err(c, RCPSP_E_CUDA, "prefix scratch allocation failed");
        }
    }
    // device block: [plan][initial lists][random words][working sets]; the
    // first three are uploaded, the working sets are written by the kernel
    auto up16 = [](size_t x) { return (x + 15) & ~static_cast<size_t>(15); };
    const size_t plan_bytes = up16(sizeof(rcpsp::CoopItem) * count);
    const size_t lists_bytes = up16(keys_total * 4);
    const size_t words_bytes = up16(random_words ? static_cast<size_t>(count) * B * P * 4 : 0);
    size_t slots_bytes = 0;
    std::vector<size_t> slot_off(count);
    for (int k = 0; k < count; ++k) {
        slot_off[k] = slots_bytes;
        const rcpsp::SlotLayout SL = rcpsp::slot_layout(items[k].h.n, items[k].tabu_len, items[k].delta);
        slots_bytes += up16(static_cast<size_t>(F) * SL.words * 4);
    }
    const size_t up_bytes = plan_bytes + lists_bytes + words_bytes;
    const size_t total = up_bytes + slots_bytes;
    if (c->coop_cap < total) {
        dev_free(c, c->coop_dev, c->coop_cap, nullptr);
        c->coop_dev = dev_alloc(c, total, nullptr);
        c->coop_cap = c->coop_dev ? total : 0;
        if (!c->coop_dev) return set_err(c, RCPSP_E_CUDA, "working-set allocation failed");
    }
    if (c->coop_host_cap < up_bytes) {
        if (c->coop_host) cudaFreeHost(c->coop_host);
        c->coop_host = nullptr;
        c->coop_host_cap = 0;
        e = cudaMallocHost(reinterpret_cast<void **>(&c->coop_host), up_bytes);
        if (e != cudaSuccess) return cuda_err(c, e, "pinned staging");
        c->coop_host_cap = up_bytes;
    }
    char *hb = c->coop_host, *db = static_cast<char *>(c->coop_dev);
    std::memset(hb, 0, up_bytes);
    auto *plan = reinterpret_cast<rcpsp::CoopItem *>(hb);
    auto *lists = reinterpret_cast<int32_t *>(hb + plan_bytes);
    for (int q = 0; q < count; ++q) {
        const int k = order[q];
        const Inst &in = c->insts[ids[k]];
        const int n = in.h.n;
        for (int f = 0; f < F; ++f)
            rcpsp::level_order(n, in.succ_off.data(), in.succ.data(),
                               slot_keys ? slot_keys + key_off[k] + static_cast<size_t>(f) * n : nullptr,
                               lists + key_off[k] + static_cast<size_t>(f) * n);
        rcpsp::CoopItem &ci = plan[q];
        ci.base = items[k];
        ci.slots = reinterpret_cast<int32_t *>(db + up_bytes + slot_off[k]);
        ci.init_lists = reinterpret_cast<const int32_t *>(db + plan_bytes) + key_off[k];
        ci.words = random_words ? reinterpret_cast<const uint32_t *>(db + plan_bytes + lists_bytes) +
                                      static_cast<size_t>(k) * B * P
                                : nullptr;
        ci.slot_words = rcpsp::slot_layout(n, items[k].tabu_len, items[k].delta).words;
    }
    if (random_words)
        std::memcpy(hb + plan_bytes + lists_bytes, random_words, static_cast<size_t>(count) * B * P * 4);
    e = cudaMemcpyAsync(db, hb, up_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->queue_dev, 0, sizeof(int) * kMaxLaunches, st);
    if (e != cudaSuccess) return cuda_err(c, e, "co-operative search upload");
    c->h2d += static_cast<long long>(up_bytes);
    // one launch per class; classes after the first run on forked streams
    // and join back before the done event
    rcpsp::CoopConfig cfg{B, F, cp->phi_max, cp->phi_steps, cp->assign_fixed, P, cp->fbi_every};
    if (launches.size() > 1 && (e = cudaEventRecord(c->fork, st)) != cudaSuccess)
        return cuda_err(c, e, "event record");
    for (size_t q = 0; q < launches.size(); ++q) {
        const CoopLaunch &L = launches[q];
        cudaStream_t sq = q == 0 ? st : c->aux[q - 1];
        if (q > 0 && (e = cudaStreamWaitEvent(sq, c->fork, 0)) != cudaSuccess) return cuda_err(c, e, "stream fork");
        e = rcpsp::launch_coop(L.G, reinterpret_cast<const rcpsp::CoopItem *>(db) + L.offset, L.count,
                               c->queue_dev + q, L.move_cap, cfg, L.nclusters * B, L.warps * 32, L.smem, sq,
                               L.prefix, L.prefix ? c->snap_dev + L.snap_off : nullptr, L.snap_words);
        if (e != cudaSuccess) return cuda_err(c, e, "co-operative search launch");
        c->kernels += 1;
        if (q > 0 && (e = cudaEventRecord(c->join[q - 1], sq)) != cudaSuccess) return cuda_err(c, e, "event record");
    }
    for (size_t q = 1; q < launches.size(); ++q)
        if ((e = cudaStreamWaitEvent(st, c->join[q - 1], 0)) != cudaSuccess) return cuda_err(c, e, "stream join");
    e = cudaEventRecord(c->done, st);
    if (e != cudaSuccess) return cuda_err(c, e, "event record");
    c->pending = true;
    return RCPSP_OK;
}

int rcpsp_tabu_search_noalloc(rcpsp_ctx *c, const int32_t *ids, int32_t count, const rcpsp_params *p,
                              void *stream) {
    HostRange range("rcpsp_tabu_search_noalloc");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (!p || count < 0 || (count > 0 && !ids)) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    if (p->iterations < 0 || p->max_swap_dist < 0 || p->tabu_len < 0 || p->tabu_len > RCPSP_MAX_TABU ||
        p->eval_mode < 0 || p->eval_mode > 2 || p->warps_per_cta < 0 || p->warps_per_cta > rcpsp::kSearchMaxWarps)
        return set_err(c, RCPSP_E_INVALID_ARG, "bad search parameters");
    const int gs = p->group_size;
    if (gs != 0 && gs != 1 && gs != 2 && gs != 4 && gs != 8 && gs != 16 && gs != 32)
        return set_err(c, RCPSP_E_INVALID_ARG, "group_size must be 0, 1, 2, 4, 8, 16 or 32");
    if (p->record_trace || p->use_graph || p->checkpoint || p->resume)
        return set_err(c, RCPSP_E_INVALID_ARG,
                       "the no-allocation search keeps no trace or state and captures no graph");
    if (p->cluster_size != 0 && p->cluster_size != 1)
        return set_err(c, RCPSP_E_INVALID_ARG, "the no-allocation search runs one CTA per search (cluster_size 0 or 1)");
    if (count > rcpsp::noalloc_max_items())
        return set_err(c, RCPSP_E_TOO_LARGE, "the no-allocation search takes at most " +
                                                 std::to_string(rcpsp::noalloc_max_items()) + " instances per call");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    if (count == 0) return RCPSP_OK;
    std::vector<LaunchItem> items(count);
    std::vector<double> cost(count);
    for (int k = 0; k < count; ++k) {
        const int id = ids[k];
        if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
            return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
        Inst &in = c->insts[id];
        LaunchItem &it = items[k];
        std::memset(&it, 0, sizeof(it));
        it.h = in.h;
        it.record = in.record;
        it.out = in.out;
        it.mode = p->eval_mode == RCPSP_EVAL_AUTO ? in.h.sel_mode : p->eval_mode;
        int dd, tl;
        rcpsp::default_search_params(in.h.n, &dd, &tl);
        // v - u never exceeds N - 3, so a larger delta names the same moves
        it.delta = std::max(1, std::min(p->max_swap_dist ? p->max_swap_dist : dd, in.h.n - 3));
        it.tabu_len = p->tabu_len ? p->tabu_len : tl;
        it.iterations = p->iterations;
        it.stop_at_cp = p->stop_at_cp ? 1 : 0;
        in.trace_iters = -1;
        cost[k] = rcpsp::estimate_cost(in.h, it.mode, it.iterations, it.delta, it.stop_at_cp != 0);
    }
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    c->noalloc_plan.resize(count);
    for (int k = 0; k < count; ++k) c->noalloc_plan[k] = items[order[k]];
    int G = gs, warps = p->warps_per_cta;
    int dG, dW;
    default_shape(c->noalloc_plan, &dG, &dW);
    if (!gs && !warps) tuned_shape(c, shape_key(c->noalloc_plan), &dG, &dW);
    if (!G) G = dG;
    if (!warps) warps = std::max(dW, (G + 31) / 32);
    const int move_cap = launch_move_cap(c->noalloc_plan);
    const size_t smem_limit = c->prop.sharedMemPerBlockOptin > 1024 ? c->prop.sharedMemPerBlockOptin - 1024 : 0;
    size_t smem = smem_bytes(c->noalloc_plan, warps * (32 / G), move_cap);
    while (smem > smem_limit && p->warps_per_cta == 0 && warps > 1) {
        --warps;
        smem = smem_bytes(c->noalloc_plan, warps * (32 / G), move_cap);
    }
    if (smem > smem_limit)
        return set_err(c, RCPSP_E_TOO_LARGE, "instance state does not fit in shared memory at this launch shape");
    const int threads = warps * 32;
    int *queue = nullptr;
    LaunchItem *plan = nullptr;
    cudaError_t e = rcpsp::noalloc_scratch(c->device, &queue, &plan);
    if (e != cudaSuccess) return cuda_err(c, e, "scratch address");
    // the same process-wide limit rcpsp_tabu_search sets, so that the value
    // only ever goes up for a launch on another thread or context
    e = rcpsp::prepare_search(G, smem_limit);
    if (e != cudaSuccess) return cuda_err(c, e, "kernel attributes");
    int per_sm = 0;
    e = rcpsp::search_occupancy(G, threads, smem, 1, &per_sm);
    if (e != cudaSuccess) return cuda_err(c, e, "occupancy");
    if (per_sm < 1) return set_err(c, RCPSP_E_TOO_LARGE, "launch shape does not fit on an SM");
    const int blocks = std::max(1, std::min(count, per_sm * c->prop.multiProcessorCount));
    const size_t ibytes = sizeof(LaunchItem) * count;
    e = cudaMemcpyAsync(plan, c->noalloc_plan.data(), ibytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, sizeof(int), st);      // the counter starts at 0
    if (e == cudaSuccess) e = rcpsp::launch_search(G, plan, count, queue, move_cap, blocks, threads, smem, st, 1);
    if (e != cudaSuccess) return cuda_err(c, e, "no-allocation search launch");
    c->h2d += static_cast<long long>(ibytes);
    c->kernels += 1;
    e = cudaEventRecord(c->done, st);
    if (e != cudaSuccess) return cuda_err(c, e, "event record");
    c->pending = true;
    return RCPSP_OK;
}

int rcpsp_autotune(rcpsp_ctx *c, const int32_t *ids, int32_t count, const rcpsp_params *p, int32_t trial_iterations,
                   void *stream, int32_t *best_group_size, int32_t *best_warps, int32_t *best_cluster_size) {
    HostRange range("rcpsp_autotune");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (!p || count <= 0 || !ids || trial_iterations < 1) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    // the signature of the real search (its parameters, not the trial's)
    std::vector<LaunchItem> items(count);
    for (int k = 0; k < count; ++k) {
        const int id = ids[k];
        if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
            return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
        const Inst &in = c->insts[id];
        LaunchItem &it = items[k];
        std::memset(&it, 0, sizeof(it));
        it.h = in.h;
        it.mode = p->eval_mode == RCPSP_EVAL_AUTO ? in.h.sel_mode : p->eval_mode;
        int dd, tl;
        rcpsp::default_search_params(in.h.n, &dd, &tl);
        // v - u never exceeds N - 3, so a larger delta names the same moves
        it.delta = std::max(1, std::min(p->max_swap_dist ? p->max_swap_dist : dd, in.h.n - 3));
        it.tabu_len = p->tabu_len ? p->tabu_len : tl;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_err(c, RCPSP_E_CUDA, "event create");
    rcpsp_params q = *p;
    q.iterations = std::min(p->iterations, trial_iterations);
    q.record_trace = 0;
    q.use_graph = 0;
    q.checkpoint = 0;
    q.resume = 0;
    int ret_G = 0, ret_W = 0, ret_C = 0, ret_count = -1;
    std::vector<std::string> tuned_keys;        // signatures of the classes tuned here
    std::vector<std::vector<std::array<int, 3>>> tuned_top;   // their three fastest shapes alone
    std::string ret_key;
    // each footprint class is tuned on its own (searches launch them apart)
    for (int cls = 0; cls < kClasses; ++cls) {
        std::vector<int32_t> cids;
        std::vector<LaunchItem> part;
        for (int k = 0; k < count; ++k)
            if (footprint_class(items[k]) == cls) {
                cids.push_back(ids[k]);
                part.push_back(items[k]);
            }
        if (cids.empty()) continue;
        const int cn = static_cast<int>(cids.size());
        const std::string key = shape_key(part);
        std::vector<rcpsp_stats> stats(cn);
        double best_rate = -1.0;
        int bG = 0, bW = 0, bC = 1;
        std::vector<std::pair<double, std::array<int, 3>>> ranked;   // (rate, shape) of every trial
        const int gsz[] = {1, 2, 4, 8, 16, 32};
        const int wcnt[] = {1, 2, 3, 4, 6, 8, 10, 12, 16};
        // clusters pay when the class has fewer searches than the GPU has SMs,
        // or when its searches are large (N > 160: long decode chains and big
        // neighbourhoods, which would otherwise leave the GPU to a few
        // long-running CTAs at the end of the call)
        const int cmax = (2 * cn <= c->prop.multiProcessorCount || cls % 3 == 2) ? 8 : 1;
        for (int C = 1; C <= cmax; C *= 2)
        for (int G : gsz)
            for (int W : wcnt) {
                const int ng = W * (32 / G);
                const int fp = cls / 3, sz = cls % 3;                        // large states fit few groups
                const int min_groups = fp <= 1 ? (sz == 0 ? 8 : 2) : (fp == 2 ? 2 : 1);
                if (ng < min_groups || ng > 256) continue;
                if (C > 1 && (G < 4 || W < 4)) continue;                     // fewer trials for clusters
                q.group_size = G;
                q.warps_per_cta = W;
                q.cluster_size = C;
                cudaEventRecord(e0, st);
                int r = rcpsp_tabu_search(c, cids.data(), cn, &q, stream);
                if (r == RCPSP_E_TOO_LARGE) continue;             // shape does not fit
                if (r == RCPSP_OK) {
                    cudaEventRecord(e1, st);
                    r = rcpsp_get_schedules(c, cids.data(), cn, nullptr, nullptr, nullptr, stats.data());
                }
                if (r != RCPSP_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return r;
                }
                float ms = 0.f;
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                long long ev = 0;
                for (const rcpsp_stats &x : stats) ev += x.evaluated;
                const double rate = ms > 0 ? static_cast<double>(ev > 0 ? ev : 1) / ms : 0.0;
                ranked.push_back({rate, {G, W, C}});
                if (rate > best_rate) {
                    best_rate = rate;
                    bG = G;
                    bW = W;
                    bC = C;
                }
            }
        // short trials can rank shapes by their first iterations only: the
        // three best are timed again with four times as many iterations
        if (ranked.size() > 1 && p->iterations > q.iterations) {
            std::stable_sort(ranked.begin(), ranked.end(),
                             [](const auto &a, const auto &b) { return a.first > b.first; });
            rcpsp_params q4 = q;
            q4.iterations = std::min(p->iterations, 4 * q.iterations);
            double best4 = -1.0;
            for (size_t t = 0; t < ranked.size() && t < 3; ++t) {
                q4.group_size = ranked[t].second[0];
                q4.warps_per_cta = ranked[t].second[1];
                q4.cluster_size = ranked[t].second[2];
                cudaEventRecord(e0, st);
                int r = rcpsp_tabu_search(c, cids.data(), cn, &q4, stream);
                if (r == RCPSP_OK) {
                    cudaEventRecord(e1, st);
                    r = rcpsp_get_schedules(c, cids.data(), cn, nullptr, nullptr, nullptr, stats.data());
                }
                if (r != RCPSP_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return r;
                }
                float ms = 0.f;
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                long long ev = 0;
                for (const rcpsp_stats &x : stats) ev += x.evaluated;
                const double rate = ms > 0 ? static_cast<double>(ev > 0 ? ev : 1) / ms : 0.0;
                if (rate > best4) {
                    best4 = rate;
                    bG = ranked[t].second[0];
                    bW = ranked[t].second[1];
                    bC = ranked[t].second[2];
                }
            }
        }
        if (!bG) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return set_err(c, RCPSP_E_TOO_LARGE, "no launch shape fits");
        }
        bool found = false;
        for (auto &e : c->tuned)
            if (e.first == key) {
                e.second = {bG, bW, bC};
                found = true;
            }
        if (!found) c->tuned.push_back({key, {bG, bW, bC}});
        if (cn > ret_count) {
            ret_count = cn;
            ret_G = bG;
            ret_W = bW;
            ret_C = bC;
            ret_key = key;
        }
        tuned_keys.push_back(key);
        std::vector<std::array<int, 3>> top;
        for (size_t t = 0; t < ranked.size() && t < 3; ++t) top.push_back(ranked[t].second);
        tuned_top.push_back(top);
    }
    // The classes of a call share the GPU, so a shape that is best for a
    // class alone can hold SMs the other classes need: with more than one
    // class, each class's three fastest shapes alone and the other cluster
    // sizes of its pick are timed with the whole call running (every other
    // class at its current shape), keeping a change only if the call gets at
    // least 3% faster.
    if (tuned_keys.size() > 1) {
        q.group_size = q.warps_per_cta = q.cluster_size = 0;
        std::vector<rcpsp_stats> stats(count);
        auto time_call = [&](double *ms_out) -> int {
            double best = 1e30;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, st);
                int r = rcpsp_tabu_search(c, ids, count, &q, stream);
                if (r == RCPSP_OK) {
                    cudaEventRecord(e1, st);
                    r = rcpsp_get_schedules(c, ids, count, nullptr, nullptr, nullptr, stats.data());
                }
                if (r != RCPSP_OK) return r;
                float ms = 0.f;
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                best = std::min(best, static_cast<double>(ms));
            }
            *ms_out = best;
            return RCPSP_OK;
        };
        double base_ms = 0;
        int r = time_call(&base_ms);
        for (size_t t = 0; r == RCPSP_OK && t < tuned_keys.size(); ++t) {
            std::array<int, 3> *sh = nullptr;
            for (auto &e : c->tuned)
                if (e.first == tuned_keys[t]) sh = &e.second;
            if (!sh) continue;
            std::vector<std::array<int, 3>> cand = tuned_top[t];
            for (int C = 1; C <= 8; C *= 2)
                if (C != (*sh)[2] && (C == 1 || ((*sh)[0] >= 4 && (*sh)[1] >= 4))) cand.push_back({(*sh)[0], (*sh)[1], C});
            const std::array<int, 3> orig = *sh;
            std::array<int, 3> keep = orig;
            for (const std::array<int, 3> &x : cand) {
                if (x == orig) continue;
                *sh = x;
                double ms = 0;
                const int rr = time_call(&ms);
                if (rr == RCPSP_E_TOO_LARGE) continue;        // does not fit at this shape
                if (rr != RCPSP_OK) {
                    r = rr;
                    break;
                }
                if (ms < 0.97 * base_ms) {
                    base_ms = ms;
                    keep = x;
                }
            }
            *sh = keep;
            if (tuned_keys[t] == ret_key) {
                ret_G = keep[0];
                ret_W = keep[1];
                ret_C = keep[2];
            }
        }
        if (r != RCPSP_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return r;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    save_tune_cache(c);
    if (best_group_size) *best_group_size = ret_G;
    if (best_warps) *best_warps = ret_W;
    if (best_cluster_size) *best_cluster_size = ret_C;
    return RCPSP_OK;
}

int rcpsp_get_schedules(rcpsp_ctx *c, const int32_t *ids, int32_t count, int32_t *order, int32_t *start,
                        int32_t *makespan, rcpsp_stats *stats) {
    HostRange range("rcpsp_get_schedules");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (count < 0 || (count > 0 && !ids)) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    // one copy per block touched
    std::vector<int> touched;
    for (int k = 0; k < count; ++k) {
        const int id = ids[k];
        if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
            return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
        touched.push_back(c->insts[id].block);
    }
    std::sort(touched.begin(), touched.end());
    touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
    std::vector<std::vector<int32_t>> host(c->blocks.size());
    for (int b : touched) {
        Block &bl = c->blocks[b];
        host[b].resize(bl.out_bytes / 4);
        cudaError_t e = cudaMemcpy(host[b].data(), static_cast<char *>(bl.ptr) + bl.out_offset, bl.out_bytes,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(c, e, "result copy");
        c->d2h += static_cast<long long>(bl.out_bytes);
    }
    size_t at = 0;
    int status = RCPSP_OK;
    for (int k = 0; k < count; ++k) {
        const Inst &in = c->insts[ids[k]];
        const int n = in.h.n;
        const int32_t *o = host[in.block].data() + in.out_word;
        const int32_t *s = o + 2 * n;
        if (order) std::memcpy(order + at, o, n * 4);
        if (start) std::memcpy(start + at, o + n, n * 4);
        at += n;
        if (makespan) makespan[k] = s[rcpsp::kOutCmax];
        if (stats) {
            rcpsp_stats &x = stats[k];
            x.evaluated = (static_cast<int64_t>(s[rcpsp::kOutEvalHi]) << 32) | static_cast<uint32_t>(s[rcpsp::kOutEvalLo]);
            x.work = (static_cast<int64_t>(s[rcpsp::kOutWorkHi]) << 32) | static_cast<uint32_t>(s[rcpsp::kOutWorkLo]);
            x.iterations = s[rcpsp::kOutIters];
            x.eval_mode = s[rcpsp::kOutMode];
            x.critical_path = in.h.cp;
            x.status = s[rcpsp::kOutStatus];
            x.t_start_ns = (static_cast<int64_t>(s[rcpsp::kOutT0Hi]) << 32) | static_cast<uint32_t>(s[rcpsp::kOutT0Lo]);
            x.t_end_ns = (static_cast<int64_t>(s[rcpsp::kOutT1Hi]) << 32) | static_cast<uint32_t>(s[rcpsp::kOutT1Lo]);
            int64_t *ta[rcpsp::kTallies] = {&x.placements, &x.steps_done, &x.update_units, &x.succ_pushes,
                                            &x.kept_words};
            for (int t = 0; t < rcpsp::kTallies; ++t)
                *ta[t] = (static_cast<int64_t>(s[rcpsp::kOutPlacedLo + 2 * t + 1]) << 32) |
                         static_cast<uint32_t>(s[rcpsp::kOutPlacedLo + 2 * t]);
        }
        if (s[rcpsp::kOutStatus] != 0) status = RCPSP_E_DEVICE;
    }
    if (status != RCPSP_OK) return set_err(c, status, "a search reported an internal error");
    return RCPSP_OK;
}

int rcpsp_get_trace(rcpsp_ctx *c, int32_t id, int32_t *trace, int32_t capacity, int32_t *written) {
    if (!c) return RCPSP_E_INVALID_ARG;
    if (!trace || capacity < 0 || !written) return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    cudaSetDevice(c->device);
    int rc = wait_done(c);
    if (rc != RCPSP_OK) return rc;
    if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
        return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
    const Inst &in = c->insts[id];
    if (in.trace_iters < 0 || !in.trace) return set_err(c, RCPSP_E_INVALID_ARG, "no trace recorded");
    int32_t words[rcpsp::kOutStats];
    cudaError_t e = cudaMemcpy(words, in.out + 2 * in.h.n, sizeof(words), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(c, e, "trace copy");
    const int32_t iters = words[rcpsp::kOutIters] - words[rcpsp::kOutIters0];   // this call's iterations
    if (static_cast<long long>(iters) * 3 > capacity) return set_err(c, RCPSP_E_INVALID_ARG, "trace buffer too small");
    if (iters > 0) {
        e = cudaMemcpy(trace, in.trace, static_cast<size_t>(iters) * 3 * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(c, e, "trace copy");
        c->d2h += static_cast<long long>(iters) * 12;
    }
    *written = iters;
    return RCPSP_OK;
}

int rcpsp_evaluate_lists(rcpsp_ctx *c, int32_t id, const int32_t *lists, int32_t count, int32_t eval_mode,
                         int32_t *start, int32_t *makespan, int64_t *work, void *stream) {
    HostRange range("rcpsp_evaluate_lists");
    if (!c) return RCPSP_E_INVALID_ARG;
    if (count < 0 || (count > 0 && !lists) || eval_mode < 0 || eval_mode > 2)
        return set_err(c, RCPSP_E_INVALID_ARG, "bad arguments");
    cudaSetDevice(c->device);
    if (id < 0 || id >= static_cast<int>(c->insts.size()) || !c->insts[id].alive)
        return set_err(c, RCPSP_E_NOT_FOUND, "unknown instance id");
    if (count == 0) return RCPSP_OK;
    const Inst &in = c->insts[id];
    const int n = in.h.n;
    // every list must be a precedence-feasible permutation with the dummies fixed
    {
        std::vector<int> pos(n);
        for (int l = 0; l < count; ++l) {
            const int32_t *L = lists + static_cast<size_t>(l) * n;
            std::fill(pos.begin(), pos.end(), -1);
            for (int p = 0; p < n; ++p) {
                if (L[p] < 0 || L[p] >= n || pos[L[p]] >= 0)
                    return set_err(c, RCPSP_E_INVALID_ARG, "list " + std::to_string(l) + " is not a permutation");
                pos[L[p]] = p;
            }
            if (L[0] != 0 || L[n - 1] != n - 1)
                return set_err(c, RCPSP_E_INVALID_ARG, "list " + std::to_string(l) + " moves a dummy activity");
            for (int i = 0; i < n; ++i)
                for (int e = in.succ_off[i]; e < in.succ_off[i + 1]; ++e)
                    if (pos[i] > pos[in.succ[e]])
                        return set_err(c, RCPSP_E_INVALID_ARG, "list " + std::to_string(l) + " violates a precedence");
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LaunchItem it;
    std::memset(&it, 0, sizeof(it));
    it.h = in.h;
    it.record = in.record;
    it.mode = eval_mode == RCPSP_EVAL_AUTO ? in.h.sel_mode : eval_mode;
    // largest of a few shapes whose profiles fit in shared memory
    const int pw = rcpsp::profile_words(it.mode, in.h.wps, in.h.ub, in.h.sum_cap);
    const int shapes[][2] = {{8, 4}, {8, 2}, {8, 1}, {16, 1}, {32, 1}};
    int G = 0, warps = 0, ngroups = 0;
    size_t smem = 0;
    for (const auto &sh : shapes) {
        const int ng = sh[1] * (32 / sh[0]);
        const rcpsp::StateLayout S =
            rcpsp::state_layout(in.h.inst_words, n, 0, 0, ng * rcpsp::align4(n), pw, ng, it.mode);
        smem = static_cast<size_t>(S.total) * 4;
        if (smem + 1024 <= c->prop.sharedMemPerBlockOptin) {
            G = sh[0];
            warps = sh[1];
            ngroups = ng;
            break;
        }
    }
    if (!G) return set_err(c, RCPSP_E_TOO_LARGE, "profile too large for shared memory");
    // output block: work [count] int64 first (8-byte aligned), then start
    // [count*N], makespan [count] and the error word, each 16-byte aligned
    auto up16 = [](size_t x) { return (x + 15) & ~static_cast<size_t>(15); };
    const size_t lbytes = static_cast<size_t>(count) * n * 4;
    const size_t o_work = 0;
    const size_t o_start = up16(static_cast<size_t>(count) * 8);
    const size_t o_cmax = o_start + up16(lbytes);
    const size_t o_err = o_cmax + up16(static_cast<size_t>(count) * 4);
    const size_t obytes = o_err + 16;
    char *dl = static_cast<char *>(dev_alloc(c, lbytes, st));
    char *dout = static_cast<char *>(dev_alloc(c, obytes, st));
    if (!dl || !dout) {
        dev_free(c, dl, lbytes, st);
        dev_free(c, dout, obytes, st);
        return set_err(c, RCPSP_E_CUDA, "device allocation failed");
    }
    long long *d_work = reinterpret_cast<long long *>(dout + o_work);
    int32_t *d_start = reinterpret_cast<int32_t *>(dout + o_start);
    int32_t *d_cmax = reinterpret_cast<int32_t *>(dout + o_cmax);
    int *d_err = reinterpret_cast<int *>(dout + o_err);
    std::vector<char> host(obytes);
    int rc = RCPSP_OK;
    cudaError_t e = cudaMemcpyAsync(dl, lists, lbytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, 4, st);
    if (e == cudaSuccess) {
        const int blocks = std::max(1, std::min((count + ngroups - 1) / ngroups, 4 * c->prop.multiProcessorCount));
        e = rcpsp::launch_evaluate(G, it, reinterpret_cast<int32_t *>(dl), count, d_start, d_cmax, d_work, d_err,
                                   blocks, warps * 32, smem, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), dout, obytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_err(c, e, "evaluate");
    dev_free(c, dl, lbytes, st);
    dev_free(c, dout, obytes, st);
    if (rc != RCPSP_OK) return rc;
    c->h2d += static_cast<long long>(lbytes);
    c->d2h += static_cast<long long>(obytes);
    c->kernels += 1;
    if (start) std::memcpy(start, host.data() + o_start, lbytes);
    if (work) std::memcpy(work, host.data() + o_work, static_cast<size_t>(count) * 8);
    if (makespan) std::memcpy(makespan, host.data() + o_cmax, static_cast<size_t>(count) * 4);
    int derr = 0;
    std::memcpy(&derr, host.data() + o_err, 4);
    if (derr) return set_err(c, RCPSP_E_DEVICE, "decode reported an internal error");
    return RCPSP_OK;
}

}  // extern "C"
