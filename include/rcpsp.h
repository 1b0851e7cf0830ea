/*
 * rcpsp.h -- C interface of the GB300 tabu-search library for the Resource
 * Constrained Project Scheduling Problem (makespan), after Bukata, Sucha and
 * Hanzalek, "Solving the RCPSP using the parallel tabu search designed for the
 * CUDA platform" (J. Parallel Distrib. Comput. 77, 2015).
 *
 * Conventions for every call:
 *   - all integers are int32 unless stated; arrays are dense and row-major;
 *   - a pointer argument documented "host" must point to host memory;
 *   - the library copies every input it is given before the call returns;
 *     the caller keeps ownership of its buffers;
 *   - device memory belongs to the context; it is taken from the allocator
 *     passed to rcpsp_create (for example PyTorch's caching allocator) or,
 *     without one, from cudaMalloc;
 *   - calls return RCPSP_OK (0) or a negative RCPSP_E_* code; the text of the
 *     last failure of a context is given by rcpsp_last_error; no call throws
 *     across the interface;
 *   - a context is used by one host thread at a time.
 */
#ifndef RCPSP_H
#define RCPSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ limits */
#define RCPSP_MAX_N 1024        /* activities, dummies included            */
#define RCPSP_MAX_M 8           /* renewable resources                      */
#define RCPSP_MAX_CAP 32767     /* largest capacity R_k                     */
#define RCPSP_MAX_HORIZON 32767 /* largest sum of durations (UB of Sec. 5.2) */
#define RCPSP_MAX_TABU 8192     /* largest |tabuList|                       */

/* ------------------------------------------------------- error codes */
enum {
    RCPSP_OK = 0,
    RCPSP_E_INVALID_ARG = -1,         /* bad pointer, size or parameter           */
    RCPSP_E_CYCLE = -2,               /* precedence graph has a cycle             */
    RCPSP_E_DUMMY = -3,               /* 0 / N-1 are not the unique source / sink
                                         with zero duration and demand            */
    RCPSP_E_DEMAND_EXCEEDS_CAP = -4,  /* r_{i,k} > R_k                            */
    RCPSP_E_TOO_LARGE = -5,           /* beyond a RCPSP_MAX_* limit or shared memory */
    RCPSP_E_CUDA = -6,                /* a CUDA runtime call failed               */
    RCPSP_E_TIMEOUT = -7,             /* a bounded wait ran out                   */
    RCPSP_E_NOT_FOUND = -8,           /* unknown instance id                      */
    RCPSP_E_DEVICE = -9               /* a kernel reported an internal error      */
};

/* Resource evaluation algorithm (Sec. 5). */
enum {
    RCPSP_EVAL_AUTO = 0,      /* per instance, by the selection rule (Sec. 5.4) */
    RCPSP_EVAL_TIME = 1,      /* time-indexed: Algs. 5-6                         */
    RCPSP_EVAL_CAPACITY = 2   /* capacity-indexed: Eq. 7 and Alg. 4             */
};

/* One instance, as in the problem statement (Sec. 2): N activities with
 * dummies 0 and N-1 (zero duration and demand, 0 the only activity without a
 * predecessor, N-1 the only one without a successor), durations d_i, M
 * resources with capacities R_k, demands r_{i,k} <= R_k, and the precedence
 * arcs E as successor lists.  Activities need not be numbered topologically.
 * All pointers are host pointers. */
typedef struct {
    int32_t n;                  /* N, dummies included, 3 <= N <= RCPSP_MAX_N  */
    int32_t m;                  /* M, 1 <= M <= RCPSP_MAX_M                     */
    const int32_t *dur;         /* [N] durations d_i >= 0, d_0 = d_{N-1} = 0    */
    const int32_t *cap;         /* [M] capacities 1 <= R_k <= RCPSP_MAX_CAP    */
    const int32_t *req;         /* [N*M] demands, req[i*M+k] = r_{i,k}          */
    const int32_t *succ_off;    /* [N+1] CSR offsets into succ                   */
    const int32_t *succ;        /* [succ_off[N]] successor lists (arcs (i,j))   */
    const int32_t *level_key;   /* [N] or NULL: order inside a level of the
                                   initial list (Sec. 4.1 "shuffling"); the
                                   list sorts by (level, key, label)          */
} rcpsp_instance;

/* Search parameters (Sec. 6, Table 2) and launch shape. */
typedef struct {
    int32_t iterations;         /* iteration limit per instance, >= 0            */
    int32_t max_swap_dist;      /* delta of the reduced neighbourhood (Sec. 4.3) */
    int32_t tabu_len;           /* |tabuList| of the simple tabu list (Sec. 4.5) */
    int32_t eval_mode;          /* RCPSP_EVAL_*                                  */
    int32_t stop_at_cp;         /* 1: stop once C*_max equals the critical path  */
    int32_t group_size;         /* lanes per neighbour decode: 1,2,4,8,16,32;
                                   0 = choose automatically                      */
    int32_t warps_per_cta;      /* 1..16; 0 = choose automatically               */
    int32_t record_trace;       /* 1: keep (u, v, C) of every iteration          */
    int32_t use_graph;          /* 1: capture the launch in a CUDA graph and
                                   replay it on later identical calls            */
    int32_t cluster_size;       /* CTAs that share one search (1, 2, 4, 8): they
                                   split its neighbourhood and exchange the best
                                   move through distributed shared memory;
                                   0 = choose automatically                      */
    int32_t checkpoint;         /* 1: keep each search's state on the device when
                                   the call ends (lists, tabu list and cache,
                                   iteration, counters), for `resume` or
                                   rcpsp_get_state                               */
    int32_t resume;             /* 1: continue each instance from its kept state
                                   for `iterations` more iterations; it must have
                                   been kept with the same swap distance, tabu
                                   length and evaluator.  Counters and the
                                   iteration count continue, so k1 iterations
                                   then k2 resumed equal k1+k2 in one call.  The
                                   trace of a resumed call holds its own
                                   iterations.                                    */
    int32_t slices;             /* scheduling of a launch class with more searches
                                   than the GPU holds at once (not of the
                                   results, which are the same either way): each
                                   search runs in `slices` slices of
                                   ceil(iterations / slices) iterations, every
                                   search's first slice before any second one,
                                   the state kept in device memory in between, so
                                   that the searches that start last do not run
                                   alone at the end of the call.  0 = choose
                                   automatically, 1 = never, 2..64 = that many in
                                   every class.  Not part of the paper.           */
} rcpsp_params;

/* Result statistics of one instance. */
typedef struct {
    int64_t evaluated;          /* neighbour schedules decoded (Sched_sec count) */
    int64_t work;               /* Alg. 5 loop steps (time-indexed) or Alg. 4
                                   loop steps (capacity-indexed) of those decodes */
    int32_t iterations;         /* iterations performed                         */
    int32_t eval_mode;          /* evaluator used (RCPSP_EVAL_TIME / _CAPACITY)  */
    int32_t critical_path;      /* critical-path length (Sec. 2)                */
    int32_t status;             /* 0, or a negative RCPSP_E_* code              */
    int64_t t_start_ns;         /* device global timer when the search started   */
    int64_t t_end_ns;           /* device global timer when its results were out */
    /* Work the decodes of the last call performed, for throughput
     * accounting (a resumed search counts only its own call).  With prefix
     * reuse a neighbour's decode restores the decoder state of the current
     * list before its first swapped position instead of placing those
     * activities again; the positions it restores are not counted here,
     * while `evaluated` and `work` above count every neighbour in full.
     * Counted: the neighbour decodes and the decodes of the current list
     * that produce the kept states (not the first and last decode of a
     * search). */
    int64_t placements;         /* activities placed (serial SGS steps, Alg. 7) */
    int64_t steps_done;         /* Alg. 5 / Alg. 4 loop steps of those placements */
    int64_t update_units;       /* time-indexed: Alg. 6 update steps (sum of
                                   d_i); capacity-indexed: Eq. 7 reads (one per
                                   resource with r_{i,k} > 0)                  */
    int64_t succ_pushes;        /* successor updates (|succ(i)| per placement)  */
    int64_t kept_words;         /* 32-bit words of kept decoder states written
                                   and read (device memory, L2-resident)       */
} rcpsp_stats;

/* Optional device allocator.  alloc returns device memory of `bytes` bytes
 * usable on `stream` (NULL on failure); release returns it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*release)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} rcpsp_allocator;

typedef struct rcpsp_ctx rcpsp_ctx;

/* Creates a context on CUDA device `device`.  `alloc` may be NULL (then
 * cudaMalloc / cudaFree are used); the struct is copied.  Errors:
 * RCPSP_E_INVALID_ARG, RCPSP_E_CUDA. */
int rcpsp_create(rcpsp_ctx **ctx, int device, const rcpsp_allocator *alloc);

/* Waits for the context's work, frees its device memory and the context.
 * RCPSP_E_INVALID_ARG for a NULL context. */
int rcpsp_destroy(rcpsp_ctx *ctx);

/* Validates `count` instances (host memory), computes for each the critical
 * path (Sec. 2), the level-ordered initial list (Sec. 4.1) and the evaluator
 * of the selection rule (Sec. 5.4), packs them and copies them to the
 * device.  Writes one id per instance to out_ids (host).  On any validation
 * error nothing is loaded and the code of the first bad instance is
 * returned (RCPSP_E_CYCLE, RCPSP_E_DUMMY, RCPSP_E_DEMAND_EXCEEDS_CAP,
 * RCPSP_E_TOO_LARGE, RCPSP_E_INVALID_ARG).  The copy goes through pinned
 * staging on a stream of the context; the call returns when the data is on
 * the device, without waiting for searches still running, so loading the
 * next batch overlaps the current search. */
int rcpsp_load_instances(rcpsp_ctx *ctx, const rcpsp_instance *inst, int32_t count,
                         int32_t *out_ids);

/* Frees the device memory of loaded instances (their ids become unknown),
 * after the context's running search.  ids: host, [count].  An unknown id
 * gives RCPSP_E_NOT_FOUND; the ids before it in the list are freed. */
int rcpsp_free_instances(rcpsp_ctx *ctx, const int32_t *ids, int32_t count);

/* Runs one tabu search per listed instance (Sec. 6: neighbourhood of swap
 * moves with Eqs. 5-6 filtering, serial-SGS decoding with the chosen
 * evaluator, best admissible move under the simple tabu list (Algs. 2-3)
 * and the aspiration rule).  The searches are grouped into launch classes
 * by footprint (per-group scratch up to 512, 2K, 8K, above 8K words) and
 * size (N up to 64, up to 160, larger); each class is one persistent launch
 * with its own shape -- lanes per decode, warps per CTA, CTAs per search --
 * the first on `cuda_stream` (a cudaStream_t; NULL = legacy default stream),
 * the others on streams of the context forked from it and joined back into
 * it, classes of more estimated work first.  With cluster_size = 0, a class
 * of one CTA per search whose neighbourhoods mostly fit one decode round
 * gives its few outliers (at most 1/16 of the class, initial list with more
 * feasible swaps than the CTA has decoding groups) a launch of their own
 * with clusters of 2-8 CTAs, started first.  A class whose iterations take
 * several decode rounds per CTA keeps the decoder state of the current list
 * every K positions and starts each neighbour's decode from the last state
 * before its first swapped position (prefix reuse; results and counts are
 * those of full decodes).  A class with at least 1.5 times as many searches
 * as its launch holds at once is sliced (rcpsp_params.slices): its searches
 * take turns in slices of iterations, so that the ones that would start last
 * do not run alone at the end; a CTA that pops a slice whose previous slice
 * another CTA still runs waits for it, and gives the search up with
 * status RCPSP_E_DEVICE only if that search makes no progress for 10 s.
 * Device memory of the call (plan, kept states, slice states) comes from
 * the context's allocator.  The call is asynchronous.  Results stay on the device until rcpsp_get_schedules.
 * ids: host, [count], loaded instances.  Errors, before anything is
 * launched: RCPSP_E_INVALID_ARG (a parameter out of range, resume without a
 * state kept with the same swap distance, tabu length and evaluator),
 * RCPSP_E_NOT_FOUND (id), RCPSP_E_TOO_LARGE (a search state that does not
 * fit in shared memory at the shape asked for), RCPSP_E_CUDA. */
int rcpsp_tabu_search(rcpsp_ctx *ctx, const int32_t *ids, int32_t count,
                      const rcpsp_params *params, void *cuda_stream);

/* Co-operating searches (Sec. 6.1, Eq. 8).  Each instance is searched by
 * `blocks` tabu searches -- one CTA each, the CTAs of one thread-block
 * cluster -- that exchange solutions through a working set F of
 * `working_set` slots in device memory.  Slot k starts from the level order
 * of Sec. 4.1 with slot k's shuffle keys, improved by the forward-backward
 * improvement (FBI) when fbi_every says so: the list's schedule decoded
 * backward on the reversed network in order of decreasing finish time
 * (ties: later list position first), then forward in order of increasing
 * mirrored start (ties: earlier position first), repeated while the
 * makespan gets strictly shorter.  Every block reads a slot, then
 * runs the search of rcpsp_tabu_search on it; when its best list since the
 * read is better than the slot it read, or after more than I_assigned
 * iterations without that (Eq. 8, quantity factor read as I_block / 5), it
 * writes its best list and tabu state back to that slot (only if better
 * than what the slot now holds) and reads the next slot round robin.  A
 * slot read more than phi_max times since its last improvement is
 * diversified on reading by phi_steps random feasible swaps.  The blocks
 * advance in lockstep and exchange in block order (writes, then reads) after
 * every iteration, so the result is deterministic and independent of the
 * launch; the paper's blocks exchange asynchronously under locks.
 * params->iterations = I_block, the iterations of each block; the result
 * (rcpsp_get_schedules) is the best list found, with iterations and
 * evaluated schedules summed over the blocks.  */
typedef struct {
    int32_t blocks;            /* B, 1..16: searches per instance (CTAs per cluster) */
    int32_t working_set;       /* |F|, 1..64 (the paper: 16)                         */
    int32_t phi_max;           /* Phi_max (the paper: 3)                             */
    int32_t phi_steps;         /* Phi_steps (the paper: 20); 0 = no diversification  */
    int32_t assign_fixed;      /* iterations per read; 0 = Eq. 8                     */
    int32_t words_per_block;   /* P: random words per block in random_words          */
    int32_t fbi_every;         /* e: slots e-1, 2e-1, ... start improved by the
                                  forward-backward improvement (Sec. 6: every
                                  second solution, e = 2); 0 = none              */
} rcpsp_coop_params;

/* Runs co-operating searches of the loaded instances `ids` (asynchronous on
 * cuda_stream, like rcpsp_tabu_search; no trace, no graph capture:
 * record_trace / use_graph / checkpoint / resume = 1 give
 * RCPSP_E_INVALID_ARG).  slot_keys (host,
 * copied, may be NULL = every slot unshuffled): for each id in order,
 * working_set rows of N shuffle keys (Sec. 4.1; all zeros = unshuffled).
 * random_words (host, copied; NULL allowed when phi_steps == 0): for each id
 * in order, blocks rows of words_per_block uint32, the words block b draws
 * its swaps from, used cyclically: each swap takes the next word w and
 * applies the floor(w * n_f / 2^32)-th of the n_f feasible swaps
 * (1 <= u < v <= N-2, v - u <= delta, Eqs. 5-6), in u-major order.  Errors:
 * RCPSP_E_INVALID_ARG (parameters), RCPSP_E_NOT_FOUND (id),
 * RCPSP_E_TOO_LARGE (state or cluster does not fit), RCPSP_E_CUDA. */
int rcpsp_coop_search(rcpsp_ctx *ctx, const int32_t *ids, int32_t count, const rcpsp_params *params,
                      const rcpsp_coop_params *coop, const int32_t *slot_keys,
                      const uint32_t *random_words, void *cuda_stream);

/* The same search as rcpsp_tabu_search, for callers that cannot allocate
 * device memory when they search: for example a serving process whose
 * device memory is owned by another allocator with a fixed budget, or a
 * host thread that must not block on the implicit device synchronisation
 * of cudaMalloc / cudaFree.  This call allocates nothing: the launch plan
 * and the work-queue counter live in a fixed 1 MiB array in the library's
 * device image, which every GPU that loads the library keeps until the
 * process exits.  Instances must already be loaded (rcpsp_load_instances
 * is where device memory is taken); results are read as usual with
 * rcpsp_get_schedules.  Limits: at most as many instances per call as the
 * array holds (8190; more gives RCPSP_E_TOO_LARGE), no trace, no graph
 * capture and no checkpoints (record_trace, use_graph, checkpoint or resume
 * = 1 gives RCPSP_E_INVALID_ARG).  The call makes one launch with one
 * launch shape for all its instances: no launch classes, no prefix reuse,
 * no slices (`slices` is ignored) and one CTA per search (cluster_size
 * other than 0 or 1 gives RCPSP_E_INVALID_ARG), because the per-class
 * queues, the kept prefix and slice states and the cluster plan would need
 * context memory.  Results are the
 * same as rcpsp_tabu_search's; throughput on batches of uneven sizes can be
 * lower.  The
 * first call on a device also looks up the array's device address with
 * that device current; make that first call before any stream capture.
 * Every call shares the one array and resets its counter: calls whose
 * searches overlap on the GPU (several contexts, or several streams, on
 * one device) race.  The paper has no counterpart of this call. */
int rcpsp_tabu_search_noalloc(rcpsp_ctx *ctx, const int32_t *ids, int32_t count,
                              const rcpsp_params *params, void *cuda_stream);

/* Chooses the launch shape -- lanes per neighbour decode (group_size),
 * warps per CTA and CTAs per search (cluster_size) -- for searches like `params` over these instances by
 * timing short trial searches (trial_iterations each, on `cuda_stream`) of
 * every shape that fits, and keeps the fastest (neighbours decoded per
 * second) in the context under the workload's signature (largest N, horizon,
 * words per step, swap distance, evaluator mix, batch size).  Instances are
 * tuned per launch class (see rcpsp_tabu_search), the unit a search launches
 * apart; classes with at most half as many searches as the GPU has SMs also
 * try clusters of 2, 4 and 8 CTAs per search; the three fastest shapes of
 * a class are timed again with four times the trial iterations (up to the
 * search's own) before one is kept.  When the call has more
 * than one class, each class's three fastest shapes and the other cluster
 * sizes of its pick are then timed with the whole call running (the classes
 * share the GPU), keeping a change only if the call gets at least 3% faster.  The returned shape (any
 * output pointer may be NULL) is the one of the largest class.  Later searches with group_size =
 * warps_per_cta = cluster_size = 0 and the same signature use it.  When the
 * environment variable RCPSP_TUNE_CACHE names a file, the table is written
 * there per device name and read back by contexts created later.  The
 * trials overwrite the instances' results.  Synchronous.  The shape is the
 * GPU's own split of the neighbourhood (Sec. 6 parallelises it over the
 * threads of a block); the paper fixes it by hand (Sec. 7). */
int rcpsp_autotune(rcpsp_ctx *ctx, const int32_t *ids, int32_t count, const rcpsp_params *params,
                   int32_t trial_iterations, void *cuda_stream, int32_t *best_group_size,
                   int32_t *best_warps, int32_t *best_cluster_size);

/* Waits for the last search of the context and copies results to host
 * buffers: order = best list W* and start = its start times S (both [sum of N
 * over the ids], concatenated in id order), makespan = C*_max [count].  Any
 * output pointer may be NULL.  stats (NULL allowed) gets [count] entries.
 * Returns RCPSP_E_DEVICE if a search reported an internal error. */
int rcpsp_get_schedules(rcpsp_ctx *ctx, const int32_t *ids, int32_t count,
                        int32_t *order, int32_t *start, int32_t *makespan,
                        rcpsp_stats *stats);

/* Copies the iteration trace of the last search of an instance run with
 * record_trace = 1: [iterations][3] = (u, v, C_max after the move), (0, 0)
 * for an iteration without an admissible move.  `capacity` is the number of
 * int32 elements of `trace` (host); *written gets the number of iterations
 * of that call (for a resumed search: the iterations it added).  Errors:
 * RCPSP_E_NOT_FOUND (id), RCPSP_E_INVALID_ARG (no trace recorded, or
 * `capacity` below 3 x those iterations). */
int rcpsp_get_trace(rcpsp_ctx *ctx, int32_t id, int32_t *trace, int32_t capacity,
                    int32_t *written);

/* Decodes `count` activity lists of one loaded instance on the device with
 * the serial SGS of Alg. 7 and the given evaluator (TIME or CAPACITY; AUTO =
 * the instance's selected one).  lists [count*N] (host): each a permutation
 * of 0..N-1 with 0 first, N-1 last and every arc pointing forward, else
 * RCPSP_E_INVALID_ARG.  Writes start [count*N], makespan [count] and work
 * [count] (Alg. 5 or Alg. 4 loop steps; any may be NULL).  Synchronous. */
int rcpsp_evaluate_lists(rcpsp_ctx *ctx, int32_t id, const int32_t *lists, int32_t count,
                         int32_t eval_mode, int32_t *start, int32_t *makespan,
                         int64_t *work, void *cuda_stream);

/* Validates one instance (host memory) and reports what
 * rcpsp_load_instances would prepare for it, without using a GPU: the
 * critical-path length (Sec. 2), the horizon UB = sum d_i (Sec. 5.2), the
 * initial list W (Sec. 4.1, [N]) and the evaluator of the selection rule
 * (Sec. 5.4).  Any output may be NULL; `msg` (msg_len bytes, may be NULL)
 * gets the reason of a failure.  Returns the same codes as loading. */
int rcpsp_prepare_instance(const rcpsp_instance *inst, int32_t *critical_path, int32_t *horizon,
                           int32_t *initial_order, int32_t *eval_mode, char *msg, int32_t msg_len);

/* Saved search state of a loaded instance (see rcpsp_params.checkpoint),
 * for keeping a search outside the context or moving it to another one.
 * rcpsp_get_state waits for the context's search, then copies the state to
 * `buf` (host, `capacity` bytes); *bytes gets its size (call with buf = NULL
 * to ask for it).  rcpsp_set_state gives the instance a state from `buf`
 * (as written by rcpsp_get_state for an instance with the same N); the next
 * search with resume = 1 continues it.  Errors: RCPSP_E_NOT_FOUND (id),
 * RCPSP_E_INVALID_ARG (no kept state, or a state that is not for this
 * instance), RCPSP_E_TOO_LARGE (capacity too small).  The paper has no
 * counterpart (its working set keeps lists and tabu lists, Sec. 6.1). */
int rcpsp_get_state(rcpsp_ctx *ctx, int32_t id, void *buf, size_t capacity, size_t *bytes);
int rcpsp_set_state(rcpsp_ctx *ctx, int32_t id, const void *buf, size_t bytes);

/* Bytes the context has copied host->device and device->host since it was
 * created (instance records, launch plans, results, traces); host. */
int rcpsp_transfer_bytes(const rcpsp_ctx *ctx, int64_t *h2d, int64_t *d2h);

/* Kernel launches the context has issued since it was created: one per
 * launch class of every search (a graph replay counts the kernels it
 * replays), one per no-allocation search and per list evaluation; host.
 * RCPSP_E_INVALID_ARG if `launches` is NULL.  An accounting call with no
 * counterpart in the paper. */
int rcpsp_kernel_launches(const rcpsp_ctx *ctx, int64_t *launches);

/* Multi-start (Sec. 4.1): `starts` independent searches of one instance,
 * start k from the level-ordered list with the shuffle keys of row k of
 * level_keys ([starts][N], host; NULL or a row of zeros = the unshuffled
 * order), keeping the one with the lowest best makespan (ties: the lowest
 * start index).  The instance is loaded `starts` times, searched in one
 * rcpsp_tabu_search call with `params` (record_trace, checkpoint and resume
 * must be 0) on cuda_stream, and freed again; the call is synchronous.
 * Outputs (host; any may be NULL): *best_start, the best start's list
 * order[N] and start times start[N], makespans[starts] of every start, and
 * stats of the best start.  Errors: those of rcpsp_load_instances and
 * rcpsp_tabu_search; RCPSP_E_INVALID_ARG for starts < 1. */
int rcpsp_multistart(rcpsp_ctx *ctx, const rcpsp_instance *inst, int32_t starts, const int32_t *level_keys,
                     const rcpsp_params *params, void *cuda_stream, int32_t *best_start, int32_t *order,
                     int32_t *start, int32_t *makespans, rcpsp_stats *stats);

/* Launch plan of the context's last rcpsp_tabu_search: one entry per
 * launch class of that call (see rcpsp_tabu_search), in launch order
 * (classes of more estimated work first). */
typedef struct {
    int32_t searches;           /* searches of the class                          */
    int32_t group_size;         /* lanes per neighbour decode                      */
    int32_t warps;              /* warps per CTA                                   */
    int32_t cluster_size;       /* CTAs per search                                 */
    int32_t ctas;               /* CTAs launched (persistent)                      */
    int32_t prefix_reuse;       /* 1: neighbours start from kept decoder states    */
    int32_t shape_source;       /* 0: built-in defaults, 1: the context's table of
                                   measured shapes (rcpsp_autotune), 2: the caller */
    int32_t slices;             /* slices per search (rcpsp_params.slices); 1: none */
    int64_t smem_bytes;         /* dynamic shared memory per CTA                   */
} rcpsp_launch_info;

/* Copies up to `capacity` entries of that plan to `out` (host; NULL with
 * capacity 0 to ask only for the count); *count gets the number of
 * classes.  An accounting call with no counterpart in the paper. */
int rcpsp_last_launches(const rcpsp_ctx *ctx, rcpsp_launch_info *out, int32_t capacity, int32_t *count);

/* Measured ceilings of the integer search path on one GPU, for its
 * roofline: the 32-bit integer ALU rate (independent chains of a logical
 * and an add per link, registers only; ops counted per thread) and the
 * shared-memory load bandwidth (16-byte loads, consecutive lanes at
 * consecutive words, no bank conflicts).  Each rate is the best of five
 * launches of one full wave (the blocks every SM holds at once), timed with
 * CUDA events, at the clocks of the run. */
typedef struct {
    double int32_ops_per_s;        /* whole GPU                                  */
    double smem_bytes_per_s;       /* whole GPU                                  */
    double int32_ms;               /* event time of the best integer launch      */
    double smem_ms;                /* event time of the best shared-memory launch */
    int32_t sms;                   /* SMs of the device                          */
} rcpsp_peaks;

/* Runs the two measurements on CUDA device `device` (a few tens of ms,
 * synchronous; it allocates and frees a few bytes of device memory and
 * restores the calling thread's current device).  Errors:
 * RCPSP_E_INVALID_ARG (NULL `out`, bad device), RCPSP_E_CUDA.  A measuring
 * call with no counterpart in the paper. */
int rcpsp_measure_peaks(int device, rcpsp_peaks *out);

/* ------------------------------------------------------------------------
 * Continuous-batching solve server.  Requests are admitted while others run,
 * as launch slots and device memory free up, and their searches overlap on
 * the GPU.  A search's result does not depend on what else is in flight.
 * ---------------------------------------------------------------------- */
typedef struct rcpsp_server rcpsp_server;

typedef struct {
    int32_t slots;              /* batches in flight (one stream each), 1..16; 0 = 8 */
    int32_t max_batch;          /* most requests per batch; 0 = 256.  A batch holds
                                   one launch class (footprint x size, see
                                   rcpsp_tabu_search) and at most 256 / 96 / 32
                                   requests of N up to 64 / 160 / more           */
    int64_t memory_budget;      /* device bytes of admitted requests; 0 = 1 GiB.
                                   A request larger than the budget is admitted
                                   alone when nothing else is in flight          */
    int32_t poll_us;            /* idle wait of the worker loop; 0 = 100 us        */
    int32_t slice_iterations;   /* > 0: time-slice requests of more iterations:
                                   each batch runs at most this many iterations
                                   of a request, whose state is then kept
                                   (rcpsp_params.checkpoint) and which goes back
                                   to the end of its queue until done, so long
                                   searches take turns with newer requests;
                                   results are those of an uninterrupted search.
                                   0 = no slicing                                 */
    int32_t max_pending;        /* > 0: most requests waiting for admission; a
                                   submission beyond it is refused with
                                   RCPSP_E_TOO_LARGE and counted as rejected (load
                                   shedding under overload).  0 = no limit        */
} rcpsp_server_config;

typedef struct {
    int64_t tag;                /* the caller's tag of the request                 */
    int32_t n;                  /* N of the instance                               */
    int32_t status;             /* 0 or a negative RCPSP_E_* code                  */
    int32_t best_cmax, iterations, eval_mode, critical_path;
    int64_t evaluated, work;    /* as in rcpsp_stats                               */
    int64_t t_submit_ns, t_launch_ns, t_done_ns;   /* host steady clock           */
    const int32_t *order;       /* [n] best list W*; owned by the server until the
                                   next rcpsp_server_poll                          */
    const int32_t *start;       /* [n] its start times S                           */
} rcpsp_completion;

typedef struct {
    int64_t submitted, rejected, admitted, completed, batches;
    int64_t inflight_requests, pending, inflight_bytes, max_inflight_bytes;
    int64_t evaluated;          /* neighbours decoded by completed requests        */
    int64_t requeued;           /* slices that ended with the request requeued     */
} rcpsp_server_stats;

/* Starts a server on `device` (cfg may be NULL for the defaults).  It owns
 * `slots` library contexts whose device memory comes from stream-ordered
 * allocations on their own streams, and one worker thread.  Before it
 * returns it maps the memory budget in the server's pool, sizes every
 * slot's pinned staging and launch plan for a full batch and loads the
 * search kernels, so that the first requests do not pay for that. */
int rcpsp_server_create(rcpsp_server **srv, int device, const rcpsp_server_config *cfg);
/* Stops the worker after the batches in flight and frees everything. */
int rcpsp_server_destroy(rcpsp_server *srv);
/* Validates one instance (as rcpsp_load_instances does; the same error
 * codes), copies it and queues it with its search parameters (record_trace,
 * use_graph, checkpoint and resume must be 0).  Requests of one launch class with identical
 * parameters share batches, in arrival order; the class whose oldest
 * request is oldest is served first.  Returns at once. */
int rcpsp_server_submit(rcpsp_server *srv, const rcpsp_instance *inst, const rcpsp_params *params,
                        int64_t tag);
/* Moves up to `capacity` finished requests into `out` (host), waiting up to
 * wait_ms for the first one; *count gets how many.  The arrays they point to
 * stay valid until the next call. */
int rcpsp_server_poll(rcpsp_server *srv, rcpsp_completion *out, int32_t capacity, int32_t *count,
                      int32_t wait_ms);
/* Counters of the server (host). */
int rcpsp_server_get_stats(rcpsp_server *srv, rcpsp_server_stats *stats);

/* Text of the last error of the context (never NULL). */
const char *rcpsp_last_error(const rcpsp_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RCPSP_H */
