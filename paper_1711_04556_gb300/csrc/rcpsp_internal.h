// Internal layout shared by the host runtime and the sm_103a kernels.
//
// One instance is packed once, at load time, into an int32 record in device
// memory whose first section has exactly the layout the search kernel uses
// in shared memory, so that staging an instance into a CTA is one contiguous
// copy.  The record is followed by the initial activity list W (Sec. 4.1).
#pragma once

#include <stdint.h>

#include "../../include/rcpsp.h"

#if defined(__CUDACC__)
#define RC_HD __host__ __device__ __forceinline__
#else
#define RC_HD inline
#endif

namespace rcpsp {

constexpr int kDefaultMoveCap = 1024;   // feasible moves one batch of decodes holds
constexpr int kSearchMaxWarps = 16;     // largest search CTA (512 threads)
constexpr int kSearchNarrowThreads = 384;   // CTAs up to this size run the 384-thread build of the kernel

// Per-instance header (64 bytes).
struct InstHeader {
    int32_t n, m, ub, cp;       // N, M, UB = sum d_i (Sec. 5.2), critical path
    int32_t sel_mode;           // evaluator of the selection rule (Sec. 5.4)
    int32_t wps;                // 32-bit words per time step of the packed profile
    int32_t lane_bits;          // 8 or 16 bits per resource inside a word
    int32_t sum_cap;            // sum R_k: length of the capacity-indexed state
    int32_t n_arcs;             // |E|
    int32_t inst_words;         // words of the shared-memory section
    int32_t record_words;       // inst_words + initial list, multiple of 4
    int32_t sum_used;           // number of (activity, resource) pairs with r_{i,k} > 0
    int32_t es_fits;            // 1: the earliest-start schedule respects every capacity
    int32_t pad[3];
};
static_assert(sizeof(InstHeader) == 64, "InstHeader is 64 bytes");

// One entry of a launch (128 bytes), ordered by estimated cost on the host.
struct LaunchItem {
    InstHeader h;
    const int32_t *record;      // packed record in device memory
    int32_t *out;               // outputs: W*[N], S*[N], then kOutStats words
    int32_t *trace;             // [iterations*3] or nullptr
    int32_t *state;             // saved search state (CkptLayout) or nullptr
    int32_t mode;               // evaluator for this search
    int32_t iterations;         // iterations of this call
    int32_t delta;              // max swap distance
    int32_t tabu_len;           // tabu list length
    int32_t stop_at_cp;
    int32_t ckpt;               // kCkpt* bits: resume from / save to `state`
    int32_t prefix_k;           // > 0: positions between kept prefix states (prefix_*)
    int32_t slice_off;          // sliced launch: first word of this search's slice state (SliceSched)
};
static_assert(sizeof(LaunchItem) == 128, "LaunchItem is 128 bytes");

enum : int { kCkptResume = 1, kCkptSave = 2 };

// One entry of a co-operative launch (160 bytes): the search of `base` run
// by a cluster of CTAs that exchange solutions through a working set F
// (Sec. 6.1) in device memory.
struct CoopItem {
    LaunchItem base;                 // instance, outputs, search parameters (no trace)
    int32_t *slots;                  // F: working_set slots of slot_words words (SlotLayout)
    const int32_t *init_lists;       // [working_set][N] initial list of every slot
    const uint32_t *words;           // [blocks][words_per_block] random words
    int32_t slot_words;
    int32_t pad;
};
static_assert(sizeof(CoopItem) == 160, "CoopItem is 160 bytes");

// Launch-wide parameters of the co-operation (identical for every item).
struct CoopConfig {
    int32_t blocks;                  // B = CTAs per cluster
    int32_t working_set;             // |F|
    int32_t phi_max, phi_steps;      // diversification
    int32_t assign_fixed;            // iterations per read; 0 = Eq. 8
    int32_t words_per_block;         // P
    int32_t fbi_every;               // FBI on slots k with k % e == e-1; 0 = none
};

constexpr int kMaxCoopBlocks = 16;   // largest cluster (non-portable above 8)
constexpr int kMaxWorkingSet = 64;

// Statistics words after W* and S* in the output block of an instance.
enum : int {
    kOutEvalLo = 0, kOutEvalHi, kOutWorkLo, kOutWorkHi,
    kOutIters, kOutCmax, kOutMode, kOutStatus,
    kOutT0Lo, kOutT0Hi, kOutT1Lo, kOutT1Hi,
    kOutIters0,                 // iterations before the call (a resumed search)
    // work the decodes of this call performed (positions restored from a
    // kept state excluded; see TallyRef)
    kOutPlacedLo, kOutPlacedHi, kOutStepsLo, kOutStepsHi, kOutUpdLo, kOutUpdHi,
    kOutSuccLo, kOutSuccHi, kOutKeptLo, kOutKeptHi,
    kOutStats
};

// Work counters of the decodes, in the order of the kOutPlaced.. words:
// activities placed, Alg. 5 (time-indexed) or Alg. 4 (capacity-indexed)
// loop steps of those placements, their Alg. 6 update steps (sum of d_i,
// time-indexed) or Eq. 7 reads (used resources, capacity-indexed),
// successor pushes (|succ(i)| per placement), and 32-bit words of kept
// decoder states written and read (prefix reuse).
enum : int { kTallyPlaced = 0, kTallySteps, kTallyUpd, kTallySucc, kTallyKept, kTallies };

RC_HD int align4(int x) { return (x + 3) & ~3; }

static_assert(RCPSP_MAX_M <= 8, "a resource index of the packed demands takes 3 bits");

// Offsets (in 32-bit words) of the shared-memory image of an instance.
struct InstLayout {
    int dur, reqw, capw, cap, cbase, reqk, poff, plist, soff, slist, words;
};

RC_HD InstLayout inst_layout(int n, int m, int wps, int n_arcs) {
    InstLayout L;
    int o = 0;
    L.dur = o;   o += align4(n);          // d_i
    L.reqw = o;  o += align4(n * wps);    // packed r_{i,k}: word w of activity i at i*wps+w
    L.capw = o;  o += 4;                  // packed R_k per word (initial profile value)
    L.cap = o;   o += 8;                  // R_k
    L.cbase = o; o += 8;                  // start of c_k in the capacity-indexed state
    L.reqk = o;  o += align4(n * m);      // used resources of i first: r_{i,k} << 3 | k, then 0
    L.poff = o;  o += align4(n + 1);      // predecessor CSR
    L.plist = o; o += align4(n_arcs);
    L.soff = o;  o += align4(n + 1);      // successor CSR
    L.slist = o; o += align4(n_arcs);
    L.words = o;
    return L;
}

// Search state and per-group scratch that follow the instance image.
struct StateLayout {
    int W, pos, Wbest, fsp, lpp, stl, tc, moves;
    int groups;          // first word of the per-warp group areas
    int prof_words;      // profile words of one group (time- or capacity-indexed)
    int group_words;     // words of one group's scratch (group_area_words)
    int total;           // words of dynamic shared memory
};

// Words of one decoding group's shared scratch.  Time-indexed: the packed
// profile (prof_words 32-bit words), then the N earliest starts in 16 bits;
// capacity-indexed: the capacity state (prof_words = sum R_k entries) and
// the N earliest starts, all in 16 bits.  Every time value is at most
// RCPSP_MAX_HORIZON (32767), so 16 bits hold it.
RC_HD int group_area_words(int mode, int prof_words, int n) {
    return mode == RCPSP_EVAL_CAPACITY ? (prof_words + n + 1) / 2 : prof_words + (n + 1) / 2;
}

RC_HD int profile_words(int mode, int wps, int ub, int sum_cap) {
    return mode == RCPSP_EVAL_CAPACITY ? sum_cap : wps * (ub > 0 ? ub : 1);
}

// Prefix reuse: a swap (u, v) leaves list positions below u as they are, so
// a neighbour's decode may start from the decoder state of the current list
// before position floor(u/K)*K.  These states -- a meta block, the profile
// (or capacity state) and the earliest starts -- are kept before positions
// K, 2K, ..., count*K < N, in a global scratch region of each CTA.  Meta
// words: frontier F, makespan so far, work so far, the Alg. 6 update steps
// (or Eq. 7 reads) and successor pushes of the positions before, and the
// words of this state.
enum : int { kPxF = 0, kPxCmax, kPxWork, kPxUpd, kPxSucc, kPxWords, kPxMeta = 8 };
RC_HD int prefix_count(int n, int K) { return K > 0 ? (n - 1) / K : 0; }
RC_HD int prefix_stride(int n, int prof_words) { return align4(kPxMeta + prof_words + n); }
RC_HD int prefix_words(int n, int prof_words, int K) { return prefix_count(n, K) * prefix_stride(n, prof_words); }

// Launch class of a search: its footprint -- per-group scratch words `gw`
// (group_area_words: profile or capacity state plus N earliest starts) up
// to 512, 2K, 8K, or more -- times its size (N up to 64, up to 160, larger).  Searches of one
// class share a launch and its shape; the finest footprint level keeps the
// capacity-indexed searches (a few hundred words per group) apart from the
// time-indexed ones of the same size, whose profiles would otherwise size
// every CTA of the launch.
constexpr int kLaunchClasses = 12;
RC_HD int launch_class(int gw, int n) {
    const int fp = gw <= 512 ? 0 : (gw <= 2048 ? 1 : (gw <= 8192 ? 2 : 3));
    const int sz = n <= 64 ? 0 : (n <= 160 ? 1 : 2);
    return fp * 3 + sz;
}

RC_HD StateLayout state_layout(int inst_words, int n, int tabu_len, int delta, int move_cap,
                               int prof_words, int ngroups, int mode) {
    StateLayout S;
    int o = inst_words;
    S.W = o;     o += align4(n);
    S.pos = o;   o += align4(n);
    S.Wbest = o; o += align4(n);
    S.fsp = o;   o += align4(n);
    S.lpp = o;   o += align4(n);
    S.stl = o;   o += align4(tabu_len);
    S.tc = o;    o += align4((n * delta + 31) / 32);
    S.moves = o; o += align4(move_cap);
    S.groups = o;
    S.prof_words = prof_words;
    S.group_words = group_area_words(mode, prof_words, n);
    o += ngroups * S.group_words;
    S.total = o;
    return S;
}

// Saved state of one search (checkpoint): a meta block, then the current
// list W, the best list W*, the tabu list and the tabu cache, in the
// kernel's shared-memory representation.  Meta words: magic, N, delta,
// |TL|, evaluator, iterations done, C, C*, tabu write index, evaluated
// (lo, hi), work (lo, hi).
enum : int {
    kCkMagic = 0, kCkN, kCkDelta, kCkTabu, kCkMode, kCkIters, kCkC, kCkCbest, kCkWidx,
    kCkEvalLo, kCkEvalHi, kCkWorkLo, kCkWorkHi, kCkMeta = 16
};
constexpr int32_t kCkptMagic = 0x52435053;

struct CkptLayout {
    int W, Wbest, stl, tc, words;
};

RC_HD CkptLayout ckpt_layout(int n, int tabu_len, int delta) {
    CkptLayout L;
    L.W = kCkMeta;
    L.Wbest = L.W + align4(n);
    L.stl = L.Wbest + align4(n);
    L.tc = L.stl + align4(tabu_len);
    L.words = L.tc + align4((n * delta + 31) / 32);
    return L;
}

// Slicing a launch (SliceSched): with more searches than resident CTAs (or
// clusters), the searches that start last would run alone at the end of the
// call while the rest of the GPU idles.  A sliced launch cuts every search
// into `nslices` runs of L = ceil(iterations / nslices) iterations: queue
// position q names slice q / count of search q % count, so every search's
// first slice is popped before any second one, and a CTA may pick up a
// slice that another CTA's previous slice left in global memory.  Between
// slices a search's state is kept in its slice state: the CkptLayout of its
// (N, |TL|, delta) followed by kSlExtra words -- the iteration count before
// the call, the start timestamp, the error word and the five work counters
// of the call so far.  sync[2i] counts the slices of search i that are done
// (nslices once it has finished; kSliceAbandoned set when a CTA gave up
// waiting for it), sync[2i + 1] its iterations so far, which a waiting CTA
// watches for progress.  nslices <= 1: no slicing.
enum : int { kSlIt0 = 0, kSlT0Lo, kSlT0Hi, kSlErr, kSlTally, kSlExtra = 16 };
static_assert(kSlTally + 2 * kTallies <= kSlExtra, "slice extras fit");
constexpr int kSliceAbandoned = 1 << 29;
constexpr int kMaxSlices = 64;

struct SliceSched {
    int nslices;
    int *sync;             // [count][2]: slices done, iterations so far (zeroed before the launch)
    int32_t *states;       // slice states, at LaunchItem::slice_off
};

RC_HD int slice_state_words(int n, int tabu_len, int delta) {
    return align4(ckpt_layout(n, tabu_len, delta).words + kSlExtra);
}

// Words of one working-set slot: the list W, the tabu list (packed pairs),
// the tabu cache (banded bits, as in shared memory), then the write index
// and the makespan of the slot's initial list (the kernel keeps the current
// makespans in shared memory).
struct SlotLayout {
    int W, stl, tc, widx, words;
};

RC_HD SlotLayout slot_layout(int n, int tabu_len, int delta) {
    SlotLayout L;
    L.W = 0;
    L.stl = align4(n);
    L.tc = L.stl + align4(tabu_len);
    L.widx = L.tc + align4((n * delta + 31) / 32);
    L.words = L.widx + 4;
    return L;
}

}  // namespace rcpsp
