// Device building blocks of the tabu-search kernels: the warp-lockstep
// decoding groups, the shared-memory view of an instance, the serial SGS
// with both resource evaluations, the tabu cache, and the evaluation of a
// whole neighbourhood.  Included by each kernel translation unit; everything
// here has internal linkage.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "rcpsp_internal.h"

namespace rcpsp {
namespace {

namespace cg = cooperative_groups;

constexpr unsigned kFull = 0xffffffffu;
constexpr int kErrHorizon = 1;     // a profile window ran past UB
constexpr int kErrWait = 4;        // a wait for a kept decoder state gave up
constexpr unsigned long long kWaitNs = 2000000000ull;   // limit of that wait

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// G lanes of a warp that decode one neighbour.  All groups of a warp run in
// lockstep: a loop whose trip count may differ between groups is driven by a
// warp-wide vote and every warp-synchronous primitive names all 32 lanes, so
// one instruction serves the 32/G neighbours of the warp at once.
template <int G>
struct Group {
    int lane;        // lane inside the group
    int gbase;       // first warp lane of the group
    __device__ Group() {
        const int wl = threadIdx.x & 31;
        lane = wl & (G - 1);
        gbase = wl & ~(G - 1);
    }
    // the group's G bits of a warp-wide ballot
    __device__ unsigned bits(unsigned warp_ballot) const {
        return G == 32 ? warp_ballot : (warp_ballot >> gbase) & ((1u << G) - 1u);
    }
    // maximum over the group; every lane of the warp calls it
    __device__ int max(int x) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) x = ::max(x, __shfl_xor_sync(kFull, x, o));
        return x;
    }
    // sum over the group; every lane of the warp calls it
    __device__ int sum(int x) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        return x;
    }
};

// Shared-memory view of one instance.
struct SInst {
    const int *dur;
    const uint32_t *reqw;
    const uint32_t *capw;
    const int *cap;
    const int *cbase;
    const int *reqk;
    const int *poff;
    const int *plist;
    const int *soff;
    const int *slist;
    int n, m, ub, wps, sum_cap;
    int n_arcs, sum_used;
    uint32_t hi;     // high bit of every packed field
};

__device__ SInst bind_instance(const int *sm, const InstHeader &h) {
    InstLayout L = inst_layout(h.n, h.m, h.wps, h.n_arcs);
    SInst I;
    I.dur = sm + L.dur;
    I.reqw = reinterpret_cast<const uint32_t *>(sm + L.reqw);
    I.capw = reinterpret_cast<const uint32_t *>(sm + L.capw);
    I.cap = sm + L.cap;
    I.cbase = sm + L.cbase;
    I.reqk = sm + L.reqk;
    I.poff = sm + L.poff;
    I.plist = sm + L.plist;
    I.soff = sm + L.soff;
    I.slist = sm + L.slist;
    I.n = h.n;
    I.m = h.m;
    I.ub = h.ub;
    I.wps = h.wps;
    I.sum_cap = h.sum_cap;
    I.n_arcs = h.n_arcs;
    I.sum_used = h.sum_used;
    I.hi = h.lane_bits == 8 ? 0x80808080u : 0x80008000u;
    return I;
}

// Copies the instance image (a multiple of 16 bytes) into shared memory.
__device__ void stage_instance(int *sm, const int32_t *record, int words) {
    const int4 *src = reinterpret_cast<const int4 *>(record);
    int4 *dst = reinterpret_cast<int4 *>(sm);
    for (int x = threadIdx.x; x < words / 4; x += blockDim.x) dst[x] = __ldg(src + x);
}

// ---------------------------------------------------------------------------
// Serial SGS (Alg. 7) of the list W with positions u and v swapped
// (u == v leaves W unchanged), decoded by one group in lockstep with the
// other groups of its warp.  A group with active == false follows the loops
// without writing its scratch.  `area` is the group's interleaved scratch:
// the time-indexed profile as 32-bit words (element e at area[e*NG]), or the
// capacity state as 16-bit entries, then es[i], the precedence earliest
// start of every activity, in 16 bits (see half_area).  Instead of
// reading the finish times of i's predecessors when i is placed (the
// precedence part of Alg. 7), every placed activity raises es[] of its successors, so the
// placement of i starts from one broadcast load; the value is the same
// maximum.  Returns C_max; `work` gets the Alg. 5 (time-indexed) or Alg. 4
// (capacity-indexed) loop steps; S_out (may be null) gets start times.
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ int activity_at(const int *W, int p, int u, int v) {
    return p == u ? W[v] : (p == v ? W[u] : W[p]);
}

// es of every successor of i := max(es, f); inactive groups write nothing.
// Earliest starts are 16-bit (every time value is at most RCPSP_MAX_HORIZON).
template <int G>
__device__ __forceinline__ void push_finish(const SInst &I, int i, int f, short *es, int NG, const Group<G> &g,
                                            bool active) {
    const int e0 = I.soff[i], ns = active ? I.soff[i + 1] - e0 : 0;
    for (int b = g.lane; b < ns; b += G) {
        short *x = es + I.slist[e0 + b] * NG;
        *x = static_cast<short>(::max(static_cast<int>(*x), f));
    }
}

template <int G>
__device__ __forceinline__ void clear_es(short *es, int n, int NG, bool active, const Group<G> &g) {
    if (active)
        for (int x = g.lane; x < n; x += G) es[x * NG] = 0;
    __syncwarp();
}

// A group's 16-bit scratch from `area` (its first word): element e of
// group gw of a warp is halfword e*NG + gw of the warp's area, so the groups
// of a warp stay interleaved element by element as in the 32-bit sections.
template <int G>
__device__ __forceinline__ short *half_area(int *area, int word_offset, int NG) {
    const int gw = (threadIdx.x & 31) / G;
    return reinterpret_cast<short *>(area - gw + word_offset * NG) + gw;
}

// Kept decoder states of the current list (prefix reuse, see prefix_count),
// in the CTA's own global scratch (L2-resident, read and written past L1):
// snapshot j (1..count) is the state before position j*K, at base +
// (j-1)*stride: the kPxMeta meta words, then the profile (time-indexed: WPS
// planes of UB words; capacity-indexed: the c_k) and the N earliest starts.
// base == nullptr: no prefix reuse.  `ready` (shared memory) counts the
// snapshots of the current list kept so far in this iteration: the producing
// group publishes each one as it is written (release), and a neighbour decode
// that restores snapshot j waits until ready >= j (acquire), so the
// neighbours start before the producer has finished.  ready == nullptr: the
// snapshots are complete before any neighbour decode starts.
struct Prefix {
    int *base;
    int K, count, stride;
    int *ready;
};

__device__ __forceinline__ int load_acquire_cta(const int *x) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];"
                 : "=r"(v)
                 : "r"(static_cast<unsigned>(__cvta_generic_to_shared(x)))
                 : "memory");
    return v;
}

__device__ __forceinline__ void store_release_cta(int *x, int v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;"
                 :
                 : "r"(static_cast<unsigned>(__cvta_generic_to_shared(x))), "r"(v)
                 : "memory");
}

// Waits until *ready >= need, for at most kWaitNs; on giving up sets
// kErrWait (the search then reports RCPSP_E_DEVICE).  The producer never
// waits on a consumer, so a correct kernel always gets there.
__device__ __forceinline__ void wait_kept(const int *ready, int need, int &err) {
    if (need <= 0 || load_acquire_cta(ready) >= need) return;
    const unsigned long long t0 = global_timer_ns();
    while (load_acquire_cta(ready) < need) {
        if (global_timer_ns() - t0 > kWaitNs) {
            err |= kErrWait;
            return;
        }
        __nanosleep(64);
    }
}

// Work counters of the decodes of a CTA (kTally* order; see rcpsp_stats):
// `t` accumulates placements, Alg. 6 update steps or Eq. 7 reads, successor
// pushes and kept-state words, and at kTallySteps the correction that turns
// the work counter (which counts every neighbour in full) into the loop
// steps performed: plus the producer's decodes, minus the steps restored
// from kept states.  `hist` counts the neighbour decodes of the current
// batch of moves by the kept state they restored (0: none).  t == nullptr:
// no counting.
struct TallyRef {
    long long *t;
    int *hist;
};

// Alg. 6 update steps (time-indexed: d_i) or Eq. 7 reads (capacity-indexed:
// resources with r_{i,k} > 0) and successor pushes of the activities at
// positions [p0, p1) of W, summed over the group; every lane of the warp
// calls it.
template <int G>
__device__ __forceinline__ void position_sums(const SInst &I, const int *W, int p0, int p1, bool cap,
                                              const Group<G> &g, int &upd, int &succ) {
    int a_u = 0, a_s = 0;
    for (int q = p0 + g.lane; q < p1; q += G) {
        const int a = W[q];
        if (cap) {
            for (int k = 0; k < I.m; ++k) a_u += I.reqk[a * I.m + k] > 0 ? 1 : 0;
        } else {
            a_u += I.dur[a];
        }
        a_s += I.soff[a + 1] - I.soff[a];
    }
    upd = g.sum(a_u);
    succ = g.sum(a_s);
}

// Keeps the meta words of snapshot j (lane 0 of the producing group): the
// running sums of the positions before j*K -- those of [(j-1)K, jK) added to
// snapshot j-1's -- and the words of the state.
template <int G>
__device__ __forceinline__ void keep_meta(const SInst &I, const int *W, const Prefix &px, int j, int *sn, bool cap,
                                          int F, int cmax, int work, int words, bool active, const Group<G> &g) {
    int upd, succ;
    position_sums<G>(I, W, (j - 1) * px.K, j * px.K, cap, g, upd, succ);
    if (active && g.lane == 0) {
        if (j >= 2) {
            upd += __ldcg(sn - px.stride + kPxUpd);
            succ += __ldcg(sn - px.stride + kPxSucc);
        }
        __stcg(sn + kPxF, F);
        __stcg(sn + kPxCmax, cmax);
        __stcg(sn + kPxWork, work);
        __stcg(sn + kPxUpd, upd);
        __stcg(sn + kPxSucc, succ);
        __stcg(sn + kPxWords, words);
    }
}

// First position a neighbour decode of swap(u, v) must place itself.
__device__ __forceinline__ int prefix_start(const Prefix &px, int u, bool produce) {
    if (!px.base || produce || u <= 0) return 0;
    return ::min(u / px.K, px.count) * px.K;
}

// Before a warp's neighbour decodes restore their kept states: wait until
// the snapshots they restore (the largest index over the warp's groups) are
// published.  Every lane of the warp calls it.
__device__ __forceinline__ void await_prefix(const Prefix &px, int p0, bool active, bool produce, int &err) {
    if (!px.ready || produce) return;
    const int need = __reduce_max_sync(kFull, active ? p0 / px.K : 0);
    wait_kept(px.ready, need, err);
}

// After the producing warp kept snapshot j: make its stores (every lane's)
// visible to the block, then publish j.  Every lane of the warp calls it.
__device__ __forceinline__ void publish_prefix(const Prefix &px, int j) {
    if (!px.ready) return;
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) store_release_cta(px.ready, j);
}

// Time-indexed decode, WPS = 32-bit words per time step of the packed profile.
template <int G, int WPS, bool PFX>
__device__ int decode_time(const SInst &I, const int *W, int u, int v, bool active, int *area, int NG,
                           const Group<G> &g, int &work, int &err, int *S_out, const Prefix &px,
                           bool produce) {
    constexpr int U = G >= 32 ? 1 : (G >= 16 ? 2 : 4);   // steps a lane tests per round
    constexpr int R = G * U;                               // steps a group tests per round (<= 32)
    const int n = I.n, ub = I.ub;
    const int ubs = ub > 0 ? ub : 1;              // stride of one resource-word plane
    uint32_t *prof = reinterpret_cast<uint32_t *>(area);
    short *esa = half_area<G>(area, WPS * ubs, NG);
    const uint32_t hi = I.hi;
    uint32_t capw[WPS];
#pragma unroll
    for (int w = 0; w < WPS; ++w) capw[w] = I.capw[w] | hi;   // profile words carry the guard bits
    // Every step starts with R_k free units (Sec. 5.2.1).  Steps at or after
    // the frontier F have not been touched by this decode, so they are not
    // stored: they are written the first time an activity covers them.
    int F = 0;
    int cmax = 0;
    const int p0 = PFX ? prefix_start(px, u, produce) : 0;
    if (PFX) await_prefix(px, p0, active, produce, err);
    if (PFX && p0 > 0) {
        // start from the kept state of the current list before position p0
        const int *sn = px.base + (p0 / px.K - 1) * px.stride;
        if (active) {
            F = __ldcg(sn + kPxF);
            cmax = __ldcg(sn + kPxCmax);
            work += __ldcg(sn + kPxWork);
#pragma unroll
            for (int w = 0; w < WPS; ++w)
                for (int t = g.lane; t < F; t += G)
                    prof[(w * ubs + t) * NG] = __ldcg(sn + kPxMeta + w * ubs + t);
            for (int x = g.lane; x < n; x += G)
                esa[x * NG] = static_cast<short>(__ldcg(sn + kPxMeta + WPS * ubs + x));
        }
        __syncwarp();
    } else {
        clear_es<G>(esa, n, NG, active, g);
    }
    const int pstart = PFX ? __reduce_min_sync(kFull, active ? p0 : n) : 0;
    int i = activity_at<G>(W, pstart < n ? pstart : 0, u, v);
    for (int p = pstart; p < n; ++p) {
        const bool act = PFX ? active && p >= p0 : active;
        if (PFX && produce && p > 0 && p % px.K == 0 && p / px.K <= px.count) {
            // keep the state before position p (warp-uniform condition)
            int *sn = px.base + (p / px.K - 1) * px.stride;
            if (active) {
#pragma unroll
                for (int w = 0; w < WPS; ++w)
                    for (int t = g.lane; t < F; t += G)
                        __stcg(sn + kPxMeta + w * ubs + t, static_cast<int>(prof[(w * ubs + t) * NG]));
                for (int x = g.lane; x < n; x += G) __stcg(sn + kPxMeta + WPS * ubs + x, static_cast<int>(esa[x * NG]));
            }
            keep_meta<G>(I, W, px, p / px.K, sn, false, F, cmax, work, kPxMeta + WPS * F + n, active, g);
            __syncwarp();
            publish_prefix(px, p / px.K);
        }
        const int inext = activity_at<G>(W, p + 1 < n ? p + 1 : p, u, v);
        const int es = esa[i * NG];
        const int d = I.dur[i];
        uint32_t rq[WPS];
#pragma unroll
        for (int w = 0; w < WPS; ++w) rq[w] = I.reqw[i * WPS + w];
        // Alg. 5: the first window [s, s+d), s >= es, whose steps all fit,
        // read off bit masks.  [s, s+k) is known to fit; a round tests the R
        // steps s+k .. s+k+R-1 (step s+k+lane+G*j in lane `lane`; steps at or
        // after F always fit) and either finds the first run of d fitting
        // steps, or keeps the trailing run of fitting steps as the new
        // verified prefix -- the same window as Alg. 5's loadTime count.
        int s = es, k = 0;
        bool done = !act || d == 0;
        while (__any_sync(kFull, !done)) {
            if (!done && s + k >= F) done = true;
            const int tlim = done ? INT_MIN : F;
            const int t0 = s + k + g.lane;
            const uint32_t *a0 = prof + t0 * NG;
            bool fit[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                fit[j] = true;
                if (t0 + G * j < tlim) {
#pragma unroll
                    for (int w = 0; w < WPS; ++w) {
                        const uint32_t x = a0[(w * ubs + G * j) * NG];
                        fit[j] = fit[j] && ((x - rq[w]) & hi) == hi;
                    }
                }
            }
            unsigned x = 0;                                       // bit o: step s+k+o fits
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if (G == 1) x |= static_cast<unsigned>(fit[j]) << j;
                else x |= g.bits(__ballot_sync(kFull, fit[j])) << (G * j);
            }
            if (!done) {
                const unsigned full = R == 32 ? 0xffffffffu : ((1u << R) - 1u);
                const int need = d - k;                           // >= 1
                const unsigned lowneed = need >= 32 ? 0xffffffffu : ((1u << need) - 1u);
                if (need <= R && (x & lowneed) == lowneed) {
                    done = true;                                  // [s, s+d) fits
                } else if (x == full) {
                    k += R;                                       // all fit, the window needs more
                } else {
                    const int b = __ffs(~x) - 1;                  // first failing step of the round
                    const int avail = R - b - 1;                  // steps after it in the round
                    const unsigned xs = b + 1 >= 32 ? 0u : (x >> (b + 1));
                    int w = -1;
                    if (d <= avail) {
                        unsigned y = xs;                          // y bit w: steps w..w+d-1 fit
                        int len = 1;
                        while (2 * len <= d) {
                            y &= y >> len;
                            len *= 2;
                        }
                        if (len < d) y &= y >> (d - len);
                        if (y) w = __ffs(y) - 1;
                    }
                    if (w >= 0) {
                        s += k + b + 1 + w;
                        done = true;
                    } else {
                        const int h = 31 - __clz(~x & full);      // last failing step of the round
                        s += k + h + 1;
                        k = R - h - 1;
                    }
                }
            }
        }
        const int f = s + d;
        if (act) {
            // Alg. 6: take r_{i,k} units over [s, s+d) (fields never borrow);
            // untouched steps in [F, s) get R_k, those in [F, s+d) R_k - r.
            if (d > 0) {
                const int fe = ::min(f, ub);
                if (f > ub) err |= kErrHorizon;
#pragma unroll 2
                for (int t = ::min(s, F) + g.lane; t < fe; t += G) {
                    uint32_t *x = prof + t * NG;
#pragma unroll
                    for (int w = 0; w < WPS; ++w) {
                        uint32_t *xw = x + w * ubs * NG;
                        *xw = (t >= F ? capw[w] : *xw) - (t >= s ? rq[w] : 0u);
                    }
                }
                F = ::max(F, fe);
            }
            if (S_out && g.lane == 0) S_out[i] = s;
            work += f - es;
            cmax = ::max(cmax, f);
        }
        push_finish<G>(I, i, f, esa, NG, g, act);
        __syncwarp();
        i = inext;
    }
    return cmax;
}

template <int G, bool PFX>
__device__ int decode_capacity(const SInst &I, const int *W, int u, int v, bool active, int *area, int NG,
                               const Group<G> &g, int &work, int &err, int *S_out, const Prefix &px,
                               bool produce) {
    const int n = I.n, m = I.m, sc = I.sum_cap;
    short *cst = half_area<G>(area, 0, NG);             // c_k, concatenated, 16-bit
    short *esa = cst + sc * NG;
    int cmax = 0;
    int wk = 0;                                        // this lane's Alg. 4 steps
    const int p0 = PFX ? prefix_start(px, u, produce) : 0;
    if (PFX) await_prefix(px, p0, active, produce, err);
    if (PFX && p0 > 0) {
        // start from the kept state of the current list before position p0
        const int *sn = px.base + (p0 / px.K - 1) * px.stride;
        if (active) {
            cmax = __ldcg(sn + kPxCmax);
            if (g.lane == 0) wk = __ldcg(sn + kPxWork);
            for (int j = g.lane; j < sc; j += G) cst[j * NG] = static_cast<short>(__ldcg(sn + kPxMeta + j));
            for (int x = g.lane; x < n; x += G) esa[x * NG] = static_cast<short>(__ldcg(sn + kPxMeta + sc + x));
        }
        __syncwarp();
    } else {
        if (active)
            for (int j = g.lane; j < sc; j += G) cst[j * NG] = 0;   // Sec. 5.1.1
        clear_es<G>(esa, n, NG, active, g);
    }
    const int pstart = PFX ? __reduce_min_sync(kFull, active ? p0 : n) : 0;
    int i = activity_at<G>(W, pstart < n ? pstart : 0, u, v);
    for (int p = pstart; p < n; ++p) {
        const bool act = PFX ? active && p >= p0 : active;
        if (PFX && produce && p > 0 && p % px.K == 0 && p / px.K <= px.count) {
            // keep the state before position p (warp-uniform condition)
            int *sn = px.base + (p / px.K - 1) * px.stride;
            const int wsum = g.sum(wk);
            if (active) {
                for (int j = g.lane; j < sc; j += G) __stcg(sn + kPxMeta + j, static_cast<int>(cst[j * NG]));
                for (int x = g.lane; x < n; x += G) __stcg(sn + kPxMeta + sc + x, static_cast<int>(esa[x * NG]));
            }
            keep_meta<G>(I, W, px, p / px.K, sn, true, 0, cmax, wsum, kPxMeta + sc + n, active, g);
            __syncwarp();
            publish_prefix(px, p / px.K);
        }
        const int inext = activity_at<G>(W, p + 1 < n ? p + 1 : p, u, v);
        const int es = esa[i * NG];
        // Eq. 7: es_res = max over used resources of c_k[R_k - r_{i,k}]
        // (the used resources of i come first in its row of reqk, each as
        // r << 3 | k; lane q takes the q-th, q+G-th, ... of them)
        int er = 0;
        if (act)
            for (int q = g.lane; q < m; q += G) {
                const int e = I.reqk[i * m + q];
                if (e == 0) break;
                const int k = e & 7, r = e >> 3;
                er = ::max(er, cst[(I.cbase[k] + I.cap[k] - r) * NG]);
            }
        er = g.max(er);
        const int s = ::max(es, er);
        const int d = I.dur[i];
        // Alg. 4, one lane per used resource (resources k = lane, lane+G, ...).
        // With T = s+d, a = #{j : c[j] > s} and b = #{j : c[j] >= T} (c_k is
        // non-increasing, and s >= c[R-r] by Eq. 7, so b <= a <= R-r), the
        // result of Alg. 4 is c with r copies of T inserted at b and the r
        // entries from a on dropped:
        //   c' = c[0..b) ++ T^r ++ c[b..a) ++ c[r+a..R),
        // and its last change is at index r+a-1, so it runs r+a loop steps.
        // (Both facts follow from the per-index form j < r: max(c[j], T);
        // j >= r: c[j-r] <= s ? c[j] : max(c[j], min(c[j-r], T)).)  The lane
        // finds a and b by two interleaved binary searches, shifts c[b..a)
        // up by r from the top down (a batch of reads before its writes, so
        // every read sees the old value) and writes T into [b, b+r).
        if (act && d > 0)
            for (int q = g.lane; q < m; q += G) {
                const int e = I.reqk[i * m + q];
                if (e == 0) break;
                const int k = e & 7, r = e >> 3;
                const int R = I.cap[k];
                const int T = s + d;
                short *ck = cst + I.cbase[k] * NG;
                int alo = 0, ahi = R - r, blo = 0, bhi = R - r;
                while (alo < ahi || blo < bhi) {
                    const int am = (alo + ahi) >> 1, bm = (blo + bhi) >> 1;
                    const int ca = ck[am * NG], cb = ck[bm * NG];
                    if (alo < ahi) {
                        if (ca > s) alo = am + 1;
                        else ahi = am;
                    }
                    if (blo < bhi) {
                        if (cb >= T) blo = bm + 1;
                        else bhi = bm;
                    }
                }
                const int a = alo, b = blo;
                int j = r + a - 1;
                for (; j - 3 >= r + b; j -= 4) {
                    const int x0 = ck[(j - r) * NG], x1 = ck[(j - 1 - r) * NG];
                    const int x2 = ck[(j - 2 - r) * NG], x3 = ck[(j - 3 - r) * NG];
                    ck[j * NG] = static_cast<short>(x0);
                    ck[(j - 1) * NG] = static_cast<short>(x1);
                    ck[(j - 2) * NG] = static_cast<short>(x2);
                    ck[(j - 3) * NG] = static_cast<short>(x3);
                }
                for (; j >= r + b; --j) ck[j * NG] = ck[(j - r) * NG];
                for (int x = b; x < b + r; ++x) ck[x * NG] = static_cast<short>(T);
                wk += r + a;                            // Alg. 4's loop steps
            }
        if (act) {
            if (S_out && g.lane == 0) S_out[i] = s;
            cmax = ::max(cmax, s + d);
        }
        push_finish<G>(I, i, s + d, esa, NG, g, act);
        __syncwarp();
        i = inext;
    }
    work += g.sum(wk);
    return cmax;
}

// One decode by the groups of a warp; PFX compiles the prefix-reuse paths in.
template <int G, bool PFX = false>
__device__ __forceinline__ int decode(const SInst &I, int mode, const int *W, int u, int v, bool active,
                                      int *area, int NG, const Group<G> &g, long long &work, int &err,
                                      int *S_out = nullptr, const Prefix &px = Prefix{nullptr, 1, 0, 0, nullptr},
                                      bool produce = false) {
    int wk = 0, c;
    if (mode == RCPSP_EVAL_CAPACITY)
        c = decode_capacity<G, PFX>(I, W, u, v, active, area, NG, g, wk, err, S_out, px, produce);
    else if (I.wps == 1)
        c = decode_time<G, 1, PFX>(I, W, u, v, active, area, NG, g, wk, err, S_out, px, produce);
    else if (I.wps == 2)
        c = decode_time<G, 2, PFX>(I, W, u, v, active, area, NG, g, wk, err, S_out, px, produce);
    else
        c = decode_time<G, 4, PFX>(I, W, u, v, active, area, NG, g, wk, err, S_out, px, produce);
    work += wk;
    return c;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(kFull, x, o);
        x = y < x ? y : x;
    }
    return x;
}

__device__ __forceinline__ long long warp_sum_i64(long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ bool tc_get(const unsigned *tc, int u, int v, int delta) {
    const int b = u * delta + (v - u - 1);
    return (tc[b >> 5] >> (b & 31)) & 1u;
}

__device__ __forceinline__ void tc_put(unsigned *tc, int u, int v, int delta, bool on) {
    const int b = u * delta + (v - u - 1);
    if (on) tc[b >> 5] |= 1u << (b & 31);
    else tc[b >> 5] &= ~(1u << (b & 31));
}

// ---------------------------------------------------------------------------
// Steps 1-3 of an iteration (Sec. 6) on the CTA's current list W: the first
// successor / last predecessor position of every position (and, with prefix
// reuse, the kept decoder states of W, see Prefix), then the feasible moves
// (with csize > 1 only this cluster rank's chunks of 32 slots),
// ballot-compacted into `moves` and decoded by the groups.  The potential
// moves are filtered in passes of up to nthr slots while the list has room
// for a whole pass (it holds move_cap moves), then the warps drain the list:
// each warp takes the next NG moves from the counter s_mq[1] and decodes
// them in lockstep, so a warp with short decodes takes more of them and the
// block meets at one barrier per full list instead of one per round.  The
// list is in (u, v) order up to the order of the warps inside a pass, so the
// longest decodes (small u, with prefix reuse) go first.  Returns the
// thread's smallest key (C_max << 32 | u << 16 | v) among admissible moves
// -- not tabu, or C_max < aspiration -- or ~0 when it saw none.  Thread 0
// adds the number of decoded neighbours to *s_eval; every thread adds its
// decode work to my_work; with tally.t, warp 0 adds the work counters of
// the decodes (see TallyRef) once per batch of moves.  Starts and ends with a __syncthreads, so the
// caller may reset its reduction word before the call.
// ---------------------------------------------------------------------------
template <int G, bool PFX = false>
__device__ __forceinline__ unsigned long long best_admissible_key(
        const SInst &I, int mode, const int *W, const int *pos, int *fsp, int *lpp, const unsigned *tc,
        int *moves, int *area, int n, int delta, int nslots, unsigned dmagic, int move_cap, int aspiration,
        int csize, unsigned crank, int *s_mq, long long *s_eval, long long &my_work, int &err,
        const Prefix &px = Prefix{nullptr, 1, 0, 0, nullptr}, TallyRef tally = TallyRef{nullptr, nullptr}) {
    constexpr int NG = 32 / G;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, wl = tid & 31;
    const int gw = wl / G;
    const Group<G> g;
    (void)warp;
    // 1. first successor / last predecessor position of every position
    for (int p = tid; p < n; p += nthr) {
        const int a = W[p];
        int f = n, l = -1;
        for (int e = I.soff[a]; e < I.soff[a + 1]; ++e) f = ::min(f, pos[I.slist[e]]);
        for (int e = I.poff[a]; e < I.poff[a + 1]; ++e) l = ::max(l, pos[I.plist[e]]);
        fsp[p] = f;
        lpp[p] = l;
    }
    const int upd_all = mode == RCPSP_EVAL_CAPACITY ? I.sum_used : I.ub;
    unsigned long long my_key = ~0ull;
    const int pass = ::min(nthr, move_cap);      // slots of one filter pass (<= move_cap)
    int base = 0;
    if (nslots <= 0) __syncthreads();            // no moves (N <= 3): nothing to keep either
    while (base < nslots) {
        const bool first = base == 0;
        if (tid == 0) {
            s_mq[0] = 0;                          // compaction cursor
            s_mq[1] = 0;                          // drain cursor
            if (first && px.ready) *px.ready = 0;   // snapshots of W kept so far
        }
        __syncthreads();
        // 2. feasible moves, compacted, pass by pass while a pass still fits
        int nm = 0;
        while (base < nslots && nm + pass <= move_cap) {
            bool ok = false;
            int code = 0;
            if (tid < pass && base + tid < nslots) {
                const int slot = base + tid;
                const int q = delta > 1 ? static_cast<int>(__umulhi(static_cast<unsigned>(slot), dmagic)) : slot;
                const int u = 1 + q;
                const int v = u + 1 + (slot - q * delta);
                const bool mine = csize == 1 || static_cast<unsigned>((slot >> 5) % csize) == crank;
                if (mine && v <= n - 2 && fsp[u] > v && lpp[v] < u) {
                    ok = true;
                    code = u | (v << 16);
                }
            }
            const unsigned b = __ballot_sync(kFull, ok);
            int wb = 0;
            if (wl == 0 && b) wb = atomicAdd(&s_mq[0], __popc(b));
            wb = __shfl_sync(kFull, wb, 0);
            if (ok) moves[wb + __popc(b & ((1u << wl) - 1u))] = code;
            nm += __syncthreads_count(ok);        // the same count in every thread
            base += pass;
        }
        // 3. decode the neighbours: the groups of a warp take NG consecutive
        // moves at a time and decode them in lockstep.  With prefix reuse,
        // warp 0 first decodes the current list and keeps its state before
        // positions K, 2K, ... (its work is not a neighbour's), publishing
        // each as it goes, while the other warps start on the moves.
        if (PFX && px.base && first && warp == 0) {
            long long w0 = 0;
            decode<G, PFX>(I, mode, W, 0, 0, gw == 0, area, NG, g, w0, err, nullptr, px, true);
            if (px.ready && wl == 0) store_release_cta(px.ready, px.count);
            if (tally.t) {
                // a full decode, and the kept states it wrote
                __syncwarp();
                int kw = 0;
                for (int j = 1 + wl; j <= px.count; j += 32) kw += __ldcg(px.base + (j - 1) * px.stride + kPxWords);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) kw += __shfl_xor_sync(kFull, kw, o);
                if (wl == 0) {
                    tally.t[kTallyPlaced] += n;
                    tally.t[kTallyUpd] += upd_all;
                    tally.t[kTallySucc] += I.n_arcs;
                    tally.t[kTallyKept] += kw;
                    tally.t[kTallySteps] += w0;
                }
            }
        }
        for (;;) {
            int q0 = 0;
            if (wl == 0) q0 = atomicAdd(&s_mq[1], NG);
            q0 = __shfl_sync(kFull, q0, 0);
            if (q0 >= nm) break;
            const int q = q0 + gw;
            const bool act = q < nm;
            const int code = act ? moves[q] : 0;
            const int u = code & 0xffff, v = code >> 16;
            const int c = decode<G, PFX>(I, mode, W, u, v, act, area, NG, g, my_work, err, nullptr, px);
            if (PFX && px.base && tally.t && act && g.lane == 0) atomicAdd(&tally.hist[::min(u / px.K, px.count)], 1);
            if (act && (!tc_get(tc, u, v, delta) || c < aspiration)) {
                const unsigned long long key =
                    (static_cast<unsigned long long>(c) << 32) | static_cast<unsigned>(code & 0xffff) << 16 |
                    static_cast<unsigned>(v);
                my_key = key < my_key ? key : my_key;
            }
        }
        if (tid == 0) *s_eval += nm;
        __syncthreads();
        if (tally.t && warp == 0) {
            // the batch's neighbour decodes: full ones, and those that
            // restored kept state j before position j*K (hist[j])
            long long v[kTallies] = {0, 0, 0, 0, 0};
            if (PFX && px.base) {
                for (int j = wl; j <= px.count; j += 32) {
                    const long long c = tally.hist[j];
                    tally.hist[j] = 0;
                    if (c == 0) continue;
                    if (j == 0) {
                        v[kTallyPlaced] += c * n;
                        v[kTallyUpd] += c * upd_all;
                        v[kTallySucc] += c * I.n_arcs;
                    } else {
                        const int *sn = px.base + (j - 1) * px.stride;
                        v[kTallyPlaced] += c * (n - j * px.K);
                        v[kTallyUpd] += c * (upd_all - __ldcg(sn + kPxUpd));
                        v[kTallySucc] += c * (I.n_arcs - __ldcg(sn + kPxSucc));
                        v[kTallyKept] += c * __ldcg(sn + kPxWords);
                        v[kTallySteps] -= c * __ldcg(sn + kPxWork);
                    }
                }
#pragma unroll
                for (int x = 0; x < kTallies; ++x) v[x] = warp_sum_i64(v[x]);
            } else {
                v[kTallyPlaced] = static_cast<long long>(nm) * n;
                v[kTallyUpd] = static_cast<long long>(nm) * upd_all;
                v[kTallySucc] = static_cast<long long>(nm) * I.n_arcs;
            }
            if (wl == 0)
                for (int x = 0; x < kTallies; ++x) tally.t[x] += v[x];
        }
    }
    return my_key;
}

// Slot / delta by a multiply-high: exact while slot * delta < 2^32, which
// holds because the host clamps delta to N - 3 (the same moves).
__device__ __forceinline__ unsigned slot_magic(int delta) {
    return delta > 1 ? 0xffffffffu / static_cast<unsigned>(delta) + 1u : 0u;
}

}  // namespace
}  // namespace rcpsp
