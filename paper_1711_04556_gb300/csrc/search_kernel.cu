// sm_103a kernels of the tabu search for the RCPSP (Bukata, Sucha, Hanzalek).
//
// One persistent CTA runs one search at a time and pops the next instance
// from a device work queue when it is done (Sec. 6: one block = one tabu
// search; the homogeneous model: instance and state stay on the device for
// the whole run).  Inside a CTA the neighbourhood is split over "groups" of
// G lanes (G = 1, 2, ..., 32, chosen at launch); a group decodes one
// neighbour at a time with the serial SGS of Alg. 7, its lanes cooperating
// on the resource scan and update.  Each group owns a private resource
// profile in shared memory, interleaved with the other groups of its warp so
// that the G lanes of every group always hit G distinct banks and the groups
// of a warp hit disjoint bank sets.
//
// Per iteration (Sec. 6):
//   1. first-successor / last-predecessor positions of the current list;
//      swap(u,v) satisfies Eqs. 5-6 iff v < firstSucc(u) and
//      u > lastPred(v) -- the same predicate, evaluated in O(1);
//   2. feasible moves of the reduced neighbourhood (v - u <= delta) are
//      ballot-compacted into shared memory (Alg. 1's filter, one pass);
//   3. the groups decode the neighbours (time-indexed: Algs. 5-6 on a
//      SWAR-packed profile; capacity-indexed: Eq. 7 and Alg. 4 in a
//      per-index closed form) and form the key (C_max, u, v) of every
//      admissible move (not tabu, or strictly better than C*_max);
//   4. warp-shuffle min, then a shared-memory atomicMin, give the move;
//   5. one thread applies it and updates the simple tabu list (Alg. 3).
//
// The kernel never spins: the work queue is a single atomicAdd.  Internal
// inconsistencies set an error word that the host reads as a status.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "kernels.h"
#include "rcpsp_internal.h"

namespace rcpsp {
namespace {

namespace cg = cooperative_groups;

constexpr unsigned kFull = 0xffffffffu;
constexpr int kErrHorizon = 1;     // a profile window ran past UB

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
// element e at area[e*NG]; the profile (or capacity state) comes first, then
// es[i], the precedence earliest start of every activity.  Instead of
// reading the finish times of i's predecessors when i is placed (Alg. 7,
// lines 3-6), every placed activity raises es[] of its successors, so the
// placement of i starts from one broadcast load; the value is the same
// maximum.  Returns C_max; `work` gets the Alg. 5 (time-indexed) or Alg. 4
// (capacity-indexed) loop steps; S_out (may be null) gets start times.
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ int activity_at(const int *W, int p, int u, int v) {
    return p == u ? W[v] : (p == v ? W[u] : W[p]);
}

// es of every successor of i := max(es, f); inactive groups write nothing.
template <int G>
__device__ __forceinline__ void push_finish(const SInst &I, int i, int f, int *es, int NG, const Group<G> &g,
                                            bool active) {
    const int e0 = I.soff[i], ns = active ? I.soff[i + 1] - e0 : 0;
    for (int b = g.lane; b < ns; b += G) {
        int *x = es + I.slist[e0 + b] * NG;
        *x = ::max(*x, f);
    }
}

template <int G>
__device__ __forceinline__ void clear_es(int *es, int n, int NG, bool active, const Group<G> &g) {
    if (active)
        for (int x = g.lane; x < n; x += G) es[x * NG] = 0;
    __syncwarp();
}

// Time-indexed decode, WPS = 32-bit words per time step of the packed profile.
template <int G, int WPS>
__device__ int decode_time(const SInst &I, const int *W, int u, int v, bool active, int *area, int NG,
                           const Group<G> &g, int &work, int &err, int *S_out) {
    constexpr int U = G >= 32 ? 1 : (G >= 16 ? 2 : 4);   // steps a lane tests per round
    constexpr int R = G * U;                               // steps a group tests per round (<= 32)
    const int n = I.n, ub = I.ub;
    const int ubs = ub > 0 ? ub : 1;              // stride of one resource-word plane
    uint32_t *prof = reinterpret_cast<uint32_t *>(area);
    int *esa = area + WPS * ubs * NG;
    const uint32_t hi = I.hi;
    uint32_t capw[WPS];
#pragma unroll
    for (int w = 0; w < WPS; ++w) capw[w] = I.capw[w];
    clear_es<G>(esa, n, NG, active, g);
    // Every step starts with R_k free units (Sec. 5.2.1).  Steps at or after
    // the frontier F have not been touched by this decode, so they are not
    // stored: they are written the first time an activity covers them.
    int F = 0;
    int cmax = 0;
    int i = activity_at<G>(W, 0, u, v);
    for (int p = 0; p < n; ++p) {
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
        bool done = !active || d == 0;
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
                        fit[j] = fit[j] && (((x | hi) - rq[w]) & hi) == hi;
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
        if (active) {
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
        push_finish<G>(I, i, f, esa, NG, g, active);
        __syncwarp();
        i = inext;
    }
    return cmax;
}

template <int G>
__device__ int decode_capacity(const SInst &I, const int *W, int u, int v, bool active, int *area, int NG,
                               const Group<G> &g, int &work, int &err, int *S_out) {
    const int n = I.n, m = I.m;
    int *cst = area;                                   // c_k, concatenated
    int *esa = area + I.sum_cap * NG;
    if (active)
        for (int j = g.lane; j < I.sum_cap; j += G) cst[j * NG] = 0;   // Sec. 5.1.1
    clear_es<G>(esa, n, NG, active, g);
    int cmax = 0;
    int i = activity_at<G>(W, 0, u, v);
    for (int p = 0; p < n; ++p) {
        const int inext = activity_at<G>(W, p + 1 < n ? p + 1 : p, u, v);
        const int es = esa[i * NG];
        // Eq. 7: es_res = max over used resources of c_k[R_k - r_{i,k}]
        int er = 0;
        if (active)
            for (int k = g.lane; k < m; k += G) {
                const int r = I.reqk[i * m + k];
                if (r > 0) er = ::max(er, cst[(I.cbase[k] + I.cap[k] - r) * NG]);
            }
        er = g.max(er);
        const int s = ::max(es, er);
        const int d = I.dur[i];
        for (int k = 0; k < m; ++k) {
            const int r = I.reqk[i * m + k];
            const bool upd = active && d > 0 && r > 0;
            int last = -1;
            if (__any_sync(kFull, upd)) {
                // Alg. 4 as a per-index closed form of its result:
                //   j <  r : c'[j] = max(c[j], s+d)
                //   j >= r : c'[j] = c[j-r] <= s ? c[j] : max(c[j], min(c[j-r], s+d))
                // c_k is non-increasing, so with a = #{j : c[j] > s} nothing at
                // j >= r + a changes (there c[j-r] <= s).  a is found chunk by
                // chunk; the update then runs from the top chunk down so that
                // c[j-r] is still old when it is read.
                const int R = I.cap[k];
                int *ck = cst + I.cbase[k] * NG;
                int a = 0;
                bool more = upd;
                for (int J = 0; __any_sync(kFull, more); J += G) {
                    const int j = J + g.lane;
                    const bool above = more && j < R && ck[j * NG] > s;
                    const unsigned m = g.bits(__ballot_sync(kFull, above));
                    if (more) {
                        a += __popc(m);
                        more = m == (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) && J + G < R;
                    }
                }
                const int top = ::min(R, r + a);            // indices that can change: [0, top)
                const int topmax = __reduce_max_sync(kFull, upd ? top : 0);
                for (int J = ((topmax - 1) / G) * G; J >= 0; J -= G) {
                    const int j = J + g.lane;
                    int old = 0, prev = 0;
                    if (upd && j < top) {
                        old = ck[j * NG];
                        if (j >= r) prev = ck[(j - r) * NG];
                    }
                    __syncwarp();
                    if (upd && j < top) {
                        const int nv = j < r ? ::max(old, s + d)
                                             : (prev <= s ? old : ::max(old, ::min(prev, s + d)));
                        if (nv != old) {
                            ck[j * NG] = nv;
                            last = ::max(last, j);
                        }
                    }
                    __syncwarp();
                }
            }
            last = g.max(last);
            if (upd) work += last + 1;                 // Alg. 4 stops after its last change
        }
        if (active) {
            if (S_out && g.lane == 0) S_out[i] = s;
            cmax = ::max(cmax, s + d);
        }
        push_finish<G>(I, i, s + d, esa, NG, g, active);
        __syncwarp();
        i = inext;
    }
    (void)err;
    return cmax;
}

template <int G>
__device__ __forceinline__ int decode(const SInst &I, int mode, const int *W, int u, int v, bool active,
                                      int *area, int NG, const Group<G> &g, long long &work, int &err,
                                      int *S_out = nullptr) {
    int wk = 0, c;
    if (mode == RCPSP_EVAL_CAPACITY) c = decode_capacity<G>(I, W, u, v, active, area, NG, g, wk, err, S_out);
    else if (I.wps == 1) c = decode_time<G, 1>(I, W, u, v, active, area, NG, g, wk, err, S_out);
    else if (I.wps == 2) c = decode_time<G, 2>(I, W, u, v, active, area, NG, g, wk, err, S_out);
    else c = decode_time<G, 4>(I, W, u, v, active, area, NG, g, wk, err, S_out);
    work += wk;
    return c;
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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
// Persistent search kernel.  With csize > 1 it runs as clusters of csize
// CTAs, one search per cluster: every CTA holds the same search state,
// examines its share of the potential moves (chunks of 32 slots, round
// robin over the cluster ranks), finds its best admissible key, and after a
// cluster barrier reads the other CTAs' keys through distributed shared
// memory; all CTAs then apply the same move.  Rank 0 pops the work queue,
// sums the counters and writes the results.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(512, 2) search_kernel(const LaunchItem *__restrict__ items, int count,
                                                      int *__restrict__ queue, int move_cap, int csize) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int s_item, s_nmoves, s_C, s_Cbest, s_widx, s_it, s_improved, s_err;
    __shared__ unsigned long long s_bestp[2], s_t0;      // best key of the iteration, by parity
    __shared__ long long s_eval, s_work;
    const unsigned crank = csize > 1 ? cg::this_cluster().block_rank() : 0u;

    constexpr int NG = 32 / G;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, wl = tid & 31;
    const int ngroups = (nthr >> 5) * NG;
    const int gw = wl / G;                     // group inside the warp
    const Group<G> g;

    for (;;) {
        if (tid == 0 && crank == 0) s_item = atomicAdd(queue, 1);
        int item;
        if (csize > 1) {
            cg::this_cluster().sync();
            item = *cg::this_cluster().map_shared_rank(&s_item, 0);
            cg::this_cluster().sync();                      // read before rank 0 pops again
        } else {
            __syncthreads();
            item = s_item;
        }
        if (item >= count) break;
        const LaunchItem it = items[item];
        const InstHeader &h = it.h;
        const int n = h.n, mode = it.mode, delta = it.delta, tl = it.tabu_len;
        const int pw = profile_words(mode, h.wps, h.ub, h.sum_cap);
        const StateLayout S = state_layout(h.inst_words, n, tl, delta, move_cap, pw, ngroups);
        stage_instance(sm, it.record, h.inst_words);
        const SInst I = bind_instance(sm, h);
        int *W = sm + S.W;
        int *pos = sm + S.pos;
        int *Wbest = sm + S.Wbest;
        int *fsp = sm + S.fsp;
        int *lpp = sm + S.lpp;
        int *stl = sm + S.stl;
        unsigned *tc = reinterpret_cast<unsigned *>(sm + S.tc);
        int *moves = sm + S.moves;
        int *area = sm + S.groups + warp * NG * S.group_words + wl / G;
        const int32_t *W0 = it.record + h.inst_words;
        for (int p = tid; p < n; p += nthr) {
            const int a = W0[p];
            W[p] = a;
            Wbest[p] = a;
            pos[a] = p;
        }
        for (int x = tid; x < tl; x += nthr) stl[x] = 0;                 // (0,0) = empty move
        for (int x = tid; x < (n * delta + 31) / 32; x += nthr) tc[x] = 0u;
        if (tid == 0) {
            s_t0 = global_timer_ns();
            s_widx = 0;
            s_it = 0;
            s_eval = 0;
            s_work = 0;
            s_err = 0;
        }
        __syncthreads();
        int err = 0;
        if (warp == 0) {
            long long w0 = 0;
            const int c0 = decode<G>(I, mode, W, 0, 0, gw == 0, area, NG, g, w0, err);
            if (gw == 0 && g.lane == 0) {
                s_C = c0;
                s_Cbest = c0;
            }
        }
        __syncthreads();
        const int nslots = n > 3 ? (n - 3) * delta : 0;
        // slot / delta by a multiply-high: exact while slot * delta < 2^32,
        // which holds because the host clamps delta to N - 3 (same moves)
        const unsigned dmagic = delta > 1 ? 0xffffffffu / static_cast<unsigned>(delta) + 1u : 0u;
        long long my_work = 0;
        for (;;) {
            if (s_it >= it.iterations || (it.stop_at_cp && s_Cbest == h.cp)) break;
            // 1. first successor / last predecessor position of every position
            for (int p = tid; p < n; p += nthr) {
                const int a = W[p];
                int f = n, l = -1;
                for (int e = I.soff[a]; e < I.soff[a + 1]; ++e) f = ::min(f, pos[I.slist[e]]);
                for (int e = I.poff[a]; e < I.poff[a + 1]; ++e) l = ::max(l, pos[I.plist[e]]);
                fsp[p] = f;
                lpp[p] = l;
            }
            const int par = s_it & 1;
            if (tid == 0) s_bestp[par] = ~0ull;
            __syncthreads();
            const int cbest = s_Cbest;
            unsigned long long my_key = ~0ull;
            for (int base = 0; base < nslots; base += move_cap) {
                const int stripe = ::min(move_cap, nslots - base);
                if (tid == 0) s_nmoves = 0;
                __syncthreads();
                // 2. feasible moves of the stripe, compacted
                for (int k0 = 0; k0 < stripe; k0 += nthr) {
                    const int k = k0 + tid;
                    bool ok = false;
                    int code = 0;
                    if (k < stripe) {
                        const int slot = base + k;
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
                    if (wl == 0 && b) wb = atomicAdd(&s_nmoves, __popc(b));
                    wb = __shfl_sync(kFull, wb, 0);
                    if (ok) moves[wb + __popc(b & ((1u << wl) - 1u))] = code;
                }
                __syncthreads();
                const int nm = s_nmoves;
                // 3. decode the neighbours
                // (the groups of a warp take consecutive moves and decode them in lockstep)
                for (int q0 = warp * NG; q0 < nm; q0 += ngroups) {
                    const int q = q0 + gw;
                    const bool act = q < nm;
                    const int code = act ? moves[q] : 0;
                    const int u = code & 0xffff, v = code >> 16;
                    const int c = decode<G>(I, mode, W, u, v, act, area, NG, g, my_work, err);
                    if (act && (!tc_get(tc, u, v, delta) || c < cbest)) {
                        const unsigned long long key =
                            (static_cast<unsigned long long>(c) << 32) | static_cast<unsigned>(code & 0xffff) << 16 |
                            static_cast<unsigned>(v);
                        my_key = key < my_key ? key : my_key;
                    }
                }
                if (tid == 0) s_eval += nm;
                __syncthreads();
            }
            // 4. best admissible move of the block, then of the cluster
            const unsigned long long wk = warp_min_u64(my_key);
            if (wl == 0 && wk != ~0ull) atomicMin(&s_bestp[par], wk);
            if (csize > 1) cg::this_cluster().sync();
            else __syncthreads();
            // 5. apply, Alg. 3 (every CTA of a cluster applies the same move)
            if (tid == 0) {
                unsigned long long kb = s_bestp[par];
                for (int r = 1; r < csize; ++r) {
                    const unsigned long long o = *cg::this_cluster().map_shared_rank(&s_bestp[par],
                                                                                  (crank + r) % csize);
                    kb = o < kb ? o : kb;
                }
                int bu = 0, bv = 0;
                s_improved = 0;
                if (kb != ~0ull) {
                    const int c = static_cast<int>(kb >> 32);
                    bu = static_cast<int>((kb >> 16) & 0xffff);
                    bv = static_cast<int>(kb & 0xffff);
                    const int a = W[bu], b = W[bv];
                    W[bu] = b;
                    W[bv] = a;
                    pos[b] = bu;
                    pos[a] = bv;
                    s_C = c;
                    if (c < s_Cbest) {
                        s_Cbest = c;
                        s_improved = 1;
                    }
                }
                const int old = stl[s_widx];
                if (old) tc_put(tc, old & 0xffff, old >> 16, delta, false);
                stl[s_widx] = bu | (bv << 16);
                if (bu | bv) tc_put(tc, bu, bv, delta, true);
                s_widx = s_widx + 1 == tl ? 0 : s_widx + 1;
                if (it.trace && crank == 0) {
                    it.trace[3 * s_it + 0] = bu;
                    it.trace[3 * s_it + 1] = bv;
                    it.trace[3 * s_it + 2] = s_C;
                }
                s_it = s_it + 1;
            }
            __syncthreads();
            if (s_improved)
                for (int p = tid; p < n; p += nthr) Wbest[p] = W[p];
        }
        // work of all groups (the lanes of a group hold the same count)
        const long long ws = warp_sum_i64(g.lane == 0 ? my_work : 0);
        if (wl == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&s_work), static_cast<unsigned long long>(ws));
        if (err) atomicOr(&s_err, err);
        __syncthreads();
        if (csize > 1) {
            // rank 0 adds up the cluster's counters; the other CTAs go on to
            // the next queue pop, which waits for rank 0
            cg::this_cluster().sync();
            if (crank == 0 && tid == 0)
                for (int r = 1; r < csize; ++r) {
                    s_eval += *cg::this_cluster().map_shared_rank(&s_eval, r);
                    s_work += *cg::this_cluster().map_shared_rank(&s_work, r);
                    s_err |= *cg::this_cluster().map_shared_rank(&s_err, r);
                }
            __syncthreads();
        }
        // outputs: W*, its schedule S*, statistics (rank 0)
        int32_t *out = it.out;
        if (crank == 0) {
        if (warp == 0) {
            long long w1 = 0;
            int e1 = 0;
            const int cb = decode<G>(I, mode, Wbest, 0, 0, gw == 0, area, NG, g, w1, e1, out + n);
            if (gw == 0) {
                if (g.lane == 0) {
                    out[2 * n + kOutCmax] = cb;
                    if (e1 || cb != s_Cbest) atomicOr(&s_err, 2);
                }
            }
        }
        for (int p = tid; p < n; p += nthr) out[p] = Wbest[p];
        __syncthreads();
        if (tid == 0) {
            int32_t *st = out + 2 * n;
            st[kOutEvalLo] = static_cast<int32_t>(s_eval & 0xffffffffll);
            st[kOutEvalHi] = static_cast<int32_t>(s_eval >> 32);
            st[kOutWorkLo] = static_cast<int32_t>(s_work & 0xffffffffll);
            st[kOutWorkHi] = static_cast<int32_t>(s_work >> 32);
            st[kOutIters] = s_it;
            st[kOutMode] = mode;
            st[kOutStatus] = s_err ? RCPSP_E_DEVICE : 0;
            const unsigned long long t1 = global_timer_ns();
            st[kOutT0Lo] = static_cast<int32_t>(s_t0 & 0xffffffffull);
            st[kOutT0Hi] = static_cast<int32_t>(s_t0 >> 32);
            st[kOutT1Lo] = static_cast<int32_t>(t1 & 0xffffffffull);
            st[kOutT1Hi] = static_cast<int32_t>(t1 >> 32);
        }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Decoding of caller-given lists (rcpsp_evaluate_lists).
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(512, 2) evaluate_kernel(LaunchItem item, const int32_t *__restrict__ lists,
                                                        int count, int32_t *__restrict__ start,
                                                        int32_t *__restrict__ cmax_out,
                                                        long long *__restrict__ work_out,
                                                        int *__restrict__ err_out) {
    extern __shared__ __align__(16) int sm[];
    constexpr int NG = 32 / G;
    const int tid = threadIdx.x, warp = tid >> 5, wl = tid & 31;
    const int ngroups = (blockDim.x >> 5) * NG;
    const int gw = wl / G;
    const int gid = warp * NG + gw;
    const Group<G> g;
    const InstHeader &h = item.h;
    const int n = h.n, mode = item.mode;
    const int pw = profile_words(mode, h.wps, h.ub, h.sum_cap);
    // per-group list buffers take the place of the move buffer
    const StateLayout S = state_layout(h.inst_words, n, 0, 0, ngroups * align4(n), pw, ngroups);
    stage_instance(sm, item.record, h.inst_words);
    __syncthreads();
    const SInst I = bind_instance(sm, h);
    int *myW = sm + S.moves + gid * align4(n);
    int *area = sm + S.groups + warp * NG * S.group_words + wl / G;
    int err = 0;
    for (int l0 = (blockIdx.x * (blockDim.x >> 5) + warp) * NG; l0 < count; l0 += gridDim.x * ngroups) {
        const int l = l0 + gw;
        const bool act = l < count;
        // an idle group follows the lockstep on the identity list, reading only
        for (int p = g.lane; p < n; p += G) myW[p] = act ? lists[static_cast<long long>(l) * n + p] : p;
        __syncwarp();
        long long wk = 0;
        const int c = decode<G>(I, mode, myW, 0, 0, act, area, NG, g, wk, err,
                                act ? start + static_cast<long long>(l) * n : nullptr);
        if (act) {
            if (g.lane == 0) {
                cmax_out[l] = c;
                work_out[l] = wk;
            }
        }
        __syncwarp();
    }
    if (err) atomicOr(err_out, err);
}

template <int G>
cudaError_t prepare_search_g(size_t smem) {
    return cudaFuncSetAttribute(search_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem));
}

template <int G>
cudaError_t occupancy_g(int threads, size_t smem, int csize, int *units) {
    if (csize <= 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(units, search_kernel<G>, threads, smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(units, search_kernel<G>, &cfg);
}

template <int G>
cudaError_t launch_search_g(const LaunchItem *items, int count, int *queue, int move_cap, int blocks,
                            int threads, size_t smem, cudaStream_t st, int csize) {
    if (csize <= 1) {
        search_kernel<G><<<blocks, threads, smem, st>>>(items, count, queue, move_cap, 1);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, search_kernel<G>, items, count, queue, move_cap, csize);
}

template <int G>
cudaError_t launch_eval_g(const LaunchItem &item, const int32_t *lists, int count, int32_t *start,
                          int32_t *cmax, long long *work, int *err, int blocks, int threads, size_t smem,
                          cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(evaluate_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    evaluate_kernel<G><<<blocks, threads, smem, st>>>(item, lists, count, start, cmax, work, err);
    return cudaGetLastError();
}

}  // namespace

#define RCPSP_DISPATCH_G(G_, CALL)                 \
    switch (G_) {                                  \
        case 1: { constexpr int GG = 1; CALL; }    \
        case 2: { constexpr int GG = 2; CALL; }    \
        case 4: { constexpr int GG = 4; CALL; }    \
        case 8: { constexpr int GG = 8; CALL; }    \
        case 16: { constexpr int GG = 16; CALL; }  \
        case 32: { constexpr int GG = 32; CALL; }  \
        default: return cudaErrorInvalidValue;     \
    }

cudaError_t prepare_search(int group_size, size_t smem) {
    RCPSP_DISPATCH_G(group_size, return prepare_search_g<GG>(smem))
}

cudaError_t search_occupancy(int group_size, int threads, size_t smem, int csize, int *units) {
    RCPSP_DISPATCH_G(group_size, return occupancy_g<GG>(threads, smem, csize, units))
}

cudaError_t launch_search(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                          int blocks, int threads, size_t smem, cudaStream_t st, int csize) {
    RCPSP_DISPATCH_G(group_size,
                     return launch_search_g<GG>(items, count, queue, move_cap, blocks, threads, smem, st, csize))
}

cudaError_t launch_evaluate(int group_size, const LaunchItem &item, const int32_t *lists, int count,
                            int32_t *start, int32_t *cmax, long long *work, int *err, int blocks, int threads,
                            size_t smem, cudaStream_t st) {
    switch (group_size) {
        case 1: return launch_eval_g<1>(item, lists, count, start, cmax, work, err, blocks, threads, smem, st);
        case 2: return launch_eval_g<2>(item, lists, count, start, cmax, work, err, blocks, threads, smem, st);
        case 4: return launch_eval_g<4>(item, lists, count, start, cmax, work, err, blocks, threads, smem, st);
        case 8: return launch_eval_g<8>(item, lists, count, start, cmax, work, err, blocks, threads, smem, st);
        case 16: return launch_eval_g<16>(item, lists, count, start, cmax, work, err, blocks, threads, smem, st);
        case 32: return launch_eval_g<32>(item, lists, count, start, cmax, work, err, blocks, threads, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcpsp
