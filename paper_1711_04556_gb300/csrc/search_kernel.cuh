// sm_103a tabu search kernel for the RCPSP (Bukata, Sucha, Hanzalek), the
// template shared by search_kernel.cu (CTAs of up to 384 threads, two per
// SM), search_kernel_wide.cu (up to 512, two per SM) and
// search_kernel_solo.cu (up to 512, one per SM), which compile in parallel.
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
// The work queue is a single atomicAdd.  The kernel waits in two places
// only, each bounded by the global timer: a CTA of a sliced launch
// (SliceSched) may pop a slice whose previous slice another CTA is still
// running, and with prefix reuse a warp's neighbour decodes may wait for a
// kept state that warp 0 of the same CTA is still writing.  Internal inconsistencies set an error word that the host reads
// as a status.
#pragma once

#include "device_search.cuh"

namespace rcpsp {
namespace {

__device__ __forceinline__ int load_acquire_gpu(const int *x) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(x) : "memory");
    return v;
}

__device__ __forceinline__ int load_relaxed_gpu(const int *x) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(x) : "memory");
    return v;
}

// Iteration at which slice `slice` of a search whose call started at
// iteration it0 and runs `iters` iterations stops: slices are
// ceil(iters / nsl) iterations long, the last one shorter.
__device__ __forceinline__ int slice_end(int it0, int iters, int slice, int nsl) {
    if (nsl <= 1) return it0 + iters;
    const int per = (iters + nsl - 1) / nsl;
    return it0 + ::min(iters, (slice + 1) * per);
}

constexpr unsigned long long kSliceWaitNs = 10000000000ull;   // 10 s without progress

// Before slice s of a search runs: wait until its slice s-1 is done (sync[0]
// reaches s).  The slice before was popped earlier by a CTA that is running
// it, so the wait ends unless that CTA stops making progress: it is given
// up, and the search abandoned, only after kSliceWaitNs without the search's
// iteration count (sync[1]) moving.  Returns 1: run slice s, 0: the search
// has finished (nothing to do), -1: gave up.
__device__ int slice_wait(int *sync, int s) {
    int d = load_acquire_gpu(sync);
    if (d < s) {
        int last = load_relaxed_gpu(sync + 1);
        unsigned long long t0 = global_timer_ns();
        while ((d = load_acquire_gpu(sync)) < s) {
            const int pr = load_relaxed_gpu(sync + 1);
            const unsigned long long t = global_timer_ns();
            if (pr != last) {
                last = pr;
                t0 = t;
            } else if (t - t0 > kSliceWaitNs) {
                atomicOr(sync, kSliceAbandoned);
                return -1;
            }
            __nanosleep(200);
        }
    }
    return d == s ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Persistent search kernel.  With csize > 1 it runs as clusters of csize
// CTAs, one search per cluster: every CTA holds the same search state,
// examines its share of the potential moves (chunks of 32 slots, round
// robin over the cluster ranks), finds its best admissible key, and after a
// cluster barrier reads the other CTAs' keys through distributed shared
// memory; all CTAs then apply the same move.  Rank 0 pops the work queue,
// sums the counters and writes the results.  NT is the most threads a CTA
// may have; MB CTAs of NT threads share an SM's registers (MB = 1: a build
// for launches whose shared memory holds one CTA per SM anyway, which may
// then take up to twice the registers).
// ---------------------------------------------------------------------------
template <int G, bool PFX, int NT, int MB>
__global__ void __launch_bounds__(NT, MB) search_kernel(const LaunchItem *__restrict__ items, int count,
                                                      int *__restrict__ queue, int move_cap, int csize,
                                                      int *__restrict__ gsnap, int gsnap_words, SliceSched sl) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int s_mq[3];   // compaction and drain cursors, kept snapshots
    __shared__ int s_item, s_C, s_Cbest, s_widx, s_it, s_improved, s_err, s_it0, s_it_end, s_slice_end;
    __shared__ int s_run;     // 1: run the popped slice, 0: skip it
    __shared__ unsigned long long s_bestp[2], s_t0;      // best key of the iteration, by parity
    __shared__ long long s_eval, s_work;
    __shared__ long long s_tally[kTallies];   // work counters of the decodes (TallyRef)
    __shared__ int s_hist[32];
    const unsigned crank = csize > 1 ? cg::this_cluster().block_rank() : 0u;

    constexpr int NG = 32 / G;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, wl = tid & 31;
    const int ngroups = (nthr >> 5) * NG;
    const int gw = wl / G;                     // group inside the warp
    const Group<G> g;

    // (the slice values below are recomputed where they are needed, from the
    // launch parameters and s_item, so that none stays live across the
    // search loop)
    for (;;) {
        if (tid == 0 && crank == 0) {
            const int q = atomicAdd(queue, 1);
            int run = 1;
            if (sl.nslices > 1 && q < count * sl.nslices) {
                const int si = q / count, k = q - si * count;
                run = slice_wait(sl.sync + 2 * k, si);
                if (run < 0) {
                    // abandoned: the search reports a device error
                    const LaunchItem &ik = items[k];
                    ik.out[2 * ik.h.n + kOutStatus] = RCPSP_E_DEVICE;
                    run = 0;
                }
            }
            s_item = q;
            s_run = run;
        }
        int item, run;
        if (csize > 1) {
            cg::this_cluster().sync();
            item = *cg::this_cluster().map_shared_rank(&s_item, 0);
            run = *cg::this_cluster().map_shared_rank(&s_run, 0);
            cg::this_cluster().sync();                      // read before rank 0 pops again
        } else {
            __syncthreads();
            item = s_item;
            run = s_run;
        }
        if (item >= count * (sl.nslices > 1 ? sl.nslices : 1)) break;
        if (!run) {
            if (csize == 1) __syncthreads();                // every thread has read s_item
            continue;
        }
        const int slice = item / count;                     // 0 unless the launch is sliced
        const int ki = item - slice * count;
        const LaunchItem &it = items[ki];
        const InstHeader &h = it.h;
        const int n = h.n, mode = it.mode, delta = it.delta, tl = it.tabu_len;
        const int pw = profile_words(mode, h.wps, h.ub, h.sum_cap);
        const int pk = PFX ? it.prefix_k : 0;
        const StateLayout S = state_layout(h.inst_words, n, tl, delta, move_cap, pw, ngroups, mode);
        const Prefix px{pk > 0 ? gsnap + static_cast<long long>(blockIdx.x) * gsnap_words : nullptr,
                        pk > 0 ? pk : 1, prefix_count(n, pk), prefix_stride(n, pw), pk > 0 ? s_mq + 2 : nullptr};
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
        const int tcw = (n * delta + 31) / 32;
        int err = 0;
        // slice state of this search (sliced launches)
        const bool from_slice = slice > 0;
        if (from_slice || (it.state && (it.ckpt & kCkptResume))) {
            // continue a saved search -- the caller's kept state, or the one
            // the previous slice of this launch left -- with lists, tabu
            // state, iteration and makespans as they were; the counters so
            // far ride on rank 0.  Read past L1: another SM wrote them.
            const CkptLayout CL = ckpt_layout(n, tl, delta);
            const int32_t *sv = from_slice ? sl.states + it.slice_off : it.state;
            for (int p = tid; p < n; p += nthr) {
                const int a = __ldcg(sv + CL.W + p);
                W[p] = a;
                pos[a] = p;
                Wbest[p] = __ldcg(sv + CL.Wbest + p);
            }
            for (int x = tid; x < tl; x += nthr) stl[x] = __ldcg(sv + CL.stl + x);
            for (int x = tid; x < tcw; x += nthr) tc[x] = static_cast<unsigned>(__ldcg(sv + CL.tc + x));
            if (tid < kTallies) {
                // the work counters are the call's: kept across slices only
                const int32_t *xt = sv + CL.words + kSlTally + 2 * tid;
                s_tally[tid] = from_slice && crank == 0
                                   ? (static_cast<long long>(static_cast<uint32_t>(__ldcg(xt))) |
                                      (static_cast<long long>(__ldcg(xt + 1)) << 32))
                                   : 0;
            }
            if (tid < 32) s_hist[tid] = 0;
            if (tid == 0) {
                s_widx = __ldcg(sv + kCkWidx);
                s_it = __ldcg(sv + kCkIters);
                if (from_slice) {
                    const int32_t *xs = sv + CL.words;
                    s_it0 = __ldcg(xs + kSlIt0);
                    s_t0 = static_cast<unsigned long long>(static_cast<uint32_t>(__ldcg(xs + kSlT0Lo))) |
                           (static_cast<unsigned long long>(static_cast<uint32_t>(__ldcg(xs + kSlT0Hi))) << 32);
                    s_err = crank == 0 ? __ldcg(xs + kSlErr) : 0;
                } else {
                    s_it0 = s_it;                 // iterations before this call
                    s_t0 = global_timer_ns();
                    s_err = 0;
                }
                s_it_end = s_it0 + it.iterations;
                s_slice_end = slice_end(s_it0, it.iterations, slice, sl.nslices);
                s_C = __ldcg(sv + kCkC);
                s_Cbest = __ldcg(sv + kCkCbest);
                const long long ev = static_cast<long long>(static_cast<uint32_t>(__ldcg(sv + kCkEvalLo))) |
                                     (static_cast<long long>(__ldcg(sv + kCkEvalHi)) << 32);
                const long long wk = static_cast<long long>(static_cast<uint32_t>(__ldcg(sv + kCkWorkLo))) |
                                     (static_cast<long long>(__ldcg(sv + kCkWorkHi)) << 32);
                s_eval = crank == 0 ? ev : 0;
                s_work = crank == 0 ? wk : 0;
            }
            __syncthreads();
        } else {
            const int32_t *W0 = it.record + h.inst_words;
            for (int p = tid; p < n; p += nthr) {
                const int a = W0[p];
                W[p] = a;
                Wbest[p] = a;
                pos[a] = p;
            }
            for (int x = tid; x < tl; x += nthr) stl[x] = 0;             // (0,0) = empty move
            for (int x = tid; x < tcw; x += nthr) tc[x] = 0u;
            if (tid < kTallies) s_tally[tid] = 0;
            if (tid < 32) s_hist[tid] = 0;
            if (tid == 0) {
                s_t0 = global_timer_ns();
                s_widx = 0;
                s_it = 0;
                s_it0 = 0;
                s_it_end = it.iterations;
                s_slice_end = slice_end(0, it.iterations, slice, sl.nslices);
                s_eval = 0;
                s_work = 0;
                s_err = 0;
            }
            __syncthreads();
            if (warp == 0) {
                long long w0 = 0;
                const int c0 = decode<G>(I, mode, W, 0, 0, gw == 0, area, NG, g, w0, err);
                if (gw == 0 && g.lane == 0) {
                    s_C = c0;
                    s_Cbest = c0;
                }
            }
            __syncthreads();
        }

        const int nslots = n > 3 ? (n - 3) * delta : 0;
        const unsigned dmagic = slot_magic(delta);
        long long my_work = 0;
        for (;;) {
            if (s_it >= s_slice_end || (it.stop_at_cp && s_Cbest == h.cp)) break;
            const int par = s_it & 1;
            if (tid == 0) s_bestp[par] = ~0ull;
            const unsigned long long my_key =
                best_admissible_key<G, PFX>(I, mode, W, pos, fsp, lpp, tc, moves, area, n, delta, nslots, dmagic,
                                       move_cap, s_Cbest, csize, crank, s_mq, &s_eval, my_work, err, px,
                                       TallyRef{s_tally, s_hist});
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
                    it.trace[3 * (s_it - s_it0) + 0] = bu;
                    it.trace[3 * (s_it - s_it0) + 1] = bv;
                    it.trace[3 * (s_it - s_it0) + 2] = s_C;
                }
                s_it = s_it + 1;
                // progress, watched by a CTA that waits for this slice
                if (sl.nslices > 1 && crank == 0)
                    *reinterpret_cast<volatile int *>(sl.sync + 2 * (s_item % count) + 1) = s_it;
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
                    for (int x = 0; x < kTallies; ++x) s_tally[x] += *cg::this_cluster().map_shared_rank(&s_tally[x], r);
                }
            __syncthreads();
        }
        // finished: the last iteration of the call is done or C* reached the
        // critical path; otherwise only this slice of a sliced launch is
        const bool done = sl.nslices <= 1 || s_it >= s_it_end || (it.stop_at_cp && s_Cbest == h.cp);
        int32_t *out = it.out;
        if (crank == 0) {
            if (done) {
                // outputs: W*, its schedule S*, statistics
                if (warp == 0) {
                    long long w1 = 0;
                    int e1 = 0;
                    const int cb = decode<G>(I, mode, Wbest, 0, 0, gw == 0, area, NG, g, w1, e1, out + n);
                    if (gw == 0 && g.lane == 0) {
                        out[2 * n + kOutCmax] = cb;
                        if (e1 || cb != s_Cbest) atomicOr(&s_err, 2);
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
                    st[kOutIters0] = s_it0;
                    for (int x = 0; x < kTallies; ++x) {
                        // loop steps performed = the work counter plus its correction
                        const long long t = x == kTallySteps ? s_work + s_tally[x] : s_tally[x];
                        st[kOutPlacedLo + 2 * x] = static_cast<int32_t>(t & 0xffffffffll);
                        st[kOutPlacedLo + 2 * x + 1] = static_cast<int32_t>(t >> 32);
                    }
                    st[kOutMode] = mode;
                    st[kOutStatus] = s_err ? RCPSP_E_DEVICE : 0;
                    const unsigned long long t1 = global_timer_ns();
                    st[kOutT0Lo] = static_cast<int32_t>(s_t0 & 0xffffffffull);
                    st[kOutT0Hi] = static_cast<int32_t>(s_t0 >> 32);
                    st[kOutT1Lo] = static_cast<int32_t>(t1 & 0xffffffffull);
                    st[kOutT1Hi] = static_cast<int32_t>(t1 >> 32);
                }
            }
            // keep the search where it stopped: for a later call to resume
            // (the caller's state), or for the next slice of this launch
            int32_t *sv = done ? ((it.state && (it.ckpt & kCkptSave)) ? it.state : nullptr)
                               : sl.states + it.slice_off;
            if (sv) {
                const CkptLayout CL = ckpt_layout(n, tl, delta);
                for (int p = tid; p < n; p += nthr) {
                    __stcg(sv + CL.W + p, W[p]);
                    __stcg(sv + CL.Wbest + p, Wbest[p]);
                }
                for (int x = tid; x < tl; x += nthr) __stcg(sv + CL.stl + x, stl[x]);
                for (int x = tid; x < tcw; x += nthr) __stcg(sv + CL.tc + x, static_cast<int32_t>(tc[x]));
                if (tid == 0) {
                    __stcg(sv + kCkMagic, kCkptMagic);
                    __stcg(sv + kCkN, n);
                    __stcg(sv + kCkDelta, delta);
                    __stcg(sv + kCkTabu, tl);
                    __stcg(sv + kCkMode, mode);
                    __stcg(sv + kCkIters, s_it);
                    __stcg(sv + kCkC, s_C);
                    __stcg(sv + kCkCbest, s_Cbest);
                    __stcg(sv + kCkWidx, s_widx);
                    __stcg(sv + kCkEvalLo, static_cast<int32_t>(s_eval & 0xffffffffll));
                    __stcg(sv + kCkEvalHi, static_cast<int32_t>(s_eval >> 32));
                    __stcg(sv + kCkWorkLo, static_cast<int32_t>(s_work & 0xffffffffll));
                    __stcg(sv + kCkWorkHi, static_cast<int32_t>(s_work >> 32));
                    if (!done) {
                        // what the call has counted so far
                        int32_t *xs = sv + CL.words;
                        __stcg(xs + kSlIt0, s_it0);
                        __stcg(xs + kSlT0Lo, static_cast<int32_t>(s_t0 & 0xffffffffull));
                        __stcg(xs + kSlT0Hi, static_cast<int32_t>(s_t0 >> 32));
                        __stcg(xs + kSlErr, s_err);
                        for (int x = 0; x < kTallies; ++x) {
                            __stcg(xs + kSlTally + 2 * x, static_cast<int32_t>(s_tally[x] & 0xffffffffll));
                            __stcg(xs + kSlTally + 2 * x + 1, static_cast<int32_t>(s_tally[x] >> 32));
                        }
                    }
                }
            }
            if (sl.nslices > 1) {
                // publish: this slice of the search is done (all of it when finished)
                __syncthreads();
                if (tid == 0) {
                    const int q = s_item, qs = q / count;
                    __threadfence();
                    atomicMax(sl.sync + 2 * (q - qs * count), done ? sl.nslices : qs + 1);
                }
            }
        }
        __syncthreads();
    }
}

template <int G, int NT, int MB>
cudaError_t prepare_search_g(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(search_kernel<G, false, NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(search_kernel<G, true, NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    return e;
}

template <int G, bool PFX, int NT, int MB>
cudaError_t occupancy_g(int threads, size_t smem, int csize, int *units) {
    if (csize <= 1)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(units, search_kernel<G, PFX, NT, MB>, threads, smem);
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
    return cudaOccupancyMaxActiveClusters(units, search_kernel<G, PFX, NT, MB>, &cfg);
}

template <int G, bool PFX, int NT, int MB>
cudaError_t launch_search_g(const LaunchItem *items, int count, int *queue, int move_cap, int blocks,
                            int threads, size_t smem, cudaStream_t st, int csize, int *gsnap, int gsnap_words,
                            SliceSched sl) {
    if (csize <= 1) {
        search_kernel<G, PFX, NT, MB><<<blocks, threads, smem, st>>>(items, count, queue, move_cap, 1, gsnap, gsnap_words,
                                                                 sl);
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
    return cudaLaunchKernelEx(&cfg, search_kernel<G, PFX, NT, MB>, items, count, queue, move_cap, csize, gsnap,
                              gsnap_words, sl);
}

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

// The entry points of one build (thread bound NT, MB CTAs per SM), for
// every group size.
template <int NT, int MB>
cudaError_t prepare_search_nt(int group_size, size_t smem) {
    RCPSP_DISPATCH_G(group_size, return (prepare_search_g<GG, NT, MB>(smem)))
}

template <int NT, int MB>
cudaError_t search_occupancy_nt(int group_size, int threads, size_t smem, int csize, int *units, bool prefix) {
    if (prefix) RCPSP_DISPATCH_G(group_size, return (occupancy_g<GG, true, NT, MB>(threads, smem, csize, units)))
    RCPSP_DISPATCH_G(group_size, return (occupancy_g<GG, false, NT, MB>(threads, smem, csize, units)))
}

template <int NT, int MB>
cudaError_t launch_search_nt(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                             int blocks, int threads, size_t smem, cudaStream_t st, int csize, bool prefix,
                             int *gsnap, int gsnap_words, SliceSched sl) {
    if (prefix)
        RCPSP_DISPATCH_G(group_size, return (launch_search_g<GG, true, NT, MB>(items, count, queue, move_cap, blocks,
                                                                           threads, smem, st, csize, gsnap,
                                                                           gsnap_words, sl)))
    RCPSP_DISPATCH_G(group_size, return (launch_search_g<GG, false, NT, MB>(items, count, queue, move_cap, blocks,
                                                                        threads, smem, st, csize, nullptr, 0, sl)))
}

}  // namespace

// The 512-thread instances (search_kernel_wide.cu) and the one-CTA-per-SM
// instances (search_kernel_solo.cu).
cudaError_t prepare_search_wide(int group_size, size_t smem);
cudaError_t search_occupancy_wide(int group_size, int threads, size_t smem, int csize, int *units, bool prefix);
cudaError_t launch_search_wide(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                               int blocks, int threads, size_t smem, cudaStream_t st, int csize, bool prefix,
                               int *gsnap, int gsnap_words, SliceSched sl);
cudaError_t prepare_search_solo(int group_size, size_t smem);
cudaError_t search_occupancy_solo(int group_size, int threads, size_t smem, int csize, int *units, bool prefix);
cudaError_t launch_search_solo(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                               int blocks, int threads, size_t smem, cudaStream_t st, int csize, bool prefix,
                               int *gsnap, int gsnap_words, SliceSched sl);

}  // namespace rcpsp
