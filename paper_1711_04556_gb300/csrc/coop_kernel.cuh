// sm_103a kernel of the co-operating tabu searches (Sec. 6.1, Eq. 8).
// Included by coop_kernel.cu (G = 1, 2, 4) and coop_kernel_wide.cu (G = 8,
// 16, 32), which compile in parallel.
//
// One instance is searched by a thread-block cluster of B CTAs; each CTA is
// one of the paper's blocks, a complete tabu search with its own list, tabu
// list and cache in shared memory, evaluating its whole neighbourhood per
// iteration exactly as the single search does.  The blocks exchange
// solutions through a working set F of |F| slots in global memory.
//
// The paper's blocks run asynchronously under read/write locks, which leaves
// the order of exchanges to the scheduler.  Here the blocks of a cluster
// advance in lockstep (one cluster barrier per iteration), and the exchange
// decisions are a deterministic function of values every CTA knows: after
// each iteration every CTA publishes its best makespan since its last read
// in distributed shared memory, and every CTA replays the same exchange plan
// -- writes in block order, then reads in block order -- on its own copy of
// the slot bookkeeping (makespan, read count Phi, iterations counter IC) and
// of every block's read state.  Only the lists and tabu states move through
// global memory: the writing CTA stores its best list, its tabu list and
// cache into the slot it read; after a second barrier the reading CTAs load
// their new slots.  A read of a slot that has been read more than Phi_max
// times without improvement applies Phi_steps random feasible swaps, each
// drawn with the next of the block's random words (an input), and decodes
// the result; a third barrier then shares the new makespans.  Eq. 8 is
// evaluated in IEEE double with correctly rounded operations only, so every
// CTA -- and the CPU reference -- gets the same iteration budget.
//
// Every wait in this kernel is a cluster barrier; the clusters never wait on
// each other, and the work queue is one atomicAdd per instance.
#pragma once

#include "device_search.cuh"
#include "kernels.h"

namespace rcpsp {
namespace {

// e^{-x} for x >= 0: (sum_{i=0..24} (-x/1024)^i / i!)^(2^10), Horner form,
// 0 for x > 700; correctly rounded operations only (no contraction).
__device__ double exp_neg(double x) {
    if (x > 700.0) return 0.0;
    const double y = __ddiv_rn(x, 1024.0);
    double t = 1.0;
    for (int i = 24; i >= 1; --i) t = __dsub_rn(1.0, __ddiv_rn(__dmul_rn(y, t), static_cast<double>(i)));
    for (int k = 0; k < 10; ++k) t = __dmul_rn(t, t);
    return t;
}

// Eq. 8 with the quantity factor read as I_block / 5:
// floor(I_block/5 * (0.8 e^{-100 (C^k/C* - 1)} + 0.2 e^{-4 IC^k / I_block})).
__device__ int assigned_iterations(int c_k, int c_star, long long ic_k, int i_block) {
    if (i_block <= 0) return 0;
    const double xq = c_star > 0
        ? __dmul_rn(100.0, __dsub_rn(__ddiv_rn(static_cast<double>(c_k), static_cast<double>(c_star)), 1.0))
        : 0.0;
    const double xi = __dmul_rn(4.0, __ddiv_rn(static_cast<double>(ic_k), static_cast<double>(i_block)));
    const double a = __dmul_rn(0.8, exp_neg(xq));
    const double b = __dmul_rn(0.2, exp_neg(xi));
    const double v = __dmul_rn(__ddiv_rn(static_cast<double>(i_block), 5.0), __dadd_rn(a, b));
    return static_cast<int>(v);       // v >= 0: truncation is the floor
}

// Potential move `slot` (u-major, v ascending) of the reduced neighbourhood.
__device__ __forceinline__ bool slot_move(int slot, int delta, unsigned dmagic, int n, const int *fsp,
                                          const int *lpp, int &u, int &v) {
    const int q = delta > 1 ? static_cast<int>(__umulhi(static_cast<unsigned>(slot), dmagic)) : slot;
    u = 1 + q;
    v = u + 1 + (slot - q * delta);
    return v <= n - 2 && fsp[u] > v && lpp[v] < u;
}

// Diversification by one warp: up to `steps` swaps, each the
// floor(w * n_f / 2^32)-th feasible move (u-major order) of the n_f feasible
// ones, w the block's next random word.  Returns the words consumed.
__device__ int diversify_warp(const SInst &I, int *W, int *pos, int *fsp, int *lpp, int n, int delta, int nslots,
                              unsigned dmagic, int steps, const uint32_t *words, int P, int cursor) {
    const int lane = threadIdx.x & 31;
    int used = 0;
    for (int s = 0; s < steps; ++s) {
        for (int p = lane; p < n; p += 32) {
            const int a = W[p];
            int f = n, l = -1;
            for (int e = I.soff[a]; e < I.soff[a + 1]; ++e) f = ::min(f, pos[I.slist[e]]);
            for (int e = I.poff[a]; e < I.poff[a + 1]; ++e) l = ::max(l, pos[I.plist[e]]);
            fsp[p] = f;
            lpp[p] = l;
        }
        __syncwarp();
        int nf = 0;
        for (int base = 0; base < nslots; base += 32) {
            int u, v;
            const bool ok = base + lane < nslots && slot_move(base + lane, delta, dmagic, n, fsp, lpp, u, v);
            nf += __popc(__ballot_sync(kFull, ok));
        }
        if (nf == 0) break;
        const uint32_t w = __ldg(words + (cursor + used) % P);
        ++used;
        const int pick = static_cast<int>((static_cast<unsigned long long>(w) * static_cast<unsigned>(nf)) >> 32);
        int acc = 0;
        for (int base = 0; base < nslots; base += 32) {
            int u = 0, v = 0;
            const bool ok = base + lane < nslots && slot_move(base + lane, delta, dmagic, n, fsp, lpp, u, v);
            const unsigned b = __ballot_sync(kFull, ok);
            const int cnt = __popc(b);
            if (acc + cnt > pick) {
                if (ok && __popc(b & ((1u << lane) - 1u)) == pick - acc) {
                    const int x = W[u], y = W[v];
                    W[u] = y;
                    W[v] = x;
                    pos[y] = u;
                    pos[x] = v;
                }
                break;
            }
            acc += cnt;
        }
        __syncwarp();
    }
    return used;
}

// Forward-backward improvement of the list W by warp 0 (group 0 decodes):
// the backward list (finish time descending, later position first) decoded
// on the reversed network, then the forward list (mirrored start ascending,
// earlier position first) decoded forward; repeated while the makespan gets
// strictly shorter.  Scratch: pos, Wx (a list), S and tau (N each).  Ends with
// W improved (or unchanged).
template <int G>
__device__ void fbi_warp(const SInst &I, int mode, int *W, int *Wx, int *pos, int *S, int *tau, int *area, int NG,
                         const Group<G> &g, int &err) {
    const int lane = threadIdx.x & 31, gw = lane / G, n = I.n;
    SInst Ir = I;                                   // the reversed network
    Ir.soff = I.poff;
    Ir.slist = I.plist;
    Ir.poff = I.soff;
    Ir.plist = I.slist;
    long long w0 = 0;
    int C = decode<G>(I, mode, W, 0, 0, gw == 0, area, NG, g, w0, err, S);
    C = __shfl_sync(kFull, C, 0);
    for (;;) {
        __syncwarp();
        for (int p = lane; p < n; p += 32) pos[W[p]] = p;
        __syncwarp();
        for (int a = lane; a < n; a += 32) {          // rank in the backward order
            const int fa = S[a] + I.dur[a], pa = pos[a];
            int r = 0;
            for (int b = 0; b < n; ++b) {
                const int fb = S[b] + I.dur[b];
                r += fb > fa || (fb == fa && pos[b] > pa);
            }
            Wx[r] = a;
        }
        __syncwarp();
        int T = decode<G>(Ir, mode, Wx, 0, 0, gw == 0, area, NG, g, w0, err, tau);
        T = __shfl_sync(kFull, T, 0);
        __syncwarp();
        for (int a = lane; a < n; a += 32) {          // rank in the forward order
            const int sa = T - tau[a] - I.dur[a], pa = pos[a];
            int r = 0;
            for (int b = 0; b < n; ++b) {
                const int sb = T - tau[b] - I.dur[b];
                r += sb < sa || (sb == sa && pos[b] < pa);
            }
            Wx[r] = a;
        }
        __syncwarp();
        int C2 = decode<G>(I, mode, Wx, 0, 0, gw == 0, area, NG, g, w0, err, S);
        C2 = __shfl_sync(kFull, C2, 0);
        if (!(C2 < C)) break;
        C = C2;
        __syncwarp();
        for (int p = lane; p < n; p += 32) W[p] = Wx[p];
    }
    __syncwarp();
}

// PFX: the variant with prefix reuse -- every CTA keeps the decoder states
// of its own current list at gsnap + blockIdx.x * gsnap_words (see Prefix),
// for the items with prefix_k > 0.
template <int G, bool PFX>
__global__ void __launch_bounds__(512, 2) coop_kernel(const CoopItem *__restrict__ items, int count,
                                                    int *__restrict__ queue, int move_cap, CoopConfig cfg,
                                                    int *__restrict__ gsnap, int gsnap_words) {
    extern __shared__ __align__(16) int sm[];
    __shared__ int s_mq[3];   // compaction and drain cursors, kept snapshots
    __shared__ int s_hist[32];
    __shared__ int s_item, s_C, s_Cbb, s_widx, s_it, s_err, s_improved;
    __shared__ unsigned long long s_best, s_t0;
    __shared__ long long s_eval, s_work;
    __shared__ long long s_tally[kTallies];   // work counters of the decodes (TallyRef)
    __shared__ int s_pub[2], s_pub_div[2];            // this CTA's best since its read, by parity
    // replicated bookkeeping: identical in every CTA of the cluster
    __shared__ int s_slotC[kMaxWorkingSet], s_slotPhi[kMaxWorkingSet], s_winner[kMaxWorkingSet];
    __shared__ long long s_slotIC[kMaxWorkingSet];
    __shared__ int s_bSlot[kMaxCoopBlocks], s_bCread[kMaxCoopBlocks], s_bSince[kMaxCoopBlocks];
    __shared__ int s_bAssigned[kMaxCoopBlocks], s_bCbb[kMaxCoopBlocks], s_bRead[kMaxCoopBlocks];
    __shared__ int s_bDiv[kMaxCoopBlocks], s_bCursor[kMaxCoopBlocks];
    __shared__ long long s_bICread[kMaxCoopBlocks];
    __shared__ int s_rp, s_Cstar, s_anyRead, s_anyDiv, s_src;

    cg::cluster_group cl = cg::this_cluster();
    const int crank = static_cast<int>(cl.block_rank());
    const int B = cfg.blocks, F = cfg.working_set;
    constexpr int NG = 32 / G;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, wl = tid & 31;
    const int ngroups = (nthr >> 5) * NG;
    const int gw = wl / G;
    const Group<G> g;

    for (;;) {
        if (tid == 0 && crank == 0) s_item = atomicAdd(queue, 1);
        cl.sync();
        const int item = *cl.map_shared_rank(&s_item, 0);
        cl.sync();                                          // read before rank 0 pops again
        if (item >= count) break;
        const CoopItem &ci = items[item];
        const LaunchItem &it = ci.base;
        const InstHeader &h = it.h;
        const int n = h.n, mode = it.mode, delta = it.delta, tl = it.tabu_len, Ib = it.iterations;
        const int pw = profile_words(mode, h.wps, h.ub, h.sum_cap);
        const StateLayout S = state_layout(h.inst_words, n, tl, delta, move_cap, pw, ngroups, mode);
        const SlotLayout SL = slot_layout(n, tl, delta);
        const int pk = PFX ? it.prefix_k : 0;
        const Prefix px{pk > 0 ? gsnap + static_cast<long long>(blockIdx.x) * gsnap_words : nullptr,
                        pk > 0 ? pk : 1, prefix_count(n, pk), prefix_stride(n, pw), pk > 0 ? s_mq + 2 : nullptr};
        const int tcw = (n * delta + 31) / 32;
        stage_instance(sm, it.record, h.inst_words);
        const SInst I = bind_instance(sm, h);
        int *W = sm + S.W;
        int *pos = sm + S.pos;
        int *Wbest = sm + S.Wbest;              // best list since the last read
        int *fsp = sm + S.fsp;
        int *lpp = sm + S.lpp;
        int *stl = sm + S.stl;
        unsigned *tc = reinterpret_cast<unsigned *>(sm + S.tc);
        int *moves = sm + S.moves;
        int *area = sm + S.groups + warp * NG * S.group_words + wl / G;
        const int nslots = n > 3 ? (n - 3) * delta : 0;
        const unsigned dmagic = slot_magic(delta);
        const uint32_t *words = ci.words ? ci.words + static_cast<long long>(crank) * cfg.words_per_block : nullptr;
        if (tid < kTallies) s_tally[tid] = 0;
        if (tid < 32) s_hist[tid] = 0;
        if (tid == 0) {
            s_t0 = global_timer_ns();
            s_eval = 0;
            s_work = 0;
            s_err = 0;
            s_it = 0;
        }
        int err = 0;
        long long my_work = 0;

        // the working set: this CTA starts the slots k = crank (mod B)
        for (int k = crank; k < F; k += B) {
            int32_t *slot = ci.slots + static_cast<long long>(k) * ci.slot_words;
            for (int p = tid; p < n; p += nthr) W[p] = __ldg(ci.init_lists + static_cast<long long>(k) * n + p);
            __syncthreads();
            if (cfg.fbi_every > 0 && k % cfg.fbi_every == cfg.fbi_every - 1) {
                if (warp == 0) fbi_warp<G>(I, mode, W, Wbest, pos, fsp, lpp, area, NG, g, err);
                __syncthreads();
            }
            if (warp == 0) {
                long long w0 = 0;
                const int c0 = decode<G>(I, mode, W, 0, 0, gw == 0, area, NG, g, w0, err);
                if (gw == 0 && g.lane == 0) s_C = c0;
            }
            for (int p = tid; p < n; p += nthr) __stcg(slot + SL.W + p, W[p]);
            for (int x = tid; x < tl; x += nthr) __stcg(slot + SL.stl + x, 0);
            for (int x = tid; x < tcw; x += nthr) __stcg(slot + SL.tc + x, 0);
            __syncthreads();
            if (tid == 0) {
                __stcg(slot + SL.widx, 0);
                __stcg(slot + SL.widx + 1, s_C);    // makespan, for the other CTAs' bookkeeping
            }
            __syncthreads();
        }
        cl.sync();                                          // slots written
        if (tid == 0) {
            s_Cstar = INT_MAX;
            for (int k = 0; k < F; ++k) {
                s_slotC[k] = __ldcg(ci.slots + static_cast<long long>(k) * ci.slot_words + SL.widx + 1);
                s_slotPhi[k] = 0;
                s_slotIC[k] = 0;
                s_Cstar = ::min(s_Cstar, s_slotC[k]);
            }
            s_rp = 0;
            for (int b = 0; b < B; ++b) s_bCursor[b] = 0;
        }

        // Replicated read plan of block b (tid 0): round robin over F.
        auto plan_read = [&](int b) {
            const int k = s_rp;
            s_rp = s_rp + 1 == F ? 0 : s_rp + 1;
            s_slotPhi[k] += 1;
            s_bSlot[b] = k;
            s_bCread[b] = s_slotC[k];
            s_bICread[b] = s_slotIC[k];
            s_bSince[b] = 0;
            s_bRead[b] = 1;
            s_bDiv[b] = s_slotPhi[k] > cfg.phi_max && cfg.phi_steps > 0;
            s_bCbb[b] = s_slotC[k];
        };
        // Eq. 8 budgets of this phase's reads, one thread per block (the
        // inputs -- the slot's makespan and IC at the read, and C* -- are
        // fixed while the reads are planned).  Every thread calls it.
        auto plan_budgets = [&]() {
            if (tid < B && s_bRead[tid])
                s_bAssigned[tid] = cfg.assign_fixed > 0
                    ? cfg.assign_fixed
                    : assigned_iterations(s_bCread[tid], s_Cstar, s_bICread[tid], Ib);
            __syncthreads();
        };
        // This CTA takes the slot its plan names; a diversified read decodes
        // its new list.  Ends with s_C, s_Cbb, Wbest and the tabu state set.
        auto load_read = [&]() {
            const int k = s_bSlot[crank];
            const int32_t *slot = ci.slots + static_cast<long long>(k) * ci.slot_words;
            for (int p = tid; p < n; p += nthr) {
                const int a = __ldcg(slot + SL.W + p);
                W[p] = a;
                pos[a] = p;
            }
            for (int x = tid; x < tl; x += nthr) stl[x] = __ldcg(slot + SL.stl + x);
            for (int x = tid; x < tcw; x += nthr) tc[x] = static_cast<unsigned>(__ldcg(slot + SL.tc + x));
            if (tid == 0) {
                s_widx = __ldcg(slot + SL.widx);
                s_C = s_bCread[crank];
            }
            __syncthreads();
            if (s_bDiv[crank]) {
                if (warp == 0) {
                    const int used = diversify_warp(I, W, pos, fsp, lpp, n, delta, nslots, dmagic, cfg.phi_steps,
                                                    words, cfg.words_per_block, s_bCursor[crank]);
                    long long w0 = 0;
                    const int c0 = decode<G>(I, mode, W, 0, 0, gw == 0, area, NG, g, w0, err);
                    if (gw == 0 && g.lane == 0) {
                        s_C = c0;
                        s_bCursor[crank] += used;
                    }
                }
                __syncthreads();
            }
            for (int p = tid; p < n; p += nthr) Wbest[p] = W[p];
            if (tid == 0) s_Cbb = s_C;
            __syncthreads();
        };
        // Shares the makespans of the diversified reads (tid 0 of every CTA
        // reads them after the barrier) and lowers C* by them.
        auto share_diversified = [&](int par) {
            if (tid == 0) s_pub_div[par] = s_Cbb;
            cl.sync();
            if (tid < B && s_bRead[tid] && s_bDiv[tid])
                s_bCbb[tid] = tid == crank ? s_Cbb : *cl.map_shared_rank(&s_pub_div[par], tid);
            __syncthreads();
            if (tid == 0)
                for (int b = 0; b < B; ++b)
                    if (s_bRead[b] && s_bDiv[b]) s_Cstar = ::min(s_Cstar, s_bCbb[b]);
        };

        // initial reads, in block order
        if (tid == 0) {
            s_anyDiv = 0;
            for (int b = 0; b < B; ++b) {
                plan_read(b);
                s_anyDiv |= s_bDiv[b];
            }
        }
        __syncthreads();
        plan_budgets();
        load_read();
        if (s_anyDiv) share_diversified(1);
        __syncthreads();

        for (;;) {
            if (s_it >= Ib || (it.stop_at_cp && s_Cstar == h.cp)) break;
            const int par = s_it & 1;
            if (tid == 0) s_best = ~0ull;
            const unsigned long long my_key =
                best_admissible_key<G, PFX>(I, mode, W, pos, fsp, lpp, tc, moves, area, n, delta, nslots, dmagic,
                                            move_cap, s_Cstar, 1, 0u, s_mq, &s_eval, my_work, err, px,
                                            TallyRef{s_tally, s_hist});
            const unsigned long long wk = warp_min_u64(my_key);
            if (wl == 0 && wk != ~0ull) atomicMin(&s_best, wk);
            __syncthreads();
            // apply the move, Alg. 3
            if (tid == 0) {
                const unsigned long long kb = s_best;
                int bu = 0, bv = 0;
                s_improved = 0;
                if (kb != ~0ull) {
                    bu = static_cast<int>((kb >> 16) & 0xffff);
                    bv = static_cast<int>(kb & 0xffff);
                    const int a = W[bu], b = W[bv];
                    W[bu] = b;
                    W[bv] = a;
                    pos[b] = bu;
                    pos[a] = bv;
                    s_C = static_cast<int>(kb >> 32);
                }
                const int old = stl[s_widx];
                if (old) tc_put(tc, old & 0xffff, old >> 16, delta, false);
                stl[s_widx] = bu | (bv << 16);
                if (bu | bv) tc_put(tc, bu, bv, delta, true);
                s_widx = s_widx + 1 == tl ? 0 : s_widx + 1;
                if (s_C < s_Cbb) {
                    s_Cbb = s_C;
                    s_improved = 1;
                }
                s_it = s_it + 1;
                s_pub[par] = s_Cbb;
            }
            __syncthreads();
            if (s_improved)
                for (int p = tid; p < n; p += nthr) Wbest[p] = W[p];
            cl.sync();                                      // every block's best published
            if (tid < B) s_bCbb[tid] = tid == crank ? s_Cbb : *cl.map_shared_rank(&s_pub[par], tid);
            __syncthreads();
            // replicated exchange plan: writes in block order, then reads
            if (tid == 0) {
                for (int b = 0; b < B; ++b) {
                    s_bSince[b] += 1;
                    s_bRead[b] = 0;
                    s_Cstar = ::min(s_Cstar, s_bCbb[b]);
                }
                for (int k = 0; k < F; ++k) s_winner[k] = -1;
                s_anyRead = 0;
                s_anyDiv = 0;
                for (int b = 0; b < B; ++b) {
                    const bool improved = s_bCbb[b] < s_bCread[b];
                    if (!(improved || s_bSince[b] > s_bAssigned[b])) continue;
                    s_bRead[b] = 2;                         // exchanges this phase
                    const int k = s_bSlot[b];
                    if (improved && s_bCbb[b] < s_slotC[k]) {
                        s_slotC[k] = s_bCbb[b];
                        s_slotIC[k] = s_bICread[b] + s_bSince[b];
                        s_slotPhi[k] = 0;
                        s_winner[k] = b;
                    } else {
                        s_slotIC[k] += s_bSince[b];
                    }
                }
                if (s_it < Ib)
                    for (int b = 0; b < B; ++b)
                        if (s_bRead[b] == 2) {
                            plan_read(b);
                            s_anyRead = 1;
                            s_anyDiv |= s_bDiv[b];
                        }
                for (int b = 0; b < B; ++b) s_bRead[b] = s_bRead[b] == 1;
            }
            __syncthreads();
            plan_budgets();
            // the last winning write of a slot stores this CTA's best list and
            // tabu state there (the slot this CTA had read; its new read is
            // already planned)
            int wslot = -1;
            for (int k = 0; k < F; ++k)
                if (s_winner[k] == crank) wslot = k;
            if (wslot >= 0) {
                int32_t *slot = ci.slots + static_cast<long long>(wslot) * ci.slot_words;
                for (int p = tid; p < n; p += nthr) __stcg(slot + SL.W + p, Wbest[p]);
                for (int x = tid; x < tl; x += nthr) __stcg(slot + SL.stl + x, stl[x]);
                for (int x = tid; x < tcw; x += nthr) __stcg(slot + SL.tc + x, static_cast<int>(tc[x]));
                if (tid == 0) __stcg(slot + SL.widx, s_widx);
            }
            if (s_anyRead) {
                cl.sync();                                  // writes visible to the readers
                if (s_bRead[crank]) load_read();
                if (s_anyDiv) share_diversified(par);
            }
            __syncthreads();
        }
        cl.sync();                                          // last writes visible
        // the result: the best slot (lowest index), unless a block's best
        // since its read is strictly better (lowest block)
        if (tid == 0) {
            int cb = s_slotC[0], src = 0;
            for (int k = 1; k < F; ++k)
                if (s_slotC[k] < cb) {
                    cb = s_slotC[k];
                    src = k;
                }
            for (int b = 0; b < B; ++b)
                if (s_bCbb[b] < cb) {
                    cb = s_bCbb[b];
                    src = F + b;
                }
            s_src = src;
            s_Cstar = cb;
        }
        __syncthreads();
        const int src = s_src;
        const bool owner = src < F ? crank == 0 : crank == src - F;
        int32_t *out = it.out;
        if (owner) {
            if (src < F) {
                const int32_t *slot = ci.slots + static_cast<long long>(src) * ci.slot_words;
                for (int p = tid; p < n; p += nthr) Wbest[p] = __ldcg(slot + SL.W + p);
                __syncthreads();
            }
            if (warp == 0) {
                long long w1 = 0;
                int e1 = 0;
                const int cb = decode<G>(I, mode, Wbest, 0, 0, gw == 0, area, NG, g, w1, e1, out + n);
                if (gw == 0 && g.lane == 0) {
                    out[2 * n + kOutCmax] = cb;
                    if (e1 || cb != s_Cstar) atomicOr(&s_err, 2);
                }
            }
            for (int p = tid; p < n; p += nthr) out[p] = Wbest[p];
        }
        const long long ws = warp_sum_i64(g.lane == 0 ? my_work : 0);
        if (wl == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&s_work), static_cast<unsigned long long>(ws));
        if (err) atomicOr(&s_err, err);
        __syncthreads();
        cl.sync();                                          // counters final in every CTA
        if (crank == 0 && tid == 0) {
            long long ev = s_eval, wsum = s_work;
            int e = s_err;
            long long ta[kTallies];
            for (int x = 0; x < kTallies; ++x) ta[x] = s_tally[x];
            for (int r = 1; r < B; ++r) {
                ev += *cl.map_shared_rank(&s_eval, r);
                wsum += *cl.map_shared_rank(&s_work, r);
                e |= *cl.map_shared_rank(&s_err, r);
                for (int x = 0; x < kTallies; ++x) ta[x] += *cl.map_shared_rank(&s_tally[x], r);
            }
            int32_t *st = out + 2 * n;
            st[kOutEvalLo] = static_cast<int32_t>(ev & 0xffffffffll);
            st[kOutEvalHi] = static_cast<int32_t>(ev >> 32);
            st[kOutWorkLo] = static_cast<int32_t>(wsum & 0xffffffffll);
            st[kOutWorkHi] = static_cast<int32_t>(wsum >> 32);
            st[kOutIters] = s_it * B;
            st[kOutIters0] = 0;
            ta[kTallySteps] += wsum;                      // loop steps performed
            for (int x = 0; x < kTallies; ++x) {
                st[kOutPlacedLo + 2 * x] = static_cast<int32_t>(ta[x] & 0xffffffffll);
                st[kOutPlacedLo + 2 * x + 1] = static_cast<int32_t>(ta[x] >> 32);
            }
            st[kOutMode] = mode;
            st[kOutStatus] = e ? RCPSP_E_DEVICE : 0;
            const unsigned long long t1 = global_timer_ns();
            st[kOutT0Lo] = static_cast<int32_t>(s_t0 & 0xffffffffull);
            st[kOutT0Hi] = static_cast<int32_t>(s_t0 >> 32);
            st[kOutT1Lo] = static_cast<int32_t>(t1 & 0xffffffffull);
            st[kOutT1Hi] = static_cast<int32_t>(t1 >> 32);
        }
        __syncthreads();
    }
}

template <int G, bool PFX>
cudaError_t coop_attributes_g(size_t smem, int csize) {
    cudaError_t e = cudaFuncSetAttribute(coop_kernel<G, PFX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e == cudaSuccess && csize > 8)
        e = cudaFuncSetAttribute(coop_kernel<G, PFX>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

cudaLaunchConfig_t coop_config(int blocks, int threads, size_t smem, cudaStream_t st, int csize,
                               cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int G, bool PFX>
cudaError_t coop_occupancy_g(int threads, size_t smem, int csize, int *clusters) {
    cudaError_t e = coop_attributes_g<G, PFX>(smem, csize);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = coop_config(csize, threads, smem, nullptr, csize, attr);
    return cudaOccupancyMaxActiveClusters(clusters, coop_kernel<G, PFX>, &cfg);
}

template <int G, bool PFX>
cudaError_t launch_coop_g(const CoopItem *items, int count, int *queue, int move_cap, const CoopConfig &cc,
                          int blocks, int threads, size_t smem, cudaStream_t st, int *gsnap, int gsnap_words) {
    cudaError_t e = coop_attributes_g<G, PFX>(smem, cc.blocks);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = coop_config(blocks, threads, smem, st, cc.blocks, attr);
    return cudaLaunchKernelEx(&cfg, coop_kernel<G, PFX>, items, count, queue, move_cap, cc, gsnap, gsnap_words);
}

// The entry points of one prefix-reuse variant for a set of group sizes.
#define RCPSP_COOP_ENTRY_POINTS(NAME, PFX_, G0, G1, G2)                                                        \
    cudaError_t coop_occupancy_##NAME(int group_size, int threads, size_t smem, int csize, int *clusters) {   \
        switch (group_size) {                                                                                  \
            case G0: return coop_occupancy_g<G0, PFX_>(threads, smem, csize, clusters);                         \
            case G1: return coop_occupancy_g<G1, PFX_>(threads, smem, csize, clusters);                         \
            case G2: return coop_occupancy_g<G2, PFX_>(threads, smem, csize, clusters);                         \
            default: return cudaErrorInvalidValue;                                                             \
        }                                                                                                      \
    }                                                                                                          \
    cudaError_t launch_coop_##NAME(int group_size, const CoopItem *items, int count, int *queue, int move_cap, \
                                   const CoopConfig &cfg, int blocks, int threads, size_t smem,                \
                                   cudaStream_t st, int *gsnap, int gsnap_words) {                             \
        switch (group_size) {                                                                                  \
            case G0: return launch_coop_g<G0, PFX_>(items, count, queue, move_cap, cfg, blocks, threads, smem, \
                                                     st, gsnap, gsnap_words);                                  \
            case G1: return launch_coop_g<G1, PFX_>(items, count, queue, move_cap, cfg, blocks, threads, smem, \
                                                     st, gsnap, gsnap_words);                                  \
            case G2: return launch_coop_g<G2, PFX_>(items, count, queue, move_cap, cfg, blocks, threads, smem, \
                                                     st, gsnap, gsnap_words);                                  \
            default: return cudaErrorInvalidValue;                                                             \
        }                                                                                                      \
    }

}  // namespace

// Per-variant entry points: coop_kernel.cu (G 1, 2, 4), coop_kernel_wide.cu
// (G 8, 16, 32), coop_kernel_pfx.cu and coop_kernel_pfx_wide.cu (the same
// with prefix reuse).
#define RCPSP_COOP_DECLARE(NAME)                                                                                 \
    cudaError_t coop_occupancy_##NAME(int group_size, int threads, size_t smem, int csize, int *clusters);     \
    cudaError_t launch_coop_##NAME(int group_size, const CoopItem *items, int count, int *queue, int move_cap, \
                                   const CoopConfig &cfg, int blocks, int threads, size_t smem,                \
                                   cudaStream_t st, int *gsnap, int gsnap_words);
RCPSP_COOP_DECLARE(narrow)
RCPSP_COOP_DECLARE(wide)
RCPSP_COOP_DECLARE(pfx_narrow)
RCPSP_COOP_DECLARE(pfx_wide)

}  // namespace rcpsp
