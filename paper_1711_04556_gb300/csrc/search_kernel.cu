// sm_103a kernels of the tabu search for the RCPSP (Bukata, Sucha, Hanzalek):
// the search kernel for CTAs of up to 384 threads (two CTAs of 384 threads
// per SM leave each thread 85 registers, so the decode loop runs without
// spills at 80), the dispatch by CTA size, and the decoding of caller-given
// lists.  The kernel itself is in search_kernel.cuh.
#include "kernels.h"
#include "search_kernel.cuh"

namespace rcpsp {
namespace {

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
    const StateLayout S = state_layout(h.inst_words, n, 0, 0, ngroups * align4(n), pw, ngroups, mode);
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

cudaError_t prepare_search(int group_size, size_t smem) {
    cudaError_t e = prepare_search_nt<kSearchNarrowThreads, 2>(group_size, smem);
    if (e == cudaSuccess) e = prepare_search_wide(group_size, smem);
    return e == cudaSuccess ? prepare_search_solo(group_size, smem) : e;
}

cudaError_t search_occupancy(int group_size, int threads, size_t smem, int csize, int *units, bool prefix,
                             bool solo) {
    if (solo) return search_occupancy_solo(group_size, threads, smem, csize, units, prefix);
    if (threads > kSearchNarrowThreads)
        return search_occupancy_wide(group_size, threads, smem, csize, units, prefix);
    return search_occupancy_nt<kSearchNarrowThreads, 2>(group_size, threads, smem, csize, units, prefix);
}

cudaError_t launch_search(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                          int blocks, int threads, size_t smem, cudaStream_t st, int csize, bool prefix,
                          int *gsnap, int gsnap_words, SliceSched sl, bool solo) {
    if (solo)
        return launch_search_solo(group_size, items, count, queue, move_cap, blocks, threads, smem, st, csize,
                                  prefix, gsnap, gsnap_words, sl);
    if (threads > kSearchNarrowThreads)
        return launch_search_wide(group_size, items, count, queue, move_cap, blocks, threads, smem, st, csize,
                                  prefix, gsnap, gsnap_words, sl);
    return launch_search_nt<kSearchNarrowThreads, 2>(group_size, items, count, queue, move_cap, blocks, threads,
                                                     smem, st, csize, prefix, gsnap, gsnap_words, sl);
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
