// Co-operative search kernels for G = 1, 2, 4 lanes per decode, and the
// dispatch of every variant (the others compile in coop_kernel_wide.cu,
// coop_kernel_pfx.cu and coop_kernel_pfx_wide.cu).
#include "coop_kernel.cuh"

namespace rcpsp {

RCPSP_COOP_ENTRY_POINTS(narrow, false, 1, 2, 4)

cudaError_t coop_occupancy(int group_size, int threads, size_t smem, int csize, int *clusters, bool prefix) {
    if (prefix)
        return group_size <= 4 ? coop_occupancy_pfx_narrow(group_size, threads, smem, csize, clusters)
                               : coop_occupancy_pfx_wide(group_size, threads, smem, csize, clusters);
    return group_size <= 4 ? coop_occupancy_narrow(group_size, threads, smem, csize, clusters)
                           : coop_occupancy_wide(group_size, threads, smem, csize, clusters);
}

cudaError_t launch_coop(int group_size, const CoopItem *items, int count, int *queue, int move_cap,
                        const CoopConfig &cfg, int blocks, int threads, size_t smem, cudaStream_t st, bool prefix,
                        int *gsnap, int gsnap_words) {
    if (prefix)
        return group_size <= 4 ? launch_coop_pfx_narrow(group_size, items, count, queue, move_cap, cfg, blocks,
                                                        threads, smem, st, gsnap, gsnap_words)
                               : launch_coop_pfx_wide(group_size, items, count, queue, move_cap, cfg, blocks,
                                                      threads, smem, st, gsnap, gsnap_words);
    return group_size <= 4 ? launch_coop_narrow(group_size, items, count, queue, move_cap, cfg, blocks, threads,
                                                smem, st, nullptr, 0)
                           : launch_coop_wide(group_size, items, count, queue, move_cap, cfg, blocks, threads, smem,
                                              st, nullptr, 0);
}

}  // namespace rcpsp
