// Co-operative search kernels for G = 1, 2, 4 lanes per decode, and the
// dispatch of every G (the wider ones compile in coop_kernel_wide.cu).
#include "coop_kernel.cuh"

namespace rcpsp {

cudaError_t coop_occupancy_narrow(int group_size, int threads, size_t smem, int csize, int *clusters) {
    switch (group_size) {
        case 1: return coop_occupancy_g<1>(threads, smem, csize, clusters);
        case 2: return coop_occupancy_g<2>(threads, smem, csize, clusters);
        case 4: return coop_occupancy_g<4>(threads, smem, csize, clusters);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_coop_narrow(int group_size, const CoopItem *items, int count, int *queue, int move_cap,
                               const CoopConfig &cfg, int blocks, int threads, size_t smem, cudaStream_t st) {
    switch (group_size) {
        case 1: return launch_coop_g<1>(items, count, queue, move_cap, cfg, blocks, threads, smem, st);
        case 2: return launch_coop_g<2>(items, count, queue, move_cap, cfg, blocks, threads, smem, st);
        case 4: return launch_coop_g<4>(items, count, queue, move_cap, cfg, blocks, threads, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t coop_occupancy(int group_size, int threads, size_t smem, int csize, int *clusters) {
    return group_size <= 4 ? coop_occupancy_narrow(group_size, threads, smem, csize, clusters)
                           : coop_occupancy_wide(group_size, threads, smem, csize, clusters);
}

cudaError_t launch_coop(int group_size, const CoopItem *items, int count, int *queue, int move_cap,
                        const CoopConfig &cfg, int blocks, int threads, size_t smem, cudaStream_t st) {
    return group_size <= 4
        ? launch_coop_narrow(group_size, items, count, queue, move_cap, cfg, blocks, threads, smem, st)
        : launch_coop_wide(group_size, items, count, queue, move_cap, cfg, blocks, threads, smem, st);
}

}  // namespace rcpsp
