// Co-operative search kernels for G = 8, 16, 32 lanes per decode.
#include "coop_kernel.cuh"

namespace rcpsp {

cudaError_t coop_occupancy_wide(int group_size, int threads, size_t smem, int csize, int *clusters) {
    switch (group_size) {
        case 8: return coop_occupancy_g<8>(threads, smem, csize, clusters);
        case 16: return coop_occupancy_g<16>(threads, smem, csize, clusters);
        case 32: return coop_occupancy_g<32>(threads, smem, csize, clusters);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_coop_wide(int group_size, const CoopItem *items, int count, int *queue, int move_cap,
                             const CoopConfig &cfg, int blocks, int threads, size_t smem, cudaStream_t st) {
    switch (group_size) {
        case 8: return launch_coop_g<8>(items, count, queue, move_cap, cfg, blocks, threads, smem, st);
        case 16: return launch_coop_g<16>(items, count, queue, move_cap, cfg, blocks, threads, smem, st);
        case 32: return launch_coop_g<32>(items, count, queue, move_cap, cfg, blocks, threads, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcpsp
