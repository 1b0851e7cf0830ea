// The tabu search kernel for CTAs of 385 to 512 threads (13 to 16 warps):
// two CTAs of 512 threads per SM leave each thread 64 registers.  Compiled
// apart from search_kernel.cu so that the two compile in parallel.
#include "search_kernel.cuh"

namespace rcpsp {

constexpr int kWideThreads = kSearchMaxWarps * 32;

cudaError_t prepare_search_wide(int group_size, size_t smem) {
    return prepare_search_nt<kWideThreads, 2>(group_size, smem);
}

cudaError_t search_occupancy_wide(int group_size, int threads, size_t smem, int csize, int *units, bool prefix) {
    return search_occupancy_nt<kWideThreads, 2>(group_size, threads, smem, csize, units, prefix);
}

cudaError_t launch_search_wide(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                               int blocks, int threads, size_t smem, cudaStream_t st, int csize, bool prefix,
                               int *gsnap, int gsnap_words, SliceSched sl) {
    return launch_search_nt<kWideThreads, 2>(group_size, items, count, queue, move_cap, blocks, threads, smem, st,
                                          csize, prefix, gsnap, gsnap_words, sl);
}

}  // namespace rcpsp
