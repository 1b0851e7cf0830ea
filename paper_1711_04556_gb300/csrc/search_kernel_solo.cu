// The tabu search kernel for launches whose shared memory holds one CTA per
// SM (up to 512 threads): a CTA then has the SM's registers to itself, so
// this build may take up to 128 a thread where the two-CTA builds stop at
// 80 (384 threads) or 64 (512).  Compiled apart so that the builds compile
// in parallel.
#include "search_kernel.cuh"

namespace rcpsp {

constexpr int kSoloThreads = kSearchMaxWarps * 32;

cudaError_t prepare_search_solo(int group_size, size_t smem) {
    return prepare_search_nt<kSoloThreads, 1>(group_size, smem);
}

cudaError_t search_occupancy_solo(int group_size, int threads, size_t smem, int csize, int *units, bool prefix) {
    return search_occupancy_nt<kSoloThreads, 1>(group_size, threads, smem, csize, units, prefix);
}

cudaError_t launch_search_solo(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                               int blocks, int threads, size_t smem, cudaStream_t st, int csize, bool prefix,
                               int *gsnap, int gsnap_words, SliceSched sl) {
    return launch_search_nt<kSoloThreads, 1>(group_size, items, count, queue, move_cap, blocks, threads, smem, st,
                                          csize, prefix, gsnap, gsnap_words, sl);
}

}  // namespace rcpsp
