// Launchers of the sm_103a kernels (search_kernel.cu).
#pragma once

#include <cuda_runtime.h>

#include "rcpsp_internal.h"

namespace rcpsp {

// Raises the dynamic shared-memory limit of the search kernel for group size G.
cudaError_t prepare_search(int group_size, size_t smem);
// Resident units of the search kernel at this shape: CTAs per SM when
// csize == 1, clusters on the whole GPU when csize > 1.
// `prefix`: the kernel variant with prefix reuse (items with prefix_k > 0).
// `solo`: the build for one CTA per SM (up to 512 threads, up to 128
// registers a thread), for launches whose shared memory allows no second.
cudaError_t search_occupancy(int group_size, int threads, size_t smem, int csize, int *units,
                             bool prefix = false, bool solo = false);
// blocks = CTAs (a multiple of csize); csize > 1 launches clusters of csize CTAs.
// With prefix reuse, CTA b keeps its decoder states at gsnap + b * gsnap_words.
// sl.nslices > 1: a sliced launch (SliceSched; sl.sync zeroed beforehand).
cudaError_t launch_search(int group_size, const LaunchItem *items, int count, int *queue, int move_cap,
                          int blocks, int threads, size_t smem, cudaStream_t st, int csize, bool prefix = false,
                          int *gsnap = nullptr, int gsnap_words = 0, SliceSched sl = SliceSched{1, nullptr, nullptr},
                          bool solo = false);
cudaError_t launch_evaluate(int group_size, const LaunchItem &item, const int32_t *lists, int count,
                            int32_t *start, int32_t *cmax, long long *work, int *err, int blocks, int threads,
                            size_t smem, cudaStream_t st);

// Co-operative search (coop_kernel.cu): clusters of cfg.blocks CTAs, one
// instance per cluster.  coop_occupancy gives the resident clusters on the
// whole GPU; blocks = CTAs of the launch, a multiple of cfg.blocks.  With
// prefix reuse CTA b keeps its decoder states at gsnap + b * gsnap_words.
cudaError_t coop_occupancy(int group_size, int threads, size_t smem, int csize, int *clusters, bool prefix = false);
cudaError_t launch_coop(int group_size, const CoopItem *items, int count, int *queue, int move_cap,
                        const CoopConfig &cfg, int blocks, int threads, size_t smem, cudaStream_t st,
                        bool prefix = false, int *gsnap = nullptr, int gsnap_words = 0);

// Fixed scratch of the no-allocation search (noalloc_scratch.cu): largest
// plan it holds, and its device address on `device` (queue counter, plan).
int noalloc_max_items();
cudaError_t noalloc_scratch(int device, int **queue, LaunchItem **plan);

}  // namespace rcpsp
