// Fixed device scratch for rcpsp_tabu_search_noalloc.
//
// The search kernel needs two pieces of global memory besides its inputs and
// outputs: the launch plan (one LaunchItem per instance) and the work-queue
// counter.  rcpsp_tabu_search takes them from the context's allocator; the
// no-allocation entry point takes them from this file-scope array instead,
// which every GPU that loads the library holds until the process exits.
//
// Layout: bytes [0, 4) hold the queue counter; the plan starts at byte 256.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"
#include "rcpsp_internal.h"

namespace rcpsp {
namespace {

constexpr size_t kScratchBytes = size_t(1) << 20;   // 1 MiB
constexpr size_t kPlanOffset = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

}  // namespace

int noalloc_max_items() { return static_cast<int>((kScratchBytes - kPlanOffset) / sizeof(LaunchItem)); }

// Device address of the scratch on `device`.  The first call for a device
// makes that device current and asks the runtime for the symbol's address
// (the host-side name of the array is not a device address); later calls
// return the cached address.
cudaError_t noalloc_scratch(int device, int **queue, LaunchItem **plan) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != device) cudaSetDevice(cur);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    }
    unsigned char *base = static_cast<unsigned char *>(g_addr[device]);
    *queue = reinterpret_cast<int *>(base);
    *plan = reinterpret_cast<LaunchItem *>(base + kPlanOffset);
    return cudaSuccess;
}

}  // namespace rcpsp
