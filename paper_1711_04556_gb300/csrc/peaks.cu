// Measured ceilings for the roofline of the integer search path
// (rcpsp_measure_peaks): the 32-bit integer ALU rate and the shared-memory
// load bandwidth of the GPU, each from a kernel that does nothing else.
//
//  * int_alu_kernel: every thread runs 8 independent chains of
//    a = (a ^ K) + b -- one logical and one add per link, which no single
//    instruction fuses -- over registers only.  Ops = 16 per thread per
//    loop iteration.
//  * smem_load_kernel: every thread loads 16 bytes per access from a 32 KiB
//    shared array, consecutive lanes at consecutive 16-byte words (no bank
//    conflicts), 8 accesses per loop iteration at offsets that change every
//    iteration, folded into an xor.
//
// Both are timed with CUDA events around the launch; each grid is one wave
// (the blocks an SM holds at once, from the occupancy calculator, times the
// SMs).
#include <cuda_runtime.h>

#include "../../include/rcpsp.h"

namespace rcpsp {
namespace {

constexpr int kIntThreads = 256;
constexpr int kSmemThreads = 256;
constexpr int kSmemWords = 2048;          // uint4 words: 32 KiB

__global__ void __launch_bounds__(kIntThreads) int_alu_kernel(unsigned *sink, int iters, unsigned seed) {
    unsigned a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed ^ (threadIdx.x * 0x9e3779b9u + c * 0x85ebca6bu + blockIdx.x);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = (a[c] ^ 0x5bd1e995u) + a[(c + 1) & 7];
    }
    unsigned x = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) x ^= a[c];
    if (x == seed) sink[blockIdx.x] = x;      // keeps the chains live
}

__global__ void __launch_bounds__(kSmemThreads) smem_load_kernel(unsigned *sink, int iters, unsigned seed) {
    __shared__ uint4 buf[kSmemWords];
    for (int x = threadIdx.x; x < kSmemWords; x += blockDim.x)
        buf[x] = make_uint4(seed + x, seed ^ x, seed * x, ~x);
    __syncthreads();
    unsigned acc0 = 0, acc1 = 0;
    for (int i = 0; i < iters; ++i) {
        const int base = threadIdx.x + (i & 7) * kSmemThreads;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint4 v = buf[(base + k * 32 * 8) & (kSmemWords - 1)];
            acc0 ^= v.x ^ v.y;
            acc1 ^= v.z ^ v.w;
        }
    }
    if ((acc0 ^ acc1) == seed) sink[blockIdx.x] = acc0;
}

}  // namespace
}  // namespace rcpsp

int rcpsp_measure_peaks(int device, rcpsp_peaks *out) {
    using namespace rcpsp;
    if (!out) return RCPSP_E_INVALID_ARG;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return RCPSP_E_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return RCPSP_E_INVALID_ARG;
    int rc = RCPSP_OK;
    cudaDeviceProp prop{};
    unsigned *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    const int sms = (cudaGetDeviceProperties(&prop, device) == cudaSuccess) ? prop.multiProcessorCount : 0;
    int int_per_sm = 0, smem_per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&int_per_sm, int_alu_kernel, kIntThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&smem_per_sm, smem_load_kernel, kSmemThreads, 0) != cudaSuccess)
        int_per_sm = smem_per_sm = 0;
    const int int_blocks = sms * int_per_sm, smem_blocks = sms * smem_per_sm;
    const int int_iters = 1 << 15, smem_iters = 1 << 13;
    if (sms <= 0 || int_blocks <= 0 || smem_blocks <= 0 ||
        cudaMalloc(&sink, sizeof(unsigned) * (int_blocks + smem_blocks)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        rc = RCPSP_E_CUDA;
    }
    double best_int = 0, best_smem = 0, int_ms = 0, smem_ms = 0;
    for (int rep = 0; rc == RCPSP_OK && rep < 5; ++rep) {
        float ms = 0;
        cudaEventRecord(e0, st);
        int_alu_kernel<<<int_blocks, kIntThreads, 0, st>>>(sink, int_iters, 0x1234567u + rep);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = RCPSP_E_CUDA;
            break;
        }
        const double ops = 16.0 * int_iters * static_cast<double>(int_blocks) * kIntThreads;
        if (ms > 0 && ops / (ms * 1e-3) > best_int) {
            best_int = ops / (ms * 1e-3);
            int_ms = ms;
        }
        cudaEventRecord(e0, st);
        smem_load_kernel<<<smem_blocks, kSmemThreads, 0, st>>>(sink + int_blocks, smem_iters, 0x7654321u + rep);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = RCPSP_E_CUDA;
            break;
        }
        const double bytes = 16.0 * 8 * smem_iters * static_cast<double>(smem_blocks) * kSmemThreads;
        if (ms > 0 && bytes / (ms * 1e-3) > best_smem) {
            best_smem = bytes / (ms * 1e-3);
            smem_ms = ms;
        }
    }
    if (rc == RCPSP_OK && cudaGetLastError() != cudaSuccess) rc = RCPSP_E_CUDA;
    if (rc == RCPSP_OK) {
        out->int32_ops_per_s = best_int;
        out->smem_bytes_per_s = best_smem;
        out->int32_ms = int_ms;
        out->smem_ms = smem_ms;
        out->sms = sms;
    }
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaSetDevice(cur);
    return rc;
}
