// cvrpsd_int_rate: the device's measured rate of 32-bit integer min/max
// instructions, the operation of the window minimum of Eq. 3 (one min per
// candidate predecessor). It is the denominator of the integer-ALU roofline
// the benchmark reports; it is not a step of the Split.
//
// Every thread runs eight independent chains; each chain alternates min and
// max against four different (lo, hi) pairs, so no instruction repeats an
// earlier one with the same operands and none can be folded away. The
// instructions are written as inline PTX, one per statement. Loop overhead
// (counter, compare, branch) is three instructions per 64 min/max.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cvrpsd.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kOpsPerIter = kChains * 8;   // 4 (min, max) pairs per chain

__device__ __forceinline__ void mn(int &x, int y) { asm volatile("min.s32 %0, %0, %1;" : "+r"(x) : "r"(y)); }
__device__ __forceinline__ void mx(int &x, int y) { asm volatile("max.s32 %0, %0, %1;" : "+r"(x) : "r"(y)); }

__global__ void __launch_bounds__(kThreads) int_rate_kernel(int iters, int base, int *sink)
{
    const int t = (int)threadIdx.x;
    int lo0 = base + t, lo1 = lo0 + 3, lo2 = lo0 + 5, lo3 = lo0 + 7;
    int hi0 = lo0 + 1000, hi1 = hi0 - 2, hi2 = hi0 - 4, hi3 = hi0 - 6;
    int x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = base * j + t;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            mn(x[j], hi0); mx(x[j], lo0);
            mn(x[j], hi1); mx(x[j], lo1);
            mn(x[j], hi2); mx(x[j], lo2);
            mn(x[j], hi3); mx(x[j], lo3);
        }
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s ^= x[j];
    if (s == 0x7fffffff) *sink = s;   // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int cvrpsd_int_rate(int32_t device, int32_t iters, double *ops_per_s, double *ms, void *stream_ptr)
{
    if (!ops_per_s || iters < 1) return CVRPSD_ERR_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    int sms = 0, per_sm = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_rate_kernel, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return CVRPSD_ERR_CUDA;
    }
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    int *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CVRPSD_OK;
    float t = 0.0f;
    if (cudaMalloc(&sink, sizeof(int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = CVRPSD_ERR_CUDA;
    } else {
        int_rate_kernel<<<grid, kThreads, 0, stream>>>(iters / 8 > 0 ? iters / 8 : 1, 1, sink);   // warm-up
        cudaEventRecord(e0, stream);
        int_rate_kernel<<<grid, kThreads, 0, stream>>>(iters, 1, sink);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || t <= 0.0f)
            rc = CVRPSD_ERR_CUDA;
    }
    if (rc == CVRPSD_OK) {
        const double ops = (double)grid * kThreads * (double)iters * kOpsPerIter;
        *ops_per_s = ops / (t * 1e-3);
        if (ms) *ms = t;
    }
    cudaGetLastError();
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}
