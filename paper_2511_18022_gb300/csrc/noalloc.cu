// cvrpsd_split_eval_noalloc: the Split of cvrpsd_split_eval for callers that
// cannot allocate device memory at call time.
//
// Who needs it: programs that give the whole device memory to their own pool
// or arena at start-up (so a library cudaMalloc would fail or fragment it),
// and latency-sensitive loops where a cudaMalloc / cudaFree could block on
// the device or fail under memory pressure. The regular entry point needs a
// context whose scratch (accumulators, tour table, list of set-aside
// scenarios) is allocated on first use; this one keeps that scratch in one
// file-scope device array instead, so it allocates nothing.
//
// The array is reserved in every device that loads the library, for as long
// as the library stays loaded. Host code must not pass the array's name to a
// kernel: on the host it is only a stand-in symbol, not a device address.
// The device address is looked up once per device with cudaGetSymbolAddress
// (on the device that is current at the first call there).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "../../include/cvrpsd.h"
#include "deque2.h"
#include "kernels.h"
#include "trace.h"
#include "tour_table.h"

namespace {

using namespace cvrpsd;

constexpr long long kMaxS = CVRPSD_NOALLOC_MAX_S;
constexpr size_t kAccBytes = 256;                                   // ACC_WORDS int64, padded
constexpr size_t kTabBytes = ((size_t)CVRPSD_MAX_N * sizeof(TourStep) + 255) / 256 * 256;
constexpr size_t kListBytes = (size_t)kMaxS * sizeof(int32_t);
constexpr size_t kScratchBytes = kAccBytes + kTabBytes + kListBytes;

// Scratch shared by every call on a device: accumulators, then the tour
// table, then the set-aside list. It keeps the last call's contents.
static __device__ __align__(256) unsigned char g_split_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    std::once_flag once;
    cudaError_t status = cudaErrorInitializationError;
    unsigned char *scratch = nullptr;   // device address of g_split_scratch
    int max_smem = 0;
    int sm_count = 0;
};
DeviceSetup g_setup[kMaxDevices];

std::mutex g_host_mutex;                // guards the host staging table below
TourStep g_host_tab[CVRPSD_MAX_N];

typedef CUresult (*GetRangeFn)(CUdeviceptr *, size_t *, CUdeviceptr);

GetRangeFn range_fn()
{
    static GetRangeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<GetRangeFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// [ptr, ptr + bytes) must be device memory of `device` inside one allocation.
bool device_buffer_ok(const void *ptr, unsigned long long bytes, int device)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
    if (a.type == cudaMemoryTypeDevice && a.device != device) return false;
    if (GetRangeFn fn = range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)ptr) == CUDA_SUCCESS &&
            (unsigned long long)(uintptr_t)ptr + bytes > (unsigned long long)base + size)
            return false;
    }
    return true;
}

}  // namespace

extern "C" int cvrpsd_split_eval_noalloc(const int32_t *tour, int32_t n, const int32_t *dist, const void *demand,
                                         int32_t demand_dtype, int64_t S, int64_t ld, int32_t Q, int32_t L,
                                         int32_t *out_cost, int64_t *out_sum, int64_t *out_infeasible,
                                         double *out_mean, void *stream_ptr)
{
    CVRPSD_TRACE("cvrpsd_split_eval_noalloc");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    if (!tour || !dist || n < 1 || n > CVRPSD_MAX_N) return CVRPSD_ERR_ARG;
    if (demand_dtype != CVRPSD_I16 && demand_dtype != CVRPSD_I32) return CVRPSD_ERR_DTYPE;
    if (S < 0 || ld < S || ld < 1 || Q < 0 || L < 1) return CVRPSD_ERR_ARG;
    if (S > kMaxS) return CVRPSD_ERR_UNSUPPORTED;   // the set-aside list holds kMaxS scenarios
    if ((unsigned long long)ld * demand_dtype > 0xFFFFFFFFull) return CVRPSD_ERR_UNSUPPORTED;
    if (L > n) L = n;
    // Each call stages its tour table through one process-wide host buffer.
    // Recorded into a graph, that copy would read the buffer at replay time,
    // after later calls have overwritten it, so a capturing stream is refused.
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &capturing) != cudaSuccess) {
        cudaGetLastError();
        return CVRPSD_ERR_CUDA;
    }
    if (capturing != cudaStreamCaptureStatusNone) return CVRPSD_ERR_UNSUPPORTED;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
        cudaGetLastError();
        return CVRPSD_ERR_CUDA;
    }
    DeviceSetup &ds = g_setup[device];
    std::call_once(ds.once, [&ds, device] {
        void *addr = nullptr;
        ds.status = cudaGetSymbolAddress(&addr, g_split_scratch);
        if (ds.status == cudaSuccess) ds.status = cudaDeviceGetAttribute(&ds.max_smem,
                                                                         cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        if (ds.status == cudaSuccess) ds.status = cudaDeviceGetAttribute(&ds.sm_count,
                                                                         cudaDevAttrMultiProcessorCount, device);
        if (ds.status == cudaSuccess) ds.scratch = static_cast<unsigned char *>(addr);
        else cudaGetLastError();
    });
    if (ds.status != cudaSuccess || !ds.scratch) return CVRPSD_ERR_CUDA;
    if (S > 0) {
        if (!device_buffer_ok(demand, ((unsigned long long)(n - 1) * ld + S) * demand_dtype, device))
            return CVRPSD_ERR_ARG;
        if (out_cost && !device_buffer_ok(out_cost, (unsigned long long)S * 4, device)) return CVRPSD_ERR_ARG;
    }

    unsigned long long *acc = reinterpret_cast<unsigned long long *>(ds.scratch);
    TourStep *tab = reinterpret_cast<TourStep *>(ds.scratch + kAccBytes);
    int32_t *list = reinterpret_cast<int32_t *>(ds.scratch + kAccBytes + kTabBytes);

    // The accumulators keep the previous call's values: start this call at zero.
    if (cudaMemsetAsync(acc, 0, ACC_WORDS * sizeof(unsigned long long), stream) != cudaSuccess) {
        cudaGetLastError();
        return CVRPSD_ERR_CUDA;
    }
    // The shared host table is read by the upload and, for the parameter-table
    // walk, by the launch (its parameters are copied when it is enqueued):
    // both happen under the lock.
    {
        std::lock_guard<std::mutex> lock(g_host_mutex);
        int32_t g0 = 0;
        char msg[256];
        const int rc = fill_tour_table(tour, n, dist, Q, g_host_tab, &g0, msg, sizeof(msg));
        if (rc) return rc;
        // From pageable host memory: the copy has read the table when this returns.
        if (cudaMemcpyAsync(tab, g_host_tab, (size_t)n * sizeof(TourStep), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess) {
            cudaGetLastError();
            return CVRPSD_ERR_CUDA;
        }


        if (S > 0) {
            SplitParams p{};
            p.tab = tab;
            p.demand = demand;
            p.ld = ld;
            p.S = S;
            p.n = n;
            p.Q = Q;
            p.L = L;
            p.g0 = g0;
            p.K = key_scale(n);
            p.out_cost = out_cost;
            p.acc = acc;
            p.ovf_list = list;
            // The parameter-table walk where it applies (no device memory beyond
            // the fixed scratch: its table travels in the launch parameters),
            // else the global-table walk.
            DequeShape shape{128, 1, 16};
            cudaError_t e = cudaSuccess;
            if (deque2_supported(p, demand_dtype)) {
                e = launch_split_deque2(p, g_host_tab, demand_dtype, shape, 0, nullptr, stream);
            } else {
                while (split_deque_smem(p, shape) > (size_t)ds.max_smem) {
                    if (shape.threads > 64) shape.threads >>= 1;
                    else return CVRPSD_ERR_UNSUPPORTED;
                }
                e = launch_split_deque(p, demand_dtype, shape, stream);
            }
            if (e != cudaSuccess ||
                launch_split_warp(p, demand_dtype, list, acc + ACC_OVERFLOW, 2 * ds.sm_count, ds.max_smem, stream) !=
                    cudaSuccess) {
                cudaGetLastError();
                return CVRPSD_ERR_CUDA;
            }
        }
    }
    if (!out_sum && !out_infeasible && !out_mean) return CVRPSD_OK;

    unsigned long long h[ACC_WORDS] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return CVRPSD_ERR_CUDA;
    }
    if (h[ACC_STATUS] & (ST_NEGATIVE_DEMAND | ST_INDEX)) return CVRPSD_ERR_DEVICE_STATUS;
    const long long sum = (long long)h[ACC_SUM], inf = (long long)h[ACC_INFEASIBLE];
    if (out_sum) *out_sum = sum;
    if (out_infeasible) *out_infeasible = inf;
    if (out_mean) *out_mean = (S - inf) > 0 ? (double)sum / (double)(S - inf) : NAN;
    return inf > 0 ? CVRPSD_WARN_INFEASIBLE : CVRPSD_OK;
}
