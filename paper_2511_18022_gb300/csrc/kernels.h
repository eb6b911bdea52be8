// Internal interface between the C ABI (api.cu) and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cvrpsd {

// Accumulator words written by the Split kernels (device). The first
// ACC_WORDS are zeroed per call; ACC_STICKY collects the status bits of every
// call until the host reads and clears it (cvrpsd_check_inputs), so that a
// call that returned without waiting still has its input errors reported.
enum AccWord { ACC_SUM = 0, ACC_INFEASIBLE = 1, ACC_OVERFLOW = 2, ACC_STATUS = 3, ACC_WORDS = 4, ACC_STICKY = 4,
               ACC_ALLOC_WORDS = 8 };

// Device status bits (ACC_STATUS, and a batch's BACC_STATUS).
enum StatusBits { ST_NEGATIVE_DEMAND = 1, ST_INDEX = 2 };

// Checked build (compile with -DCVRPSD_CHECKED=1): every index a Split kernel
// forms from data (table rows, scenario columns, list entries) is compared
// with its buffer before use; a bad one sets ST_INDEX in `status` and the
// access is skipped. Nothing traps. The regular build compiles the checks
// away.
#ifndef CVRPSD_CHECKED
#define CVRPSD_CHECKED 0
#endif
#ifdef __CUDACC__
__device__ __forceinline__ bool index_ok(bool ok, unsigned long long *status)
{
#if CVRPSD_CHECKED
    if (!ok) atomicOr(status, (unsigned long long)ST_INDEX);
    return ok;
#else
    (void)status;
    (void)ok;
    return true;
#endif
}
#endif

// One tour position as the kernels read it: the demand row of sigma_i and the
// scenario-independent cost term C_i (see api.cu: C_i = c(sigma_i,0) +
// c(0,sigma_{i+1}) - c(sigma_i,sigma_{i+1}) for i < n, and for i = n the full
// tail D[n] + c(sigma_n, 0)).
struct TourStep {
    int32_t row;
    int32_t c;
};

struct SplitParams {
    const TourStep *tab;          // device [n]
    const void *demand;           // device [n][ld]
    int64_t ld;                   // row pitch, elements
    int64_t S;                    // scenarios
    int32_t n, Q, L;              // L > n means no route-length limit
    int32_t g0;                   // c(0, sigma_1)
    uint32_t K;                   // key scale: power of two > n
    int32_t *out_cost;            // device [S] or nullptr
    unsigned long long *acc;      // device [ACC_WORDS]
    int32_t *ovf_list;            // device [S]: scenarios the deque could not hold
    int16_t *pred;                // device [n][ldp] or nullptr: optimal predecessor of each position
    long long ldp;
};

struct DequeShape {
    int threads;    // 64, 128, 256
    int spt;        // 1, 2
    int ring;       // 16, 32, 64
};

// Deque kernel, one thread per `spt` scenarios. esize = 2 or 4.
cudaError_t launch_split_deque(const SplitParams &p, int esize, const DequeShape &shape,
                               cudaStream_t stream);
cudaError_t launch_split_deque_i16_cap(const SplitParams &p, const DequeShape &s, cudaStream_t st);
cudaError_t launch_split_deque_i16_nocap(const SplitParams &p, const DequeShape &s, cudaStream_t st);
cudaError_t launch_split_deque_i32_cap(const SplitParams &p, const DequeShape &s, cudaStream_t st);
cudaError_t launch_split_deque_i32_nocap(const SplitParams &p, const DequeShape &s, cudaStream_t st);

// Dynamic shared memory of the deque kernel: its rings ([spt][ring][threads] int2).
inline size_t split_deque_smem(const SplitParams &p, const DequeShape &shape)
{
    (void)p;
    return (size_t)shape.spt * shape.ring * shape.threads * 8;
}

// Warp-per-scenario kernel. If `list` is non-null it evaluates the scenarios
// named in list[0 .. *count) (count lives on the device); otherwise all S.
// `max_smem` is the device's opt-in shared memory per block.
cudaError_t launch_split_warp(const SplitParams &p, int esize, const int32_t *list,
                              const unsigned long long *count, int grid_ctas, int max_smem,
                              cudaStream_t stream);
inline size_t split_warp_smem_per_warp(int n) { return (size_t)2 * (n + 1) * sizeof(int); }

// ---- batches of tours (one persistent launch) ----

// One tour of a batch, as the batch kernels read it.
struct TourDev {
    const TourStep *tab;          // device [n]
    const void *demand;           // device [n][ld]
    long long ld;
    int32_t *out_cost;            // device [S] or nullptr
    int32_t n, Q, L, g0;          // L > n: no route-length limit
    uint32_t K;
    int32_t pad;
};

// Batch accumulator header; per tour three words follow: sum, infeasible
// count, status bits.
enum BatchAccWord { BACC_COUNTER = 0, BACC_LIST = 1, BACC_STATUS = 2, BACC_WORDS = 4 };
enum BatchStatusBits { BST_LIST_FULL = 1 };   // shares its word with ST_INDEX (2)

struct BatchParams {
    const TourDev *tours;         // device [T]
    const int2 *items;            // device [n_items]: (tour, scenario tile), in processing order;
                                  // nullptr: item = tour * tiles + tile
    int n_items;
    int tiles;                    // scenario tiles per tour (with items == nullptr)
    long long S;                  // scenarios per tour
    unsigned long long *acc;      // device [BACC_WORDS + 3 T]
    int2 *list;                   // device [list_cap]: set-aside (tour, scenario)
    long long list_cap;
    int max_n;                    // largest tour
    int walk2;                    // int16 demands and keys that cannot wrap in every tour: the
                                  // second walk runs the one-scenario-per-thread shapes
};

// Dynamic shared memory of the batch kernel: rings, then the current tour's table.
inline size_t split_batch_smem(int max_n, const DequeShape &shape)
{
    return (size_t)shape.spt * shape.ring * shape.threads * 8 + (size_t)max_n * sizeof(TourStep);
}
// Persistent deque kernel over all work items; with configure_only it only
// sets the kernel's shared-memory limit (call before stream capture) and
// reports blocks per SM in *blocks_per_sm.
cudaError_t launch_split_batch(const BatchParams &b, int esize, bool lcap, const DequeShape &shape, int grid,
                               bool configure_only, int *blocks_per_sm, cudaStream_t stream);
// The batch kernel on the second walk (split_batch2.cu), which
// launch_split_batch picks where b.walk2 is set and the shape has one
// scenario per thread.
bool batch2_shape_compiled(const DequeShape &s);
cudaError_t launch_split_batch2_cap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                    int *blocks_per_sm, cudaStream_t stream);
cudaError_t launch_split_batch2_nocap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                      int *blocks_per_sm, cudaStream_t stream);
// Whether every key K (P + Q) + p of an int16 walk stays below 2^31 (demands
// read unclamped: one bad demand may add up to 65535 before the walk freezes).
inline bool batch2_keys_fit(long long n, long long Q, long long K)
{
    return K * (n * Q + 65535 + Q) + n < (1LL << 31);
}
cudaError_t launch_split_batch_i16_cap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                       int *blocks_per_sm, cudaStream_t stream);
cudaError_t launch_split_batch_i16_nocap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                         int *blocks_per_sm, cudaStream_t stream);
cudaError_t launch_split_batch_i32_cap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                       int *blocks_per_sm, cudaStream_t stream);
cudaError_t launch_split_batch_i32_nocap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                         int *blocks_per_sm, cudaStream_t stream);
// Whether the batch kernel is compiled for this (threads, spt, ring).
bool batch_shape_compiled(const DequeShape &s);
cudaError_t launch_split_warp_batch(const BatchParams &b, int esize, int grid_ctas, int max_smem, bool configure_only,
                                    cudaStream_t stream);

// Sequence-parallel Split for few scenarios (seqpar.cu).
struct SeqParParams {
    const TourStep *tab;          // device [n]
    const void *demand;           // device [n][ld]
    long long ld;
    int S, n, Q, L, g0;
    int blocks;                   // ceil(n / block)
    int32_t *lo;                  // scratch [S][n]: window starts
    int32_t *flags;               // scratch [S]: nonzero = hand to the warp kernel
    int32_t *mats;                // scratch [S][blocks][W][W]: block transfer matrices
    int32_t *out_cost;            // device [S] or nullptr
    unsigned long long *acc;      // device [ACC_WORDS]
    int32_t *list;                // device [S]: scenarios for the warp kernel
};
cudaError_t launch_seqpar(const SeqParParams &a, int esize, cudaStream_t st);
int seqpar_blocks(int n);
int seqpar_width();

// Local search on the device (search.cu).
cudaError_t launch_neighbors(const int32_t *base, int n, const int32_t *moves, int M, int32_t *out, cudaStream_t st);
cudaError_t launch_tour_tables(const int32_t *tours, int T, int n, const int32_t *dist, int32_t *D_out,
                               TourStep *tabs, TourDev *descs, const void *demand, long long ld, int Q, int L,
                               uint32_t K, cudaStream_t st);
cudaError_t launch_tour_means(const unsigned long long *acc, int T, long long S, double *mean, long long *sum,
                              long long *inf, cudaStream_t st);
cudaError_t launch_topk(const float *scores, int M, int k, int32_t *idx_out, cudaStream_t st);
cudaError_t launch_gather_rows(const int32_t *in, int rows, int n, const int32_t *idx, int R, int32_t *out,
                               cudaStream_t st);
cudaError_t launch_accept_best(const int32_t *tours, int T, int n, const double *cost, int32_t *cur,
                               double *cur_cost, double *trace, cudaStream_t st);

// Copy a [n][ld_in] demand matrix into a [n][ld_out] one of another element
// type (first S columns); values outside int16 set *saturated (device flag).
cudaError_t launch_convert_demand(const void *in, int esize_in, long long ld_in, void *out, int esize_out,
                                  long long ld_out, int n, long long S, unsigned int *saturated,
                                  cudaStream_t stream);

// Scenario generator.
struct GenParams {
    uint64_t seed;
    int32_t kind;
    const int32_t *mu;            // device [n]
    const int32_t *region;        // device [n]
    int32_t n;
    int64_t S, ld;
    void *out;
};
cudaError_t launch_gen_demand(const GenParams &g, int esize, cudaStream_t stream);

}  // namespace cvrpsd
