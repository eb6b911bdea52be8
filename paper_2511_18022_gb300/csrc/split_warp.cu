// Transition-parallel Split: one warp evaluates one scenario (the second
// level of parallelism of Section 3: the candidate predecessors of a position). For each position i the 32 lanes take the
// candidates p of the feasible window [mask(i), i-1] of Eq. 2/3 in a strided
// pattern and a warp min-reduction picks the best, so the cost per position
// is O(|window| / 32 + log 32) and no candidate bound is needed. It serves the
// scenarios the deque kernel sets aside, and any tour when forced.
//
// Per warp, shared memory holds the scenario's prefix loads P[0..n] (demands
// loaded by all lanes at once, then a warp scan) and the values
// g[0..n] with g(p) = f(p) + c(0, sigma_{p+1}) - D[p+1] (see split_deque.cuh).
// The window start mask(i) is the smallest p >= i - L with
// P(i) - P(p) <= Q, tracked by a pointer that only moves forward.
#include <stdint.h>

#include "kernels.h"
#include "tour_table.h"

namespace cvrpsd {

struct WarpResult {
    int cost;      // f(n), INT32_MAX if infeasible
    bool bad;      // some demand > Q
    bool neg;      // some demand < 0
};

// Evaluates scenario s of one tour with the calling (full) warp. P and g are
// this warp's shared arrays of n + 1 ints each.
template <typename DT>
__device__ WarpResult warp_split_scenario(const TourStep *tab, int n, int Q, int L, int g0, const DT *dem,
                                          long long ld, long long s, int *P, int *g, unsigned long long *status,
                                          int16_t *pred = nullptr, long long ldp = 0)
{
    const int lane = threadIdx.x & 31;
    // Demands in tour order, clamped to Q+1 (anything above Q is infeasible).
    bool neg = false, bad = false;
    for (int i = 1 + lane; i <= n; i += 32) {
        const int row = tab[i - 1].row & kRowMask;
        int q = index_ok(row < n && s >= 0 && s < ld, status) ? (int)dem[(long long)row * ld + s] : 0;
        if (q < 0) { neg = true; q = 0; }
        if (q > Q) { bad = true; q = Q + 1; }
        P[i] = q;
    }
    __syncwarp();
    // Inclusive prefix sums, 32 positions at a time.
    int carry = 0;
    for (int b = 1; b <= n; b += 32) {
        const int i = b + lane;
        int v = i <= n ? P[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (i <= n) P[i] = v + carry;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) { P[0] = 0; g[0] = g0; }
    WarpResult r;
    r.neg = __any_sync(0xffffffffu, neg);
    r.bad = __any_sync(0xffffffffu, bad);
    __syncwarp();
    r.cost = INT32_MAX;
    if (!r.bad) {
        int lo = 0;
        for (int i = 1; i <= n; ++i) {
            const int Pi = P[i];
            if (i - lo > L) lo = i - L;
            while (Pi - P[lo] > Q) ++lo;            // same on every lane
            int m = INT32_MAX, at = INT32_MAX;
            for (int c = lo + lane; c < i; c += 32) {
                const int v = g[c];
                if (v < m) { m = v; at = c; }          // first (smallest) c of this lane's minimum
            }
            const int mm = __reduce_min_sync(0xffffffffu, m);
            const int gi = tab[i - 1].c + mm;
            if (pred) {                                 // smallest optimal predecessor
                const int p = __reduce_min_sync(0xffffffffu, m == mm ? at : INT32_MAX);
                if (lane == 0) pred[(long long)(i - 1) * ldp + s] = (int16_t)p;
            }
            if (lane == 0) g[i] = gi;
            __syncwarp();
        }
        r.cost = g[n];
    }
    __syncwarp();
    return r;
}

template <typename DT>
__global__ void __launch_bounds__(128) split_warp_kernel(SplitParams p, const int32_t *list,
                                                         const unsigned long long *count)
{
    extern __shared__ __align__(16) int wsmem[];
    const int n = p.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    int *P = wsmem + (size_t)w * 2 * (n + 1);
    int *g = P + (n + 1);
    const long long total = list ? (long long)*count : p.S;
    const DT *dem = reinterpret_cast<const DT *>(p.demand);

    long long sum = 0;
    unsigned inf = 0, status = 0;
    for (long long item = (long long)blockIdx.x * wpb + w; item < total;
         item += (long long)gridDim.x * wpb) {
        const long long s = list ? (long long)list[item] : item;
        if (!index_ok(s >= 0 && s < p.S, p.acc + ACC_STATUS)) continue;   // warp-uniform
        const WarpResult r = warp_split_scenario<DT>(p.tab, n, p.Q, p.L, p.g0, dem, p.ld, s, P, g,
                                                     p.acc + ACC_STATUS, p.pred, p.ldp);
        if (lane == 0) {
            if (r.neg) status |= ST_NEGATIVE_DEMAND;
            if (r.bad) ++inf; else sum += r.cost;
            if (p.out_cost) p.out_cost[s] = r.cost;
        }
    }
    if (lane == 0) {
        if (sum) atomicAdd(p.acc + ACC_SUM, (unsigned long long)sum);
        if (inf) atomicAdd(p.acc + ACC_INFEASIBLE, (unsigned long long)inf);
        if (status) {
            atomicOr(p.acc + ACC_STATUS, (unsigned long long)status);
            atomicOr(p.acc + ACC_STICKY, (unsigned long long)status);
        }
    }
}

// Set-aside (tour, scenario) pairs of a batch; per-tour sums, infeasible
// counts and status words follow the batch header in `acc`.
template <typename DT>
__global__ void __launch_bounds__(128) split_warp_batch_kernel(BatchParams b)
{
    extern __shared__ __align__(16) int wsmem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    int *P = wsmem + (size_t)w * 2 * (b.max_n + 1);
    int *g = P + (b.max_n + 1);
    const unsigned long long cnt = b.acc[BACC_LIST];
    const long long total = (long long)(cnt < (unsigned long long)b.list_cap ? cnt : (unsigned long long)b.list_cap);
    unsigned long long *tacc = b.acc + BACC_WORDS;
    for (long long item = (long long)blockIdx.x * wpb + w; item < total;
         item += (long long)gridDim.x * wpb) {
        const int2 e = b.list[item];
        if (!index_ok(e.x >= 0 && e.y >= 0 && e.y < b.S, b.acc + BACC_STATUS)) continue;   // warp-uniform
        const TourDev td = b.tours[e.x];
        const WarpResult r = warp_split_scenario<DT>(td.tab, td.n, td.Q, td.L, td.g0,
                                                     reinterpret_cast<const DT *>(td.demand), td.ld, e.y, P, g,
                                                     b.acc + BACC_STATUS);
        if (lane == 0) {
            if (r.neg) atomicOr(tacc + 3 * e.x + 2, (unsigned long long)ST_NEGATIVE_DEMAND);
            if (r.bad) atomicAdd(tacc + 3 * e.x + 1, 1ull);
            else atomicAdd(tacc + 3 * e.x, (unsigned long long)r.cost);
            if (td.out_cost) td.out_cost[e.y] = r.cost;
        }
    }
}

static int warps_for(size_t per_warp, int max_smem)
{
    int warps = 4;
    while (warps > 1 && (size_t)warps * per_warp > (size_t)max_smem) --warps;
    return per_warp > (size_t)max_smem ? 0 : warps;
}

cudaError_t launch_split_warp(const SplitParams &p, int esize, const int32_t *list,
                              const unsigned long long *count, int grid_ctas, int max_smem,
                              cudaStream_t stream)
{
    const size_t per_warp = split_warp_smem_per_warp(p.n);
    const int warps = warps_for(per_warp, max_smem);
    if (!warps) return cudaErrorInvalidValue;
    const int threads = 32 * warps;
    const size_t smem = (size_t)warps * per_warp;
    if (esize == 2) {
        auto k = split_warp_kernel<int16_t>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid_ctas, threads, smem, stream>>>(p, list, count);
    } else {
        auto k = split_warp_kernel<int32_t>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid_ctas, threads, smem, stream>>>(p, list, count);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_warp_batch(const BatchParams &b, int esize, int grid_ctas, int max_smem, bool configure_only,
                                    cudaStream_t stream)
{
    const size_t per_warp = split_warp_smem_per_warp(b.max_n);
    const int warps = warps_for(per_warp, max_smem);
    if (!warps) return cudaErrorInvalidValue;
    const size_t smem = (size_t)warps * per_warp;
    auto k = esize == 2 ? split_warp_batch_kernel<int16_t> : split_warp_batch_kernel<int32_t>;
    if (configure_only)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid_ctas, 32 * warps, smem, stream>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_split_deque(const SplitParams &p, int esize, const DequeShape &shape,
                               cudaStream_t stream)
{
    const bool cap = p.L < p.n;
    if (esize == 2) return cap ? launch_split_deque_i16_cap(p, shape, stream)
                               : launch_split_deque_i16_nocap(p, shape, stream);
    return cap ? launch_split_deque_i32_cap(p, shape, stream)
               : launch_split_deque_i32_nocap(p, shape, stream);
}

}  // namespace cvrpsd
