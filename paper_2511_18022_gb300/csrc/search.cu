// Device-side pieces of the local search around the Split: neighbour tours
// from 2-opt / relocate moves, per-tour tables built on the device, a
// many-tours-one-instance Split on the persistent batch kernel, and a
// bitonic top-k. Everything stays on the device so that a search iteration
// needs no host round trip.
#include <stdint.h>

#include "kernels.h"
#include "tour_table.h"

namespace cvrpsd {

// Move (type, a, b) applied to `base` (positions 0..n-1):
//   type 0, 2-opt: reverse positions a..b (a <= b);
//   type 1, relocate: take the customer at position a out and put it back so
//           that it ends at position b (positions between shift by one).
__device__ __forceinline__ int move_source(int k, int type, int a, int b)
{
    if (type == 0) {
        if (a > b) { const int t = a; a = b; b = t; }
        return (k >= a && k <= b) ? a + b - k : k;
    }
    if (a == b) return k;
    if (a < b) return k < a ? k : (k < b ? k + 1 : (k == b ? a : k));
    return k < b ? k : (k == b ? a : (k <= a ? k - 1 : k));
}

__global__ void neighbors_kernel(const int32_t *base, int n, const int32_t *moves, int M, int32_t *out)
{
    for (int m = blockIdx.x; m < M; m += gridDim.x) {
        // positions outside 0..n-1 are clamped: every read stays inside the base tour
        const int type = moves[3 * m];
        const int a = min(max(moves[3 * m + 1], 0), n - 1), b = min(max(moves[3 * m + 2], 0), n - 1);
        for (int k = threadIdx.x; k < n; k += blockDim.x) out[(long long)m * n + k] = base[move_source(k, type, a, b)];
    }
}

cudaError_t launch_neighbors(const int32_t *base, int n, const int32_t *moves, int M, int32_t *out, cudaStream_t st)
{
    if (M == 0) return cudaSuccess;
    neighbors_kernel<<<M < 4096 ? M : 4096, 128, 0, st>>>(base, n, moves, M, out);
    return cudaGetLastError();
}

// Tables of T tours of one instance (as fill_tour_table builds them on the
// host): one block per tour, positions spread over the threads. The
// per-block flag for C_i <= 0 is an OR over kPrefetch consecutive positions.
__global__ void tour_tables_kernel(const int32_t *tours, int T, int n, const int32_t *dist, int32_t *D_out,
                                   TourStep *tabs, TourDev *descs, const void *demand, long long ld, int Q, int L,
                                   uint32_t K)
{
    __shared__ long long s_len[32];
    const long long N1 = (long long)n + 1;
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
        const int32_t *tour = tours + (long long)t * n;
        TourStep *tab = tabs + (long long)t * n;
        long long len = 0;
        const int rounds = (n + blockDim.x - 1) / blockDim.x;
        for (int r = 0; r < rounds; ++r) {
            const int k = r * blockDim.x + threadIdx.x;
            int c = 0, row = 0;
            if (k < n) {
                const int cu = min(max(tour[k], 1), n);           // ids outside 1..n are clamped
                row = cu - 1;
                if (k + 1 < n) {
                    const int nx = min(max(tour[k + 1], 1), n);
                    const int edge = dist[(long long)cu * N1 + nx];
                    len += edge;
                    c = dist[(long long)cu * N1] + dist[nx] - edge;
                }
            }
            // blocks of kPrefetch positions are aligned inside a warp (32 % kPrefetch == 0)
            const unsigned nonpos = __ballot_sync(0xffffffffu, k < n - 1 && c <= 0);
            const int lane = threadIdx.x & 31;
            const unsigned group = (nonpos >> (lane & ~(kPrefetch - 1))) & ((1u << kPrefetch) - 1);
            if (k < n) {
                if ((k % kPrefetch) == 0 && group) row |= kRowFlagNonPositive;
                tab[k].row = row;
                if (k + 1 < n) tab[k].c = c;
            }
        }
        // tour length D[n] for C_n = D[n] + c(sigma_n, 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len += __shfl_xor_sync(0xffffffffu, len, o);
        if ((threadIdx.x & 31) == 0) s_len[threadIdx.x >> 5] = len;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long Dn = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) Dn += s_len[w];
            const int last = min(max(tour[n - 1], 1), n);
            tab[n - 1].c = (int32_t)(Dn + dist[(long long)last * N1]);
            if (D_out) D_out[t] = (int32_t)Dn;
            TourDev d;
            d.tab = tab;
            d.demand = demand;
            d.ld = ld;
            d.out_cost = nullptr;
            d.n = n;
            d.Q = Q;
            d.L = L;
            d.g0 = dist[min(max(tour[0], 1), n)];
            d.K = K;
            d.pad = 0;
            descs[t] = d;
        }
        __syncthreads();
    }
}

cudaError_t launch_tour_tables(const int32_t *tours, int T, int n, const int32_t *dist, int32_t *D_out,
                               TourStep *tabs, TourDev *descs, const void *demand, long long ld, int Q, int L,
                               uint32_t K, cudaStream_t st)
{
    if (T == 0) return cudaSuccess;
    tour_tables_kernel<<<T < 8192 ? T : 8192, 256, 0, st>>>(tours, T, n, dist, D_out, tabs, descs, demand, ld, Q, L, K);
    return cudaGetLastError();
}

// Per-tour SAA outputs from the batch accumulators.
__global__ void tour_means_kernel(const unsigned long long *acc, int T, long long S, double *mean, long long *sum,
                                  long long *inf)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const unsigned long long *w = acc + BACC_WORDS + 3 * t;
    const long long s = (long long)w[0], i = (long long)w[1];
    if (sum) sum[t] = s;
    if (inf) inf[t] = i;
    if (mean) mean[t] = (S - i) > 0 ? (double)s / (double)(S - i) : __longlong_as_double(0x7ff8000000000000LL);
}

cudaError_t launch_tour_means(const unsigned long long *acc, int T, long long S, double *mean, long long *sum,
                              long long *inf, cudaStream_t st)
{
    if (T == 0) return cudaSuccess;
    tour_means_kernel<<<(T + 255) / 256, 256, 0, st>>>(acc, T, S, mean, sum, inf);
    return cudaGetLastError();
}

// k smallest scores (ties: smaller index first) of M <= 16384, one block:
// bitonic sort of (score, index) pairs padded to a power of two.
__global__ void topk_kernel(const float *scores, int M, int k, int32_t *idx_out)
{
    extern __shared__ unsigned long long keys[];
    int P = 1;
    while (P < M) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned int bits = 0xFFFFFFFFu;
        if (i < M) {
            const float f = scores[i];
            unsigned int u = __float_as_uint(f);
            bits = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // order-preserving map of floats
            if (f != f) bits = 0xFFFFFFFFu;                        // NaN last
        }
        keys[i] = ((unsigned long long)bits << 32) | (unsigned int)i;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = keys[i], b = keys[j];
                    if ((a > b) == up) { keys[i] = b; keys[j] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) idx_out[i] = (int32_t)(keys[i] & 0xFFFFFFFFu);
}

cudaError_t launch_topk(const float *scores, int M, int k, int32_t *idx_out, cudaStream_t st)
{
    int P = 1;
    while (P < M) P <<= 1;
    const size_t smem = (size_t)P * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    topk_kernel<<<1, 1024, smem, st>>>(scores, M, k, idx_out);
    return cudaGetLastError();
}

// Gather rows: out[r] = in[idx[r]] for rows of n ints.
__global__ void gather_rows_kernel(const int32_t *in, int rows, int n, const int32_t *idx, int R, int32_t *out)
{
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const long long src = (long long)min(max(idx[r], 0), rows - 1) * n;   // clamped into the source
        for (int k = threadIdx.x; k < n; k += blockDim.x) out[(long long)r * n + k] = in[src + k];
    }
}

cudaError_t launch_gather_rows(const int32_t *in, int rows, int n, const int32_t *idx, int R, int32_t *out,
                               cudaStream_t st)
{
    if (R == 0 || rows < 1) return cudaSuccess;
    gather_rows_kernel<<<R < 4096 ? R : 4096, 128, 0, st>>>(in, rows, n, idx, R, out);
    return cudaGetLastError();
}

// The search's acceptance, one block: the cheapest of T costs (smallest
// index among equal costs; a NaN cost compares false and is never taken),
// accepted when strictly cheaper than *cur_cost, in which case its tour
// replaces cur. trace (optional) gets the current cost after the step.
constexpr int kAcceptThreads = 256;

__global__ void __launch_bounds__(kAcceptThreads) accept_best_kernel(const int32_t *tours, int T, int n,
                                                                     const double *cost, int32_t *cur,
                                                                     double *cur_cost, double *trace)
{
    __shared__ double s_c[kAcceptThreads / 32];
    __shared__ int s_i[kAcceptThreads / 32];
    __shared__ int s_take;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    double best = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    int bi = T;                                                   // none yet
    for (int j = tid; j < T; j += kAcceptThreads) {
        const double c = cost[j];
        if (c < best) best = c, bi = j;       // ascending j: the first of equal costs stays
    }
    // (cost, index) minimum over the block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oc = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oc < best || (oc == best && oi < bi)) best = oc, bi = oi;
    }
    if (lane == 0) s_c[w] = best, s_i[w] = bi;
    __syncthreads();
    if (tid == 0) {
        for (int k = 1; k < kAcceptThreads / 32; ++k)
            if (s_c[k] < best || (s_c[k] == best && s_i[k] < bi)) best = s_c[k], bi = s_i[k];
        const double cc = *cur_cost;
        const bool take = bi < T && best < cc;
        if (take) *cur_cost = best;
        if (trace) *trace = take ? best : cc;
        s_take = take ? bi : -1;
    }
    __syncthreads();
    const int b = s_take;
    if (b >= 0)
        for (int k = tid; k < n; k += kAcceptThreads) cur[k] = tours[(long long)b * n + k];
}

cudaError_t launch_accept_best(const int32_t *tours, int T, int n, const double *cost, int32_t *cur,
                               double *cur_cost, double *trace, cudaStream_t st)
{
    accept_best_kernel<<<1, kAcceptThreads, 0, st>>>(tours, T, n, cost, cur, cur_cost, trace);
    return cudaGetLastError();
}

}  // namespace cvrpsd
