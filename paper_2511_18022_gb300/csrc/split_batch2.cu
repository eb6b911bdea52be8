// Batched Split on the second deque walk (split_deque2.cuh): the persistent
// item loop of split_batch.cu (blocks take (tour, tile of T scenarios) items
// from an atomic counter, longest tours first, and copy a tour's table into
// shared memory when they move to it), with each thread walking its scenario
// by the second walk's rules: int16 demands read unclamped, tests of the
// route length and of ring overflow once per span of 8 positions, no
// frozen flag in the tests, front walks that read only keys, back-pop skip
// bits and a vote-free first back step. The table differs from the
// single-tour walk's only in where it lives: shared memory instead of the
// launch parameters, with the skip bit and the block flag derived while it
// is copied. One scenario per thread, int16 demands, rings of 16 or more,
// keys that cannot wrap (the host checks every tour).
#include "split_deque2.cuh"

namespace cvrpsd {

// Shared-memory table entry of position i at byte (i - 1) * 8: x = demand
// row | kTab2NoBack (no back pops at i) | kTab2SharedGeneral (on the first
// entry of a prefetch block holding some C_i <= 0 with i < n), y = C_i.
constexpr uint32_t kTab2SharedGeneral = 1u << 30;
constexpr uint32_t kTab2SharedRowMask = kTab2SharedGeneral - 1u;

struct TabShared2 {
    uint32_t a;   // shared-window address of entry 0
    static constexpr int kCap = 1 << 30;
    __device__ __forceinline__ uint2 entry(int i) const
    {
        const int2 v = lds2(a + (uint32_t)(i - 1) * 8u);
        return make_uint2((uint32_t)v.x, (uint32_t)v.y);
    }
    __device__ __forceinline__ uint32_t row(int i) const
    {
        return (uint32_t)lds1(a + (uint32_t)(i - 1) * 8u) & kTab2SharedRowMask;
    }
    __device__ __forceinline__ bool general(int i0) const
    {
        return ((uint32_t)lds1(a + (uint32_t)(i0 - 1) * 8u) & kTab2SharedGeneral) != 0;
    }
};

// Blocks an SM holds: shared memory for the rings and a table of up to 1024
// positions (1 KB reserved per block), at most 2048 threads and 32 blocks.
// The registers this leaves (40 or more) keep the per-item tour parameters
// out of local memory.
template <int R, int T>
constexpr int b2_min_blocks()
{
    constexpr int by_smem = 233472 / (R * T * 8 + 8192 + 1024);
    constexpr int by_threads = 2048 / T;
    constexpr int m = by_smem < by_threads ? by_smem : by_threads;
    return m < 1 ? 1 : (m > 32 ? 32 : m);
}

template <int R, int T, bool LCAP>
__global__ void __launch_bounds__(T, b2_min_blocks<R, T>()) split_batch2_kernel(BatchParams b)
{
    extern __shared__ __align__(16) unsigned char smem[];   // rings [R][T], then the table
    __shared__ int s_item;
    __shared__ long long s_sum[T / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t rs = (uint32_t)__cvta_generic_to_shared(smem);
    uint2 *tabp = reinterpret_cast<uint2 *>(smem + (size_t)R * T * 8);
    const TabShared2 tab{rs + (uint32_t)R * T * 8};
    unsigned long long *tacc = b.acc + BACC_WORDS;
    unsigned long long *status = b.acc + BACC_STATUS;
    int cur = -1;
    for (;;) {
        __syncthreads();                          // the previous item is finished everywhere
        if (tid == 0) s_item = (int)atomicAdd(reinterpret_cast<unsigned int *>(b.acc + BACC_COUNTER), 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= b.n_items) break;
        const int2 it = b.items ? b.items[item] : make_int2(item / b.tiles, item % b.tiles);
        if (!index_ok(it.x >= 0 && it.y >= 0 && (long long)it.y * T < b.S, status)) continue;
        const TourDev td = b.tours[it.x];
        const int t = it.x;
        if (t != cur) {   // block-uniform; the loop-top barrier has retired the previous item
            for (int k = tid; k < td.n; k += T) {
                const int ck = td.tab[k].c;
                uint32_t x = (uint32_t)(td.tab[k].row & kRowMask);
                // position k + 1 >= 2 with C_k > 0 and C_{k+1} > C_k: no back pops
                if (k >= 1) {
                    const int cp = td.tab[k - 1].c;
                    if (cp > 0 && ck > cp) x |= kTab2NoBack;
                }
                if (k % kPrefetch2 == 0) {
                    bool np = false;
                    for (int u = k; u < k + kPrefetch2 && u < td.n - 1; ++u) np |= td.tab[u].c <= 0;
                    if (np) x |= kTab2SharedGeneral;
                }
                tabp[k] = make_uint2(x, (uint32_t)ck);
            }
            __syncthreads();
            cur = t;
        }
        Walk2Params p{};
        p.demand = td.demand;
        p.S = b.S;
        p.n = td.n;
        p.Q = td.Q;
        p.L = td.L;
        p.g0 = td.g0;
        p.K = td.K;
        p.pitch = (uint32_t)(td.ld * 2);
        p.status = status;
        const long long s = (long long)it.y * T + tid;
        bool aside = false;
        const int c = walk2_scenario<int16_t, R, T, LCAP, true>(p, tab, s, rs, (uint32_t)tid * 8u, aside);
        long long sum = 0;
        if (s < b.S) {
            if (aside) {
                const unsigned long long idx = atomicAdd(b.acc + BACC_LIST, 1ull);
                if ((long long)idx < b.list_cap) b.list[idx] = make_int2(t, (int)s);
                else atomicOr(status, (unsigned long long)BST_LIST_FULL);
            } else {
                sum = c;
                if (td.out_cost) td.out_cost[s] = c;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) s_sum[w] = sum;
        __syncthreads();
        if (tid == 0) {
            long long tot = 0;
#pragma unroll
            for (int k = 0; k < T / 32; ++k) tot += s_sum[k];
            if (tot) atomicAdd(tacc + 3 * t, (unsigned long long)tot);
        }
    }
}

template <int R, int T, bool LCAP>
static cudaError_t launch2_one(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                               int *blocks_per_sm, cudaStream_t stream)
{
    auto kern = split_batch2_kernel<R, T, LCAP>;
    const size_t smem = split_batch_smem(b.max_n, shape);
    if (configure_only) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return blocks_per_sm ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, T, smem)
                             : cudaSuccess;
    }
    kern<<<grid, T, smem, stream>>>(b);
    return cudaGetLastError();
}

// Shapes of the batch kernel's list with one scenario per thread.
#define CVRPSD_BATCH2_SHAPES(X)                                                                 \
    X(32, 16) X(32, 32) X(32, 64) X(64, 16) X(64, 32) X(64, 64) X(128, 16) X(128, 32)            \
    X(128, 64) X(256, 16) X(256, 32) X(512, 16)

template <bool LCAP>
static cudaError_t dispatch2(const BatchParams &b, const DequeShape &s, int grid, bool configure_only,
                             int *blocks_per_sm, cudaStream_t st)
{
#define CVRPSD_CASE(T_, R_)                                                            \
    if (s.threads == T_ && s.spt == 1 && s.ring == R_)                                \
        return launch2_one<R_, T_, LCAP>(b, s, grid, configure_only, blocks_per_sm, st);
    CVRPSD_BATCH2_SHAPES(CVRPSD_CASE)
#undef CVRPSD_CASE
    return cudaErrorInvalidValue;
}

#if CVRPSD_BATCH2_PART == 0
bool batch2_shape_compiled(const DequeShape &s)
{
#define CVRPSD_CASE(T_, R_) if (s.threads == T_ && s.spt == 1 && s.ring == R_) return true;
    CVRPSD_BATCH2_SHAPES(CVRPSD_CASE)
#undef CVRPSD_CASE
    return false;
}

cudaError_t launch_split_batch2_cap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                    int *blocks_per_sm, cudaStream_t stream)
{
    return dispatch2<true>(b, shape, grid, configure_only, blocks_per_sm, stream);
}
#else
cudaError_t launch_split_batch2_nocap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                      int *blocks_per_sm, cudaStream_t stream)
{
    return dispatch2<false>(b, shape, grid, configure_only, blocks_per_sm, stream);
}
#endif

}  // namespace cvrpsd
