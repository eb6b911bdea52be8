// Batched Split: many giant tours, each with its own scenario matrix, in one
// persistent launch. Blocks take work items (tour, tile of T * SPT
// scenarios) from an atomic counter in the order the host chose (largest
// tours first), copy the tour's table into shared memory when the tour
// changes (blocks hop between tours, so a shared copy beats L1 here), and
// walk the tile exactly as the single-tour kernel does. Each block adds its
// tile's cost sum to the tour's accumulator.
#include "split_deque.cuh"

namespace cvrpsd {

template <typename DT, int SPT, int R, int T, bool LCAP>
__global__ void __launch_bounds__(T) split_batch_kernel(BatchParams b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ long long s_sum[T / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    unsigned long long *tacc = b.acc + BACC_WORDS;
    // the current tour's table follows the rings
    TourStep *tabp = reinterpret_cast<TourStep *>(smem + (size_t)SPT * R * T * 8);
    const uint32_t tab_s = sbase + (uint32_t)SPT * R * T * 8;
    int cur = -1;
    for (;;) {
        __syncthreads();                          // the previous item is finished everywhere
        if (tid == 0) s_item = (int)atomicAdd(reinterpret_cast<unsigned int *>(b.acc + BACC_COUNTER), 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= b.n_items) break;
        const int2 it = b.items ? b.items[item] : make_int2(item / b.tiles, item % b.tiles);
        if (!index_ok(it.x >= 0 && it.y >= 0 && (long long)it.y * T * SPT < b.S, b.acc + BACC_STATUS)) continue;
        const TourDev td = b.tours[it.x];
        const int t = it.x;
        if (t != cur) {   // block-uniform; the loop-top barrier has retired the previous item
            for (int k = tid; k < td.n; k += T) tabp[k] = td.tab[k];
            __syncthreads();
            cur = t;
        }
        const TabShared tabref{tab_s};
        const long long s_first = ((long long)it.y * T + tid) * SPT;
        unsigned long long *acc = b.acc;
        int2 *list = b.list;
        const long long cap = b.list_cap;
        long long sum = split_thread<DT, SPT, R, T, LCAP>(
            td.demand, td.ld, b.S, s_first, td.n, td.Q, td.L, td.K, td.g0, sbase, tabref, tid, td.out_cost,
            [acc, list, cap, t](long long s) {
                const unsigned long long idx = atomicAdd(acc + BACC_LIST, 1ull);
                if ((long long)idx < cap) list[idx] = make_int2(t, (int)s);
                else atomicOr(acc + BACC_STATUS, (unsigned long long)BST_LIST_FULL);
            },
            b.acc + BACC_STATUS);
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

template <typename DT, int SPT, int R, int T, bool LCAP>
static cudaError_t launch_one(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                              int *blocks_per_sm, cudaStream_t stream)
{
    auto kern = split_batch_kernel<DT, SPT, R, T, LCAP>;
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

// Launch shapes compiled for the batch kernel (threads, scenarios per
// thread, ring): scenarios per block 32..512 with rings of 16, 32 and 64
// entries (64 only up to 128 threads: larger blocks of 64-entry rings leave
// room for one block per SM; 512 threads only with rings of 16).
#define CVRPSD_BATCH_SHAPES(X)                                                                  \
    X(32, 1, 16) X(32, 1, 32) X(32, 1, 64) X(32, 2, 16) X(32, 2, 32) X(32, 2, 64)               \
    X(64, 1, 16) X(64, 1, 32) X(64, 1, 64) X(64, 2, 16) X(64, 2, 32) X(64, 2, 64)               \
    X(128, 1, 16) X(128, 1, 32) X(128, 1, 64) X(128, 2, 16) X(128, 2, 32)                      \
    X(256, 1, 16) X(256, 1, 32) X(256, 2, 16) X(512, 1, 16)

template <typename DT, bool LCAP>
static cudaError_t dispatch(const BatchParams &b, const DequeShape &s, int grid, bool configure_only,
                            int *blocks_per_sm, cudaStream_t st)
{
#define CVRPSD_CASE(T_, SPT_, R_)                                                      \
    if (s.threads == T_ && s.spt == SPT_ && s.ring == R_)                             \
        return launch_one<DT, SPT_, R_, T_, LCAP>(b, s, grid, configure_only, blocks_per_sm, st);
    CVRPSD_BATCH_SHAPES(CVRPSD_CASE)
#undef CVRPSD_CASE
    return cudaErrorInvalidValue;
}

#if CVRPSD_BATCH_PART == 0
bool batch_shape_compiled(const DequeShape &s)
{
#define CVRPSD_CASE(T_, SPT_, R_) if (s.threads == T_ && s.spt == SPT_ && s.ring == R_) return true;
    CVRPSD_BATCH_SHAPES(CVRPSD_CASE)
#undef CVRPSD_CASE
    return false;
}

cudaError_t launch_split_batch_i16_cap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                       int *blocks_per_sm, cudaStream_t stream)
{
    return dispatch<int16_t, true>(b, shape, grid, configure_only, blocks_per_sm, stream);
}

cudaError_t launch_split_batch(const BatchParams &b, int esize, bool lcap, const DequeShape &shape, int grid,
                               bool configure_only, int *blocks_per_sm, cudaStream_t stream)
{
    if (esize == 2 && b.walk2 && batch2_shape_compiled(shape))
        return lcap ? launch_split_batch2_cap(b, shape, grid, configure_only, blocks_per_sm, stream)
                    : launch_split_batch2_nocap(b, shape, grid, configure_only, blocks_per_sm, stream);
    if (esize == 2)
        return lcap ? launch_split_batch_i16_cap(b, shape, grid, configure_only, blocks_per_sm, stream)
                    : launch_split_batch_i16_nocap(b, shape, grid, configure_only, blocks_per_sm, stream);
    return lcap ? launch_split_batch_i32_cap(b, shape, grid, configure_only, blocks_per_sm, stream)
                : launch_split_batch_i32_nocap(b, shape, grid, configure_only, blocks_per_sm, stream);
}
#elif CVRPSD_BATCH_PART == 1
cudaError_t launch_split_batch_i16_nocap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                         int *blocks_per_sm, cudaStream_t stream)
{
    return dispatch<int16_t, false>(b, shape, grid, configure_only, blocks_per_sm, stream);
}
#elif CVRPSD_BATCH_PART == 2
cudaError_t launch_split_batch_i32_cap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                       int *blocks_per_sm, cudaStream_t stream)
{
    return dispatch<int32_t, true>(b, shape, grid, configure_only, blocks_per_sm, stream);
}
#else
cudaError_t launch_split_batch_i32_nocap(const BatchParams &b, const DequeShape &shape, int grid, bool configure_only,
                                         int *blocks_per_sm, cudaStream_t stream)
{
    return dispatch<int32_t, false>(b, shape, grid, configure_only, blocks_per_sm, stream);
}
#endif

}  // namespace cvrpsd
