// Instantiations and launcher of the deque Split kernel. The template
// arguments are split over translation units (CVRPSD_DEQUE_PART) so that the
// build compiles them in parallel.
#include "split_deque.cuh"

namespace cvrpsd {

template <typename DT, int SPT, int R, int T, bool LCAP, bool PRED = false>
static cudaError_t launch_one(const SplitParams &p, const DequeShape &shape, cudaStream_t stream)
{
    auto kern = split_deque_kernel<DT, SPT, R, T, LCAP, PRED>;
    const size_t smem = split_deque_smem(p, shape);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long per_block = (long long)T * SPT;
    const long long blocks = (p.S + per_block - 1) / per_block;
    kern<<<(unsigned)blocks, T, smem, stream>>>(p);
    return cudaGetLastError();
}

template <typename DT, bool LCAP>
static cudaError_t dispatch_shape(const SplitParams &p, const DequeShape &s, cudaStream_t st)
{
    if (p.pred) {   // route recovery: one scenario per thread
        if (s.spt == 1 && s.threads == 128 && s.ring == 16) return launch_one<DT, 1, 16, 128, LCAP, true>(p, s, st);
        if (s.spt == 1 && s.threads == 128 && s.ring == 32) return launch_one<DT, 1, 32, 128, LCAP, true>(p, s, st);
        if (s.spt == 1 && s.threads == 256 && s.ring == 32) return launch_one<DT, 1, 32, 256, LCAP, true>(p, s, st);
        return launch_one<DT, 1, 16, 256, LCAP, true>(p, DequeShape{256, 1, 16}, st);
    }
#define CVRPSD_CASE(T_, SPT_, R_) \
    if (s.threads == T_ && s.spt == SPT_ && s.ring == R_) return launch_one<DT, SPT_, R_, T_, LCAP>(p, s, st);
#define CVRPSD_CASES_T(T_) \
    CVRPSD_CASE(T_, 1, 16) CVRPSD_CASE(T_, 1, 32) CVRPSD_CASE(T_, 1, 64) \
    CVRPSD_CASE(T_, 2, 16) CVRPSD_CASE(T_, 2, 32) CVRPSD_CASE(T_, 2, 64)
    CVRPSD_CASES_T(64) CVRPSD_CASES_T(128) CVRPSD_CASES_T(256)
    CVRPSD_CASE(128, 1, 8) CVRPSD_CASE(256, 1, 8)
#undef CVRPSD_CASES_T
#undef CVRPSD_CASE
    return cudaErrorInvalidValue;
}

#if CVRPSD_DEQUE_PART == 0
cudaError_t launch_split_deque_i16_cap(const SplitParams &p, const DequeShape &s, cudaStream_t st)
{ return dispatch_shape<int16_t, true>(p, s, st); }
#elif CVRPSD_DEQUE_PART == 1
cudaError_t launch_split_deque_i16_nocap(const SplitParams &p, const DequeShape &s, cudaStream_t st)
{ return dispatch_shape<int16_t, false>(p, s, st); }
#elif CVRPSD_DEQUE_PART == 2
cudaError_t launch_split_deque_i32_cap(const SplitParams &p, const DequeShape &s, cudaStream_t st)
{ return dispatch_shape<int32_t, true>(p, s, st); }
#elif CVRPSD_DEQUE_PART == 3
cudaError_t launch_split_deque_i32_nocap(const SplitParams &p, const DequeShape &s, cudaStream_t st)
{ return dispatch_shape<int32_t, false>(p, s, st); }
#endif

}  // namespace cvrpsd
