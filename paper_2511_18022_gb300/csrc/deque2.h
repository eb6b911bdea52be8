// Internal interface of the second deque walk (split_deque2.cuh): its
// parameter blocks and launcher.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "tour_table.h"

namespace cvrpsd {

// Table capacities of the kernel-parameter tour table: 8 KB for tours up to
// 1024 customers, and the largest that fits the 32 KB parameter space.
constexpr int kTab2Small = 1024;
constexpr int kTab2Large = 4032;

// Tour positions per prefetch block of the second walk: its demands are
// loaded one block ahead (at full occupancy four positions hide the load
// latency, and the walk then fits 32 registers).
constexpr int kPrefetch2 = 4;

// Table entry of position i (index i - 1): x = the demand row of sigma_i in
// the low bits, plus kTab2NoBack when no scenario can pop the deque's back
// at i (C_{i-1} > 0 and C_i > C_{i-1}, see split_deque2.cuh); y = C_i. Bit m
// of nonpos marks prefetch block m (positions 1 + m * kPrefetch2 ...) as
// holding some C_i <= 0 with i < n.
constexpr uint32_t kTab2NoBack = 1u << 31;
constexpr uint32_t kTab2RowMask = kTab2NoBack - 1u;

template <int CAP>
struct TabParam {
    uint2 e[CAP];
    uint32_t nonpos[(CAP / kPrefetch2 + 31) / 32];
    static constexpr int kCap = CAP;
#ifdef __CUDACC__
    // The walk's view of a table (see TabShared2 for the batch kernel's).
    __device__ __forceinline__ uint2 entry(int i) const { return e[i - 1]; }
    __device__ __forceinline__ uint32_t row(int i) const { return e[i - 1].x & kTab2RowMask; }
    __device__ __forceinline__ bool general(int i0) const
    {
        const int m = (i0 - 1) / kPrefetch2;
        return (nonpos[m >> 5] >> (m & 31)) & 1u;
    }
#endif
};

struct Walk2Params {
    const void *demand;        // device [n][ld]
    long long S;               // scenarios
    long long stride;          // grid * T: scenario step between a thread's rounds
    int32_t n, Q, L, g0;       // L > n: no route-length limit
    uint32_t K;                // key scale: power of two > n
    uint32_t pitch;            // bytes between demand rows
    int32_t *out_cost;         // device [S] or nullptr
    unsigned long long *acc;   // device [ACC_WORDS]
    int32_t *ovf_list;         // device [S]
    unsigned long long *status;   // device word for index-check status bits
};

// Whether the second walk can run this Split (otherwise the first walk runs):
// no predecessor output, n <= kTab2Large, demand rows addressable with
// 32-bit byte offsets, and for int16 demands Q < 32768 (a negative demand
// read as unsigned then exceeds Q).
bool deque2_supported(const SplitParams &p, int esize);

// Launch it. `tab` is the host copy of the tour table (TourStep rows with
// the block flag); rounds = 0 gives one scenario per thread, rounds >= 1 a
// grid of ceil(tiles / rounds) blocks, each walking up to `rounds` tiles of
// T scenarios. *shape_ran receives the (threads, ring) actually launched.
cudaError_t launch_split_deque2(const SplitParams &p, const TourStep *tab, int esize, const DequeShape &shape,
                                int rounds, DequeShape *shape_ran, cudaStream_t stream);

}  // namespace cvrpsd
