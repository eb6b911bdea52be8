// Scenario-parallel Split: one thread evaluates SPT scenarios of one giant
// tour, walking the tour positions i = 1..n in order (the first of the two
// levels of parallelism of Section 3: independent scenarios).
//
// The segment cost of Eq. 1 separates into a part of the first position and a
// part of the last (both scenario-independent), so with
//   g(p) = f(p) + c(0, sigma_{p+1}) - D[p+1]      (D = cumulative tour length)
// the recursion becomes g(i) = C_i + min_{p in W(i)} g(p), W(i) = [mask(i), i-1]
// the feasible window of Eq. 2/3 (also p >= i - L), and f(n) = C_n + min g.
// Both ends of W(i) are non-decreasing in i (demands are >= 0), so the window
// minimum is kept by a monotone double-ended queue: each candidate enters
// once and leaves once, O(1) amortised per (scenario, position) instead of
// the O(|W|) scan of Eq. 3.
//
// Deque entries are (g(p), x(p)) with x(p) = K * (P(p) + Q) + p (mod 2^32),
// P the prefix load and K = 2^k > n. Candidate p is capacity-feasible at i iff
// x(p) - K * P(i) >= 0 as a signed 32-bit difference (exact while the true
// difference stays below 2^31, which the host guarantees for feasible
// scenarios: (Q + 1) * K + n < 2^31). The route-length test p >= i - L is the
// cached expiry step e = p + L + 1 of the front entry.
//
// A scenario with a demand above Q (or a negative one) has no valid walk
// here; a running unsigned maximum of its demands flags it, and flagged
// scenarios, like those whose deque outgrows the R-entry ring, are handed to
// the warp kernel, which evaluates them exactly. The ring of each scenario
// lives in shared memory, laid out [R][T] (warp accesses never conflict) and
// addressed by byte offsets that wrap with a mask. Demands are read straight
// from HBM with streaming loads of SPT adjacent scenarios, prefetched one
// block of kPrefetch tour positions ahead.
#pragma once

#include <stdint.h>

#include "kernels.h"
#include "tour_table.h"

namespace cvrpsd {

template <typename DT, int SPT> struct DemandVec;
template <> struct DemandVec<int16_t, 1> { using T = short; };
template <> struct DemandVec<int16_t, 2> { using T = short2; };
template <> struct DemandVec<int32_t, 1> { using T = int; };
template <> struct DemandVec<int32_t, 2> { using T = int2; };

// Demands of this thread's SPT scenarios at one tour position, as ints.
template <typename DT, int SPT>
__device__ __forceinline__ void load_demands(const char *__restrict__ base, int row, uint32_t ldb,
                                             bool full, int nvalid, int (&q)[SPT])
{
    const char *ptr = base + (unsigned long long)(uint32_t)row * ldb;
    if (SPT == 1 || full) {
        using V = typename DemandVec<DT, SPT>::T;
        const V v = __ldcs(reinterpret_cast<const V *>(ptr));
        if constexpr (SPT == 1) {
            q[0] = (int)v;
        } else {
            q[0] = (int)v.x;
            q[1] = (int)v.y;
        }
    } else {
        const DT *e = reinterpret_cast<const DT *>(ptr);
#pragma unroll
        for (int j = 0; j < SPT; ++j) q[j] = (j < nvalid) ? (int)e[j] : 0;
    }
}

struct Deque {
    int fg;            // front entry: g
    uint32_t fx;       //              x
    int fe;            //              route-length expiry step
    int bg;            // back entry: g
    uint32_t hoff;     // byte offset of the front slot within the ring
    uint32_t boff;     // byte offset of the back slot
    uint32_t pk;       // K * prefix load
    uint32_t qmax;     // largest demand seen, as unsigned (negatives are huge)
    bool ovf;          // the ring was too small
};

// 32-bit shared-memory accesses (the ring and the tour table are addressed by
// shared-window byte addresses, which keeps address arithmetic to one add).
__device__ __forceinline__ int2 lds2(uint32_t a)
{
    int2 v;
    asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ int lds1(uint32_t a)
{
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts2(uint32_t a, int x, int y)
{
    asm volatile("st.shared.v2.s32 [%0], {%1, %2};" ::"r"(a), "r"(x), "r"(y) : "memory");
}

// Tour table (TourStep = {row, c}, entry i-1 for position i) as the walk
// reads it. Every lane of a block reads the same entry (all threads walk the
// same tour position), so either way a read is one broadcast.
// TabGlobal: straight from global memory with read-only loads (the
// single-tour kernel: the table stays in L1 and shared memory is left to the
// rings). TabShared: from a copy in shared memory (the batch kernel, whose
// blocks move between tours).
struct TabShared {
    uint32_t a;   // shared-window address of entry 0
    __device__ __forceinline__ int row(int i) const { return lds1(a + (uint32_t)(i - 1) * 8u); }
    __device__ __forceinline__ int c(int i) const { return lds1(a + (uint32_t)(i - 1) * 8u + 4u); }
};
struct TabGlobal {
    const int *p;   // entry 0 as two ints (row, c)
    __device__ __forceinline__ int row(int i) const { return __ldg(p + 2 * (i - 1)); }
    __device__ __forceinline__ int c(int i) const { return __ldg(p + 2 * (i - 1) + 1); }
};

template <int R, int T>
struct Ring {
    static constexpr uint32_t kStride = T * 8u;            // bytes between slots of one thread
    static constexpr uint32_t kMask = R * T * 8u - 1u;     // ring bytes - 1 (power of two)
    __device__ static __forceinline__ uint32_t next(uint32_t off) { return (off + kStride) & kMask; }
    __device__ static __forceinline__ uint32_t prev(uint32_t off) { return (off - kStride) & kMask; }
};

// One position of the walk. PUSH: positions 1..n-1 add candidate i; the last
// position only reads the window minimum, returned as f(n).
//
// Pops at both ends run as warp-uniform loops: every lane executes each
// iteration (loads included) and applies it only if it still has an entry to
// drop, so the warp never splits on this data-dependent control flow; the
// loop ends when no lane has anything left (vote). Each scenario's walk is
// exactly the sequential deque walk.
//
// The walk uses min(q, Q) for the load: a scenario with a larger (or a
// negative) demand is flagged by qmax and re-evaluated elsewhere, and with
// the clamp the back entry (candidate i-1) is always in the window, so the
// front walk stops there at the latest. GENERAL: some C_i <= 0 in this block
// (the host marks such blocks); only then can the new value min + C_i
// undercut the front, so that back pops may empty the deque.
//
// PRED: back entries are dropped only when strictly larger, so among equal
// minima the oldest stays in front and the front is the smallest optimal
// predecessor (the tie rule of route recovery).
template <int R, int T, bool LCAP, bool PUSH, bool GENERAL, bool PRED = false>
__device__ __forceinline__ int dq_step(Deque &d, uint32_t ring, int q, int i, int ci, uint32_t K,
                                       uint32_t xi, int L, int Q, int *argmin = nullptr)
{
    using RG = Ring<R, T>;
    d.qmax = max(d.qmax, (uint32_t)q);
    d.pk += (uint32_t)min(q, Q) * K;
    // front: drop entries that left the window. A scenario whose ring has
    // overflowed is frozen (no more pops): its ring no longer holds a valid
    // deque, and the warp kernel recomputes it anyway; this keeps every pop
    // loop bounded.
    bool pf = (((int)(d.fx - d.pk) < 0) | (LCAP & (i >= d.fe))) & !d.ovf;
    while (__any_sync(0xffffffffu, pf)) {
        const uint32_t nh = RG::next(d.hoff);
        const int2 e = lds2(ring + nh);
        d.hoff = pf ? nh : d.hoff;
        d.fg = pf ? e.x : d.fg;
        d.fx = pf ? (uint32_t)e.y : d.fx;
        if (LCAP) d.fe = pf ? (int)((uint32_t)e.y & (K - 1)) + L + 1 : d.fe;
        pf = pf & (((int)(d.fx - d.pk) < 0) | (LCAP & (i >= d.fe)));
    }
    const int gi = d.fg + ci;
    if (PRED) *argmin = (int)(d.fx & (K - 1));   // the optimal predecessor, before the push
    if (!PUSH) return gi;
    const uint32_t x = d.pk + xi;               // K * (P(i) + Q) + i
    bool pb = (PRED ? d.bg > gi : d.bg >= gi) & !d.ovf;
    if (!GENERAL) {
        // back: drop entries not smaller than gi (the front is smaller)
        while (__any_sync(0xffffffffu, pb)) {
            const uint32_t bp = RG::prev(d.boff);
            const int below = lds1(ring + bp);
            d.boff = pb ? bp : d.boff;
            d.bg = pb ? below : d.bg;
            pb = pb & (PRED ? below > gi : below >= gi);
        }
        d.boff = RG::next(d.boff);
        // the new back slot is the front's: the ring already holds R entries
        d.ovf |= d.boff == d.hoff;
    } else {
        // back pops may reach the front: the new entry then becomes the front
        bool empty = false;
        while (__any_sync(0xffffffffu, pb)) {
            const bool emp = d.boff == d.hoff;
            const uint32_t bp = RG::prev(d.boff);
            const int below = lds1(ring + bp);
            empty |= pb & emp;
            d.boff = pb ? bp : d.boff;
            d.bg = pb ? below : d.bg;
            pb = pb & !emp & (PRED ? below > gi : below >= gi);
        }
        d.boff = RG::next(d.boff);
        d.ovf |= (d.boff == d.hoff) & !empty;
        d.hoff = empty ? d.boff : d.hoff;
        d.fg = empty ? gi : d.fg;
        d.fx = empty ? x : d.fx;
        if (LCAP) d.fe = empty ? i + L + 1 : d.fe;
    }
    // On overflow this store overwrites the front slot; the front itself
    // is held in registers and the scenario is frozen and set aside.
    sts2(ring + d.boff, gi, (int)x);
    d.bg = gi;
    return gi;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block reduction of (sum, infeasible count, status) and one atomic per block.
__device__ __forceinline__ void block_accumulate(long long sum, unsigned inf, unsigned status,
                                                 unsigned long long *acc)
{
    __shared__ long long s_sum[32];
    __shared__ unsigned s_inf[32], s_st[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    sum = warp_sum_ll(sum);
    inf = __reduce_add_sync(0xffffffffu, inf);
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0) { s_sum[w] = sum; s_inf[w] = inf; s_st[w] = status; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        sum = lane < nw ? s_sum[lane] : 0;
        inf = lane < nw ? s_inf[lane] : 0;
        status = lane < nw ? s_st[lane] : 0;
        sum = warp_sum_ll(sum);
        inf = __reduce_add_sync(0xffffffffu, inf);
        status = __reduce_or_sync(0xffffffffu, status);
        if (lane == 0) {
            if (sum) atomicAdd(acc + ACC_SUM, (unsigned long long)sum);
            if (inf) atomicAdd(acc + ACC_INFEASIBLE, (unsigned long long)inf);
            if (status) atomicOr(acc + ACC_STATUS, (unsigned long long)status);
        }
    }
}

// Positions of one prefetch block. GUARD: the block may run past n; the last
// position reads f(n) instead of pushing. `tab` reads the tour table; the
// block's first row carries the host's flag for a C_i <= 0 inside the block.
template <typename DT, int SPT, int R, int T, bool LCAP, bool GUARD, bool GENERAL, bool PRED, typename TB>
__device__ __forceinline__ void walk_steps(Deque (&d)[SPT], const uint32_t (&ring)[SPT], const int (&q)[kPrefetch][SPT],
                                           const TB &tab, int i0, int n, uint32_t K, uint32_t QK, int L, int Q,
                                           int (&out)[SPT], int16_t *pred, long long ldp)
{
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
        const int i = i0 + u;
        if (GUARD && i > n) break;
        const int ci = tab.c(i);
        const uint32_t xi = QK + (uint32_t)i;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            int p = 0;
            if (!GUARD || i < n) dq_step<R, T, LCAP, true, GENERAL, PRED>(d[j], ring[j], q[u][j], i, ci, K, xi, L, Q, &p);
            else out[j] = dq_step<R, T, LCAP, false, GENERAL, PRED>(d[j], ring[j], q[u][j], i, ci, K, xi, L, Q, &p);
            if (PRED && pred) pred[(long long)(i - 1) * ldp + j] = (int16_t)p;
        }
    }
}

template <typename DT, int SPT, int R, int T, bool LCAP, bool GUARD, bool PRED, typename TB>
__device__ __forceinline__ void walk_block(Deque (&d)[SPT], const uint32_t (&ring)[SPT], const int (&q)[kPrefetch][SPT],
                                           const TB &tab, int i0, int n, uint32_t K, uint32_t QK, int L, int Q,
                                           int (&out)[SPT], int16_t *pred, long long ldp)
{
    if (tab.row(i0) & kRowFlagNonPositive)
        walk_steps<DT, SPT, R, T, LCAP, GUARD, true, PRED>(d, ring, q, tab, i0, n, K, QK, L, Q, out, pred, ldp);
    else
        walk_steps<DT, SPT, R, T, LCAP, GUARD, false, PRED>(d, ring, q, tab, i0, n, K, QK, L, Q, out, pred, ldp);
}

// Demands of positions i0 .. i0 + kPrefetch - 1. Positions past n re-read row
// n (in bounds, unused), which keeps the loads free of branches.
template <typename DT, int SPT, bool CLAMP = true, typename TB>
__device__ __forceinline__ void prefetch_block(const char *base, const TB &tab, int i0, int n, uint32_t ldb,
                                               bool full, int nvalid, unsigned long long *status,
                                               int (&q)[kPrefetch][SPT])
{
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
        const int i = CLAMP ? min(i0 + u, n) : i0 + u;
        if (!index_ok(i >= 1 && i <= n, status)) {
#pragma unroll
            for (int j = 0; j < SPT; ++j) q[u][j] = 0;
            continue;
        }
        const int row = tab.row(i) & kRowMask;
        if (!index_ok(row < n, status)) {
#pragma unroll
            for (int j = 0; j < SPT; ++j) q[u][j] = 0;
            continue;
        }
        load_demands<DT, SPT>(base, row, ldb, full, nvalid, q[u]);
    }
}

// The walk of one thread: SPT adjacent scenarios s_first.. of one tour whose
// table is read through `tab` (TabGlobal or TabShared); the rings start at
// shared address `rings`. Writes f(n) of feasible scenarios to out_cost (if
// given), returns the sum of those costs, and passes every scenario it sets
// aside to `set_aside(s)`. Threads with no scenario (s_first >= S) walk
// column 0 and report nothing: every lane must take part in the pop votes.
template <typename DT, int SPT, int R, int T, bool LCAP, typename SetAside, bool PRED = false, typename TB>
__device__ __forceinline__ long long split_thread(const void *demand, long long ld, long long S, long long s_first,
                                                  int n, int Q, int L, uint32_t K, int g0, uint32_t rings,
                                                  TB tab, int tid, int32_t *out_cost, SetAside set_aside,
                                                  unsigned long long *status, int16_t *pred_base = nullptr,
                                                  long long ldp = 0)
{
    using RG = Ring<R, T>;
    const long long rem = S - s_first;
    const bool full = rem >= SPT;
    const int nvalid = rem >= SPT ? SPT : (int)(rem > 0 ? rem : 0);
    const uint32_t ldb = (uint32_t)(ld * (long long)sizeof(DT));
    const char *base = reinterpret_cast<const char *>(demand) + (nvalid ? s_first : 0) * (long long)sizeof(DT);
    const uint32_t QK = (uint32_t)Q * K;
    // Route recovery runs with one scenario per thread; a thread without a
    // scenario writes no predecessors.
    static_assert(!PRED || SPT == 1, "predecessor output needs one scenario per thread");
    int16_t *pred = PRED && nvalid ? pred_base + s_first : nullptr;

    Deque d[SPT];
    uint32_t ring[SPT];
    int out[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        ring[j] = rings + (uint32_t)j * R * T * 8;
        d[j].hoff = d[j].boff = (uint32_t)tid * 8u;
        d[j].fg = d[j].bg = g0;
        d[j].fx = QK;                               // x(0) = K * (0 + Q) + 0
        d[j].fe = L + 1;
        d[j].pk = 0;
        d[j].qmax = 0;
        d[j].ovf = false;
        out[j] = 0;
        sts2(ring[j] + d[j].hoff, g0, (int)QK);
    }

    int qa[kPrefetch][SPT], qb[kPrefetch][SPT];
    prefetch_block<DT, SPT>(base, tab, 1, n, ldb, full, nvalid, status, qa);
    int i0 = 1;
    // Double blocks whose positions, and those of the next prefetch, are all
    // below n: no guards or clamps.
    for (; i0 + 3 * kPrefetch - 1 < n; i0 += 2 * kPrefetch) {
        prefetch_block<DT, SPT, false>(base, tab, i0 + kPrefetch, n, ldb, full, nvalid, status, qb);
        walk_block<DT, SPT, R, T, LCAP, false, PRED>(d, ring, qa, tab, i0, n, K, QK, L, Q, out, pred, ldp);
        prefetch_block<DT, SPT, false>(base, tab, i0 + 2 * kPrefetch, n, ldb, full, nvalid, status, qa);
        walk_block<DT, SPT, R, T, LCAP, false, PRED>(d, ring, qb, tab, i0 + kPrefetch, n, K, QK, L, Q, out, pred, ldp);
    }
    // The remaining positions i0 .. n (qa holds i0 .. i0 + kPrefetch - 1).
    for (; i0 <= n; i0 += 2 * kPrefetch) {
        prefetch_block<DT, SPT>(base, tab, i0 + kPrefetch, n, ldb, full, nvalid, status, qb);
        walk_block<DT, SPT, R, T, LCAP, true, PRED>(d, ring, qa, tab, i0, n, K, QK, L, Q, out, pred, ldp);
        if (i0 + kPrefetch > n) break;
        prefetch_block<DT, SPT>(base, tab, i0 + 2 * kPrefetch, n, ldb, full, nvalid, status, qa);
        walk_block<DT, SPT, R, T, LCAP, true, PRED>(d, ring, qb, tab, i0 + kPrefetch, n, K, QK, L, Q, out, pred, ldp);
    }

    long long sum = 0;
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        if (j >= nvalid) continue;
        const long long s = s_first + j;
        if (d[j].ovf || d[j].qmax > (uint32_t)Q) {
            // deque too small, a demand above Q, or a negative demand: the
            // warp kernel evaluates (and classifies) this scenario
            set_aside(s);
            continue;
        }
        sum += out[j];
        if (out_cost) out_cost[s] = out[j];
    }
    return sum;
}

#ifndef CVRPSD_D1_TPSM
#define CVRPSD_D1_TPSM 0
#endif
template <int T>
constexpr int d1_min_blocks() { return CVRPSD_D1_TPSM > 0 ? CVRPSD_D1_TPSM / T : 1; }

template <typename DT, int SPT, int R, int T, bool LCAP, bool PRED = false>
__global__ void __launch_bounds__(T, d1_min_blocks<T>()) split_deque_kernel(SplitParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];   // SPT rings of R*T*8 bytes
    const int n = p.n;
    const int tid = threadIdx.x;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    // The tour table stays in global memory (L1-resident, one broadcast per
    // read): shared memory holds only the rings, which leaves room for more
    // resident blocks.
    const TabGlobal tab{reinterpret_cast<const int *>(p.tab)};
    const long long s_first = ((long long)blockIdx.x * T + tid) * SPT;
    unsigned long long *acc = p.acc;
    int32_t *list = p.ovf_list;
    const long long S = p.S;
    auto set_aside = [acc, list, S](long long s) {
        const unsigned long long idx = atomicAdd(acc + ACC_OVERFLOW, 1ull);
        if (index_ok(idx < (unsigned long long)S, acc + ACC_STATUS)) list[idx] = (int32_t)s;
    };
    const long long sum = split_thread<DT, SPT, R, T, LCAP, decltype(set_aside), PRED>(
        p.demand, p.ld, p.S, s_first, n, p.Q, p.L, p.K, p.g0, sbase, tab, tid, p.out_cost, set_aside,
        p.acc + ACC_STATUS, p.pred, p.ldp);
    block_accumulate(sum, 0u, 0u, p.acc);
}

}  // namespace cvrpsd
