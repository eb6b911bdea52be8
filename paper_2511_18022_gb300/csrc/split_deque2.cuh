// Scenario-parallel Split, second walk: the same monotone-deque recursion as
// split_deque.cuh (one thread per scenario, Section 3's scenario level;
// Eq. 1-3 through the separable segment cost, see there), with less fixed
// work per position. The walk is bound by instruction issue and by the
// integer ALU pipe (compares, selects, logic, which that pipe executes at
// half the issue rate), so every change below removes instructions from one
// of the two:
//
//  - The tour table is a kernel parameter (__grid_constant__), read at a
//    block-uniform index from the constant bank: no global table loads, and
//    the demand address is one wide multiply-add (row * pitch + column).
//  - int16 demands are read as unsigned 16-bit values. A demand above Q (a
//    negative one reads as >= 32768 > Q) expires every deque entry, the back
//    one included; the front walk notices when it would pass the back,
//    marks the scenario bad and freezes it. So the per-position clamp and
//    running maximum of the first walk are gone (int32 demands keep them).
//  - When n * Q * K + (Q + 1) * K + n < 2^31 (checked on the host), keys
//    never wrap and the capacity test is one signed compare (NOWRAP).
//  - A frozen scenario (ring overflow or a bad demand) only sets a flag that
//    the front and back tests carry; with rings of 16 or more and keys that
//    cannot wrap, a frozen lane instead keeps walking a consistent deque and
//    the tests carry no flag (fold_frozen).
//  - A front walk moves only the front slot and reads only keys; the new
//    front's (g, key) is read from its slot once the walk ends.
//  - Where C_{i-1} > 0 and C_i > C_{i-1}, no scenario can pop the deque's
//    back at position i (dq2_step gives the argument); the host marks those
//    positions and the walk skips the back test and its vote there.
//  - The rings are a static shared array (a slot's address is its masked
//    byte offset plus a constant), and with rings of 8 entries and 32
//    registers per thread the SM holds 2048 threads of the walk.
//  - The grid may be smaller than one thread per scenario: a thread then
//    walks scenarios s, s + G*T, ... (every thread of a block the same
//    number of times).
//  - The route-length test of the front and (rings of 16 or more) the
//    ring-overflow test of a push run once per span of two prefetch blocks
//    (8 positions), not per position: the front's position p is the low
//    bits of its key, and fronts only move to later positions, so no front
//    reaches its length limit inside a span that starts with every front
//    younger than L + 1 - 8 positions before the span's last position; a
//    ring that starts a span at most R - 8 entries full cannot fill inside
//    it (a position pushes once). A span where some lane of the warp fails
//    either test walks the exact per-position tests (rare: the mean window
//    is far shorter than L and the deque far shorter than the ring).
//
// Set-aside scenarios (ring too small, a demand above Q, a negative demand)
// go to the warp kernel exactly as before.
#pragma once

#include <stdint.h>

#include "deque2.h"
#include "kernels.h"
#include "split_deque.cuh"
#include "tour_table.h"

namespace cvrpsd {

struct Deque2 {
    int fg;          // front entry: g
    int fx;          // front key K * (P(p) + Q) + p
    int bg;          // back entry: g
    uint32_t h;      // byte offset of the front slot in the block's rings
    uint32_t b;      // byte offset of the back slot
    uint32_t pk;     // K * P(i)
    uint32_t qmax;   // int32 demands only: largest demand seen (unsigned)
    bool frozen;     // ring overflow or a bad demand: set aside, no more pops
};

// Signed capacity test of a key against K * P(i): wrapping difference, or a
// plain compare when keys cannot wrap.
template <bool NOWRAP>
__device__ __forceinline__ bool key_expired(int x, uint32_t pk)
{
    if (NOWRAP) return x < (int)pk;
    return (int)((uint32_t)x - pk) < 0;
}

// Whether the front of key x has passed its route-length limit at position
// i (its position p = x mod K, limit p + L + 1).
__device__ __forceinline__ bool front_too_long(int x, int i, uint32_t K, int L)
{
    return i >= (int)((uint32_t)x & (K - 1u)) + L + 1;
}

// Rings of 16 or more: the overflow test moves to the block; smaller rings
// test every push.
template <int R> __host__ __device__ constexpr bool block_ovf() { return R >= 16; }

// Frozen lanes that keep walking (keys that cannot wrap, rings of 16 or
// more): a frozen lane's result is discarded, so it only has to stay a
// consistent deque, and then the front and back tests need no frozen flag.
// A ring overflow restarts the deque from the entry just pushed (its slot is
// the one the push overwrote); a demand above Q leaves the front on the back
// entry. Either way every later front walk ends at the back (or freezes
// there again) and every back walk at the front, as for any other lane.
template <int R, bool NOWRAP> __host__ __device__ constexpr bool fold_frozen() { return NOWRAP && block_ovf<R>(); }

// One position. PUSH: candidate i enters (positions 1..n-1); the last
// position only reads the window minimum. GENERAL: some C_i <= 0 in this
// block, so back pops may empty the deque (see split_deque.cuh). LTEST: test
// the front's route-length limit; OVF: test the push for ring overflow.
template <int R, int T, bool LTEST, bool OVF, bool NOWRAP, bool CLAMP, bool PUSH, bool GENERAL>
__device__ __forceinline__ int dq2_step(Deque2 &d, uint32_t q, int i, int ci, uint32_t K, uint32_t xi, int L, int Q,
                                        uint32_t rs, bool noback)
{
    constexpr uint32_t kStride = T * 8u;
    constexpr uint32_t kMask = R * T * 8u - 1u;
    if (CLAMP) {
        d.qmax = max(d.qmax, q);
        q = min(q, (uint32_t)Q);
    }
    d.pk += q * K;
    bool pf = key_expired<NOWRAP>(d.fx, d.pk) | (LTEST && front_too_long(d.fx, i, K, L));
    if (!fold_frozen<R, NOWRAP>()) pf = pf & !d.frozen;
    // Front pops. The walk reads only the keys and moves h; the new front's
    // (g, key) is read once after it. Reaching the back entry with it expired
    // means a demand above Q (only possible without CLAMP): the scenario is
    // bad and frozen, its front left on the back entry. The slot at h always
    // holds the front (a frozen lane's overwritten slot included, which only
    // that lane reads).
    if (__any_sync(0xffffffffu, pf)) {
        do {
            const bool last = d.h == d.b;
            const uint32_t nh = (d.h + kStride) & kMask;
            const int key = lds1(rs + nh + 4u);
            if (!CLAMP && last && pf) {
                d.frozen = true;
                pf = false;
            }
            d.h = pf ? nh : d.h;
            pf = pf & (key_expired<NOWRAP>(key, d.pk) | (LTEST && front_too_long(key, i, K, L)));
        } while (__any_sync(0xffffffffu, pf));
        const int2 e = lds2(rs + d.h);
        d.fg = e.x;
        d.fx = e.y;
    }
    const int gi = d.fg + ci;
    if (!PUSH) return gi;
    const int x = (int)(d.pk + xi);       // K * (P(i) + Q) + i
    constexpr bool kFold = fold_frozen<R, NOWRAP>();
    // In a GENERAL block only the positions with C_i <= 0 need the back walk
    // that may empty the deque: with C_i > 0 the new value exceeds the
    // front's, so the back walk stops there as in any other block.
    if (!GENERAL || ci > 0) {
        if (!noback) {
            bool pb = (d.bg >= gi) & (kFold || !d.frozen);
            // Where the back can pop at all (C_i <= C_{i-1} or C_{i-1} <= 0),
            // nearly every warp pops at least once (lanes whose front did
            // not move pop the back whenever C_i <= C_{i-1}): the first step
            // runs without a vote.
            {
                const uint32_t bp = (d.b - kStride) & kMask;
                const int below = lds1(rs + bp);
                d.b = pb ? bp : d.b;
                d.bg = pb ? below : d.bg;
                pb = pb & (below >= gi);
            }
            while (__any_sync(0xffffffffu, pb)) {
                const uint32_t bp = (d.b - kStride) & kMask;
                const int below = lds1(rs + bp);
                d.b = pb ? bp : d.b;
                d.bg = pb ? below : d.bg;
                pb = pb & (below >= gi);
            }
        }
        d.b = (d.b + kStride) & kMask;
        if (OVF) {
            const bool ovf = d.b == d.h;            // the ring already held R entries
            d.frozen |= ovf;
            if (kFold && ovf) d.fg = gi, d.fx = x;
        }
    } else {
        bool pb = (d.bg >= gi) & (kFold || !d.frozen);
        bool empty = false;
        while (__any_sync(0xffffffffu, pb)) {
            const bool emp = d.b == d.h;
            const uint32_t bp = (d.b - kStride) & kMask;
            const int below = lds1(rs + bp);
            empty |= pb & emp;
            d.b = pb ? bp : d.b;
            d.bg = pb ? below : d.bg;
            pb = pb & !emp & (below >= gi);
        }
        d.b = (d.b + kStride) & kMask;
        if (empty) {
            d.h = d.b;
            d.fg = gi;
            d.fx = x;
        } else if (OVF) {
            const bool ovf = d.b == d.h;
            d.frozen |= ovf;
            if (kFold && ovf) d.fg = gi, d.fx = x;
        }
    }
    sts2(rs + d.b, gi, x);
    d.bg = gi;
    return gi;
}

template <typename DT> struct Dem2;
template <> struct Dem2<int16_t> { using T = unsigned short; };
template <> struct Dem2<int32_t> { using T = unsigned int; };

template <typename DT, typename TB>
__device__ __forceinline__ uint32_t load_dem2(const char *base, const TB &tab, int i, uint32_t pitch,
                                              int n, unsigned long long *status)
{
    if (!index_ok(i >= 1 && i <= n && i <= TB::kCap, status)) return 0u;
    const uint32_t row = tab.row(i);
    if (!index_ok(row < (uint32_t)n, status)) return 0u;
    return (uint32_t)__ldcs(reinterpret_cast<const typename Dem2<DT>::T *>(base + (unsigned long long)row * pitch));
}

// Positions i0 .. i0 + kPrefetch2 - 1 (GUARD: the block may reach past n).
template <typename DT, int R, int T, bool LTEST, bool OVF, bool NOWRAP, bool GUARD, bool GENERAL, typename TB>
__device__ __forceinline__ void walk2_steps(Deque2 &d, const uint32_t (&q)[kPrefetch2], const TB &tab,
                                            int i0, int n, uint32_t K, uint32_t QK, int L, int Q, uint32_t rs, int &out)
{
    constexpr bool CLAMP = sizeof(DT) == 4;
#pragma unroll
    for (int u = 0; u < kPrefetch2; ++u) {
        const int i = i0 + u;
        if (GUARD && i > n) break;
        const uint2 e = tab.entry(i);
        const int ci = (int)e.y;
        const bool noback = (e.x & kTab2NoBack) != 0;
        const uint32_t xi = QK + (uint32_t)i;
        if (!GUARD || i < n)
            dq2_step<R, T, LTEST, OVF, NOWRAP, CLAMP, true, GENERAL>(d, q[u], i, ci, K, xi, L, Q, rs, noback);
        else
            out = dq2_step<R, T, LTEST, OVF, NOWRAP, CLAMP, false, GENERAL>(d, q[u], i, ci, K, xi, L, Q, rs, noback);
    }
}

// Whether some lane of the warp needs the exact per-position tests in the
// SPAN positions from i0: its front may reach the route-length limit, or its
// ring may fill.
template <int R, int T, bool LCAP, bool NOWRAP, int SPAN>
__device__ __forceinline__ bool walk2_exact(const Deque2 &d, int i0, uint32_t K, int L)
{
    constexpr uint32_t kStride = T * 8u;
    constexpr uint32_t kMask = R * T * 8u - 1u;
    if (!LCAP && !block_ovf<R>()) return false;
    bool risk = false;
    if (LCAP) risk = (int)((uint32_t)d.fx & (K - 1u)) + L < i0 + SPAN - 1;
    if (block_ovf<R>()) risk |= ((d.b - d.h) & kMask) > (uint32_t)(R - SPAN - 1) * kStride;
    if (!fold_frozen<R, NOWRAP>()) risk = risk & !d.frozen;   // a frozen lane no longer pops
    return __any_sync(0xffffffffu, risk);
}

template <typename DT, int R, int T, bool LCAP, bool NOWRAP, bool GUARD, typename TB>
__device__ __forceinline__ void walk2_block(Deque2 &d, const uint32_t (&q)[kPrefetch2], const TB &tab,
                                            int i0, int n, uint32_t K, uint32_t QK, int L, int Q, uint32_t rs,
                                            bool exact, int &out)
{
    constexpr bool kBlockOvf = block_ovf<R>();
    const bool general = tab.general(i0);
    if (exact) {
        if (general)
            walk2_steps<DT, R, T, LCAP, true, NOWRAP, GUARD, true>(d, q, tab, i0, n, K, QK, L, Q, rs, out);
        else
            walk2_steps<DT, R, T, LCAP, true, NOWRAP, GUARD, false>(d, q, tab, i0, n, K, QK, L, Q, rs, out);
    } else {
        if (general)
            walk2_steps<DT, R, T, false, !kBlockOvf, NOWRAP, GUARD, true>(d, q, tab, i0, n, K, QK, L, Q, rs, out);
        else
            walk2_steps<DT, R, T, false, !kBlockOvf, NOWRAP, GUARD, false>(d, q, tab, i0, n, K, QK, L, Q, rs, out);
    }
}

template <typename DT, bool CLAMPI, typename TB>
__device__ __forceinline__ void prefetch2(const char *base, const TB &tab, int i0, int n, uint32_t pitch,
                                          unsigned long long *status, uint32_t (&q)[kPrefetch2])
{
#pragma unroll
    for (int u = 0; u < kPrefetch2; ++u)
        q[u] = load_dem2<DT>(base, tab, CLAMPI ? min(i0 + u, n) : i0 + u, pitch, n, status);
}

// The walk of one scenario (column s; a thread past S walks column 0 and
// reports nothing: every lane takes part in the votes). Returns f(n) or
// sets *aside.
template <typename DT, int R, int T, bool LCAP, bool NOWRAP, typename TB>
__device__ __forceinline__ int walk2_scenario(const Walk2Params &p, const TB &tab, long long s,
                                              uint32_t rs, uint32_t slot0, bool &aside)
{
    const int n = p.n, Q = p.Q, L = p.L;
    const uint32_t K = p.K;
    const uint32_t QK = (uint32_t)Q * K;
    const char *base = reinterpret_cast<const char *>(p.demand) + (s < p.S ? s : 0) * (long long)sizeof(DT);
    Deque2 d;
    d.h = d.b = slot0;
    d.fg = d.bg = p.g0;
    d.fx = (int)QK;                 // x(0) = K * (0 + Q) + 0
    d.pk = 0;
    d.qmax = 0;
    d.frozen = false;
    sts2(rs + slot0, p.g0, (int)QK);
    int out = 0;
    uint32_t qa[kPrefetch2], qb[kPrefetch2];
    const uint32_t pitch = p.pitch;
    unsigned long long *status = p.status;
    prefetch2<DT, true>(base, tab, 1, n, pitch, status, qa);
    int i0 = 1;
    // One exactness vote covers both prefetch blocks of an iteration.
    constexpr int kSpan = 2 * kPrefetch2;
    for (; i0 + 3 * kPrefetch2 - 1 < n; i0 += 2 * kPrefetch2) {
        prefetch2<DT, false>(base, tab, i0 + kPrefetch2, n, pitch, status, qb);
        const bool ex = walk2_exact<R, T, LCAP, NOWRAP, kSpan>(d, i0, K, L);
        walk2_block<DT, R, T, LCAP, NOWRAP, false>(d, qa, tab, i0, n, K, QK, L, Q, rs, ex, out);
        prefetch2<DT, false>(base, tab, i0 + 2 * kPrefetch2, n, pitch, status, qa);
        walk2_block<DT, R, T, LCAP, NOWRAP, false>(d, qb, tab, i0 + kPrefetch2, n, K, QK, L, Q, rs, ex, out);
    }
    for (; i0 <= n; i0 += 2 * kPrefetch2) {
        prefetch2<DT, true>(base, tab, i0 + kPrefetch2, n, pitch, status, qb);
        const bool ex = walk2_exact<R, T, LCAP, NOWRAP, kSpan>(d, i0, K, L);
        walk2_block<DT, R, T, LCAP, NOWRAP, true>(d, qa, tab, i0, n, K, QK, L, Q, rs, ex, out);
        if (i0 + kPrefetch2 > n) break;
        prefetch2<DT, true>(base, tab, i0 + 2 * kPrefetch2, n, pitch, status, qa);
        walk2_block<DT, R, T, LCAP, NOWRAP, true>(d, qb, tab, i0 + kPrefetch2, n, K, QK, L, Q, rs, ex, out);
    }
    aside = d.frozen || d.qmax > (uint32_t)Q;
    return out;
}

// The walk is compiled for 2048 resident threads per SM (the most an SM
// holds): 32 registers a thread, and with rings of 8 its blocks fit the
// shared memory too. Full occupancy measured 4 % faster than the compiler's
// own choice (40 registers, 12 blocks of 128). Rings of 16 fit fewer blocks
// by shared memory (6 of 256 threads), but giving those kernels the 40
// registers that would allow measured 16 % slower (the compiler then moves
// table work from the uniform datapath to the vector pipes).
constexpr int kD2ThreadsPerSM = 2048;
template <int R, int T>
constexpr int d2_min_blocks() { return kD2ThreadsPerSM / T; }

template <typename DT, int R, int T, bool LCAP, bool NOWRAP, int CAP>
__global__ void __launch_bounds__(T, d2_min_blocks<R, T>()) split_deque2_kernel(const Walk2Params p, const __grid_constant__ TabParam<CAP> tab)
{
    // Rings [R][T] of (g, key) slots: thread t's slot k is at byte
    // (k * T + t) * 8, so a warp's accesses never conflict.
    __shared__ __align__(16) int2 rings[R * T];
    const int tid = threadIdx.x;
    const uint32_t rs = (uint32_t)__cvta_generic_to_shared(rings);
    const uint32_t slot0 = (uint32_t)tid * 8u;
    long long sum = 0;
    // Every thread of a block runs the same number of rounds (the test is
    // on the block's first scenario), so block-wide code after the loop is
    // reached by all.
    for (long long sb = (long long)blockIdx.x * T; sb < p.S; sb += p.stride) {
        const long long s = sb + tid;
        bool aside = false;
        const int c = walk2_scenario<DT, R, T, LCAP, NOWRAP>(p, tab, s, rs, slot0, aside);
        if (s < p.S) {
            if (aside) {
                const unsigned long long idx = atomicAdd(p.acc + ACC_OVERFLOW, 1ull);
                if (index_ok(idx < (unsigned long long)p.S, p.status)) p.ovf_list[idx] = (int32_t)s;
            } else {
                sum += c;
                if (p.out_cost) p.out_cost[s] = c;
            }
        }
    }
    block_accumulate(sum, 0u, 0u, p.acc);
}

}  // namespace cvrpsd
