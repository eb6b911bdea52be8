// Instantiations and launcher of the second deque walk (split_deque2.cuh).
// The template arguments are spread over translation units
// (CVRPSD_DEQUE2_PART) so that the build compiles them in parallel.
#include "split_deque2.cuh"

namespace cvrpsd {

cudaError_t dispatch_deque2_i16_cap_fast(const Walk2Params &p, const void *tab, const DequeShape &s, long long grid,
                                         cudaStream_t st);
cudaError_t dispatch_deque2_i16_nocap_fast(const Walk2Params &p, const void *tab, const DequeShape &s,
                                           long long grid, cudaStream_t st);
cudaError_t dispatch_deque2_general(const Walk2Params &p, const void *tab, int esize, bool lcap, bool nowrap,
                                    bool large, const DequeShape &s, long long grid, cudaStream_t st);
cudaError_t dispatch_deque2_i32(const Walk2Params &p, const void *tab, bool lcap, bool nowrap, bool large,
                                const DequeShape &s, long long grid, cudaStream_t st);

// A launch's parameters may take at most 32764 bytes.
static_assert(sizeof(TabParam<kTab2Large>) + sizeof(Walk2Params) <= 32764, "tour table too large for the parameters");

template <typename DT, int R, int T, bool LCAP, bool NOWRAP, int CAP>
static cudaError_t launch2(const Walk2Params &p, const void *tab, long long grid, cudaStream_t st)
{
    split_deque2_kernel<DT, R, T, LCAP, NOWRAP, CAP>
        <<<(unsigned)grid, T, 0, st>>>(p, *static_cast<const TabParam<CAP> *>(tab));
    return cudaGetLastError();
}

// One instantiation class: demand type, route-length cap, key range, table
// capacity. `shapes` lists the (threads, ring) pairs compiled for it; others
// fall back to (128, 16).
#define CVRPSD_D2_SHAPE(T_, R_)                                                                        \
    if (s.threads == T_ && s.ring == R_) return launch2<DT, R_, T_, LCAP, NOWRAP, CAP>(p, tab, grid, st);

template <typename DT, bool LCAP, bool NOWRAP, int CAP>
static cudaError_t dispatch_wide(const Walk2Params &p, const void *tab, const DequeShape &s, long long grid,
                                 cudaStream_t st)
{
    CVRPSD_D2_SHAPE(64, 8) CVRPSD_D2_SHAPE(64, 16) CVRPSD_D2_SHAPE(128, 8) CVRPSD_D2_SHAPE(128, 16)
    CVRPSD_D2_SHAPE(256, 8) CVRPSD_D2_SHAPE(256, 16)
    return cudaErrorInvalidValue;
}

template <typename DT, bool LCAP, bool NOWRAP, int CAP>
static cudaError_t dispatch_narrow(const Walk2Params &p, const void *tab, const DequeShape &s, long long grid,
                                   cudaStream_t st)
{
    CVRPSD_D2_SHAPE(128, 16)
    return cudaErrorInvalidValue;
}
#undef CVRPSD_D2_SHAPE

#if CVRPSD_DEQUE2_PART == 0
cudaError_t dispatch_deque2_i16_cap_fast(const Walk2Params &p, const void *tab, const DequeShape &s, long long grid,
                                         cudaStream_t st)
{ return dispatch_wide<int16_t, true, true, kTab2Small>(p, tab, s, grid, st); }

namespace {

// Keys K * (P + Q) + p and K * P(i) stay below 2^31 for every position a
// walk reaches before it freezes: without the clamp (int16) a bad demand can
// add up to 65535 once.
bool keys_fit(const SplitParams &p, int esize)
{
    const long long K = p.K, n = p.n, Q = p.Q;
    const long long last = esize == 2 ? 65535 : Q;
    return K * (n * Q + last + Q) + n < (1LL << 31);
}

// Picks the compiled kernel class of this Split and launches it.
cudaError_t route(const Walk2Params &w, const void *tab, const SplitParams &p, int esize, const DequeShape &s,
                  long long grid, cudaStream_t st)
{
    const bool lcap = p.L < p.n, nowrap = keys_fit(p, esize), large = p.n > kTab2Small;
    if (esize == 4) return dispatch_deque2_i32(w, tab, lcap, nowrap, large, s, grid, st);
    if (nowrap && !large) {
        cudaError_t e = lcap ? dispatch_deque2_i16_cap_fast(w, tab, s, grid, st)
                             : dispatch_deque2_i16_nocap_fast(w, tab, s, grid, st);
        if (e != cudaErrorInvalidValue) return e;
    }
    return dispatch_deque2_general(w, tab, esize, lcap, nowrap, large, s, grid, st);
}

// The shape that runs: the requested one if its class compiles it, else (128, 16).
DequeShape compiled_shape(const SplitParams &p, int esize, const DequeShape &s)
{
    const bool wide = esize == 2 && keys_fit(p, esize) && p.n <= kTab2Small;
    const bool listed = (s.threads == 64 || s.threads == 128 || s.threads == 256) && (s.ring == 8 || s.ring == 16);
    if (wide && listed) return DequeShape{s.threads, 1, s.ring};
    return DequeShape{128, 1, 16};
}

}  // namespace

bool deque2_supported(const SplitParams &p, int esize)
{
    if (p.pred || p.n > kTab2Large || p.n < 1) return false;
    if ((unsigned long long)p.ld * esize > 0xFFFFFFFFull) return false;   // 32-bit row pitch
    if ((unsigned long long)(p.n - 1) * (unsigned long long)p.ld * esize + (unsigned long long)p.S * esize >
        0xFFFFFFFFull)
        return false;
    return esize == 4 || p.Q < 32768;
}

cudaError_t launch_split_deque2(const SplitParams &p, const TourStep *tab, int esize, const DequeShape &shape,
                                int rounds, DequeShape *shape_ran, cudaStream_t stream)
{
    const DequeShape s = compiled_shape(p, esize, shape);
    if (shape_ran) *shape_ran = s;
    // The table as the kernel reads it, built in a host buffer large enough
    // for either capacity (passed by value as the launch's parameters).
    static thread_local TabParam<kTab2Large> big;
    static thread_local TabParam<kTab2Small> small;
    const bool large = p.n > kTab2Small;
    uint2 *e = large ? big.e : small.e;
    uint32_t *nonpos = large ? big.nonpos : small.nonpos;
    const size_t words = large ? sizeof(big.nonpos) / 4 : sizeof(small.nonpos) / 4;
    for (size_t k = 0; k < words; ++k) nonpos[k] = 0;
    const unsigned long long pitch = (unsigned long long)p.ld * esize;
    for (int k = 0; k < p.n; ++k) {
        e[k].x = (uint32_t)(tab[k].row & kRowMask);
        e[k].y = (uint32_t)tab[k].c;
        // Position k + 1 >= 2 with C_k > 0 and C_{k+1} > C_k: no back pops.
        if (k >= 1 && tab[k - 1].c > 0 && tab[k].c > tab[k - 1].c) e[k].x |= kTab2NoBack;
        // C_{k+1} <= 0 (k + 1 < n) marks its prefetch block.
        if (k + 1 < p.n && tab[k].c <= 0) {
            const int m = k / kPrefetch2;
            nonpos[m >> 5] |= 1u << (m & 31);
        }
    }
    Walk2Params w{};
    w.demand = p.demand;
    w.S = p.S;
    w.n = p.n;
    w.Q = p.Q;
    w.L = p.L;
    w.g0 = p.g0;
    w.K = p.K;
    w.out_cost = p.out_cost;
    w.acc = p.acc;
    w.ovf_list = p.ovf_list;
    w.status = p.acc + ACC_STATUS;
    w.pitch = (uint32_t)pitch;
    const long long tiles = (p.S + s.threads - 1) / s.threads;
    const long long grid = rounds > 0 ? (tiles + rounds - 1) / rounds : tiles;
    w.stride = grid * s.threads;
    return route(w, large ? (const void *)&big : (const void *)&small, p, esize, s, grid, stream);
}
#elif CVRPSD_DEQUE2_PART == 1
cudaError_t dispatch_deque2_i16_nocap_fast(const Walk2Params &p, const void *tab, const DequeShape &s,
                                           long long grid, cudaStream_t st)
{ return dispatch_wide<int16_t, false, true, kTab2Small>(p, tab, s, grid, st); }
#elif CVRPSD_DEQUE2_PART == 2
// Every other combination, with the (128, 16) shape only.
cudaError_t dispatch_deque2_general(const Walk2Params &p, const void *tab, int esize, bool lcap, bool nowrap,
                                    bool large, const DequeShape &s, long long grid, cudaStream_t st)
{
#define CVRPSD_D2_CLASS(DT_, LCAP_, NOWRAP_, CAP_)                                                     \
    if ((esize == (int)sizeof(DT_)) && lcap == LCAP_ && nowrap == NOWRAP_ && (CAP_ == kTab2Large) == large) \
        return dispatch_narrow<DT_, LCAP_, NOWRAP_, CAP_>(p, tab, s, grid, st);
    CVRPSD_D2_CLASS(int16_t, true, false, kTab2Small) CVRPSD_D2_CLASS(int16_t, false, false, kTab2Small)
    CVRPSD_D2_CLASS(int16_t, true, true, kTab2Large) CVRPSD_D2_CLASS(int16_t, false, true, kTab2Large)
    CVRPSD_D2_CLASS(int16_t, true, false, kTab2Large) CVRPSD_D2_CLASS(int16_t, false, false, kTab2Large)
#undef CVRPSD_D2_CLASS
    return cudaErrorInvalidValue;
}
#elif CVRPSD_DEQUE2_PART == 3
cudaError_t dispatch_deque2_i32(const Walk2Params &p, const void *tab, bool lcap, bool nowrap, bool large,
                                const DequeShape &s, long long grid, cudaStream_t st)
{
#define CVRPSD_D2_CLASS(LCAP_, NOWRAP_, CAP_)                                                          \
    if (lcap == LCAP_ && nowrap == NOWRAP_ && (CAP_ == kTab2Large) == large)                          \
        return dispatch_narrow<int32_t, LCAP_, NOWRAP_, CAP_>(p, tab, s, grid, st);
    CVRPSD_D2_CLASS(true, true, kTab2Small) CVRPSD_D2_CLASS(false, true, kTab2Small)
    CVRPSD_D2_CLASS(true, false, kTab2Small) CVRPSD_D2_CLASS(false, false, kTab2Small)
    CVRPSD_D2_CLASS(true, true, kTab2Large) CVRPSD_D2_CLASS(false, true, kTab2Large)
    CVRPSD_D2_CLASS(true, false, kTab2Large) CVRPSD_D2_CLASS(false, false, kTab2Large)
#undef CVRPSD_D2_CLASS
    return cudaErrorInvalidValue;
}
#endif

}  // namespace cvrpsd
