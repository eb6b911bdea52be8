// Host construction of the per-tour position table read by every Split kernel.
#pragma once

#include <stdint.h>
#include <stdio.h>

#include <vector>

#include "../../include/cvrpsd.h"
#include "kernels.h"

namespace cvrpsd {

#ifndef CVRPSD_PREFETCH
#define CVRPSD_PREFETCH 8
#endif
constexpr int kPrefetch = CVRPSD_PREFETCH;   // tour positions per prefetch block of the deque kernels

// Set in tab[i0 - 1].row, for the first position i0 = 1 + m * kPrefetch of
// each block, when some position i of that block with i < n has C_i <= 0:
// only such a block can see the deque emptied by a new entry.
constexpr int32_t kRowFlagNonPositive = 1 << 30;
constexpr int32_t kRowMask = kRowFlagNonPositive - 1;

inline uint32_t key_scale(int n)
{
    uint32_t K = 1;
    while (K <= (uint32_t)n) K <<= 1;
    return K;
}

// Validates the tour (a permutation of 1..n) and the distances it uses (>= 0)
// and fills tab[0..n): row of sigma_i and
//   C_i = c(sigma_i, 0) + c(0, sigma_{i+1}) - c(sigma_i, sigma_{i+1})   (i < n)
//   C_n = D[n] + c(sigma_n, 0),  D[n] = sum_{t<n} c(sigma_t, sigma_{t+1}),
// with g0 = c(0, sigma_1). Checks that every value the kernels form fits
// int32. Returns 0 or an error code, with a message in err.
inline int fill_tour_table(const int32_t *tour, int n, const int32_t *dist, int Q, TourStep *tab, int32_t *g0,
                           char *err, size_t errlen)
{
    if (!tour || !dist) {
        snprintf(err, errlen, "tour and dist are required");
        return CVRPSD_ERR_ARG;
    }
    const long long N1 = (long long)n + 1;
    std::vector<unsigned char> seen((size_t)n + 1, 0);
    for (int k = 0; k < n; ++k) {
        const int c = tour[k];
        if (c < 1 || c > n) {
            snprintf(err, errlen, "tour[%d] = %d is not a customer id in 1..%d", k, c, n);
            return CVRPSD_ERR_ARG;
        }
        if (seen[c]) {
            snprintf(err, errlen, "customer %d appears twice in the tour", c);
            return CVRPSD_ERR_ARG;
        }
        seen[c] = 1;
    }
    long long singles = 0, Dn = 0, maxc = 0;
    for (int k = 0; k < n; ++k) {
        const int c = tour[k];
        const long long out0 = dist[c], back = dist[(long long)c * N1];
        const long long nxt = k + 1 < n ? dist[(long long)c * N1 + tour[k + 1]] : 0;
        if (out0 < 0 || back < 0 || nxt < 0) {
            snprintf(err, errlen, "negative distance at tour position %d", k + 1);
            return CVRPSD_ERR_ARG;
        }
        singles += out0 + back;
        Dn += nxt;
        if (out0 > maxc) maxc = out0;
        if (back > maxc) maxc = back;
        if (nxt > maxc) maxc = nxt;
    }
    // |g| <= singles + D[n] + max c; every intermediate is bounded by that sum.
    if (singles + Dn + 3 * maxc >= (1LL << 30)) {
        snprintf(err, errlen, "route costs up to %lld do not fit the int32 arithmetic", singles + Dn + 3 * maxc);
        return CVRPSD_ERR_OVERFLOW;
    }
    const long long K = key_scale(n);
    if ((long long)(Q + 1LL) * K + n >= (1LL << 31)) {
        snprintf(err, errlen, "Q = %d too large for n = %d (need (Q+1)*%lld + n < 2^31)", Q, n, K);
        return CVRPSD_ERR_UNSUPPORTED;
    }
    for (int k = 0; k < n; ++k) {
        const int c = tour[k];
        tab[k].row = c - 1;
        if (k + 1 < n) {
            const int d = tour[k + 1];
            tab[k].c = (int32_t)(dist[(long long)c * N1] + dist[d] - dist[(long long)c * N1 + d]);
        } else {
            tab[k].c = (int32_t)(Dn + dist[(long long)c * N1]);
        }
    }
    for (int b = 0; b < n; b += kPrefetch) {
        bool nonpos = false;
        for (int k = b; k < b + kPrefetch && k < n - 1; ++k) nonpos |= tab[k].c <= 0;
        if (nonpos) tab[b].row |= kRowFlagNonPositive;
    }
    *g0 = dist[tour[0]];
    return CVRPSD_OK;
}

}  // namespace cvrpsd
