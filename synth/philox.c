/*
 * Philox4x32-10 words for a grid of counters (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011): the same function
 * as synth/rng.py's philox4x32_10, in C so that full-size scenario matrices
 * (10^9 counters) are generated in seconds. Input synthesis only; it holds
 * none of the Split's arithmetic.
 *
 * For every index row r < ni and scenario column j < ns, the counter is
 * (s[j], index[r], domain, 0) and the key (k0, k1); words 0 and 1 of the
 * output block go to w0[r * ns + j] and w1[r * ns + j].
 */
#include <stdint.h>

static void philox_block(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;    /* Weyl key increments */
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];   /* round multipliers */
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)p1;
        c[3] = (uint32_t)p0;
        c[0] = n0;
        c[2] = n2;
    }
}

void synth_philox_words(const int64_t *s, int64_t ns, const int64_t *index, int64_t ni, uint32_t domain,
                        uint32_t k0, uint32_t k1, uint32_t *w0, uint32_t *w1)
{
    for (int64_t r = 0; r < ni; ++r) {
        for (int64_t j = 0; j < ns; ++j) {
            uint32_t c[4] = {(uint32_t)s[j], (uint32_t)index[r], domain, 0u};
            philox_block(c, k0, k1);
            w0[r * ns + j] = c[0];
            w1[r * ns + j] = c[1];
        }
    }
}
