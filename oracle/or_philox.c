/* CPU oracle (test infrastructure only): Philox-4x32-10 counter-based
 * generator, written from its published definition (Salmon, Moraes, Dror,
 * Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Sec. 4.2):
 * ten rounds of two 32x32->64 multiplications with multipliers 0xD2511F53
 * and 0xCD9E8D57, key schedule bumped by the Weyl constants 0x9E3779B9 and
 * 0xBB67AE85 between rounds. */
#include "or_internal.h"

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double or_rnd(uint32_t seed, uint32_t kind, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    uint32_t ctr[4] = {a, b, c, d >> 2}, key[2] = {seed, kind}, out[4];
    or_philox(ctr, key, out);
    return (double)(out[d & 3u] >> 8) * (1.0 / 16777216.0);
}

void or_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    or_philox(ctr, key, out);
}

double or_uniform(uint32_t seed, uint32_t kind, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    return or_rnd(seed, kind, a, b, c, d);
}
