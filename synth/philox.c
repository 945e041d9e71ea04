/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), written from its published
 * definition: ten rounds of two 32x32->64 multiplies with the Weyl key bump.
 *
 * Input generation only: this file holds no arithmetic of the GEMM method.
 *
 * Word i of a stream is lane (i % 4) of Philox(counter, key) with
 *   counter = { lo32(i / 4), hi32(i / 4), stream, 0 },  key = { lo32(seed), hi32(seed) }.
 */
#include <stdint.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Fill out[0..n) with words first_word .. first_word+n-1 of stream `stream`. */
void synth_philox_fill(uint64_t seed, uint32_t stream, uint64_t first_word, uint64_t n, uint32_t* out) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t i = 0;
    while (i < n) {
        uint64_t w = first_word + i;
        uint64_t blk = w >> 2;
        uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), stream, 0u};
        uint32_t r[4];
        synth_philox4x32_10(ctr, key, r);
        for (uint32_t lane = (uint32_t)(w & 3u); lane < 4u && i < n; ++lane, ++i) out[i] = r[lane];
    }
}
