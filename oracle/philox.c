/*
 * Oracle -- TEST INFRASTRUCTURE ONLY.
 * Philox4x32-10 counter-based generator, written from its published definition
 * (J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11, Sec. 4): ten rounds of two 32x32->64 multiplies with the
 * multipliers 0xD2511F53 / 0xCD9E8D57, the counter words permuted and xor-ed with
 * the key, and the key bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85
 * between rounds.  Pinned by the authors' known-answer vectors in the tests.
 */
#include "oracle.h"

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) orc_philox_block(ctr + 4 * i, key + 2 * i, out + 4 * i);
}
