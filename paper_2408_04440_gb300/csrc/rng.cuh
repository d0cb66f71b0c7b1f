// rng.cuh -- the counter-based normal generator of the library (device
// code shared by the sampler and the emulation nugget): Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, SC'11) at counter {p mod 2^32, p >> 32,
// column, stream id}, key {seed mod 2^32, seed >> 32}; two 53-bit uniforms
// u1 in (0,1], u2 in [0,1); Box-Muller gives rows 2p (cosine) and 2p+1 (sine).
#pragma once
#include <stdint.h>

namespace {

__device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Normals of pair p (rows 2p, 2p+1) of column col, written at z[0], z[1].
__device__ inline void normal_pair(uint64_t seed, uint32_t stream_id, long p, int col, int nrows, double *z) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t c[4] = {(uint32_t)((uint64_t)p & 0xffffffffu), (uint32_t)((uint64_t)p >> 32), (uint32_t)col,
                   stream_id};
  philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  uint64_t a = ((uint64_t)c[0] << 21) | (uint64_t)(c[1] >> 11);
  uint64_t b = ((uint64_t)c[2] << 21) | (uint64_t)(c[3] >> 11);
  double u1 = ((double)a + 1.0) * 0x1.0p-53;
  double u2 = (double)b * 0x1.0p-53;
  double rad = sqrt(-2.0 * log(u1));
  double th = two_pi * u2;
  z[0] = rad * cos(th);
  if (2 * p + 1 < nrows) z[1] = rad * sin(th);
}

}  // namespace
