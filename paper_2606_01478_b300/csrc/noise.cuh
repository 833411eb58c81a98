// Sampling noise shared by the sampling rollouts and the MPPI update: the
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller
// transform.  Both kernels draw the normals of sample id (lo, hi) at step k
// from counter (lo, hi, k, 0) under the 64-bit seed as key, so the update
// regenerates exactly the noise the rollouts used.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace cf {
namespace noise {

// Round r of Philox4x32-10 xors the key (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85)
// into the high product halves.  The round keys depend on the seed alone, so a
// kernel can build the ten once and reuse them for every draw.
__device__ __forceinline__ uint2 philox_round_key(uint32_t k0, uint32_t k1, uint32_t r) {
  return make_uint2(k0 + r * 0x9E3779B9u, k1 + r * 0xBB67AE85u);
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], const uint2* keys) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint2 k = keys[r];
    // one widening multiply gives both halves of each 32 x 32 -> 64-bit product
    unsigned long long p0, p1;
    asm("mul.wide.u32 %0, %1, 0xD2511F53;" : "=l"(p0) : "r"(c[0]));
    asm("mul.wide.u32 %0, %1, 0xCD9E8D57;" : "=l"(p1) : "r"(c[2]));
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k.x, n2 = hi0 ^ c[3] ^ k.y;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  uint2 keys[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) keys[r] = philox_round_key(k0, k1, r);
  philox4x32_10(c, keys);
}

// Two standard normals from two words: u = ((w >> 9) + 0.5) 2^-23 (exact),
// r = sqrt(-2 ln u1), angle 2 pi u2 (evaluated as 2 pi u2 - pi, in [-pi, pi)).
__device__ __forceinline__ float2 box_muller(uint32_t w1, uint32_t w2) {
  // the float with a zero exponent and mantissa w >> 9 is 1 + (w >> 9) 2^-23;
  // subtracting 1 - 2^-24 is exact and leaves ((w >> 9) + 0.5) 2^-23
  const float u1 = __uint_as_float((w1 >> 9) + 0x3F800000u) - 0.99999994039535522f;
  const float u2 = __uint_as_float((w2 >> 9) + 0x3F800000u) - 0.99999994039535522f;
  const float r = sqrt_approx(-2.f * logf(u1));  // within 1 ulp of the rounded root
  float s, c;
  __sincosf(fmaf(6.28318530717958648f, u2, -3.14159265358979324f), &s, &c);
  return make_float2(-r * c, -r * s);
}

}  // namespace noise
}  // namespace cf
