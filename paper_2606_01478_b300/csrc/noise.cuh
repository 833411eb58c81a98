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

// Rounds FIRST..9 of Philox4x32-10 on the counter block c.
template <int FIRST>
__device__ __forceinline__ void philox_rounds(uint32_t c[4], const uint2* keys) {
#pragma unroll
  for (int r = FIRST; r < 10; ++r) {
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

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], const uint2* keys) {
  philox_rounds<0>(c, keys);
}

// The blocks of the counters (lo, hi, k, 0), k = 0, 1, 2, ..., of one sample id.
// In the first round only the product k 0xCD9E8D57 depends on k: the product of
// lo and the key words it meets are fixed, and k 0xCD9E8D57 grows by the
// multiplier at each step (a 64-bit add in place of a multiply).  The words equal
// philox4x32_10 of each counter.
struct PhiloxSteps {
  uint32_t x0, x2, x3;      // hi ^ key0.x, high(lo 0xD2511F53) ^ key0.y, low(lo 0xD2511F53)
  unsigned long long km;    // k 0xCD9E8D57 for the next block
  __device__ __forceinline__ PhiloxSteps(uint32_t lo, uint32_t hi, const uint2* keys) {
    unsigned long long p0;
    asm("mul.wide.u32 %0, %1, 0xD2511F53;" : "=l"(p0) : "r"(lo));
    const uint2 k = keys[0];
    x0 = hi ^ k.x;
    x2 = (uint32_t)(p0 >> 32) ^ k.y;
    x3 = (uint32_t)p0;
    km = 0ull;
  }
  // the block of the next counter (k = 0 first)
  __device__ __forceinline__ void next(uint32_t c[4], const uint2* keys) {
    c[0] = (uint32_t)(km >> 32) ^ x0;
    c[1] = (uint32_t)km;
    c[2] = x2;
    c[3] = x3;
    philox_rounds<1>(c, keys);
    km += 0xCD9E8D57ull;
  }
};

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  uint2 keys[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) keys[r] = philox_round_key(k0, k1, r);
  philox4x32_10(c, keys);
}

// -2 ln u for u = ((w >> 9) + 0.5) 2^-23.  Away from 1 the hardware base-2
// logarithm (lg2.approx: absolute error about 2^-22 for arguments in [0.5, 1),
// a few ulp relative below) gives it as -2 ln 2 log2 u; within 2^-8 of 1, where
// that absolute error would dominate the small result, v = 1 - u is exact
// (both are multiples of 2^-24) and -ln(1 - v) = v + v^2/2 + v^3/3 + ... is
// summed to the cubic term (relative remainder below v^3 / 3 < 2^-25).  At the
// switch, -2 ln u = 0.0078 and the logarithm's error moves sqrt(-2 ln u) by
// under 2e-6; the root then carries that error alone.
__device__ __forceinline__ float minus_two_log_uniform(float u) {
  const float v = 1.f - u;
  float l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(u));
  const float near_one = 2.f * v * fmaf(v, fmaf(v, 1.f / 3.f, 0.5f), 1.f);
  return v < 0.00390625f ? near_one : -1.38629436111989061f * l2;  // 2 ln 2
}

// Two standard normals from two words: u = ((w >> 9) + 0.5) 2^-23 (exact),
// r = sqrt(-2 ln u1), angle 2 pi u2 (evaluated as 2 pi u2 - pi, in [-pi, pi)).
__device__ __forceinline__ float2 box_muller(uint32_t w1, uint32_t w2) {
  // the float with a zero exponent and mantissa w >> 9 is 1 + (w >> 9) 2^-23;
  // subtracting 1 - 2^-24 is exact and leaves ((w >> 9) + 0.5) 2^-23
  const float u1 = __uint_as_float((w1 >> 9) + 0x3F800000u) - 0.99999994039535522f;
  const float r = sqrt_approx(minus_two_log_uniform(u1));
  // 2 pi u2 - pi from m2 = 1 + (w2 >> 9) 2^-23 = u2 + 1 - 2^-24 in one multiply-add:
  // 2 pi m2 - (2 pi (1 - 2^-24) + pi), the constant rounded to float (error 1.4e-7;
  // 2 pi and pi as their floats)
  const float m2 = __uint_as_float((w2 >> 9) + 0x3F800000u);
  float s, c;
  __sincosf(fmaf(6.28318530717958648f, m2, -9.42477784853068f), &s, &c);
  return make_float2(-r * c, -r * s);
}

}  // namespace noise
}  // namespace cf
