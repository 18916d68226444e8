// Counter-based Gaussian test matrices on the device (Algorithm 4.1 step 1).
//
// Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw ("Parallel
// random numbers: as easy as 1, 2, 3", SC'11): ten rounds over a 4 x 32-bit
// counter with a 2 x 32-bit key; each round forms the 64-bit products of
// counter words 0 and 2 with 0xD2511F53 and 0xCD9E8D57 and remixes
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
// advances by (0x9E3779B9, 0xBB67AE85) between rounds.  Uniforms are
// (2 (x >> 9) + 1) 2^-24, in (0, 1) and exact in float32; normals come from
// the Box-Muller transform.  Element (i, j) of a drawn matrix uses counter
// (j / 4, i, stream, 0) and takes output j % 4.
#pragma once

#include <stdint.h>

namespace rsvd {

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
}

__device__ __forceinline__ float bits_to_uniform(uint32_t x) {
  return __uint2float_rn(((x >> 9) << 1) | 1u) * 5.9604644775390625e-08f;  // * 2^-24, exact
}

// Four standard normals for counter (g, i, stream, 0).
__device__ __forceinline__ float4 gaussian4(uint2 key, uint32_t g, uint32_t i, uint32_t stream) {
  const uint4 w = philox4x32_10(make_uint4(g, i, stream, 0u), key);
  const float u0 = bits_to_uniform(w.x), u1 = bits_to_uniform(w.y);
  const float u2 = bits_to_uniform(w.z), u3 = bits_to_uniform(w.w);
  const float r01 = sqrtf(-2.0f * logf(u0));
  const float r23 = sqrtf(-2.0f * logf(u2));
  float s01, c01, s23, c23;
  sincospif(2.0f * u1, &s01, &c01);
  sincospif(2.0f * u3, &s23, &c23);
  return make_float4(r01 * c01, r01 * s01, r23 * c23, r23 * s23);
}

}  // namespace rsvd
