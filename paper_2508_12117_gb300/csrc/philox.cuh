// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based generator
// keying the Langevin noise and the minibatch permutation.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spider {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;
constexpr uint32_t kTagNoise = 0x4E4F4953u;    // 'NOIS'
constexpr uint32_t kTagFeistel = 0x46454953u;  // 'FEIS'

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += kPhiloxW0;
      k.y += kPhiloxW1;
    }
#ifdef __CUDA_ARCH__
    uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
#else
    uint64_t p0 = (uint64_t)kPhiloxM0 * c.x, p1 = (uint64_t)kPhiloxM1 * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// (floor(w / 2^9) + 1/2) * 2^-23, exact in FP32, inside (0, 1)
__device__ __forceinline__ float unit_from_word(uint32_t w) {
  return (float)(w >> 9) * 1.1920928955078125e-07f + 5.9604644775390625e-08f;
}

// Box-Muller: two words -> two standard normals
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb) {
  float u1 = unit_from_word(wa), u2 = unit_from_word(wb);
  float rad = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(rad * c, rad * s);
}

// s-th element of a keyed permutation of [0, n): balanced 4-round Feistel on
// 2h bits, round function = low h bits of Philox word 0 of (R, round, 0, 'FEIS'),
// cycle-walking back into range.  Returns -1 if the walk exceeds its bound.
__host__ __device__ __forceinline__ int64_t feistel_index(int64_t s, int64_t n, uint64_t seed) {
  int bits = 0;
  for (uint64_t v = (uint64_t)(n - 1); v; v >>= 1) ++bits;
  if (bits < 2) bits = 2;
  bits += bits & 1;
  const int h = bits / 2;
  const uint64_t mask = (1ull << h) - 1;
  const uint2 key = seed_key(seed);
  uint64_t x = (uint64_t)s;
  for (int walk = 0; walk < 4096; ++walk) {
    uint64_t L = x >> h, R = x & mask;
    for (int r = 0; r < 4; ++r) {
      uint4 w = philox4x32_10(make_uint4((uint32_t)R, (uint32_t)r, 0u, kTagFeistel), key);
      uint64_t F = (uint64_t)w.x & mask;
      uint64_t nl = R;
      R = L ^ F;
      L = nl;
    }
    x = (L << h) | R;
    if (x < (uint64_t)n) return (int64_t)x;
  }
  return -1;
}

}  // namespace spider
