// Host-side rounding of FP32 weights to the tensor-core operand formats
// (BF16 and E4M3), shared by the weight-image builder and its CPU test.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

namespace spider {

// round-to-nearest-even FP32 -> BF16 on the host
inline uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// FP32 -> E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; largest
// finite 448, no infinities), round to nearest even, saturating at 448.
inline uint8_t to_e4m3(float f) {
  uint8_t sign = std::signbit(f) ? 0x80 : 0;
  double a = std::fabs((double)f);
  if (!(a == a)) return 0x7F;                        // NaN
  if (a >= 448.0) return sign | 0x7E;                // saturate
  // candidates on the E4M3 grid around a: spacing 2^(e-3) for a in [2^e, 2^(e+1)), e >= -6;
  // below 2^-6 the grid is the subnormal one, spacing 2^-9
  int e = 0;
  if (a > 0) {
    std::frexp(a, &e);                               // a = m 2^e, m in [0.5, 1)
    e -= 1;                                          // a in [2^e, 2^(e+1))
  }
  if (a == 0 || e < -6) e = -6;
  const double q = std::ldexp(1.0, e - 3);          // grid spacing
  double k = std::floor(a / q);
  const double rem = a - k * q;
  if (rem > 0.5 * q || (rem == 0.5 * q && std::fmod(k, 2.0) != 0)) k += 1;
  const double v = k * q;                            // rounded magnitude (may reach 2^(e+1))
  if (v == 0) return sign;
  if (v < std::ldexp(1.0, -6)) return sign | (uint8_t)(v / std::ldexp(1.0, -9));   // subnormal
  int ev = 0;
  const double mv = std::frexp(v, &ev);              // v = mv 2^ev, mv in [0.5, 1)
  const int E = ev - 1 + 7;                          // biased exponent
  const int Mt = (int)std::lround((mv * 2.0 - 1.0) * 8.0);
  if (E > 15 || (E == 15 && Mt > 6)) return sign | 0x7E;
  return sign | (uint8_t)(E << 3) | (uint8_t)Mt;
}

}  // namespace spider
