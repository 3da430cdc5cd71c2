// FP64 -> FP16 rounding shared by the FP16 store, its right-hand sides and the
// symmetric store's FP16 lo term.
#pragma once
#include <stdint.h>

namespace pide {

// fp16 bits of v * 2^-k, rounded to nearest even from v's FP64 bits; zero and
// FP64 subnormals give a signed zero, values beyond 65504 saturate to 65504.
__device__ __forceinline__ uint16_t f16_bits_scaled(double v, int k) {
  const uint64_t x = (uint64_t)__double_as_longlong(v);
  const uint16_t sign = (uint16_t)((x >> 48) & 0x8000u);
  const int eb = (int)((x >> 52) & 0x7FF);
  if (eb == 0) return sign;
  if (eb == 0x7FF) return (uint16_t)(sign | 0x7BFFu);
  const int E = eb - 1023 - k;                   // v * 2^-k = m * 2^(E - 52)
  if (E > 15) return (uint16_t)(sign | 0x7BFFu);
  const uint64_t m = (x & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  // normal: q = m / 2^42 in [2^10, 2^11], bits = ((E + 14) << 10) + q (a carry
  // to 2^11 moves into the exponent); subnormal: q = m / 2^(28 - E), quantum 2^-24
  const int shift = E >= -14 ? 42 : 28 - E;
  if (shift > 53) return sign;                   // below half the smallest subnormal
  uint64_t q = m >> shift;
  const uint64_t rest = m & ((1ull << shift) - 1);
  const uint64_t half = 1ull << (shift - 1);
  if (rest > half || (rest == half && (q & 1u))) ++q;
  uint32_t bits = (uint32_t)q + (E >= -14 ? (uint32_t)(E + 14) << 10 : 0u);
  if (bits > 0x7BFFu) bits = 0x7BFFu;
  return (uint16_t)(sign | bits);
}

}  // namespace pide
