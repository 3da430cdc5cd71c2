// FP64 -> FP16 rounding shared by the FP16 store, its right-hand sides and the
// symmetric store's FP16 lo term.
#pragma once
#include <stdint.h>

namespace pide {

// fp16 bits of v * 2^-k, rounded to nearest even from v's FP64 bits; zero and
// FP64 subnormals give a signed zero, values beyond 65504 saturate to 65504.
__device__ __forceinline__ uint16_t f16_bits_scaled_any(double v, int k) {
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

// The same, with the common case -- a normal FP16 result -- on 32-bit integer
// operations: the 10 fraction bits are FP64 fraction bits 51..42 (bits 19..10
// of the high word), the rounding bit is fraction bit 41 (bit 9) and the
// sticky bits are everything below it; other cases take the general routine.
__device__ __forceinline__ uint16_t f16_bits_scaled(double v, int k) {
  const uint64_t x = (uint64_t)__double_as_longlong(v);
  const uint32_t xh = (uint32_t)(x >> 32), xl = (uint32_t)x;
  const int eb = (int)((xh >> 20) & 0x7FFu);
  const int E = eb - 1023 - k;
  if (eb == 0 || eb == 0x7FF || E < -14 || E > 15) return f16_bits_scaled_any(v, k);
  uint32_t q = ((xh >> 10) & 0x3FFu) | 0x400u;
  const uint32_t rbit = (xh >> 9) & 1u;
  const uint32_t sticky = (xh & 0x1FFu) | xl;
  q += rbit & ((sticky != 0u ? 1u : 0u) | (q & 1u));
  uint32_t bits = q + ((uint32_t)(E + 14) << 10);
  if (bits > 0x7BFFu) bits = 0x7BFFu;
  return (uint16_t)(((xh >> 16) & 0x8000u) | bits);
}

}  // namespace pide
