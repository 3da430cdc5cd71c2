// Double-float arithmetic on the integer and FP32 pipes: FP64 values split
// into two floats (47 significant bits), error-free products (FMA) and sums
// (Knuth's two-sum), and the FP64 formula of the Eq. (3) stencil for the nodes
// whose inputs fall outside the split's range.  Shared by the refinement
// residual (residual_df.cu) and the batched plans' residual (batched.cu).
#pragma once

#include "common.cuh"

namespace pide {
namespace {

// x = h + l with h = x truncated to 24 significant bits and l = the next 23
// bits (47 in all): integer operations and one FP32 subtraction.  Returns
// the binary64 exponent field E of x.  Inputs with E < 920 (|x| < 2^-103,
// including 0) give h = l = 0; the split is exact to 47 bits for
// 920 <= E <= 1150 (|x| < 2^128); above that the caller takes the FP64 route.
// With sticky = true the dropped low bits set the last bit of l (round to
// odd), so that a later rounding of h + l to 8 or 24 bits equals the
// rounding of x itself.
template <bool sticky>
__device__ __forceinline__ uint32_t split47(double x, float& h, float& l) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
  // the exponent field's low 9 bits and the top 23 fraction bits, shifted onto
  // binary32's fields; E - 896 rebiases 1023 -> 127 (adding 128 is the same
  // modulo 512)
  const uint32_t t = __funnelshift_l(lo, hi, 3);
  const uint32_t hb = ((t + 0x40000000u) & 0x7FFFFFFFu) | (hi & 0x80000000u);
  // l: the 29 fraction bits below h, top 23 of them, as 2^(e_h - 23) * q / 2^23
  const uint32_t base = (hb & 0xFF800000u) - 0x0B800000u;
  uint32_t q = (lo >> 6) & 0x007FFFFFu;
  if (sticky) q |= (lo & 0x3Fu) ? 1u : 0u;
  const float hh = __uint_as_float(hb);
  const float ll = __fsub_rn(__uint_as_float(base | q), __uint_as_float(base));
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const bool tiny = e < 920u;
  h = tiny ? 0.f : hh;
  l = tiny ? 0.f : ll;
  return e;
}

// As split47, with inputs at or above 2^128 (and Inf, NaN) marked as h = NaN:
// a stencil that touches one gives a NaN result and takes the FP64 route.
__device__ __forceinline__ void split_marked(double x, float& h, float& l) {
  float hh, ll;
  const uint32_t e = split47<false>(x, hh, ll);
  h = e > 1150u ? __int_as_float(0x7FC00000) : hh;
  l = ll;
}

// Exponent-field limits of the fast route.  A node is evaluated in
// double-float when none of its inputs reaches 2^128 (E <= 1150) and its own
// scale max(|f_p|, |u_p|) is at least 2^-60 (E >= 963): the inputs below
// 2^-103 that the split drops then change r by at most 2^-102, within the
// 2^-42 (|f_p| + |u_p| + ...) error bound.  Other nodes take the FP64 formula.
constexpr uint32_t E_SPLIT_MAX = 1150u, E_NODE_MIN = 963u;

// (sh, sl) += (ah, al); two-sum of the high parts, low parts added.
__device__ __forceinline__ void df_add(float& sh, float& sl, float ah, float al) {
  const float s = __fadd_rn(sh, ah);
  const float v = __fsub_rn(s, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(ah, v));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(al, e));
}

// (sh, sl) += (wh + wl)(uh + ul); the product's error term from an FMA.
__device__ __forceinline__ void df_fma(float& sh, float& sl, float wh, float wl, float uh,
                                       float ul) {
  const float ph = __fmul_rn(wh, uh);
  float pl = __fmaf_rn(wh, uh, -ph);
  pl = __fmaf_rn(wh, ul, pl);
  pl = __fmaf_rn(wl, uh, pl);
  df_add(sh, sl, ph, pl);
}

// bfloat16 of s + e rounded to nearest even, for s = fl(s + e) and
// |e| <= ulp(s) / 2: s's own rounding is right unless s sits exactly half-way
// between two bfloat16 values, where the sign of e decides.
__device__ __forceinline__ __nv_bfloat16 bf16_of_pair(float s, float e) {
  uint32_t x = __float_as_uint(s);
  if ((x & 0xFFFFu) == 0x8000u && e != 0.f)
    x += (((__float_as_uint(e) ^ x) >> 31) != 0u) ? 0xFFFFFFFFu : 1u;
  return __float2bfloat16_rn(__uint_as_float(x));
}

// The FP64 formula for one node (out-of-range inputs).  Not inlined, so that
// the fast route's warps never issue its FP64 instructions.
__device__ __noinline__ double residual_node_fp64(const double* __restrict__ bc,
                                                  const double* __restrict__ uc,
                                                  const double* __restrict__ w4,
                                                  const double* __restrict__ lift, int n, int mx,
                                                  int plane, int p) {
  const int c = p % mx, pp = plane == n ? p : p % plane;
  double r = lift ? bc[p] + (lift[p] - uc[p]) : bc[p] - uc[p];
  if (c > 0) r = fma(w4[p], uc[p - 1], r);
  if (c < mx - 1) r = fma(w4[n + p], uc[p + 1], r);
  if (pp >= mx) r = fma(w4[2 * n + p], uc[p - mx], r);
  if (pp + mx < plane) r = fma(w4[3 * n + p], uc[p + mx], r);
  if (p >= plane) r = fma(w4[4 * (size_t)n + p], uc[p - plane], r);
  if (p + plane < n) r = fma(w4[5 * (size_t)n + p], uc[p + plane], r);
  return r;
}

__device__ __noinline__ void split_f64_slow(double r, float& s, float& e) {
  s = __double2float_rn(r);
  e = __double2float_rn(r - (double)s);
}

__device__ __noinline__ __nv_bfloat16 bf16_of_f64_slow(double v) { return __double2bfloat16(v); }

__device__ __forceinline__ bool is_zero(double x) {
  return ((uint64_t)__double_as_longlong(x) << 1) == 0;
}

// bfloat16 of x rounded to nearest even with integer operations (binary64
// exponent field E: 897..1150 exactly; below 2^-134 the result is a signed
// zero); the rest through CUDA's conversion, outside the inlined code.
__device__ __forceinline__ __nv_bfloat16 bf16_of_f64(double v) {
  const uint64_t x = (uint64_t)__double_as_longlong(v);
  const uint32_t hi = (uint32_t)(x >> 32);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint16_t sign = (uint16_t)((hi >> 16) & 0x8000u);
  if (e < 889u) return __ushort_as_bfloat16(sign);
  if (e < 897u || e > E_SPLIT_MAX) return bf16_of_f64_slow(v);
  // 45 dropped fraction bits: above half up, exactly half to even
  uint32_t r = ((e - 896u) << 7) | (uint32_t)((x >> 45) & 0x7Fu);
  const uint64_t rest = x & 0x1FFFFFFFFFFFull;
  const uint64_t half = 0x100000000000ull;
  if (rest > half || (rest == half && (r & 1u))) r += 1u;
  return __ushort_as_bfloat16((uint16_t)(sign | r));
}

}  // namespace
}  // namespace pide
