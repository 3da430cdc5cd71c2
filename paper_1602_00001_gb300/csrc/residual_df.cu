// The refinement residual of Eq. (3) without the FP64 pipe.
//
// r = f - L u = b (+ lift) - u_p + sum_q w_pq u_q is the only FP64 arithmetic
// left in a refinement sweep, and GB300 runs FP64 at a small fraction of its
// FP32 rate: evaluated with FP64 instructions the stencil is bound by the
// FP64 pipe at ~4x the time its 18 bytes per node take from HBM.  Here every
// FP64 input is split into two floats with integer operations (x = h + l,
// 47 significant bits) and the stencil is evaluated in double-float
// arithmetic: error-free products (FMA) and error-free sums (Knuth's
// two-sum), so the computed residual carries an absolute error of about
// 2^-45 (|u_p| + sum_q w_pq |u_q|), far below the error of the BF16/FP8
// stored inverse it feeds and below the 1e-6 accuracy the refinement targets.
// Values outside the float range of the split (|x| < 2^-103 or >= 2^128,
// except 0) send their node back to the FP64 formula.
//
// Boundary neighbours carry zero weights in the split weight arrays, so the
// kernel loads every neighbour from a clamped index without branches.
#include "common.cuh"

namespace pide {
namespace {

// x = h + l with h = x truncated to 24 significant bits and l = the next 23
// bits (47 in all); x = 0 gives h = l = 0.  Integer operations and one FP32
// subtraction.  Returns false when x != 0 lies outside 2^-103 <= |x| < 2^128.
// With sticky = true the dropped low bits set the last bit of l (round to
// odd), so that a later rounding of h + l to 8 or 24 bits equals the
// rounding of x itself.
template <bool sticky>
__device__ __forceinline__ bool split47(double x, float& h, float& l) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
  // exponent field E (11 bits) and the top 23 fraction bits, shifted so that
  // E's low 9 bits land on binary32's exponent field; E - 896 rebiases
  // 1023 -> 127 (adding 128 is the same modulo 512)
  const uint32_t t = __funnelshift_l(lo, hi, 3);
  const uint32_t hb = ((t + 0x40000000u) & 0x7FFFFFFFu) | (hi & 0x80000000u);
  // l: the 29 fraction bits below h, top 23 of them, as 2^(e_h - 23) * q / 2^23
  const uint32_t base = (hb & 0xFF800000u) - 0x0B800000u;
  uint32_t q = (lo >> 6) & 0x007FFFFFu;
  if (sticky) q |= (lo & 0x3Fu) ? 1u : 0u;
  const float hh = __uint_as_float(hb);
  const float ll = __fsub_rn(__uint_as_float(base | q), __uint_as_float(base));
  const bool zero = (bits << 1) == 0;
  h = zero ? 0.f : hh;
  l = zero ? 0.f : ll;
  const uint32_t e = (hi >> 20) & 0x7FFu;
  return zero || (e - 920u <= 230u);
}

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

// bfloat16 bits of s + e rounded to nearest even, for s = fl(s + e) and
// |e| <= ulp(s) / 2: s's own rounding is right unless s sits exactly half-way
// between two bfloat16 values, where the sign of e decides.
__device__ __forceinline__ __nv_bfloat16 bf16_of_pair(float s, float e) {
  uint32_t x = __float_as_uint(s);
  if ((x & 0xFFFFu) == 0x8000u && e != 0.f)
    x += (((__float_as_uint(e) ^ x) >> 31) != 0u) ? 0xFFFFFFFFu : 1u;
  return __float2bfloat16_rn(__uint_as_float(x));
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <int RF>
__device__ __forceinline__ void store_r(void* R, size_t idx, float s, float e, float isc) {
  if constexpr (RF == RF_BF16) {
    reinterpret_cast<__nv_bfloat16*>(R)[idx] = bf16_of_pair(s, e);
  } else if constexpr (RF == RF_F32) {
    reinterpret_cast<float*>(R)[idx] = s;
  } else {
    reinterpret_cast<__nv_fp8_e4m3*>(R)[idx] = __nv_fp8_e4m3(s * isc);
  }
}

// Weights of the residual split into float pairs; zero toward boundary
// neighbours (their values enter through the lift).  wh[p] = (W, E, S, N).
__global__ void wsplit_kernel(const double* __restrict__ w4, int n, int mx,
                              float4* __restrict__ wh, float4* __restrict__ wl) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int c = p % mx;
    const double w[4] = {c > 0 ? w4[p] : 0.0, c < mx - 1 ? w4[n + p] : 0.0,
                         p >= mx ? w4[2 * n + p] : 0.0, p + mx < n ? w4[3 * n + p] : 0.0};
    float h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] = __double2float_rn(w[k]);
      l[k] = __double2float_rn(w[k] - (double)h[k]);
    }
    wh[p] = make_float4(h[0], h[1], h[2], h[3]);
    wl[p] = make_float4(l[0], l[1], l[2], l[3]);
  }
}

constexpr int DF_COLS = 2;   // columns per thread: the weights are loaded once for both

// r = f - u_p + sum_q w_pq u_q for columns blockIdx.y * DF_COLS + k, written to R
// (BF16 rounded to nearest from the pair, FP32, or e4m3 after the column scale);
// optionally max |r| per column into colmax_r.
template <int RF>
__global__ void __launch_bounds__(256) residual_df_kernel(
    const double* __restrict__ b, const double* __restrict__ u, int n, int mx, int B, int ldr,
    const float4* __restrict__ wh4, const float4* __restrict__ wl4,
    const double* __restrict__ w4, const double* __restrict__ lift, void* __restrict__ R,
    const float* __restrict__ col_scale, double* __restrict__ colmax_r, int track,
    const uint32_t* __restrict__ flags) {
  __shared__ float red[DF_COLS][8];
  if (flags && flags[FLAG_DONE]) return;
  const int cbase = blockIdx.y * DF_COLS;
  float isc[DF_COLS], mxr[DF_COLS];
#pragma unroll
  for (int k = 0; k < DF_COLS; ++k) {
    isc[k] = (RF == RF_E4M3 && cbase + k < B) ? 1.0f / col_scale[cbase + k] : 1.0f;
    mxr[k] = 0.f;
  }
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const float4 wh = wh4[p], wl = wl4[p];
    const int pw = p > 0 ? p - 1 : p, pe = p + 1 < n ? p + 1 : p;
    const int ps = p >= mx ? p - mx : p, pn = p + mx < n ? p + mx : p;
    float lh = 0.f, ll = 0.f;
    const bool lok = lift ? split47<false>(lift[p], lh, ll) : true;
#pragma unroll
    for (int k = 0; k < DF_COLS; ++k) {
      const int col = cbase + k;
      if (col >= B) break;
      const double* uc = u + (size_t)col * n;
      const double bp = b[(size_t)col * n + p];
      const double u0 = uc[p], uw = uc[pw], ue = uc[pe], us = uc[ps], un = uc[pn];
      float bh, bl, h0, l0, hw, lw, he, le, hs, ls, hn, ln;
      bool ok = split47<false>(bp, bh, bl);
      ok &= split47<false>(u0, h0, l0);
      ok &= split47<false>(uw, hw, lw);
      ok &= split47<false>(ue, he, le);
      ok &= split47<false>(us, hs, ls);
      ok &= split47<false>(un, hn, ln);
      float s, e;
      if (ok && lok) {
        float sh = bh, sl = bl;
        if (lift) df_add(sh, sl, lh, ll);
        df_add(sh, sl, -h0, -l0);
        df_fma(sh, sl, wh.x, wl.x, hw, lw);
        df_fma(sh, sl, wh.y, wl.y, he, le);
        df_fma(sh, sl, wh.z, wl.z, hs, ls);
        df_fma(sh, sl, wh.w, wl.w, hn, ln);
        s = __fadd_rn(sh, sl);
        e = __fsub_rn(sl, __fsub_rn(s, sh));
      } else {
        // outside the split's range: the FP64 formula
        const int c = p % mx;
        double r = lift ? bp + (lift[p] - u0) : bp - u0;
        if (c > 0) r = fma(w4[p], uw, r);
        if (c < mx - 1) r = fma(w4[n + p], ue, r);
        if (p >= mx) r = fma(w4[2 * n + p], us, r);
        if (p + mx < n) r = fma(w4[3 * n + p], un, r);
        s = __double2float_rn(r);
        e = __double2float_rn(r - (double)s);
      }
      store_r<RF>(R, (size_t)col * ldr + p, s, e, isc[k]);
      if (track) mxr[k] = fmaxf(mxr[k], fabsf(s));
    }
  }
  if (track) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < DF_COLS; ++k) {
      float v = mxr[k];
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < DF_COLS && cbase + (int)threadIdx.x < B) {
      float v = 0.f;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v = fmaxf(v, red[threadIdx.x][q]);
      atomic_max_nonneg(&colmax_r[cbase + threadIdx.x], (double)v);
    }
  }
}

// Prep for BF16 right-hand sides, forward mode: R = bf16(b + lift), rounded to
// nearest from the exact pair (the sticky split makes the 47-bit pair round
// like the FP64 value); optionally max |f| per column.
__global__ void prep_df_bf16_kernel(const double* __restrict__ b, int n, int ldr,
                                    const double* __restrict__ lift,
                                    __nv_bfloat16* __restrict__ R, double* __restrict__ colmax_b,
                                    int track) {
  __shared__ float red[8];
  const int col = blockIdx.y;
  const double* bc = b + (size_t)col * n;
  float mx = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const double bp = bc[p];
    const double lp = lift ? lift[p] : 0.0;
    float bh, bl, lh = 0.f, ll = 0.f, s;
    __nv_bfloat16 q;
    if (split47<true>(bp, bh, bl) && (!lift || split47<true>(lp, lh, ll))) {
      if (lift) df_add(bh, bl, lh, ll);
      s = __fadd_rn(bh, bl);
      q = bf16_of_pair(s, __fsub_rn(bl, __fsub_rn(s, bh)));
    } else {
      const double f = bp + lp;
      s = __double2float_rn(f);
      q = __double2bfloat16(f);
    }
    R[(size_t)col * ldr + p] = q;
    if (track) mx = fmaxf(mx, fabsf(s));
  }
  if (track) {
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      float v = 0.f;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v = fmaxf(v, red[q]);
      atomic_max_nonneg(&colmax_b[col], (double)v);
    }
  }
}

}  // namespace

pide_status launch_wsplit(pide_ctx* c, cudaStream_t st) {
  const int g = (c->n + 255) / 256 < c->num_sms * 8 ? (c->n + 255) / 256 : c->num_sms * 8;
  wsplit_kernel<<<g > 0 ? g : 1, 256, 0, st>>>(c->w, c->n, c->mx, c->wsp, c->wsp + c->n);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_residual_df(pide_ctx* c, const double* b, const double* u, int B,
                               const double* lift, int rfmt, void* R, int ldr,
                               const float* col_scale, double* colmax_r, bool track,
                               const uint32_t* flags, cudaStream_t st) {
  if (B == 0) return PIDE_OK;
  int gx = (c->n + 255) / 256;
  if (gx > 1024) gx = 1024;
  const dim3 g(gx, (B + DF_COLS - 1) / DF_COLS, 1);
  const float4* wh = c->wsp;
  const float4* wl = c->wsp + c->n;
  const int t = track ? 1 : 0;
  switch (rfmt) {
    case RF_BF16: residual_df_kernel<RF_BF16><<<g, 256, 0, st>>>(b, u, c->n, c->mx, B, ldr, wh, wl, c->w, lift, R, col_scale, colmax_r, t, flags); break;
    case RF_F32: residual_df_kernel<RF_F32><<<g, 256, 0, st>>>(b, u, c->n, c->mx, B, ldr, wh, wl, c->w, lift, R, col_scale, colmax_r, t, flags); break;
    case RF_E4M3: residual_df_kernel<RF_E4M3><<<g, 256, 0, st>>>(b, u, c->n, c->mx, B, ldr, wh, wl, c->w, lift, R, col_scale, colmax_r, t, flags); break;
    default: return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_prep_df_bf16(pide_ctx* c, const double* b, int B, const double* lift,
                                bool track, cudaStream_t st) {
  if (B == 0) return PIDE_OK;
  int gx = (c->n + 255) / 256;
  if (gx > 1024) gx = 1024;
  prep_df_bf16_kernel<<<dim3(gx, B, 1), 256, 0, st>>>(b, c->n, c->ld, lift,
                                                      (__nv_bfloat16*)c->R,
                                                      c->colmax + c->ws_B, track ? 1 : 0);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

}  // namespace pide

// Test hook: the double-float residual written as FP32 to r_dev[B][n] (ld n).
extern "C" pide_status pide_selftest_residual_df(pide_handle h, const double* b_dev,
                                                 const double* u_dev, const double* g_dev,
                                                 float* r_dev, int32_t B, void* stream) {
  using namespace pide;
  if (!h || !b_dev || !u_dev || !r_dev || B < 0) {
    set_error("pide_selftest_residual_df: bad argument");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const double* lift = nullptr;
  if (g_dev) {
    PIDE_TRY(launch_lift(h, g_dev, st));
    lift = h->lift;
  }
  return launch_residual_df(h, b_dev, u_dev, B, lift, RF_F32, r_dev, h->n, nullptr, nullptr,
                            false, nullptr, st);
}
