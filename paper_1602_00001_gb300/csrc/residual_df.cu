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
#include "df_arith.cuh"

namespace pide {
namespace {

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <int RF>
__device__ __forceinline__ void store_r(void* R, size_t idx, float s, float e, float isc) {
  if constexpr (RF == RF_BF16) {
    reinterpret_cast<__nv_bfloat16*>(R)[idx] = bf16_of_pair(s, e);
  } else if constexpr (RF == RF_F32) {
    reinterpret_cast<float*>(R)[idx] = s;
  } else if constexpr (RF == RF_F16) {
    // isc a power of two: s * isc exact; saturating at 65504
    reinterpret_cast<__half*>(R)[idx] = __float2half_rn(fminf(fmaxf(s * isc, -65504.0f), 65504.0f));
  } else {
    reinterpret_cast<__nv_fp8_e4m3*>(R)[idx] = __nv_fp8_e4m3(s * isc);
  }
}

// Weights of the residual split into float pairs; zero toward boundary
// neighbours (their values enter through the lift).  wh[p] = (W, E, S, N),
// wl[p] the low parts, and for a 3-D grid wz[p] = (D hi, U hi, D lo, U lo).
__global__ void wsplit_kernel(const double* __restrict__ w4, int n, int mx, int plane,
                              float4* __restrict__ wh, float4* __restrict__ wl,
                              float4* __restrict__ wz) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int c = p % mx, pp = p % plane;
    const double w[6] = {c > 0 ? w4[p] : 0.0, c < mx - 1 ? w4[n + p] : 0.0,
                         pp >= mx ? w4[2 * n + p] : 0.0, pp + mx < plane ? w4[3 * n + p] : 0.0,
                         (wz && p >= plane) ? w4[4 * (size_t)n + p] : 0.0,
                         (wz && p + plane < n) ? w4[5 * (size_t)n + p] : 0.0};
    float h[6], l[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      h[k] = __double2float_rn(w[k]);
      l[k] = __double2float_rn(w[k] - (double)h[k]);
    }
    wh[p] = make_float4(h[0], h[1], h[2], h[3]);
    wl[p] = make_float4(l[0], l[1], l[2], l[3]);
    if (wz) wz[p] = make_float4(h[4], h[5], l[4], l[5]);
  }
}

// Launch shapes of the shared-memory kernel (PIDE_TUNE_RESID_SHAPE): SM_NR
// nodes per thread, a tile of 256 * SM_NR nodes per block.
constexpr int SM_NRS[4] = {4, 8, 2, 16};
constexpr size_t SMEM_MAX = 48 * 1024;   // larger halos (very wide grids) take the register kernel
constexpr size_t SMEM_MAX_3D = 200 * 1024;  // 3-D halos (one z-plane each side), opt-in shared memory

__device__ __forceinline__ int clampi(int q, int n) { return q < 0 ? 0 : (q >= n ? n - 1 : q); }

// Register kernel (grids too wide for the shared-memory halo):
// r = f - u_p + sum_q w_pq u_q for nodes p0 .. p0 + DF_NR - 1 (flat index; a
// grid row's end needs no test since the weights toward boundary nodes are
// zero) of columns blockIdx.y * DF_COLS + k, written to R (BF16 rounded to
// nearest from the pair, FP32, or e4m3 after the column scale); optionally
// max |r| per column into colmax_r.
template <int RF, int DF_NR, int DF_COLS>
__global__ void __launch_bounds__(256, 2) residual_df_reg_kernel(
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
    isc[k] = ((RF == RF_E4M3 || RF == RF_F16) && cbase + k < B) ? 1.0f / col_scale[cbase + k] : 1.0f;
    mxr[k] = 0.f;
  }
  const int stride = DF_NR * gridDim.x * blockDim.x;
  for (int p0 = DF_NR * (blockIdx.x * blockDim.x + threadIdx.x); p0 < n; p0 += stride) {
    float4 wh[DF_NR], wl[DF_NR];
    float lh[DF_NR], ll[DF_NR];
    uint32_t el[DF_NR];
#pragma unroll
    for (int k = 0; k < DF_NR; ++k) {
      const int p = clampi(p0 + k, n);
      wh[k] = wh4[p];
      wl[k] = wl4[p];
      el[k] = lift ? split47<false>(lift[p], lh[k], ll[k]) : 0u;
      if (!lift) lh[k] = ll[k] = 0.f;
    }
#pragma unroll
    for (int cc = 0; cc < DF_COLS; ++cc) {
      const int col = cbase + cc;
      if (col >= B) break;
      const double* uc = u + (size_t)col * n;
      const double* bc = b + (size_t)col * n;
      // row values u[p0 - 1 .. p0 + DF_NR], the rows below and above, and b
      float rh[DF_NR + 2], rl[DF_NR + 2], sh_[DF_NR], sl_[DF_NR], nh[DF_NR], nl[DF_NR];
      float bh[DF_NR], bl[DF_NR];
      uint32_t er[DF_NR + 2], es[DF_NR], en[DF_NR], eb[DF_NR];
#pragma unroll
      for (int j = 0; j < DF_NR + 2; ++j) er[j] = split47<false>(uc[clampi(p0 - 1 + j, n)], rh[j], rl[j]);
#pragma unroll
      for (int k = 0; k < DF_NR; ++k) {
        es[k] = split47<false>(uc[clampi(p0 + k - mx, n)], sh_[k], sl_[k]);
        en[k] = split47<false>(uc[clampi(p0 + k + mx, n)], nh[k], nl[k]);
        eb[k] = split47<false>(bc[clampi(p0 + k, n)], bh[k], bl[k]);
      }
#pragma unroll
      for (int k = 0; k < DF_NR; ++k) {
        const int p = p0 + k;
        if (p >= n) break;
        const uint32_t emax = max(max(max(er[k], er[k + 1]), max(er[k + 2], es[k])),
                                  max(max(en[k], eb[k]), el[k]));
        const uint32_t enode = max(max(er[k + 1], eb[k]), el[k]);
        float s, e;
        if (emax <= E_SPLIT_MAX && enode >= E_NODE_MIN) {
          float ah = bh[k], al = bl[k];
          if (lift) df_add(ah, al, lh[k], ll[k]);
          df_add(ah, al, -rh[k + 1], -rl[k + 1]);
          df_fma(ah, al, wh[k].x, wl[k].x, rh[k], rl[k]);
          df_fma(ah, al, wh[k].y, wl[k].y, rh[k + 2], rl[k + 2]);
          df_fma(ah, al, wh[k].z, wl[k].z, sh_[k], sl_[k]);
          df_fma(ah, al, wh[k].w, wl[k].w, nh[k], nl[k]);
          s = __fadd_rn(ah, al);
          e = __fsub_rn(al, __fsub_rn(s, ah));
        } else {
          split_f64_slow(residual_node_fp64(bc, uc, w4, lift, n, mx, n, p), s, e);
        }
        store_r<RF>(R, (size_t)col * ldr + p, s, e, isc[cc]);
        if (track) mxr[cc] = fmaxf(mxr[cc], fabsf(s));
      }
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

// Packed pairs: lane x of every float2 belongs to column 2y, lane y to
// column 2y + 1, so that one FADD2 / FMUL2 / FFMA2 instruction advances both.
// a - b is formed as fma(b, -1, a): the product is exact, so the result is the
// correctly rounded difference, in one instruction without a negated operand.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// (sh, sl) += (ah, al - q): two-sum of the high parts; the low part arrives
// as al and a term q to subtract (q = 0.f2 when there is none).
__device__ __forceinline__ void df_add2(float2& sh, float2& sl, float2 ah, float2 al, float2 q) {
  const float2 s = __fadd2_rn(sh, ah);
  const float2 v = sub2(s, sh);
  const float2 e = __fadd2_rn(sub2(sh, sub2(s, v)), sub2(ah, v));
  sh = s;
  sl = __fadd2_rn(sl, __fadd2_rn(al, sub2(e, q)));
}

// (sh, sl) -= (ah, al): two-sum of sh and -ah written with subtractions
// (each rounding is symmetric under negation, so the error term is exact).
__device__ __forceinline__ void df_sub2(float2& sh, float2& sl, float2 ah, float2 al) {
  const float2 s = sub2(sh, ah);
  const float2 v = sub2(s, sh);
  const float2 e = sub2(sub2(sh, sub2(s, v)), __fadd2_rn(ah, v));
  sh = s;
  sl = __fadd2_rn(sl, sub2(e, al));
}

// (sh, sl) += (wh + wl)(uh + ul).  With nw = -wh, nv = -wl:
// ph = wh uh, q = ph - wh uh (exact, = minus the product's error) - wh ul - wl uh.
__device__ __forceinline__ void df_fma2(float2& sh, float2& sl, float wh, float nw, float nv,
                                        float2 uh, float2 ul) {
  const float2 w = make_float2(wh, wh), wn = make_float2(nw, nw), vn = make_float2(nv, nv);
  const float2 ph = __fmul2_rn(w, uh);
  float2 q = __ffma2_rn(wn, uh, ph);
  q = __ffma2_rn(wn, ul, q);
  q = __ffma2_rn(vn, uh, q);
  df_add2(sh, sl, ph, make_float2(0.f, 0.f), q);
}

// Shared-memory kernel: block (x, y) takes the tile of T = 256 * SM_NR nodes
// from P0 = x * T and the column pair 2y, 2y + 1.  It stages u of both
// columns over [P0 - mx - 1, P0 + T + mx + 1) (the tile and one grid row of
// halo on each side; zero outside 0..n-1) into shared memory as split values,
// float4 (hi_a, hi_b, lo_a, lo_b), so each value is split once; thread t then
// evaluates nodes P0 + t + 256 k for both columns at once: the five stencil
// values are consecutive-per-lane shared loads.  A column past B is computed
// on zeros and not stored.  The fast route needs max(|f_p|, |u_p|) >= 2^-60
// and a finite result (a value at or above 2^128 is staged as NaN); other
// nodes take the FP64 route.
template <int RF, int SM_NR, bool DIM3>
__device__ __forceinline__ void residual_df_tile(
    const double* __restrict__ b, const double* __restrict__ u, int n, int mx, int plane, int B,
    int ldr, const float4* __restrict__ wh4, const float4* __restrict__ wl4,
    const float4* __restrict__ wz4, const double* __restrict__ w4,
    const double* __restrict__ lift, void* __restrict__ R, const float* __restrict__ col_scale,
    double* __restrict__ colmax_r, int track, const uint32_t* __restrict__ flags, int pf) {
  extern __shared__ float4 su[];   // [L]
  __shared__ float red[2][8];
  if (flags && flags[FLAG_DONE]) return;
  constexpr int T = 256 * SM_NR;
  const int halo = DIM3 ? plane : mx;   // farthest neighbour: one z-plane (3-D) or one row (2-D)
  const int L = T + 2 * halo + 2;
  const int P0 = blockIdx.x * T;
  const int q0 = P0 - halo - 1;
  const int ca = 2 * blockIdx.y, cb = ca + 1;
  const bool has_b = cb < B;
  const double* ua = u + (size_t)ca * n;
  const double* ub = u + (size_t)(has_b ? cb : ca) * n;
  if (pf > 0) {
    // L2 prefetch of the same tile of the column pair pf pairs ahead (the
    // blocks that will run a few rounds later), 128-byte lines, in bounds
    const int fa = ca + 2 * pf;
    if (fa < B) {
      const int lo = q0 < 0 ? 0 : q0, hi = (q0 + L < n) ? q0 + L : n;
      const int blo = P0, bhi = (P0 + T < n) ? P0 + T : n;
      const int nu = (hi - lo + 15) / 16, nb = (bhi - blo + 15) / 16;
      const int ncol = (fa + 1 < B) ? 2 : 1;
      for (int i = threadIdx.x; i < ncol * (nu + nb); i += 256) {
        const int col = fa + i / (nu + nb), j = i % (nu + nb);
        const double* a = (j < nu) ? u + (size_t)col * n + lo + 16 * j
                                   : b + (size_t)col * n + blo + 16 * (j - nu);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
      }
    }
  }
  // staging: STAGE_UNROLL rows of loads in flight per thread before any split
  constexpr int STAGE_UNROLL = 4;
  for (int i0 = threadIdx.x; i0 < L; i0 += 256 * STAGE_UNROLL) {
    double va[STAGE_UNROLL], vb[STAGE_UNROLL];
#pragma unroll
    for (int j = 0; j < STAGE_UNROLL; ++j) {
      const int q = q0 + i0 + 256 * j;
      const bool in = i0 + 256 * j < L && q >= 0 && q < n;
      va[j] = in ? ua[q] : 0.0;
      vb[j] = (in && has_b) ? ub[q] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < STAGE_UNROLL; ++j) {
      const int i = i0 + 256 * j;
      if (i < L) {
        float ha, la, hb, lb;
        split_marked(va[j], ha, la);
        split_marked(vb[j], hb, lb);
        su[i] = make_float4(ha, hb, la, lb);
      }
    }
  }
  __syncthreads();
  const float isa = (RF == RF_E4M3 || RF == RF_F16) ? 1.0f / col_scale[ca] : 1.0f;
  const float isb = ((RF == RF_E4M3 || RF == RF_F16) && has_b) ? 1.0f / col_scale[cb] : 1.0f;
  float mxa = 0.f, mxb = 0.f;
  const double* ba = b + (size_t)ca * n;
  const double* bb = b + (size_t)(has_b ? cb : ca) * n;
#pragma unroll 2
  for (int k = 0; k < SM_NR; ++k) {
    const int p = P0 + (int)threadIdx.x + 256 * k;
    if (p >= n) break;
    const float4 wh = wh4[p], wl = wl4[p];
    float lh = 0.f, ll = 0.f;
    if (lift) split_marked(lift[p], lh, ll);
    float bha, bla, bhb = 0.f, blb = 0.f;
    split_marked(ba[p], bha, bla);
    if (has_b) split_marked(bb[p], bhb, blb);
    const int i = p - q0;
    const float4 c0 = su[i], cw = su[i - 1], ce = su[i + 1], cs = su[i - mx], cn = su[i + mx];
    float2 ah = make_float2(bha, bhb), al = make_float2(bla, blb);
    if (lift) df_add2(ah, al, make_float2(lh, lh), make_float2(ll, ll), make_float2(0.f, 0.f));
    df_sub2(ah, al, make_float2(c0.x, c0.y), make_float2(c0.z, c0.w));
    df_fma2(ah, al, wh.x, -wh.x, -wl.x, make_float2(cw.x, cw.y), make_float2(cw.z, cw.w));
    df_fma2(ah, al, wh.y, -wh.y, -wl.y, make_float2(ce.x, ce.y), make_float2(ce.z, ce.w));
    df_fma2(ah, al, wh.z, -wh.z, -wl.z, make_float2(cs.x, cs.y), make_float2(cs.z, cs.w));
    df_fma2(ah, al, wh.w, -wh.w, -wl.w, make_float2(cn.x, cn.y), make_float2(cn.z, cn.w));
    if (DIM3) {
      const float4 wz = wz4[p];
      const float4 cd = su[i - plane], cu = su[i + plane];
      df_fma2(ah, al, wz.x, -wz.x, -wz.z, make_float2(cd.x, cd.y), make_float2(cd.z, cd.w));
      df_fma2(ah, al, wz.y, -wz.y, -wz.w, make_float2(cu.x, cu.y), make_float2(cu.z, cu.w));
    }
    const float2 s = __fadd2_rn(ah, al);
    const float2 e = sub2(al, sub2(s, ah));
    float sa = s.x, ea = e.x, sb = s.y, eb = e.y;
    if (!(fmaxf(fmaxf(fabsf(c0.x), fabsf(bha)), fabsf(lh)) >= 0x1p-60f) ||
        !(fabsf(sa) <= 3.4028234e38f))
      split_f64_slow(residual_node_fp64(ba, ua, w4, lift, n, mx, DIM3 ? plane : n, p), sa, ea);
    store_r<RF>(R, (size_t)ca * ldr + p, sa, ea, isa);
    if (track) mxa = fmaxf(mxa, fabsf(sa));
    if (has_b) {
      if (!(fmaxf(fmaxf(fabsf(c0.y), fabsf(bhb)), fabsf(lh)) >= 0x1p-60f) ||
          !(fabsf(sb) <= 3.4028234e38f))
        split_f64_slow(residual_node_fp64(bb, ub, w4, lift, n, mx, DIM3 ? plane : n, p), sb, eb);
      store_r<RF>(R, (size_t)cb * ldr + p, sb, eb, isb);
      if (track) mxb = fmaxf(mxb, fabsf(sb));
    }
  }
  if (track) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
      mxa = fmaxf(mxa, __shfl_xor_sync(0xffffffffu, mxa, o));
      mxb = fmaxf(mxb, __shfl_xor_sync(0xffffffffu, mxb, o));
    }
    if (lane == 0) {
      red[0][w] = mxa;
      red[1][w] = mxb;
    }
    __syncthreads();
    if (threadIdx.x < 2 && (threadIdx.x == 0 || has_b)) {
      float v = 0.f;
      for (int q = 0; q < 8; ++q) v = fmaxf(v, red[threadIdx.x][q]);
      atomic_max_nonneg(&colmax_r[ca + threadIdx.x], (double)v);
    }
  }
}

#define RESIDUAL_DF_ARGS                                                                       \
  const double* __restrict__ b, const double* __restrict__ u, int n, int mx, int plane, int B,  \
      int ldr, const float4* __restrict__ wh4, const float4* __restrict__ wl4,                  \
      const float4* __restrict__ wz4, const double* __restrict__ w4,                            \
      const double* __restrict__ lift, void* __restrict__ R, const float* __restrict__ col_scale, \
      double* __restrict__ colmax_r, int track, const uint32_t* __restrict__ flags, int pf

template <int RF, int SM_NR, bool DIM3>
__global__ void __launch_bounds__(256) residual_df_kernel(RESIDUAL_DF_ARGS) {
  residual_df_tile<RF, SM_NR, DIM3>(b, u, n, mx, plane, B, ldr, wh4, wl4, wz4, w4, lift, R,
                                    col_scale, colmax_r, track, flags, pf);
}
#undef RESIDUAL_DF_ARGS

// Prep for BF16 right-hand sides, forward mode: R = bf16(b + lift) rounded to
// nearest (integer rounding of b alone; with a lift, from the exact pair of
// the sticky split); optionally max |f| per column.
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
    __nv_bfloat16 q;
    // |f| for the column maximum, to FP32 accuracy (not the BF16 value)
    float af = 0.f;
    if (!lift) {
      q = bf16_of_f64(bp);
      if (track) af = fabsf(__double2float_rn(bp));
    } else {
      float bh, bl, lh, ll;
      const double lp = lift[p];
      const uint32_t e1 = split47<true>(bp, bh, bl), e2 = split47<true>(lp, lh, ll);
      // both in the split's exact range (or exactly zero)
      const bool ok = (e1 >= 920u || is_zero(bp)) && (e2 >= 920u || is_zero(lp)) &&
                      e1 <= E_SPLIT_MAX && e2 <= E_SPLIT_MAX;
      if (ok) {
        df_add(bh, bl, lh, ll);
        const float s = __fadd_rn(bh, bl);
        q = bf16_of_pair(s, __fsub_rn(bl, __fsub_rn(s, bh)));
        af = fabsf(s);
      } else {
        q = bf16_of_f64_slow(bp + lp);
        if (track) af = fabsf(__double2float_rn(bp + lp));
      }
    }
    R[(size_t)col * ldr + p] = q;
    if (track) mx = fmaxf(mx, af);
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
  wsplit_kernel<<<g > 0 ? g : 1, 256, 0, st>>>(c->w, c->n, c->mx, plane_of(c), c->wsp,
                                               c->wsp + c->n,
                                               c->dims == 3 ? c->wsp + 2 * (size_t)c->n : nullptr);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

template <int NR, bool DIM3>
static pide_status launch_df_smem(pide_ctx* c, const double* b, const double* u, int B,
                                  const double* lift, int rfmt, void* R, int ldr,
                                  const float* col_scale, double* colmax_r, int t,
                                  const uint32_t* flags, size_t smem, cudaStream_t st) {
  const dim3 g((c->n + 256 * NR - 1) / (256 * NR), (B + 1) / 2, 1);
  const float4* wh = c->wsp;
  const float4* wl = c->wsp + c->n;
  const float4* wz = DIM3 ? c->wsp + 2 * (size_t)c->n : nullptr;
  const int plane = plane_of(c);
  switch (rfmt) {
    case RF_BF16: {
      auto k = residual_df_kernel<RF_BF16, NR, DIM3>;
      if (smem > 48 * 1024)
        PIDE_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<g, 256, smem, st>>>(b, u, c->n, c->mx, plane, B, ldr, wh, wl, wz, c->w, lift, R, col_scale, colmax_r, t, flags, c->resid_prefetch);
      break;
    }
    case RF_F32: {
      auto k = residual_df_kernel<RF_F32, NR, DIM3>;
      if (smem > 48 * 1024)
        PIDE_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<g, 256, smem, st>>>(b, u, c->n, c->mx, plane, B, ldr, wh, wl, wz, c->w, lift, R, col_scale, colmax_r, t, flags, c->resid_prefetch);
      break;
    }
    case RF_F16: {
      auto k = residual_df_kernel<RF_F16, NR, DIM3>;
      if (smem > 48 * 1024)
        PIDE_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<g, 256, smem, st>>>(b, u, c->n, c->mx, plane, B, ldr, wh, wl, wz, c->w, lift, R, col_scale, colmax_r, t, flags, c->resid_prefetch);
      break;
    }
    default: {
      auto k = residual_df_kernel<RF_E4M3, NR, DIM3>;
      if (smem > 48 * 1024)
        PIDE_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<g, 256, smem, st>>>(b, u, c->n, c->mx, plane, B, ldr, wh, wl, wz, c->w, lift, R, col_scale, colmax_r, t, flags, c->resid_prefetch);
      break;
    }
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_residual_df(pide_ctx* c, const double* b, const double* u, int B,
                               const double* lift, int rfmt, void* R, int ldr,
                               const float* col_scale, double* colmax_r, bool track,
                               const uint32_t* flags, cudaStream_t st) {
  if (B == 0) return PIDE_OK;
  if (rfmt != RF_BF16 && rfmt != RF_F32 && rfmt != RF_E4M3 && rfmt != RF_F16) return PIDE_EINVAL;
  const int t = track ? 1 : 0;
  const bool three = c->dims == 3;
  // default (-1): 8 nodes per thread (16 in 3-D stages relatively less halo
  // but measured slower at 32^3: 1.05 against 0.85 ms per step, 98 KB of
  // shared memory per block leaves two blocks per SM)
  const int nr = c->resid_shape < 0 ? 8 : SM_NRS[c->resid_shape & 3];
  const size_t halo = three ? (size_t)plane_of(c) : (size_t)c->mx;
  const size_t smem = (256 * (size_t)nr + 2 * halo + 2) * sizeof(float4);
  if (three) {
    // a z-plane of halo on each side; beyond SMEM_MAX_3D the caller uses the FP64 stencil
    if (smem > SMEM_MAX_3D) return PIDE_EUNSUPPORTED;
    switch (nr) {
      case 16: return launch_df_smem<16, true>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
      case 8: return launch_df_smem<8, true>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
      case 2: return launch_df_smem<2, true>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
      default: return launch_df_smem<4, true>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
    }
  }
  if (smem <= SMEM_MAX) {
    switch (nr) {
      case 16: return launch_df_smem<16, false>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
      case 8: return launch_df_smem<8, false>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
      case 2: return launch_df_smem<2, false>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
      default: return launch_df_smem<4, false>(c, b, u, B, lift, rfmt, R, ldr, col_scale, colmax_r, t, flags, smem, st);
    }
  }
  constexpr int NR = 4, COLS = 2;
  int gx = (c->n + 256 * NR - 1) / (256 * NR);
  if (gx > 1024) gx = 1024;
  const dim3 g(gx, (B + COLS - 1) / COLS, 1);
  const float4* wh = c->wsp;
  const float4* wl = c->wsp + c->n;
  switch (rfmt) {
    case RF_BF16: residual_df_reg_kernel<RF_BF16, NR, COLS><<<g, 256, 0, st>>>(b, u, c->n, c->mx, B, ldr, wh, wl, c->w, lift, R, col_scale, colmax_r, t, flags); break;
    case RF_F32: residual_df_reg_kernel<RF_F32, NR, COLS><<<g, 256, 0, st>>>(b, u, c->n, c->mx, B, ldr, wh, wl, c->w, lift, R, col_scale, colmax_r, t, flags); break;
    case RF_F16: residual_df_reg_kernel<RF_F16, NR, COLS><<<g, 256, 0, st>>>(b, u, c->n, c->mx, B, ldr, wh, wl, c->w, lift, R, col_scale, colmax_r, t, flags); break;
    default: residual_df_reg_kernel<RF_E4M3, NR, COLS><<<g, 256, 0, st>>>(b, u, c->n, c->mx, B, ldr, wh, wl, c->w, lift, R, col_scale, colmax_r, t, flags); break;
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
