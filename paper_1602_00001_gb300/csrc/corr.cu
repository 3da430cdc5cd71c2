// PIDE_BF16_FP8 / PIDE_FP16_FP8: the BF16 store Q = bf16(L^-1) (or the scaled
// FP16 store) plus an e4m3 correction term.
//
// The refinement's error contraction per sweep is set by how far the stored
// inverse is from L^-1: with BF16 alone (8 significant bits) it is ~0.1-0.16
// per sweep at 198^2 unknowns and grows with the grid.  The correction term
// C = e4m3((L^-1 - Q) / s_p), s_p = max_q |L^-1 - Q|_pq / 448 per row, adds
// about four more bits at half the BF16 contraction's cost (the FP8 tensor
// pipe runs at twice the BF16 rate), and the sweeps that add it contract
// roughly 16x harder.  Its right-hand side is the BF16 R of the same sweep,
// taken to e4m3 with a per-column scale t_j = max_p |R_pj| / 448; the GEMM's
// epilogue multiplies by s_p t_j and adds into u.
#include "common.cuh"

namespace pide {

namespace {

__device__ __forceinline__ float block_max_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  return red[0];
}

// The stored value of entry e of row p: BF16, or FP16 times the row's
// power-of-two scale (exact in FP64).
__device__ __forceinline__ double stored_hi(const void* Q, const float* hi_scale, size_t e, int p) {
  if (hi_scale)
    return (double)__half2float(reinterpret_cast<const __half*>(Q)[e]) * (double)hi_scale[p];
  return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Q)[e]);
}

// One CTA per row p of the FP64 inverse G: D = G - Q (Q the stored BF16 or
// scaled FP16 value; D exact in FP64), s_p = float(max|D| / 448) (1 for an
// all-zero D), C = e4m3(float(D / s_p)).
__global__ void to_corr_kernel(const double* __restrict__ G, size_t ld, int n,
                               const void* __restrict__ Q, const float* __restrict__ hi_scale,
                               __nv_fp8_e4m3* __restrict__ C, float* __restrict__ scale) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  const double* row = G + (size_t)p * ld;
  double mx = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x)
    mx = fmax(mx, fabs(row[q] - stored_hi(Q, hi_scale, (size_t)p * ld + q, p)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) red[0] = mx;
  }
  __syncthreads();
  mx = red[0];
  const float s = mx > 0.0 ? (float)(mx / 448.0) : 1.0f;
  if (threadIdx.x == 0) scale[p] = s;
  const double inv = 1.0 / (double)s;
  for (int q = threadIdx.x; q < (int)ld; q += blockDim.x) {
    double x = 0.0;
    if (q < n) x = (row[q] - stored_hi(Q, hi_scale, (size_t)p * ld + q, p)) * inv;
    C[(size_t)p * ld + q] = __nv_fp8_e4m3((float)x);
  }
}

template <typename T2>
__device__ __forceinline__ float2 to_float2(T2 v);
template <>
__device__ __forceinline__ float2 to_float2<__nv_bfloat162>(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <>
__device__ __forceinline__ float2 to_float2<__half2>(__half2 v) { return __half22float2(v); }

// One CTA per column j of R (BF16, or FP16 in units of its power-of-two column
// scale rs_j): t_j = float(max|R_j| / 448) (1 for a zero column),
// Rc_j = e4m3(R_j * float(1 / t_j)), and the scale the GEMM applies, t_j rs_j
// (exact: rs_j is a power of two); entries at and beyond n (the row padding,
// which may hold another format's bytes) count as zero.  Both passes read the
// column (2 n bytes, L1/L2-resident for the second).
template <typename T2>
__global__ void corr_rhs_kernel(const T2* __restrict__ R, int n, int ld,
                                const float* __restrict__ r_scale,
                                __nv_fp8_e4m3* __restrict__ Rc, float* __restrict__ col_scale,
                                const uint32_t* __restrict__ flags) {
  __shared__ float red[32];
  if (flags && flags[FLAG_DONE]) return;
  const int j = blockIdx.x;
  const T2* r2 = R + (size_t)j * (ld / 2);
  const int half = ld / 2;                 // ld is a multiple of 64
  // 16-byte loads: four pairs per thread and step
  const uint4* r8 = reinterpret_cast<const uint4*>(r2);
  float mx = 0.0f;
  for (int q4 = threadIdx.x; q4 < half / 4; q4 += blockDim.x) {
    const uint4 raw = r8[q4];
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = 4 * q4 + i;
      float2 v = to_float2<T2>(*reinterpret_cast<const T2*>(&w[i]));
      if (2 * q >= n) v.x = 0.0f;
      if (2 * q + 1 >= n) v.y = 0.0f;
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  }
  mx = block_max_f(mx, red);
  const float t = mx > 0.0f ? (float)((double)mx / 448.0) : 1.0f;
  if (threadIdx.x == 0) col_scale[j] = r_scale ? t * r_scale[j] : t;
  const float isc = 1.0f / t;
  __nv_fp8x2_e4m3* o2 = reinterpret_cast<__nv_fp8x2_e4m3*>(
      reinterpret_cast<uint8_t*>(Rc) + (size_t)j * ld);
  for (int q4 = threadIdx.x; q4 < half / 4; q4 += blockDim.x) {
    const uint4 raw = r8[q4];
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
    uint16_t o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = 4 * q4 + i;
      float2 v = to_float2<T2>(*reinterpret_cast<const T2*>(&w[i]));
      if (2 * q >= n) v.x = 0.0f;
      if (2 * q + 1 >= n) v.y = 0.0f;
      o[i] = __nv_fp8x2_e4m3(make_float2(v.x * isc, v.y * isc)).__x;
    }
    reinterpret_cast<uint2*>(o2)[q4] = make_uint2((uint32_t)o[0] | ((uint32_t)o[1] << 16),
                                                  (uint32_t)o[2] | ((uint32_t)o[3] << 16));
  }
}

}  // namespace

pide_status quantize_corr(pide_ctx* c, const double* G, cudaStream_t st) {
  const size_t total = (size_t)c->n * c->ld;
  PIDE_CUDA_TRY(cudaMallocAsync(&c->corr, total, st));
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&c->corr_scale, c->n * sizeof(float), st));
  // after quantize_store: D is taken against the stored value itself
  const float* hi_scale = c->prec == PIDE_FP16 ? c->row_scale : nullptr;
  to_corr_kernel<<<c->n, 256, 0, st>>>(G, c->ld, c->n, c->inv, hi_scale,
                                       (__nv_fp8_e4m3*)c->corr, c->corr_scale);
  PIDE_CUDA_TRY(cudaGetLastError());
  c->store_bytes += total + c->n * sizeof(float);
  return PIDE_OK;
}

pide_status launch_corr_rhs(pide_ctx* c, int B, cudaStream_t st) {
  if (B == 0) return PIDE_OK;
  if (!c->corr || !c->Rc) return PIDE_EINVAL;
  ProfScope ps(c, st, 2);
  if (c->prec == PIDE_FP16)
    corr_rhs_kernel<__half2><<<B, 256, 0, st>>>((const __half2*)c->R, c->n, c->ld, c->col_scale,
                                                (__nv_fp8_e4m3*)c->Rc, c->col_scale_c, c->flags);
  else
    corr_rhs_kernel<__nv_bfloat162><<<B, 256, 0, st>>>((const __nv_bfloat162*)c->R, c->n, c->ld,
                                                       nullptr, (__nv_fp8_e4m3*)c->Rc,
                                                       c->col_scale_c, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_apply_corr(pide_ctx* c, int B, double* u, cudaStream_t st) {
  if (B == 0) return PIDE_OK;
  c->tail.pending = false;
  pide_status s;
  {
    ProfScope ps(c, st, 3);   // its own class: the FP8 GEMM, timed apart from the BF16 applies
    s = launch_gemm_tc(c, B, u, true, st, 0, true);
  }
  if (s != PIDE_OK) {
    c->tail.pending = false;
    return s;
  }
  return launch_tail_reduce(c, st);
}

}  // namespace pide
