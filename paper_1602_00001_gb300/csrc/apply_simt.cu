// Step 3 on the CUDA cores: u (=|+=) Q(S^-1) R.
//
//  * gemv_kernel: few right-hand sides (B <= 8).  The apply is bound by HBM:
//    each stored entry is read once with 16-byte vector loads, multiplied by
//    the right-hand side slice held in shared memory (FP32, or FP64 for the
//    FP64 store) and reduced across the warp with shuffles.  When the slice
//    does not fit in shared memory the K range is split over blockIdx.y and
//    the partial sums are added atomically into the FP64 result.
//  * gemm_simt_kernel: FP64 / FP32 stores with many right-hand sides (the
//    FP64 comparator and the FP32 format), register-tiled 64 x 64 tiles.
#include "common.cuh"

namespace pide {

namespace {

template <int KIND> struct Elem;
template <> struct Elem<KIND_F64> { using TA = double; using TX = double; static constexpr int VEC = 2; };
template <> struct Elem<KIND_F32> { using TA = float; using TX = float; static constexpr int VEC = 4; };
template <> struct Elem<KIND_BF16> { using TA = __nv_bfloat16; using TX = float; static constexpr int VEC = 8; };
template <> struct Elem<KIND_FP8> { using TA = __nv_fp8_e4m3; using TX = float; static constexpr int VEC = 16; };
template <> struct Elem<KIND_FP8X2> { using TA = __nv_fp8_e4m3; using TX = float; static constexpr int VEC = 16; };
template <> struct Elem<KIND_F16> { using TA = __half; using TX = float; static constexpr int VEC = 8; };

template <int KIND>
__device__ __forceinline__ void unpack(const uint4& raw, float (&out)[Elem<KIND>::VEC]) {
  if constexpr (KIND == KIND_F32) {
    out[0] = __uint_as_float(raw.x); out[1] = __uint_as_float(raw.y);
    out[2] = __uint_as_float(raw.z); out[3] = __uint_as_float(raw.w);
  } else if constexpr (KIND == KIND_BF16) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      out[2 * i] = __uint_as_float(w[i] << 16);
      out[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  } else if constexpr (KIND == KIND_F16) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
      out[2 * i] = f.x;
      out[2 * i + 1] = f.y;
    }
  } else {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        __nv_fp8_e4m3 v;
        v.__x = (uint8_t)(w[i] >> (8 * b));
        out[4 * i + b] = (float)v;
      }
    }
  }
}

template <int KIND, int NB, int GEMV_UNROLL>
__global__ void __launch_bounds__(1024) gemv_kernel(
    const void* __restrict__ A_, const void* __restrict__ Alo_, const float* __restrict__ row_scale,
    const float* __restrict__ col_scale, int n, int ld, const void* __restrict__ R_, int ldr,
    int B, double* __restrict__ u, int accumulate, int kchunk, const uint32_t* __restrict__ flags) {
  using TA = typename Elem<KIND>::TA;
  using TX = typename Elem<KIND>::TX;
  constexpr int VEC = Elem<KIND>::VEC;
  constexpr bool LO = (KIND == KIND_FP8X2);
  if (flags && flags[FLAG_DONE]) return;
  extern __shared__ __align__(16) uint8_t shm[];
  TX* xs = reinterpret_cast<TX*>(shm);
  const TX* R = reinterpret_cast<const TX*>(R_);
  const int k0 = blockIdx.y * kchunk;
  const int klen = min(kchunk, n - k0);
  for (int e = threadIdx.x; e < NB * kchunk; e += blockDim.x) {
    const int c = e / kchunk, q = e - c * kchunk;
    xs[e] = (c < B && q < klen) ? R[(size_t)c * ldr + k0 + q] : (TX)0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int tw = gridDim.x * nwarps;
  const bool split = gridDim.y > 1;
  for (int row = blockIdx.x * nwarps + warp; row < n; row += tw) {
    const TA* arow = reinterpret_cast<const TA*>(A_) + (size_t)row * ld + k0;
    const TA* lrow = LO ? reinterpret_cast<const TA*>(Alo_) + (size_t)row * ld + k0 : nullptr;
    TX acc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = (TX)0;
    for (int q0 = lane * VEC; q0 < klen; q0 += 32 * VEC * GEMV_UNROLL) {
      uint4 raw[GEMV_UNROLL], rawlo[GEMV_UNROLL];
#pragma unroll
      for (int uu = 0; uu < GEMV_UNROLL; ++uu) {
        const int q = q0 + uu * 32 * VEC;
        if (q < klen) {
          raw[uu] = __ldcs(reinterpret_cast<const uint4*>(arow + q));
          if constexpr (LO) rawlo[uu] = __ldcs(reinterpret_cast<const uint4*>(lrow + q));
        } else {
          raw[uu] = make_uint4(0, 0, 0, 0);
          if constexpr (LO) rawlo[uu] = make_uint4(0, 0, 0, 0);
        }
      }
#pragma unroll
      for (int uu = 0; uu < GEMV_UNROLL; ++uu) {
        const int q = q0 + uu * 32 * VEC;
        if (q >= klen) break;
        if constexpr (KIND == KIND_F64) {
          const double a0 = __longlong_as_double(((unsigned long long)raw[uu].y << 32) | raw[uu].x);
          const double a1 = __longlong_as_double(((unsigned long long)raw[uu].w << 32) | raw[uu].z);
#pragma unroll
          for (int c = 0; c < NB; ++c) {
            acc[c] = fma(a0, xs[c * kchunk + q], acc[c]);
            acc[c] = fma(a1, xs[c * kchunk + q + 1], acc[c]);
          }
        } else {
          float a[VEC];
          unpack<KIND>(raw[uu], a);
          if constexpr (LO) {
            float al[VEC];
            unpack<KIND>(rawlo[uu], al);
#pragma unroll
            for (int v = 0; v < VEC; ++v) a[v] += al[v];
          }
#pragma unroll
          for (int c = 0; c < NB; ++c) {
            const float4* x4 = reinterpret_cast<const float4*>(xs + c * kchunk + q);
#pragma unroll
            for (int v4 = 0; v4 < VEC / 4; ++v4) {
              const float4 xv = x4[v4];
              acc[c] = fmaf(a[4 * v4 + 0], xv.x, acc[c]);
              acc[c] = fmaf(a[4 * v4 + 1], xv.y, acc[c]);
              acc[c] = fmaf(a[4 * v4 + 2], xv.z, acc[c]);
              acc[c] = fmaf(a[4 * v4 + 3], xv.w, acc[c]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      TX v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[c] = v;
    }
    if (lane == 0) {
      const double rs = row_scale ? (double)row_scale[row] : 1.0;
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        if (c >= B) break;
        double val = (double)acc[c] * rs;
        if (col_scale) val *= (double)col_scale[c];
        double* dst = u + (size_t)c * n + row;
        if (split) atomicAdd(dst, val);
        else *dst = accumulate ? *dst + val : val;
      }
    }
  }
}

template <typename TA, typename TX, int KS>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const TA* __restrict__ A, int n, int ld,
                                                        const TX* __restrict__ X, int ldx, int B,
                                                        double* __restrict__ u, int accumulate,
                                                        const uint32_t* __restrict__ flags) {
  if (flags && flags[FLAG_DONE]) return;
  __shared__ TA As[KS][65];
  __shared__ TX Xs[KS][65];
  const int p0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  TA acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (TA)0;
  for (int k0 = 0; k0 < n; k0 += KS) {
    for (int e = threadIdx.x; e < 64 * KS; e += 256) {
      const int rr = e / KS, kk = e - rr * KS;
      const int gk = k0 + kk;
      const int gp = p0 + rr, gr = r0 + rr;
      As[kk][rr] = (gp < n && gk < n) ? A[(size_t)gp * ld + gk] : (TA)0;
      Xs[kk][rr] = (gr < B && gk < n) ? (TA)X[(size_t)gr * ldx + gk] : (TX)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      TA av[4], xv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) xv[j] = (TA)Xs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], xv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 16 * j;
    if (r >= B) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = p0 + tx + 16 * i;
      if (p >= n) continue;
      double* dst = u + (size_t)r * n + p;
      const double v = (double)acc[i][j];
      *dst = accumulate ? *dst + v : v;
    }
  }
}

template <int KIND, int NB, int UNROLL>
pide_status gemv_launch(pide_ctx* c, int B, int col0, double* u, bool accumulate,
                        cudaStream_t st) {
  using TX = typename Elem<KIND>::TX;
  constexpr int VEC = Elem<KIND>::VEC;
  const int unit = 32 * VEC * UNROLL;
  const size_t smem_cap = 200 * 1024;
  int kchunk = (int)(smem_cap / (NB * sizeof(TX)));
  kchunk = (kchunk / unit) * unit;
  const int npad = ((c->n + unit - 1) / unit) * unit;
  if (kchunk > npad) kchunk = npad;
  const int ksplit = (c->n + kchunk - 1) / kchunk;
  const size_t smem = (size_t)NB * kchunk * sizeof(TX);
  auto kern = gemv_kernel<KIND, NB, UNROLL>;
  PIDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int bcols = B - col0 < NB ? B - col0 : NB;
  double* uc = u + (size_t)col0 * c->n;
  if (ksplit > 1 && !accumulate)
    PIDE_CUDA_TRY(cudaMemsetAsync(uc, 0, (size_t)bcols * c->n * sizeof(double), st));
  const size_t esz = rhs_elem_bytes(rhs_format(c, B));
  const void* R = (const uint8_t*)c->R + (size_t)col0 * c->ld * esz;
  dim3 grid(c->num_sms, ksplit);
  kern<<<grid, c->gemv_threads, smem, st>>>(c->inv, c->inv_lo, c->row_scale, nullptr, c->n, c->ld,
                                            R, c->ld, bcols, uc, accumulate ? 1 : 0, kchunk,
                                            c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

template <int KIND, int NB>
pide_status gemv_unroll(pide_ctx* c, int B, int col0, double* u, bool accumulate, cudaStream_t st) {
  // FP8X2 keeps two vectors per load slot: cap its unroll to stay within 64 registers
  if (c->gemv_unroll >= 8 && KIND != KIND_FP8X2) return gemv_launch<KIND, NB, 8>(c, B, col0, u, accumulate, st);
  return gemv_launch<KIND, NB, 4>(c, B, col0, u, accumulate, st);
}

template <int KIND>
pide_status gemv_dispatch(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st) {
  for (int col0 = 0; col0 < B; col0 += 8) {
    const int left = B - col0;
    pide_status s;
    if (left == 1) s = gemv_unroll<KIND, 1>(c, B, col0, u, accumulate, st);
    else if (left == 2) s = gemv_unroll<KIND, 2>(c, B, col0, u, accumulate, st);
    else if (left <= 4) s = gemv_unroll<KIND, 4>(c, B, col0, u, accumulate, st);
    else s = gemv_unroll<KIND, 8>(c, B, col0, u, accumulate, st);
    if (s != PIDE_OK) return s;
  }
  return PIDE_OK;
}

}  // namespace

pide_status launch_gemv(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st) {
  switch (c->prec) {
    case PIDE_FP64: return gemv_dispatch<KIND_F64>(c, B, u, accumulate, st);
    case PIDE_FP32: return gemv_dispatch<KIND_F32>(c, B, u, accumulate, st);
    case PIDE_BF16: return gemv_dispatch<KIND_BF16>(c, B, u, accumulate, st);
    case PIDE_FP8: return gemv_dispatch<KIND_FP8>(c, B, u, accumulate, st);
    case PIDE_FP8X2: return gemv_dispatch<KIND_FP8X2>(c, B, u, accumulate, st);
    case PIDE_FP16: return gemv_dispatch<KIND_F16>(c, B, u, accumulate, st);   // row scales applied
  }
  return PIDE_EINVAL;
}

pide_status launch_gemm_simt(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st) {
  dim3 grid((c->n + 63) / 64, (B + 63) / 64);
  if (c->prec == PIDE_FP64) {
    gemm_simt_kernel<double, double, 16><<<grid, 256, 0, st>>>(
        (const double*)c->inv, c->n, c->ld, (const double*)c->R, c->ld, B, u, accumulate ? 1 : 0,
        c->flags);
  } else if (c->prec == PIDE_FP32) {
    gemm_simt_kernel<float, float, 32><<<grid, 256, 0, st>>>(
        (const float*)c->inv, c->n, c->ld, (const float*)c->R, c->ld, B, u, accumulate ? 1 : 0,
        c->flags);
  } else {
    return PIDE_EUNSUPPORTED;
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

}  // namespace pide
