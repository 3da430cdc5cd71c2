// PIDE_FP16: the inverse and the right-hand sides in IEEE half precision with
// power-of-two scales.
//
// BF16 keeps 8 significant bits and needs no scale; FP16 keeps 11 but spans
// only 2^-24 .. 65504, so each row p of the inverse is stored as
// fp16(L^-1_p / s_p) with s_p = 2^k_p chosen so that the row's largest entry
// lands in [2^14, 2^15), and each right-hand side column j as fp16(f_j / t_j)
// with t_j = 2^k_j putting its largest entry in [2^11, 2^12) (headroom for the
// refinement's residuals, which reuse t_j and are far smaller than f).  Entries
// down to ~2^-29 of the row (column) maximum stay normal.  Powers of two make
// every scaling exact; the GEMM epilogue multiplies the FP32 accumulator by
// s_p t_j.  The conversions round to nearest even directly from the FP64 bit
// pattern with integer operations (no FP64 instruction, no double rounding).
#include "common.cuh"
#include "f16_round.cuh"

namespace pide {

namespace {

// largest |x| as FP64 bits (non-negative doubles order like their bit patterns)
__device__ __forceinline__ uint64_t abs_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ uint64_t block_max_u64(uint64_t v, unsigned long long* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t w = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
      v = w > v ? w : v;
    }
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  return red[0];
}

// exponent k of the power-of-two scale that puts a maximum with FP64 bits mx in
// [2^(top-1), 2^top); 0 for a zero maximum; kept inside FP32's normal range
__device__ __forceinline__ int pow2_scale_exp(uint64_t mx, int top) {
  if (mx == 0) return 0;
  const int e = (int)(mx >> 52) - 1022;          // mx in [2^(e-1), 2^e)
  int k = e - top;
  if (k < -126) k = -126;
  if (k > 127) k = 127;
  return k;
}

// One CTA per row: s_p = 2^k, Q_p = fp16(G_p / s_p), zero padding to ld.
__global__ void to_f16_kernel(const double* __restrict__ G, size_t ld, int n,
                              __half* __restrict__ Q, float* __restrict__ row_scale) {
  __shared__ unsigned long long red[32];
  const int p = blockIdx.x;
  const double* row = G + (size_t)p * ld;
  uint64_t mx = 0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const uint64_t a = abs_bits(row[q]);
    mx = a > mx ? a : mx;
  }
  mx = block_max_u64(mx, red);
  const int k = pow2_scale_exp(mx, 15);
  if (threadIdx.x == 0) row_scale[p] = ldexpf(1.0f, k);
  for (int q = threadIdx.x; q < (int)ld; q += blockDim.x)
    Q[(size_t)p * ld + q] = __ushort_as_half(q < n ? f16_bits_scaled(row[q], k) : (uint16_t)0);
}

__device__ __forceinline__ double rhs_value(const double* __restrict__ bc, int p, int mode,
                                            const double* __restrict__ dinv,
                                            const double* __restrict__ lift) {
  const double v = bc[p];
  if (mode == 1) return v * dinv[p];
  return lift ? v + lift[p] : v;
}

// One CTA per column: f = b + lift (mode 0) or b / d (mode 1); t_j = 2^k with
// max|f_j| / t_j in [2^11, 2^12); R_j = fp16(f_j / t_j); optionally max|f_j|.
__global__ void prep_f16_kernel(const double* __restrict__ b, int n, int ldr, int mode,
                                const double* __restrict__ dinv, const double* __restrict__ lift,
                                __half* __restrict__ R, float* __restrict__ col_scale,
                                double* __restrict__ colmax_b, int track) {
  __shared__ unsigned long long red[32];
  const int col = blockIdx.x;
  const double* bc = b + (size_t)col * n;
  uint64_t mx = 0;
  // four independent loads in flight per thread
  const int step = 4 * blockDim.x;
  for (int p0 = threadIdx.x; p0 < n; p0 += step) {
    double v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = p0 + i * blockDim.x;
      v[i] = p < n ? rhs_value(bc, p, mode, dinv, lift) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint64_t a = abs_bits(v[i]);
      mx = a > mx ? a : mx;
    }
  }
  mx = block_max_u64(mx, red);
  const int k = pow2_scale_exp(mx, 12);
  if (threadIdx.x == 0) {
    col_scale[col] = ldexpf(1.0f, k);
    if (track) colmax_b[col] = __longlong_as_double((long long)mx);
  }
  // second pass (from L2), again four loads in flight per thread
  for (int p0 = threadIdx.x; p0 < n; p0 += step) {
    double v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = p0 + i * blockDim.x;
      v[i] = p < n ? rhs_value(bc, p, mode, dinv, lift) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = p0 + i * blockDim.x;
      if (p < n) R[(size_t)col * ldr + p] = __ushort_as_half(f16_bits_scaled(v[i], k));
    }
  }
}

}  // namespace

pide_status quantize_store_f16(pide_ctx* c, const double* G, cudaStream_t st) {
  const size_t total = (size_t)c->n * c->ld;
  PIDE_CUDA_TRY(cudaMallocAsync(&c->inv, total * sizeof(__half), st));
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&c->row_scale, c->n * sizeof(float), st));
  to_f16_kernel<<<c->n, 256, 0, st>>>(G, c->ld, c->n, (__half*)c->inv, c->row_scale);
  PIDE_CUDA_TRY(cudaGetLastError());
  c->store_bytes = total * sizeof(__half) + c->n * sizeof(float);
  return PIDE_OK;
}

pide_status launch_prep_f16(pide_ctx* c, const double* b, int B, int mode, const double* lift,
                            bool track, cudaStream_t st) {
  if (B == 0) return PIDE_OK;
  ProfScope ps(c, st, 2);
  // 1024 threads per column: fewer columns in flight, so that the second pass
  // over a column finds it in L2
  prep_f16_kernel<<<B, 1024, 0, st>>>(b, c->n, c->ld, mode, c->dinv, lift, (__half*)c->R,
                                      c->col_scale, c->colmax + c->ws_B, track ? 1 : 0);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

}  // namespace pide
