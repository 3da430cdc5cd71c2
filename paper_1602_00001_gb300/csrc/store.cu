// The stored inverse: FP64 -> FP32 / BF16 / e4m3 (single term or hi + lo)
// conversion with per-row scales, and row read-back for tests.
//
// The paper's Table 1 stores the inverse rounded to a few decimal digits; the
// GPU stores it in a binary low-precision format instead and wins the
// accuracy back by iterative refinement against the FP64 stencil residual.
// FP8 rows are scaled by s_p = max_q |G_pq| / 448 (448 = largest finite
// e4m3), the hi term is e4m3(G/s) and the lo term e4m3(G/s - hi), so that
// hi + lo carries about twice the mantissa bits of one e4m3 value.
#include "common.cuh"

namespace pide {

namespace {

__global__ void to_f32_kernel(const double* __restrict__ G, float* __restrict__ out, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = (float)G[e];
}

__global__ void to_bf16_kernel(const double2* __restrict__ G, __nv_bfloat162* __restrict__ out,
                               size_t total2) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total2;
       e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = G[e];
    __nv_bfloat162 o;
    o.x = __double2bfloat16(v.x);
    o.y = __double2bfloat16(v.y);
    out[e] = o;
  }
}

// One CTA per row: scale, then hi (and lo) e4m3 terms.
__global__ void to_fp8_kernel(const double* __restrict__ G, size_t ld, int n,
                              __nv_fp8_e4m3* __restrict__ hi, __nv_fp8_e4m3* __restrict__ lo,
                              float* __restrict__ row_scale) {
  __shared__ double red[32];
  const int p = blockIdx.x;
  const double* row = G + (size_t)p * ld;
  double mx = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) mx = fmax(mx, fabs(row[q]));
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
  if (threadIdx.x == 0) row_scale[p] = s;
  const double inv = 1.0 / (double)s;
  for (int q = threadIdx.x; q < (int)ld; q += blockDim.x) {
    const double x = q < n ? row[q] * inv : 0.0;
    const __nv_fp8_e4m3 h((float)x);
    hi[(size_t)p * ld + q] = h;
    if (lo) lo[(size_t)p * ld + q] = __nv_fp8_e4m3((float)(x - (double)(float)h));
  }
}

__global__ void row_to_f64_kernel(const void* __restrict__ inv, const void* __restrict__ inv_lo,
                                  const float* __restrict__ row_scale, int fmt, size_t ld, int n,
                                  int p, double* __restrict__ out,
                                  const __nv_fp8_e4m3* __restrict__ corr,
                                  const float* __restrict__ corr_scale) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const size_t e = (size_t)p * ld + q;
    double v;
    switch (fmt) {
      case PIDE_FP64: v = reinterpret_cast<const double*>(inv)[e]; break;
      case PIDE_FP32: v = reinterpret_cast<const float*>(inv)[e]; break;
      case PIDE_BF16:
        // with the e4m3 correction term: Q + s_p C, exact in FP64
        v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(inv)[e]);
        if (corr) v += (double)(float)corr[e] * (double)corr_scale[p];
        break;
      case PIDE_FP16:
        v = (double)__half2float(reinterpret_cast<const __half*>(inv)[e]) * (double)row_scale[p];
        if (corr) v += (double)(float)corr[e] * (double)corr_scale[p];
        break;
      default: {
        v = (float)reinterpret_cast<const __nv_fp8_e4m3*>(inv)[e];
        if (inv_lo) v += (float)reinterpret_cast<const __nv_fp8_e4m3*>(inv_lo)[e];
        v *= row_scale[p];
      }
    }
    out[q] = v;
  }
}

// Table 1's rounding of the inverse: x -> sign(x) floor(|x| 10^k + 1/2) / 10^k,
// each operation rounded separately in FP64 (no FMA contraction), so that the
// same input gives the same decimal as a plain FP64 evaluation of the formula.
__global__ void round_decimal_kernel(double* __restrict__ G, size_t ld, int n, double scale) {
  const size_t total = (size_t)n * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double x = G[e];
    const double m = floor(__dadd_rn(__dmul_rn(fabs(x), scale), 0.5));
    G[e] = copysign(__ddiv_rn(m, scale), x);
  }
}

}  // namespace

pide_status quantize_store(pide_ctx* c, const double* G, cudaStream_t st) {
  const size_t total = (size_t)c->n * c->ld;
  const int grid = c->num_sms * 8;
  switch (c->prec) {
    case PIDE_FP32:
      PIDE_CUDA_TRY(cudaMallocAsync(&c->inv, total * sizeof(float), st));
      to_f32_kernel<<<grid, 256, 0, st>>>(G, (float*)c->inv, total);
      c->store_bytes = total * sizeof(float);
      break;
    case PIDE_BF16:
      PIDE_CUDA_TRY(cudaMallocAsync(&c->inv, total * sizeof(__nv_bfloat16), st));
      to_bf16_kernel<<<grid, 256, 0, st>>>((const double2*)G, (__nv_bfloat162*)c->inv, total / 2);
      c->store_bytes = total * sizeof(__nv_bfloat16);
      break;
    case PIDE_FP16:
      return quantize_store_f16(c, G, st);
    case PIDE_FP8:
    case PIDE_FP8X2:
      PIDE_CUDA_TRY(cudaMallocAsync(&c->inv, total, st));
      if (c->prec == PIDE_FP8X2) PIDE_CUDA_TRY(cudaMallocAsync(&c->inv_lo, total, st));
      PIDE_CUDA_TRY(cudaMallocAsync((void**)&c->row_scale, c->n * sizeof(float), st));
      to_fp8_kernel<<<c->n, 256, 0, st>>>(G, c->ld, c->n, (__nv_fp8_e4m3*)c->inv,
                                          (__nv_fp8_e4m3*)c->inv_lo, c->row_scale);
      c->store_bytes = total * (c->prec == PIDE_FP8X2 ? 2 : 1) + c->n * sizeof(float);
      break;
    default:
      return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

}  // namespace pide

extern "C" pide_status pide_get_inverse_row(pide_handle h, int32_t p, double* dst_host) {
  using namespace pide;
  if (!h || !dst_host || p < 0 || p >= h->n) {
    set_error("pide_get_inverse_row: bad argument");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  double* tmp = nullptr;
  PIDE_CUDA_TRY(cudaMalloc(&tmp, h->n * sizeof(double)));
  row_to_f64_kernel<<<64, 256>>>(h->inv, h->inv_lo, h->row_scale, (int)h->prec, (size_t)h->ld,
                                 h->n, p, tmp, (const __nv_fp8_e4m3*)h->corr, h->corr_scale);
  cudaError_t e = cudaMemcpy(dst_host, tmp, h->n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  PIDE_CUDA_TRY(e);
  return PIDE_OK;
}

extern "C" pide_status pide_round_inverse_decimal(pide_handle h, int32_t digits, void* stream) {
  using namespace pide;
  if (!h || digits < 0 || digits > 15) {
    set_error("pide_round_inverse_decimal: bad argument (digits in [0, 15])");
    return PIDE_EINVAL;
  }
  if (h->prec != PIDE_FP64) {
    set_error("pide_round_inverse_decimal: FP64 handles only");
    return PIDE_EUNSUPPORTED;
  }
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  double scale = 1.0;
  for (int k = 0; k < digits; ++k) scale *= 10.0;   // exact for digits <= 15
  round_decimal_kernel<<<h->num_sms * 8, 256, 0, (cudaStream_t)stream>>>((double*)h->inv,
                                                                         (size_t)h->ld, h->n, scale);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}
