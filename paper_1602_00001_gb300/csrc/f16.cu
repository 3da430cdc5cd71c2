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
#include <cooperative_groups.h>

#include "common.cuh"
#include "f16_round.cuh"

namespace cg = cooperative_groups;

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

// The same prep with a cluster of PREP_CL CTAs per column: each CTA reads its
// slice of f from HBM once into shared memory (as FP64), the cluster agrees on
// the column maximum through distributed shared memory, then each CTA converts
// its slice from shared memory -- one HBM pass instead of two (the second from
// L2) and no per-column serial chain.  With Rc it also writes the e4m3 copy of
// R for the correction term, exactly as corr_rhs_kernel would from R: its
// scale is max|R| / 448, and max|R| is the FP16 value of max|f| / t_j (the
// rounding is monotone).
// Clusters of 8 CTAs of 256 threads: an eighth of a column per CTA (39 KB at
// 198^2), five CTAs per SM; measured 0.18 ms per B = 1024 prep at 198^2 against
// 0.20 ms for clusters of 4 x 512 threads (two CTAs per SM).
constexpr int PREP_CL = 8;
constexpr int PREP_THREADS = 256;

__global__ void __cluster_dims__(PREP_CL, 1, 1) __launch_bounds__(PREP_THREADS)
prep_f16_cluster_kernel(const double* __restrict__ b, int n, int ldr, int mode,
                        const double* __restrict__ dinv, const double* __restrict__ lift,
                        __half* __restrict__ R, float* __restrict__ col_scale,
                        double* __restrict__ colmax_b, int track, int chunk,
                        uint8_t* __restrict__ Rc, float* __restrict__ col_scale_c) {
  extern __shared__ double sf[];            // [chunk]: this CTA's slice of f
  __shared__ unsigned long long red[32];
  __shared__ unsigned long long cta_max;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int col = blockIdx.y;
  const int p0 = rank * chunk;
  const int len = max(0, min(chunk, n - p0));
  const double* bc = b + (size_t)col * n;
  uint64_t mx = 0;
  // pass 1: HBM -> shared memory, eight loads in flight per thread
  for (int i0 = threadIdx.x; i0 < len; i0 += 8 * PREP_THREADS) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * PREP_THREADS;
      v[u] = i < len ? rhs_value(bc, p0 + i, mode, dinv, lift) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * PREP_THREADS;
      if (i < len) sf[i] = v[u];
      const uint64_t a = abs_bits(v[u]);
      mx = a > mx ? a : mx;
    }
  }
  mx = block_max_u64(mx, red);
  if (threadIdx.x == 0) cta_max = mx;
  cluster.sync();
  if (threadIdx.x == 0) {
    uint64_t m = 0;
    for (int r = 0; r < PREP_CL; ++r) {
      const uint64_t x = *cluster.map_shared_rank(&cta_max, r);
      m = x > m ? x : m;
    }
    red[0] = m;
  }
  // every remote read is done before any CTA of the cluster goes on (or exits)
  cluster.sync();
  mx = red[0];
  const int k = pow2_scale_exp(mx, 12);
  if (rank == 0 && threadIdx.x == 0) {
    col_scale[col] = ldexpf(1.0f, k);
    if (track) colmax_b[col] = __longlong_as_double((long long)mx);
  }
  float isc_c = 0.0f;
  if (Rc) {
    const float mxr = fabsf(__half2float(__ushort_as_half(
        f16_bits_scaled(__longlong_as_double((long long)mx), k))));
    const float t = mxr > 0.0f ? (float)((double)mxr / 448.0) : 1.0f;
    if (rank == 0 && threadIdx.x == 0) col_scale_c[col] = t * ldexpf(1.0f, k);
    isc_c = 1.0f / t;
  }
  // pass 2: shared memory -> R (pairs of FP16), and the e4m3 pairs of Rc
  __half2* R2 = reinterpret_cast<__half2*>(R + (size_t)col * ldr + p0);
  __nv_fp8x2_e4m3* C2 = Rc ? reinterpret_cast<__nv_fp8x2_e4m3*>(Rc + (size_t)col * ldr + p0) : nullptr;
  for (int i = 2 * threadIdx.x; i < len; i += 2 * PREP_THREADS) {
    const bool two = i + 1 < len;
    const uint16_t h0 = f16_bits_scaled(sf[i], k);
    const uint16_t h1 = two ? f16_bits_scaled(sf[i + 1], k) : (uint16_t)0;
    if (two) {
      R2[i >> 1] = __halves2half2(__ushort_as_half(h0), __ushort_as_half(h1));
    } else {
      R[(size_t)col * ldr + p0 + i] = __ushort_as_half(h0);
    }
    if (C2) {
      const float v0 = __half2float(__ushort_as_half(h0)), v1 = __half2float(__ushort_as_half(h1));
      const __nv_fp8x2_e4m3 q(make_float2(v0 * isc_c, v1 * isc_c));
      if (two) C2[i >> 1] = q;
      else Rc[(size_t)col * ldr + p0 + i] = (uint8_t)(q.__x & 0xFFu);
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
                            bool track, cudaStream_t st, bool with_corr) {
  if (B == 0) return PIDE_OK;
  ProfScope ps(c, st, 2);
  // one cluster of CTAs per column while an eighth of a column fits a CTA's shared memory
  const int chunk = ((c->n + PREP_CL - 1) / PREP_CL + 7) / 8 * 8;
  const size_t smem = (size_t)chunk * sizeof(double);
  if (c->prep_cluster && smem <= 110 * 1024 && B <= 65535 && (!with_corr || c->Rc)) {
    PIDE_CUDA_TRY(cudaFuncSetAttribute(prep_f16_cluster_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    prep_f16_cluster_kernel<<<dim3(PREP_CL, B), PREP_THREADS, smem, st>>>(
        b, c->n, c->ld, mode, c->dinv, lift, (__half*)c->R, c->col_scale, c->colmax + c->ws_B,
        track ? 1 : 0, chunk, with_corr ? (uint8_t*)c->Rc : nullptr,
        with_corr ? c->col_scale_c : nullptr);
    PIDE_CUDA_TRY(cudaGetLastError());
    return PIDE_OK;
  }
  if (with_corr) {
    PIDE_TRY(launch_prep_f16(c, b, B, mode, lift, track, st, false));
    return launch_corr_rhs(c, B, st);
  }
  // 1024 threads per column: fewer columns in flight, so that the second pass
  // over a column finds it in L2
  prep_f16_kernel<<<B, 1024, 0, st>>>(b, c->n, c->ld, mode, c->dinv, lift, (__half*)c->R,
                                      c->col_scale, c->colmax + c->ws_B, track ? 1 : 0);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

}  // namespace pide
