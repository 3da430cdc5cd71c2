// Step 3 for one right-hand side through the symmetric form of the inverse.
//
// L^-1 = S^-1 D with S = D L symmetric (the conservative form of Eq. 3), so
// u = L^-1 r = S^-1 (D r): only the lower triangle of S^-1 has to be read.
// For B = 1 the apply is bound by HBM bytes, so reading one triangle halves
// them.  Storing one triangle makes the rounding error of the stored matrix
// exactly symmetric, and a symmetric error matrix has about twice the
// spectral radius of an unstructured one with the same entry size
// (semicircle vs circular law), so refinement contracts half as fast.  The
// triangle is therefore kept in two terms, hi = bf16(S^-1) and
// lo = fp16((S^-1 - hi) / sigma_p) with one power-of-two scale sigma_p per row
// (the row's largest |S^-1 - hi| in [2^14, 2^15)): ~19 significant bits in the
// bytes of the full one-term L^-1, so that one apply alone reaches ~1e-7.
// Layout: packed 128 x 128 tiles of the lower block triangle, tile (i, j),
// i >= j, at offset (i (i + 1) / 2 + j) * 128 * 128, row-major inside the tile
// (rows/columns past n are zero), hi and lo in two arrays of that layout.  Each
// tile is read once and used twice: y_i += A_ij x_j and, below the diagonal,
// y_j += A_ij^T x_i, with A_pq = hi_pq + sigma_p lo_pq for the stored row p in
// both uses.
//
// Kernel: persistent CTAs of 256 threads take equal contiguous ranges of
// tiles in row-major tile order.  Thread t loads 16-byte vectors t + 256 k
// (k < 8): row (t >> 4) + 16 k, columns 8 (t & 15) .. + 7.  Within a tile the
// products are summed in FP32 and the sums reach y in FP64: row partials stay
// in FP32 registers for at most 8 tiles of a block row (64 terms per thread),
// are reduced across the 16 lanes of a row and added to y; column partials are
// reduced per tile through shared memory; both through FP64 atomics, which run
// in L2 and spare GB300's slow FP64 pipe.  (With FP32 chains across a whole
// block row, ~1200 terms, one apply stayed at ~8e-7 of the solution whatever
// the store's precision; FP64 row registers cost a third of the bandwidth.)
// x = D r is formed on the fly from the FP32 residual and d.  A final kernel
// adds y into the FP64 solution.
#include <cmath>

#include "common.cuh"
#include "f16_round.cuh"

namespace pide {
namespace {

constexpr int T = 128;

__device__ __forceinline__ int tile_row(long long t) {
  int i = (int)floor((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)(i + 1) * (i + 2) / 2 <= t) ++i;
  while ((long long)i * (i + 1) / 2 > t) --i;
  return i;
}

__device__ __forceinline__ void bf16x8(const uint4& raw, float (&a)[8]) {
  const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    a[2 * q] = __uint_as_float(w[q] << 16);
    a[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
  }
}

__device__ __forceinline__ void f16x8(const uint4& raw, float (&a)[8]) {
  const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[q]));
    a[2 * q] = f.x;
    a[2 * q + 1] = f.y;
  }
}

__global__ void __launch_bounds__(256, 2) symv_bf16_kernel(const uint4* __restrict__ P,
                                                        const uint4* __restrict__ Plo,
                                                        const float* __restrict__ sigma,
                                                        long long ntiles,
                                                        int n, const float* __restrict__ r,
                                                        const float* __restrict__ df,
                                                        double* __restrict__ y,
                                                        const uint32_t* __restrict__ flags) {
  if (flags[FLAG_DONE]) return;
  __shared__ float red[2][8][T];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int s = t & 15, r0 = t >> 4;
  const long long t0 = ntiles * blockIdx.x / gridDim.x;
  const long long t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;
  int i = tile_row(t0);
  int j = (int)(t0 - (long long)i * (i + 1) / 2);
  float rowacc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) rowacc[k] = 0.f;
  int since_flush = 0;
  int buf = 0;
  for (long long tt = t0; tt < t1; ++tt) {
    const uint4* tile = P + tt * (T * T / 8);
    const uint4* tlo = Plo + tt * (T * T / 8);
    uint4 raw[8], rlo[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      raw[k] = __ldcs(tile + t + 256 * k);
      rlo[k] = __ldcs(tlo + t + 256 * k);
    }
    float xj[8];
    const int cb = j * T + 8 * s;
#pragma unroll
    for (int q = 0; q < 8; ++q) xj[q] = (cb + q < n) ? r[cb + q] * df[cb + q] : 0.f;
    const bool off = (i != j);
    float xi[8], sg[8];
    float colacc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int row = i * T + r0 + 16 * k;
      xi[k] = (off && row < n) ? r[row] * df[row] : 0.f;
      sg[k] = row < n ? sigma[row] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) colacc[q] = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float a[8], al[8];
      bf16x8(raw[k], a);
      f16x8(rlo[k], al);
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fmaf(al[q], sg[k], a[q]);
      float acc = rowacc[k];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        acc = fmaf(a[q], xj[q], acc);
        colacc[q] = fmaf(a[q], xi[k], colacc[q]);
      }
      rowacc[k] = acc;
    }
    if (off) {
#pragma unroll
      for (int q = 0; q < 8; ++q) colacc[q] += __shfl_xor_sync(0xffffffffu, colacc[q], 16);
      if (lane < 16) {
#pragma unroll
        for (int q = 0; q < 8; ++q) red[buf][warp][8 * s + q] = colacc[q];
      }
      __syncthreads();
      if (t < T) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) v += red[buf][w][t];
        const int col = j * T + t;
        if (col < n) atomicAdd(y + col, (double)v);
      }
      buf ^= 1;
    }
    // next tile; flush the row partials when the block row ends or after 8 tiles
    ++j;
    if (j > i || tt + 1 == t1 || ++since_flush == 8) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float v = rowacc[k];
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        const int row = i * T + r0 + 16 * k;
        if (s == 0 && row < n) atomicAdd(y + row, (double)v);
        rowacc[k] = 0.f;
      }
      since_flush = 0;
      if (j > i) {
        ++i;
        j = 0;
      }
    }
  }
}

// u (=|+=) y, then y = 0 for the next apply.
__global__ void symv_finish_kernel(double* __restrict__ y, double* __restrict__ u, int n,
                                   int accumulate, const uint32_t* __restrict__ flags) {
  if (flags[FLAG_DONE]) return;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const double v = y[p];
    u[p] = accumulate ? u[p] + v : v;
    y[p] = 0.0;
  }
}

// Row scales of the lo term: sigma_p = 2^k with max_q |v_pq - bf16(v_pq)| / sigma_p
// in [2^14, 2^15) (1 for a zero row), v = S^-1 = L^-1 D^-1 from the FP64 L^-1; one
// CTA per row.  The maximum is taken on the FP64 bit patterns.
__global__ void sym_scale_kernel(const double* __restrict__ G, size_t ld, int n,
                                 const double* __restrict__ dinv, float* __restrict__ sigma) {
  __shared__ unsigned long long red[8];
  const int p = blockIdx.x;
  unsigned long long mx = 0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const double v = G[(size_t)p * ld + q] * dinv[q];
    const double dlo = v - (double)__bfloat162float(__double2bfloat16(v));
    const unsigned long long a = (unsigned long long)__double_as_longlong(dlo) & 0x7FFFFFFFFFFFFFFFull;
    mx = a > mx ? a : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = w > mx ? w : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = red[w] > mx ? red[w] : mx;
    int k = 0;
    if (mx) {
      k = (int)(mx >> 52) - 1022 - 15;       // mx in [2^(e-1), 2^e), e = biased - 1022
      k = k < -126 ? -126 : (k > 127 ? 127 : k);
    }
    sigma[p] = ldexpf(1.0f, k);
  }
}

// Pack S^-1 into lower tiles: hi = bf16(v), lo = fp16((v - hi) / sigma_p), both
// rounded to nearest from FP64; one CTA per tile.
__global__ void pack_sym_kernel(const double* __restrict__ G, size_t ld, int n,
                                const double* __restrict__ dinv, const float* __restrict__ sigma,
                                __nv_bfloat16* __restrict__ P, __half* __restrict__ Plo) {
  const long long tt = blockIdx.x;
  const int i = tile_row(tt);
  const int j = (int)(tt - (long long)i * (i + 1) / 2);
  __nv_bfloat16* tile = P + tt * (long long)(T * T);
  __half* tlo = Plo + tt * (long long)(T * T);
  for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
    const int a = e / T, c = e % T;
    const int p = i * T + a, q = j * T + c;
    const double v = (p < n && q < n) ? G[(size_t)p * ld + q] * dinv[q] : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(v);
    tile[e] = h;
    const int k = p < n ? ilogbf(sigma[p]) : 0;
    tlo[e] = __ushort_as_half(f16_bits_scaled(v - (double)__bfloat162float(h), k));
  }
}

__global__ void to_float_kernel(const double* __restrict__ d, float* __restrict__ f, int n) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    f[p] = (float)d[p];
}

}  // namespace

pide_status build_sym_store(pide_ctx* c, const double* G, cudaStream_t st) {
  const int nt = (c->n + T - 1) / T;
  const long long ntiles = (long long)nt * (nt + 1) / 2;
  const size_t bytes = (size_t)ntiles * T * T * sizeof(__nv_bfloat16);
  PIDE_CUDA_TRY(cudaMallocAsync(&c->sym, bytes, st));
  PIDE_CUDA_TRY(cudaMallocAsync(&c->sym_lo, bytes, st));
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&c->dfl, (size_t)c->n * sizeof(float), st));
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&c->sym_scale, (size_t)c->n * sizeof(float), st));
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&c->ysum, (size_t)c->n * sizeof(double), st));
  PIDE_CUDA_TRY(cudaMemsetAsync(c->ysum, 0, (size_t)c->n * sizeof(double), st));
  c->sym_tiles = ntiles;
  c->sym_bytes = 2 * bytes;
  to_float_kernel<<<c->num_sms, 256, 0, st>>>(c->d, c->dfl, c->n);
  PIDE_CUDA_TRY(cudaGetLastError());
  sym_scale_kernel<<<c->n, 256, 0, st>>>(G, (size_t)c->ld, c->n, c->dinv, c->sym_scale);
  PIDE_CUDA_TRY(cudaGetLastError());
  pack_sym_kernel<<<(unsigned)ntiles, 256, 0, st>>>(G, (size_t)c->ld, c->n, c->dinv, c->sym_scale,
                                                   (__nv_bfloat16*)c->sym, (__half*)c->sym_lo);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_symv(pide_ctx* c, double* u, bool accumulate, cudaStream_t st) {
  const int grid = c->num_sms * 2;
  symv_bf16_kernel<<<grid, 256, 0, st>>>((const uint4*)c->sym, (const uint4*)c->sym_lo,
                                         c->sym_scale, c->sym_tiles, c->n,
                                         (const float*)c->R, c->dfl, c->ysum, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  symv_finish_kernel<<<c->num_sms * 2, 256, 0, st>>>(c->ysum, u, c->n, accumulate ? 1 : 0,
                                                      c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

}  // namespace pide
