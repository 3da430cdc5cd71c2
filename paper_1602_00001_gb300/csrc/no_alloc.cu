// pide_apply_noalloc: a refined apply that allocates no device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a caller
// that owns a fixed memory pool and forbids other allocations, one that runs
// inside a region where an allocation would synchronise the device or fail
// (for example a real-time loop, or a plugin that receives only pre-sized
// buffers from its host application).  Such a caller still passes its own
// input and output buffers; the one scratch buffer this apply needs (the
// FP32 right-hand side / residual handed from the stencil to the product)
// lives in a fixed array compiled into the library instead of the handle's
// workspace.
//
// Limits: at most NOALLOC_MAX_COLS = 8 right-hand sides and
// NOALLOC_MAX_N = 65536 unknowns per call (2 MiB of scratch).  Every GPU that
// loads the library holds that array until the process exits.
//
// The scratch array is shared by every call in the process: each call
// overwrites what it needs before reading it (nothing in it has to start at
// zero), and two calls whose work overlaps on the GPU (different streams, or
// different threads) race on it -- serialise them.
//
// The product here is a plain warp-per-row matrix-vector kernel reading the
// right-hand side from the scratch array; the numbers match pide_apply up to
// FP32 summation order.
#include <mutex>

#include "common.cuh"

namespace pide {
namespace {

constexpr int NOALLOC_MAX_COLS = 8;
constexpr int NOALLOC_MAX_N = 65536;
constexpr size_t NOALLOC_SCRATCH_FLOATS = (size_t)NOALLOC_MAX_COLS * NOALLOC_MAX_N;

// File-scope scratch: [NOALLOC_MAX_COLS][n] FP32 right-hand side / residual.
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

// Host code cannot use g_noalloc_scratch as a device address; its address on
// each device is looked up once (cudaGetSymbolAddress, that device current)
// and kept here.
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

pide_status noalloc_scratch(int dev, float** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("pide_apply_noalloc: device ordinal out of range");
    return PIDE_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("pide_apply_noalloc: cudaGetSymbolAddress failed: ") +
                cudaGetErrorString(e));
      return PIDE_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_addr[dev];
  return PIDE_OK;
}

// R[col][p] = float(b) (first apply) or float(b - L u) (FP64 residual of Eq. 3).
__global__ void noalloc_rhs_kernel(const double* __restrict__ b, const double* __restrict__ u,
                                   const double* __restrict__ w4, int n, int mx, int residual,
                                   float* __restrict__ R) {
  const int col = blockIdx.y;
  const double* bc = b + (size_t)col * n;
  const double* uc = u + (size_t)col * n;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double r = bc[p];
    if (residual) {
      const int c = p % mx;
      r -= uc[p];
      if (c > 0) r = fma(w4[p], uc[p - 1], r);
      if (c < mx - 1) r = fma(w4[n + p], uc[p + 1], r);
      if (p >= mx) r = fma(w4[2 * n + p], uc[p - mx], r);
      if (p + mx < n) r = fma(w4[3 * n + p], uc[p + mx], r);
    }
    R[(size_t)col * n + p] = (float)r;
  }
}

__device__ __forceinline__ float stored_entry(const void* inv, const void* inv_lo, int fmt,
                                              size_t e) {
  switch (fmt) {
    case PIDE_FP64: return (float)reinterpret_cast<const double*>(inv)[e];
    case PIDE_FP32: return reinterpret_cast<const float*>(inv)[e];
    case PIDE_BF16: return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(inv)[e]);
    case PIDE_FP16: return __half2float(reinterpret_cast<const __half*>(inv)[e]);   // row scale outside
    default: {
      float v = (float)reinterpret_cast<const __nv_fp8_e4m3*>(inv)[e];
      if (inv_lo) v += (float)reinterpret_cast<const __nv_fp8_e4m3*>(inv_lo)[e];
      return v;
    }
  }
}

// One warp per row p: u[col][p] (=|+=) scale_p * sum_q Q[p][q] R[col][q].
// The FP64 store is read in FP64 and summed in FP64.
__global__ void __launch_bounds__(256) noalloc_gemv_kernel(
    const void* __restrict__ inv, const void* __restrict__ inv_lo,
    const float* __restrict__ row_scale, int fmt, int ld, int n, int B,
    const float* __restrict__ R, double* __restrict__ u, int accumulate) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    double acc[NOALLOC_MAX_COLS];
#pragma unroll
    for (int c = 0; c < NOALLOC_MAX_COLS; ++c) acc[c] = 0.0;
    const size_t row = (size_t)p * ld;
    for (int q = lane; q < n; q += 32) {
      const double a = fmt == PIDE_FP64 ? reinterpret_cast<const double*>(inv)[row + q]
                                        : (double)stored_entry(inv, inv_lo, fmt, row + q);
#pragma unroll
      for (int c = 0; c < NOALLOC_MAX_COLS; ++c)
        if (c < B) acc[c] = fma(a, (double)R[(size_t)c * n + q], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NOALLOC_MAX_COLS; ++c) {
      double v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[c] = v;
    }
    if (lane == 0) {
      const double s = row_scale ? (double)row_scale[p] : 1.0;
      for (int c = 0; c < B; ++c) {
        double* dst = u + (size_t)c * n + p;
        *dst = accumulate ? *dst + acc[c] * s : acc[c] * s;
      }
    }
  }
}

}  // namespace
}  // namespace pide

using namespace pide;

extern "C" pide_status pide_apply_noalloc(pide_handle h, const double* b_dev, double* u_dev,
                                          int32_t B, int32_t sweeps, void* stream) {
  if (!h || B < 0 || sweeps < 0 || (B > 0 && (!b_dev || !u_dev || b_dev == u_dev))) {
    set_error("pide_apply_noalloc: bad argument (handle, pointers, B >= 0, sweeps >= 0, b != u)");
    return PIDE_EINVAL;
  }
  if (B > NOALLOC_MAX_COLS || h->n > NOALLOC_MAX_N) {
    set_error("pide_apply_noalloc: at most " + std::to_string(NOALLOC_MAX_COLS) +
              " right-hand sides and " + std::to_string(NOALLOC_MAX_N) +
              " unknowns per call (got B = " + std::to_string(B) + ", n = " +
              std::to_string(h->n) + "); use pide_apply for larger problems");
    return PIDE_EINVAL;
  }
  if (h->dims == 3) {
    set_error("pide_apply_noalloc: 2-D grids only");
    return PIDE_EUNSUPPORTED;
  }
  if (B == 0) return PIDE_OK;
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  float* R = nullptr;
  PIDE_TRY(noalloc_scratch(h->device, &R));
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 rgrid((h->n + 255) / 256, B);
  const int ggrid = h->num_sms * 8;
  const int fmt = (int)h->prec;
  noalloc_rhs_kernel<<<rgrid, 256, 0, st>>>(b_dev, u_dev, h->w, h->n, h->mx, 0, R);
  PIDE_CUDA_TRY(cudaGetLastError());
  noalloc_gemv_kernel<<<ggrid, 256, 0, st>>>(h->inv, h->inv_lo, h->row_scale, fmt, h->ld, h->n,
                                             B, R, u_dev, 0);
  PIDE_CUDA_TRY(cudaGetLastError());
  for (int k = 0; k < sweeps; ++k) {
    noalloc_rhs_kernel<<<rgrid, 256, 0, st>>>(b_dev, u_dev, h->w, h->n, h->mx, 1, R);
    PIDE_CUDA_TRY(cudaGetLastError());
    noalloc_gemv_kernel<<<ggrid, 256, 0, st>>>(h->inv, h->inv_lo, h->row_scale, fmt, h->ld,
                                               h->n, B, R, u_dev, 1);
    PIDE_CUDA_TRY(cudaGetLastError());
  }
  return PIDE_OK;
}
