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
// rewrites all of it that it reads (the right-hand side and its zero padding)
// before reading it, so nothing has to start at zero, and two calls whose work
// overlaps on the GPU (different streams, or different threads) race on it --
// serialise them.
//
// What it computes: the same refinement as pide_apply (first apply, then
// `sweeps` times an FP64 stencil residual and an apply-accumulate), with every
// right-hand side handed to the stored inverse in FP32 (pide_apply hands the
// tensor cores FP16, BF16 or e4m3).  The e4m3 correction term of a *_FP8 store
// joins the applies its correction mask selects, as in pide_apply.  So the two
// entry points agree once the refinement has converged, not apply by apply;
// an FP64 store needs two sweeps to come back from the FP32 right-hand side to
// FP64 accuracy.  The product is a CUDA-core matrix-vector kernel: FP32
// accumulation (FP64 for the FP64 store), 16-byte loads of the stored rows,
// four rows per warp sharing each load of the right-hand side.
#include <mutex>

#include "common.cuh"

namespace pide {
namespace {

constexpr int NOALLOC_MAX_COLS = 8;
constexpr int NOALLOC_MAX_N = 65536;
constexpr size_t NOALLOC_SCRATCH_FLOATS = (size_t)NOALLOC_MAX_COLS * NOALLOC_MAX_N;

// File-scope scratch: [NOALLOC_MAX_COLS][ldr] FP32 right-hand side / residual,
// ldr = n rounded up to 16 (<= NOALLOC_MAX_N), zero past n.
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

// R[col][p] = float(b) (first apply) or float(b - L u) (FP64 residual of Eq. 3)
// for p < n, and 0 for n <= p < ldr.
__global__ void noalloc_rhs_kernel(const double* __restrict__ b, const double* __restrict__ u,
                                   const double* __restrict__ w4, int n, int ldr, int mx,
                                   int residual, float* __restrict__ R) {
  const int col = blockIdx.y;
  const double* bc = b + (size_t)col * n;
  const double* uc = u + (size_t)col * n;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < ldr; p += gridDim.x * blockDim.x) {
    double r = 0.0;
    if (p < n) {
      r = bc[p];
      if (residual) {
        const int c = p % mx;
        r -= uc[p];
        if (c > 0) r = fma(w4[p], uc[p - 1], r);
        if (c < mx - 1) r = fma(w4[n + p], uc[p + 1], r);
        if (p >= mx) r = fma(w4[2 * n + p], uc[p - mx], r);
        if (p + mx < n) r = fma(w4[3 * n + p], uc[p + mx], r);
      }
    }
    R[(size_t)col * ldr + p] = (float)r;
  }
}

// Stored entries per 16-byte load, and their conversion to FP32.
template <int KIND> struct Store;
template <> struct Store<KIND_F64> { static constexpr int V = 2; };
template <> struct Store<KIND_F32> { static constexpr int V = 4; };
template <> struct Store<KIND_BF16> { static constexpr int V = 8; };
template <> struct Store<KIND_F16> { static constexpr int V = 8; };
template <> struct Store<KIND_FP8> { static constexpr int V = 16; };

__device__ __forceinline__ float e4m3_value(uint32_t byte) {
  __nv_fp8_e4m3 v;
  v.__x = (uint8_t)byte;
  return (float)v;
}

template <int KIND>
__device__ __forceinline__ void to_float(const uint4& raw, float (&a)[Store<KIND>::V]) {
  const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
  if constexpr (KIND == KIND_F32) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = __uint_as_float(w[i]);
  } else if constexpr (KIND == KIND_BF16) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[2 * i] = __uint_as_float(w[i] << 16);
      a[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  } else if constexpr (KIND == KIND_F16) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
      a[2 * i] = f.x;
      a[2 * i + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) a[4 * i + k] = e4m3_value(w[i] >> (8 * k));
  }
}

// The second term of a row, V e4m3 entries at the same positions: the FP8X2
// lo term (same row scale) or the e4m3 correction term (its own row scale).
// load_second fetches its V bytes, second_term converts them.
template <int V>
__device__ __forceinline__ uint4 load_second(const uint8_t* p) {
  if constexpr (V == 16) {
    return __ldcs(reinterpret_cast<const uint4*>(p));
  } else if constexpr (V == 8) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
    return make_uint4(v.x, v.y, 0u, 0u);
  } else if constexpr (V == 4) {
    return make_uint4(__ldcs(reinterpret_cast<const unsigned int*>(p)), 0u, 0u, 0u);
  } else {
    return make_uint4((uint32_t)p[0] | ((uint32_t)p[1] << 8), 0u, 0u, 0u);
  }
}

template <int V>
__device__ __forceinline__ void second_term(const uint4& raw, float (&a)[V]) {
  const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
  for (int k = 0; k < V; ++k) a[k] = e4m3_value(w[k >> 2] >> (8 * (k & 3)));
}

// u[c][p] (=|+=) scale_p * sum_q A[p][q] R[c][q] for the ROWS rows of each warp.
// A[p][q] = Q + ratio_p * T (T: the FP8X2 lo term with ratio 1, or the
// correction term C with ratio c_p / s_p), accumulated in FP32 and scaled by
// s_p (the row scale, 1 for BF16 and FP32) in FP64 at the end.
template <int KIND, int ROWS>
__global__ void __launch_bounds__(256) noalloc_gemv_kernel(
    const void* __restrict__ inv, const uint8_t* __restrict__ second,
    const float* __restrict__ row_scale, const float* __restrict__ second_scale, int ld, int n,
    int ldr, int B, const float* __restrict__ R, double* __restrict__ u, int accumulate) {
  constexpr int V = Store<KIND>::V;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int p0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * ROWS; p0 < n; p0 += warps * ROWS) {
    float acc[ROWS][NOALLOC_MAX_COLS];
    float ratio[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
#pragma unroll
      for (int c = 0; c < NOALLOC_MAX_COLS; ++c) acc[r][c] = 0.0f;
      const int p = min(p0 + r, n - 1);
      const float s = row_scale ? row_scale[p] : 1.0f;
      ratio[r] = second ? (second_scale ? second_scale[p] / s : 1.0f) : 0.0f;
    }
    for (int q = lane * V; q < ldr; q += 32 * V) {
      // every row's loads are issued before any is converted
      uint4 raw[ROWS];
      uint4 raw2[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const size_t e = (size_t)min(p0 + r, n - 1) * ld + q;
        raw[r] = __ldcs(reinterpret_cast<const uint4*>(
            reinterpret_cast<const uint8_t*>(inv) + e * (16 / V)));
        if (second) raw2[r] = load_second<V>(second + e);
      }
      float a[ROWS][V];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        to_float<KIND>(raw[r], a[r]);
        if (second) {
          float t[V];
          second_term<V>(raw2[r], t);
#pragma unroll
          for (int v = 0; v < V; ++v) a[r][v] = fmaf(ratio[r], t[v], a[r][v]);
        }
      }
#pragma unroll
      for (int c = 0; c < NOALLOC_MAX_COLS; ++c) {
        if (c >= B) break;
        const float4* x4 = reinterpret_cast<const float4*>(R + (size_t)c * ldr + q);
#pragma unroll
        for (int v4 = 0; v4 < V / 4; ++v4) {
          const float4 x = __ldg(x4 + v4);
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            acc[r][c] = fmaf(a[r][4 * v4 + 0], x.x, acc[r][c]);
            acc[r][c] = fmaf(a[r][4 * v4 + 1], x.y, acc[r][c]);
            acc[r][c] = fmaf(a[r][4 * v4 + 2], x.z, acc[r][c]);
            acc[r][c] = fmaf(a[r][4 * v4 + 3], x.w, acc[r][c]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int c = 0; c < NOALLOC_MAX_COLS; ++c)
        for (int o = 16; o > 0; o >>= 1) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], o);
    // lane r * 8 + c writes row p0 + r, column c
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int c = 0; c < NOALLOC_MAX_COLS; ++c)
        if (lane == r * NOALLOC_MAX_COLS + c && c < B && p0 + r < n) {
          const int p = p0 + r;
          const double s = row_scale ? (double)row_scale[p] : 1.0;
          double* dst = u + (size_t)c * n + p;
          const double v = (double)acc[r][c] * s;
          *dst = accumulate ? *dst + v : v;
        }
  }
}

// The FP64 store: one warp per row, FP64 products and sums.
__global__ void __launch_bounds__(256) noalloc_gemv_f64_kernel(
    const double* __restrict__ inv, int ld, int n, int ldr, int B, const float* __restrict__ R,
    double* __restrict__ u, int accumulate) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += warps) {
    double acc[NOALLOC_MAX_COLS];
#pragma unroll
    for (int c = 0; c < NOALLOC_MAX_COLS; ++c) acc[c] = 0.0;
    const double* row = inv + (size_t)p * ld;
    for (int q = lane * 2; q < ldr; q += 64) {
      const double2 a = __ldcs(reinterpret_cast<const double2*>(row + q));
#pragma unroll
      for (int c = 0; c < NOALLOC_MAX_COLS; ++c) {
        if (c >= B) break;
        const float2 x = __ldg(reinterpret_cast<const float2*>(R + (size_t)c * ldr + q));
        acc[c] = fma(a.x, (double)x.x, acc[c]);
        acc[c] = fma(a.y, (double)x.y, acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NOALLOC_MAX_COLS; ++c)
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
#pragma unroll
    for (int c = 0; c < NOALLOC_MAX_COLS; ++c)
      if (lane == c && c < B) {
        double* dst = u + (size_t)c * n + p;
        *dst = accumulate ? *dst + acc[c] : acc[c];
      }
  }
}

pide_status launch_noalloc_gemv(pide_ctx* c, const float* R, int ldr, int B, double* u,
                                bool accumulate, bool corrected, cudaStream_t st) {
  const int acc = accumulate ? 1 : 0;
  const int threads = 256;
  if (c->prec == PIDE_FP64) {
    int grid = (c->n + 7) / 8;
    if (grid > c->num_sms * 16) grid = c->num_sms * 16;
    noalloc_gemv_f64_kernel<<<grid, threads, 0, st>>>((const double*)c->inv, c->ld, c->n, ldr, B,
                                                      R, u, acc);
    return PIDE_OK;
  }
  // the second term: the FP8X2 lo term, or the correction term in the applies that add it
  const uint8_t* second = nullptr;
  const float* second_scale = nullptr;
  if (c->prec == PIDE_FP8X2) {
    second = (const uint8_t*)c->inv_lo;
  } else if (corrected && c->corr) {
    second = (const uint8_t*)c->corr;
    second_scale = c->corr_scale;
  }
  const float* rs = (c->prec == PIDE_FP16 || c->prec == PIDE_FP8 || c->prec == PIDE_FP8X2)
                        ? c->row_scale : nullptr;
  auto grid_for = [&](int rows) {
    int g = (c->n + rows * 8 - 1) / (rows * 8);
    return g > c->num_sms * 16 ? c->num_sms * 16 : g;
  };
  switch (c->prec) {
    case PIDE_FP32:
      noalloc_gemv_kernel<KIND_F32, 4><<<grid_for(4), threads, 0, st>>>(
          c->inv, second, rs, second_scale, c->ld, c->n, ldr, B, R, u, acc);
      break;
    case PIDE_BF16:
      noalloc_gemv_kernel<KIND_BF16, 4><<<grid_for(4), threads, 0, st>>>(
          c->inv, second, rs, second_scale, c->ld, c->n, ldr, B, R, u, acc);
      break;
    case PIDE_FP16:
      noalloc_gemv_kernel<KIND_F16, 4><<<grid_for(4), threads, 0, st>>>(
          c->inv, second, rs, second_scale, c->ld, c->n, ldr, B, R, u, acc);
      break;
    default:   // PIDE_FP8, PIDE_FP8X2 (e4m3 hi (+ lo) with the row scale)
      noalloc_gemv_kernel<KIND_FP8, 2><<<grid_for(2), threads, 0, st>>>(
          c->inv, second, rs, second_scale, c->ld, c->n, ldr, B, R, u, acc);
      break;
  }
  return PIDE_OK;
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
  const int ldr = (h->n + 15) / 16 * 16;           // <= NOALLOC_MAX_N and <= h->ld
  int gx = (ldr + 255) / 256;
  if (gx > 1024) gx = 1024;
  const dim3 rgrid(gx, B);
  // apply k adds the e4m3 correction term when bit k of the handle's mask is set
  auto corrected = [&](int k) { return h->corr && k < 31 && ((h->corr_mask >> k) & 1); };
  noalloc_rhs_kernel<<<rgrid, 256, 0, st>>>(b_dev, u_dev, h->w, h->n, ldr, h->mx, 0, R);
  PIDE_CUDA_TRY(cudaGetLastError());
  PIDE_TRY(launch_noalloc_gemv(h, R, ldr, B, u_dev, false, corrected(0), st));
  PIDE_CUDA_TRY(cudaGetLastError());
  for (int k = 0; k < sweeps; ++k) {
    noalloc_rhs_kernel<<<rgrid, 256, 0, st>>>(b_dev, u_dev, h->w, h->n, ldr, h->mx, 1, R);
    PIDE_CUDA_TRY(cudaGetLastError());
    PIDE_TRY(launch_noalloc_gemv(h, R, ldr, B, u_dev, true, corrected(k + 1), st));
    PIDE_CUDA_TRY(cudaGetLastError());
  }
  return PIDE_OK;
}
