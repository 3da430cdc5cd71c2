// Batched apply over independent problems: uneven grids, ragged column
// counts, FP32 or BF16 stored inverses, all in one launch per phase.
//
// A plan (pide_batch_create) uploads a problem table and two device work
// lists once:
//   tile items  (problem, 64-row tile, 64-column tile), ordered largest work
//               first (n_k x columns), pulled by persistent CTAs from an
//               atomic counter -- the apply of every problem in ONE launch;
//   column items (problem, column) -- prep and FP64 residual of every problem
//               in one launch each;
//   BF16 problems go to a grouped tcgen05 launch instead of the SIMT one:
//               (problem, 128-row tile, 64-column tile) items whose TMA maps
//               come from a device array of per-problem descriptors.
// pide_batch_run then issues prep, apply, and `sweeps` x (residual, apply):
// 2 + 2*sweeps launches for the whole set, optionally replayed from a CUDA
// graph captured on the first run.  Each problem may cap its own sweep count
// (an FP32 store needs fewer than a BF16 one): its items are skipped in the
// phases past its cap.  The apply is a register-tiled FP32 SIMT contraction
// (4 x 4 results per thread, columns contiguous per thread so warps past a
// problem's last column skip their arithmetic).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "df_arith.cuh"

namespace pide {
namespace {

struct BatchProb {
  const void* inv;      // [n][ld] FP32 or BF16 stored inverse
  const double* w;      // [4][n] Eq. (3) weights
  const float4* wsp;    // [2][n] the weights split into float pairs (hi, then lo), zero
                        // toward boundary neighbours
  const double* b;      // [B][n]
  double* u;            // [B][n]
  float* R;             // [B][ld] FP32 right-hand side / residual
  int ld, n, mx, B, fmt;  // fmt: 0 FP32, 1 BF16
  int pad;                // sweeps this problem runs (phases past it are skipped)
  int rbf16;              // 1: R holds BF16 for the grouped tensor-core apply, 0: FP32
};

// SIMT apply of the FP32 (and non-tensor-core BF16) problems.  An item is
// (problem, row tile, column tile, shape): the tile holds SB_OUT = 8192 outputs
// as TM x TN with TN = 16, 32 or 64 columns (the smallest that covers the
// problem's B, so small batches waste no lanes) and TM = 8192 / TN rows.
// 256 threads, each 8 rows x 4 columns; K in steps of 16, double-buffered in
// shared memory; A read as 16-byte vectors (4 FP32 or 4 BF16 entries).
constexpr int SB_K = 16;
constexpr int SB_OUT = 8192;
constexpr int SB_TMMAX = 512;
constexpr int SB_APAD = SB_TMMAX + 4;
constexpr int SB_XPAD = 64 + 4;
// FP32 problems stage A row-major through asynchronous copies instead:
// [TM][SB_APITCH] per stage (16 K values and 4 of padding per row).
constexpr int SB_APITCH = SB_K + 4;
constexpr int SB_A_FLOATS = (2 * SB_K * SB_APAD > 2 * SB_TMMAX * SB_APITCH)
                                ? 2 * SB_K * SB_APAD : 2 * SB_TMMAX * SB_APITCH;
constexpr size_t SB_SMEM = (size_t)(SB_A_FLOATS + 2 * SB_K * SB_XPAD) * sizeof(float);

__device__ __forceinline__ int sb_tn(int code) { return code == 0 ? 16 : (code == 1 ? 32 : 64); }

// four consecutive entries of row gp from column gk (gk a multiple of 4; zero past n)
__device__ __forceinline__ float4 load_a4(const BatchProb& P, int gp, int gk) {
  if (gp >= P.n || gk >= P.n) return make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t idx = (size_t)gp * P.ld + gk;
  if (gk + 3 < P.n) {
    if (P.fmt == 0) return *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(P.inv) + idx);
    const uint2 raw = *reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(P.inv) + idx);
    return make_float4(__uint_as_float(raw.x << 16), __uint_as_float(raw.x & 0xFFFF0000u),
                       __uint_as_float(raw.y << 16), __uint_as_float(raw.y & 0xFFFF0000u));
  }
  float v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = gk + j;
    v[j] = k < P.n ? (P.fmt == 0 ? reinterpret_cast<const float*>(P.inv)[idx + j]
                                 : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(P.inv)[idx + j]))
                   : 0.f;
  }
  return make_float4(v[0], v[1], v[2], v[3]);
}

// four consecutive entries of right-hand side gc from row gk (zero past n or past B)
__device__ __forceinline__ float4 load_x4(const BatchProb& P, int gc, bool col_ok, int gk) {
  if (!col_ok || gk >= P.n) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float* src = P.R + (size_t)gc * P.ld + gk;
  if (gk + 3 < P.n) return *reinterpret_cast<const float4*>(src);
  return make_float4(src[0], gk + 1 < P.n ? src[1] : 0.f, gk + 2 < P.n ? src[2] : 0.f, 0.f);
}

template <int TN>
__device__ __forceinline__ void simt_tile(const BatchProb& P, int p0, int c0, int accumulate,
                                          float* __restrict__ sA, float* __restrict__ sX) {
  constexpr int TM = SB_OUT / TN;
  constexpr int CG = TN / 4;             // column groups of 4
  constexpr int AL = TM / 64;            // float4 loads of A per thread and K step
  const int t = threadIdx.x;
  const int cg = t % CG, rg = t / CG;    // this thread: rows rg*8 .. +7, columns cg*4 .. +3
  const int ncols = min(TN, P.B - c0);
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float4 ra[AL], rx = make_float4(0.f, 0.f, 0.f, 0.f);
  const bool xloader = t < TN * 4;
  const int xc = t >> 2, xk = (t & 3) * 4;
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < AL; ++q) {
      const int e = t + 256 * q;
      ra[q] = load_a4(P, p0 + (e >> 2), k0 + (e & 3) * 4);
    }
    if (xloader) rx = load_x4(P, c0 + xc, xc < ncols, k0 + xk);
  };
  auto store = [&](int buf) {
    float* A = sA + buf * SB_K * SB_APAD;
#pragma unroll
    for (int q = 0; q < AL; ++q) {
      const int e = t + 256 * q;
      const int r = e >> 2, k = (e & 3) * 4;
      A[(k + 0) * SB_APAD + r] = ra[q].x;
      A[(k + 1) * SB_APAD + r] = ra[q].y;
      A[(k + 2) * SB_APAD + r] = ra[q].z;
      A[(k + 3) * SB_APAD + r] = ra[q].w;
    }
    if (xloader) {
      float* X = sX + buf * SB_K * SB_XPAD;
      X[(xk + 0) * SB_XPAD + xc] = rx.x;
      X[(xk + 1) * SB_XPAD + xc] = rx.y;
      X[(xk + 2) * SB_XPAD + xc] = rx.z;
      X[(xk + 3) * SB_XPAD + xc] = rx.w;
    }
  };
  const int nk = (P.n + SB_K - 1) / SB_K;
  load(0);
  store(0);
  __syncthreads();
  for (int ks = 0; ks < nk; ++ks) {
    const int buf = ks & 1;
    if (ks + 1 < nk) load((ks + 1) * SB_K);
    const float* A = sA + buf * SB_K * SB_APAD + rg * 8;
    const float* X = sX + buf * SB_K * SB_XPAD + cg * 4;
#pragma unroll
    for (int kk = 0; kk < SB_K; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(A + kk * SB_APAD);
      const float4 a1 = *reinterpret_cast<const float4*>(A + kk * SB_APAD + 4);
      const float4 x = *reinterpret_cast<const float4*>(X + kk * SB_XPAD);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], xv[j], acc[i][j]);
    }
    if (ks + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cg * 4 + j;
    if (c >= ncols) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = p0 + rg * 8 + i;
      if (p >= P.n) continue;
      double* dst = P.u + (size_t)(c0 + c) * P.n + p;
      *dst = accumulate ? *dst + (double)acc[i][j] : (double)acc[i][j];
    }
  }
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The same tile for an FP32 problem, A staged without a register round trip:
// 16-byte asynchronous copies into a row-major [TM][SB_APITCH] tile (zero-fill
// past n), read back with one 16-byte shared load per row and four K values.
// The thread's 8 rows are rg + RG i (RG = TM / 8), so that the 8 rows a warp
// reads at once are consecutive: stride 20 floats puts them in 8 distinct
// 4-bank groups.  No transposed scalar stores (the SIMT tile's main cost).
template <int TN>
__device__ __forceinline__ void simt_tile_async(const BatchProb& P, int p0, int c0, int accumulate,
                                                float* __restrict__ sA, float* __restrict__ sX) {
  constexpr int TM = SB_OUT / TN;
  constexpr int CG = TN / 4;
  constexpr int RG = TM / 8;
  constexpr int AC = TM * 4 / 256;       // 16-byte chunks of A per thread and K step
  const int t = threadIdx.x;
  const int cg = t % CG, rg = t / CG;
  const int ncols = min(TN, P.B - c0);
  const float* inv = reinterpret_cast<const float*>(P.inv);
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float4 rx = make_float4(0.f, 0.f, 0.f, 0.f);
  const bool xloader = t < TN * 4;
  const int xc = t >> 2, xk = (t & 3) * 4;
  auto issue_a = [&](int k0, int buf) {
    float* A = sA + buf * TM * SB_APITCH;
#pragma unroll
    for (int q = 0; q < AC; ++q) {
      const int c = t + 256 * q;
      const int r = c >> 2, kq = c & 3;
      const int gp = p0 + r, gk = k0 + kq * 4;
      int bytes = 0;
      const float* src = inv;
      if (gp < P.n && gk < P.n) {
        bytes = 4 * min(4, P.n - gk);
        src = inv + (size_t)gp * P.ld + gk;
      }
      cp_async16(A + r * SB_APITCH + kq * 4, src, bytes);
    }
    cp_async_commit();
  };
  auto store_x = [&](int buf) {
    if (xloader) {
      float* X = sX + buf * SB_K * SB_XPAD;
      X[(xk + 0) * SB_XPAD + xc] = rx.x;
      X[(xk + 1) * SB_XPAD + xc] = rx.y;
      X[(xk + 2) * SB_XPAD + xc] = rx.z;
      X[(xk + 3) * SB_XPAD + xc] = rx.w;
    }
  };
  const int nk = (P.n + SB_K - 1) / SB_K;
  issue_a(0, 0);
  if (xloader) rx = load_x4(P, c0 + xc, xc < ncols, xk);
  store_x(0);
  cp_async_wait_all();
  __syncthreads();
  for (int ks = 0; ks < nk; ++ks) {
    const int buf = ks & 1;
    if (ks + 1 < nk) {
      issue_a((ks + 1) * SB_K, buf ^ 1);
      if (xloader) rx = load_x4(P, c0 + xc, xc < ncols, (ks + 1) * SB_K + xk);
    }
    const float* A = sA + buf * TM * SB_APITCH + rg * SB_APITCH;
    const float* X = sX + buf * SB_K * SB_XPAD + cg * 4;
#pragma unroll
    for (int kq = 0; kq < 4; ++kq) {
      float4 a[8], x[4];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        a[i] = *reinterpret_cast<const float4*>(A + i * RG * SB_APITCH + kq * 4);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        x[kk] = *reinterpret_cast<const float4*>(X + (kq * 4 + kk) * SB_XPAD);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float xv[4] = {x[kk].x, x[kk].y, x[kk].z, x[kk].w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float av = kk == 0 ? a[i].x : (kk == 1 ? a[i].y : (kk == 2 ? a[i].z : a[i].w));
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av, xv[j], acc[i][j]);
        }
      }
    }
    if (ks + 1 < nk) store_x(buf ^ 1);
    cp_async_wait_all();
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cg * 4 + j;
    if (c >= ncols) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = p0 + rg + RG * i;
      if (p >= P.n) continue;
      double* dst = P.u + (size_t)(c0 + c) * P.n + p;
      *dst = accumulate ? *dst + (double)acc[i][j] : (double)acc[i][j];
    }
  }
}

__global__ void __launch_bounds__(256) batched_apply_kernel(const BatchProb* __restrict__ probs,
                                                            const int4* __restrict__ items,
                                                            int nitems, int* __restrict__ counter,
                                                            int accumulate, int phase, int sb_async) {
  extern __shared__ float sb_smem[];
  float* sA = sb_smem;
  float* sX = sb_smem + SB_A_FLOATS;
  __shared__ int s_item;
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const int4 w = items[it];
    const BatchProb P = probs[w.x];
    if (phase > P.pad) continue;                      // this problem already ran its sweeps
    const int tn = sb_tn(w.w);
    const int p0 = w.y * (SB_OUT / tn), c0 = w.z * tn;
    if (P.fmt == 0 && sb_async) {
      if (w.w == 0) simt_tile_async<16>(P, p0, c0, accumulate, sA, sX);
      else if (w.w == 1) simt_tile_async<32>(P, p0, c0, accumulate, sA, sX);
      else simt_tile_async<64>(P, p0, c0, accumulate, sA, sX);
    } else if (w.w == 0) simt_tile<16>(P, p0, c0, accumulate, sA, sX);
    else if (w.w == 1) simt_tile<32>(P, p0, c0, accumulate, sA, sX);
    else simt_tile<64>(P, p0, c0, accumulate, sA, sX);
  }
}

// Prep (residual == 0): R = q(b).  Residual: R = q(b - L u), the Eq. (3)
// stencil in double-float arithmetic on the integer and FP32 pipes (each FP64
// input split into two floats, error-free products and sums: absolute error
// ~2^-45 (|u_p| + sum_q w_pq |u_q|)); nodes with inputs outside the split's
// range, or whose own scale max(|b_p|, |u_p|) is below 2^-60, take the FP64
// formula.  q: FP32 (rounded from the pair) or BF16 (rounded to nearest from the
// pair, or from b's FP64 bits in the prep).
__global__ void __launch_bounds__(256) batched_vec_kernel(const BatchProb* __restrict__ probs,
                                                          const int2* __restrict__ items,
                                                          int residual, int phase) {
  const int2 w = items[blockIdx.x];
  const BatchProb P = probs[w.x];
  if (phase > P.pad) return;
  const int col = w.y;
  const double* bc = P.b + (size_t)col * P.n;
  const double* uc = P.u + (size_t)col * P.n;
  float* Rc = P.R + (size_t)col * P.ld;
  __nv_bfloat16* Rb = reinterpret_cast<__nv_bfloat16*>(P.R) + (size_t)col * P.ld;
  const int n = P.n, mx = P.mx;
  const float4* wh4 = P.wsp;
  const float4* wl4 = P.wsp + n;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    if (!residual) {
      const double bp = bc[p];
      if (P.rbf16) {
        Rb[p] = bf16_of_f64(bp);
      } else {
        float bh, bl;
        const uint32_t e = split47<false>(bp, bh, bl);
        Rc[p] = (e <= E_SPLIT_MAX && (e >= 920u || is_zero(bp))) ? __fadd_rn(bh, bl)
                                                                   : __double2float_rn(bp);
      }
      continue;
    }
    // neighbours from clamped indices: the split weights toward boundary nodes are zero
    const double vw = uc[p > 0 ? p - 1 : 0], ve = uc[p + 1 < n ? p + 1 : n - 1];
    const double vs = uc[p >= mx ? p - mx : 0], vn = uc[p + mx < n ? p + mx : n - 1];
    const double vp = uc[p], bp = bc[p];
    float wh_, wl_, eh, el, sh_, sl_, nh, nl, ph, pl, bh, bl;
    const uint32_t ew = split47<false>(vw, wh_, wl_), ee = split47<false>(ve, eh, el);
    const uint32_t es = split47<false>(vs, sh_, sl_), en = split47<false>(vn, nh, nl);
    const uint32_t ep = split47<false>(vp, ph, pl), eb = split47<false>(bp, bh, bl);
    const uint32_t emax = max(max(max(ew, ee), max(es, en)), max(ep, eb));
    float s, e;
    if (emax <= E_SPLIT_MAX && max(ep, eb) >= E_NODE_MIN) {
      const float4 wh = wh4[p], wl = wl4[p];
      float ah = bh, al = bl;
      df_add(ah, al, -ph, -pl);
      df_fma(ah, al, wh.x, wl.x, wh_, wl_);
      df_fma(ah, al, wh.y, wl.y, eh, el);
      df_fma(ah, al, wh.z, wl.z, sh_, sl_);
      df_fma(ah, al, wh.w, wl.w, nh, nl);
      s = __fadd_rn(ah, al);
      e = __fsub_rn(al, __fsub_rn(s, ah));
    } else {
      split_f64_slow(residual_node_fp64(bc, uc, P.w, nullptr, n, mx, n, p), s, e);
    }
    if (P.rbf16) Rb[p] = bf16_of_pair(s, e);
    else Rc[p] = s;
  }
}


// ---------------------------------------------------------------------------
// BF16 and FP32 problems: grouped tcgen05 launches.  Same pipeline as the
// main tensor-core apply (TMA producer warp, single-thread MMA issuer, four
// epilogue warps, 2 TMEM accumulators), but every (problem, 128-row tile,
// BN-column tile) item takes its TMA maps from a device array of per-problem
// descriptors, so problems of any size share the launch.  A BF16 problem
// contracts on kind::f16 (64 K values per 128-byte stage row); an FP32
// problem on kind::tf32 (32 K values per row): the tensor cores read each FP32
// entry of the stored inverse and of the FP32 right-hand side with TF32's 10
// explicit mantissa bits, and the refinement's FP64 residual wins the rest
// back.  The column-tile width BN (32, 64 or 128) is per problem (the
// PIDE_TUNE_BATCH_BN knob, which the autotuner sets); each width present in a
// plan is one launch per phase.
struct alignas(64) GroupProb {
  CUtensorMap tmA;      // stored L^-1 of the problem (box 128 bytes x 128 rows)
  CUtensorMap tmR;      // its right-hand-side workspace (box 128 bytes x BN rows)
  double* u;
  int n, B, num_kb, cap;
  int tf32;             // 1: FP32 store on kind::tf32, 0: BF16 on kind::f16
};

constexpr int G_A_BYTES = 128 * 128;
// stages of the grouped kernel for a column-tile width (~160-192 KB of shared memory)
constexpr int g_stages(int bn) { return bn >= 128 ? 6 : 8; }
constexpr size_t g_smem(int bn) {
  return 1024 + (size_t)g_stages(bn) * (G_A_BYTES + bn * 128) + 256;
}

template <int GBN>
__global__ void __launch_bounds__(192, 1) grouped_gemm_kernel(const GroupProb* __restrict__ probs,
                                                              const int4* __restrict__ items,
                                                              int nitems, int accumulate, int phase,
                                                              uint32_t* __restrict__ flags) {
  constexpr int GSTAGES = g_stages(GBN);
  constexpr int G_B_BYTES = GBN * 128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + GSTAGES * G_A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + GSTAGES * G_B_BYTES);
  uint64_t* empty = full + GSTAGES;
  uint64_t* tfull = empty + GSTAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int q = 0; q < GSTAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 128);
    }
    mbar_init(drain, 1);
    *abort_s = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 2 * GBN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    const uint64_t pol_a = policy_evict_first();
    int st = 0;
    uint32_t ph = 0, issued = 0, issued_ph = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      const int4 w = items[it];
      const GroupProb* P = probs + w.x;
      if (phase > P->cap) continue;
      const CUtensorMap* mA = &P->tmA;
      const CUtensorMap* mR = &P->tmR;
      prefetch_tmap(mA);
      prefetch_tmap(mR);
      for (int kb = 0; kb < P->num_kb; ++kb) {
        if (!mbar_wait_bounded(&empty[st], ph ^ 1, abort_s)) {
          ok = false;
          break;
        }
        // 128 bytes of K per stage row: 64 BF16 or 32 FP32 values
        const int kx = P->tf32 ? kb * 32 : kb * 64;
        mbar_expect_tx(&full[st], G_A_BYTES + G_B_BYTES);
        tma_load_2d_hint(sA + st * G_A_BYTES, mA, &full[st], kx, w.y * 128, pol_a);
        tma_load_2d(sB + st * G_B_BYTES, mR, &full[st], kx, w.z * GBN);
        issued |= 1u << st;
        issued_ph = (issued_ph & ~(1u << st)) | (ph << st);
        if (++st == GSTAGES) {
          st = 0;
          ph ^= 1;
        }
      }
    }
    if (!ok) {
      atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_TMA);
      *abort_s = 1;
      volatile int never = 0;
      for (int q = 0; q < GSTAGES; ++q)
        if (issued & (1u << q)) mbar_wait_bounded(&full[q], (issued_ph >> q) & 1u, &never);
    }
  } else if (warp == 1 && lane == 0) {
    // instruction descriptors: F32 accumulator (bits 4-5 = 1), A and B formats
    // (bits 7-9, 10-12: 1 = BF16 for kind::f16, 2 = TF32 for kind::tf32), both
    // K-major, N / 8 (bits 17-22), M / 16 (bits 24-28)
    const uint32_t shape = ((uint32_t)(GBN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t idesc_bf16 = (1u << 4) | (1u << 7) | (1u << 10) | shape;
    const uint32_t idesc_tf32 = (1u << 4) | (2u << 7) | (2u << 10) | shape;
    int st = 0, acc = 0;
    uint32_t ph = 0, acc_ph = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      const int4 w = items[it];
      const GroupProb* P = probs + w.x;
      if (phase > P->cap) continue;
      if (!mbar_wait_bounded(&tempty[acc], acc_ph ^ 1, abort_s)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * GBN);
      const int nkb = P->num_kb;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait_bounded(&full[st], ph, abort_s)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(sA + st * G_A_BYTES);
        const uint32_t b_addr = smem_u32(sB + st * G_B_BYTES);
        // four MMAs per stage, 32 bytes of K each (K = 16 BF16 or 8 TF32)
        if (P->tf32) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_tf32(d_tmem, smem_desc_sw128(a_addr + k * 32), smem_desc_sw128(b_addr + k * 32),
                     idesc_tf32, (kb > 0 || k > 0) ? 1u : 0u);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            mma_f16(d_tmem, smem_desc_sw128(a_addr + k * 32), smem_desc_sw128(b_addr + k * 32),
                    idesc_bf16, (kb > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&empty[st]);
        if (++st == GSTAGES) {
          st = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(&tfull[acc]);
      acc ^= 1;
      if (acc == 0) acc_ph ^= 1;
    }
    if (!ok) {
      atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_MMA);
      *abort_s = 1;
    }
    mma_commit(drain);
    volatile int never = 0;
    if (!mbar_wait_bounded(drain, 0, &never)) atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_DRAIN);
  } else if (warp >= 2) {
    const int quarter = warp & 3;
    const int row_in_tile = quarter * 32 + lane;
    int acc = 0;
    uint32_t acc_ph = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
      const int4 w = items[it];
      const GroupProb* P = probs + w.x;
      if (phase > P->cap) continue;
      bool ok = mbar_wait_bounded(&tfull[acc], acc_ph, abort_s);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_EPI);
          *abort_s = 1;
        }
        break;
      }
      tc_fence_after();
      const int n = P->n, B = P->B;
      double* u = P->u;
      const int p = w.y * 128 + row_in_tile;
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * GBN);
#pragma unroll 1
      for (int ch = 0; ch < GBN / 32; ++ch) {
        uint32_t v[32];
        tmem_ld_32x32b_x32(tbase + ch * 32, v);
        tmem_ld_wait();
        const int colbase = w.z * GBN + ch * 32;
        if (p < n) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = colbase + j;
            if (col < B) {
              double* dst = u + (size_t)col * n + p;
              const double val = f32_to_f64(__uint_as_float(v[j]));
              *dst = accumulate ? *dst + val : val;
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[acc]);
      acc ^= 1;
      if (acc == 0) acc_ph ^= 1;
    }
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, 2 * GBN);
  }
}

}  // namespace
}  // namespace pide

struct pide_batch {
  int nprob = 0, nitems = 0, ncolitems = 0;
  // grouped tensor-core items (BF16 and FP32 problems), one list per column-tile
  // width BN = 32, 64, 128
  int ngitems = 0;
  int ngitems_bn[3] = {0, 0, 0};
  pide::GroupProb* d_gprobs = nullptr;
  int4* d_gitems_bn[3] = {nullptr, nullptr, nullptr};
  int nsimt_shape[3] = {0, 0, 0};      // SIMT problems per tile width (16, 32, 64 columns)
  int ntf32 = 0;                       // FP32 problems on the TF32 tensor cores
  uint32_t* d_flags = nullptr;
  pide::BatchProb* d_probs = nullptr;
  int4* d_items = nullptr;
  int2* d_colitems = nullptr;
  int* d_counter = nullptr;   // one counter per apply launch of a run (reset by memset)
  int counters = 0;
  int num_sms = 0, device = 0;
  std::vector<pide_handle> hs;
  // graph replay, keyed by sweep count
  int graph_sweeps = -1;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
};

using namespace pide;

static void batch_free(pide_batch* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->d_probs) cudaFree(p->d_probs);
  if (p->d_items) cudaFree(p->d_items);
  if (p->d_colitems) cudaFree(p->d_colitems);
  if (p->d_counter) cudaFree(p->d_counter);
  if (p->d_gprobs) cudaFree(p->d_gprobs);
  for (int4* q : p->d_gitems_bn)
    if (q) cudaFree(q);
  if (p->d_flags) cudaFree(p->d_flags);
  delete p;
}

extern "C" pide_status pide_batch_create(const pide_handle* hs, int32_t nprob,
                                         const double* const* b, double* const* u,
                                         const int32_t* Bs, const int32_t* sweeps_k,
                                         pide_batch_handle* out) {
  if (out) *out = nullptr;
  if (!out || nprob < 0 || (nprob > 0 && (!hs || !b || !u || !Bs))) {
    set_error("pide_batch_create: bad argument");
    return PIDE_EINVAL;
  }
  for (int k = 0; k < nprob; ++k)
    if (hs[k] && hs[k]->dims == 3) {
      set_error("pide_batch_create: batched problems are 2-D grids");
      return PIDE_EUNSUPPORTED;
    }
  pide_batch* p = new pide_batch();
  std::vector<BatchProb> probs(nprob);
  struct Item { int prob, mt, ct; double cost; int shape = 0; };
  std::vector<Item> items, gitems_bn[3];
  std::vector<GroupProb> gprobs;
  std::vector<int> gindex(nprob, -1);
  std::vector<int2> colitems;
  int dev = -1;
  for (int k = 0; k < nprob; ++k) {
    pide_handle h = hs[k];
    if (!h || Bs[k] < 0 || (Bs[k] > 0 && (!b[k] || !u[k] || b[k] == u[k])) || Bs[k] > 65535) {
      batch_free(p);
      set_error("pide_batch_create: bad problem " + std::to_string(k));
      return PIDE_EINVAL;
    }
    if (h->prec != PIDE_FP32 && h->prec != PIDE_BF16) {
      batch_free(p);
      set_error("pide_batch_create: batched apply serves FP32 and BF16 stores");
      return PIDE_EUNSUPPORTED;
    }
    if (dev < 0) dev = h->device;
    if (h->device != dev) {
      batch_free(p);
      set_error("pide_batch_create: all handles must live on one device");
      return PIDE_EINVAL;
    }
    PIDE_CUDA_TRY(cudaSetDevice(h->device));
    pide_status s = ensure_workspace(h, Bs[k] > 0 ? Bs[k] : 1);
    if (s != PIDE_OK) {
      batch_free(p);
      return s;
    }
    probs[k] = BatchProb{h->inv, h->w, h->wsp, b[k], u[k], (float*)h->R, h->ld, h->n, h->mx, Bs[k],
                         h->prec == PIDE_FP32 ? 0 : 1,
                         sweeps_k ? (sweeps_k[k] < 0 ? 0 : sweeps_k[k]) : 1 << 30, 0};
    const bool tc_bf16 = h->prec == PIDE_BF16 && h->tmA_ok;
    const bool tc_tf32 = h->prec == PIDE_FP32 && h->batch_tc;
    if ((tc_bf16 || tc_tf32) && Bs[k] > 0) {
      // tensor cores: (problem, 128-row tile, BN-column tile) items with this problem's
      // maps; BN from the problem's knob, else the narrowest width that covers its
      // columns in one tile (each further column tile streams the inverse again)
      const int bn = h->batch_bn > 0 ? h->batch_bn : (Bs[k] <= 32 ? 32 : (Bs[k] <= 64 ? 64 : 128));
      const int bcode = bn == 32 ? 0 : (bn == 64 ? 1 : 2);
      GroupProb g;
      std::memset(&g, 0, sizeof(g));
      pide_status es = PIDE_OK;
      if (tc_bf16) {
        g.tmA = h->tmA;
        es = encode_2d(&g.tmR, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, h->R, h->n, h->ws_B,
                       (uint64_t)h->ld * 2, 64, bn);
      } else {
        es = encode_2d(&g.tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, h->inv, h->n, h->n,
                       (uint64_t)h->ld * 4, 32, 128);
        if (es == PIDE_OK)
          es = encode_2d(&g.tmR, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, h->R, h->n, h->ws_B,
                         (uint64_t)h->ld * 4, 32, bn);
      }
      if (es != PIDE_OK) {
        batch_free(p);
        return es;
      }
      g.u = u[k];
      g.n = h->n;
      g.B = Bs[k];
      g.tf32 = tc_tf32 ? 1 : 0;
      p->ntf32 += g.tf32;
      g.num_kb = tc_tf32 ? (h->n + 31) / 32 : (h->n + 63) / 64;
      g.cap = probs[k].pad;
      probs[k].rbf16 = tc_bf16 ? 1 : 0;
      gindex[k] = (int)gprobs.size();
      gprobs.push_back(g);
      const int mt = (h->n + 127) / 128, ct = (Bs[k] + bn - 1) / bn;
      // cost: K bytes streamed per item (an FP32 K block holds half the values)
      for (int i = 0; i < mt; ++i)
        for (int j = 0; j < ct; ++j) gitems_bn[bcode].push_back({gindex[k], i, j, (double)g.num_kb});
    } else if (Bs[k] > 0) {
      // SIMT: the tile width from the problem's knob, else the narrowest that
      // covers B (16, 32 or 64 columns)
      int code = Bs[k] <= 16 ? 0 : (Bs[k] <= 32 ? 1 : 2);
      if (h->batch_tn > 0) code = h->batch_tn == 16 ? 0 : (h->batch_tn == 32 ? 1 : 2);
      p->nsimt_shape[code] += 1;
      const int tn = code == 0 ? 16 : (code == 1 ? 32 : 64), tm = SB_OUT / tn;
      const int mt = (h->n + tm - 1) / tm, ct = (Bs[k] + tn - 1) / tn;
      for (int i = 0; i < mt; ++i)
        for (int j = 0; j < ct; ++j) items.push_back({k, i, j, (double)h->n * tm * tn, code});
    }
    for (int c = 0; c < Bs[k]; ++c) colitems.push_back(make_int2(k, c));
    p->hs.push_back(h);
    p->num_sms = h->num_sms;
    p->device = h->device;
  }
  // largest work first, so the tail of the dynamic schedule is made of small items
  std::stable_sort(items.begin(), items.end(),
                   [](const Item& a, const Item& c) { return a.cost > c.cost; });
  std::vector<int4> it4(items.size());
  for (size_t i = 0; i < items.size(); ++i) it4[i] = make_int4(items[i].prob, items[i].mt, items[i].ct, items[i].shape);
  std::vector<int4> g4[3];
  for (int q = 0; q < 3; ++q) {
    std::stable_sort(gitems_bn[q].begin(), gitems_bn[q].end(),
                     [](const Item& a, const Item& c) { return a.cost > c.cost; });
    for (const Item& t : gitems_bn[q]) g4[q].push_back(make_int4(t.prob, t.mt, t.ct, 0));
    p->ngitems_bn[q] = (int)g4[q].size();
    p->ngitems += p->ngitems_bn[q];
  }
  p->nprob = nprob;
  p->nitems = (int)it4.size();
  p->ncolitems = (int)colitems.size();
  p->counters = 64;
  auto fail = [&](cudaError_t e) {
    set_error(std::string("pide_batch_create: ") + cudaGetErrorString(e));
    batch_free(p);
    return e == cudaErrorMemoryAllocation ? PIDE_ENOMEM : PIDE_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaMalloc((void**)&p->d_probs, std::max<size_t>(1, probs.size()) * sizeof(BatchProb))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&p->d_items, std::max<size_t>(1, it4.size()) * sizeof(int4))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&p->d_colitems, std::max<size_t>(1, colitems.size()) * sizeof(int2))) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc((void**)&p->d_counter, p->counters * sizeof(int))) != cudaSuccess) return fail(e);
  if (!probs.empty() && (e = cudaMemcpy(p->d_probs, probs.data(), probs.size() * sizeof(BatchProb), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if (!it4.empty() && (e = cudaMemcpy(p->d_items, it4.data(), it4.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if (!colitems.empty() && (e = cudaMemcpy(p->d_colitems, colitems.data(), colitems.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if (!gprobs.empty()) {
    if ((e = cudaMalloc((void**)&p->d_gprobs, gprobs.size() * sizeof(GroupProb))) != cudaSuccess) return fail(e);
    for (int q = 0; q < 3; ++q)
      if (!g4[q].empty() &&
          (e = cudaMalloc((void**)&p->d_gitems_bn[q], g4[q].size() * sizeof(int4))) != cudaSuccess)
        return fail(e);
    if ((e = cudaMalloc((void**)&p->d_flags, FLAG_COUNT * sizeof(uint32_t))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(p->d_flags, 0, FLAG_COUNT * sizeof(uint32_t))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(p->d_gprobs, gprobs.data(), gprobs.size() * sizeof(GroupProb), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    for (int q = 0; q < 3; ++q)
      if (!g4[q].empty() && (e = cudaMemcpy(p->d_gitems_bn[q], g4[q].data(), g4[q].size() * sizeof(int4),
                                            cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    if ((e = cudaFuncSetAttribute(grouped_gemm_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_smem(32))) != cudaSuccess) return fail(e);
    if ((e = cudaFuncSetAttribute(grouped_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_smem(64))) != cudaSuccess) return fail(e);
    if ((e = cudaFuncSetAttribute(grouped_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_smem(128))) != cudaSuccess) return fail(e);
  }
  *out = p;
  return PIDE_OK;
}

static pide_status batch_apply(pide_batch* p, int phase, cudaStream_t st) {
  if (p->nitems > 0) {
    const int grid_apply = std::min(p->nitems, p->num_sms * 2);
    PIDE_CUDA_TRY(cudaFuncSetAttribute(batched_apply_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SB_SMEM));
    batched_apply_kernel<<<grid_apply, 256, SB_SMEM, st>>>(p->d_probs, p->d_items, p->nitems,
                                                           p->d_counter + phase, phase > 0, phase, 1);
    PIDE_CUDA_TRY(cudaGetLastError());
  }
  // one grouped launch per column-tile width present in the plan
  for (int q = 0; q < 3; ++q) {
    const int ni = p->ngitems_bn[q];
    if (ni == 0) continue;
    const int grid = std::min(ni, p->num_sms);
    if (q == 0)
      grouped_gemm_kernel<32><<<grid, 192, g_smem(32), st>>>(p->d_gprobs, p->d_gitems_bn[q], ni,
                                                             phase > 0, phase, p->d_flags);
    else if (q == 1)
      grouped_gemm_kernel<64><<<grid, 192, g_smem(64), st>>>(p->d_gprobs, p->d_gitems_bn[q], ni,
                                                             phase > 0, phase, p->d_flags);
    else
      grouped_gemm_kernel<128><<<grid, 192, g_smem(128), st>>>(p->d_gprobs, p->d_gitems_bn[q], ni,
                                                               phase > 0, phase, p->d_flags);
    PIDE_CUDA_TRY(cudaGetLastError());
  }
  return PIDE_OK;
}

static pide_status batch_enqueue(pide_batch* p, int sweeps, cudaStream_t st) {
  if (p->nitems == 0 && p->ngitems == 0) return PIDE_OK;
  if (1 + sweeps > p->counters) {
    set_error("pide_batch_run: at most 63 sweeps");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, (1 + sweeps) * sizeof(int), st));
  batched_vec_kernel<<<p->ncolitems, 256, 0, st>>>(p->d_probs, p->d_colitems, 0, 0);
  PIDE_CUDA_TRY(cudaGetLastError());
  PIDE_TRY(batch_apply(p, 0, st));
  for (int k = 0; k < sweeps; ++k) {
    batched_vec_kernel<<<p->ncolitems, 256, 0, st>>>(p->d_probs, p->d_colitems, 1, k + 1);
    PIDE_CUDA_TRY(cudaGetLastError());
    PIDE_TRY(batch_apply(p, k + 1, st));
  }
  return PIDE_OK;
}

extern "C" pide_status pide_batch_run(pide_batch_handle p, int32_t sweeps, int32_t use_graph,
                                      void* stream) {
  if (!p || sweeps < 0) {
    set_error("pide_batch_run: bad argument");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (!use_graph || st == nullptr) return batch_enqueue(p, sweeps, st);
  if (p->exec == nullptr || p->graph_sweeps != sweeps) {
    if (p->exec) {
      cudaGraphExecDestroy(p->exec);
      p->exec = nullptr;
    }
    PIDE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    pide_status s = batch_enqueue(p, sweeps, st);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != PIDE_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    PIDE_CUDA_TRY(e);
    e = cudaGraphInstantiate(&p->exec, g, 0);
    cudaGraphDestroy(g);
    PIDE_CUDA_TRY(e);
    p->graph_sweeps = sweeps;
  }
  PIDE_CUDA_TRY(cudaGraphLaunch(p->exec, st));
  return PIDE_OK;
}

extern "C" pide_status pide_batch_get_info(pide_batch_handle p, pide_batch_info* out) {
  if (!p || !out) {
    set_error("pide_batch_get_info: bad argument");
    return PIDE_EINVAL;
  }
  std::memset(out, 0, sizeof(*out));
  out->nprob = p->nprob;
  out->simt_items = p->nitems;
  out->tc_items = p->ngitems;
  for (int q = 0; q < 3; ++q) {
    out->tc_items_bn[q] = p->ngitems_bn[q];
    out->simt_problems_tn[q] = p->nsimt_shape[q];
    out->apply_launches += p->ngitems_bn[q] > 0 ? 1 : 0;
  }
  out->apply_launches += p->nitems > 0 ? 1 : 0;
  out->tf32_problems = p->ntf32;
  return PIDE_OK;
}

extern "C" void pide_batch_destroy(pide_batch_handle p) {
  if (!p) return;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  batch_free(p);
}

extern "C" pide_status pide_apply_batched_impl(const pide_handle* hs, int32_t nprob,
                                               const double* const* b, double* const* u,
                                               const int32_t* Bs, int32_t sweeps, void* stream) {
  pide_batch_handle p = nullptr;
  PIDE_TRY(pide_batch_create(hs, nprob, b, u, Bs, nullptr, &p));
  pide_status s = pide_batch_run(p, sweeps, 0, stream);
  if (s == PIDE_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) s = PIDE_ECUDA;
  batch_free(p);
  return s;
}
