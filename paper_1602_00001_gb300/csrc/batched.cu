// Batched apply over independent problems: uneven grids, ragged column
// counts, FP32 or BF16 stored inverses, all in one launch per phase.
//
// A plan (pide_batch_create) uploads a problem table and two device work
// lists once:
//   tile items  (problem, 128-row tile, 64-column tile), ordered largest work
//               first (n_k x columns), pulled by persistent CTAs from an
//               atomic counter -- the apply of every problem in ONE launch;
//   column items (problem, column) -- prep and FP64 residual of every problem
//               in one launch each.
// pide_batch_run then issues prep, apply, and `sweeps` x (residual, apply):
// 2 + 2*sweeps launches for the whole set, optionally replayed from a CUDA
// graph captured on the first run.  Each problem may cap its own sweep count
// (an FP32 store needs fewer than a BF16 one): its items are skipped in the
// phases past its cap.  The apply is a register-tiled FP32 SIMT contraction
// (8 x 4 results per thread, columns contiguous per thread so warps past a
// problem's last column skip their arithmetic).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace pide {
namespace {

struct BatchProb {
  const void* inv;      // [n][ld] FP32 or BF16 stored inverse
  const double* w;      // [4][n] Eq. (3) weights
  const double* b;      // [B][n]
  double* u;            // [B][n]
  float* R;             // [B][ld] FP32 right-hand side / residual
  int ld, n, mx, B, fmt;  // fmt: 0 FP32, 1 BF16
  int pad;                // sweeps this problem runs (phases past it are skipped)
};

constexpr int BM = 128;  // rows per tile item
constexpr int BT = 64;   // columns per tile item
constexpr int BK = 32;   // K step

__device__ __forceinline__ float load_a(const BatchProb& P, size_t idx) {
  if (P.fmt == 0) return reinterpret_cast<const float*>(P.inv)[idx];
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(P.inv)[idx]);
}

// 128 x 64 output tile per item, 256 threads: thread (tx, ty) owns rows
// 4 tx .. +3 and 64 + 4 tx .. +3 and columns 4 ty .. +3 (32 accumulators);
// per k it reads three float4 from shared memory for 32 FMAs.
__global__ void __launch_bounds__(256) batched_apply_kernel(const BatchProb* __restrict__ probs,
                                                            const int4* __restrict__ items,
                                                            int nitems, int* __restrict__ counter,
                                                            int accumulate, int phase) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Xs[BK][BT + 4];
  __shared__ int s_item;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const int4 w = items[it];
    const BatchProb P = probs[w.x];
    if (phase > P.pad) continue;                      // this problem already ran its sweeps
    const int p0 = w.y * BM, c0 = w.z * BT;
    const int ncols = min(BT, P.B - c0);
    const bool active = ty * 4 < ncols;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < P.n; k0 += BK) {
#pragma unroll
      for (int q = 0; q < (BM * BK) / 256; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int r = e / BK, kk = e % BK;
        const int gk = k0 + kk, gp = p0 + r;
        As[kk][r] = (gp < P.n && gk < P.n) ? load_a(P, (size_t)gp * P.ld + gk) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < (BT * BK) / 256; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int r = e / BK, kk = e % BK;
        const int gk = k0 + kk;
        Xs[kk][r] = (r < ncols && gk < P.n) ? P.R[(size_t)(c0 + r) * P.ld + gk] : 0.f;
      }
      __syncthreads();
      if (active) {
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
          const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][4 * tx]);
          const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + 4 * tx]);
          const float4 xv = *reinterpret_cast<const float4*>(&Xs[kk][4 * ty]);
          const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], xs[j], acc[i][j]);
        }
      }
      __syncthreads();
    }
    if (active) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = ty * 4 + j;
        if (c >= ncols) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int p = p0 + (i < 4 ? 4 * tx + i : 64 + 4 * tx + (i - 4));
          if (p >= P.n) continue;
          double* dst = P.u + (size_t)(c0 + c) * P.n + p;
          *dst = accumulate ? *dst + (double)acc[i][j] : (double)acc[i][j];
        }
      }
    }
  }
}

// Prep (residual == 0): R = float(b).  Residual: R = float(b - L u), FP64.
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
  const int n = P.n, mx = P.mx;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double r = bc[p];
    if (residual) {
      const int c = p % mx;
      r -= uc[p];
      if (c > 0) r = fma(P.w[p], uc[p - 1], r);
      if (c < mx - 1) r = fma(P.w[n + p], uc[p + 1], r);
      if (p >= mx) r = fma(P.w[2 * n + p], uc[p - mx], r);
      if (p + mx < n) r = fma(P.w[3 * n + p], uc[p + mx], r);
    }
    Rc[p] = (float)r;
  }
}

}  // namespace
}  // namespace pide

struct pide_batch {
  int nprob = 0, nitems = 0, ncolitems = 0;
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
  pide_batch* p = new pide_batch();
  std::vector<BatchProb> probs(nprob);
  struct Item { int prob, mt, ct; double cost; };
  std::vector<Item> items;
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
    probs[k] = BatchProb{h->inv, h->w, b[k], u[k], (float*)h->R, h->ld, h->n, h->mx, Bs[k],
                         h->prec == PIDE_FP32 ? 0 : 1,
                         sweeps_k ? (sweeps_k[k] < 0 ? 0 : sweeps_k[k]) : 1 << 30};
    const int mt = (h->n + BM - 1) / BM, ct = (Bs[k] + BT - 1) / BT;
    for (int i = 0; i < mt; ++i)
      for (int j = 0; j < ct; ++j) {
        const int cols = std::min(BT, Bs[k] - j * BT);
        items.push_back({k, i, j, (double)h->n * ((cols + 3) / 4)});
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
  for (size_t i = 0; i < items.size(); ++i) it4[i] = make_int4(items[i].prob, items[i].mt, items[i].ct, 0);
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
  *out = p;
  return PIDE_OK;
}

static pide_status batch_enqueue(pide_batch* p, int sweeps, cudaStream_t st) {
  if (p->nitems == 0) return PIDE_OK;
  if (1 + sweeps > p->counters) {
    set_error("pide_batch_run: at most 63 sweeps");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, (1 + sweeps) * sizeof(int), st));
  const int grid_apply = std::min(p->nitems, p->num_sms * 4);
  batched_vec_kernel<<<p->ncolitems, 256, 0, st>>>(p->d_probs, p->d_colitems, 0, 0);
  PIDE_CUDA_TRY(cudaGetLastError());
  batched_apply_kernel<<<grid_apply, 256, 0, st>>>(p->d_probs, p->d_items, p->nitems,
                                                   p->d_counter, 0, 0);
  PIDE_CUDA_TRY(cudaGetLastError());
  for (int k = 0; k < sweeps; ++k) {
    batched_vec_kernel<<<p->ncolitems, 256, 0, st>>>(p->d_probs, p->d_colitems, 1, k + 1);
    PIDE_CUDA_TRY(cudaGetLastError());
    batched_apply_kernel<<<grid_apply, 256, 0, st>>>(p->d_probs, p->d_items, p->nitems,
                                                     p->d_counter + 1 + k, 1, k + 1);
    PIDE_CUDA_TRY(cudaGetLastError());
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
