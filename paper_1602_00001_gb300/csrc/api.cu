// C ABI of libpide (declared in include/pide.h): handle life cycle, the
// refinement driver around the apply kernels, host-buffer apply, adjoint,
// batched apply, persistence and profiling.
#include <cudaTypedefs.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace pide {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

size_t rhs_elem_bytes(int rfmt) {
  switch (rfmt) {
    case RF_F64: return 8;
    case RF_F32: return 4;
    case RF_BF16: return 2;
    default: return 1;
  }
}

int rhs_format(const pide_ctx* c, int B) {
  switch (c->prec) {
    case PIDE_FP64: return RF_F64;
    case PIDE_FP32: return RF_F32;
    case PIDE_BF16: return B <= c->gemv_max_b ? RF_F32 : RF_BF16;
    case PIDE_FP16: return B <= c->gemv_max_b ? RF_F32 : RF_F16;
    default: return B <= c->gemv_max_b ? RF_F32 : RF_E4M3;
  }
}

ProfScope::ProfScope(pide_ctx* c_, cudaStream_t st_, int cls_) : c(c_), st(st_), cls(cls_) {
  if (c && c->prof_on) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
}

ProfScope::~ProfScope() {
  if (a) {
    cudaEventRecord(b, st);
    c->prof_events.push_back({a, b, cls});
  }
}

// ---------------------------------------------------------------- TMA maps

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

pide_status encode_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base,
                             uint64_t inner, uint64_t outer, uint64_t row_bytes, uint32_t box_in,
                             uint32_t box_out) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return PIDE_EUNSUPPORTED;
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_in, box_out};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
    return PIDE_ECUDA;
  }
  return PIDE_OK;
}

pide_status make_tma_maps(pide_ctx* c) {
  c->tmA_ok = false;
  if (c->prec == PIDE_BF16 || c->prec == PIDE_FP16) {
    PIDE_TRY(encode_2d(&c->tmA, c->prec == PIDE_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                       c->inv, c->n, c->n, (uint64_t)c->ld * 2, 64, 128));
  } else if (c->prec == PIDE_FP8 || c->prec == PIDE_FP8X2) {
    PIDE_TRY(encode_2d(&c->tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, c->inv, c->n, c->n,
                       (uint64_t)c->ld, 128, 128));
    if (c->prec == PIDE_FP8X2)
      PIDE_TRY(encode_2d(&c->tmA_lo, CU_TENSOR_MAP_DATA_TYPE_UINT8, c->inv_lo, c->n, c->n,
                         (uint64_t)c->ld, 128, 128));
    else
      c->tmA_lo = c->tmA;
  } else {
    return PIDE_OK;
  }
  if (c->corr)
    PIDE_TRY(encode_2d(&c->tmA_corr, CU_TENSOR_MAP_DATA_TYPE_UINT8, c->corr, c->n, c->n,
                       (uint64_t)c->ld, 128, 128));
  c->tmA_ok = true;
  return PIDE_OK;
}

pide_status make_tma_rhs(pide_ctx* c, int bn) {
  if (c->prec == PIDE_BF16 || c->prec == PIDE_FP16)
    return encode_2d(&c->tmR, c->prec == PIDE_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                     c->R, c->n, c->ws_B, (uint64_t)c->ld * 2, 64, bn);
  return encode_2d(&c->tmR, CU_TENSOR_MAP_DATA_TYPE_UINT8, c->R, c->n, c->ws_B, (uint64_t)c->ld,
                   128, bn);
}

pide_status make_tma_rhs_corr(pide_ctx* c, int bn) {
  if (!c->Rc) return PIDE_EINVAL;
  return encode_2d(&c->tmRc, CU_TENSOR_MAP_DATA_TYPE_UINT8, c->Rc, c->n, c->ws_B,
                   (uint64_t)c->ld, 128, bn);
}

// ---------------------------------------------------------------- workspace

pide_status ensure_workspace(pide_ctx* c, int B) {
  // the SM-pair GEMM's partial tiles (B > 128 only): four 256 x 256 FP32 slots
  // per pair (80 MB at 152 SMs), allocated once so that a captured apply
  // allocates nothing
  if (!c->tail_ws && B > 128 &&
      (c->prec == PIDE_BF16 || c->prec == PIDE_FP8 || c->prec == PIDE_FP8X2 ||
       c->prec == PIDE_FP16)) {
    const int slots = 4 * (c->num_sms / 2 > 0 ? c->num_sms / 2 : 1);
    PIDE_CUDA_TRY(cudaMalloc((void**)&c->tail_ws, (size_t)slots * 256 * 256 * sizeof(float)));
    c->tail_slots = slots;
  }
  if (B <= c->ws_B && c->R) return PIDE_OK;
  int nb = B < 16 ? 16 : B;
  if (c->R) cudaFree(c->R);
  if (c->col_scale) cudaFree(c->col_scale);
  if (c->colmax) cudaFree(c->colmax);
  if (c->Rf) cudaFree(c->Rf);
  if (c->Rc) cudaFree(c->Rc);
  if (c->col_scale_c) cudaFree(c->col_scale_c);
  c->R = nullptr;
  c->col_scale = nullptr;
  c->colmax = nullptr;
  c->Rf = nullptr;
  c->Rc = nullptr;
  c->col_scale_c = nullptr;
  c->ws_B = 0;
  const size_t esz = c->prec == PIDE_FP64 ? 8 : 4;
  PIDE_CUDA_TRY(cudaMalloc(&c->R, (size_t)nb * c->ld * esz));
  PIDE_CUDA_TRY(cudaMemset(c->R, 0, (size_t)nb * c->ld * esz));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->col_scale, (size_t)nb * sizeof(float)));
  if (c->prec == PIDE_FP8 || c->prec == PIDE_FP8X2)
    PIDE_CUDA_TRY(cudaMalloc((void**)&c->Rf, (size_t)nb * c->ld * sizeof(float)));
  if (c->corr) {
    PIDE_CUDA_TRY(cudaMalloc(&c->Rc, (size_t)nb * c->ld));
    PIDE_CUDA_TRY(cudaMalloc((void**)&c->col_scale_c, (size_t)nb * sizeof(float)));
  }
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->colmax, 3 * (size_t)nb * sizeof(double)));
  PIDE_CUDA_TRY(cudaMemset(c->colmax, 0, 3 * (size_t)nb * sizeof(double)));
  c->ws_B = nb;
  return PIDE_OK;
}

// ---------------------------------------------------------------- apply

static pide_status apply_dispatch(pide_ctx* c, int B, double* u, bool accumulate,
                                  cudaStream_t st, int col0) {
  ProfScope ps(c, st, 0);
  if (col0 == 0 && B == 1 && c->sym && c->symv) return launch_symv(c, u, accumulate, st);
  if (col0 == 0 && B <= c->gemv_max_b) return launch_gemv(c, B, u, accumulate, st);
  if (col0 == 0 && (c->prec == PIDE_FP64 || c->prec == PIDE_FP32))
    return launch_gemm_simt(c, B, u, accumulate, st);
  return launch_gemm_tc(c, B, u + (size_t)col0 * c->n, accumulate, st, col0);
}

pide_status launch_apply(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                         int col0) {
  if (B == 0) return PIDE_OK;
  c->tail.pending = false;
  const pide_status s = apply_dispatch(c, B, u, accumulate, st, col0);
  if (s != PIDE_OK) {
    c->tail.pending = false;
    return s;
  }
  return launch_tail_reduce(c, st);   // after the apply's own profile scope
}

// Refinement with the FP64 residual of one column group hidden under the
// tensor-core apply of the other.  Columns split into groups A = [0, Ba) and
// B = [Ba, B).  Main stream: apply(A), apply(B), apply(A), ...; aux stream
// (lower priority): residual(A) after apply(A), residual(B) after apply(B).
// The residual runs on the FP64 pipe and the apply on the tensor pipe, so
// they share the SMs with little interference.  Events fork the aux stream
// from the caller's stream and join it back (graph-capturable).
static pide_status solve_overlapped(pide_ctx* c, const double* b, int mode, const double* lift,
                                    double* x, int B, int sweeps, int rf, cudaStream_t st) {
  const int Ba = ((B / 2 + 127) / 128) * 128;
  const int Bb = B - Ba;
  const int g0[2] = {0, Ba}, gn[2] = {Ba, Bb};
  cudaEvent_t fork = c->ev[0], appl[2] = {c->ev[1], c->ev[2]}, res = c->ev[3];
  PIDE_CUDA_TRY(cudaEventRecord(fork, st));
  PIDE_CUDA_TRY(cudaStreamWaitEvent(c->aux, fork, 0));
  if (rf == RF_E4M3) PIDE_TRY(launch_fp8_scales(c, b, nullptr, B, mode, lift, false, st));
  PIDE_TRY(launch_prep(c, b, B, mode, lift, rf, false, st));
  for (int k = 0; k <= sweeps; ++k) {
    for (int g = 0; g < 2; ++g) {
      if (k > 0) PIDE_CUDA_TRY(cudaStreamWaitEvent(st, c->ev[4 + g], 0));
      PIDE_TRY(launch_apply(c, gn[g], x, k > 0, st, g0[g]));
      if (k == sweeps) continue;
      PIDE_CUDA_TRY(cudaEventRecord(appl[g], st));
      PIDE_CUDA_TRY(cudaStreamWaitEvent(c->aux, appl[g], 0));
      if (rf == RF_E4M3)
        PIDE_TRY(launch_fp8_scales(c, b, x, gn[g], mode, lift, true, c->aux, g0[g]));
      PIDE_TRY(launch_residual_persistent(c, b, x, gn[g], mode, lift, rf, c->aux, g0[g]));
      PIDE_CUDA_TRY(cudaEventRecord(c->ev[4 + g], c->aux));
    }
  }
  PIDE_CUDA_TRY(cudaEventRecord(res, c->aux));
  PIDE_CUDA_TRY(cudaStreamWaitEvent(st, res, 0));
  return PIDE_OK;
}

// L x = f with x = Q(L^-1) q(f), then `sweeps` refinement sweeps
// x += Q(L^-1) q(f - L x), the residual in FP64 (or double-float).  mode 0:
// f = b + lift (Eq. 3); mode 1 (adjoint): f = b / d, so that
// x = L^-1 D^-1 b = S^-1 b.  With an e4m3 correction term, apply k (0: the
// first, k: sweep k) adds C e4m3(q(r)) when bit k of corr_mask is set.  FP16
// right-hand sides take their power-of-two column scales once, from f, in the
// prep; every residual of the solve reuses them.  hist (device, or NULL):
// hist[k] = worst-column relative residual after apply k, recorded from the
// refinement's own residuals (which are then tracked even without a tolerance).
pide_status solve_s(pide_ctx* c, const double* b, int mode, const double* lift, double* x,
                    int B, int sweeps, double tol, cudaStream_t st, double* hist) {
  PIDE_TRY(ensure_workspace(c, B));
  PIDE_CUDA_TRY(cudaMemsetAsync(c->flags, 0, FLAG_COUNT * sizeof(uint32_t), st));
  PIDE_CUDA_TRY(cudaMemsetAsync(c->colmax, 0, 3 * (size_t)c->ws_B * sizeof(double), st));
  const int rf = rhs_format(c, B);
  const bool tensor = B > c->gemv_max_b && (c->prec == PIDE_BF16 || c->prec == PIDE_FP8 ||
                                            c->prec == PIDE_FP8X2 || c->prec == PIDE_FP16);
  // the e4m3 correction term joins the applies that corr_mask selects (tensor path)
  const bool corr = c->corr && tensor && (c->prec == PIDE_BF16 || c->prec == PIDE_FP16);
  auto corr_at = [&](int k) { return corr && k < 31 && ((c->corr_mask >> k) & 1); };
  const bool track = tol > 0 || hist;
  if (c->overlap && tensor && tol <= 0 && sweeps > 0 && B >= 512 && c->aux && !corr &&
      rf != RF_F16 && !hist)
    return solve_overlapped(c, b, mode, lift, x, B, sweeps, rf, st);
  // Low-precision stores take the double-float residual (its ~2^-45 |u|
  // rounding is far below their own error) unless the caller's tolerance
  // asks for a residual below 1e-8 of |f|, which only the FP64 stencil resolves.
  const bool emul = c->resid_emul && mode == 0 &&
                    (c->prec == PIDE_BF16 || c->prec == PIDE_FP8 || c->prec == PIDE_FP8X2 ||
                     c->prec == PIDE_FP16) &&
                    (tol <= 0 || tol >= 1e-8);
  if (rf == RF_E4M3) PIDE_TRY(launch_fp8_scales(c, b, nullptr, B, mode, lift, false, st));
  // FP16: the prep writes the correction term's e4m3 copy of R in the same pass
  const bool fused_corr = rf == RF_F16 && corr_at(0);
  if (rf == RF_F16) PIDE_TRY(launch_prep_f16(c, b, B, mode, lift, track, st, fused_corr));
  else PIDE_TRY(launch_prep(c, b, B, mode, lift, rf, track, st, emul));
  if (corr_at(0) && !fused_corr) PIDE_TRY(launch_corr_rhs(c, B, st));
  PIDE_TRY(launch_apply(c, B, x, false, st));
  if (corr_at(0)) PIDE_TRY(launch_apply_corr(c, B, x, st));
  for (int k = 0; k < sweeps; ++k) {
    if (rf == RF_E4M3 && tol <= 0 && !hist) {
      PIDE_TRY(launch_residual_fp8(c, b, x, B, mode, lift, st, emul));
      PIDE_TRY(launch_apply(c, B, x, true, st));
      continue;
    }
    if (rf == RF_E4M3) PIDE_TRY(launch_fp8_scales(c, b, x, B, mode, lift, true, st));
    PIDE_TRY(launch_residual(c, b, x, B, mode, lift, rf, true, nullptr, track, true, st, 0,
                             emul));
    if (hist && k < HIST_MAX) PIDE_TRY(launch_record(c, B, hist + k, tol <= 0, st));
    if (tol > 0) PIDE_TRY(launch_check(c, B, tol, st));
    if (corr_at(k + 1)) PIDE_TRY(launch_corr_rhs(c, B, st));
    PIDE_TRY(launch_apply(c, B, x, true, st));
    if (corr_at(k + 1)) PIDE_TRY(launch_apply_corr(c, B, x, st));
  }
  return PIDE_OK;
}

static pide_status fill_info(pide_ctx* c, const double* b, const double* x, int B, int mode,
                             const double* lift, int sweeps, double tol, cudaStream_t st,
                             pide_info* info, bool timed = true) {
  // one more residual, tracked, ignoring the early-exit flag
  PIDE_CUDA_TRY(cudaMemsetAsync(c->colmax, 0, (size_t)c->ws_B * sizeof(double), st));
  if (tol <= 0) {
    PIDE_CUDA_TRY(cudaMemsetAsync(c->colmax + c->ws_B, 0, (size_t)c->ws_B * sizeof(double), st));
    PIDE_TRY(launch_colmax_b(c, b, B, mode, lift, st));
  }
  PIDE_TRY(launch_residual(c, b, x, B, mode, lift, RF_F64, false, nullptr, true, false, st));
  std::vector<double> cm(2 * (size_t)c->ws_B);
  uint32_t fl[FLAG_COUNT];
  double r0 = 0.0;
  PIDE_CUDA_TRY(cudaMemcpyAsync(cm.data(), c->colmax, cm.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
  PIDE_CUDA_TRY(cudaMemcpyAsync(fl, c->flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
  PIDE_CUDA_TRY(cudaMemcpyAsync(&r0, c->hist, sizeof(double), cudaMemcpyDeviceToHost, st));
  PIDE_CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.0f;
  if (timed && cudaEventElapsedTime(&ms, c->tev[0], c->tev[1]) != cudaSuccess) ms = 0.0f;
  info->ms = ms;
  double worst = 0.0;
  for (int k = 0; k < B; ++k) {
    const double den = cm[c->ws_B + k];
    const double r = den > 0 ? cm[k] / den : cm[k];
    if (r > worst) worst = r;
  }
  info->rel_residual = worst;
  info->setup_ms = c->setup_ms;
  if (tol > 0) {
    info->converged = worst <= tol ? 1 : 0;
    info->sweeps = (int)fl[FLAG_SWEEPS];
  } else {
    info->converged = 1;
    info->sweeps = sweeps;
  }
  // geometric mean of the per-sweep residual ratios: (r_K / r_0)^(1/K)
  info->contraction = std::nan("");
  if (info->sweeps > 0 && r0 > 0.0)
    info->contraction = std::pow(worst / r0, 1.0 / info->sweeps);
  if (fl[FLAG_ERROR]) {
    set_error("device-side wait timed out (code " + std::to_string(fl[FLAG_ERROR]) + ")");
    return PIDE_ETIMEOUT;
  }
  if (tol > 0 && !info->converged) {
    set_error("tolerance not reached within max_sweeps");
    return PIDE_ENOTCONV;
  }
  return PIDE_OK;
}

static pide_status check_device_error(pide_ctx* c, cudaStream_t st) {
  uint32_t e = 0;
  PIDE_CUDA_TRY(cudaMemcpyAsync(&e, c->flags + FLAG_ERROR, sizeof(e), cudaMemcpyDeviceToHost, st));
  PIDE_CUDA_TRY(cudaStreamSynchronize(st));
  if (e) {
    set_error("device-side wait timed out (code " + std::to_string(e) + ")");
    return PIDE_ETIMEOUT;
  }
  return PIDE_OK;
}

}  // namespace pide

using namespace pide;

// ---------------------------------------------------------------- setup / destroy

static bool valid_grid(const pide_grid* g) {
  return g && g->nx >= 3 && g->ny >= 3 && std::isfinite(g->h) && g->h > 0 &&
         (int64_t)(g->nx - 2) * (g->ny - 2) < (int64_t)1 << 30;
}

static pide_status setup_operator(pide_ctx* c, int nx, int ny, int nz, double h, int dims,
                                  const double* eps_host, cudaStream_t st) {
  c->dims = dims;
  c->nx = nx;
  c->ny = ny;
  c->nz = dims == 3 ? nz : 1;
  c->h = h;
  c->mx = nx - 2;
  c->my = ny - 2;
  c->mz = dims == 3 ? nz - 2 : 1;
  c->n = c->mx * c->my * c->mz;
  c->ld = ((c->n + 63) / 64) * 64;
  const size_t N = (size_t)nx * ny * c->nz;
  const int faces = dims == 3 ? 6 : 4;
  c->eps_host.assign(N, 1.0);
  if (eps_host) {
    for (size_t k = 0; k < N; ++k) {
      if (!std::isfinite(eps_host[k]) || !(eps_host[k] > 0.0)) {
        set_error("eps must be finite and > 0 at every node");
        return PIDE_EINVAL;
      }
      c->eps_host[k] = eps_host[k];
    }
  }
  PIDE_CUDA_TRY(cudaGetDevice(&c->device));
  cudaDeviceProp prop;
  PIDE_CUDA_TRY(cudaGetDeviceProperties(&prop, c->device));
  if (prop.major != 10 || prop.minor != 3) {
    set_error("this library is built for sm_103a (GB300); device is sm_" +
              std::to_string(prop.major) + std::to_string(prop.minor));
    return PIDE_EUNSUPPORTED;
  }
  c->num_sms = prop.multiProcessorCount;
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->eps, N * sizeof(double)));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->cf, faces * (size_t)c->n * sizeof(double)));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->d, (size_t)c->n * sizeof(double)));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->dinv, (size_t)c->n * sizeof(double)));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->w, faces * (size_t)c->n * sizeof(double)));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->lift, (size_t)c->n * sizeof(double)));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->flags, FLAG_COUNT * sizeof(uint32_t)));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->hist, HIST_MAX * sizeof(double)));
  PIDE_CUDA_TRY(cudaMemset(c->hist, 0, HIST_MAX * sizeof(double)));
  for (int k = 0; k < 2; ++k) PIDE_CUDA_TRY(cudaEventCreate(&c->tev[k]));

  PIDE_CUDA_TRY(cudaMemset(c->flags, 0, FLAG_COUNT * sizeof(uint32_t)));
  int prio_lo = 0, prio_hi = 0;
  PIDE_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  PIDE_CUDA_TRY(cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, prio_lo));
  for (int k = 0; k < 6; ++k) PIDE_CUDA_TRY(cudaEventCreateWithFlags(&c->ev[k], cudaEventDisableTiming));
  PIDE_CUDA_TRY(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
  for (int k = 0; k < 6; ++k) PIDE_CUDA_TRY(cudaEventCreateWithFlags(&c->hev[k], cudaEventDisableTiming));
  PIDE_CUDA_TRY(cudaStreamCreateWithFlags(&c->dstream, cudaStreamNonBlocking));
  for (int k = 0; k < 9; ++k) PIDE_CUDA_TRY(cudaEventCreateWithFlags(&c->sev[k], cudaEventDisableTiming));
  PIDE_CUDA_TRY(cudaMemcpyAsync(c->eps, c->eps_host.data(), N * sizeof(double),
                                cudaMemcpyHostToDevice, st));
  PIDE_TRY(launch_assemble(c, st));
  PIDE_CUDA_TRY(cudaMalloc((void**)&c->wsp, (dims == 3 ? 3 : 2) * (size_t)c->n * sizeof(float4)));
  PIDE_TRY(launch_wsplit(c, st));
  return PIDE_OK;
}

// Arguments of the measured format choice (pide_setup_auto / PIDE_AUTO).
struct AutoArgs {
  double target = 0.5e-6;
  const double* probe_host = nullptr;
  int nprobe = 16;
  int max_sweeps = 8;
};

// Steps 1-2 for a 2-D (dims 2) or 3-D (dims 3) grid: assemble, invert in FP64,
// quantise (PIDE_AUTO: the store the measurement chooses); the handle is
// returned only when every step succeeded.
static pide_status setup_handle(int nx, int ny, int nz, double h, int dims, const double* eps_host,
                                pide_precision p, void* stream, pide_handle* out,
                                const AutoArgs& aa = AutoArgs()) {
  if (eps_host) {
    const size_t N = (size_t)nx * ny * (dims == 3 ? nz : 1);
    for (size_t k = 0; k < N; ++k)
      if (!std::isfinite(eps_host[k]) || !(eps_host[k] > 0.0)) {
        set_error("eps must be finite and > 0 at every node");
        return PIDE_EINVAL;
      }
  }
  // host-side fault injection for tests: pretend the device allocation failed
  if (const char* f = std::getenv("PIDE_FAULT_ALLOC")) {
    if (f[0] == '1') {
      set_error("PIDE_FAULT_ALLOC=1: injected allocation failure");
      return PIDE_ENOMEM;
    }
  }
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  pide_ctx* c = new pide_ctx();
  // the BF16 / FP16 store plus its e4m3 correction term
  const bool want_corr = p == PIDE_BF16_FP8 || p == PIDE_FP16_FP8;
  const bool want_auto = p == PIDE_AUTO;
  if (want_auto) p = PIDE_FP64;                 // until the measurement has chosen
  if (p == PIDE_BF16_FP8) p = PIDE_BF16;
  if (p == PIDE_FP16_FP8) {
    p = PIDE_FP16;
    c->corr_mask = 1;                             // FP16: correct the first apply
  }
  c->prec = p;
  pide_status s = setup_operator(c, nx, ny, nz, h, dims, eps_host, st);
  double* G = nullptr;
  if (s == PIDE_OK) {
    const size_t bytes = (size_t)c->n * c->ld * sizeof(double);
    cudaError_t e = cudaMalloc((void**)&G, bytes);
    if (e != cudaSuccess) {
      set_error(std::string("allocating the FP64 inverse: ") + cudaGetErrorString(e));
      s = e == cudaErrorMemoryAllocation ? PIDE_ENOMEM : PIDE_ECUDA;
    } else if ((e = cudaMemsetAsync(G, 0, bytes, st)) != cudaSuccess) {
      set_error(cudaGetErrorString(e));
      s = PIDE_ECUDA;
    }
  }
  if (s == PIDE_OK) s = build_inverse_fp64(c, G, st);
  if (s == PIDE_OK && want_auto) {
    // leaves the chosen store quantised in the handle
    s = auto_select(c, G, aa.target, aa.probe_host, aa.nprobe, aa.max_sweeps, st);
    p = c->prec;
  }
  if (s == PIDE_OK) {
    if (p == PIDE_FP64) {
      c->inv = G;
      c->store_bytes = (size_t)c->n * c->ld * sizeof(double);
      G = nullptr;
    } else {
      if (!want_auto) s = quantize_store(c, G, st);
      if (s == PIDE_OK && want_corr) s = quantize_corr(c, G, st);
      // B = 1 of both 16-bit stores: the symmetric two-term BF16 form of S^-1
      if (s == PIDE_OK && (p == PIDE_BF16 || p == PIDE_FP16)) s = build_sym_store(c, G, st);
    }
  }
  if (s == PIDE_OK) s = make_tma_maps(c);
  if (s == PIDE_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("setup kernels: ") + cudaGetErrorString(e));
      s = PIDE_ECUDA;
    }
  }
  if (G) cudaFree(G);
  if (s != PIDE_OK) {
    pide_destroy(c);
    return s;
  }
  c->setup_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = c;
  return PIDE_OK;
}

extern "C" pide_status pide_setup(const pide_grid* g, const double* eps_host, pide_precision p,
                                  void* stream, pide_handle* out) {
  if (out) *out = nullptr;
  if (!out || !valid_grid(g) || (int)p < 0 || (int)p > 8) {
    set_error("pide_setup: bad argument");
    return PIDE_EINVAL;
  }
  return setup_handle(g->nx, g->ny, 1, g->h, 2, eps_host, p, stream, out);
}

extern "C" pide_status pide_setup_auto(const pide_grid* g, const double* eps_host, double target,
                                       const double* probe_host, int32_t nprobe,
                                       int32_t max_sweeps, void* stream, pide_handle* out) {
  if (out) *out = nullptr;
  if (!out || !valid_grid(g) || !(target > 0.0 && target <= 0.1) || nprobe < 1 || nprobe > 256 ||
      max_sweeps < 0 || max_sweeps > 30) {
    set_error("pide_setup_auto: bad argument (grid, target in (0, 0.1], nprobe in [1, 256], "
              "max_sweeps in [0, 30])");
    return PIDE_EINVAL;
  }
  AutoArgs aa;
  aa.target = target;
  aa.probe_host = probe_host;
  aa.nprobe = nprobe;
  aa.max_sweeps = max_sweeps;
  return setup_handle(g->nx, g->ny, 1, g->h, 2, eps_host, PIDE_AUTO, stream, out, aa);
}

extern "C" pide_status pide_get_auto_report(pide_handle h, pide_auto_report* out) {
  if (!h || !out || !h->has_auto) {
    set_error("pide_get_auto_report: bad argument (handle from pide_setup_auto, out)");
    return PIDE_EINVAL;
  }
  *out = h->auto_rep;
  return PIDE_OK;
}

extern "C" pide_status pide_setup_3d(const pide_grid3* g, const double* eps_host,
                                     pide_precision p, void* stream, pide_handle* out) {
  if (out) *out = nullptr;
  const bool ok = g && g->nx >= 3 && g->ny >= 3 && g->nz >= 3 && std::isfinite(g->h) && g->h > 0 &&
                  (int64_t)(g->nx - 2) * (g->ny - 2) * (g->nz - 2) < (int64_t)1 << 30;
  if (!out || !ok || (int)p < 0 || (int)p > 8) {
    set_error("pide_setup_3d: bad argument");
    return PIDE_EINVAL;
  }
  return setup_handle(g->nx, g->ny, g->nz, g->h, 3, eps_host, p, stream, out);
}

extern "C" void pide_destroy(pide_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  void* ptrs[] = {h->sym, h->sym_lo, h->sym_scale, h->dfl, h->ysum, h->Rf, h->eps, h->cf, h->d, h->dinv, h->w, h->wsp, h->inv, h->inv_lo, h->row_scale, h->R, h->col_scale,
                  h->corr, h->corr_scale, h->Rc, h->col_scale_c,
                  h->lift, h->colmax, h->flags, h->hist, h->hbuf_b, h->hbuf_u, h->sbuf_in, h->sbuf_out,
                  h->tail_ws};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& ev : h->prof_events) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->hev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->sev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->tev)
    if (e) cudaEventDestroy(e);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  if (h->dstream) cudaStreamDestroy(h->dstream);
  delete h;
}

// ---------------------------------------------------------------- apply entry points

static pide_status check_apply_args(pide_handle h, const void* b, const void* u, int32_t B,
                                    int32_t sweeps) {
  if (!h || B < 0 || sweeps < 0 || (B > 0 && (!b || !u)) || (B > 0 && b == u) || B > 65535) {
    set_error("bad argument (handle, pointers, B in [0, 65535], sweeps >= 0, b != u)");
    return PIDE_EINVAL;
  }
  return PIDE_OK;
}

// PIDE_SWEEPS_AUTO -> the sweep count pide_setup_auto measured for the handle.
static pide_status resolve_sweeps(pide_handle h, int32_t* sweeps) {
  if (h && *sweeps == PIDE_SWEEPS_AUTO) {
    if (h->sweeps_hint < 0) {
      set_error("PIDE_SWEEPS_AUTO needs a handle from pide_setup_auto");
      return PIDE_EINVAL;
    }
    *sweeps = h->sweeps_hint;
  }
  return PIDE_OK;
}

extern "C" pide_status pide_apply(pide_handle h, const double* b_dev, double* u_dev, int32_t B,
                                  int32_t max_sweeps, double tol, const double* g_dev,
                                  void* stream, pide_info* info) {
  PIDE_TRY(resolve_sweeps(h, &max_sweeps));
  PIDE_TRY(check_apply_args(h, b_dev, u_dev, B, max_sweeps));
  if (B == 0) {
    if (info) *info = pide_info{0, 1, 0.0, h->setup_ms, std::nan(""), 0.0};
    return PIDE_OK;
  }
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (info) PIDE_CUDA_TRY(cudaEventRecord(h->tev[0], st));
  const double* lift = nullptr;
  if (g_dev) {
    PIDE_TRY(launch_lift(h, g_dev, st));
    lift = h->lift;
  }
  PIDE_TRY(solve_s(h, b_dev, 0, lift, u_dev, B, max_sweeps, tol, st, info ? h->hist : nullptr));
  if (info) {
    PIDE_CUDA_TRY(cudaEventRecord(h->tev[1], st));
    return fill_info(h, b_dev, u_dev, B, 0, lift, max_sweeps, tol, st, info);
  }
  return PIDE_OK;
}

extern "C" pide_status pide_apply_host(pide_handle h, const double* b_host, double* u_host,
                                       int32_t B, int32_t max_sweeps, double tol, void* stream,
                                       pide_info* info) {
  PIDE_TRY(resolve_sweeps(h, &max_sweeps));
  PIDE_TRY(check_apply_args(h, b_host, u_host, B, max_sweeps));
  if (B == 0) return PIDE_OK;
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (B > h->hbuf_B) {
    if (h->hbuf_b) cudaFree(h->hbuf_b);
    if (h->hbuf_u) cudaFree(h->hbuf_u);
    h->hbuf_b = h->hbuf_u = nullptr;
    h->hbuf_B = 0;
    PIDE_CUDA_TRY(cudaMalloc((void**)&h->hbuf_b, (size_t)B * h->n * sizeof(double)));
    PIDE_CUDA_TRY(cudaMalloc((void**)&h->hbuf_u, (size_t)B * h->n * sizeof(double)));
    h->hbuf_B = B;
  }
  const size_t bytes = (size_t)B * h->n * sizeof(double);
  if (B >= 512 && tol <= 0 && !info && h->cstream) {
    // Two column chunks: the copy stream moves chunk 1 in while chunk 0 is
    // solved, and chunk 0 out while chunk 1 is solved.
    const int B0 = ((B / 2 + 127) / 128) * 128;
    const int c0[2] = {0, B0}, cn[2] = {B0, B - B0};
    cudaEvent_t fork = h->hev[0], in[2] = {h->hev[1], h->hev[2]}, done[2] = {h->hev[3], h->hev[4]},
                out = h->hev[5];
    PIDE_CUDA_TRY(cudaEventRecord(fork, st));
    PIDE_CUDA_TRY(cudaStreamWaitEvent(h->cstream, fork, 0));
    for (int q = 0; q < 2; ++q) {
      const size_t off = (size_t)c0[q] * h->n;
      PIDE_CUDA_TRY(cudaMemcpyAsync(h->hbuf_b + off, b_host + off, (size_t)cn[q] * h->n * sizeof(double),
                                    cudaMemcpyHostToDevice, h->cstream));
      PIDE_CUDA_TRY(cudaEventRecord(in[q], h->cstream));
    }
    for (int q = 0; q < 2; ++q) {
      const size_t off = (size_t)c0[q] * h->n;
      PIDE_CUDA_TRY(cudaStreamWaitEvent(st, in[q], 0));
      PIDE_TRY(solve_s(h, h->hbuf_b + off, 0, nullptr, h->hbuf_u + off, cn[q], max_sweeps, tol, st));
      PIDE_CUDA_TRY(cudaEventRecord(done[q], st));
      PIDE_CUDA_TRY(cudaStreamWaitEvent(h->cstream, done[q], 0));
      PIDE_CUDA_TRY(cudaMemcpyAsync(u_host + off, h->hbuf_u + off, (size_t)cn[q] * h->n * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->cstream));
    }
    PIDE_CUDA_TRY(cudaEventRecord(out, h->cstream));
    PIDE_CUDA_TRY(cudaStreamWaitEvent(st, out, 0));
    return check_device_error(h, st);
  }
  if (info) PIDE_CUDA_TRY(cudaEventRecord(h->tev[0], st));
  PIDE_CUDA_TRY(cudaMemcpyAsync(h->hbuf_b, b_host, bytes, cudaMemcpyHostToDevice, st));
  PIDE_TRY(solve_s(h, h->hbuf_b, 0, nullptr, h->hbuf_u, B, max_sweeps, tol, st,
                   info ? h->hist : nullptr));
  PIDE_CUDA_TRY(cudaMemcpyAsync(u_host, h->hbuf_u, bytes, cudaMemcpyDeviceToHost, st));
  if (info) {
    PIDE_CUDA_TRY(cudaEventRecord(h->tev[1], st));
    return fill_info(h, h->hbuf_b, h->hbuf_u, B, 0, nullptr, max_sweeps, tol, st, info);
  }
  return check_device_error(h, st);
}

// Eq. (1) with time: a sequence of right-hand sides (or charge densities) in
// host memory solved chunk by chunk.  Slot q = i & 1 of the two device slots
// holds chunk i; its input copy (cstream) waits until chunk i - 2 has been
// solved, its solve (st) waits for that copy and for the output copy of
// chunk i - 2 (dstream), and its output copy waits for the solve, so chunk
// i's solve runs under chunk i + 1's input copy and chunk i - 1's output copy.
extern "C" pide_status pide_solve_stream(pide_handle h, const double* in_host, double* u_host,
                                         int64_t T, int32_t chunk, int32_t sweeps,
                                         int32_t charge, void* stream) {
  PIDE_TRY(resolve_sweeps(h, &sweeps));
  if (!h || T < 0 || chunk < 1 || chunk > 65535 || sweeps < 0 || (T > 0 && (!in_host || !u_host)) ||
      (const void*)in_host == (const void*)u_host) {
    set_error("pide_solve_stream: bad argument (handle, pointers, T >= 0, chunk in [1, 65535], "
              "sweeps >= 0, in != u)");
    return PIDE_EINVAL;
  }
  if (T == 0) return PIDE_OK;
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int cols = (int)(T < chunk ? T : chunk);
  if (cols > h->sbuf_cols) {
    if (h->sbuf_in) cudaFree(h->sbuf_in);
    if (h->sbuf_out) cudaFree(h->sbuf_out);
    h->sbuf_in = h->sbuf_out = nullptr;
    h->sbuf_cols = 0;
    PIDE_CUDA_TRY(cudaMalloc((void**)&h->sbuf_in, 2 * (size_t)cols * h->n * sizeof(double)));
    PIDE_CUDA_TRY(cudaMalloc((void**)&h->sbuf_out, 2 * (size_t)cols * h->n * sizeof(double)));
    h->sbuf_cols = cols;
  }
  PIDE_TRY(ensure_workspace(h, cols));
  const size_t slot = (size_t)cols * h->n;
  cudaEvent_t fork = h->sev[0], copied_in[2] = {h->sev[1], h->sev[2]},
              solved[2] = {h->sev[3], h->sev[4]}, copied_out[2] = {h->sev[5], h->sev[6]},
              end_in = h->sev[7], end_out = h->sev[8];
  // the copy streams start after the work already queued on st
  PIDE_CUDA_TRY(cudaEventRecord(fork, st));
  PIDE_CUDA_TRY(cudaStreamWaitEvent(h->cstream, fork, 0));
  PIDE_CUDA_TRY(cudaStreamWaitEvent(h->dstream, fork, 0));
  // Chunk schedule: a half chunk first and last, so that only a smaller copy
  // is exposed at each end (the first input copy precedes every solve, the last
  // output copy follows them); full chunks between.
  std::vector<std::pair<int64_t, int>> chunks;
  if (T <= cols) {
    chunks.emplace_back(0, (int)T);
  } else {
    const int r = cols / 2 > 0 ? cols / 2 : 1;
    chunks.emplace_back(0, r);
    int64_t c0 = r, rest = T - r;
    while (rest > (int64_t)cols + r) {
      chunks.emplace_back(c0, cols);
      c0 += cols;
      rest -= cols;
    }
    if (rest > r) {
      chunks.emplace_back(c0, (int)(rest - r));
      chunks.emplace_back(c0 + rest - r, r);
    } else {
      chunks.emplace_back(c0, (int)rest);
    }
  }
  const int64_t nchunks = (int64_t)chunks.size();
  for (int64_t i = 0; i < nchunks; ++i) {
    const int q = (int)(i & 1);
    const int64_t c0 = chunks[i].first;
    const int nc = chunks[i].second;
    const size_t off = (size_t)c0 * h->n, bytes = (size_t)nc * h->n * sizeof(double);
    double* din = h->sbuf_in + q * slot;
    double* dout = h->sbuf_out + q * slot;
    if (i >= 2) PIDE_CUDA_TRY(cudaStreamWaitEvent(h->cstream, solved[q], 0));
    PIDE_CUDA_TRY(cudaMemcpyAsync(din, in_host + off, bytes, cudaMemcpyHostToDevice, h->cstream));
    PIDE_CUDA_TRY(cudaEventRecord(copied_in[q], h->cstream));
    PIDE_CUDA_TRY(cudaStreamWaitEvent(st, copied_in[q], 0));
    if (i >= 2) PIDE_CUDA_TRY(cudaStreamWaitEvent(st, copied_out[q], 0));
    if (charge) PIDE_TRY(launch_rhs_from_charge(h, din, din, nc, st));
    PIDE_TRY(solve_s(h, din, 0, nullptr, dout, nc, sweeps, 0.0, st));
    PIDE_CUDA_TRY(cudaEventRecord(solved[q], st));
    PIDE_CUDA_TRY(cudaStreamWaitEvent(h->dstream, solved[q], 0));
    PIDE_CUDA_TRY(cudaMemcpyAsync(u_host + off, dout, bytes, cudaMemcpyDeviceToHost, h->dstream));
    PIDE_CUDA_TRY(cudaEventRecord(copied_out[q], h->dstream));
  }
  PIDE_CUDA_TRY(cudaEventRecord(end_in, h->cstream));
  PIDE_CUDA_TRY(cudaEventRecord(end_out, h->dstream));
  PIDE_CUDA_TRY(cudaStreamWaitEvent(st, end_in, 0));
  PIDE_CUDA_TRY(cudaStreamWaitEvent(st, end_out, 0));
  return check_device_error(h, st);
}

extern "C" pide_status pide_residual(pide_handle h, const double* b_dev, const double* u_dev,
                                     double* r_dev, int32_t B, void* stream) {
  if (!h || B < 0 || (B > 0 && (!b_dev || !u_dev || !r_dev)) || r_dev == b_dev || r_dev == u_dev) {
    set_error("pide_residual: bad argument");
    return PIDE_EINVAL;
  }
  if (B == 0) return PIDE_OK;
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  PIDE_TRY(ensure_workspace(h, B));
  return launch_residual(h, b_dev, u_dev, B, 0, nullptr, RF_F64, false, r_dev, false, false,
                         (cudaStream_t)stream);
}

extern "C" pide_status pide_rhs_from_charge(pide_handle h, const double* rho_dev, double* b_dev,
                                            int32_t B, void* stream) {
  if (!h || B < 0 || (B > 0 && (!rho_dev || !b_dev))) {
    set_error("pide_rhs_from_charge: bad argument");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  return launch_rhs_from_charge(h, rho_dev, b_dev, B, (cudaStream_t)stream);
}

extern "C" pide_status pide_apply_backward(pide_handle h, const double* gout_dev,
                                           const double* u_dev, const double* b_dev,
                                           double* db_dev, double* deps_dev, int32_t B,
                                           int32_t max_sweeps, void* stream) {
  PIDE_TRY(check_apply_args(h, gout_dev, u_dev, B, max_sweeps));
  if (B > 0 && (!b_dev)) {
    set_error("pide_apply_backward: b_dev is required");
    return PIDE_EINVAL;
  }
  if (B == 0) return PIDE_OK;
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  cudaStream_t st = (cudaStream_t)stream;
  double* mu = nullptr;
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&mu, (size_t)B * h->n * sizeof(double), st));
  pide_status s = solve_s(h, gout_dev, 1, nullptr, mu, B, max_sweeps, 0.0, st);
  if (s == PIDE_OK && db_dev) s = launch_scale_d(h, mu, db_dev, B, st);
  if (s == PIDE_OK && deps_dev) s = launch_face_grad(h, mu, u_dev, b_dev, B, deps_dev, st);
  cudaFreeAsync(mu, st);
  if (s != PIDE_OK) return s;
  return PIDE_OK;
}

extern "C" pide_status pide_reserve(pide_handle h, int32_t Bmax) {
  if (!h || Bmax < 0) {
    set_error("pide_reserve: bad argument");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  return ensure_workspace(h, Bmax);
}

// ---------------------------------------------------------------- batched

extern "C" pide_status pide_apply_batched_impl(const pide_handle* hs, int32_t nprob,
                                               const double* const* b, double* const* u,
                                               const int32_t* Bs, int32_t sweeps, void* stream);

extern "C" pide_status pide_apply_batched(const pide_handle* hs, int32_t nprob,
                                          const double* const* b, double* const* u,
                                          const int32_t* Bs, int32_t sweeps, void* stream) {
  if (nprob < 0 || (nprob > 0 && (!hs || !b || !u || !Bs)) || sweeps < 0) {
    set_error("pide_apply_batched: bad argument");
    return PIDE_EINVAL;
  }
  for (int k = 0; k < nprob; ++k) PIDE_TRY(check_apply_args(hs[k], b[k], u[k], Bs[k], sweeps));
  return pide_apply_batched_impl(hs, nprob, b, u, Bs, sweeps, stream);
}

// ---------------------------------------------------------------- persistence

namespace {
struct FileHeader {
  char magic[8];
  int32_t version, nx, ny, prec, n, ld;
  double h;
  uint64_t eps_hash;
  uint64_t store_bytes;
};

// Version 2 (3-D grids) follows the header with this block.
struct FileHeader3 {
  int32_t nz, dims;
};

uint64_t fnv1a(const void* data, size_t len) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t hsh = 1469598103934665603ull;
  for (size_t k = 0; k < len; ++k) {
    hsh ^= p[k];
    hsh *= 1099511628211ull;
  }
  return hsh;
}
}  // namespace

extern "C" pide_status pide_save(pide_handle h, const char* path) {
  if (!h || !path) {
    set_error("pide_save: bad argument");
    return PIDE_EINVAL;
  }
  PIDE_CUDA_TRY(cudaSetDevice(h->device));
  PIDE_CUDA_TRY(cudaDeviceSynchronize());
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error(std::string("cannot open ") + path);
    return PIDE_EINVAL;
  }
  const size_t main_bytes = (size_t)h->n * h->ld *
                            (h->prec == PIDE_FP64 ? 8 : h->prec == PIDE_FP32 ? 4 :
                             (h->prec == PIDE_BF16 || h->prec == PIDE_FP16) ? 2 : 1);
  FileHeader hd{};
  std::memcpy(hd.magic, "PIDEINV1", 8);
  hd.version = h->dims == 3 ? 2 : 1;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.prec = !h->corr ? (int)h->prec : h->prec == PIDE_FP16 ? (int)PIDE_FP16_FP8 : (int)PIDE_BF16_FP8;
  hd.n = h->n;
  hd.ld = h->ld;
  hd.h = h->h;
  hd.eps_hash = fnv1a(h->eps_host.data(), h->eps_host.size() * sizeof(double));
  hd.store_bytes = main_bytes;
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  if (hd.version == 2) {
    const FileHeader3 h3{h->nz, h->dims};
    ok = ok && std::fwrite(&h3, sizeof(h3), 1, f) == 1;
  }
  ok = ok && std::fwrite(h->eps_host.data(), sizeof(double), h->eps_host.size(), f) == h->eps_host.size();
  std::vector<char> buf(1 << 26);
  auto dump = [&](const void* dev, size_t bytes) {
    for (size_t off = 0; ok && off < bytes; off += buf.size()) {
      const size_t len = std::min(buf.size(), bytes - off);
      ok = cudaMemcpy(buf.data(), (const char*)dev + off, len, cudaMemcpyDeviceToHost) == cudaSuccess;
      ok = ok && std::fwrite(buf.data(), 1, len, f) == len;
    }
  };
  dump(h->inv, main_bytes);
  if (h->inv_lo) dump(h->inv_lo, main_bytes);
  if (h->row_scale) dump(h->row_scale, (size_t)h->n * sizeof(float));
  if (h->corr) {
    dump(h->corr, (size_t)h->n * h->ld);
    dump(h->corr_scale, (size_t)h->n * sizeof(float));
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    set_error(std::string("writing ") + path + " failed");
    return PIDE_ECUDA;
  }
  return PIDE_OK;
}

extern "C" pide_status pide_load(const char* path, void* stream, pide_handle* out) {
  if (!path || !out) {
    set_error("pide_load: bad argument");
    return PIDE_EINVAL;
  }
  *out = nullptr;
  auto t0 = std::chrono::steady_clock::now();
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("cannot open ") + path);
    return PIDE_EINVAL;
  }
  FileHeader hd{};
  bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, "PIDEINV1", 8) == 0 &&
            (hd.version == 1 || hd.version == 2);
  FileHeader3 h3{1, 2};
  if (ok && hd.version == 2) ok = std::fread(&h3, sizeof(h3), 1, f) == 1 && h3.dims == 3;
  pide_grid g{hd.nx, hd.ny, hd.h};
  if (!ok || !valid_grid(&g) || hd.prec < 0 || hd.prec > 7 || h3.nz < 1 ||
      (h3.dims == 3 && (h3.nz < 3 || (int64_t)(hd.nx - 2) * (hd.ny - 2) * (h3.nz - 2) >= (int64_t)1 << 30))) {
    std::fclose(f);
    set_error(std::string(path) + ": not a pide inverse file");
    return PIDE_EINVAL;
  }
  std::vector<double> eps((size_t)hd.nx * hd.ny * (h3.dims == 3 ? h3.nz : 1));
  ok = std::fread(eps.data(), sizeof(double), eps.size(), f) == eps.size();
  if (!ok || fnv1a(eps.data(), eps.size() * sizeof(double)) != hd.eps_hash) {
    std::fclose(f);
    set_error(std::string(path) + ": eps block corrupt (hash mismatch)");
    return PIDE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  pide_ctx* c = new pide_ctx();
  const bool has_corr = hd.prec == PIDE_BF16_FP8 || hd.prec == PIDE_FP16_FP8;
  c->prec = hd.prec == PIDE_BF16_FP8 ? PIDE_BF16 : hd.prec == PIDE_FP16_FP8 ? PIDE_FP16
                                                 : (pide_precision)hd.prec;
  if (hd.prec == PIDE_FP16_FP8) c->corr_mask = 1;
  pide_status s = setup_operator(c, g.nx, g.ny, h3.nz, g.h, h3.dims, eps.data(), st);
  if (s == PIDE_OK && (c->n != hd.n || c->ld != hd.ld)) {
    set_error("pide_load: header sizes do not match the grid");
    s = PIDE_EINVAL;
  }
  std::vector<char> buf(1 << 26);
  auto load = [&](void** dev, size_t bytes) -> pide_status {
    cudaError_t e = cudaMalloc(dev, bytes);
    if (e != cudaSuccess) {
      set_error(cudaGetErrorString(e));
      return PIDE_ENOMEM;
    }
    for (size_t off = 0; off < bytes; off += buf.size()) {
      const size_t len = std::min(buf.size(), bytes - off);
      if (std::fread(buf.data(), 1, len, f) != len) {
        set_error("pide_load: file truncated");
        return PIDE_EINVAL;
      }
      if (cudaMemcpy((char*)*dev + off, buf.data(), len, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("pide_load: upload failed");
        return PIDE_ECUDA;
      }
    }
    return PIDE_OK;
  };
  if (s == PIDE_OK) s = load(&c->inv, hd.store_bytes);
  if (s == PIDE_OK && c->prec == PIDE_FP8X2) s = load(&c->inv_lo, hd.store_bytes);
  if (s == PIDE_OK && (c->prec == PIDE_FP8 || c->prec == PIDE_FP8X2 || c->prec == PIDE_FP16))
    s = load((void**)&c->row_scale, (size_t)c->n * sizeof(float));
  if (s == PIDE_OK && has_corr) s = load(&c->corr, (size_t)c->n * c->ld);
  if (s == PIDE_OK && has_corr) s = load((void**)&c->corr_scale, (size_t)c->n * sizeof(float));
  std::fclose(f);
  if (s == PIDE_OK) {
    c->store_bytes = hd.store_bytes * (c->prec == PIDE_FP8X2 ? 2 : 1) +
                     (c->prec == PIDE_FP16 ? c->n * sizeof(float) : 0) +
                     (has_corr ? (size_t)c->n * c->ld + c->n * sizeof(float) : 0);
    s = make_tma_maps(c);
  }
  if (s == PIDE_OK && cudaStreamSynchronize(st) != cudaSuccess) s = PIDE_ECUDA;
  if (s != PIDE_OK) {
    pide_destroy(c);
    return s;
  }
  c->setup_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = c;
  return PIDE_OK;
}

// ---------------------------------------------------------------- queries, profiling

extern "C" pide_status pide_get_handle_info(pide_handle h, pide_handle_info* out) {
  if (!h || !out) {
    set_error("pide_get_handle_info: bad argument");
    return PIDE_EINVAL;
  }
  out->n = h->n;
  out->ld = h->ld;
  out->precision = !h->corr ? (int32_t)h->prec
                  : h->prec == PIDE_FP16 ? (int32_t)PIDE_FP16_FP8 : (int32_t)PIDE_BF16_FP8;
  out->num_sms = h->num_sms;
  out->store_bytes = h->store_bytes;
  out->setup_ms = h->setup_ms;
  out->dims = h->dims;
  out->sweeps_hint = h->sweeps_hint;
  return PIDE_OK;
}

extern "C" pide_status pide_profile_begin(pide_handle h) {
  if (!h) {
    set_error("pide_profile_begin: bad argument");
    return PIDE_EINVAL;
  }
  h->prof_on = true;
  return PIDE_OK;
}

extern "C" pide_status pide_profile_end(pide_handle h, pide_profile* out) {
  if (!h || !out) {
    set_error("pide_profile_end: bad argument");
    return PIDE_EINVAL;
  }
  h->prof_on = false;
  std::memset(out, 0, sizeof(*out));
  pide_status s = PIDE_OK;
  for (auto& ev : h->prof_events) {
    if (cudaEventSynchronize(ev.b) != cudaSuccess) s = PIDE_ECUDA;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) {
      out->ms[ev.cls] += ms;
      out->launches[ev.cls] += 1;
    }
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  h->prof_events.clear();
  return s;
}

extern "C" pide_status pide_set_tuning(pide_handle h, int32_t key, int32_t value) {
  if (!h) {
    set_error("pide_set_tuning: NULL handle");
    return PIDE_EINVAL;
  }
  switch (key) {
    case PIDE_TUNE_GEMV_THREADS:
      if (value < 128 || value > 1024 || value % 32) break;
      h->gemv_threads = value;
      return PIDE_OK;
    case PIDE_TUNE_GEMV_UNROLL:
      if (value != 4 && value != 8) break;
      h->gemv_unroll = value;
      return PIDE_OK;
    case PIDE_TUNE_GEMV_MAX_B:
      if (value < 1 || value > 8) break;
      h->gemv_max_b = value;
      return PIDE_OK;
    case PIDE_TUNE_GEMM_BN:
      if (value != 128 && value != 256) break;
      h->gemm_bn_large = value;
      return PIDE_OK;
    case PIDE_TUNE_GEMM_STREAMK:
      if (value < 0 || value > 2) break;
      h->gemm_streamk = value;
      return PIDE_OK;
    case PIDE_TUNE_OVERLAP:
      if (value != 0 && value != 1) break;
      h->overlap = value;
      return PIDE_OK;
    case PIDE_TUNE_RESID_CTAS:
      if (value < 1 || value > 8) break;
      h->resid_ctas_per_sm = value;
      return PIDE_OK;
    case PIDE_TUNE_SYMV:
      if (value != 0 && value != 1) break;
      h->symv = value;
      return PIDE_OK;
    case PIDE_TUNE_RESID_EMUL:
      if (value != 0 && value != 1) break;
      h->resid_emul = value;
      return PIDE_OK;
    case PIDE_TUNE_RESID_SHAPE:
      if (value < -1 || value > 3) break;
      h->resid_shape = value;
      return PIDE_OK;
    case PIDE_TUNE_GEMM_2CTA:
      if (value != 0 && value != 1) break;
      h->gemm_2cta = value;
      return PIDE_OK;
    case PIDE_TUNE_GEMM_A_HINT:
      if (value < 0 || value > 2) break;
      h->gemm_a_hint = value;
      return PIDE_OK;
    case PIDE_TUNE_RESID_PREFETCH:
      if (value < 0 || value > 4096) break;
      h->resid_prefetch = value;
      return PIDE_OK;
    case PIDE_TUNE_CORR_MASK:
      if (value < 0 || value >= (1 << 30)) break;
      h->corr_mask = value;
      return PIDE_OK;
    case PIDE_TUNE_GEMM_U_HINT:
      if (value < 0 || value > 1) break;
      h->gemm_u_hint = value;
      return PIDE_OK;
    case PIDE_TUNE_BATCH_TC:
      if (value != 0 && value != 1) break;
      h->batch_tc = value;
      return PIDE_OK;
    case PIDE_TUNE_BATCH_BN:
      if (value != 0 && value != 32 && value != 64 && value != 128) break;
      h->batch_bn = value;
      return PIDE_OK;
    case PIDE_TUNE_BATCH_TN:
      if (value != 0 && value != 16 && value != 32 && value != 64) break;
      h->batch_tn = value;
      return PIDE_OK;
    case PIDE_TUNE_PREP_CLUSTER:
      if (value != 0 && value != 1) break;
      h->prep_cluster = value;
      return PIDE_OK;
  }
  set_error("pide_set_tuning: unknown key or value out of range");
  return PIDE_EINVAL;
}

extern "C" pide_status pide_get_tuning(pide_handle h, int32_t key, int32_t* value) {
  if (!h || !value) {
    set_error("pide_get_tuning: bad argument");
    return PIDE_EINVAL;
  }
  switch (key) {
    case PIDE_TUNE_GEMV_THREADS: *value = h->gemv_threads; return PIDE_OK;
    case PIDE_TUNE_GEMV_UNROLL: *value = h->gemv_unroll; return PIDE_OK;
    case PIDE_TUNE_GEMV_MAX_B: *value = h->gemv_max_b; return PIDE_OK;
    case PIDE_TUNE_GEMM_BN: *value = h->gemm_bn_large; return PIDE_OK;
    case PIDE_TUNE_GEMM_STREAMK: *value = h->gemm_streamk; return PIDE_OK;
    case PIDE_TUNE_OVERLAP: *value = h->overlap; return PIDE_OK;
    case PIDE_TUNE_RESID_CTAS: *value = h->resid_ctas_per_sm; return PIDE_OK;
    case PIDE_TUNE_SYMV: *value = h->symv; return PIDE_OK;
    case PIDE_TUNE_RESID_EMUL: *value = h->resid_emul; return PIDE_OK;
    case PIDE_TUNE_RESID_SHAPE: *value = h->resid_shape; return PIDE_OK;
    case PIDE_TUNE_GEMM_2CTA: *value = h->gemm_2cta; return PIDE_OK;
    case PIDE_TUNE_GEMM_A_HINT: *value = h->gemm_a_hint; return PIDE_OK;
    case PIDE_TUNE_RESID_PREFETCH: *value = h->resid_prefetch; return PIDE_OK;
    case PIDE_TUNE_CORR_MASK: *value = h->corr_mask; return PIDE_OK;
    case PIDE_TUNE_GEMM_U_HINT: *value = h->gemm_u_hint; return PIDE_OK;
    case PIDE_TUNE_BATCH_TC: *value = h->batch_tc; return PIDE_OK;
    case PIDE_TUNE_BATCH_BN: *value = h->batch_bn; return PIDE_OK;
    case PIDE_TUNE_BATCH_TN: *value = h->batch_tn; return PIDE_OK;
    case PIDE_TUNE_PREP_CLUSTER: *value = h->prep_cluster; return PIDE_OK;
  }
  set_error("pide_get_tuning: unknown key");
  return PIDE_EINVAL;
}

extern "C" const char* pide_status_string(pide_status s) {
  switch (s) {
    case PIDE_OK: return "ok";
    case PIDE_EINVAL: return "invalid argument";
    case PIDE_ENOMEM: return "out of memory";
    case PIDE_ECUDA: return "CUDA error";
    case PIDE_ENOTCONV: return "refinement did not reach the tolerance";
    case PIDE_ETIMEOUT: return "device-side wait timed out";
    case PIDE_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

// One thread waits on an mbarrier that nothing will complete, with a short
// cycle budget: the bounded-wait path every kernel uses gives up, records the
// error word and returns, and the host reports PIDE_ETIMEOUT.
__global__ void timeout_probe_kernel(long long budget, uint32_t* flags) {
  __shared__ uint64_t bar;
  __shared__ int abort_s;
  mbar_init(&bar, 1);
  abort_s = 0;
  fence_barrier_init();
  if (!mbar_wait_bounded(&bar, 0, &abort_s, budget)) flags[FLAG_ERROR] = DEV_TIMEOUT_MMA;
  mbar_arrive(&bar);   // complete the phase so nothing is left pending
}

extern "C" pide_status pide_selftest_wait_timeout(int64_t budget_cycles, void* stream) {
  if (budget_cycles <= 0 || budget_cycles > (int64_t)PIDE_WAIT_BUDGET_CYCLES) {
    set_error("pide_selftest_wait_timeout: budget out of range");
    return PIDE_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* fl = nullptr;
  PIDE_CUDA_TRY(cudaMalloc((void**)&fl, FLAG_COUNT * sizeof(uint32_t)));
  cudaMemsetAsync(fl, 0, FLAG_COUNT * sizeof(uint32_t), st);
  timeout_probe_kernel<<<1, 1, 0, st>>>((long long)budget_cycles, fl);
  cudaError_t e = cudaGetLastError();
  uint32_t code = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&code, fl + FLAG_ERROR, sizeof(code), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(fl);
  PIDE_CUDA_TRY(e);
  if (code) {
    set_error("bounded wait expired as requested (code " + std::to_string(code) + ")");
    return PIDE_ETIMEOUT;
  }
  return PIDE_OK;
}

// Bit-for-bit comparison of the integer-pipe conversions with CUDA's own.
__global__ void convert_selftest_kernel(const double* __restrict__ x, const float* __restrict__ f,
                                        long long n, uint16_t* __restrict__ bf_mine,
                                        uint16_t* __restrict__ bf_cuda, double* __restrict__ d_mine,
                                        double* __restrict__ d_cuda) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    bf_mine[i] = f64_to_bf16_bits(x[i]);
    bf_cuda[i] = __bfloat16_as_ushort(__double2bfloat16(x[i]));
    d_mine[i] = f32_to_f64(f[i]);
    d_cuda[i] = (double)f[i];
  }
}

extern "C" pide_status pide_selftest_convert(const double* x_dev, const float* f_dev, int64_t n,
                                             uint16_t* bf_mine, uint16_t* bf_cuda,
                                             double* d_mine, double* d_cuda, void* stream) {
  if (n < 0 || (n > 0 && (!x_dev || !f_dev || !bf_mine || !bf_cuda || !d_mine || !d_cuda))) {
    set_error("pide_selftest_convert: bad argument");
    return PIDE_EINVAL;
  }
  if (n == 0) return PIDE_OK;
  convert_selftest_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(x_dev, f_dev, (long long)n,
                                                                 bf_mine, bf_cuda, d_mine, d_cuda);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

extern "C" const char* pide_last_error(void) { return g_last_error.c_str(); }

extern "C" int32_t pide_version(void) { return 1; }
