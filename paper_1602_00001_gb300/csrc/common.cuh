// Internal declarations shared by the CUDA translation units of libpide.
// Nothing here is part of the public ABI (include/pide.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pide.h"

namespace pide {

// ---------------------------------------------------------------- errors

void set_error(const std::string& msg);

#define PIDE_CUDA_TRY(expr)                                                   \
  do {                                                                        \
    cudaError_t e__ = (expr);                                                 \
    if (e__ != cudaSuccess) {                                                 \
      ::pide::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__)); \
      return e__ == cudaErrorMemoryAllocation ? PIDE_ENOMEM : PIDE_ECUDA;     \
    }                                                                         \
  } while (0)

#define PIDE_TRY(expr)                 \
  do {                                 \
    pide_status s__ = (expr);          \
    if (s__ != PIDE_OK) return s__;    \
  } while (0)

// Device-side error word values (ctx->flags[1]).
enum : uint32_t { DEV_OK = 0, DEV_TIMEOUT_TMA = 1, DEV_TIMEOUT_MMA = 2, DEV_TIMEOUT_EPI = 3,
                  DEV_TIMEOUT_DRAIN = 4 };

// Flag words in device memory.
enum { FLAG_DONE = 0, FLAG_ERROR = 1, FLAG_SWEEPS = 2, FLAG_WHERE = 3, FLAG_COUNT = 8 };

// ---------------------------------------------------------------- context

enum ApplyKind { KIND_F64 = 0, KIND_F32 = 1, KIND_BF16 = 2, KIND_FP8 = 3, KIND_FP8X2 = 4, KIND_F16 = 6 };

struct pide_ctx_impl;

}  // namespace pide

struct pide_ctx {
  // grid and operator (dims 2: nx x ny nodes; dims 3: nx x ny x nz nodes, x fastest)
  int dims = 2;
  int nx = 0, ny = 0, nz = 1, mx = 0, my = 0, mz = 1, n = 0;
  double h = 0.0;
  pide_precision prec = PIDE_FP64;
  int device = 0, num_sms = 0;
  int ld = 0;                       // row stride of the stored inverse (elements)
  double* eps = nullptr;            // [(nz)][ny][nx] node permittivity
  double* cf = nullptr;             // [4 or 6][n] face eps of each interior node: W, E, S, N (, D, U)
  double* d = nullptr;              // [n] diagonal of S (sum of face eps)
  double* dinv = nullptr;           // [n] 1 / d
  double* w = nullptr;              // [4 or 6][n] Eq. (3) weights w = cf / d
  float4* wsp = nullptr;            // [2 or 3][n] w as float pairs, zero toward boundary nodes:
                                    // (W,E,S,N) hi, (W,E,S,N) lo (, (D hi, U hi, D lo, U lo))
  std::vector<double> eps_host;     // kept for save/load
  // stored inverse L^-1 = S^-1 D (the interior block of the Fig. 3 inverse)
  void* inv = nullptr;              // [n][ld] FP64 / FP32 / BF16 / FP16 / e4m3 (hi)
  void* inv_lo = nullptr;           // [n][ld] e4m3 lo term (FP8X2)
  float* row_scale = nullptr;       // [n] per-row scale (FP8 formats; FP16: powers of two)
  // PIDE_BF16_FP8 / PIDE_FP16_FP8: e4m3 correction term of the BF16 or FP16 store
  // (prec stays PIDE_BF16 / PIDE_FP16)
  void* corr = nullptr;             // [n][ld] e4m3((L^-1 - bf16(L^-1)) / corr_scale)
  float* corr_scale = nullptr;      // [n] its per-row scale
  int corr_mask = 2;                // applies that add it: bit 0 the first, bit k sweep k
  size_t store_bytes = 0;
  void* sym = nullptr;              // packed lower 128x128 BF16 tiles of S^-1, hi term (B = 1 apply)
  void* sym_lo = nullptr;           // same layout, lo term fp16((S^-1 - hi) / sigma_p)
  float* sym_scale = nullptr;       // [n] sigma_p: power-of-two scale of row p's lo term
  long long sym_tiles = 0;
  size_t sym_bytes = 0;
  float* dfl = nullptr;             // [n] d as float (x = D r formed on the fly)
  double* ysum = nullptr;           // [n] accumulation of the symmetric apply (FP64 atomics)
  bool tmA_ok = false;
  CUtensorMap tmA, tmA_lo;          // TMA maps over the stored inverse (tensor-core formats)
  CUtensorMap tmA_corr;             // over the correction term (PIDE_BF16_FP8)
  // workspace (grown on demand; pide_reserve pre-sizes it)
  int ws_B = 0;
  void* R = nullptr;                // [ws_B][ld] quantised right-hand side / residual
  float* col_scale = nullptr;       // [ws_B] per-column scale (FP8 formats; FP16: powers of two)
  float* Rf = nullptr;              // [ws_B][ld] FP32 residual before FP8 quantisation
  void* Rc = nullptr;               // [ws_B][ld] e4m3 copy of the BF16 R for the correction term
  float* col_scale_c = nullptr;     // [ws_B] its per-column scale
  CUtensorMap tmRc;
  double* lift = nullptr;           // [n] boundary lifting sum_q w_pq g_q
  double* colmax = nullptr;         // [3][ws_B] column maxima: |r|, |b|, raw (FP8 scales)
  uint32_t* flags = nullptr;        // FLAG_COUNT words
  double* hbuf_b = nullptr;         // device staging for pide_apply_host
  double* hbuf_u = nullptr;
  int hbuf_B = 0;
  void* tmR_ptr = nullptr;          // which R buffer tmR describes
  int tmR_rows = 0;
  CUtensorMap tmR;
  // launch-shape knobs (pide_set_tuning; the autotuner sets them)
  int gemm_bn_large = 256;          // BN for B > 128: 128 or 256
  int gemm_streamk = 1;             // stream-K tail after the full data-parallel waves
  int gemm_2cta = 1;                // B > 128 on SM pairs (tcgen05 cta_group::2)
  int gemm_a_hint = 2;              // L2 policy of the inverse's TMA loads (policy_for_a)
  int gemm_u_hint = 1;              // epilogue's u loads/stores: 0 plain, 1 L2 evict-first
  int max_pairs = 0;                // SM pairs resident at once for that kernel (queried once)
  // K-split last round of the SM-pair GEMM: FP32 partial tiles (one 256 x 256
  // slot per pair, allocated with the workspace) and the reduction that the
  // GEMM's caller launches after the GEMM's own profile scope
  float* tail_ws = nullptr;
  int tail_slots = 0;
  struct TailReduce {
    bool pending = false;
    double* u = nullptr;            // the GEMM's u (already offset to its first column)
    int B = 0, n_tiles = 0, first_tile = 0, tiles = 0, P = 0, accumulate = 0;
  } tail;
  int overlap = 0;                  // residual of one column group under the GEMM of the other
  int resid_ctas_per_sm = 2;        // residual grid under a concurrent GEMM (CTAs of 256 per SM)
  cudaStream_t aux = nullptr;       // low-priority stream for the overlapped residuals
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaStream_t cstream = nullptr;   // host<->device copies of pide_apply_host
  cudaEvent_t hev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // pide_solve_stream: two device slots of `sbuf_cols` columns for the input and
  // the solution, copies in on cstream and out on dstream
  cudaStream_t dstream = nullptr;
  cudaEvent_t sev[9] = {};
  double* sbuf_in = nullptr;
  double* sbuf_out = nullptr;
  int sbuf_cols = 0;
  int gemv_max_b = 1;               // largest B sent to the GEMV kernel (tcgen05 above)
  int gemv_threads = 1024;          // GEMV block size (multiple of 32, <= 1024)
  int gemv_unroll = 8;              // 16-byte loads in flight per lane: 4 or 8
  int symv = 1;                     // B = 1 through the packed symmetric S^-1 (half the bytes)
  int resid_emul = 1;               // refinement residual in double-float (off the FP64 pipe)
  int resid_shape = -1;             // its launch shape: -1 default (8 nodes per thread); 0..3: 4, 8, 2, 16
  int resid_prefetch = 4;           // its L2 prefetch distance in column pairs (0: none)
  int prep_cluster = 1;             // FP16 prep: one CTA cluster per column, one HBM pass
  // batched plans (pide_batch_create reads them per problem; the autotuner sets them)
  int batch_tc = 1;                 // FP32 store: 1 TF32 tensor cores, 0 FP32 SIMT tiles
  int batch_bn = 0;                 // tensor-core column tile 32, 64 or 128 (0: the narrowest covering B)
  int batch_tn = 0;                 // SIMT tile width 16, 32 or 64 (0: the narrowest covering B)
  // refinement history of a pide_apply that fills pide_info: the worst-column
  // relative residual after apply k (k < HIST_MAX), and events timing the call
  double* hist = nullptr;
  cudaEvent_t tev[2] = {nullptr, nullptr};
  // pide_setup_auto: what was measured, and the sweep count it chose
  bool has_auto = false;
  pide_auto_report auto_rep = {};
  int sweeps_hint = -1;
  // profiling
  bool prof_on = false;
  struct Ev { cudaEvent_t a, b; int cls; };
  std::vector<Ev> prof_events;
  double setup_ms = 0.0;
};

namespace pide {

// Nodes in one z-plane of the interior (3-D), or all of them (2-D): the
// distance between up/down neighbours, and the bound that makes the 2-D
// stencil's up/down terms vanish.
inline int plane_of(const pide_ctx* c) { return c->dims == 3 ? c->mx * c->my : c->n; }

// ---------------------------------------------------------------- launchers
// (each returns a pide_status; kernels are enqueued on `st`)

pide_status launch_assemble(pide_ctx* c, cudaStream_t st);
pide_status launch_rhs_from_charge(pide_ctx* c, const double* rho, double* b, int B, cudaStream_t st);
pide_status launch_lift(pide_ctx* c, const double* g, cudaStream_t st);
pide_status build_inverse_fp64(pide_ctx* c, double* G, cudaStream_t st);   // G = L^-1 (FP64)
pide_status quantize_store(pide_ctx* c, const double* G, cudaStream_t st);

// RHS preparation: R = q(f), f = b + lift (mode 0) or f = b / d (mode 1, adjoint).
// emul: BF16 forward prep through the integer/FP32 pipes (same codes as FP64).
pide_status launch_prep(pide_ctx* c, const double* b, int B, int mode, const double* lift,
                        int rfmt, bool track, cudaStream_t st, bool emul = false);
// Residual: R = q(f - L u) (FP64 stencil); optional column max of |r| into colmax.
// col0: first column of a column group (b, u, R rows, scales and maxima offset by it).
// emul: forward residuals written only to R take the double-float kernel.
pide_status launch_residual(pide_ctx* c, const double* b, const double* u, int B, int mode,
                            const double* lift, int rfmt, bool write_R, double* r_out, bool track,
                            bool honor_done, cudaStream_t st, int col0 = 0, bool emul = false);
pide_status launch_check(pide_ctx* c, int B, double tol, cudaStream_t st);
// *slot = max over columns of colmax[c] / max|f_c| (the residual just tracked);
// reset: zero colmax afterwards (the tolerance check does it when tol > 0).
// Skipped once the tolerance flag marks the solve done.
pide_status launch_record(pide_ctx* c, int B, double* slot, bool reset, cudaStream_t st);
constexpr int HIST_MAX = 64;
// The refined solve of step 3 (api.cu): x = Q(L^-1) q(f), then `sweeps` sweeps
// x += Q(L^-1) q(f - L x); hist (device, may be NULL): per-sweep residual record.
pide_status solve_s(pide_ctx* c, const double* b, int mode, const double* lift, double* x,
                    int B, int sweeps, double tol, cudaStream_t st, double* hist = nullptr);
// The workspace sized for another right-hand-side format is released (select.cu).
void drop_workspace(pide_ctx* c);
// PIDE_AUTO (select.cu): measure the candidate stores against G = L^-1 (FP64) and
// leave the chosen one quantised in the handle (prec, corr, corr_mask, sweeps_hint).
pide_status auto_select(pide_ctx* c, const double* G, double target, const double* probe_host,
                        int nprobe, int max_sweeps, cudaStream_t st);
// FP8 right-hand sides in one FP64 pass: residual to FP32 scratch with the column
// maxima, per-column scale, then e4m3 quantisation of the scratch into R.
pide_status launch_residual_fp8(pide_ctx* c, const double* b, const double* u, int B, int mode,
                                const double* lift, cudaStream_t st, bool emul = false);
// Double-float residual (residual_df.cu): weights split once per operator, then
// r = f - L u (forward mode) into R[B][ldr] as BF16 / FP32 / e4m3 (col_scale).
pide_status launch_wsplit(pide_ctx* c, cudaStream_t st);
pide_status launch_residual_df(pide_ctx* c, const double* b, const double* u, int B,
                               const double* lift, int rfmt, void* R, int ldr,
                               const float* col_scale, double* colmax_r, bool track,
                               const uint32_t* flags, cudaStream_t st);
pide_status launch_prep_df_bf16(pide_ctx* c, const double* b, int B, const double* lift,
                                bool track, cudaStream_t st);
// FP16 right-hand sides (f16.cu): per column t_j = 2^k with max|f_j| / t_j in
// [2^11, 2^12) into col_scale, R = fp16(f / t_j) rounded to nearest from FP64;
// the refinement's residuals reuse t_j.
// with_corr: also write the e4m3 copy Rc of R and its column scales (what
// launch_corr_rhs does), in the same pass.
pide_status launch_prep_f16(pide_ctx* c, const double* b, int B, int mode, const double* lift,
                            bool track, cudaStream_t st, bool with_corr = false);
pide_status quantize_store_f16(pide_ctx* c, const double* G, cudaStream_t st);
// Residual with a small persistent grid (num_sms * resid_ctas_per_sm blocks), for the
// overlapped schedule; writes R only.
pide_status launch_residual_persistent(pide_ctx* c, const double* b, const double* u, int B,
                                      int mode, const double* lift, int rfmt, cudaStream_t st,
                                      int col0);
// FP8 right-hand sides: per-column scale max|f~|/448 (prep) or max|r~|/448 (residual).
pide_status launch_fp8_scales(pide_ctx* c, const double* b, const double* u, int B, int mode,
                              const double* lift, bool from_residual, cudaStream_t st,
                              int col0 = 0);
pide_status launch_colmax_b(pide_ctx* c, const double* b, int B, int mode, const double* lift,
                            cudaStream_t st);

// Apply: u (=|+=) Q(L^-1) R for B columns.
pide_status launch_apply(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                         int col0 = 0);
// PIDE_BF16_FP8: R (BF16) -> Rc = e4m3(R / t_j), t_j = max|R_j| / 448; then
// u += s_p t_j (C Rc) on the tensor cores.
pide_status launch_corr_rhs(pide_ctx* c, int B, cudaStream_t st);
pide_status launch_apply_corr(pide_ctx* c, int B, double* u, cudaStream_t st);
pide_status quantize_corr(pide_ctx* c, const double* G, cudaStream_t st);
int rhs_format(const pide_ctx* c, int B);   // element format R must hold for this B

// tensor-core GEMM (BF16, FP8X2) and SIMT paths
pide_status launch_gemm_tc(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                           int col0 = 0, bool corr = false);
// the same on pairs of SMs (tcgen05 cta_group::2, 256 x 256 tiles), for B > 128
pide_status launch_gemm_tc2(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                            int col0 = 0, bool corr = false);
// Adds the FP32 partial tiles of a K-split last round (left by the SM-pair GEMM
// in c->tail) to u, in profile class 4; nothing when none is pending.
pide_status launch_tail_reduce(pide_ctx* c, cudaStream_t st);
pide_status launch_gemv(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st);
pide_status build_sym_store(pide_ctx* c, const double* G, cudaStream_t st);   // G = L^-1 (FP64)
pide_status launch_symv(pide_ctx* c, double* u, bool accumulate, cudaStream_t st);
pide_status launch_gemm_simt(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st);

pide_status launch_face_grad(pide_ctx* c, const double* mu, const double* u, const double* b,
                             int B, double* deps, cudaStream_t st);
pide_status launch_scale_d(pide_ctx* c, const double* mu, double* db, int B, cudaStream_t st);

pide_status ensure_workspace(pide_ctx* c, int B);
pide_status make_tma_maps(pide_ctx* c);
// 2-D tiled TMA map, 128-byte swizzle, zero fill out of bounds.
pide_status encode_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                      uint64_t outer, uint64_t row_bytes, uint32_t box_in, uint32_t box_out);
pide_status make_tma_rhs(pide_ctx* c, int bn);
pide_status make_tma_rhs_corr(pide_ctx* c, int bn);   // tmRc over Rc (e4m3)

// event profiling around one launch of class `cls`
struct ProfScope {
  pide_ctx* c; cudaStream_t st; int cls; cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(pide_ctx* c_, cudaStream_t st_, int cls_);
  ~ProfScope();
};

enum RhsFmt { RF_F64 = 0, RF_F32 = 1, RF_BF16 = 2, RF_E4M3 = 3, RF_F16 = 4 };

size_t rhs_elem_bytes(int rfmt);

// ---------------------------------------------------------------- device helpers

#ifdef __CUDACC__

// Budget for every spin-wait on an mbarrier, in SM clock cycles (~1 s).
#define PIDE_WAIT_BUDGET_CYCLES (2000000000ll)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and leaves the barrier alone) once the cycle
// budget is spent or *abort becomes non-zero.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort_flag,
                                                  long long budget = PIDE_WAIT_BUDGET_CYCLES) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) return false;
  }
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tiled TMA load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Same with an L2 cache-policy hint.
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar,
                                                 int x, int y, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// FP64 loads and stores with an L2 cache-policy hint (the GEMM epilogues' u)
__device__ __forceinline__ double ld_f64_hint(const double* p, uint64_t policy) {
  double v;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(policy));
  return v;
}
__device__ __forceinline__ void st_f64_hint(double* p, double v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(policy)
               : "memory");
}

// L2 policy for the streamed inverse: 0 evict-first, 1 evict-normal, 2 evict-last
__device__ __forceinline__ uint64_t policy_for_a(int hint) {
  return hint == 0 ? policy_evict_first() : (hint == 1 ? policy_evict_normal() : policy_evict_last());
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---- IEEE 754 conversions on the integer pipe.  GB300's FP64 pipe is
// narrow (about 1 TFLOP/s); conversions issued there compete with the FP64
// stencil and the FP64 accumulation of u.  These follow the binary formats'
// definitions (sign | biased exponent | fraction) and hand the rare
// special cases (zero handled here; subnormal, overflow, inf, NaN) to the
// hardware conversion.

// binary32 -> binary64, exact.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t x = __float_as_uint(f);
  const uint32_t e = (x >> 23) & 0xFFu;
  if ((x & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)((uint64_t)x << 32));
  if (e == 0u || e == 0xFFu) return (double)f;
  const uint64_t bits = ((uint64_t)(x & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                        ((uint64_t)(x & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// binary64 -> bfloat16 bits, round to nearest, ties to even.  bfloat16 keeps
// 7 fraction bits with binary32's exponent range: the 45 dropped fraction
// bits decide the rounding (above half: up; exactly half: to even).
__device__ __forceinline__ uint16_t f64_to_bf16_bits(double v) {
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const uint32_t sign = (uint32_t)(u >> 48) & 0x8000u;
  const int eb = (int)((u >> 52) & 0x7FF) - 896;   // rebias 1023 -> 127
  if ((u << 1) == 0) return (uint16_t)sign;
  if (eb <= 0 || eb >= 255) return __bfloat16_as_ushort(__double2bfloat16(v));
  const uint64_t m = u & 0xFFFFFFFFFFFFFull;
  uint32_t r = ((uint32_t)eb << 7) | (uint32_t)(m >> 45);
  const uint64_t rest = m & 0x1FFFFFFFFFFFull;
  const uint64_t half = 0x100000000000ull;
  if (rest > half || (rest == half && (r & 1u))) r += 1u;
  return (uint16_t)(sign | r);
}

// ---- tcgen05 (5th-generation tensor cores, accumulators in TMEM)

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16/F16 inputs, F32 accumulate)
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// kind::tf32: FP32 operands in shared memory read as TF32 (10 explicit
// mantissa bits), F32 accumulate; K = 8 per instruction (32 bytes per row,
// the same byte step as kind::f16's K = 16).
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// kind::f8f6f4 (here: e4m3 x e4m3, F32 accumulate)
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on `bar` when every previously issued tcgen05.mma of this thread completes.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread t gets row (lane base + t).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile stored with the
// 128-byte swizzle (rows of 128 bytes, 8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  desc |= (uint64_t)(16 >> 4) << 16;                 // leading byte offset (unused for SW128 K-major)
  desc |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8-row group
  desc |= (uint64_t)1 << 46;                         // descriptor version (tcgen05)
  desc |= (uint64_t)2 << 61;                         // swizzle: 128B
  return desc;
}

#endif  // __CUDACC__

}  // namespace pide
