// Step 3 on the 5th-generation tensor cores: U (=|+=) Q(S^-1) * R for many
// right-hand sides, the dense contraction at the heart of the direct method.
//
//   A = stored inverse, [n][ld] row-major (K = q contiguous)  -> K-major operand
//   B = right-hand sides R, [B][ld] row-major (K contiguous)   -> K-major operand
//   D[p][col] accumulates in TMEM (FP32); the epilogue writes the FP64 result
//   u[col][p] (one right-hand side per row of u), adding to it during sweeps.
//
// Persistent, warp-specialised kernel, one CTA per SM (192 threads):
//   warp 0  TMA producer: 128 x BK tiles of A and BN x BK tiles of R per stage,
//           128-byte swizzle, STAGES-deep ring of shared-memory buffers
//   warp 1  allocates TMEM, one thread issues tcgen05.mma (M=128, N=BN) and
//           commits each stage back to the producer and each finished tile to
//           the epilogue
//   warps 2-5  epilogue: tcgen05.ld 32 lanes x 32 columns at a time, scale,
//           FP64 read-modify-write of u (coalesced along p)
// The accumulator is double-buffered in TMEM (2 x BN columns) so the epilogue
// of tile t overlaps the main loop of tile t+1.  Tiles are ordered with the
// right-hand-side tile fastest, so the CTAs that share one 128-row slab of the
// inverse run at the same time and the slab is read from HBM about once.
//
// Schedule: data-parallel waves plus a stream-K tail (Osama, Merrill, Cecka,
// Garland, "Stream-K: Work-centric Parallel Decomposition for Dense
// Matrix-Matrix Multiplication on the GPU", PPoPP 2023).  All but the last
// one-and-a-bit waves of tiles go round-robin to the CTAs whole; the tiles
// left over are cut into k-block units and every CTA takes an equal,
// contiguous share, so no SM idles in a partial last wave.  A CTA that holds
// only part of a tile's K range adds its partial sum into u with FP64 atomic
// adds (those tiles are zeroed first when the apply overwrites u).
//
// FP8X2: A is the e4m3 hi term and A_lo the lo term (per-row scale in the
// epilogue); both multiply the same e4m3 R tile and accumulate into the same
// TMEM tile, i.e. one contraction with K doubled.
//
// Every wait on an mbarrier is bounded (about a second): on expiry the kernel
// records an error word, lets the other roles leave, waits (bounded) for its
// outstanding copies and MMAs, frees TMEM and returns.
#include "common.cuh"

namespace pide {

namespace {

constexpr int BM = 128;
constexpr int ROW_BYTES = 128;    // K extent of one stage: one 128-byte swizzle row

template <int BN, bool FP8>
struct TcCfg {
  static constexpr int A_BYTES = BM * ROW_BYTES;           // 16 KB
  static constexpr int B_BYTES = BN * ROW_BYTES;
  static constexpr int K_ELEMS = FP8 ? 128 : 64;            // elements per stage along K
  static constexpr int K_PER_MMA_BYTES = 32;                // 16 bf16 or 32 e4m3
  static constexpr int MMAS_PER_STAGE = ROW_BYTES / K_PER_MMA_BYTES;
  static constexpr uint32_t TMEM_COLS = (2 * BN < 32) ? 32 : 2 * BN;
};

// The (tile, k-block range) segments one CTA works through, identical for all
// roles.  Data-parallel part: tiles blockIdx.x, +G, ... below dp_tiles.
// Stream-K part: the remaining 128-row slabs x k-blocks are split evenly over
// groups of T = n_tiles consecutive CTAs; the T CTAs of a group walk the same
// (slab, k-range) in lockstep, one right-hand-side tile each, so every slab
// of the inverse is still fetched from HBM about once.
struct SegIter {
  int G, T, dp_tiles, num_kb, t_dp, j, base_m;
  long long u, u1;
  __device__ SegIter(int dp, int nkb, int n_tiles, int m_tiles, int sk)
      : G((int)gridDim.x), T(n_tiles), dp_tiles(dp), num_kb(nkb), t_dp((int)blockIdx.x) {
    const int NG = G / T;
    const int g = (int)blockIdx.x / T;
    j = (int)blockIdx.x - g * T;
    base_m = dp_tiles / T;
    const long long U = sk ? (long long)(m_tiles - base_m) * nkb : 0;
    if (NG > 0 && g < NG) {
      u = U * g / NG;
      u1 = U * (g + 1) / NG;
    } else {
      u = u1 = 0;
    }
  }
  __device__ bool next(int& tile, int& kb0, int& kb1) {
    if (t_dp < dp_tiles) {
      tile = t_dp;
      kb0 = 0;
      kb1 = num_kb;
      t_dp += G;
      return true;
    }
    if (u < u1) {
      const int m = base_m + (int)(u / num_kb);
      tile = m * T + j;
      kb0 = (int)(u % num_kb);
      const long long left = u1 - u;
      kb1 = (kb0 + left < num_kb) ? kb0 + (int)left : num_kb;
      u += kb1 - kb0;
      return true;
    }
    return false;
  }
};

template <int BN, int STAGES, int MODE>   // MODE 0: BF16, 1: FP8 (hi only), 2: FP8X2 (hi + lo), 3: FP16 (row/column scales)
__global__ void __launch_bounds__(192, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
               const __grid_constant__ CUtensorMap tmR, int n, int B, int rrow0, int num_kb,
               int dp_tiles, int sk, double* __restrict__ u, int accumulate,
               const float* __restrict__ row_scale, const float* __restrict__ col_scale,
               uint32_t* __restrict__ flags, int a_hint, int u_hint) {
  constexpr bool FP8 = MODE == 1 || MODE == 2;   // kind::f8f6f4 (else kind::f16)
  constexpr bool SCALED = MODE != 0;              // epilogue applies row and column scales
  constexpr bool LO = MODE == 2;
  using C = TcCfg<BN, FP8>;
  constexpr int A_STAGE = LO ? 2 * C::A_BYTES : C::A_BYTES;
  constexpr uint32_t STAGE_TX = A_STAGE + C::B_BYTES;

  if (flags[FLAG_DONE]) return;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * C::B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (B + BN - 1) / BN;
  const int m_tiles = (n + BM - 1) / BM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 128);
    }
    mbar_init(drain, 1);
    *abort_s = 0;
    fence_barrier_init();
    prefetch_tmap(&tmA);
    if (LO) prefetch_tmap(&tmAlo);
    prefetch_tmap(&tmR);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    const uint64_t pol_a = policy_for_a(a_hint);    // the inverse streams through L2 once
    const uint64_t pol_r = policy_evict_last();    // the right-hand sides are re-read by every slab
    int s = 0;
    uint32_t ph = 0;
    uint32_t issued = 0;                            // bit s: stage s has a copy in flight
    uint32_t issued_ph = 0;                         // parity of that copy's phase
    bool ok = true;
    SegIter it(dp_tiles, num_kb, n_tiles, m_tiles, sk);
    int tile, kb0, kb1;
    while (ok && it.next(tile, kb0, kb1)) {
      const int mt = tile / n_tiles, nt = tile - mt * n_tiles;
      for (int kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait_bounded(&empty[s], ph ^ 1, abort_s)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full[s], STAGE_TX);
        const int kx = kb * C::K_ELEMS;
        tma_load_2d_hint(sA + s * A_STAGE, &tmA, &full[s], kx, mt * BM, pol_a);
        if (LO) tma_load_2d_hint(sA + s * A_STAGE + C::A_BYTES, &tmAlo, &full[s], kx, mt * BM, pol_a);
        tma_load_2d_hint(sB + s * C::B_BYTES, &tmR, &full[s], kx, rrow0 + nt * BN, pol_r);
        issued |= 1u << s;
        issued_ph = (issued_ph & ~(1u << s)) | (ph << s);
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    if (!ok) {
      atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_TMA);
      *abort_s = 1;
      // wait (bounded, ignoring the abort flag) for our own copies still in flight
      volatile int never = 0;
      for (int t = 0; t < STAGES; ++t)
        if (issued & (1u << t)) mbar_wait_bounded(&full[t], (issued_ph >> t) & 1u, &never);
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    uint32_t idesc = (1u << 4)                                  // D: F32
                     | ((MODE == 0 ? 1u : 0u) << 7)             // A: BF16 / F16 (kind::f16), E4M3 (kind::f8f6f4)
                     | ((MODE == 0 ? 1u : 0u) << 10)            // B: same
                     | ((uint32_t)(BN >> 3) << 17)              // N
                     | ((uint32_t)(BM >> 4) << 24);             // M
    int s = 0;
    uint32_t ph = 0;
    int acc = 0;
    uint32_t acc_ph = 0;
    bool ok = true;
    SegIter it(dp_tiles, num_kb, n_tiles, m_tiles, sk);
    int tile, kb0, kb1;
    while (ok && it.next(tile, kb0, kb1)) {
      if (!mbar_wait_bounded(&tempty[acc], acc_ph ^ 1, abort_s)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
      for (int kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait_bounded(&full[s], ph, abort_s)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(sA + s * A_STAGE);
        const uint32_t b_addr = smem_u32(sB + s * C::B_BYTES);
#pragma unroll
        for (int k = 0; k < C::MMAS_PER_STAGE; ++k) {
          const uint64_t bdesc = smem_desc_sw128(b_addr + k * C::K_PER_MMA_BYTES);
          const uint64_t adesc = smem_desc_sw128(a_addr + k * C::K_PER_MMA_BYTES);
          const uint32_t accum = (kb > kb0 || k > 0) ? 1u : 0u;
          if (FP8) mma_f8(d_tmem, adesc, bdesc, idesc, accum);
          else mma_f16(d_tmem, adesc, bdesc, idesc, accum);
          if (LO) {
            const uint64_t ldesc = smem_desc_sw128(a_addr + C::A_BYTES + k * C::K_PER_MMA_BYTES);
            mma_f8(d_tmem, ldesc, bdesc, idesc, 1u);
          }
        }
        mma_commit(&empty[s]);                     // frees the stage when these MMAs finish
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(&tfull[acc]);                     // tile done -> epilogue
      acc ^= 1;
      if (acc == 0) acc_ph ^= 1;
    }
    if (!ok) {
      atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_MMA);
      *abort_s = 1;
    }
    // drain: every MMA issued above has finished once this commit arrives
    mma_commit(drain);
    volatile int never = 0;
    if (!mbar_wait_bounded(drain, 0, &never)) atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_DRAIN);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;                  // TMEM lanes 32*quarter .. +31
    const uint64_t upol = policy_evict_first();     // used when u_hint
    const int row_in_tile = quarter * 32 + lane;
    int acc = 0;
    uint32_t acc_ph = 0;
    SegIter it(dp_tiles, num_kb, n_tiles, m_tiles, sk);
    int tile, kb0, kb1;
    while (it.next(tile, kb0, kb1)) {
      const int mt = tile / n_tiles, nt = tile - mt * n_tiles;
      const bool whole = (kb0 == 0 && kb1 == num_kb);
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
      const int p = mt * BM + row_in_tile;
      const bool prow = p < n;
      const float rs = (SCALED && prow) ? row_scale[p] : 1.0f;
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t v[32];
        tmem_ld_32x32b_x32(tbase + ch * 32, v);
        tmem_ld_wait();
        const int colbase = nt * BN + ch * 32;
        if (prow) {
          // the 32 old values first: loads issued together instead of one
          // load-add-store round trip per column (the stores through u
          // could alias later loads, so the compiler keeps them in order)
          double old[32];
          if (accumulate && whole) {
            if (u_hint) {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                old[j] = (colbase + j < B) ? ld_f64_hint(u + (size_t)(colbase + j) * n + p, upol) : 0.0;
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                old[j] = (colbase + j < B) ? u[(size_t)(colbase + j) * n + p] : 0.0;
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = colbase + j;
            if (col < B) {
              // scales applied in FP32 (powers of two for FP16: exact; the FP8
              // apply is good to ~2^-8 anyway);
              // one FP64 operation per element: the add into u
              float a = __uint_as_float(v[j]);
              if (SCALED) a = a * rs * col_scale[col];
              const double val = f32_to_f64(a);
              double* dst = u + (size_t)col * n + p;
              if (!whole) atomicAdd(dst, val);
              else if (u_hint) st_f64_hint(dst, accumulate ? old[j] + val : val, upol);
              else *dst = accumulate ? old[j] + val : val;
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
    tmem_dealloc(tmem_base, C::TMEM_COLS);
  }
}

// Zero the output tiles that the stream-K tail will build from atomic partial sums.
__global__ void zero_tiles_kernel(double* __restrict__ u, int n, int B, int bm, int bn,
                                  int n_tiles, int first_tile, const uint32_t* __restrict__ flags) {
  if (flags[FLAG_DONE]) return;
  const int tile = first_tile + blockIdx.x;
  const int mt = tile / n_tiles, nt = tile - mt * n_tiles;
  for (int e = threadIdx.x; e < bm * bn; e += blockDim.x) {
    const int col = nt * bn + e / bm, p = mt * bm + e % bm;
    if (col < B && p < n) u[(size_t)col * n + p] = 0.0;
  }
}

template <int BN, int STAGES, int MODE>
pide_status launch_tc(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st, int col0,
                      bool corr) {
  using C = TcCfg<BN, MODE == 1 || MODE == 2>;
  constexpr int A_STAGE = (MODE == 2) ? 2 * C::A_BYTES : C::A_BYTES;
  const size_t smem = 1024 + (size_t)STAGES * (A_STAGE + C::B_BYTES) + 256;
  PIDE_TRY(corr ? make_tma_rhs_corr(c, BN) : make_tma_rhs(c, BN));
  auto kern = gemm_tc_kernel<BN, STAGES, MODE>;
  PIDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int m_tiles = (c->n + BM - 1) / BM;
  const int n_tiles = (B + BN - 1) / BN;
  const int tiles = m_tiles * n_tiles;
  const int num_kb = (c->n + C::K_ELEMS - 1) / C::K_ELEMS;
  int grid, dp_tiles;
  if (!c->gemm_streamk || tiles % c->num_sms == 0 || n_tiles > c->num_sms) {
    grid = tiles < c->num_sms ? tiles : c->num_sms;
    dp_tiles = tiles;
  } else {
    // all but the last one-and-a-bit waves whole; dp_tiles a whole number of slabs
    grid = c->num_sms;
    dp_tiles = tiles < grid ? 0 : ((tiles / grid - 1) * grid / n_tiles) * n_tiles;
  }
  const int sk = dp_tiles < tiles ? 1 : 0;
  if (sk && !accumulate) {
    zero_tiles_kernel<<<tiles - dp_tiles, 256, 0, st>>>(u, c->n, B, BM, BN, n_tiles, dp_tiles,
                                                         c->flags);
    PIDE_CUDA_TRY(cudaGetLastError());
  }
  // the correction term: e4m3 C against Rc, scales s_p (rows) and t_j (columns)
  const CUtensorMap& A = corr ? c->tmA_corr : c->tmA;
  const CUtensorMap& Alo = corr ? c->tmA_corr : c->tmA_lo;
  const CUtensorMap& R = corr ? c->tmRc : c->tmR;
  const float* rs = corr ? c->corr_scale : c->row_scale;
  const float* cs = corr ? c->col_scale_c + col0 : (MODE != 0 ? c->col_scale + col0 : nullptr);
  kern<<<grid, 192, smem, st>>>(A, Alo, R, c->n, B, col0, num_kb, dp_tiles, sk, u,
                                accumulate ? 1 : 0, rs, cs, c->flags, c->gemm_a_hint,
                                c->gemm_u_hint);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

template <int MODE>
pide_status launch_tc_mode(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                           int col0, bool corr = false) {
  // BN: the smallest supported tile that covers B (up to 256); stages fill ~200 KB.
  if (MODE == 0 || MODE == 3) {
    if (B <= 32) return launch_tc<32, 10, MODE>(c, B, u, accumulate, st, col0, corr);
    if (B <= 64) return launch_tc<64, 8, MODE>(c, B, u, accumulate, st, col0, corr);
    if (B <= 128 || c->gemm_bn_large == 128) return launch_tc<128, 6, MODE>(c, B, u, accumulate, st, col0, corr);
    return launch_tc<256, 4, MODE>(c, B, u, accumulate, st, col0, corr);
  } else if (MODE == 1) {
    if (B <= 32) return launch_tc<32, 10, MODE>(c, B, u, accumulate, st, col0, corr);
    if (B <= 64) return launch_tc<64, 8, MODE>(c, B, u, accumulate, st, col0, corr);
    if (B <= 128 || c->gemm_bn_large == 128) return launch_tc<128, 6, MODE>(c, B, u, accumulate, st, col0, corr);
    return launch_tc<256, 4, MODE>(c, B, u, accumulate, st, col0, corr);
  } else {
    if (B <= 32) return launch_tc<32, 6, MODE>(c, B, u, accumulate, st, col0, corr);
    if (B <= 64) return launch_tc<64, 5, MODE>(c, B, u, accumulate, st, col0, corr);
    if (B <= 128 || c->gemm_bn_large == 128) return launch_tc<128, 4, MODE>(c, B, u, accumulate, st, col0, corr);
    return launch_tc<256, 3, MODE>(c, B, u, accumulate, st, col0, corr);
  }
}

}  // namespace

pide_status launch_zero_tiles(pide_ctx* c, double* u, int B, int bm, int bn, int n_tiles,
                              int first_tile, int count, cudaStream_t st) {
  if (count <= 0) return PIDE_OK;
  zero_tiles_kernel<<<count, 256, 0, st>>>(u, c->n, B, bm, bn, n_tiles, first_tile, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_gemm_tc(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                           int col0, bool corr) {
  if (c->gemm_2cta && B > 128 && c->gemm_bn_large == 256)
    return launch_gemm_tc2(c, B, u, accumulate, st, col0, corr);
  if (!c->tmA_ok) {
    set_error("tensor-core apply: TMA maps were not created");
    return PIDE_EUNSUPPORTED;
  }
  if (corr) return launch_tc_mode<1>(c, B, u, true, st, col0, true);
  switch (c->prec) {
    case PIDE_BF16: return launch_tc_mode<0>(c, B, u, accumulate, st, col0);
    case PIDE_FP8: return launch_tc_mode<1>(c, B, u, accumulate, st, col0);
    case PIDE_FP8X2: return launch_tc_mode<2>(c, B, u, accumulate, st, col0);
    case PIDE_FP16: return launch_tc_mode<3>(c, B, u, accumulate, st, col0);
    default: return PIDE_EUNSUPPORTED;
  }
}

}  // namespace pide
