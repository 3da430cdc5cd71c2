// Step 3 on pairs of SMs: the same contraction as gemm_tc.cu, U (=|+=) Q(S^-1) R,
// with 256 x 256 output tiles computed by tcgen05.mma.cta_group::2.
//
// A cluster of two CTAs owns one output tile of 256 rows (p) x 256 columns
// (right-hand sides).  CTA r of the pair stages rows 128 r .. 128 r + 127 of the
// A tile and columns 128 r .. 128 r + 127 of the right-hand-side tile; the MMA
// issued by CTA 0 reads both CTAs' halves and leaves rows 128 r .. of the
// accumulator in CTA r's tensor memory (all 256 columns).  Per SM and stage
// this stages 32 KB of operands (16 KB of A, 16 KB of R) for the work that the
// single-SM kernel (M = 128, N = 256) stages 48 KB for, so shared-memory and
// L2 -> SM traffic per flop fall by a third and more pipeline stages fit.
//
// Synchronisation across the pair:
//   full[s]   in CTA 0: both CTAs' TMA copies of stage s complete on it (the
//             copy's .cta_group::2 form may name the peer's barrier); CTA 0's
//             producer sets the expected bytes of both halves
//   empty[s]  in both CTAs: the MMA commit is multicast to the pair
//   tfull[a]  in both CTAs: multicast commit when accumulator a holds a tile
//   tempty[a] in CTA 0: all 256 epilogue threads of the pair arrive on it
// Every wait is bounded as in the single-SM kernel; on expiry the kernel
// records an error word and leaves through the same teardown (a cluster
// barrier, then the pair's collective TMEM release).
//
// Schedule: persistent clusters take whole tiles cid, cid + G, ... (G clusters).
// The r tiles of the last, partial round can be cut into P ranges of k-blocks
// each, dealt round-robin to the clusters (the choice of P is in launch_tc2);
// a piece writes its scaled FP32 partial tile to a slot of a workspace and a
// separate reduction kernel adds the P partials of each tile to u.  At 198^2
// unknowns and B = 1024 (616 tiles on 76 pairs: 8 rounds and 8 tiles) the
// ninth round of whole tiles cost as much as a full one.
#include "common.cuh"

namespace pide {

namespace {

constexpr int BM2 = 256;          // output rows per cluster tile (128 per CTA)
constexpr int BN2 = 256;          // right-hand sides per cluster tile (128 staged per CTA)
constexpr int HALF = 128;
constexpr int ROW_BYTES2 = 128;   // one 128-byte swizzle row of K per stage
constexpr int TC2_NACC = 2;       // accumulators per pair (512 TMEM columns)

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared::cluster address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA tile load into this CTA's shared memory, completion on an mbarrier that
// may live in the peer CTA (cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map,
                                                 uint32_t mbar_cluster, int x, int y,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar_cluster), "r"(x), "r"(y), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t mbar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(mbar_cluster)
               : "memory");
}

__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void mma_pair_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                             uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_pair_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on the barrier at this shared offset in both CTAs of the pair
// when the MMAs issued so far complete.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  const uint16_t mask = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// Arrive once on this CTA's barrier when the MMAs issued so far complete.
__device__ __forceinline__ void mma_commit_pair_local(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// The (tile, k-range) segments of one cluster: whole tiles cid, cid + G, ...
// below dp_tiles, then the pieces of the last round: piece g = cid, cid + G,
// ... below pieces = r P is piece q = g mod P of tile dp_tiles + g / P, and
// its partial goes to slot g.  Pieces are numbered tile by tile, so the
// clusters that run at the same time hold the same K-range of neighbouring
// tiles (the column tiles of one slab share their A rows in L2).
struct SegIter2 {
  int G, t_dp, dp_tiles, num_kb, P, pieces, g;
  __device__ SegIter2(int dp, int nkb, int P_, int pieces_)
      : G((int)gridDim.x / 2), t_dp((int)blockIdx.x / 2), dp_tiles(dp), num_kb(nkb), P(P_),
        pieces(pieces_), g((int)blockIdx.x / 2) {}
  __device__ bool next(int& tile, int& kb0, int& kb1, int& slot) {
    if (t_dp < dp_tiles) {
      tile = t_dp;
      kb0 = 0;
      kb1 = num_kb;
      slot = -1;
      t_dp += G;
      return true;
    }
    if (g < pieces) {
      const int t = g / P, q = g - t * P;
      tile = dp_tiles + t;
      kb0 = (int)((long long)num_kb * q / P);
      kb1 = (int)((long long)num_kb * (q + 1) / P);
      slot = g;
      g += G;
      return true;
    }
    return false;
  }
};

// NACC accumulators of 256 columns in tensor memory (2: the epilogue of one
// tile overlaps the main loop of the next).
template <int STAGES, int MODE, int NACC>   // MODE 0: BF16, 1: FP8 (hi only), 2: FP8X2 (hi + lo), 3: FP16 (row/column scales)
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
gemm_tc2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
                const __grid_constant__ CUtensorMap tmR, int n, int B, int rrow0, int num_kb,
                int dp_tiles, int P, int pieces, double* __restrict__ u, int accumulate,
                const float* __restrict__ row_scale, const float* __restrict__ col_scale,
                float* __restrict__ ws, uint32_t* __restrict__ flags, int a_hint, int u_hint) {
  constexpr bool FP8 = MODE == 1 || MODE == 2;   // kind::f8f6f4 (else kind::f16)
  constexpr bool SCALED = MODE != 0;              // epilogue applies row and column scales
  constexpr bool LO = MODE == 2;
  constexpr int A_BYTES = HALF * ROW_BYTES2;                  // 16 KB
  constexpr int A_STAGE = LO ? 2 * A_BYTES : A_BYTES;
  constexpr int B_BYTES = HALF * ROW_BYTES2;                  // 16 KB
  constexpr int K_ELEMS = FP8 ? 128 : 64;
  constexpr int K_PER_MMA_BYTES = 32;
  constexpr int MMAS_PER_STAGE = ROW_BYTES2 / K_PER_MMA_BYTES;
  constexpr uint32_t PAIR_TX = 2u * (A_STAGE + B_BYTES);      // both CTAs' bytes of a stage
  constexpr uint32_t TMEM_COLS = NACC * BN2;

  // the flag is read by both CTAs of the pair alike, so a pair leaves together
  if (flags[FLAG_DONE]) return;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_s = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int n_tiles = (B + BN2 - 1) / BN2;
  const int m_tiles = (n + BM2 - 1) / BM2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 2 * 128);
    }
    mbar_init(drain, 1);
    *abort_s = 0;
    fence_barrier_init();
    prefetch_tmap(&tmA);
    if (LO) prefetch_tmap(&tmAlo);
    prefetch_tmap(&tmR);
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_slot, TMEM_COLS);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();            // both CTAs' barriers and TMEM exist before any cross-CTA use
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer (both CTAs)
    const uint64_t pol_a = policy_for_a(a_hint);
    const uint64_t pol_r = policy_evict_last();
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    SegIter2 it(dp_tiles, num_kb, P, pieces);
    int tile, kb0, kb1, slot;
    while (ok && it.next(tile, kb0, kb1, slot)) {
      const int mt = tile / n_tiles, nt = tile - mt * n_tiles;
      const int arow = mt * BM2 + (int)rank * HALF;
      const int rrow = rrow0 + nt * BN2 + (int)rank * HALF;
      for (int kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait_bounded(&empty[s], ph ^ 1, abort_s)) {
          ok = false;
          break;
        }
        const uint32_t fbar = mapa_shared(smem_u32(&full[s]), 0);
        if (leader) mbar_expect_tx(&full[s], PAIR_TX);
        const int kx = kb * K_ELEMS;
        tma_load_2d_pair(sA + s * A_STAGE, &tmA, fbar, kx, arow, pol_a);
        if (LO) tma_load_2d_pair(sA + s * A_STAGE + A_BYTES, &tmAlo, fbar, kx, arow, pol_a);
        tma_load_2d_pair(sB + s * B_BYTES, &tmR, fbar, kx, rrow, pol_r);
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
    }
    if (!ok) {
      atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_TMA);
      *abort_s = 1;
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ------------------------------------------------------------ MMA issuer (CTA 0)
    const uint32_t idesc = (1u << 4)                            // D: F32
                           | ((MODE == 0 ? 1u : 0u) << 7)             // A: BF16 / F16 / E4M3
                           | ((MODE == 0 ? 1u : 0u) << 10)            // B: same
                           | ((uint32_t)(BN2 >> 3) << 17)       // N = 256
                           | ((uint32_t)(BM2 >> 4) << 24);      // M = 256 (two SMs)
    int s = 0;
    uint32_t ph = 0;
    int acc = 0;
    uint32_t acc_ph = 0;
    bool ok = true;
    SegIter2 it(dp_tiles, num_kb, P, pieces);
    int tile, kb0, kb1, slot;
    while (ok && it.next(tile, kb0, kb1, slot)) {
      if (!mbar_wait_bounded(&tempty[acc], acc_ph ^ 1, abort_s)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN2);
      for (int kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait_bounded(&full[s], ph, abort_s)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(sA + s * A_STAGE);
        const uint32_t b_addr = smem_u32(sB + s * B_BYTES);
#pragma unroll
        for (int k = 0; k < MMAS_PER_STAGE; ++k) {
          const uint64_t bdesc = smem_desc_sw128(b_addr + k * K_PER_MMA_BYTES);
          const uint64_t adesc = smem_desc_sw128(a_addr + k * K_PER_MMA_BYTES);
          const uint32_t accum = (kb > kb0 || k > 0) ? 1u : 0u;
          if (FP8) mma_pair_f8(d_tmem, adesc, bdesc, idesc, accum);
          else mma_pair_f16(d_tmem, adesc, bdesc, idesc, accum);
          if (LO) {
            const uint64_t ldesc = smem_desc_sw128(a_addr + A_BYTES + k * K_PER_MMA_BYTES);
            mma_pair_f8(d_tmem, ldesc, bdesc, idesc, 1u);
          }
        }
        mma_commit_pair(&empty[s]);                // frees stage s in both CTAs
        if (++s == STAGES) {
          s = 0;
          ph ^= 1;
        }
      }
      if (!ok) break;
      mma_commit_pair(&tfull[acc]);                // tile done -> both epilogues
      if (++acc == NACC) {
        acc = 0;
        acc_ph ^= 1;
      }
    }
    if (!ok) {
      atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_MMA);
      *abort_s = 1;
    }
    mma_commit_pair_local(drain);
    volatile int never = 0;
    if (!mbar_wait_bounded(drain, 0, &never)) atomicExch(&flags[FLAG_ERROR], DEV_TIMEOUT_DRAIN);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int quarter = warp & 3;
    const uint64_t upol = policy_evict_first();     // used when u_hint
    const int row_in_tile = quarter * 32 + lane;
    int acc = 0;
    uint32_t acc_ph = 0;
    SegIter2 it(dp_tiles, num_kb, P, pieces);
    int tile, kb0, kb1, slot;
    while (it.next(tile, kb0, kb1, slot)) {
      const int mt = tile / n_tiles, nt = tile - mt * n_tiles;
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
      const int p = mt * BM2 + (int)rank * HALF + row_in_tile;
      const bool prow = p < n;
      const float rs = (SCALED && prow) ? row_scale[p] : 1.0f;
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN2);
#pragma unroll 1
      for (int ch = 0; ch < BN2 / 32; ++ch) {
        uint32_t v[32];
        tmem_ld_32x32b_x32(tbase + ch * 32, v);
        tmem_ld_wait();
        const int colbase = nt * BN2 + ch * 32;
        if (slot >= 0) {
          // a K-piece: the scaled partial to its slot, [column][row] within the
          // tile (a warp stores 32 consecutive rows of one column); zero outside
          // the rows and columns of u
          float* wcol = ws + (size_t)slot * (BM2 * BN2) + (size_t)(ch * 32) * BM2 +
                        (int)rank * HALF + row_in_tile;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = colbase + j;
            float a = 0.0f;
            if (prow && col < B) {
              a = __uint_as_float(v[j]);
              if (SCALED) a = a * rs * col_scale[col];
            }
            wcol[(size_t)j * BM2] = a;
          }
        } else if (prow) {
          // the 32 old values first: loads issued together instead of one
          // load-add-store round trip per column
          double old[32];
          if (accumulate) {
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
              float a = __uint_as_float(v[j]);
              if (SCALED) a = a * rs * col_scale[col];
              const double val = f32_to_f64(a);
              double* dst = u + (size_t)col * n + p;
              if (u_hint) st_f64_hint(dst, accumulate ? old[j] + val : val, upol);
              else *dst = accumulate ? old[j] + val : val;
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive_cluster(mapa_shared(smem_u32(&tempty[acc]), 0));
      if (++acc == NACC) {
        acc = 0;
        acc_ph ^= 1;
      }
    }
  }

  // Teardown: every role of both CTAs is done (the MMA issuer drained its
  // MMAs, so no MMA still reads either CTA's shared memory), then the pair
  // releases its tensor memory together.
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  if (warp == 1) tmem_dealloc_pair(tmem_base, TMEM_COLS);
}

// u (=|+=) the sum of the P partial tiles of each tile of the K-split last
// round, in piece order.  Block (x, t): 256 consecutive rows of one column of
// tail tile t, so partial loads and u accesses are coalesced.  The partials
// are summed as a float pair with Knuth's two-sum (each step exact in its high
// part, ~2^-48 of the sum in all) and widened to FP64 with integer operations:
// two FP64 additions per element instead of 2P + 1 conversions and additions
// on GB300's narrow FP64 pipe, which bounded the first version (56 tiles of 4
// pieces: 68 us, as long as reading the partials alone).
__global__ void __launch_bounds__(256)
tail_reduce_kernel(double* __restrict__ u, const float* __restrict__ ws, int n, int B,
                   int n_tiles, int first_tile, int P, int accumulate,
                   const uint32_t* __restrict__ flags) {
  if (flags[FLAG_DONE]) return;
  const int t = (int)blockIdx.y;
  const int tile = first_tile + t;
  const int mt = tile / n_tiles, nt = tile - mt * n_tiles;
  const int e = (int)blockIdx.x * 256 + (int)threadIdx.x;   // column-in-tile * 256 + row
  const int p = mt * BM2 + (e & (BM2 - 1));
  const int col = nt * BN2 + (e >> 8);
  if (p >= n || col >= B) return;
  double* dst = u + (size_t)col * n + p;
  const double old = accumulate ? *dst : 0.0;
  const float* src = ws + (size_t)t * P * (BM2 * BN2) + e;
  float sh = 0.0f, sl = 0.0f;
#pragma unroll 4
  for (int q = 0; q < P; ++q) {
    const float x = src[(size_t)q * (BM2 * BN2)];
    const float s = __fadd_rn(sh, x);
    const float v = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(x, v));
    sh = s;
    sl = __fadd_rn(sl, err);
  }
  const double sum = f32_to_f64(sh) + f32_to_f64(sl);
  *dst = accumulate ? old + sum : sum;
}

}  // namespace

pide_status launch_tail_reduce(pide_ctx* c, cudaStream_t st) {
  if (!c->tail.pending) return PIDE_OK;
  const pide_ctx::TailReduce t = c->tail;
  c->tail.pending = false;
  ProfScope ps(c, st, 4);
  tail_reduce_kernel<<<dim3(BM2 * BN2 / 256, t.tiles), 256, 0, st>>>(
      t.u, c->tail_ws, c->n, t.B, t.n_tiles, t.first_tile, t.P, t.accumulate, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

template <int STAGES, int MODE, int NACC>
static pide_status launch_tc2(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                              int col0, bool corr) {
  constexpr int A_STAGE = (MODE == 2 ? 2 : 1) * HALF * ROW_BYTES2;
  constexpr int B_BYTES = HALF * ROW_BYTES2;
  const size_t smem = 1024 + (size_t)STAGES * (A_STAGE + B_BYTES) + 256;
  PIDE_TRY(corr ? make_tma_rhs_corr(c, HALF) : make_tma_rhs(c, HALF));
  auto kern = gemm_tc2_kernel<STAGES, MODE, NACC>;
  PIDE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (c->max_pairs <= 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (c->num_sms / 2), 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = smem;
    int nc = 0;
    PIDE_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nc, (void*)kern, &cfg));
    c->max_pairs = nc > 0 ? nc : 1;
  }
  const int G = c->max_pairs;                               // clusters resident at once
  const int m_tiles = (c->n + BM2 - 1) / BM2;
  const int n_tiles = (B + BN2 - 1) / BN2;
  const int tiles = m_tiles * n_tiles;
  constexpr int KE = (MODE == 1 || MODE == 2) ? 128 : 64;   // K elements per stage
  const int num_kb = (c->n + KE - 1) / KE;
  // Whole rounds of tiles, then the last round's r tiles cut along K into P
  // pieces each (at least 8 k-blocks), dealt round-robin to the G pairs: the
  // round then takes ceil(r P / G) / P of a tile's time instead of one, and the
  // reduction of the r P partial tiles about as long as half a k-block each
  // (measured: 8 x 9 partials in 11 us, 56 x 4 in 37 us, against 0.34 us per
  // k-block of 64).  P minimises the sum (the smallest P within 1 % of a tile
  // of the best); no split unless it saves 5 % of a tile.  At 198^2, B = 1024:
  // r = 8 of G = 76, P = 8.  With gemm_streamk = 2 the reduction's cost is left
  // out (any split that shortens the round by 1 % is taken).
  const int full = tiles / G, rest = tiles - full * G;
  int P = 0;
  if (c->gemm_streamk && rest > 0 && c->tail_ws) {
    int pmax = num_kb / 8;
    if (pmax > c->tail_slots / rest) pmax = c->tail_slots / rest;
    const double per_partial = c->gemm_streamk == 2 ? 0.0 : 0.5;
    auto cost = [&](int p) {
      return (double)((rest * p + G - 1) / G) / p + per_partial * rest * p / num_kb;
    };
    double best = 1.0;
    for (int p = 2; p <= pmax; ++p) best = cost(p) < best ? cost(p) : best;
    if (best < (c->gemm_streamk == 2 ? 0.99 : 0.95))
      for (int p = 2; p <= pmax; ++p)
        if (cost(p) <= best + 0.01) {
          P = p;
          break;
        }
  }
  const int clusters = P ? G : (tiles < G ? tiles : G);
  const int dp_tiles = P ? full * G : tiles;
  const int pieces = P ? rest * P : 0;
  // the correction term: e4m3 C against Rc, scales s_p (rows) and t_j (columns)
  const CUtensorMap& A = corr ? c->tmA_corr : c->tmA;
  const CUtensorMap& Alo = corr ? c->tmA_corr : c->tmA_lo;
  const CUtensorMap& R = corr ? c->tmRc : c->tmR;
  const float* rs = corr ? c->corr_scale : c->row_scale;
  const float* cs = corr ? c->col_scale_c + col0 : (MODE != 0 ? c->col_scale + col0 : nullptr);
  kern<<<2 * clusters, 192, smem, st>>>(A, Alo, R, c->n, B, col0, num_kb, dp_tiles, P, pieces,
                                        u, accumulate ? 1 : 0, rs, cs, c->tail_ws, c->flags,
                                        c->gemm_a_hint, c->gemm_u_hint);
  PIDE_CUDA_TRY(cudaGetLastError());
  if (P) {
    c->tail.pending = true;
    c->tail.u = u;
    c->tail.B = B;
    c->tail.n_tiles = n_tiles;
    c->tail.first_tile = dp_tiles;
    c->tail.tiles = rest;
    c->tail.P = P;
    c->tail.accumulate = accumulate ? 1 : 0;
  }
  return PIDE_OK;
}

// B > 128 on pairs of SMs (256 x 256 tiles); stages fill ~200 KB per SM.
pide_status launch_gemm_tc2(pide_ctx* c, int B, double* u, bool accumulate, cudaStream_t st,
                            int col0, bool corr) {
  if (!c->tmA_ok) {
    set_error("tensor-core apply: TMA maps were not created");
    return PIDE_EUNSUPPORTED;
  }
  if (corr) return launch_tc2<6, 1, TC2_NACC>(c, B, u, true, st, col0, true);
  switch (c->prec) {
    case PIDE_BF16: return launch_tc2<6, 0, TC2_NACC>(c, B, u, accumulate, st, col0, false);
    case PIDE_FP8: return launch_tc2<6, 1, TC2_NACC>(c, B, u, accumulate, st, col0, false);
    case PIDE_FP8X2: return launch_tc2<4, 2, TC2_NACC>(c, B, u, accumulate, st, col0, false);
    case PIDE_FP16: return launch_tc2<6, 3, TC2_NACC>(c, B, u, accumulate, st, col0, false);
    default: return PIDE_EUNSUPPORTED;
  }
}

}  // namespace pide
