// Step 2 ("using any standard matrix inversion method"): the dense inverse of
// the symmetric conservative operator S = D L, formed in FP64 on the GPU.
//
// S is block tridiagonal over the slowest grid index: on a 2-D grid the m =
// ny-2 blocks are grid rows (k = nx-2 nodes, A_a tridiagonal: d on the
// diagonal, -eps of the x faces beside it), on a 3-D grid the m = nz-2 blocks
// are z-planes (k = (nx-2)(ny-2) nodes, A_a the in-plane 5-point operator:
// -eps of the x faces at distance 1 within a row, of the y faces at distance
// nx-2).  The couplings S_{a,a+1} = -diag(eps of the faces between blocks a and
// a+1) are diagonal in both cases (y faces in 2-D, z faces in 3-D).
// Block elimination from both ends gives the whole inverse G = S^-1:
//   backward Schur complements  Sg_{m-1} = A_{m-1},
//                               Sg_a = A_a - C_a Sg_{a+1}^-1 C_a      (C_a = faces to block a+1)
//   forward Schur complements   Df_0 = A_0,
//                               Df_a = A_a - C_{a-1} Df_{a-1}^-1 C_{a-1}
//   diagonal blocks             G_aa = (A_a - C_{a-1} Df_{a-1}^-1 C_{a-1} - C_a Sg_{a+1}^-1 C_a)^-1
//   blocks below the diagonal   G_{a,j} = M_a G_{a-1,j},  M_a = Sg_a^-1 C_{a-1}   (a > j)
//   blocks above                G_{j,a} = G_{a,j}^T        (S symmetric)
// The two chains are sequences of k x k inversions (one CTA each, run side by
// side); the diagonal blocks are m independent inversions; the rest is a
// wavefront of batched k x k x k FP64 GEMMs, O(n^2 k) flops in total instead
// of O(n^3) for dense LU.  Finally L^-1 = G D (Eq. 3's rows are D^-1 S).
#include "common.cuh"

namespace pide {

namespace {

// In-place Gauss-Jordan inversion of a k x k SPD matrix (no pivoting needed:
// every pivot of an SPD matrix is positive).  All threads of the block take part.
__device__ void gj_invert(double* A, int k, size_t lda, double* s_row, double* s_col,
                          double* s_rp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int piv = 0; piv < k; ++piv) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      s_row[t] = A[(size_t)piv * lda + t];
      s_col[t] = A[(size_t)t * lda + piv];
    }
    __syncthreads();
    const double pinv = 1.0 / s_row[piv];
    for (int t = threadIdx.x; t < k; t += blockDim.x) s_rp[t] = s_row[t] * pinv;
    __syncthreads();
    for (int i = warp; i < k; i += nw) {
      const double ci = s_col[i];
      double* row = A + (size_t)i * lda;
      if (i == piv) {
        for (int j = lane; j < k; j += 32) row[j] = (j == piv) ? pinv : s_rp[j];
      } else {
        for (int j = lane; j < k; j += 32) row[j] = (j == piv) ? -ci * pinv : fma(-ci, s_rp[j], row[j]);
      }
    }
    __syncthreads();
  }
}

// The block structure: k nodes per block, m blocks, rows of mxb nodes inside
// a block when the block is a 3-D plane (mxb = 0: the block is one 2-D row),
// face arrays of the in-block neighbours and of the couplings to the next and
// the previous block.
struct BlockOp {
  const double* cf;   // face eps, structure of arrays: W, E, S, N (, D, U)
  const double* d;
  int n, k, m, mxb;
  int f_next, f_prev;  // face array index of the coupling to block a+1 / a-1
};

__device__ __forceinline__ double block_A(const BlockOp& op, int a, int r, int c) {
  const int p = a * op.k + r;
  const size_t n = (size_t)op.n;
  if (r == c) return op.d[p];
  if (op.mxb == 0) {                        // 2-D: tridiagonal grid row
    if (c == r + 1) return -op.cf[n + p];   // east face of (a, r)
    if (c == r - 1) return -op.cf[p];       // west face of (a, r)
    return 0.0;
  }
  const int x = r % op.mxb;                 // 3-D: 5-point plane operator
  if (c == r + 1 && x < op.mxb - 1) return -op.cf[n + p];
  if (c == r - 1 && x > 0) return -op.cf[p];
  if (c == r + op.mxb) return -op.cf[3 * n + p];
  if (c == r - op.mxb) return -op.cf[2 * n + p];
  return 0.0;
}

// blockIdx.x == 0: backward chain into Gb[a] = Sg_a^-1; == 1: forward chain into Gf[a] = Df_a^-1.
__global__ void __launch_bounds__(1024) chain_kernel(BlockOp op, double* __restrict__ Gb,
                                                     double* __restrict__ Gf) {
  extern __shared__ double sh[];
  const int k = op.k, m = op.m;
  double* s_row = sh;
  double* s_col = sh + k;
  double* s_rp = sh + 2 * k;
  const size_t n = (size_t)op.n;
  const bool backward = (blockIdx.x == 0);
  const size_t kk = (size_t)k * k;
  for (int step = 0; step < m; ++step) {
    const int a = backward ? (m - 1 - step) : step;
    double* T = (backward ? Gb : Gf) + (size_t)a * kk;
    const bool has_prev = backward ? (a < m - 1) : (a > 0);
    const double* P = has_prev ? ((backward ? Gb : Gf) + (size_t)(backward ? a + 1 : a - 1) * kk) : nullptr;
    // coupling faces: backward to block a+1, forward to block a-1
    const double* C = op.cf + (size_t)(backward ? op.f_next : op.f_prev) * n + (size_t)a * k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int r = e / k, c = e - r * k;
      double v = block_A(op, a, r, c);
      if (has_prev) v -= C[r] * P[e] * C[c];
      T[e] = v;
    }
    __syncthreads();
    gj_invert(T, k, k, s_row, s_col, s_rp);
  }
}

// Diagonal blocks of the inverse, one CTA per block row a, written in place
// into G at block (a, a).
__global__ void __launch_bounds__(1024) diag_kernel(BlockOp op, const double* __restrict__ Gb,
                                                    const double* __restrict__ Gf,
                                                    double* __restrict__ G, size_t ld) {
  extern __shared__ double sh[];
  const int a = blockIdx.x;
  const int k = op.k, m = op.m;
  const size_t n = (size_t)op.n;
  const size_t kk = (size_t)k * k;
  double* T = G + (size_t)a * k * ld + (size_t)a * k;
  const double* Cs = op.cf + (size_t)op.f_prev * n + (size_t)a * k;
  const double* Cn = op.cf + (size_t)op.f_next * n + (size_t)a * k;
  const double* Pf = (a > 0) ? Gf + (size_t)(a - 1) * kk : nullptr;
  const double* Pb = (a < m - 1) ? Gb + (size_t)(a + 1) * kk : nullptr;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int r = e / k, c = e - r * k;
    double v = block_A(op, a, r, c);
    if (Pf) v -= Cs[r] * Pf[e] * Cs[c];
    if (Pb) v -= Cn[r] * Pb[e] * Cn[c];
    T[(size_t)r * ld + c] = v;
  }
  __syncthreads();
  gj_invert(T, k, ld, sh, sh + k, sh + 2 * k);
}

// M_a = Sg_a^-1 diag(faces of block a to block a-1) for a >= 1, in place over Gb[a].
__global__ void mscale_kernel(BlockOp op, double* __restrict__ Gb) {
  const int k = op.k, m = op.m;
  const size_t kk = (size_t)k * k;
  const size_t total = (size_t)(m - 1) * kk;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int a = 1 + (int)(e / kk);
    const int c = (int)((e % kk) % k);
    Gb[kk + e] *= op.cf[(size_t)op.f_prev * op.n + (size_t)a * k + c];
  }
}

// One wavefront step s: for every j with a = j + s < m, G(a, j) = M_a G(a-1, j).
// 64 x 64 output tile per CTA, 256 threads with 4 x 4 results each, K in steps of 16.
__global__ void __launch_bounds__(256) wave_dgemm(const double* __restrict__ Mw,
                                                  double* __restrict__ G, size_t ld, int k,
                                                  int s) {
  __shared__ double As[16][65];
  __shared__ double Xs[16][65];
  const int j = blockIdx.z, a = j + s;
  const double* A = Mw + (size_t)a * k * k;
  const double* X = G + (size_t)(a - 1) * k * ld + (size_t)j * k;
  double* C = G + (size_t)a * k * ld + (size_t)j * k;
  const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.0;
  for (int k0 = 0; k0 < k; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int r = e >> 4, kk = e & 15;
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < k && gk < k) ? A[(size_t)gr * k + gk] : 0.0;
      const int kk2 = e >> 6, cc = e & 63;
      const int gk2 = k0 + kk2, gc = col0 + cc;
      Xs[kk2][cc] = (gk2 < k && gc < k) ? X[(size_t)gk2 * ld + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], xv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = Xs[kk][tx + 16 * q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = fma(av[i], xv[q], acc[i][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= k) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = col0 + tx + 16 * q;
      if (c < k) C[(size_t)r * ld + c] = acc[i][q];
    }
  }
}

// L^-1 = S^-1 D: scale column q by d_q (the stored inverse is that of Eq. 3's rows).
__global__ void colscale_kernel(double* __restrict__ G, size_t ld, int n,
                                const double* __restrict__ d) {
  const size_t total = (size_t)n * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % ld);
    if (q < n) G[e] *= d[q];
  }
}

// Upper blocks from the lower ones: G[p][q] = G[q][p] when block(p) < block(q).
__global__ void mirror_kernel(double* __restrict__ G, size_t ld, int n, int k) {
  __shared__ double t[32][33];
  const int tr = blockIdx.y * 32, tc = blockIdx.x * 32;   // destination tile (rows tr.., cols tc..)
  if ((tr + 31) / k >= tc / k && tr / k >= (tc + 31) / k) return;  // no element strictly above
  // load the source tile: rows tc.., cols tr.. (transposed position)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int sr = tc + r, sc = tr + threadIdx.x;
    t[r][threadIdx.x] = (sr < n && sc < n) ? G[(size_t)sr * ld + sc] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int dr = tr + r, dc = tc + threadIdx.x;
    if (dr < n && dc < n && dr / k < dc / k) G[(size_t)dr * ld + dc] = t[threadIdx.x][r];
  }
}

}  // namespace

pide_status build_inverse_fp64(pide_ctx* c, double* G, cudaStream_t st) {
  const bool three = c->dims == 3;
  const int k = three ? c->mx * c->my : c->mx, m = three ? c->mz : c->my;
  const BlockOp op{c->cf, c->d, c->n, k, m, three ? c->mx : 0, three ? 5 : 3, three ? 4 : 2};
  const size_t kk = (size_t)k * k;
  double* work = nullptr;
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&work, 2 * (size_t)m * kk * sizeof(double), st));
  double* Gb = work;
  double* Gf = work + (size_t)m * kk;
  const size_t shm = 3 * (size_t)k * sizeof(double);
  if (shm > 48 * 1024) {
    PIDE_CUDA_TRY(cudaFuncSetAttribute(chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    PIDE_CUDA_TRY(cudaFuncSetAttribute(diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  }
  chain_kernel<<<2, 1024, shm, st>>>(op, Gb, Gf);
  PIDE_CUDA_TRY(cudaGetLastError());
  diag_kernel<<<m, 1024, shm, st>>>(op, Gb, Gf, G, (size_t)c->ld);
  PIDE_CUDA_TRY(cudaGetLastError());
  if (m > 1) {
    mscale_kernel<<<c->num_sms * 4, 256, 0, st>>>(op, Gb);
    PIDE_CUDA_TRY(cudaGetLastError());
    const int tiles = (k + 63) / 64;
    for (int s = 1; s < m; ++s) {
      dim3 grid(tiles, tiles, m - s);
      wave_dgemm<<<grid, 256, 0, st>>>(Gb, G, (size_t)c->ld, k, s);
      PIDE_CUDA_TRY(cudaGetLastError());
    }
    dim3 mg((c->n + 31) / 32, (c->n + 31) / 32);
    mirror_kernel<<<mg, dim3(32, 8), 0, st>>>(G, (size_t)c->ld, c->n, k);
    PIDE_CUDA_TRY(cudaGetLastError());
  }
  colscale_kernel<<<c->num_sms * 8, 256, 0, st>>>(G, (size_t)c->ld, c->n, c->d);
  PIDE_CUDA_TRY(cudaGetLastError());
  PIDE_CUDA_TRY(cudaFreeAsync(work, st));
  return PIDE_OK;
}

}  // namespace pide
