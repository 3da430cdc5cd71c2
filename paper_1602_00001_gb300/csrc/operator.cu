// Operator kernels: assembly of the 5-point system (Eq. 2/3), right-hand
// side preparation, the FP64 stencil residual, and the adjoint face gradient.
//
// Layout: interior node p = a*mx + c (a = i-1, c = j-1, j fastest, the order of
// Fig. 3 restricted to the interior).  cf holds four face permittivities per
// node, structure of arrays: cf[0*n+p] west (j-1), cf[1*n+p] east (j+1),
// cf[2*n+p] south (i-1), cf[3*n+p] north (i+1).  d[p] = their sum, so that
// S = D - (off-diagonal face terms) is symmetric and L = D^-1 S is the row of
// Eq. (3): u_p - sum_q w_pq u_q with w = cf / d (stored in w, same layout).
// The stored inverse is L^-1 itself, so every right-hand side is in the
// Eq. (3) form and the residual is r = b - u + sum_q w_pq u_q.
#include "common.cuh"

namespace pide {

namespace {

__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

// Step 1 (assembly): face eps by harmonic mean of the two node values, d = sum.
__global__ void assemble_kernel(const double* __restrict__ eps, int nx, int ny,
                                double* __restrict__ cf, double* __restrict__ d,
                                double* __restrict__ w4, double* __restrict__ dinv) {
  const int mx = nx - 2, my = ny - 2, n = mx * my;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int a = p / mx, c = p - a * mx;
    const int i = a + 1, j = c + 1;
    const double e0 = eps[i * nx + j];
    const double w = harmonic(e0, eps[i * nx + j - 1]);
    const double e = harmonic(e0, eps[i * nx + j + 1]);
    const double s = harmonic(e0, eps[(i - 1) * nx + j]);
    const double no = harmonic(e0, eps[(i + 1) * nx + j]);
    cf[p] = w;
    cf[n + p] = e;
    cf[2 * n + p] = s;
    cf[3 * n + p] = no;
    const double dp = w + e + s + no;
    d[p] = dp;
    dinv[p] = 1.0 / dp;
    w4[p] = w / dp;
    w4[n + p] = e / dp;
    w4[2 * n + p] = s / dp;
    w4[3 * n + p] = no / dp;
  }
}

// The same on an nx x ny x nz node grid (the 7-point flux form): six faces per
// interior node p = (z*my + y)*mx + x, in the order W, E, S, N, D, U.
__global__ void assemble3d_kernel(const double* __restrict__ eps, int nx, int ny, int nz,
                                  double* __restrict__ cf, double* __restrict__ d,
                                  double* __restrict__ w6, double* __restrict__ dinv) {
  const int mx = nx - 2, my = ny - 2, mz = nz - 2;
  const int n = mx * my * mz;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int x = p % mx, y = (p / mx) % my, z = p / (mx * my);
    const size_t sx = 1, sy = nx, sz = (size_t)nx * ny;
    const size_t q = (size_t)(z + 1) * sz + (size_t)(y + 1) * sy + (x + 1);
    const double e0 = eps[q];
    const double f[6] = {harmonic(e0, eps[q - sx]), harmonic(e0, eps[q + sx]),
                         harmonic(e0, eps[q - sy]), harmonic(e0, eps[q + sy]),
                         harmonic(e0, eps[q - sz]), harmonic(e0, eps[q + sz])};
    double dp = 0.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      cf[(size_t)k * n + p] = f[k];
      dp += f[k];
    }
    d[p] = dp;
    dinv[p] = 1.0 / dp;
#pragma unroll
    for (int k = 0; k < 6; ++k) w6[(size_t)k * n + p] = f[k] / dp;
  }
}

// 3-D lift: lift_p = sum over boundary neighbours q of w_pq g_q, g = [nz][ny][nx].
__global__ void lift3d_kernel(const double* __restrict__ g, const double* __restrict__ w6, int nx,
                              int ny, int nz, double* __restrict__ lift) {
  const int mx = nx - 2, my = ny - 2, mz = nz - 2;
  const int n = mx * my * mz;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int x = p % mx, y = (p / mx) % my, z = p / (mx * my);
    const size_t sy = nx, sz = (size_t)nx * ny;
    const size_t q = (size_t)(z + 1) * sz + (size_t)(y + 1) * sy + (x + 1);
    double s = 0.0;
    if (x == 0) s += w6[p] * g[q - 1];
    if (x == mx - 1) s += w6[(size_t)n + p] * g[q + 1];
    if (y == 0) s += w6[2 * (size_t)n + p] * g[q - sy];
    if (y == my - 1) s += w6[3 * (size_t)n + p] * g[q + sy];
    if (z == 0) s += w6[4 * (size_t)n + p] * g[q - sz];
    if (z == mz - 1) s += w6[5 * (size_t)n + p] * g[q + sz];
    lift[p] = s;
  }
}

// b = -h^2 rho / d  (flux form of Eq. 1 divided by the node's total face eps)
__global__ void rhs_from_charge_kernel(const double* __restrict__ rho, double* __restrict__ b,
                                       const double* __restrict__ d, int n, long long total,
                                       double h2) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(k % n);
    b[k] = -h2 * rho[k] / d[p];   // one division per entry; not on the refined path
  }
}

// lift_p = sum over boundary neighbours q of w_pq g_q  (Fig. 3's boundary
// columns moved to the right side of Eq. 3)
__global__ void lift_kernel(const double* __restrict__ g, const double* __restrict__ cf, int nx,
                            int ny, double* __restrict__ lift) {
  const int mx = nx - 2, my = ny - 2, n = mx * my;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int a = p / mx, c = p - a * mx;
    const int i = a + 1, j = c + 1;
    double s = 0.0;
    if (c == 0) s += cf[p] * g[i * nx + j - 1];
    if (c == mx - 1) s += cf[n + p] * g[i * nx + j + 1];
    if (a == 0) s += cf[2 * n + p] * g[(i - 1) * nx + j];
    if (a == my - 1) s += cf[3 * n + p] * g[(i + 1) * nx + j];
    lift[p] = s;
  }
}

template <int RF>
__device__ __forceinline__ void store_rhs(void* R, size_t idx, double v, float inv_scale) {
  if constexpr (RF == RF_F64) {
    reinterpret_cast<double*>(R)[idx] = v;
  } else if constexpr (RF == RF_F32) {
    reinterpret_cast<float*>(R)[idx] = (float)v;
  } else if constexpr (RF == RF_BF16) {
    reinterpret_cast<__nv_bfloat16*>(R)[idx] = __double2bfloat16(v);
  } else if constexpr (RF == RF_F16) {
    // in units of the column's power-of-two scale, saturating at 65504
    const float x = fminf(fmaxf((float)(v * (double)inv_scale), -65504.0f), 65504.0f);
    reinterpret_cast<__half*>(R)[idx] = __float2half_rn(x);
  } else {
    reinterpret_cast<__nv_fp8_e4m3*>(R)[idx] = __nv_fp8_e4m3((float)(v * (double)inv_scale));
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// Prep: the right-hand side the stored L^-1 is applied to,
//   mode 0 (forward):  f = b + lift           (Eq. 3 right side)
//   mode 1 (adjoint):  f = g / d              (S mu = g  <=>  L mu = D^-1 g)
// R[col][p] = q(f); optionally colmax_b[col] = max_p |f_p|.
template <int RF>
__global__ void prep_kernel(const double* __restrict__ b, int n, int ldr, int mode,
                            const double* __restrict__ dinv, const double* __restrict__ lift,
                            void* __restrict__ R, const float* __restrict__ col_scale,
                            double* __restrict__ colmax_b, int track) {
  __shared__ double red[32];
  const int col = blockIdx.y;
  const double* bc = b + (size_t)col * n;
  const float isc = col_scale ? 1.0f / col_scale[col] : 1.0f;
  double mx = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double f = bc[p];
    if (mode == 1) f *= dinv[p];
    else if (lift) f += lift[p];
    store_rhs<RF>(R, (size_t)col * ldr + p, f, isc);
    if (track) mx = fmax(mx, fabs(f));
  }
  if (track) {
    mx = block_max(mx, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&colmax_b[col], mx);
  }
}

// Residual of Eq. (3), FP64, five FP64 operations per node:
//   r = f - L u = f - u_p + sum_q w_pq u_q   (interior neighbours q only)
// with f as in prep.  Written quantised to R (the next apply's right side),
// optionally in full to r_out, and its column max |r| into colmax_r.
template <int RF, bool DIM3>
__global__ void residual_kernel(const double* __restrict__ b, const double* __restrict__ u,
                                int n, int mx, int plane, int ldr, int mode,
                                const double* __restrict__ w4,
                                const double* __restrict__ dinv, const double* __restrict__ lift,
                                void* __restrict__ R, const float* __restrict__ col_scale,
                                double* __restrict__ r_out, double* __restrict__ colmax_r,
                                int track, const uint32_t* __restrict__ flags) {
  __shared__ double red[32];
  if (flags && flags[FLAG_DONE]) return;
  const int col = blockIdx.y;
  const double* uc = u + (size_t)col * n;
  const double* bc = b + (size_t)col * n;
  const float isc = col_scale ? 1.0f / col_scale[col] : 1.0f;
  double mxr = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int c = p % mx;
    const int pp = DIM3 ? p % plane : p;   // index inside a z-plane (2-D: the whole grid)
    double r;
    if (mode == 1) r = fma(bc[p], dinv[p], -uc[p]);
    else if (lift) r = bc[p] + (lift[p] - uc[p]);
    else r = bc[p] - uc[p];
    if (c > 0) r = fma(w4[p], uc[p - 1], r);
    if (c < mx - 1) r = fma(w4[n + p], uc[p + 1], r);
    if (pp >= mx) r = fma(w4[2 * n + p], uc[p - mx], r);
    if (pp + mx < plane) r = fma(w4[3 * n + p], uc[p + mx], r);
    if (DIM3) {
      if (p >= plane) r = fma(w4[4 * (size_t)n + p], uc[p - plane], r);
      if (p + plane < n) r = fma(w4[5 * (size_t)n + p], uc[p + plane], r);
    }
    if (R) store_rhs<RF>(R, (size_t)col * ldr + p, r, isc);
    if (r_out) r_out[(size_t)col * n + p] = r;
    if (track) mxr = fmax(mxr, fabs(r));
  }
  if (track) {
    mxr = block_max(mxr, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&colmax_r[col], mxr);
  }
}

// The same residual over a flat index (column * n + p) with a small persistent
// grid: used under a concurrently running tensor-core apply, where a full-size
// grid would crowd the SMs' warp schedulers that the GEMM's single-thread TMA
// and MMA issuers depend on.
template <int RF, bool DIM3>
__global__ void residual_flat_kernel(const double* __restrict__ b, const double* __restrict__ u,
                                     int n, int mx, int plane, int B, int ldr, int mode,
                                     const double* __restrict__ w4,
                                     const double* __restrict__ dinv,
                                     const double* __restrict__ lift, void* __restrict__ R,
                                     const float* __restrict__ col_scale,
                                     const uint32_t* __restrict__ flags) {
  if (flags && flags[FLAG_DONE]) return;
  const long long total = (long long)B * n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(k / n);
    const int p = (int)(k - (long long)col * n);
    const int c = p % mx;
    const int pp = DIM3 ? p % plane : p;
    const double* uc = u + (size_t)col * n;
    // streaming loads (evict-first): keep the concurrent GEMM's operands in L2
    const double bp = __ldcs(b + k);
    const double up = __ldcs(uc + p);
    double r;
    if (mode == 1) r = fma(bp, dinv[p], -up);
    else if (lift) r = bp + (lift[p] - up);
    else r = bp - up;
    if (c > 0) r = fma(w4[p], __ldcs(uc + p - 1), r);
    if (c < mx - 1) r = fma(w4[n + p], __ldcs(uc + p + 1), r);
    if (pp >= mx) r = fma(w4[2 * n + p], __ldcs(uc + p - mx), r);
    if (pp + mx < plane) r = fma(w4[3 * n + p], __ldcs(uc + p + mx), r);
    if (DIM3) {
      if (p >= plane) r = fma(w4[4 * (size_t)n + p], __ldcs(uc + p - plane), r);
      if (p + plane < n) r = fma(w4[5 * (size_t)n + p], __ldcs(uc + p + plane), r);
    }
    const float isc = col_scale ? 1.0f / col_scale[col] : 1.0f;
    store_rhs<RF>(R, (size_t)col * ldr + p, r, isc);
  }
}

// Convergence check between sweeps: done once every column satisfies
// max|r| <= tol * max|f/d|.  Resets the residual maxima for the next sweep.
__global__ void check_kernel(double* colmax, const double* colmax_b, int B, double tol,
                             uint32_t* flags) {
  __shared__ int bad;
  if (flags[FLAG_DONE]) return;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < B; c += blockDim.x) {
    if (colmax[c] > tol * colmax_b[c]) bad = 1;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < B; c += blockDim.x) colmax[c] = 0.0;
  if (threadIdx.x == 0) {
    if (!bad) flags[FLAG_DONE] = 1;
    else flags[FLAG_SWEEPS] += 1;
  }
}

// Refinement record: *slot = max over columns of max|r_c| / max|f_c| for the
// residual the last tracked launch wrote into colmax (a zero column counts its
// absolute residual); reset: clear colmax for the next sweep.
__global__ void record_kernel(double* colmax, const double* colmax_b, int B, double* slot,
                              int reset, const uint32_t* flags) {
  __shared__ double red[32];
  if (flags[FLAG_DONE]) return;
  double worst = 0.0;
  for (int c = threadIdx.x; c < B; c += blockDim.x) {
    const double den = colmax_b[c];
    worst = fmax(worst, den > 0.0 ? colmax[c] / den : colmax[c]);
  }
  worst = block_max(worst, red);
  if (threadIdx.x == 0) *slot = worst;
  if (reset) {
    __syncthreads();
    for (int c = threadIdx.x; c < B; c += blockDim.x) colmax[c] = 0.0;
  }
}

// Column maxima of |f| (the prep right side) without writing R.
__global__ void colmax_b_kernel(const double* __restrict__ b, int n, int mode,
                                const double* __restrict__ dinv, const double* __restrict__ lift,
                                double* __restrict__ colmax_b) {
  __shared__ double red[32];
  const int col = blockIdx.y;
  const double* bc = b + (size_t)col * n;
  double mx = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double f = bc[p];
    if (mode == 1) f *= dinv[p];
    else if (lift) f += lift[p];
    mx = fmax(mx, fabs(f));
  }
  mx = block_max(mx, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&colmax_b[col], mx);
}

// Adjoint, per node a of the grid: dLoss/deps_a = sum over the node's faces f
// (to node b) of T_f * 2 eps_b^2 / (eps_a + eps_b)^2, where
//   T_f = sum_cols mu_p b_p + mu_q b_q - (mu_p - mu_q)(u_p - u_q)
// and a boundary endpoint contributes mu = 0, no b term and u = 0.
//
// Two passes.  face_t_kernel forms T_f once per face -- the faces toward the
// +x, +y (and +z) neighbour of every node -- in a block of 32 consecutive
// nodes (coalesced loads of mu, u and b) by FG_GROUPS column groups whose
// partial sums are added in group order through shared memory.
// face_combine_kernel then gives each node the sum over its faces in the
// order -x, +x, -y, +y (-z, +z).  Both are deterministic.  The first version
// (one thread per node looping over all B columns of its faces, every face
// formed twice) took 88 us for a 128^2 grid at B = 32 on GB300's FP64 pipe.
constexpr int FG_GROUPS = 8;

template <int DIMS>
__global__ void __launch_bounds__(32 * FG_GROUPS)
face_t_kernel(const double* __restrict__ mu, const double* __restrict__ u,
              const double* __restrict__ b, int nx, int ny, int nz, int B,
              double* __restrict__ Tf) {
  __shared__ double part[FG_GROUPS][32];
  const int mx = nx - 2, my = ny - 2, mz = DIMS == 3 ? nz - 2 : 1;
  const int n = mx * my * mz;
  const int nzz = DIMS == 3 ? nz : 1;
  const int N = nx * ny * nzz;
  const int node = (int)blockIdx.x * 32 + (int)threadIdx.x;
  const int g = (int)threadIdx.y;
  const int j = node % nx, i = (node / nx) % ny, l = DIMS == 3 ? node / (nx * ny) : 0;
  const bool valid = node < N;
  const bool in_a = valid && (DIMS != 3 || (l > 0 && l < nz - 1)) && i > 0 && i < ny - 1 &&
                    j > 0 && j < nx - 1;
  const int pa = in_a ? ((DIMS == 3 ? (l - 1) * my : 0) + (i - 1)) * mx + (j - 1) : -1;
#pragma unroll
  for (int d = 0; d < DIMS; ++d) {
    const int j2 = j + (d == 0), i2 = i + (d == 1), l2 = l + (d == 2);
    const bool exists = valid && j2 < nx && i2 < ny && l2 < nzz;
    const bool in_b = exists && (DIMS != 3 || (l2 > 0 && l2 < nz - 1)) && i2 > 0 &&
                      i2 < ny - 1 && j2 > 0 && j2 < nx - 1;
    double T = 0.0;
    if (in_a || in_b) {
      const int pb = in_b ? ((DIMS == 3 ? (l2 - 1) * my : 0) + (i2 - 1)) * mx + (j2 - 1) : -1;
      for (int c = g; c < B; c += FG_GROUPS) {
        const size_t o = (size_t)c * n;
        const double mua = in_a ? mu[o + pa] : 0.0, mub = in_b ? mu[o + pb] : 0.0;
        const double ua = in_a ? u[o + pa] : 0.0, ub = in_b ? u[o + pb] : 0.0;
        const double ba = in_a ? b[o + pa] : 0.0, bb = in_b ? b[o + pb] : 0.0;
        T += mua * ba + mub * bb - (mua - mub) * (ua - ub);
      }
    }
    part[g][threadIdx.x] = T;
    __syncthreads();
    if (g == 0 && valid) {
      double sum = part[0][threadIdx.x];
#pragma unroll
      for (int q = 1; q < FG_GROUPS; ++q) sum += part[q][threadIdx.x];
      Tf[(size_t)d * N + node] = sum;
    }
    __syncthreads();
  }
}

template <int DIMS>
__global__ void face_combine_kernel(const double* __restrict__ Tf, const double* __restrict__ eps,
                                    int nx, int ny, int nz, double* __restrict__ deps) {
  const int nzz = DIMS == 3 ? nz : 1;
  const int N = nx * ny * nzz;
  const int plane = nx * ny;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N;
       node += gridDim.x * blockDim.x) {
    const int j = node % nx, i = (node / nx) % ny, l = DIMS == 3 ? node / plane : 0;
    const double ea = eps[node];
    double acc = 0.0;
    // faces -x, +x, -y, +y, -z, +z: T_f is stored at the face's lower node
    const int step[3] = {1, nx, plane};
    const int coord[3] = {j, i, l}, extent[3] = {nx, ny, nzz};
#pragma unroll
    for (int k = 0; k < 2 * DIMS; ++k) {
      const int d = k >> 1;
      const bool up = k & 1;
      if (up ? coord[d] + 1 >= extent[d] : coord[d] == 0) continue;
      const int other = up ? node + step[d] : node - step[d];
      const double T = Tf[(size_t)d * N + (up ? node : other)];
      const double eb = eps[other];
      acc += T * 2.0 * eb * eb / ((ea + eb) * (ea + eb));
    }
    deps[node] += acc;
  }
}

__global__ void scale_d_kernel(const double* __restrict__ mu, const double* __restrict__ d,
                               double* __restrict__ out, int n, long long total) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = mu[k] * d[k % n];
}

inline int grid_for(long long work, int block, int num_sms) {
  long long g = (work + block - 1) / block;
  long long cap = (long long)num_sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

pide_status launch_assemble(pide_ctx* c, cudaStream_t st) {
  if (c->dims == 3)
    assemble3d_kernel<<<grid_for(c->n, 256, c->num_sms), 256, 0, st>>>(c->eps, c->nx, c->ny, c->nz,
                                                                        c->cf, c->d, c->w, c->dinv);
  else
    assemble_kernel<<<grid_for(c->n, 256, c->num_sms), 256, 0, st>>>(c->eps, c->nx, c->ny, c->cf,
                                                                      c->d, c->w, c->dinv);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_rhs_from_charge(pide_ctx* c, const double* rho, double* b, int B,
                                   cudaStream_t st) {
  const long long total = (long long)B * c->n;
  if (total == 0) return PIDE_OK;
  ProfScope ps(c, st, 2);
  rhs_from_charge_kernel<<<grid_for(total, 256, c->num_sms), 256, 0, st>>>(rho, b, c->d, c->n,
                                                                          total, c->h * c->h);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_lift(pide_ctx* c, const double* g, cudaStream_t st) {
  if (c->dims == 3)
    lift3d_kernel<<<grid_for(c->n, 256, c->num_sms), 256, 0, st>>>(g, c->w, c->nx, c->ny, c->nz,
                                                                    c->lift);
  else
    lift_kernel<<<grid_for(c->n, 256, c->num_sms), 256, 0, st>>>(g, c->w, c->nx, c->ny, c->lift);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

static dim3 col_grid(int n, int B) {
  int gx = (n + 255) / 256;
  if (gx > 1024) gx = 1024;
  return dim3(gx, B, 1);
}

pide_status launch_prep(pide_ctx* c, const double* b, int B, int mode, const double* lift,
                        int rfmt, bool track, cudaStream_t st, bool emul) {
  if (B == 0) return PIDE_OK;
  ProfScope ps(c, st, 2);
  if (emul && mode == 0 && rfmt == RF_BF16) return launch_prep_df_bf16(c, b, B, lift, track, st);
  if (rfmt == RF_F16) return PIDE_EINVAL;   // FP16 right-hand sides: launch_prep_f16 (scales first)
  dim3 g = col_grid(c->n, B);
  double* cmb = c->colmax + c->ws_B;
  const int t = track ? 1 : 0;
  switch (rfmt) {
    case RF_F64: prep_kernel<RF_F64><<<g, 256, 0, st>>>(b, c->n, c->ld, mode, c->dinv, lift, c->R, nullptr, cmb, t); break;
    case RF_F32: prep_kernel<RF_F32><<<g, 256, 0, st>>>(b, c->n, c->ld, mode, c->dinv, lift, c->R, nullptr, cmb, t); break;
    case RF_BF16: prep_kernel<RF_BF16><<<g, 256, 0, st>>>(b, c->n, c->ld, mode, c->dinv, lift, c->R, nullptr, cmb, t); break;
    default: prep_kernel<RF_E4M3><<<g, 256, 0, st>>>(b, c->n, c->ld, mode, c->dinv, lift, c->R, c->col_scale, cmb, t); break;
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_residual(pide_ctx* c, const double* b, const double* u, int B, int mode,
                            const double* lift, int rfmt, bool write_R, double* r_out, bool track,
                            bool honor_done, cudaStream_t st, int col0, bool emul) {
  if (B == 0) return PIDE_OK;
  ProfScope ps(c, st, 1);
  dim3 g = col_grid(c->n, B);
  const size_t off = (size_t)col0 * c->n;
  b += off;
  u += off;
  if (r_out) r_out += off;
  void* R = write_R ? (void*)((uint8_t*)c->R + (size_t)col0 * c->ld * rhs_elem_bytes(rfmt)) : nullptr;
  const uint32_t* fl = honor_done ? c->flags : nullptr;
  double* cm = c->colmax + col0;
  const int t = track ? 1 : 0;
  if (emul && mode == 0 && R && !r_out && rfmt != RF_F64) {
    const pide_status s = launch_residual_df(c, b, u, B, lift, rfmt, R, c->ld,
                                             (rfmt == RF_E4M3 || rfmt == RF_F16) ? c->col_scale + col0 : nullptr,
                                             cm, track, fl, st);
    if (s != PIDE_EUNSUPPORTED) return s;      // else: the FP64 stencil below
  }
  switch (rfmt) {
    case RF_F64: (c->dims == 3 ? residual_kernel<RF_F64, true> : residual_kernel<RF_F64, false>)<<<g, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), c->ld, mode, c->w, c->dinv, lift, R, nullptr, r_out, cm, t, fl); break;
    case RF_F32: (c->dims == 3 ? residual_kernel<RF_F32, true> : residual_kernel<RF_F32, false>)<<<g, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), c->ld, mode, c->w, c->dinv, lift, R, nullptr, r_out, cm, t, fl); break;
    case RF_BF16: (c->dims == 3 ? residual_kernel<RF_BF16, true> : residual_kernel<RF_BF16, false>)<<<g, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), c->ld, mode, c->w, c->dinv, lift, R, nullptr, r_out, cm, t, fl); break;
    case RF_F16: (c->dims == 3 ? residual_kernel<RF_F16, true> : residual_kernel<RF_F16, false>)<<<g, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), c->ld, mode, c->w, c->dinv, lift, R, c->col_scale + col0, r_out, cm, t, fl); break;
    default: (c->dims == 3 ? residual_kernel<RF_E4M3, true> : residual_kernel<RF_E4M3, false>)<<<g, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), c->ld, mode, c->w, c->dinv, lift, R, c->col_scale + col0, r_out, cm, t, fl); break;
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_residual_persistent(pide_ctx* c, const double* b, const double* u, int B,
                                      int mode, const double* lift, int rfmt, cudaStream_t st,
                                      int col0) {
  if (B == 0) return PIDE_OK;
  ProfScope ps(c, st, 1);
  const size_t off = (size_t)col0 * c->n;
  b += off;
  u += off;
  void* R = (uint8_t*)c->R + (size_t)col0 * c->ld * rhs_elem_bytes(rfmt);
  const int grid = c->num_sms * c->resid_ctas_per_sm;
  const float* cs = c->col_scale + col0;
  if (rfmt == RF_F16) return PIDE_EUNSUPPORTED;
  switch (rfmt) {
    case RF_F32: (c->dims == 3 ? residual_flat_kernel<RF_F32, true> : residual_flat_kernel<RF_F32, false>)<<<grid, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), B, c->ld, mode, c->w, c->dinv, lift, R, nullptr, c->flags); break;
    case RF_BF16: (c->dims == 3 ? residual_flat_kernel<RF_BF16, true> : residual_flat_kernel<RF_BF16, false>)<<<grid, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), B, c->ld, mode, c->w, c->dinv, lift, R, nullptr, c->flags); break;
    case RF_E4M3: (c->dims == 3 ? residual_flat_kernel<RF_E4M3, true> : residual_flat_kernel<RF_E4M3, false>)<<<grid, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), B, c->ld, mode, c->w, c->dinv, lift, R, cs, c->flags); break;
    default: (c->dims == 3 ? residual_flat_kernel<RF_F64, true> : residual_flat_kernel<RF_F64, false>)<<<grid, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), B, c->ld, mode, c->w, c->dinv, lift, R, nullptr, c->flags); break;
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_check(pide_ctx* c, int B, double tol, cudaStream_t st) {
  ProfScope ps(c, st, 3);
  check_kernel<<<1, 256, 0, st>>>(c->colmax, c->colmax + c->ws_B, B, tol, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_record(pide_ctx* c, int B, double* slot, bool reset, cudaStream_t st) {
  ProfScope ps(c, st, 3);
  record_kernel<<<1, 256, 0, st>>>(c->colmax, c->colmax + c->ws_B, B, slot, reset ? 1 : 0,
                                   c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_colmax_b(pide_ctx* c, const double* b, int B, int mode, const double* lift,
                            cudaStream_t st) {
  if (B == 0) return PIDE_OK;
  colmax_b_kernel<<<col_grid(c->n, B), 256, 0, st>>>(b, c->n, mode, c->dinv, lift,
                                                     c->colmax + c->ws_B);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_face_grad(pide_ctx* c, const double* mu, const double* u, const double* b,
                             int B, double* deps, cudaStream_t st) {
  ProfScope ps(c, st, 3);
  const int N = c->nx * c->ny * c->nz;
  double* Tf = nullptr;
  PIDE_CUDA_TRY(cudaMallocAsync((void**)&Tf, (size_t)c->dims * N * sizeof(double), st));
  const dim3 grid((N + 31) / 32), block(32, FG_GROUPS);
  if (c->dims == 3) {
    face_t_kernel<3><<<grid, block, 0, st>>>(mu, u, b, c->nx, c->ny, c->nz, B, Tf);
    face_combine_kernel<3><<<grid_for(N, 256, c->num_sms), 256, 0, st>>>(Tf, c->eps, c->nx, c->ny,
                                                                        c->nz, deps);
  } else {
    face_t_kernel<2><<<grid, block, 0, st>>>(mu, u, b, c->nx, c->ny, 1, B, Tf);
    face_combine_kernel<2><<<grid_for(N, 256, c->num_sms), 256, 0, st>>>(Tf, c->eps, c->nx, c->ny,
                                                                        1, deps);
  }
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(Tf, st);
  if (e != cudaSuccess) {
    set_error(std::string("face gradient: ") + cudaGetErrorString(e));
    return PIDE_ECUDA;
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_scale_d(pide_ctx* c, const double* mu, double* db, int B, cudaStream_t st) {
  const long long total = (long long)B * c->n;
  if (total == 0) return PIDE_OK;
  scale_d_kernel<<<grid_for(total, 256, c->num_sms), 256, 0, st>>>(mu, c->d, db, c->n, total);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

namespace {

// FP8 right-hand sides: max |f~| per column (prep) ...
__global__ void colmax_raw_prep_kernel(const double* __restrict__ b, int n, int mode,
                                       const double* __restrict__ dinv,
                                       const double* __restrict__ lift,
                                       double* __restrict__ colmax_raw) {
  __shared__ double red[32];
  const int col = blockIdx.y;
  const double* bc = b + (size_t)col * n;
  double mx = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double f = bc[p];
    if (mode == 1) f *= dinv[p];
    else if (lift) f += lift[p];
    mx = fmax(mx, fabs(f));
  }
  mx = block_max(mx, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&colmax_raw[col], mx);
}

// ... and the per-column scale max/448 (448 = largest finite e4m3); resets the maxima.
__global__ void finalize_scale_kernel(double* __restrict__ colmax_raw, float* __restrict__ col_scale,
                                      int B, const uint32_t* __restrict__ flags) {
  if (flags && flags[FLAG_DONE]) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < B; c += gridDim.x * blockDim.x) {
    const double m = colmax_raw[c];
    col_scale[c] = m > 0.0 ? (float)(m / 448.0) : 1.0f;
    colmax_raw[c] = 0.0;
  }
}

}  // namespace

namespace {
__global__ void finalize_scale_kernel(double* __restrict__ colmax_raw, float* __restrict__ col_scale,
                                      int B, const uint32_t* __restrict__ flags);
__global__ void quantize_e4m3_kernel(const float* __restrict__ Rf, int n, int ld,
                                     const float* __restrict__ col_scale,
                                     __nv_fp8_e4m3* __restrict__ R,
                                     const uint32_t* __restrict__ flags) {
  if (flags[FLAG_DONE]) return;
  const int col = blockIdx.y;
  const float isc = 1.0f / col_scale[col];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    R[(size_t)col * ld + p] = __nv_fp8_e4m3(Rf[(size_t)col * ld + p] * isc);   // FP32: off the FP64 pipe
}
}  // namespace

pide_status launch_residual_fp8(pide_ctx* c, const double* b, const double* u, int B, int mode,
                                const double* lift, cudaStream_t st, bool emul) {
  if (B == 0) return PIDE_OK;
  ProfScope ps(c, st, 1);
  dim3 g = col_grid(c->n, B);
  double* raw = c->colmax + 2 * (size_t)c->ws_B;
  pide_status sdf = PIDE_EUNSUPPORTED;
  if (emul && mode == 0)
    sdf = launch_residual_df(c, b, u, B, lift, RF_F32, c->Rf, c->ld, nullptr, raw, true, c->flags,
                             st);
  if (sdf != PIDE_OK && sdf != PIDE_EUNSUPPORTED) return sdf;
  if (sdf == PIDE_EUNSUPPORTED) {
    (c->dims == 3 ? residual_kernel<RF_F32, true> : residual_kernel<RF_F32, false>)<<<g, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), c->ld, mode, c->w, c->dinv,
                                               lift, c->Rf, nullptr, nullptr, raw, 1, c->flags);
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  finalize_scale_kernel<<<(B + 255) / 256, 256, 0, st>>>(raw, c->col_scale, B, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  quantize_e4m3_kernel<<<g, 256, 0, st>>>(c->Rf, c->n, c->ld, c->col_scale,
                                          (__nv_fp8_e4m3*)c->R, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

pide_status launch_fp8_scales(pide_ctx* c, const double* b, const double* u, int B, int mode,
                              const double* lift, bool from_residual, cudaStream_t st, int col0) {
  if (B == 0) return PIDE_OK;
  ProfScope ps(c, st, 2);
  dim3 g = col_grid(c->n, B);
  double* raw = c->colmax + 2 * (size_t)c->ws_B + col0;
  b += (size_t)col0 * c->n;
  if (u) u += (size_t)col0 * c->n;
  if (from_residual) {
    (c->dims == 3 ? residual_kernel<RF_F64, true> : residual_kernel<RF_F64, false>)<<<g, 256, 0, st>>>(b, u, c->n, c->mx, plane_of(c), c->ld, mode, c->w, c->dinv, lift,
                                               nullptr, nullptr, nullptr, raw, 1, c->flags);
  } else {
    colmax_raw_prep_kernel<<<g, 256, 0, st>>>(b, c->n, mode, c->dinv, lift, raw);
  }
  PIDE_CUDA_TRY(cudaGetLastError());
  finalize_scale_kernel<<<(B + 255) / 256, 256, 0, st>>>(raw, c->col_scale + col0, B, c->flags);
  PIDE_CUDA_TRY(cudaGetLastError());
  return PIDE_OK;
}

}  // namespace pide
