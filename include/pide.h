/*
 * pide.h -- C ABI of the GB300 dense-inverse Poisson apply.
 *
 * The method (Dourbal & Pekker, "A New Numerical Method for Fast Solution of
 * Partial Integro-Differential Equations"): assemble the 5-point system of
 * Eq. (2)/(3) on an nx x ny node grid (Fig. 3: boundary nodes are identity
 * rows), invert it once ("The solution steps", step 2), then obtain every
 * solution by one matrix-vector product with the inverse (step 3):
 *
 *     u = L_eps^-1 b          for many right-hand sides b at once.
 *
 * Notation used throughout.
 *   Grid: nodes (i, j), 0 <= i < ny (y), 0 <= j < nx (x), spacing h in both
 *     directions (Eq. 2).  Interior nodes 1 <= i <= ny-2, 1 <= j <= nx-2;
 *     n = (nx-2)*(ny-2) unknowns, ordered as in Fig. 3 restricted to the
 *     interior: index (i-1)*(nx-2) + (j-1), j fastest.
 *   Operator (Eq. 3): row p reads u_p - sum_q w_pq u_q = b_p, with face
 *     permittivity eps_pq = harmonic mean of the two node values and
 *     w_pq = eps_pq / d_p, d_p = sum of the four face values of node p.  At
 *     eps = 1 every w is 0.25 (Fig. 3).  Equivalently S u = D b with
 *     D = diag(d), S = D L symmetric positive definite.
 *   Right-hand side: b is the Eq. (3) right side at interior nodes.  From a
 *     charge density (Eq. 1) it is b = -h^2 rho / d (pide_rhs_from_charge).
 *   Boundary values: zero unless a boundary array g is given.
 *
 * Conventions.
 *   - Every *_dev pointer is CUDA device memory owned by the caller, laid out
 *     [B][n] (one right-hand side per row, row stride n), float64 unless stated.
 *   - The handle owns the inverse, its quantised copy, scales and workspace.
 *   - All work is ordered on the given cudaStream_t (passed as void*; NULL =
 *     the legacy default stream).  Calls return after enqueueing unless an
 *     output lives on the host (pide_info, pide_apply_host, pide_save).
 *   - No call throws; each returns a pide_status.  pide_last_error() returns
 *     a message for the last failure on the calling thread.
 *   - One handle may be used from one host thread at a time.
 */
#ifndef PIDE_H
#define PIDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pide_ctx* pide_handle;
typedef struct pide_batch* pide_batch_handle;

typedef enum {
  PIDE_OK = 0,
  PIDE_EINVAL = 1,       /* bad argument (size, NULL pointer, eps <= 0, NaN) */
  PIDE_ENOMEM = 2,       /* device or host allocation failed */
  PIDE_ECUDA = 3,        /* a CUDA runtime or driver call failed */
  PIDE_ENOTCONV = 4,     /* tol not reached within max_sweeps (u is written) */
  PIDE_ETIMEOUT = 5,     /* a bounded device-side wait gave up (kernel returned) */
  PIDE_EUNSUPPORTED = 6  /* valid request this build cannot serve */
} pide_status;

/* Storage/contraction format of the inverse (step 2's result). */
typedef enum {
  PIDE_FP64 = 0,   /* plain FP64 inverse, FP64 apply (the comparator) */
  PIDE_FP32 = 1,   /* FP32 inverse, FP32 SIMT apply, FP64 refinement */
  PIDE_BF16 = 2,   /* BF16 inverse, tensor-core apply (FP32 accumulate), FP64 refinement */
  PIDE_FP8 = 3,    /* e4m3 inverse with per-row scales (single term; study only) */
  PIDE_FP8X2 = 4,  /* e4m3 hi + lo terms with per-row scales, FP8 tensor cores */
  PIDE_BF16_FP8 = 5, /* BF16 inverse Q plus an e4m3 correction term C with its own per-row
                       scales s_p: C = e4m3((L^-1 - Q) / s_p).  Every apply contracts Q on the
                       BF16 tensor cores; the applies that PIDE_TUNE_CORR_MASK selects add
                       s_p t_j (C e4m3(R / t_j)) on the FP8 tensor cores (t_j = max|R_j| / 448),
                       which cuts that sweep's error by a further ~2^-4 (B = 2..65535 only:
                       B = 1 and the batched entry points use Q alone) */
  PIDE_FP16 = 6,    /* FP16 inverse Q_p = fp16(L^-1_p / s_p) with power-of-two row scales s_p
                       (row maximum in [2^14, 2^15)), FP16 right-hand sides with power-of-two
                       column scales t_j set once per apply from the first right-hand side
                       (column maximum in [2^11, 2^12)), tensor-core apply on the FP16 pipe
                       (the BF16 rate) with u += s_p t_j acc: 11 significant bits where BF16
                       has 8.  The scales are kept in FP32's normal range: a right-hand-side
                       column whose largest |f| lies above ~2^139 saturates at 65504 and one
                       below ~2^-115 loses bits to FP16 subnormals.  B = 1 uses the symmetric
                       two-term store as PIDE_BF16 does; not served by the batched entry
                       points */
  PIDE_FP16_FP8 = 7, /* PIDE_FP16 plus the e4m3 correction term of PIDE_BF16_FP8, taken against
                       the FP16 store; PIDE_TUNE_CORR_MASK defaults to 1 (the first apply) */
  PIDE_AUTO = 8     /* setup only: the store is chosen by measurement, as pide_setup_auto does
                       with its defaults (target 0.5e-6, 16 built-in probe right-hand sides,
                       at most 8 sweeps); the handle then reports the chosen format */
} pide_precision;

/* max_sweeps value of pide_apply, pide_apply_host and pide_solve_stream that
 * takes the sweep count measured for the handle by pide_setup_auto (EINVAL on
 * a handle that was not set up that way). */
#define PIDE_SWEEPS_AUTO (-1)

typedef struct {
  int32_t nx;      /* nodes along x including the two boundary nodes, >= 3 */
  int32_t ny;      /* nodes along y including the two boundary nodes, >= 3 */
  double h;        /* grid spacing (Eq. 2), > 0 */
} pide_grid;

/* A 3-D node grid: nx x ny x nz nodes including boundary nodes, spacing h. */
typedef struct {
  int32_t nx, ny, nz;   /* each >= 3 */
  double h;
} pide_grid3;

typedef struct {
  int32_t sweeps;        /* refinement sweeps executed */
  int32_t converged;     /* 1 if tol was met (always 1 when tol <= 0) */
  double rel_residual;   /* max over columns of ||b - L u||_inf / ||b||_inf (FP64) */
  double setup_ms;       /* wall time of pide_setup for this handle */
  double contraction;    /* measured per-sweep contraction of the refinement:
                            (rel_residual / r_0)^(1/sweeps), r_0 = the same worst-column
                            relative residual after the first apply, i.e. the geometric mean
                            of ||r_k||_inf / ||r_k-1||_inf; NaN when no sweep ran */
  double ms;             /* device time of the call's work (CUDA events on its stream), from
                            the right-hand-side prep to the last apply; pide_apply_host
                            includes its copies */
} pide_info;

/* One stored format measured by pide_setup_auto. */
typedef struct {
  int32_t precision;     /* pide_precision of the candidate store */
  int32_t corr_mask;     /* applies that add its e4m3 correction term (0: none) */
  int32_t sweeps;        /* fewest sweeps whose Eq. (6) error met the target on the probe;
                            -1 if max_sweeps did not reach it */
  double error;          /* Eq. (6) error on the probe after those sweeps (after max_sweeps
                            when the target was missed), against the FP64 inverse */
  double contraction;    /* geometric-mean error ratio per sweep (sweeps above 1e-12) */
  double cost;           /* modelled cost of one refined apply in 16-bit GEMM units:
                            (1 + sweeps) x (1, or 28 for FP32) + 0.5 per corrected apply
                            + 0.15 per sweep (residual and prep) */
} pide_auto_candidate;

typedef struct {
  double target;         /* Eq. (6) error the probe had to reach */
  int32_t nprobe;        /* probe right-hand sides */
  int32_t max_sweeps;
  int32_t ncand;         /* entries of cand[] that were measured */
  int32_t chosen;        /* index into cand[] of the store the handle keeps */
  pide_auto_candidate cand[6];
} pide_auto_report;

typedef struct {
  int32_t n;             /* unknowns */
  int32_t ld;            /* row stride (elements) of the stored inverse */
  int32_t precision;     /* pide_precision */
  int32_t num_sms;       /* SMs of the device the handle lives on */
  size_t store_bytes;    /* bytes of the stored inverse (+ scales) read per apply */
  double setup_ms;
  int32_t dims;          /* 2 (pide_setup) or 3 (pide_setup_3d) */
  int32_t sweeps_hint;   /* sweeps measured by pide_setup_auto (what PIDE_SWEEPS_AUTO takes);
                            -1 for handles set up with an explicit format or loaded */
} pide_handle_info;

/* Per-kernel-class event timing, recorded on the launching stream. */
typedef struct {
  int32_t launches[5];   /* [0] apply (GEMM/GEMV) [1] residual [2] rhs prep (with the
                            e4m3 copy of R for the correction term) [3] other: the
                            correction term's FP8 GEMM, the tolerance check, the
                            adjoint's face gradients [4] reduce: the sums of the
                            K-split last round of a tensor-core apply on SM pairs
                            (PIDE_TUNE_GEMM_STREAMK) */
  double ms[5];          /* summed CUDA-event time per class */
} pide_profile;

/*
 * pide_setup -- steps 1 and 2: assemble the operator (Eq. 2/3, Fig. 3) from
 * node permittivity and form its inverse.
 *   g         grid (nx, ny >= 3, h > 0).
 *   eps_host  [ny][nx] float64 node permittivity on the HOST, every value
 *             finite and > 0 (NULL means eps = 1, the case of Eq. 2).
 *   p         storage format of the inverse.  The inverse is always formed
 *             in FP64 on the GPU (block-tridiagonal elimination), then
 *             quantised; the FP64 copy is kept only for PIDE_FP64.  BF16 and
 *             FP16 handles (with or without the correction term) also keep
 *             the lower triangle of the symmetric S^-1 in 128 x 128 tiles of
 *             two terms (BF16 hi + FP16 lo with a power-of-two scale per row,
 *             the size of the one-term L^-1) for one-column applies.
 *   stream    cudaStream_t for all setup work (the call synchronises it).
 *   out       receives the new handle (NULL on failure).
 * Errors: EINVAL (bad grid, eps), ENOMEM, ECUDA, EUNSUPPORTED (not sm_103).
 * Environment: PIDE_FAULT_ALLOC=1 makes the call fail with ENOMEM before any
 * device work (host-side fault injection for tests).
 */
pide_status pide_setup(const pide_grid* g, const double* eps_host, pide_precision p,
                       void* stream, pide_handle* out);

/*
 * pide_setup_3d -- the same for an nx x ny x nz node grid (the paper states its
 * problem for N grid points; the worked case is 2-D): the 7-point flux form
 * with harmonic face permittivity, each interior row divided by its total face
 * permittivity (weight 1/6 at eps = 1), identity rows at boundary nodes.
 *   eps_host  [nz][ny][nx] node permittivity (x fastest), or NULL for eps = 1.
 * Interior unknowns p = ((k-1)(ny-2) + (i-1))(nx-2) + (j-1) for node (k, i, j)
 * (z, y, x).  The handle serves pide_apply, pide_apply_host, pide_solve_stream,
 * pide_residual, pide_rhs_from_charge (b = -h^2 rho / d with the six-face d),
 * boundary values g [nz][ny][nx] in pide_apply, the tuning and profiling
 * hooks, pide_apply_backward (six-face dLoss/deps, deps_dev [nz][ny][nx]) and
 * pide_save / pide_load.  The batched plans and pide_apply_noalloc return
 * PIDE_EUNSUPPORTED for it.  The FP64
 * inverse is formed by block elimination over z-planes: setup cost grows as
 * ((nx-2)(ny-2))^3 (nz-2) on GB300's FP64 pipe (seconds at 32^3 unknowns).
 */
pide_status pide_setup_3d(const pide_grid3* g, const double* eps_host, pide_precision p,
                          void* stream, pide_handle* out);

/*
 * pide_setup_auto -- pide_setup with the stored format chosen by measurement.
 * The paper rounds the inverse to k decimal digits and measures the error
 * against the exact solution for each k (Table 1, and the numerical example's
 * rounding of the inverse); here the candidate binary stores of the inverse are
 * each measured by the error their refined apply reaches.  After step 2 the
 * FP64 inverse G is held once; for each candidate -- FP16 + e4m3 correction in
 * the first apply, FP16, BF16 + e4m3 correction in the first sweep, BF16, in
 * that order, and FP32 only when none of them reaches the target -- the store
 * is quantised from G, the probe right-hand sides are solved with
 * k = 0, 1, ... max_sweeps refinement sweeps, and the Eq. (6) error against
 * G's own FP64 apply is taken after each k.  The handle keeps the candidate
 * of lowest modelled cost (pide_auto_candidate.cost) among those that reached
 * the target (ties: the earlier one), with that sweep count as its
 * sweeps_hint (pide_apply with max_sweeps = PIDE_SWEEPS_AUTO uses it).
 *   target      Eq. (6) error to reach on the probe, in (0, 0.1].
 *   probe_host  [nprobe][n] float64 right-hand sides on the HOST (Eq. 3 form),
 *               or NULL for built-in probes: column j is b = -h^2 rho / d for a
 *               charge rho of four Gaussian blobs (width 0.05, centres uniform in
 *               [0.2, 0.8] along each axis, amplitudes uniform in [-1, 1]) drawn
 *               from a counter-based generator (splitmix64) seeded by j.
 *   nprobe      1 .. 256 probe columns.
 *   max_sweeps  0 .. 30.
 * The other arguments are pide_setup's.  Setup holds G and one candidate
 * store at a time (12.3 GB + 4.6 GB at 198^2 unknowns) and takes a few
 * milliseconds per probe solve beyond pide_setup.  pide_get_auto_report
 * returns what was measured.  Errors: those of pide_setup; EINVAL for target,
 * nprobe or max_sweeps out of range.
 */
pide_status pide_setup_auto(const pide_grid* g, const double* eps_host, double target,
                            const double* probe_host, int32_t nprobe, int32_t max_sweeps,
                            void* stream, pide_handle* out);

/* The measurements behind a pide_setup_auto handle (EINVAL for other handles). */
pide_status pide_get_auto_report(pide_handle h, pide_auto_report* out);

/* Release every device and host resource of the handle (NULL is a no-op). */
void pide_destroy(pide_handle h);

/*
 * pide_apply -- step 3 with iterative refinement:
 *   u = Q(L^-1) b;  then up to max_sweeps times  u += Q(L^-1) (b - L u),
 * where Q(.) is the stored inverse (with the e4m3 correction term added in
 * the applies PIDE_TUNE_CORR_MASK selects, for the *_FP8 stores) and the
 * residual b - L u is taken to FP64 accuracy (FP64 stencil, or double-float
 * on the integer/FP32 pipes) with the 5-point stencil of Eq. (3).  The
 * residual reaches the tensor cores in the store's right-hand-side format
 * (BF16; FP16 with the column scales of b; e4m3 with per-column scales).
 *   b_dev     [B][n] right-hand sides (Eq. 3 form, interior nodes).
 *   u_dev     [B][n] solutions (written; must not alias b_dev).
 *   B         number of right-hand sides, >= 0 (0 is a no-op).
 *   max_sweeps  refinement sweeps (0 = a single apply).
 *   tol       > 0: stop early once ||b - L u||_inf <= tol ||b||_inf for every
 *             column (checked on the device; later kernels return at once);
 *             <= 0: run exactly max_sweeps sweeps.
 *   g_dev     [ny][nx] boundary values on the device, or NULL for zero.
 *   info      if non-NULL the call synchronises the stream and fills it.
 * Errors: EINVAL, ENOMEM (workspace), ECUDA, ETIMEOUT, ENOTCONV (only when
 * info is non-NULL and tol > 0 was not reached; u is still written).
 */
pide_status pide_apply(pide_handle h, const double* b_dev, double* u_dev, int32_t B,
                       int32_t max_sweeps, double tol, const double* g_dev,
                       void* stream, pide_info* info);

/*
 * pide_apply_host -- pide_apply on HOST buffers: copies b to the device,
 * applies, copies u back and synchronises.  b_host/u_host are [B][n] float64
 * (pinned memory makes the copies asynchronous-capable and fast).  For
 * B >= 512 with tol <= 0 and no info, the columns go in two chunks and the
 * copies of one chunk run on an internal stream under the other's solve.
 */
pide_status pide_apply_host(pide_handle h, const double* b_host, double* u_host, int32_t B,
                            int32_t max_sweeps, double tol, void* stream, pide_info* info);

/*
 * pide_solve_stream -- a time sequence of T right-hand sides (Eq. 1 with a
 * time-dependent charge, one solve per time step) from HOST memory:
 * in_host[T][n] float64 holds b (charge = 0) or the charge density rho
 * (charge = 1: b = -h^2 rho / d on the device, as pide_rhs_from_charge), and
 * u_host[T][n] receives the solutions.  The columns go through two device
 * slots of `chunk` columns (chunk in [1, 65535]; allocated by the handle on
 * first use, 4 * chunk * n * 8 bytes, kept for later calls): the copy of
 * chunk i + 1 to the device and of chunk i - 1 to the host run on internal
 * streams under the refined solve of chunk i (max_sweeps refinement sweeps,
 * fixed count).  When T > chunk the first and the last piece are a half
 * chunk, so that little copy time is left outside the solves.  Pinned host memory is needed for the copies to overlap.
 * Ordered after the work already on `stream`; returns after synchronising.
 * in_host and u_host must not overlap.
 */
pide_status pide_solve_stream(pide_handle h, const double* in_host, double* u_host, int64_t T,
                              int32_t chunk, int32_t max_sweeps, int32_t charge, void* stream);

/*
 * pide_residual -- r = b - L u at interior nodes (Eq. 3 as a matrix-free
 * 5-point stencil, FP64, zero boundary values).  b, u, r are [B][n]; r may
 * alias neither b nor u.
 */
pide_status pide_residual(pide_handle h, const double* b_dev, const double* u_dev,
                          double* r_dev, int32_t B, void* stream);

/*
 * pide_rhs_from_charge -- b = -h^2 rho / d: the Eq. (3) right side for a
 * charge density rho of Eq. (1) (flux form; at eps = 1 this is -h^2 rho / 4).
 * rho, b are [B][n]; b may alias rho.
 */
pide_status pide_rhs_from_charge(pide_handle h, const double* rho_dev, double* b_dev,
                                 int32_t B, void* stream);

/*
 * pide_apply_backward -- adjoint of u = L(eps)^-1 b (b held fixed).  Given
 * gout = dLoss/du, with mu = S^-1 gout (solved with the same stored inverse
 * and FP64 refinement):
 *   db   = dLoss/db = D mu                                   [B][n]
 *   deps = dLoss/deps (node permittivity, [ny][nx]), ACCUMULATED into deps_dev:
 *          per face f = (p,q): sum over columns of
 *          mu_p b_p + mu_q b_q - (mu_p - mu_q)(u_p - u_q)  (boundary node: mu = 0,
 *          no b term, u = 0), chained through the harmonic mean
 *          d eps_f / d eps_a = 2 eps_b^2 / (eps_a + eps_b)^2.
 * u_dev must be the forward solution for b_dev.  db_dev or deps_dev may be NULL.
 * Scratch (mu, B x n doubles; the face sums, 2 or 3 x nodes doubles) comes from
 * the stream-ordered allocator (cudaMallocAsync / cudaFreeAsync on `stream`).
 * The deps sums are deterministic (fixed order, no atomics).
 * Not in the paper: the gradient follows from differentiating L u = b.
 */
pide_status pide_apply_backward(pide_handle h, const double* gout_dev, const double* u_dev,
                                const double* b_dev, double* db_dev, double* deps_dev,
                                int32_t B, int32_t max_sweeps, void* stream);

/*
 * Batched apply (not in the paper; the many-problem form of step 3): nprob
 * independent problems -- handles of any grid size with FP32 or BF16 stores --
 * each with its own column count Bs[k] and device buffers b[k], u[k]
 * ([Bs[k]][n_k] float64).  A plan uploads one problem table and two device
 * work lists: (problem, 64-row tile, 64-column tile) items, largest first,
 * for the apply, and (problem, column) items for the right-hand-side prep and
 * the FP64 residual.  Each phase of the refinement then runs as ONE launch
 * over all problems: 2 + 2*sweeps launches per run.
 *
 * pide_batch_create  builds the plan (allocates; synchronous).  Handles must
 *                    outlive the plan and share one device; b/u pointers are
 *                    fixed in the plan.  sweeps_k (may be NULL): per-problem
 *                    cap on the refinement sweeps (a problem skips the phases
 *                    past its cap).  EUNSUPPORTED for FP64/FP8 stores.
 * pide_batch_run     enqueues one refined batched apply with `sweeps` sweeps.
 *                    use_graph != 0 (and a non-NULL stream): the launches are
 *                    captured into a CUDA graph on the first run with a given
 *                    sweep count and replayed after that.
 * pide_batch_destroy releases the plan (synchronises the device).
 * pide_apply_batched create + run + synchronise + destroy in one call.
 */
pide_status pide_batch_create(const pide_handle* hs, int32_t nprob, const double* const* b,
                              double* const* u, const int32_t* Bs, const int32_t* sweeps_k,
                              pide_batch_handle* out);
pide_status pide_batch_run(pide_batch_handle p, int32_t sweeps, int32_t use_graph, void* stream);

/* The shapes a plan launches (what the problems' PIDE_TUNE_BATCH_* knobs chose). */
typedef struct {
  int32_t nprob;
  int32_t simt_items;          /* SIMT tile items per apply phase */
  int32_t tc_items;            /* grouped tensor-core items per apply phase */
  int32_t tc_items_bn[3];      /* of those, items with column tiles 32, 64, 128 wide */
  int32_t simt_problems_tn[3]; /* problems on SIMT tiles 16, 32, 64 columns wide */
  int32_t tf32_problems;       /* FP32 problems contracted on the TF32 tensor cores */
  int32_t apply_launches;      /* apply launches per phase */
} pide_batch_info;
pide_status pide_batch_get_info(pide_batch_handle p, pide_batch_info* out);
void pide_batch_destroy(pide_batch_handle p);
pide_status pide_apply_batched(const pide_handle* hs, int32_t nprob, const double* const* b,
                               double* const* u, const int32_t* Bs, int32_t sweeps,
                               void* stream);

/*
 * pide_apply_noalloc -- pide_apply(h, b, u, B, sweeps, tol = 0, g = NULL)
 * without any device allocation, for callers that cannot call cudaMalloc
 * (a fixed memory pool, a real-time loop, a host application that hands out
 * only pre-sized buffers).  The paper has no counterpart: it is a deployment
 * variant of step 3.  The caller passes b and u ([B][n] float64, device);
 * the FP32 scratch right-hand side lives in a fixed array inside the library
 * (2 MiB, held by every GPU that loads the library until exit), so B <= 8
 * and n <= 65536, else EINVAL with a message.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) -- make that
 * first call before any stream capture.  All calls share the array: calls
 * whose work overlaps on the GPU race and must be serialised.
 * What it computes: the refinement of pide_apply (first apply, then `sweeps`
 * times an FP64 stencil residual and an apply-accumulate) with every
 * right-hand side handed to the stored inverse in FP32, where pide_apply
 * hands the tensor cores FP16, BF16 or e4m3; the e4m3 correction term of a
 * *_FP8 store joins the applies its correction mask selects, as in pide_apply.
 * The two therefore agree once the refinement has converged, not apply by
 * apply (an FP64 store needs two sweeps to come back from the FP32 right-hand
 * side to FP64 accuracy).  The product runs on the CUDA cores (FP32 sums; FP64
 * for the FP64 store): at 198^2 unknowns one apply takes ~0.7 ms at B = 1 and
 * ~2 ms at B = 8.
 */
pide_status pide_apply_noalloc(pide_handle h, const double* b_dev, double* u_dev, int32_t B,
                               int32_t sweeps, void* stream);

/* Reserve workspace for up to Bmax columns now, so later pide_apply calls with
 * B <= Bmax allocate nothing (required before capturing them in a CUDA graph). */
pide_status pide_reserve(pide_handle h, int32_t Bmax);

/* Persist / restore the stored inverse (+ scales) with a header of grid,
 * format and an FNV-1a hash of eps; pide_load rebuilds the operator from the
 * saved eps and skips step 2. */
pide_status pide_save(pide_handle h, const char* path);
pide_status pide_load(const char* path, void* stream, pide_handle* out);

pide_status pide_get_handle_info(pide_handle h, pide_handle_info* out);

/* Event timing of every kernel the handle launches between begin and end
 * (end synchronises the stream).  Off unless begun. */
pide_status pide_profile_begin(pide_handle h);
pide_status pide_profile_end(pide_handle h, pide_profile* out);

/* Copy row p of the stored inverse L^-1 (converted to float64, scales
 * applied; PIDE_BF16_FP8: Q + s_p C, exact) to host memory dst[n]: lets tests
 * check individual entries. */
pide_status pide_get_inverse_row(pide_handle h, int32_t p, double* dst_host);

/* Table 1's experiment: round every entry of the stored inverse of an FP64
 * handle to `digits` digits after the decimal point, in place, half away from
 * zero, x -> sign(x) floor(|x| 10^digits + 1/2) / 10^digits with each FP64
 * operation rounded separately (digits in [0, 15]).  Later applies of the
 * handle use the rounded inverse.  FP64 handles only (PIDE_EUNSUPPORTED
 * otherwise).  Stream-ordered. */
pide_status pide_round_inverse_decimal(pide_handle h, int32_t digits, void* stream);

/* Launch-shape knobs of the apply kernels (set by the autotuner; results do
 * not depend on them beyond FP32 summation order).
 *   PIDE_TUNE_GEMV_THREADS  GEMV block size: 128..1024, multiple of 32 (default 1024)
 *   PIDE_TUNE_GEMV_UNROLL   16-byte loads in flight per lane: 4 or 8 (default 8)
 *   PIDE_TUNE_GEMV_MAX_B    largest B served by the GEMV instead of the GEMM: 1..8 (default 1)
 *   PIDE_TUNE_GEMM_BN       tensor-core tile width for B > 128: 128 or 256 (default 256)
 *   PIDE_TUNE_GEMM_STREAMK  1 (default): split the last partial wave of tiles over all SMs by
 *                           k-blocks.  Single SMs (B <= 128 or GEMM_BN 128): FP64 atomic
 *                           partial sums.  SM pairs: the r tiles of the last partial
 *                           round are cut into P K-ranges each (at least 8 k-blocks),
 *                           dealt round-robin to the pairs, with P chosen to shorten that
 *                           round plus the reduction the most, and only when that saves
 *                           5 % of a tile (e.g. r = 8 of 76 pairs at 198^2: P = 8); the
 *                           pieces write FP32 partial tiles to a handle-owned buffer (80
 *                           MB at 152 SMs) and a reduction kernel adds them to u, in
 *                           piece order (deterministic).  2: the same, leaving the
 *                           reduction's cost out of the choice (r = 56: P = 4, three
 *                           pieces on most pairs); 0: whole tiles only
 *   PIDE_TUNE_OVERLAP       1: for B >= 512 with tol <= 0, split the columns in
 *                           two groups and run each group's FP64 residual on a
 *                           low-priority internal stream under the other group's
 *                           tensor-core apply; 0 (default): one stream, whole batch per
 *                           phase (measured faster on GB300: the two overlapped kernels
 *                           slow each other by more than the residual's time)
 *   PIDE_TUNE_RESID_CTAS    residual CTAs (256 threads) per SM while overlapped: 1..8 (default 2)
 *   PIDE_TUNE_SYMV          1 (default): BF16 and FP16 handles apply B = 1 through the packed
 *                           lower triangle of the symmetric S^-1 (L^-1 = S^-1 D) in two terms
 *                           (BF16 hi + row-scaled FP16 lo), ~19 significant bits for the bytes
 *                           of the one-term L^-1, summed in FP32 within 8 tiles and FP64
 *                           across them: one apply reaches ~5e-7 at 198^2 unknowns;
 *                           0: through the one-term L^-1 (GEMV)
 *   PIDE_TUNE_RESID_EMUL    1 (default): BF16 / FP16 / FP8 / FP8X2 handles evaluate the
 *                           refinement residual (forward mode, and the BF16 prep) on the integer and
 *                           FP32 pipes: each FP64 input split into two floats (47
 *                           significant bits), the stencil in error-free float arithmetic,
 *                           absolute error ~2^-45 (|u_p| + sum_q w_pq |u_q|); skipped when
 *                           0 < tol < 1e-8, where only the FP64 stencil resolves the residual.
 *                           0: the FP64 stencil always.  pide_residual and the rel_residual
 *                           of pide_info are always FP64.
 *   PIDE_TUNE_RESID_SHAPE   launch shape of that residual kernel: nodes per thread (a tile of
 *                           256 x that many nodes per block, two columns per block):
 *                           -1 (default): 8; 0: 4, 1: 8, 2: 2, 3: 16
 *   PIDE_TUNE_GEMM_2CTA     1 (default): for B > 128 (with GEMM_BN 256) the tensor-core apply runs
 *                           on pairs of SMs (tcgen05 cta_group::2, 256 x 256 tiles, each SM
 *                           staging half of each operand tile); 0: one SM per 128 x 256 tile
 *   PIDE_TUNE_GEMM_A_HINT   L2 policy of the tensor-core apply's loads of the stored inverse:
 *                           0 evict-first, 1 evict-normal, 2 (default) evict-last (measured
 *                           on the SM-pair kernel at 198^2, B = 1024: 6.9 GB of DRAM reads per
 *                           launch with evict-first, 4.8 GB with either other policy; the
 *                           refined step 2 % shorter with evict-last than evict-normal, three
 *                           alternating runs each on one box)
 *   PIDE_TUNE_RESID_PREFETCH  the refinement residual's L2 prefetch distance, in column pairs:
 *                           each block prefetches its tile of the pair that many pairs ahead
 *                           (0 = none, up to 4096; default 4: the 2-D residual at 158^2 and
 *                           198^2 unknowns, B = 1024, 12-15% faster, 3-D unchanged)
 *   PIDE_TUNE_CORR_MASK       PIDE_BF16_FP8 / PIDE_FP16_FP8 handles: bit k set = apply k adds
 *                           the e4m3 correction term (bit 0: the first apply, bit k: refinement
 *                           sweep k; 0 .. 2^30 - 1; default 2 for PIDE_BF16_FP8, the first
 *                           sweep: at 198^2 unknowns, B = 1024, two sweeps then reach ~2e-7 where
 *                           BF16 alone needs four; default 1 for PIDE_FP16_FP8)
 *   PIDE_TUNE_GEMM_U_HINT     tensor-core GEMM epilogues: 1 (default) = load and store u with
 *                           an L2 evict-first hint (keeps the streamed inverse's lines in L2:
 *                           at 198^2, B = 1024, DRAM reads per accumulating launch 6.5 -> 5.2 GB,
 *                           same time), 0 = plain
 * Batched plans read three more knobs of each problem's handle when they are created:
 *   PIDE_TUNE_BATCH_TC        FP32 stores: 1 (default) = contract on the tensor cores as TF32
 *                           (kind::tf32: 10 explicit mantissa bits of each stored entry and
 *                           right-hand-side value, FP32 accumulate) in the grouped launch, the
 *                           FP64 residual refining the result; 0 = the FP32 SIMT tiles (FP32
 *                           products)
 *   PIDE_TUNE_BATCH_BN        grouped tensor-core launch: column-tile width 32, 64 or 128
 *                           (0 = default: the narrowest that covers the problem's B in one
 *                           tile); each width present in a plan is one launch per phase
 *   PIDE_TUNE_BATCH_TN        SIMT tiles: width 16, 32 or 64 columns (0 = default: the narrowest
 *                           covering the problem's B)
 *   PIDE_TUNE_PREP_CLUSTER    FP16 right-hand-side prep: 1 (default) = a cluster of 8 CTAs per
 *                           column holds the column in shared memory (one HBM pass; with the
 *                           correction term in the first apply it also writes the e4m3 copy of R),
 *                           up to ~112K unknowns; 0 = one CTA per column reading it twice */
typedef enum {
  PIDE_TUNE_GEMV_THREADS = 0,
  PIDE_TUNE_GEMV_UNROLL = 1,
  PIDE_TUNE_GEMV_MAX_B = 2,
  PIDE_TUNE_GEMM_BN = 3,
  PIDE_TUNE_GEMM_STREAMK = 4,
  PIDE_TUNE_OVERLAP = 5,
  PIDE_TUNE_RESID_CTAS = 6,
  PIDE_TUNE_SYMV = 7,
  PIDE_TUNE_RESID_EMUL = 8,
  PIDE_TUNE_RESID_SHAPE = 9,
  PIDE_TUNE_GEMM_2CTA = 10,
  PIDE_TUNE_GEMM_A_HINT = 11,
  PIDE_TUNE_RESID_PREFETCH = 12,
  PIDE_TUNE_CORR_MASK = 13,
  PIDE_TUNE_GEMM_U_HINT = 14,
  PIDE_TUNE_BATCH_TC = 15,
  PIDE_TUNE_BATCH_BN = 16,
  PIDE_TUNE_BATCH_TN = 17,
  PIDE_TUNE_PREP_CLUSTER = 18
} pide_tune_key;
pide_status pide_set_tuning(pide_handle h, int32_t key, int32_t value);
pide_status pide_get_tuning(pide_handle h, int32_t key, int32_t* value);

/* Fault-handling self test (no fault is raised): one GPU thread waits on a
 * barrier that nothing completes, with a budget of budget_cycles SM cycles
 * (1 .. 2e9).  The bounded wait gives up, the kernel returns, and the call
 * reports PIDE_ETIMEOUT with the device context intact -- the same path every
 * kernel's mbarrier waits take. */
pide_status pide_selftest_wait_timeout(int64_t budget_cycles, void* stream);

/* Conversion self test: for n device inputs, writes the library's own
 * integer-pipe conversions (binary64 -> bfloat16 round-to-nearest-even bits,
 * binary32 -> binary64) beside CUDA's, so a test can compare them bit for bit. */
/* Residual self test: the double-float residual kernel the refinement uses
 * (PIDE_TUNE_RESID_EMUL), r = f - L u with f = b (+ the lift of the boundary
 * values g_dev[ny*nx], or none when NULL), written as FP32 to r_dev[B][n] so
 * a test can compare it with the exact residual.  Device buffers, stream-ordered. */
pide_status pide_selftest_residual_df(pide_handle h, const double* b_dev, const double* u_dev,
                                      const double* g_dev, float* r_dev, int32_t B, void* stream);

pide_status pide_selftest_convert(const double* x_dev, const float* f_dev, int64_t n,
                                  uint16_t* bf_mine, uint16_t* bf_cuda, double* d_mine,
                                  double* d_cuda, void* stream);

const char* pide_status_string(pide_status s);
const char* pide_last_error(void);
int32_t pide_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PIDE_H */
