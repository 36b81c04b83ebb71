/*
 * az.h -- C ABI of the GB300 AZ solver for oversampled periodised-Gaussian RBF
 * least-squares systems (Zhou & Huybrechs, "Efficient least squares
 * approximation and collocation methods using radial basis functions",
 * arXiv 2308.14490).
 *
 * Problem (Sec. 2.2-2.3, Sec. 5.1-5.2): N equispaced centers per box
 * [-T_d, T_d] (Eq. set_centers), an s-fold oversampled grid of L = s N points
 * (Eq. set_Xtilde), the kept points X = grid ∩ Omega (Eqs. set_X, set_X_2d) and
 * the rectangular system A a ≈ b with A_ij = phi_per_j(x_i), phi the Gaussian
 * exp(-eps^2 r^2) (Eq. rbf) periodised over the box (Eq. periodic_rbf).
 * Solver: Algorithm 1 (AZ) with Z* the plain inverse of the full-box problem
 * (Sec. 3.1 Eq. B_pinv, Sec. 3.2.2) and a randomised truncated solve of the
 * low-rank step 1 (Sec. 3.2.3).
 *
 * Conventions shared by every entry point
 *  - Array arguments whose name ends in _dev are DEVICE pointers owned by the
 *    caller; the library never frees them.  The handle owns only its internal
 *    buffers (symbols, index maps, sketch factors, workspace).
 *  - Matrices are column-major with a leading dimension >= the row count.
 *  - Row order of right-hand sides: the kept grid points in lexicographic order
 *    of the grid index (1D: increasing i; 2D: i = ix*Ly + iy, x-major, the
 *    paper's j = (m-1) N^y + n ordering of Sec. 5.1), followed, for
 *    collocation, by the boundary points in the order given.
 *  - Coefficient order: j (1D) or jx*Ny + jy (2D).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered and asynchronous except where noted
 *    (az_setup synchronises once to learn M; a non-NULL relres_host forces a
 *    synchronisation).
 *  - No exception crosses the ABI.  Every failure returns a status and sets a
 *    thread-local message readable with az_last_error().
 *  - Environment: AZ_SKETCH_CLUSTER=1 runs the FP64 Z* chain of square 2D grids
 *    (L = 64, 128, 256 per dimension, s = 2) as one cluster-resident kernel per
 *    column pair (16-CTA clusters, the grid in distributed shared memory)
 *    instead of three passes through device memory; read at az_setup.
 *  - Supported sizes: dim 1 or 2; n[d] and s[d] powers of two; s[d] <= 8;
 *    L per dimension <= 2^24 (1D) or <= 4096 (2D).  Other sizes return
 *    AZ_ERR_ARG.
 */
#ifndef AZ_GB300_H
#define AZ_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct az_setup_t* az_handle;

typedef enum {
  AZ_OK = 0,
  AZ_ERR_ARG = 1,        /* invalid argument or unsupported size */
  AZ_ERR_OOM = 2,        /* device allocation failed */
  AZ_ERR_ADMISSION = 3,  /* footprint above the caller's budget */
  AZ_ERR_CUDA = 4,       /* a CUDA runtime call or kernel launch failed */
  AZ_ERR_NUMERIC = 5,    /* non-finite values, or the factorisation broke down */
  AZ_ERR_TIMEOUT = 6     /* a bounded device wait gave up */
} az_status;

enum { AZ_FP64 = 0, AZ_MIXED = 1 };
enum { AZ_GAUSS = 0, AZ_NEG_LAPLACE_GAUSS = 1 };

typedef struct {
  int32_t dim;     /* 1 or 2 */
  int64_t n[2];    /* centers per dimension (N_x, N_y); n[1] ignored in 1D */
  int32_t s[2];    /* oversampling factor per dimension (Eq. set_Xtilde) */
  double T[2];     /* half box widths: box = prod_d [-T_d, T_d] */
} az_grid;

typedef struct {
  int32_t precision;    /* AZ_FP64, or AZ_MIXED: FP32 transforms and FP64 factor work and residual.
                           In 1D the mixed sketch is FP32.  In 2D (dim = 2) the mixed setup sketches
                           and factorises in FP64 and keeps W in FP64: an FP32 sketch misplaces the
                           fitted subspace there (relres gaps ~1e-5).  Only the solve's transforms,
                           stencils and projection then run in FP32, and the update x = z + W u
                           reads the FP64 W */
  int32_t k;            /* sketch width r + p (number of random columns, Sec. 3.2.3), 1..4096; 0 = adaptive:
                           widths 64, 128, ... until the k-th singular value of the sketch is below
                           1e-7 (FP64) or 1e-4 (mixed) of the largest (az_get_info reports the k used);
                           each wider attempt keeps the narrower one's sketch columns and sketches only
                           the new ones, so the result equals a fixed-width setup at the final width.
                           A width above M + n_boundary (the number of rows of the sketch) is reduced
                           to it; the first columns of R are kept */
  double tau_svd;       /* relative truncation of the low-rank solve (0 = default: 1e-8).  The narrow
                           (k <= 64) factorisation works on the Gram matrix and resolves singular values
                           down to about 1e-8 of the largest, so in AZ_FP64 a tau_svd below 1e-8 takes the
                           Householder factorisation of the wide sketches at any width */
  double tau_sym;       /* symbol truncation: S_k^{-1} := 0 if S_k <= tau_sym^2 max S (0 = exact) */
  uint64_t seed;        /* Philox key of the random test matrix */
  int32_t refine_steps; /* FP64-residual refinement steps per solve (default 1 in MIXED, 0 in FP64) ; -1 = default */
  double k0;            /* collocation (AZ_NEG_LAPLACE_GAUSS) only: wavenumber of the Helmholtz operator
                           -(Laplacian + k0^2) of Sec. 6.2 (0 = Poisson); the interior rows are
                           -(Laplacian + k0^2) phi_j / (2 eps^2) */
  const double* bnormal; /* collocation only: device array, n_boundary x dim (the layout of the boundary
                           points), or NULL.  A point with a nonzero (unit, outward) normal n gets the
                           Neumann row n . grad phi_j(p) / eps (Sec. 6.3), the others the Dirichlet row
                           phi_j(p); both are multiplied by the boundary weight.  az_collocate scales the
                           Neumann data du/dn by weight / eps.  Copied at setup; NULL = all Dirichlet */
} az_options;

typedef struct {
  int64_t N;            /* number of coefficients */
  int64_t L;            /* grid points of the full box */
  int64_t M;            /* kept grid points */
  int64_t Mb;           /* boundary rows (collocation) */
  int32_t k;            /* sketch width */
  int32_t rank;         /* numerical rank kept by the truncated solve */
  int32_t rank_gram;    /* directions kept by the first (Gram) orthogonalisation pass */
  int32_t precision;
  double sigma_max;     /* largest singular value of the sketch Y */
  double sigma_min_kept;/* smallest kept singular value */
  size_t device_bytes;  /* bytes held by the handle */
  int32_t jacobi_sweeps;/* sweeps taken by the small factor's one-sided Jacobi SVD */
} az_info_t;

/* Build a solver for one problem.  (Sec. 3.2.3 "Step 0" and step 1's sketch.)
 *   g               grid description (copied).
 *   omega_mask_dev  uint8, one byte per grid point in grid-index order, 1 = in
 *                   Omega.  Required.
 *   boundary_pts_dev  double, n_boundary x dim row-major (x, y pairs) or NULL.
 *   eps             Gaussian shape parameter (> 0).
 *   kernel          AZ_GAUSS (approximation, Sec. 2-5) or AZ_NEG_LAPLACE_GAUSS
 *                   (collocation -(Lap + k0^2) u = f, Sec. 6.1-6.3, k0 from the
 *                   options; rows divided by 2 eps^2, the normalisation of
 *                   Example 6.1; 1D or 2D).
 *   boundary_weight weight w of the boundary rows (collocation), else ignored.
 *   opt             options (copied); NULL = defaults.
 *   out             receives the handle.
 * Omega = the whole box with no boundary rows (and tau_sym = 0) is the periodic
 * problem of Sec. 3.1: the perturbation is exactly zero, the sketch is skipped
 * and solves apply Z* alone (rank 0).
 * Synchronises `stream` once (to learn M).  Errors: AZ_ERR_ARG for bad sizes
 * or pointers, and for AZ_MIXED with eps h < 0.504 (the FP32 symbol inverse
 * would amplify rounding past 1e-3; use AZ_FP64), AZ_ERR_OOM, AZ_ERR_CUDA,
 * AZ_ERR_NUMERIC. */
az_status az_setup(const az_grid* g, const uint8_t* omega_mask_dev, const double* boundary_pts_dev,
                   int64_t n_boundary, double eps, int32_t kernel, double boundary_weight,
                   const az_options* opt, void* stream, az_handle* out);

/* Least-squares solve A x ≈ b for nrhs right-hand sides (Algorithm 1, plus
 * `refine_steps` steps x += AZ(b - A x) with the residual in FP64).
 *   b_dev  (M [+ Mb]) x nrhs, leading dimension ldb, FP64.
 *   x_dev  N x nrhs, leading dimension ldx, FP64 (overwritten).
 *   relres_host  optional host array of nrhs: ||A x - b|| / ||b|| (forces a sync;
 *                then also reports AZ_ERR_TIMEOUT, once, if a tensor-core
 *                pipeline wait of this handle timed out). */
az_status az_solve(az_handle h, const double* b_dev, int64_t ldb, int64_t nrhs, double* x_dev,
                   int64_t ldx, void* stream, double* relres_host);

/* Poisson collocation solve (Sec. 6.2): interior data f at the M kept points
 * and Dirichlet data g at the Mb boundary points; the interior rows and f are
 * divided by 2 eps^2 and the boundary rows and g multiplied by the setup's
 * boundary weight before the least-squares solve.  Requires a setup with
 * kernel = AZ_NEG_LAPLACE_GAUSS.  The scaled data go through a buffer the
 * handle owns (M + Mb rows by one solve chunk): stream-ordered, no allocation
 * and, without relres_host, no synchronisation, so the call can be captured
 * in a CUDA graph; calls on one handle from overlapping streams race on that
 * buffer. */
az_status az_collocate(az_handle h, const double* f_int_dev, int64_t ldf, const double* g_bnd_dev,
                       int64_t ldg, int64_t nrhs, double* x_dev, int64_t ldx, void* stream,
                       double* relres_host);

/* Values of the expansion sum_j x_j phi_j on the s_test-fold refinement of the
 * box grid ((s_test N_d) points per dimension, grid-index order), FP64.
 *   out_dev  (prod_d s_test N_d) x nrhs, leading dimension ldo. */
az_status az_evaluate(az_handle h, const double* x_dev, int64_t ldx, int64_t nrhs, int32_t s_test,
                      double* out_dev, int64_t ldo, void* stream);

/* Operator applications in FP64 (the paper's A and Z*, for tests and users).
 *   az_apply_A:     y = A x    (x: N x nrhs, y: (M+Mb) x nrhs)   Sec. 2.3, Sec. 6.2
 *   az_apply_Zstar: x = Z* y   (y: (M+Mb) x nrhs, x: N x nrhs)    Sec. 3.2.2 (boundary columns zero) */
az_status az_apply_A(az_handle h, const double* x_dev, int64_t ldx, int64_t nrhs, double* y_dev,
                     int64_t ldy, void* stream);
az_status az_apply_Zstar(az_handle h, const double* y_dev, int64_t ldy, int64_t nrhs, double* x_dev,
                         int64_t ldx, void* stream);

/* Copies of internal arrays (device destination pointers, FP64):
 *   AZ_ARRAY_SYMBOL  the full-box symbol Ghat on the grid in natural frequency
 *                    order (L values; 2D: [kx][ky]) -- Lemma 4.2 / Eq. explicit_d
 *   AZ_ARRAY_SKETCH  Y = (I - A Z*) A R, (M+Mb) x k, ld = M+Mb     -- Sec. 3.2.3
 *   AZ_ARRAY_W       W = (I - Z* A) R, N x k, ld = N
 *   AZ_ARRAY_R       the Rademacher test matrix R, N x k, ld = N (+1/-1)
 *   AZ_ARRAY_UT      U_tau, (M+Mb) x rank, ld = M+Mb (orthonormal basis kept)
 *   AZ_ARRAY_SIGMA   the kept singular values (rank values)
 *   AZ_ARRAY_KEPT    the kept grid indices (M values, as doubles) */
enum { AZ_ARRAY_SYMBOL = 0, AZ_ARRAY_SKETCH = 1, AZ_ARRAY_W = 2, AZ_ARRAY_R = 3, AZ_ARRAY_UT = 4,
       AZ_ARRAY_SIGMA = 5, AZ_ARRAY_KEPT = 6 };
az_status az_get_array(az_handle h, int32_t which, double* dst_dev, void* stream);

/* Sizes and factorisation results of a handle.  Waits (on the host) for the
 * handle's latest factorisation (az_setup or az_refactor) only, not for solves
 * in flight on other streams.  Returns AZ_ERR_TIMEOUT (once; the flag is then
 * cleared) if a launch that has completed raised the tensor-core pipeline's
 * wait-timeout flag. */
az_status az_get_info(az_handle h, az_info_t* info);

/* Device bytes a setup of this size would hold (symbols, maps, sketch and
 * factors, plus the workspace for `nrhs_max` simultaneous right-hand sides). */
az_status az_query_footprint(const az_grid* g, int64_t M, int64_t n_boundary, const az_options* opt,
                             int64_t nrhs_max, size_t* bytes);

void az_destroy(az_handle h);

/* Thread-local text of the last failure in this thread ("" if none). */
const char* az_last_error(void);

/* The Rademacher test matrix alone: R (N x k, ld = N, FP64 +1/-1) from the
 * Philox4x32-10 layout counter = (row/128, column, 0, 0), key = (seed low,
 * seed high), bit (row % 32) of word ((row % 128)/32), set = +1.
 * k <= 65535; larger k returns AZ_ERR_ARG. */
az_status az_rademacher(int64_t N, int32_t k, uint64_t seed, double* R_dev, void* stream);

/* az_rademacher without any device allocation, for callers that cannot call
 * cudaMalloc: for example a serving process whose caching allocator already
 * holds the free device memory (a fresh cudaMalloc would fail or force the
 * cache to be released), or code on a latency-critical path where cudaMalloc
 * and cudaFree may synchronise the device.  The paper has no counterpart; it is
 * a deployment variant of az_rademacher with identical output.
 *   Scratch: a fixed 4 MiB device array inside the library (kept by every GPU
 *   that loads it until the process exits).  Limits: k * ceil(N/32) <= 2^20,
 *   i.e. at most 2^25 entries of R, and k <= 65535; larger sizes return
 *   AZ_ERR_ARG.
 *   Each call made outside stream capture looks up the array's device address
 *   for the current device (so an address from a context that cudaDeviceReset
 *   destroyed is never reused); a call under capture reuses the address of the
 *   last uncaptured call on that device.  Make the first call on each device
 *   before any stream capture, and again after a cudaDeviceReset.  All calls share the one array, so calls that overlap on the GPU
 *   (different streams or threads without ordering) race on it and must be
 *   serialised by the caller.  Stream-ordered, no synchronisation. */
az_status az_rademacher_noalloc(int64_t N, int32_t k, uint64_t seed, double* R_dev, void* stream);

/* Recompute every setup step (index map, symbol, test matrix with a new
 * seed, sketch, factorisation) on an existing handle, without allocating and
 * without synchronising.  The index map and symbol are computed on `stream`.
 * For approximation setups with k <= 64 the sketch and factorisation (steps 2-3
 * of Algorithm 1's setup) then run on the handle's own high-priority stream, so
 * that the next az_solve's first Z* pass overlaps them: every later call on the
 * handle that uses the factors (az_solve, az_get_array, az_get_info, the next
 * az_refactor) waits for them on its own stream, whichever stream that is.
 * Synchronising `stream` alone does not cover the factorisation; az_get_info
 * does.  Other setups run every step on `stream`.  A factorisation breakdown
 * is reported by the next az_get_info (status is checked lazily). */
az_status az_refactor(az_handle h, uint64_t seed, void* stream);

/* Instrumentation (not part of the paper's method).
 * az_launch_count: kernels launched by this library since it was loaded.
 * az_profile_begin / az_profile_end: while enabled, every kernel launch is
 * bracketed by CUDA events on its stream and attributed to its kernel class
 * with its algorithmic bytes (inputs read once + outputs written once);
 * az_profile_end synchronises on those events.  az_profile_query(i, ...)
 * returns entry i (name, launches, total milliseconds, total bytes) or
 * AZ_ERR_ARG past the last entry. */
int64_t az_launch_count(void);

/* Test hook for the failure path of the tensor-core projection (not part of
 * the paper's method): the next launch of that kernel (in any handle) stops
 * issuing its TMA copies at pipeline iteration `iteration` and bounds each of
 * its waits by wait_ns nanoseconds instead of one second.  Its consumers' waits
 * then run out; every CTA stops issuing work, waits (bounded) for its own
 * copies and MMAs, frees its tensor memory and returns, and the call that
 * reads the handle's status (az_solve with relres_host, or az_get_info)
 * returns AZ_ERR_TIMEOUT once.  One-shot; AZ_ERR_ARG for iteration < 0 or
 * wait_ns <= 0. */
az_status az_debug_tc_withhold(int32_t iteration, int64_t wait_ns);

/* Test hook for the FP64 output of the mixed path (not part of the paper's
 * method): out[i] = the FP64 number nearest to a[i] + b[i] (ties to even),
 * computed by the routine the solve uses to write x = x_fp32 + correction
 * without FP64 arithmetic; it must equal (double)a[i] + (double)b[i] bit for
 * bit.  a, b: n FP32 values, out: n FP64 values, all device memory owned by
 * the caller; enqueued on `stream` (a cudaStream_t, NULL = legacy default),
 * no synchronisation.  AZ_ERR_ARG for n < 0 or a null pointer with n > 0. */
az_status az_debug_f32_sum_f64(const float* a, const float* b, double* out, int64_t n, void* stream);

/* Test hook for the first Gram of the mixed factorisation (G1 = Y^T Y of the
 * sketch, the SVQB pass that replaces the SVD of Sec. 3.2.3): G (k x k FP64,
 * column-major, device) = Y^T Y for Y (M x k FP32, column-major, leading
 * dimension ldy, device) by route 0, exact FP32 products with double-float
 * sums on the FP32 pipe, or route 1, the exact split on the tensor cores (BF16
 * slices of the power-of-two-scaled columns, per-CTA slice-pair sums exact in
 * FP32, FP64 fold; k <= 24, ldy a multiple of 4, Y 16-byte aligned).  Both
 * are what az_setup uses.  Allocates its own scratch and synchronises
 * `stream` (a cudaStream_t, NULL = legacy default).  AZ_ERR_ARG for bad
 * sizes; AZ_ERR_TIMEOUT if a tensor-core pipeline wait ran out. */
az_status az_debug_gram(const float* Y, int64_t ldy, int32_t k, int64_t M, double* G, int32_t route, void* stream);
void az_profile_begin(void);
az_status az_profile_end(void);
az_status az_profile_query(int32_t i, char* name, int32_t name_len, int64_t* launches, double* ms,
                           double* bytes);

#ifdef __cplusplus
}
#endif
#endif
