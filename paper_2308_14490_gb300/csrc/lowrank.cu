// Low-rank factorisation and projections (S6, S7, S9).
//
// The paper's step 1 (Sec. 3.2.3) takes an SVD of the sketch Y = (A - A Z* A) R.
// Here Y is tall (M rows) and narrow (k columns), and numerically rank
// deficient (its trailing singular values are rounding noise).  The
// factorisation is the CholeskyQR2 pattern with a rank-revealing first pass:
//   pass 1 (SVQB): G1 = Y^T Y, G1 = V Lambda V^T, Q1 = Y V_r1 Lambda_r1^{-1/2}
//   pass 2 (Cholesky): G2 = Q1^T Q1 = R2^T R2, Q = Q1 R2^{-1}
// so Y V_r1 = Q R2 Lambda^{1/2}; the small factor Rs = R2 Lambda^{1/2} is
// decomposed by a one-sided Jacobi SVD, Rs = U_R Sigma V_R^T, and the
// truncated solve keeps sigma_i > tau sigma_1.  Stored: U_tau = Q U_R[:, :r]
// (formed as Q1 T with T = R2^{-1} U_R[:, :r]) and VS = V_r1 V_R[:, :r]
// Sigma^{-1}, so that u = VS U_tau^T g.
#include <cmath>
#include "lowrank.cuh"

namespace az {

#define AZ_LCHECK()                                                                                  \
  do {                                                                                               \
    cudaError_t _e = cudaGetLastError();                                                             \
    if (_e != cudaSuccess) { set_error(std::string("kernel launch: ") + cudaGetErrorString(_e)); return AZ_ERR_CUDA; } \
  } while (0)

static constexpr int GRAM_ROWS = 2048;  // rows per CTA of the Gram partials
static constexpr int GRAM_TILE = 64;    // rows staged per step

int gram_blocks(int64_t M) { return (int)std::max<int64_t>(1, (M + GRAM_ROWS - 1) / GRAM_ROWS); }

// Each CTA: rows [b*GRAM_ROWS, ...), all (a, c) pairs; A and B tiles staged in
// shared memory as double; per-thread FP64 accumulators.
template <typename TA, typename TB>
__global__ void k_gram_partial(const TA* __restrict__ A, int64_t lda, int ka, const TB* __restrict__ B, int64_t ldb,
                               int kb, int64_t M, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sA = (double*)smem_raw;             // GRAM_TILE x ka  [row*ka + a]
  double* sB = sA + GRAM_TILE * ka;           // GRAM_TILE x kb
  const int npair = ka * kb;
  const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS;
  const int64_t r1 = (M < r0 + GRAM_ROWS) ? M : r0 + GRAM_ROWS;
  constexpr int MAXP = 8;
  double acc[MAXP];
#pragma unroll
  for (int q = 0; q < MAXP; ++q) acc[q] = 0.0;
  for (int64_t rb = r0; rb < r1; rb += GRAM_TILE) {
    const int nr = (int)((r1 - rb) < GRAM_TILE ? (r1 - rb) : GRAM_TILE);
    __syncthreads();
    for (int t = threadIdx.x; t < GRAM_TILE * ka; t += blockDim.x) {
      int a = t / GRAM_TILE, rr = t % GRAM_TILE;
      sA[rr * ka + a] = rr < nr ? (double)A[(int64_t)a * lda + rb + rr] : 0.0;
    }
    for (int t = threadIdx.x; t < GRAM_TILE * kb; t += blockDim.x) {
      int c = t / GRAM_TILE, rr = t % GRAM_TILE;
      sB[rr * kb + c] = rr < nr ? (double)B[(int64_t)c * ldb + rb + rr] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
      int p = threadIdx.x + q * blockDim.x;
      if (p < npair) {
        int a = p % ka, c = p / ka;
        double s = 0.0;
        for (int rr = 0; rr < nr; ++rr) s = fma(sA[rr * ka + a], sB[rr * kb + c], s);
        acc[q] += s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < MAXP; ++q) {
    int p = threadIdx.x + q * blockDim.x;
    if (p < npair) partial[(int64_t)blockIdx.x * npair + p] = acc[q];
  }
}
__global__ void k_gram_reduce(const double* __restrict__ partial, int nblk, int npair, double* __restrict__ G) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * npair + p];
  G[p] = s;  // column-major ka x kb: p = a + c*ka
}
template <typename TA, typename TB>
az_status launch_gram(const TA* A, int64_t lda, int ka, const TB* B, int64_t ldb, int kb, int64_t M,
                      double* partial, double* G, cudaStream_t st) {
  const int npair = ka * kb;
  int threads = 256;
  while (threads * 8 < npair && threads < 1024) threads *= 2;
  if (threads * 8 < npair) { set_error("gram: too many columns for this kernel"); return AZ_ERR_ARG; }
  const int nblk = gram_blocks(M);
  size_t sm = (size_t)GRAM_TILE * (ka + kb) * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_gram_partial<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gram_partial<TA, TB><<<nblk, threads, sm, st>>>(A, lda, ka, B, ldb, kb, M, partial);
  k_gram_reduce<<<(npair + 255) / 256, 256, 0, st>>>(partial, nblk, npair, G);
  AZ_LCHECK();
  return AZ_OK;
}

// out = A * S : thread per (row, output column), S in shared memory.
template <typename TA, typename TO>
__global__ void k_tsprod(const TA* __restrict__ A, int64_t lda, int k, const double* __restrict__ S, int r, int64_t M,
                         TO* __restrict__ out, int64_t ldo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sS = (double*)smem_raw;
  for (int t = threadIdx.x; t < k * r; t += blockDim.x) sS[t] = S[(t / r) + (int64_t)(t % r) * k] ;  // sS[a*r + c] = S[a, c]
  __syncthreads();
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double acc[64];
  const int rr = min(r, 64);
  for (int c = 0; c < rr; ++c) acc[c] = 0.0;
  for (int a = 0; a < k; ++a) {
    double v = (double)A[(int64_t)a * lda + m];
    for (int c = 0; c < rr; ++c) acc[c] = fma(v, sS[a * r + c], acc[c]);
  }
  for (int c = 0; c < rr; ++c) out[(int64_t)c * ldo + m] = (TO)acc[c];
}
template <typename TA, typename TO>
az_status launch_tsprod(const TA* A, int64_t lda, int k, const double* S, int r, int64_t M, TO* out, int64_t ldo,
                        cudaStream_t st) {
  if (r > 64) { set_error("tsprod: r > 64 not supported by this kernel"); return AZ_ERR_ARG; }
  size_t sm = (size_t)k * r * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_tsprod<TA, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_tsprod<TA, TO><<<(unsigned)((M + 127) / 128), 128, sm, st>>>(A, lda, k, S, r, M, out, ldo);
  AZ_LCHECK();
  return AZ_OK;
}

// ---------------------------------------------------------------- one-CTA small dense work
// One-sided (Hestenes) Jacobi on the columns of a (m x n, column-major in
// shared memory, ld m): rotates column pairs until they are mutually
// orthogonal; V (n x n) accumulates the rotations.  Round-robin pair order, one
// warp per pair.  After convergence column j has norm sigma_j and
// a[:, j] / sigma_j is the left singular vector.
__device__ void jacobi_onesided(double* a, int m, int n, double* V, int* flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // identity V
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) V[t] = (t % n == t / n) ? 1.0 : 0.0;
  __syncthreads();
  const int nn = (n + 1) & ~1;  // even count for round-robin (a dummy column if n odd)
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int step = 0; step < nn - 1; ++step) {
      for (int pr = warp; pr < nn / 2; pr += nwarps) {
        // round-robin pairing: positions 0..nn-1, position 0 fixed
        int p0 = pr, p1 = nn - 1 - pr;
        auto idx = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + step) % (nn - 1)); };
        int i = idx(p0), j = idx(p1);
        if (i > j) { int tt = i; i = j; j = tt; }
        if (j >= n) continue;
        double al = 0, be = 0, ga = 0;
        for (int r = lane; r < m; r += 32) {
          double x = a[i * m + r], y = a[j * m + r];
          al += x * x; be += y * y; ga += x * y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (fabs(ga) > 1e-15 * sqrt(al * be) && ga != 0.0) {
          double zeta = (be - al) / (2.0 * ga);
          double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int r = lane; r < m; r += 32) {
            double x = a[i * m + r], y = a[j * m + r];
            a[i * m + r] = c * x - s * y;
            a[j * m + r] = s * x + c * y;
          }
          for (int r = lane; r < n; r += 32) {
            double x = V[i * n + r], y = V[j * n + r];
            V[i * n + r] = c * x - s * y;
            V[j * n + r] = s * x + c * y;
          }
          if (lane == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (*flag == 0) break;
    __syncthreads();
  }
}

// sort columns of (a, V) by decreasing norm; norms into sig
__device__ void sort_by_norm(double* a, int m, int n, double* V, double* sig, double* tmp) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0;
    for (int r = 0; r < m; ++r) s += a[j * m + r] * a[j * m + r];
    sig[j] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // selection sort on indices (n <= 64)
    for (int i = 0; i < n; ++i) {
      int best = i;
      for (int j = i + 1; j < n; ++j) if (sig[j] > sig[best]) best = j;
      if (best != i) {
        double t = sig[i]; sig[i] = sig[best]; sig[best] = t;
        for (int r = 0; r < m; ++r) { double u = a[i * m + r]; a[i * m + r] = a[best * m + r]; a[best * m + r] = u; }
        for (int r = 0; r < n; ++r) { double u = V[i * n + r]; V[i * n + r] = V[best * n + r]; V[best * n + r] = u; }
      }
    }
  }
  __syncthreads();
  (void)tmp;
}

__global__ void k_factor1(const double* __restrict__ G1, int k, double taug, double floor2, double* V, double* lam,
                          double* B1, FactorInfo* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* a = (double*)smem_raw;   // k x k
  double* sV = a + k * k;          // k x k
  double* sg = sV + k * k;         // k
  __shared__ int flag;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) a[t] = G1[t];
  __syncthreads();
  jacobi_onesided(a, k, k, sV, &flag);
  sort_by_norm(a, k, k, sV, sg, nullptr);
  // G1 SPD: the column norms of G1 V are the eigenvalues lambda
  __shared__ int r1s;
  if (threadIdx.x == 0) {
    int r1 = 0;
    double l1 = sg[0];
    bool finite = isfinite(l1);
    for (int j = 0; j < k; ++j) if (sg[j] > taug * taug * l1 && sg[j] > floor2 && isfinite(sg[j])) ++r1;
    r1s = r1;
    info->r1 = r1;
    info->status = finite ? 0 : 2;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int row = t % k, col = t / k;
    V[t] = sV[t];
    B1[t] = col < r1s ? sV[col * k + row] / sqrt(sg[col]) : 0.0;
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) lam[t] = sg[t];
}
az_status launch_factor1(const double* G1, int k, double taug, double floor2, double* V, double* lam, double* B1,
                         FactorInfo* info, cudaStream_t st) {
  if (k > 64) { set_error("factor: k > 64 not supported by the one-CTA factorisation"); return AZ_ERR_ARG; }
  size_t sm = (2 * (size_t)k * k + k) * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_factor1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_factor1<<<1, 1024, sm, st>>>(G1, k, taug, floor2, V, lam, B1, info);
  AZ_LCHECK();
  return AZ_OK;
}

__global__ void k_factor2(const double* __restrict__ G2, int k, const double* __restrict__ V, const double* __restrict__ lam,
                          double tau, double floor, double* T, double* VS, double* sig, FactorInfo* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* R = (double*)smem_raw;   // r1 x r1 (column-major ld k), Cholesky factor, upper
  double* A = R + k * k;           // Rs, then rotated
  double* VR = A + k * k;          // k x k
  double* sg = VR + k * k;
  __shared__ int flag;
  __shared__ int fail;
  const int r1 = info->r1;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) { R[t] = 0.0; A[t] = 0.0; }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  // copy upper part of G2[:r1,:r1] into R (column-major, ld k)
  for (int t = threadIdx.x; t < r1 * r1; t += blockDim.x) {
    int i = t % r1, j = t / r1;
    if (i <= j) R[j * k + i] = G2[(int64_t)j * k + i];
  }
  __syncthreads();
  // right-looking Cholesky, upper: G2 = R^T R
  for (int j = 0; j < r1; ++j) {
    if (threadIdx.x == 0) {
      double d = R[j * k + j];
      if (!(d > 0.0) || !isfinite(d)) { fail = 1; d = 1.0; }
      R[j * k + j] = sqrt(d);
    }
    __syncthreads();
    double djj = R[j * k + j];
    for (int c = j + 1 + threadIdx.x; c < r1; c += blockDim.x) R[c * k + j] /= djj;
    __syncthreads();
    for (int t = threadIdx.x; t < r1 * r1; t += blockDim.x) {
      int i = t % r1, c = t / r1;
      if (i > j && c >= i) R[c * k + i] -= R[i * k + j] * R[c * k + j];
    }
    __syncthreads();
  }
  // Rs = R diag(sqrt(lam)) (r1 x r1, column-major ld r1 in A)
  for (int t = threadIdx.x; t < r1 * r1; t += blockDim.x) {
    int i = t % r1, j = t / r1;
    A[j * r1 + i] = (i <= j ? R[j * k + i] : 0.0) * sqrt(lam[j]);
  }
  __syncthreads();
  jacobi_onesided(A, r1, r1, VR, &flag);
  sort_by_norm(A, r1, r1, VR, sg, nullptr);
  __shared__ int rs;
  if (threadIdx.x == 0) {
    int r = 0;
    double s1 = r1 > 0 ? sg[0] : 0.0;
    for (int j = 0; j < r1; ++j) if (sg[j] > tau * s1 && sg[j] > floor) ++r;
    rs = r;
    info->r = r;
    info->sigma_max = s1;
    info->sigma_min_kept = r > 0 ? sg[r - 1] : 0.0;
    if (fail) info->status = 1;
  }
  __syncthreads();
  const int r = rs;
  // U_R[:, c] = A[:, c] / sg[c]  (in A, ld r1); T = R^{-1} U_R[:, :r]  (back substitution, thread per column)
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) T[(int64_t)c * k + i] = 0.0;
    if (c < r) {
      for (int i = r1 - 1; i >= 0; --i) {
        double s = A[c * r1 + i] / sg[c];
        for (int l = i + 1; l < r1; ++l) s -= R[l * k + i] * T[(int64_t)c * k + l];
        T[(int64_t)c * k + i] = s / R[i * k + i];
      }
    }
  }
  // VS = V[:, :r1] VR[:, :r] Sigma^{-1}  (k x k, zero beyond r)
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int i = t % k, c = t / k;
    double s = 0.0;
    if (c < r) {
      for (int l = 0; l < r1; ++l) s += V[(int64_t)l * k + i] * VR[c * r1 + l];
      s /= sg[c];
    }
    VS[t] = s;
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) sig[t] = t < r1 ? sg[t] : 0.0;
}
az_status launch_factor2(const double* G2, int k, const double* V, const double* lam, double tau, double floor,
                         double* T, double* VS, double* sig, FactorInfo* info, cudaStream_t st) {
  if (k > 64) { set_error("factor: k > 64 not supported by the one-CTA factorisation"); return AZ_ERR_ARG; }
  size_t sm = (3 * (size_t)k * k + k) * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_factor2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_factor2<<<1, 1024, sm, st>>>(G2, k, V, lam, tau, floor, T, VS, sig, info);
  AZ_LCHECK();
  return AZ_OK;
}

__global__ void k_small_mm(const double* VS, int k, const double* c, int n, double* u) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * n) return;
  int i = t % k, j = t / k;
  double s = 0;
  for (int l = 0; l < k; ++l) s += VS[(int64_t)l * k + i] * c[(int64_t)j * k + l];
  u[t] = s;
}
az_status launch_small_mm(const double* VS, int k, const double* c, int n, double* u, cudaStream_t st) {
  k_small_mm<<<(k * n + 255) / 256, 256, 0, st>>>(VS, k, c, n, u);
  AZ_LCHECK();
  return AZ_OK;
}

template <typename TW, typename TZ>
__global__ void k_update_x(const TW* __restrict__ W, int64_t ldw, int k, const double* __restrict__ u,
                           const TZ* __restrict__ z, int64_t ldz, int64_t N, double* __restrict__ x, int64_t ldx,
                           int accumulate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* su = (double*)smem_raw;
  const int c = blockIdx.y;
  for (int t = threadIdx.x; t < k; t += blockDim.x) su[t] = u[(int64_t)c * k + t];
  __syncthreads();
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s = (double)z[(int64_t)c * ldz + j];
  for (int a = 0; a < k; ++a) s = fma((double)W[(int64_t)a * ldw + j], su[a], s);
  double* xp = x + (int64_t)c * ldx + j;
  *xp = accumulate ? *xp + s : s;
}
template <typename TW, typename TZ>
az_status launch_update_x(const TW* W, int64_t ldw, int k, const double* u, const TZ* z, int64_t ldz, int64_t N,
                          int nrhs, double* x, int64_t ldx, bool accumulate, cudaStream_t st) {
  dim3 grid((unsigned)((N + 255) / 256), nrhs);
  k_update_x<TW, TZ><<<grid, 256, k * sizeof(double), st>>>(W, ldw, k, u, z, ldz, N, x, ldx, accumulate ? 1 : 0);
  AZ_LCHECK();
  return AZ_OK;
}

template az_status launch_gram<float, float>(const float*, int64_t, int, const float*, int64_t, int, int64_t, double*, double*, cudaStream_t);
template az_status launch_gram<double, double>(const double*, int64_t, int, const double*, int64_t, int, int64_t, double*, double*, cudaStream_t);
template az_status launch_gram<float, double>(const float*, int64_t, int, const double*, int64_t, int, int64_t, double*, double*, cudaStream_t);
template az_status launch_tsprod<float, double>(const float*, int64_t, int, const double*, int, int64_t, double*, int64_t, cudaStream_t);
template az_status launch_tsprod<double, double>(const double*, int64_t, int, const double*, int, int64_t, double*, int64_t, cudaStream_t);
template az_status launch_tsprod<double, float>(const double*, int64_t, int, const double*, int, int64_t, float*, int64_t, cudaStream_t);
template az_status launch_update_x<float, float>(const float*, int64_t, int, const double*, const float*, int64_t, int64_t, int, double*, int64_t, bool, cudaStream_t);
template az_status launch_update_x<double, double>(const double*, int64_t, int, const double*, const double*, int64_t, int64_t, int, double*, int64_t, bool, cudaStream_t);

}  // namespace az
