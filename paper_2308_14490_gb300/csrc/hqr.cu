// Blocked Householder QR of the tall sketch Y (M x k, FP64, M >= k) and the
// application of its Q, for the wide low-rank step (the truncated solve of
// Algorithm 1 step 1, Sec. 3.2.3: U_tau = Q U_R from the SVD R = U_R S V^T).
//
// Panels of NB columns.  Within a panel, column j is reduced by one
// Householder reflector H_j = I - tau_j v_j v_j^T (v_j(j) = 1, LAPACK's
// convention): a deterministic reduction of the dot products of column j with
// the panel's remaining columns, one block that forms beta, tau and the
// scaled dot products, and one update of the rows below the diagonal (FP64
// arithmetic: the panel work is O(M k NB)).  The panel's reflectors are then
// accumulated in compact WY form, Q_p = I - V T V^T with T upper triangular
// (T(i,i) = tau_i, T(0:i, i) = -tau_i T(0:i,0:i) V(:,0:i)^T v_i), and the
// trailing columns are updated as A -= V (T^T (V^T A)) with the tall
// products on the double-float tiles of dfgemm.cu (FP64 tiles where the
// setup needs them): O(M k^2) work that GB300 would otherwise run on its
// FP64 pipe.  Q [U; 0] applies the panels in reverse, X -= V (T (V^T X)).
#include <algorithm>
#include <vector>

#include "dfgemm.cuh"
#include "hqr.cuh"
#include "profile.cuh"

namespace az {

namespace {

constexpr int NB = 64;          // panel width
constexpr int DOT_WARPS = 8;

// part[b * NB + (c - j)] = sum over this block's rows m > j of A[m, j] A[m, c],
// c in [j, c1)
__global__ void __launch_bounds__(DOT_WARPS * 32) k_hqr_dots(const double* __restrict__ A, int64_t M, int64_t lda,
                                                             int j, int c1, int64_t rows_per_blk,
                                                             double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = j + 1 + (int64_t)blockIdx.x * rows_per_blk;
  const int64_t m1 = std::min<int64_t>(M, m0 + rows_per_blk);
  const double* aj = A + (int64_t)j * lda;
  for (int c = j + warp; c < c1; c += DOT_WARPS) {
    const double* ac = A + (int64_t)c * lda;
    double s = 0.0;
    for (int64_t m = m0 + lane; m < m1; m += 32) s = fma(aj[m], ac[m], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[(int64_t)blockIdx.x * NB + (c - j)] = s;
  }
}

// beta, tau and the scaled products of column j (one block of NB threads):
//   hs[0] = 1 / (alpha - beta) (the scale of v below the diagonal),
//   hs[1 + c - j] = tau * v^T A[:, c] for c in (j, c1);
// row j takes its part of the update and A[j, j] = beta.
__global__ void k_hqr_reflect(double* __restrict__ A, int64_t lda, int j, int c1, const double* __restrict__ part,
                              int nblk, double* __restrict__ tau, double* __restrict__ hs) {
  __shared__ double s[NB];
  __shared__ double sc[2];   // scale, tau
  const int t = threadIdx.x, nc = c1 - j;
  if (t < nc) {
    double a = 0.0;
    for (int b = 0; b < nblk; ++b) a += part[(int64_t)b * NB + t];
    s[t] = a;
  }
  __syncthreads();
  if (t == 0) {
    const double alpha = A[(int64_t)j * lda + j];
    const double x2 = s[0];
    double tj = 0.0, scale = 0.0, beta = alpha;
    if (x2 > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + x2), alpha);
      tj = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    tau[j] = tj;
    sc[0] = scale;
    sc[1] = tj;
    hs[0] = scale;
    A[(int64_t)j * lda + j] = beta;
  }
  __syncthreads();
  if (t > 0 && t < nc) {
    const int c = j + t;
    double* arow = A + (int64_t)c * lda + j;
    const double w = *arow + sc[0] * s[t];   // v^T A[:, c], v = [1; scale A[j+1:, j]]
    const double tw = sc[1] * w;
    hs[1 + t] = tw;
    *arow -= tw;
  }
}

// rows m > j: v_m = scale A[m, j] (stored in place), A[m, c] -= v_m hs[1 + c - j]
__global__ void k_hqr_apply(double* __restrict__ A, int64_t M, int64_t lda, int j, int c1,
                            const double* __restrict__ hs) {
  __shared__ double h[NB + 1];
  const int nc = c1 - j;
  if (threadIdx.x <= nc) h[threadIdx.x] = hs[threadIdx.x];
  __syncthreads();
  const int64_t m = j + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const double v = A[(int64_t)j * lda + m] * h[0];
  A[(int64_t)j * lda + m] = v;
  for (int t = 1; t < nc; ++t) {
    double* p = A + (int64_t)(j + t) * lda + m;
    *p = fma(-v, h[1 + t], *p);
  }
}

// V of a panel, explicit: V[m, c] (rows m >= j0, ld ldv) = 0 above the
// diagonal, 1 on it, the stored reflector below
__global__ void k_hqr_vbuf(const double* __restrict__ A, int64_t M, int64_t lda, int j0, int nbp,
                           double* __restrict__ V, int64_t ldv) {
  const int64_t m = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (m >= M || c >= nbp) return;
  const int64_t d = m - (j0 + c);
  V[(int64_t)c * ldv + m] = d < 0 ? 0.0 : (d == 0 ? 1.0 : A[(int64_t)(j0 + c) * lda + m]);
}

// T of the panel (upper triangular nbp x nbp, ld NB) from G = V^T V and tau
__global__ void k_hqr_larft(const double* __restrict__ G, int nbp, const double* __restrict__ tau,
                            double* __restrict__ T) {
  __shared__ double Ts[NB * NB];
  __shared__ double y[NB];
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) Ts[t] = 0.0;
  __syncthreads();
  for (int i = 0; i < nbp; ++i) {
    // T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i)
    const int r = threadIdx.x;
    if (r < i) {
      double a = 0.0;
      for (int l = r; l < i; ++l) a = fma(Ts[r + l * NB], G[l + (int64_t)i * nbp], a);
      y[r] = -tau[i] * a;
    }
    __syncthreads();
    if (r < i) Ts[r + i * NB] = y[r];
    if (r == 0) Ts[i + i * NB] = tau[i];
    __syncthreads();
  }
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) T[t] = Ts[t];
}

// W2 = -op(T) W1 (nbp x n, ld nbp); op = T^T (trans) or T
__global__ void k_hqr_tw(const double* __restrict__ T, int nbp, const double* __restrict__ W1, int64_t n, bool trans,
                         double* __restrict__ W2) {
  const int i = threadIdx.x;
  const int64_t c = blockIdx.x;
  if (i >= nbp || c >= n) return;
  double a = 0.0;
  if (trans) {
    for (int l = 0; l <= i; ++l) a = fma(T[l + i * NB], W1[l + c * nbp], a);   // (T^T)(i, l) = T(l, i), l <= i
  } else {
    for (int l = i; l < nbp; ++l) a = fma(T[i + l * NB], W1[l + c * nbp], a);  // T(i, l), l >= i
  }
  W2[i + c * nbp] = -a;
}

}  // namespace

struct HQR {
  int64_t M = 0;
  int k = 0;
  bool f64 = false;
  int npanel = 0;
  int nblk = 0;
  int64_t rows_per_blk = 0;
  double* part = nullptr;   // nblk x NB dot partials
  double* hs = nullptr;     // NB + 1
  double* tau = nullptr;    // k
  double* T = nullptr;      // npanel x NB x NB
  double* V = nullptr;      // M x NB explicit panel reflectors
  double* G = nullptr;      // NB x NB
  double* W1 = nullptr;     // NB x k
  double* W2 = nullptr;     // NB x k
  double* tpart = nullptr;  // split-K partials of the tall products
  std::vector<void*> allocs;
};

static az_status hq_alloc(HQR* q, void** p, size_t bytes, size_t* tot) {
  if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed in the Householder QR workspace (" + std::to_string(bytes) + " bytes)");
    return AZ_ERR_OOM;
  }
  q->allocs.push_back(*p);
  *tot += bytes;
  return AZ_OK;
}

az_status hqr_create(HQR** out, int64_t M, int k, bool f64, size_t* bytes) {
  HQR* q = new HQR();
  *out = q;
  q->M = M;
  q->k = k;
  q->f64 = f64;
  q->npanel = (k + NB - 1) / NB;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) { cudaGetLastError(); sms = 1; }
  q->nblk = 2 * sms;
  q->rows_per_blk = (M + q->nblk - 1) / q->nblk;
  size_t tot = 0;
  AZ_TRY(hq_alloc(q, (void**)&q->part, (size_t)q->nblk * NB * 8, &tot));
  AZ_TRY(hq_alloc(q, (void**)&q->hs, (NB + 1) * 8, &tot));
  AZ_TRY(hq_alloc(q, (void**)&q->tau, (size_t)k * 8, &tot));
  AZ_TRY(hq_alloc(q, (void**)&q->T, (size_t)q->npanel * NB * NB * 8, &tot));
  AZ_TRY(hq_alloc(q, (void**)&q->V, (size_t)M * NB * 8, &tot));
  AZ_TRY(hq_alloc(q, (void**)&q->G, NB * NB * 8, &tot));
  AZ_TRY(hq_alloc(q, (void**)&q->W1, (size_t)NB * k * 8, &tot));
  AZ_TRY(hq_alloc(q, (void**)&q->W2, (size_t)NB * k * 8, &tot));
  size_t pm = 0;
  for (int n = 1; n <= k; n = n < 64 ? n + 1 : n + 64) pm = std::max(pm, (size_t)df_tn_splits(M, NB, std::min(n, k)) * NB * std::min(n, k));
  pm = std::max(pm, (size_t)df_tn_splits(M, NB, k) * NB * k);
  pm = std::max(pm, (size_t)df_tn_splits(M, NB, NB) * NB * NB);
  AZ_TRY(hq_alloc(q, (void**)&q->tpart, pm * 8, &tot));
  *bytes = tot;
  return AZ_OK;
}

void hqr_destroy(HQR* q) {
  if (!q) return;
  for (void* p : q->allocs) cudaFree(p);
  delete q;
}

// A (M x k, ld lda) -> R in its upper triangle, the reflectors below it, tau
// and the panels' T factors in the workspace.  Launches only.
az_status hqr_factor(HQR* q, double* A, int64_t lda, cudaStream_t st) {
  const int64_t M = q->M;
  const int k = q->k;
  for (int p = 0; p < q->npanel; ++p) {
    const int j0 = p * NB, nbp = std::min(NB, k - j0), c1 = j0 + nbp;
    {
      ProfScope ps("hqr_panel", (double)(M - j0) * nbp * 8.0 * 2, st, 3 * nbp);
      for (int jj = 0; jj < nbp; ++jj) {
        const int j = j0 + jj;
        k_hqr_dots<<<q->nblk, DOT_WARPS * 32, 0, st>>>(A, M, lda, j, c1, q->rows_per_blk, q->part);
        k_hqr_reflect<<<1, NB, 0, st>>>(A, lda, j, c1, q->part, q->nblk, q->tau, q->hs);
        const int64_t rows = M - j - 1;
        if (rows > 0) k_hqr_apply<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(A, M, lda, j, c1, q->hs);
      }
      AZ_CUDA(cudaGetLastError());
    }
    // compact WY: V explicit, G = V^T V, T
    {
      ProfScope ps("hqr_wy", (double)(M - j0) * nbp * 8.0 * 2, st, 2);
      dim3 vg((unsigned)((M - j0 + 255) / 256), nbp);
      k_hqr_vbuf<<<vg, 256, 0, st>>>(A, M, lda, j0, nbp, q->V, M);
      AZ_CUDA(cudaGetLastError());
    }
    AZ_TRY((launch_df_tn<double, double>(q->V + j0, M, nbp, q->V + j0, M, nbp, M - j0, q->tpart, q->G, st, q->f64)));
    k_hqr_larft<<<1, NB, 0, st>>>(q->G, nbp, q->tau + j0, q->T + (size_t)p * NB * NB);
    AZ_CUDA(cudaGetLastError());
    // trailing columns: A -= V (T^T (V^T A))
    const int n = k - c1;
    if (n > 0) {
      double* Atr = A + (int64_t)c1 * lda + j0;
      AZ_TRY((launch_df_tn<double, double>(q->V + j0, M, nbp, Atr, lda, n, M - j0, q->tpart, q->W1, st, q->f64)));
      k_hqr_tw<<<(unsigned)n, NB, 0, st>>>(q->T + (size_t)p * NB * NB, nbp, q->W1, n, true, q->W2);
      AZ_CUDA(cudaGetLastError());
      AZ_TRY((launch_df_update<double, double>(q->V + j0, M, nbp, q->W2, n, Atr, lda, M - j0, Atr, lda, false, st,
                                               nullptr, q->f64)));
    }
  }
  return AZ_OK;
}

// X (M x ncols, ld ldx) := Q X with Q = H_0 H_1 ... from hqr_factor (A holds
// the reflectors).  Launches only.
az_status hqr_apply_q(HQR* q, const double* A, int64_t lda, double* X, int64_t ldx, int ncols, cudaStream_t st) {
  const int64_t M = q->M;
  const int k = q->k;
  if (ncols > k) { set_error("hqr_apply_q: more columns than the factor's workspace"); return AZ_ERR_ARG; }
  for (int p = q->npanel - 1; p >= 0; --p) {
    const int j0 = p * NB, nbp = std::min(NB, k - j0);
    {
      ProfScope ps("hqr_wy", (double)(M - j0) * nbp * 8.0 * 2, st, 1);
      dim3 vg((unsigned)((M - j0 + 255) / 256), nbp);
      k_hqr_vbuf<<<vg, 256, 0, st>>>(A, M, lda, j0, nbp, q->V, M);
      AZ_CUDA(cudaGetLastError());
    }
    double* Xp = X + j0;
    AZ_TRY((launch_df_tn<double, double>(q->V + j0, M, nbp, Xp, ldx, ncols, M - j0, q->tpart, q->W1, st, q->f64)));
    k_hqr_tw<<<(unsigned)ncols, NB, 0, st>>>(q->T + (size_t)p * NB * NB, nbp, q->W1, ncols, false, q->W2);
    AZ_CUDA(cudaGetLastError());
    AZ_TRY((launch_df_update<double, double>(q->V + j0, M, nbp, q->W2, ncols, Xp, ldx, M - j0, Xp, ldx, false, st,
                                             nullptr, q->f64)));
  }
  return AZ_OK;
}

}  // namespace az
