// Low-rank step for wide sketches (k > 64): Householder QR of the sketch
// (cuSOLVER geqrf / orgqr: backward stable, no Gram squaring; the Gram routes
// cannot resolve the singular values near tau = 1e-8 sigma_1 that resolved 2D
// sketches have), FP64 SVD of the k x k triangular factor (cuSOLVER gesvd),
// and hand-written double-float kernels for the tall products U_tau = Q U_R,
// c = U_tau^T g and x = z + W u (dfgemm.cu).  Same outputs as the narrow path:
// U_tau ((M+Mb) x k, zero beyond the rank), VS = V_R Sigma^{-1} (k x k), sigma,
// and the FactorInfo record.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <string>

#include "dfgemm.cuh"
#include "hqr.cuh"
#include "lowrank.cuh"
#include "tc_tsgram.cuh"
#include "lowrank_large.cuh"
#include "profile.cuh"

namespace az {

#define AZ_SOL(call)                                                                        \
  do {                                                                                      \
    cusolverStatus_t _s = (call);                                                           \
    if (_s != CUSOLVER_STATUS_SUCCESS) {                                                    \
      set_error(std::string(#call) + ": cuSOLVER status " + std::to_string((int)_s));       \
      return AZ_ERR_CUDA;                                                                   \
    }                                                                                       \
  } while (0)
#define AZ_BLAS(call)                                                                       \
  do {                                                                                      \
    cublasStatus_t _s = (call);                                                             \
    if (_s != CUBLAS_STATUS_SUCCESS) {                                                      \
      set_error(std::string(#call) + ": cuBLAS status " + std::to_string((int)_s));         \
      return AZ_ERR_CUDA;                                                                   \
    }                                                                                       \
  } while (0)

struct LargeK {
  cusolverDnHandle_t sol = nullptr;
  cublasHandle_t blas = nullptr;
  bool fp64 = false;
  int64_t M = 0;
  int k = 0;
  void* work = nullptr;      // cuSOLVER workspace
  int lwork_qr = 0, lwork_svd = 0;
  void* blas_ws = nullptr;   // cuBLAS workspace (no allocation inside GEMM calls)
  int* devinfo = nullptr;    // 3 ints: geqrf, orgqr, gesvd
  void* tau = nullptr;       // k (T)
  double* R = nullptr;       // k x k (overwritten by gesvd)
  double* U = nullptr;       // k x k
  double* VT = nullptr;      // k x k
  double* S = nullptr;       // k
  void* UR = nullptr;        // k x k, T: U_R with columns >= rank zeroed
  double* part = nullptr;    // split-K partials of the double-float projection
  int cols_max = 0;          // right-hand sides per projection call
  bool prod64 = false;       // tall products in FP64 arithmetic (else double-float)
  HQR* hqr = nullptr;        // FP64 storage: the hand-written blocked Householder QR
};

static az_status lk_alloc(void** p, size_t bytes) {
  if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed in the wide-sketch factorisation (" + std::to_string(bytes) + " bytes)");
    return AZ_ERR_OOM;
  }
  return AZ_OK;
}

az_status large_create(LargeK** out, int64_t M, int k, bool fp64, void* A_probe, size_t* bytes, int cols_max,
                       bool prod64) {
  LargeK* L = new LargeK();
  *out = L;
  L->prod64 = prod64;
  L->fp64 = fp64;
  L->M = M;
  L->k = k;
  L->cols_max = cols_max;
  AZ_SOL(cusolverDnCreate(&L->sol));
  AZ_BLAS(cublasCreate(&L->blas));
  size_t tot = 0;
  const size_t ts = fp64 ? 8 : 4;
  int lq = 0, lo = 0, ls = 0;
  if (fp64) {
    size_t hb = 0;
    AZ_TRY(hqr_create(&L->hqr, M, k, prod64, &hb));
    tot += hb;
  } else {
    AZ_SOL(cusolverDnSgeqrf_bufferSize(L->sol, (int)M, k, (float*)A_probe, (int)M, &lq));
    AZ_SOL(cusolverDnSorgqr_bufferSize(L->sol, (int)M, k, k, (float*)A_probe, (int)M, (float*)A_probe, &lo));
  }
  AZ_SOL(cusolverDnDgesvd_bufferSize(L->sol, k, k, &ls));
  L->lwork_qr = std::max(lq, lo);
  L->lwork_svd = ls;
  const size_t wbytes = std::max((size_t)L->lwork_qr * ts, (size_t)L->lwork_svd * 8);
  AZ_TRY(lk_alloc(&L->work, wbytes)); tot += wbytes;
  AZ_TRY(lk_alloc(&L->blas_ws, 32 << 20)); tot += 32 << 20;
  AZ_BLAS(cublasSetWorkspace(L->blas, L->blas_ws, 32 << 20));
  AZ_TRY(lk_alloc((void**)&L->devinfo, 4 * sizeof(int)));
  AZ_TRY(lk_alloc(&L->tau, (size_t)k * ts));
  AZ_TRY(lk_alloc((void**)&L->R, (size_t)k * k * 8));
  AZ_TRY(lk_alloc((void**)&L->U, (size_t)k * k * 8));
  AZ_TRY(lk_alloc((void**)&L->VT, (size_t)k * k * 8));
  AZ_TRY(lk_alloc((void**)&L->S, (size_t)k * 8));
  AZ_TRY(lk_alloc(&L->UR, (size_t)k * k * ts));
  tot += (size_t)k * (4 * k * 8 + 8 + k * ts + ts);
  // the projection's split-K partials for every column count up to cols_max
  size_t pmax = 0;
  for (int nb = 1; nb <= cols_max; nb = nb < 64 ? nb + 1 : nb + 64)
    pmax = std::max(pmax, (size_t)df_tn_splits(M, k, std::min(nb, cols_max)) * k * std::min(nb, cols_max));
  pmax = std::max(pmax, (size_t)df_tn_splits(M, k, cols_max) * k * cols_max);
  for (int nb = 1; nb <= std::min(64, cols_max); ++nb) pmax = std::max(pmax, tc_tsgram_wide_partial(M, k, nb));
  AZ_TRY(lk_alloc((void**)&L->part, pmax * 8));
  tot += pmax * 8;
  *bytes = tot;
  return AZ_OK;
}

void large_destroy(LargeK* L) {
  if (!L) return;
  if (L->hqr) hqr_destroy(L->hqr);
  if (L->sol) cusolverDnDestroy(L->sol);
  if (L->blas) cublasDestroy(L->blas);
  for (void* p : {L->work, L->blas_ws, (void*)L->devinfo, L->tau, (void*)L->R, (void*)L->U, (void*)L->VT,
                  (void*)L->S, L->UR, (void*)L->part})
    if (p) cudaFree(p);
  delete L;
}

template <typename T>
__global__ void k_extract_R(const T* __restrict__ A, int64_t lda, int k, double* __restrict__ R) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * k) return;
  int i = t % k, j = t / k;
  R[t] = j >= i ? (double)A[i + (int64_t)j * lda] : 0.0;
}

// rank and small outputs from the SVD R = U S V^T (U, VT from gesvd)
template <typename T>
__global__ void k_svd_outputs(const double* __restrict__ S, const double* __restrict__ U, const double* __restrict__ VT,
                              int k, double tau, double floor, const int* __restrict__ devinfo, T* __restrict__ UR,
                              double* __restrict__ VS, double* __restrict__ sig, FactorInfo* info) {
  __shared__ int rs;
  if (threadIdx.x == 0) {
    int r = 0;
    const double s1 = S[0];
    for (int j = 0; j < k; ++j) if (S[j] > tau * s1 && S[j] > floor && isfinite(S[j])) ++r;
    rs = r;
    info->r1 = k;
    info->r = r;
    info->sigma_max = s1;
    info->sigma_min_kept = r > 0 ? S[r - 1] : 0.0;
    info->pad = 0;
    info->status = (devinfo[0] != 0 || devinfo[1] != 0 || devinfo[2] != 0 || !isfinite(s1)) ? 2 : 0;
  }
  __syncthreads();
  const int r = rs;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t % k, c = t / k;
    UR[t] = c < r ? (T)U[t] : (T)0;
    VS[t] = c < r ? VT[c + (int64_t)i * k] / S[c] : 0.0;   // V[i, c] / sigma_c
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) sig[t] = S[t];
}

template <typename T>
az_status large_factor_t(LargeK* L, const T* Y, int64_t ldy, T* A, T* Ut, int64_t ldu, double tau, double floor, double* VS,
                         double* sig, FactorInfo* info, cudaStream_t st) {
  const int64_t M = L->M;
  const int k = L->k;
  AZ_SOL(cusolverDnSetStream(L->sol, st));
  AZ_BLAS(cublasSetStream(L->blas, st));
  AZ_CUDA(cudaMemcpy2DAsync(A, M * sizeof(T), Y, ldy * sizeof(T), M * sizeof(T), k, cudaMemcpyDeviceToDevice, st));
  AZ_CUDA(cudaMemsetAsync(L->devinfo, 0, 4 * sizeof(int), st));
  if constexpr (sizeof(T) == 8) {
    // hand-written blocked Householder QR (R above the diagonal of A)
    AZ_TRY(hqr_factor(L->hqr, (double*)A, M, st));
    k_extract_R<T><<<(k * k + 255) / 256, 256, 0, st>>>(A, M, k, L->R);
    AZ_CUDA(cudaGetLastError());
  } else {
    ProfScope ps("wide_geqrf_f32", 2.0 * M * k * sizeof(T), st, 0);
    AZ_SOL(cusolverDnSgeqrf(L->sol, (int)M, k, (float*)A, (int)M, (float*)L->tau, (float*)L->work, L->lwork_qr,
                            L->devinfo));
    ps.close();
    k_extract_R<T><<<(k * k + 255) / 256, 256, 0, st>>>(A, M, k, L->R);
    AZ_CUDA(cudaGetLastError());
    ProfScope ps2("wide_orgqr_f32", 2.0 * M * k * sizeof(T), st, 0);
    AZ_SOL(cusolverDnSorgqr(L->sol, (int)M, k, k, (float*)A, (int)M, (float*)L->tau, (float*)L->work, L->lwork_qr,
                            L->devinfo + 1));
  }
  ProfScope ps3("wide_gesvd_f64", 8.0 * 4 * k * k, st, 0);
  AZ_SOL(cusolverDnDgesvd(L->sol, 'A', 'A', k, k, L->R, k, L->S, L->U, k, L->VT, k, (double*)L->work, L->lwork_svd,
                          nullptr, L->devinfo + 2));
  ps3.close();
  k_svd_outputs<T><<<1, 256, 0, st>>>(L->S, L->U, L->VT, k, tau, floor, L->devinfo, (T*)L->UR, VS, sig, info);
  AZ_CUDA(cudaGetLastError());
  // U_tau = Q U_R (columns beyond the rank are zero)
  const T one = 1, zero = 0;
  if constexpr (sizeof(T) == 8) {
    // Q [U_R; 0] by the reflectors, in reverse panel order
    AZ_CUDA(cudaMemsetAsync(Ut, 0, (size_t)ldu * k * sizeof(T), st));
    AZ_CUDA(cudaMemcpy2DAsync(Ut, ldu * sizeof(T), L->UR, (size_t)k * sizeof(T), (size_t)k * sizeof(T), k,
                              cudaMemcpyDeviceToDevice, st));
    AZ_TRY(hqr_apply_q(L->hqr, (const double*)A, M, (double*)Ut, ldu, k, st));
  } else {
    AZ_BLAS(cublasSgemm(L->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)M, k, k, (const float*)&one, (const float*)A, (int)M,
                        (const float*)L->UR, k, (const float*)&zero, (float*)Ut, (int)ldu));
  }
  return AZ_OK;
}

az_status large_factor(LargeK* L, const void* Y, int64_t ldy, void* A, void* Ut, int64_t ldu, double tau, double floor, double* VS,
                       double* sig, FactorInfo* info, cudaStream_t st) {
  return L->fp64 ? large_factor_t<double>(L, (const double*)Y, ldy, (double*)A, (double*)Ut, ldu, tau, floor, VS, sig, info, st)
                 : large_factor_t<float>(L, (const float*)Y, ldy, (float*)A, (float*)Ut, ldu, tau, floor, VS, sig, info, st);
}

// c[k x n] = Ut^T g   (FP64 result).  f32: Ut and g are FP32 (the mixed
// path's projection): on the tensor cores (split TF32, FP32-level accuracy)
// for n <= 64, else in double-float; FP64: double-float (or FP64 arithmetic).
// tc_err: the tensor-core pipeline's wait-timeout flag.
az_status large_project(LargeK* L, const void* Ut, int64_t ldu, const void* g, int64_t ldg, int n, double* c,
                        cudaStream_t st, bool f32, int* tc_err) {
  if (n > L->cols_max) { set_error("wide projection: more columns than the setup's chunk"); return AZ_ERR_ARG; }
  if (f32 && n <= 64 && tc_err && tc_tsgram_wide_ok(Ut, ldu, L->k, g, ldg, n))
    return launch_tc_tsgram_wide((const float*)Ut, ldu, L->k, (const float*)g, ldg, n, L->M, L->part, c, tc_err, st);
  if (f32)
    return launch_df_tn<float, float>((const float*)Ut, ldu, L->k, (const float*)g, ldg, n, L->M, L->part, c, st);
  return launch_df_tn<double, double>((const double*)Ut, ldu, L->k, (const double*)g, ldg, n, L->M, L->part, c, st,
                                      L->prod64);
}

// x (=|+=) z + W u in double-float.  w64 with z32 (the FP64-sketch mixed path)
// and w64 alone (FP64): x from the FP64-accurate sum.  FP32 W (the FP32-sketch
// mixed path): the sum is rounded to FP32 and also written back to z, so that
// x is exactly the FP32 value z holds (the first pass's residual is formed
// from that FP32 solution).
az_status large_update(LargeK* L, const void* W, int64_t ldw, const double* u, void* z, int64_t ldz, int64_t N, int n,
                       double* x, int64_t ldx, bool accumulate, cudaStream_t st, bool w64, bool z32) {
  if (w64 && z32)
    return launch_df_update<double, float>((const double*)W, ldw, L->k, u, n, (const float*)z, ldz, N, x, ldx,
                                           accumulate, st);
  if (w64)
    return launch_df_update<double, double>((const double*)W, ldw, L->k, u, n, (const double*)z, ldz, N, x, ldx,
                                            accumulate, st, nullptr, L->prod64);
  return launch_df_update<float, float>((const float*)W, ldw, L->k, u, n, (const float*)z, ldz, N, x, ldx, accumulate,
                                        st, (float*)z);
}

}  // namespace az
