// Low-rank step for wide sketches (k > 64): Householder QR of the sketch
// (cuSOLVER geqrf / orgqr: backward stable, no Gram squaring), FP64 SVD of the
// k x k triangular factor, and cuBLAS GEMMs for the tall products
// (U_tau = Q U_R, c = U_tau^T g, x = z + W u).  Same outputs as the narrow
// path: U_tau ((M+Mb) x k, zero beyond the rank), VS = V_R Sigma^{-1}
// (k x k), sigma, and the FactorInfo record.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <string>

#include "lowrank.cuh"
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
  void* c32 = nullptr;       // k x 64 (mixed: FP32 projection)
  void* u32 = nullptr;       // k x 64 (mixed: FP32 copy of u)
};

static az_status lk_alloc(void** p, size_t bytes) {
  if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed in the wide-sketch factorisation (" + std::to_string(bytes) + " bytes)");
    return AZ_ERR_OOM;
  }
  return AZ_OK;
}

az_status large_create(LargeK** out, int64_t M, int k, bool fp64, void* A_probe, size_t* bytes) {
  LargeK* L = new LargeK();
  *out = L;
  L->fp64 = fp64;
  L->M = M;
  L->k = k;
  AZ_SOL(cusolverDnCreate(&L->sol));
  AZ_BLAS(cublasCreate(&L->blas));
  size_t tot = 0;
  const size_t ts = fp64 ? 8 : 4;
  int lq = 0, lo = 0, ls = 0;
  if (fp64) {
    AZ_SOL(cusolverDnDgeqrf_bufferSize(L->sol, (int)M, k, (double*)A_probe, (int)M, &lq));
    AZ_SOL(cusolverDnDorgqr_bufferSize(L->sol, (int)M, k, k, (double*)A_probe, (int)M, (double*)A_probe, &lo));
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
  AZ_TRY(lk_alloc(&L->c32, (size_t)k * 64 * 4));
  AZ_TRY(lk_alloc(&L->u32, (size_t)k * 64 * 4));
  tot += (size_t)k * (4 * k * 8 + 8 + k * ts + 2 * 64 * 4 + ts);
  *bytes = tot;
  return AZ_OK;
}

void large_destroy(LargeK* L) {
  if (!L) return;
  if (L->sol) cusolverDnDestroy(L->sol);
  if (L->blas) cublasDestroy(L->blas);
  for (void* p : {L->work, L->blas_ws, (void*)L->devinfo, L->tau, (void*)L->R, (void*)L->U, (void*)L->VT,
                  (void*)L->S, L->UR, L->c32, L->u32})
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
  ProfScope ps(sizeof(T) == 8 ? "wide_qr_svd_f64" : "wide_qr_svd_f32", 2.0 * M * k * sizeof(T) * 3, st);
  AZ_SOL(cusolverDnSetStream(L->sol, st));
  AZ_BLAS(cublasSetStream(L->blas, st));
  AZ_CUDA(cudaMemcpy2DAsync(A, M * sizeof(T), Y, ldy * sizeof(T), M * sizeof(T), k, cudaMemcpyDeviceToDevice, st));
  AZ_CUDA(cudaMemsetAsync(L->devinfo, 0, 4 * sizeof(int), st));
  if (sizeof(T) == 8) {
    AZ_SOL(cusolverDnDgeqrf(L->sol, (int)M, k, (double*)A, (int)M, (double*)L->tau, (double*)L->work, L->lwork_qr,
                            L->devinfo));
  } else {
    AZ_SOL(cusolverDnSgeqrf(L->sol, (int)M, k, (float*)A, (int)M, (float*)L->tau, (float*)L->work, L->lwork_qr,
                            L->devinfo));
  }
  k_extract_R<T><<<(k * k + 255) / 256, 256, 0, st>>>(A, M, k, L->R);
  AZ_CUDA(cudaGetLastError());
  if (sizeof(T) == 8) {
    AZ_SOL(cusolverDnDorgqr(L->sol, (int)M, k, k, (double*)A, (int)M, (double*)L->tau, (double*)L->work,
                            L->lwork_qr, L->devinfo + 1));
  } else {
    AZ_SOL(cusolverDnSorgqr(L->sol, (int)M, k, k, (float*)A, (int)M, (float*)L->tau, (float*)L->work, L->lwork_qr,
                            L->devinfo + 1));
  }
  AZ_SOL(cusolverDnDgesvd(L->sol, 'A', 'A', k, k, L->R, k, L->S, L->U, k, L->VT, k, (double*)L->work, L->lwork_svd,
                          nullptr, L->devinfo + 2));
  k_svd_outputs<T><<<1, 256, 0, st>>>(L->S, L->U, L->VT, k, tau, floor, L->devinfo, (T*)L->UR, VS, sig, info);
  AZ_CUDA(cudaGetLastError());
  // U_tau = Q U_R (columns beyond the rank are zero)
  const T one = 1, zero = 0;
  if (sizeof(T) == 8) {
    AZ_BLAS(cublasDgemm(L->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)M, k, k, (const double*)&one, (const double*)A, (int)M,
                        (const double*)L->UR, k, (const double*)&zero, (double*)Ut, (int)ldu));
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

__global__ void k_f2d_cols(const float* __restrict__ a, int n, double* __restrict__ b) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (double)a[t];
}
__global__ void k_d2f_cols(const double* __restrict__ a, int n, float* __restrict__ b) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

// c[k x n] = Ut^T g   (FP64 result); f32: Ut and g are FP32 (the mixed
// path's projection), else FP64
az_status large_project(LargeK* L, const void* Ut, int64_t ldu, const void* g, int64_t ldg, int n, double* c,
                        cudaStream_t st, bool f32) {
  ProfScope ps("wide_proj", (double)L->M * (L->k + n) * (f32 ? 4 : 8), st);
  AZ_BLAS(cublasSetStream(L->blas, st));
  if (!f32) {
    const double one = 1, zero = 0;
    AZ_BLAS(cublasDgemm(L->blas, CUBLAS_OP_T, CUBLAS_OP_N, L->k, n, (int)L->M, &one, (const double*)Ut, (int)ldu,
                        (const double*)g, (int)ldg, &zero, c, L->k));
  } else {
    const float one = 1, zero = 0;
    AZ_BLAS(cublasSgemm(L->blas, CUBLAS_OP_T, CUBLAS_OP_N, L->k, n, (int)L->M, &one, (const float*)Ut, (int)ldu,
                        (const float*)g, (int)ldg, &zero, (float*)L->c32, L->k));
    k_f2d_cols<<<(L->k * n + 255) / 256, 256, 0, st>>>((const float*)L->c32, L->k * n, c);
    AZ_CUDA(cudaGetLastError());
  }
  return AZ_OK;
}

__global__ void k_store_x(const float* __restrict__ zf, int64_t ldz, const double* __restrict__ zd, int64_t N,
                          double* __restrict__ x, int64_t ldx, int accumulate) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (j >= N) return;
  const double v = zf ? cvt<double>(zf[(int64_t)c * ldz + j]) : zd[(int64_t)c * ldz + j];
  double* xp = x + (int64_t)c * ldx + j;
  *xp = accumulate ? *xp + v : v;
}

// z += W u (in place, in the precision of W), then x (=|+=) z.  In the mixed
// path z then holds the exact FP32 value of the new solution increment.
// w64 with z32 (the FP64-sketch mixed path): x (=|+=) z first, then x += W u in
// FP64, so that the update is consistent with the FP64 sketch Y = A W.
az_status large_update(LargeK* L, const void* W, int64_t ldw, const double* u, void* z, int64_t ldz, int64_t N, int n,
                       double* x, int64_t ldx, bool accumulate, cudaStream_t st, bool w64, bool z32) {
  ProfScope ps("wide_update", (double)N * (L->k * (w64 ? 8 : 4) + 2 * n * (z32 ? 4 : 8)) +
                                  (double)N * n * 8 * (accumulate ? 2 : 1), st);
  AZ_BLAS(cublasSetStream(L->blas, st));
  dim3 grid((unsigned)((N + 255) / 256), n);
  if (w64 && z32) {
    k_store_x<<<grid, 256, 0, st>>>((const float*)z, ldz, nullptr, N, x, ldx, accumulate ? 1 : 0);
    AZ_CUDA(cudaGetLastError());
    const double one = 1;
    AZ_BLAS(cublasDgemm(L->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, n, L->k, &one, (const double*)W, (int)ldw, u, L->k,
                        &one, x, (int)ldx));
    return AZ_OK;
  }
  if (w64) {
    const double one = 1;
    AZ_BLAS(cublasDgemm(L->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, n, L->k, &one, (const double*)W, (int)ldw, u, L->k,
                        &one, (double*)z, (int)ldz));
  } else {
    k_d2f_cols<<<(L->k * n + 255) / 256, 256, 0, st>>>(u, L->k * n, (float*)L->u32);
    const float one = 1;
    AZ_BLAS(cublasSgemm(L->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, n, L->k, &one, (const float*)W, (int)ldw,
                        (const float*)L->u32, L->k, &one, (float*)z, (int)ldz));
  }
  k_store_x<<<grid, 256, 0, st>>>(w64 ? nullptr : (const float*)z, ldz, w64 ? (const double*)z : nullptr, N, x,
                                  ldx, accumulate ? 1 : 0);
  AZ_CUDA(cudaGetLastError());
  return AZ_OK;
}

}  // namespace az
