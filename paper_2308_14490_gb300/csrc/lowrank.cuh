// Low-rank step of Algorithm 1 (S6, S7, S9): Gram products, the SVQB + Cholesky
// orthogonalisation of the sketch Y, the truncated SVD of its small factor, and
// the per-solve projections.
#pragma once
#include "az_internal.cuh"

namespace az {

// Device-side record of the factorisation (read lazily by the host).
struct FactorInfo {
  int32_t r1;          // directions kept by the Gram pass
  int32_t r;           // rank kept by the truncated SVD
  int32_t status;      // 0 ok, 1 Cholesky breakdown, 2 non-finite
  int32_t pad;
  double sigma_max;
  double sigma_min_kept;
  double ar_fro;       // ||A R||_F (noise floor reference)
};

// G[ka x kb] = A^T B over M rows, FP64 accumulation, deterministic order.
// partial must hold nblk*ka*kb doubles (nblk = gram_blocks(M)).
int gram_blocks(int64_t M);
template <typename TA, typename TB>
az_status launch_gram(const TA* A, int64_t lda, int ka, const TB* B, int64_t ldb, int kb, int64_t M,
                      double* partial, double* G, cudaStream_t st, bool fast = false);
// G (ka x kb) = sum over nblk per-block partials (partial[b * ka * kb + a + c * ka]).
az_status launch_gram_reduce(const double* partial, int nblk, int ka, int kb, double* G, cudaStream_t st);
// out[M x r] = A[M x k] * S[k x r] (S FP64, column-major ld k), FP64 accumulation.
template <typename TA, typename TO>
az_status launch_tsprod(const TA* A, int64_t lda, int k, const double* S, int r, int64_t M, TO* out, int64_t ldo,
                        cudaStream_t st);
// out[M x r] = A[M x k] S (A FP32, S FP64) with double-float accumulation (r <= 32)
template <typename TO>
az_status launch_tsprod_df(const float* A, int64_t lda, int k, const double* S, int r, int64_t M, TO* out, int64_t ldo,
                           cudaStream_t st);
// First pass: eigen-decomposition of G1 (k x k) by one-sided Jacobi; keeps
// lambda_i > taug^2 lambda_1 (and above the rounding floor); writes
// B1 = V_keep Lambda^{-1/2} (k x k, zero columns beyond r1) and V, lambda.
az_status launch_factor1(const double* G1, int k, double taug, double floor2, double* V, double* lam, double* B1,
                         FactorInfo* info, cudaStream_t st);
// Second pass: R2 = chol(G2[:r1,:r1]); Rs = R2 diag(sqrt(lam)); SVD of Rs;
// rank r = #(sigma > tau sigma_1, > floor); T = R2^{-1} U_R[:, :r] (k x k, zero
// beyond r), VS = V_keep V_R[:, :r] Sigma^{-1} (k x k, zero beyond r), sigma.
az_status launch_factor2(const double* G2, int k, const double* V, const double* lam, double tau, double floor,
                         double* T, double* VS, double* sig, FactorInfo* info, cudaStream_t st, bool f32jac = false);
// u[k x n] = VS[k x k] c[k x n]
az_status launch_small_mm(const double* VS, int k, const double* c, int n, double* u, cudaStream_t st);
// x[:, c] = (accumulate ? x : 0) + z[:, c] + W u[:, c]  (N rows)
template <typename TW, typename TZ>
// x = z + W u (accumulate: x += z + W u; xbase: x = xbase + z + W u with xbase
// FP32, ld ldz; x may be null when only the exact FP32 copy xf is wanted)
az_status launch_update_x(const TW* W, int64_t ldw, int k, const double* u, const TZ* z, int64_t ldz, int64_t N,
                          int nrhs, double* x, int64_t ldx, bool accumulate, cudaStream_t st, float* xf = nullptr,
                          const float* xbase = nullptr);

}  // namespace az
