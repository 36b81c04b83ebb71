// Double-float (FP32-pair) tall products of the wide low-rank step: about 48
// significant bits at FP32-pipe throughput (GB300's FP64 pipe runs at 1/58 of
// the FP32 rate).  Deterministic summation order.
#pragma once
#include "az_internal.cuh"

namespace az {

// Row splits launch_df_tn uses for an M-row contraction into ka x nb outputs;
// its scratch `part` must hold df_tn_splits(M, ka, nb) * ka * nb doubles.
int df_tn_splits(int64_t M, int ka, int nb);

// C (ka x nb, column-major, ld ka, FP64) = A^T B, A: M x ka (ld lda), B: M x nb (ld ldb).
// f64: FP64 arithmetic instead of double-float.
template <typename TA, typename TB>
az_status launch_df_tn(const TA* A, int64_t lda, int ka, const TB* B, int64_t ldb, int nb, int64_t M, double* part,
                       double* C, cudaStream_t st, bool f64 = false);

// x (N x nb, ld ldx) (=|+=) z + W u;  W: N x k (ld ldw), u: k x nb (ld k, FP64),
// z: N x nb (ld ldz) or null (zero).  zf (FP32 z only): round the result to FP32, store it in
// zf (ld ldz; may be z itself) and set x to exactly that value.
template <typename TW, typename TZ>
az_status launch_df_update(const TW* Wm, int64_t ldw, int k, const double* u, int nb, const TZ* z, int64_t ldz,
                           int64_t N, double* x, int64_t ldx, bool accumulate, cudaStream_t st, float* zf = nullptr,
                           bool f64 = false);

}  // namespace az
