// Blocked Householder QR of a tall FP64 matrix (panels of 64 columns, compact
// WY, tall products in double-float or FP64 arithmetic) and the application
// of its Q.  Used by the wide low-rank step (k > 64).
#pragma once
#include "az_internal.cuh"

namespace az {

struct HQR;
// Workspace for an M x k factorisation (M >= k); f64: FP64 arithmetic in the
// tall products instead of double-float.  *bytes receives the device bytes.
az_status hqr_create(HQR** out, int64_t M, int k, bool f64, size_t* bytes);
void hqr_destroy(HQR* q);
// A (M x k, ld lda): R in the upper triangle, reflectors below.  Launches only.
az_status hqr_factor(HQR* q, double* A, int64_t lda, cudaStream_t st);
// X (M x ncols <= k) := Q X.  Launches only.
az_status hqr_apply_q(HQR* q, const double* A, int64_t lda, double* X, int64_t ldx, int ncols, cudaStream_t st);

}  // namespace az
