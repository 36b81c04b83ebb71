// Wide-sketch (k > 64) low-rank step: Householder QR + FP64 SVD of R + GEMMs.
#pragma once
#include "lowrank.cuh"

namespace az {
struct LargeK;
// A_probe: a device array of at least M x k elements of the working precision
// (only used to size the solver workspace).  *bytes receives the device bytes held.
// cols_max: right-hand-side columns per projection call (sizes the scratch);
// prod64: FP64 tall products in FP64 arithmetic instead of double-float.
az_status large_create(LargeK** out, int64_t M, int k, bool fp64, void* A_probe, size_t* bytes, int cols_max,
                       bool prod64);
void large_destroy(LargeK* L);
// From the sketch Y (M x k): U_tau (M x k, zero beyond rank), VS (k x k), sigma, info.  A: M x k scratch.
az_status large_factor(LargeK* L, const void* Y, int64_t ldy, void* A, void* Ut, int64_t ldu, double tau, double floor, double* VS,
                       double* sig, FactorInfo* info, cudaStream_t st);
// c = Ut^T g; f32: Ut and g FP32 (tensor cores for n <= 64), else FP64;
// tc_err: device flag raised by a tensor-core pipeline wait that timed out
az_status large_project(LargeK* L, const void* Ut, int64_t ldu, const void* g, int64_t ldg, int n, double* c,
                        cudaStream_t st, bool f32, int* tc_err);
// x (=|+=) z + W u; w64: W FP64 (else FP32), z32: z FP32 (else the precision of W)
az_status large_update(LargeK* L, const void* W, int64_t ldw, const double* u, void* z, int64_t ldz, int64_t N, int n,
                       double* x, int64_t ldx, bool accumulate, cudaStream_t st, bool w64, bool z32);
}  // namespace az
