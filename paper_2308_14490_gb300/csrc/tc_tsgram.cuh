// Tall-skinny product G = A^T B (A: M x ka, B: M x kb, FP32, column-major,
// M long) on the 5th-generation tensor cores: TMA tiles, tcgen05.mma
// (kind::tf32) with split operands for FP32-level accuracy, accumulators in
// tensor memory.  Used in the mixed path for the projection c = U_tau^T g of
// the truncated low-rank solve in step 1 of Algorithm 1 (Sec. 3.2.3).
#pragma once
#include <cstdint>

#include "az_internal.cuh"

namespace az {

// Limits of the tensor-core path: ka, kb <= 64; lda, ldb multiples of 4
// (16-byte row strides for TMA); A, B 16-byte aligned.
bool tc_tsgram_ok(const void* A, int64_t lda, int ka, const void* B, int64_t ldb, int kb);

// G (ka x kb, column-major, FP64) = A^T B.  partial: >= tc_tsgram_blocks() *
// ka * kb doubles of scratch.  err: device int, set to a nonzero code if a
// pipeline wait timed out (the result is then invalid).
az_status launch_tc_tsgram(const float* A, int64_t lda, int ka, const float* B, int64_t ldb, int kb, int64_t M,
                           double* partial, double* G, int* err, cudaStream_t st);
int tc_tsgram_blocks();

// The same product for wide A (any ka; kb <= 64): grid rows take 64-column
// chunks of A, so A is read once and B once per chunk (from L2).  partial:
// >= tc_tsgram_wide_partial(M, ka, kb) doubles.
bool tc_tsgram_wide_ok(const void* A, int64_t lda, int ka, const void* B, int64_t ldb, int kb);
size_t tc_tsgram_wide_partial(int64_t M, int ka, int kb);
az_status launch_tc_tsgram_wide(const float* A, int64_t lda, int ka, const float* B, int64_t ldb, int kb, int64_t M,
                                double* partial, double* G, int* err, cudaStream_t st);
// Exact G = Y^T Y (k x k, FP64, column-major) for FP32 Y (M x k, ld ldy) on
// the tensor cores: BF16 slices of the power-of-two-scaled columns, exact
// per-CTA sums of every slice pair, folded in FP64.  k <= 24, ldy a multiple
// of 4, Y 16-byte aligned.  partial: >= tc_gram_oz_blocks(M) * k * k doubles;
// err as for launch_tc_tsgram.
bool tc_gram_oz_ok(const void* Y, int64_t ldy, int k, int64_t M);
int tc_gram_oz_blocks(int64_t M);
az_status launch_tc_gram_oz(const float* Y, int64_t ldy, int k, int64_t M, double* partial, double* G, int* err,
                            cudaStream_t st);
// Test hook: the next launch stops issuing TMA copies at `iteration` (so its
// consumers' waits run out) and bounds every wait by wait_ns.  One-shot.
void tc_tsgram_debug_withhold(int iteration, uint64_t wait_ns);

}  // namespace az
