// The 2D Z* chain fused into one cluster-resident kernel (16-CTA clusters,
// distributed shared memory, FP64): square grids L x L with L = 64, 128, 256
// and s = 2.
#pragma once
#include "az_internal.cuh"

namespace az {

// The grid takes the fused kernel and the device runs its 16-CTA clusters.
bool zstar_cluster_ok(const Geom& g, cudaStream_t st);
// Column pairs [pair0, pair0 + npairs) of the compact input v (M rows, ld ldv,
// ncols columns): out = R - Z* v with R from the Rademacher bits, or Z* v
// when bits is null (N rows, ld ldo).  H: Ghat / S on the grid, natural
// order.  tw: the master twiddle table w_4096^j followed by the stage table
// of the register FFTs.  err: raised (AZ_ERR_TIMEOUT semantics) if a cluster barrier wait
// ran out.
az_status launch_zstar_cluster(const Geom& g, const double* v, int64_t ldv, int ncols, const int32_t* pos2m,
                               const double* H, const uint32_t* bits, int64_t nw, double* out, int64_t ldo,
                               const double2* tw, int pair0, int npairs, int* err, cudaStream_t st);

}  // namespace az
