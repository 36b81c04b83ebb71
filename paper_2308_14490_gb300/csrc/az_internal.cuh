// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/az.h"
#include "fft.cuh"

namespace az {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
#define AZ_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t _e = (call);                                                                   \
    if (_e != cudaSuccess) {                                                                   \
      ::az::set_error(std::string(#call) + ": " + cudaGetErrorString(_e) + " (" + __FILE__ + \
                      ":" + std::to_string(__LINE__) + ")");                                  \
      return AZ_ERR_CUDA;                                                                      \
    }                                                                                          \
  } while (0)
#define AZ_TRY(expr)              \
  do {                            \
    az_status _s = (expr);        \
    if (_s != AZ_OK) return _s;   \
  } while (0)

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: two 32x32->64 multiplies per round, 10 rounds, key
// bumped by the Weyl constants between rounds.  Same bit layout as documented in
// include/az.h (counter = (row/128, column, 0, 0), key = seed).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// floor division for possibly negative numerators (positive divisor)
__host__ __device__ __forceinline__ int64_t fdiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__host__ __device__ __forceinline__ int64_t fmod_pos(int64_t a, int64_t b) { int64_t r = a % b; return r < 0 ? r + b : r; }

// Rademacher value of R[j, col] from the packed bit matrix (N/32 words per column).
__device__ __forceinline__ float rad_bit(const uint32_t* __restrict__ bits, int64_t nw, int64_t j, int col) {
  const uint32_t w = __ldg(bits + (int64_t)col * nw + (j >> 5));
  return ((w >> (j & 31)) & 1u) ? 1.0f : -1.0f;
}

// ---------------------------------------------------------------- geometry
// FFT grid of the L-grid: 1D L = D0*D1 (natural index n0*D1 + n1; spectrum
// position (k0,k1) holds frequency k0 + D0*k1); 2D D0 = Lx, D1 = Ly.
// N-grid: G0 x N1 with N1 = D1/s_last (1D: G0 = D0; 2D: G0 = Nx).
struct Geom {
  int dim;
  int64_t n[2];     // centers per dim
  int s[2];         // oversampling per dim
  int64_t Ld[2];    // L per dim
  double T[2];
  int64_t N, L;
  int D0, D1, logD0, logD1;   // L-grid FFT factorisation
  int G0, N1, logG0, logN1;   // N-grid (fold output) factorisation
  int Rg, Rstride, Fq;        // fold: rows per group, row stride, within-row alias count
  int Wst32[2], Wst64[2];     // stencil half-widths (grid units of the L-grid)
  int logN, logs[2], logn[2], logLd[2], logRg;
};

// Device tables owned by a setup.
struct Tables {
  double2* tw64[2] = {nullptr, nullptr};   // twiddles for D0 / D1 lengths
  float2* tw32[2] = {nullptr, nullptr};
  double2* twN64 = nullptr;                // twiddles for N1 (fold inverse) and G0 (col inverse)
  float2* twN32 = nullptr;
  double2* twG64 = nullptr;
  float2* twG32 = nullptr;
  // big twiddles for the four-step (1D): w_L^m = A[m >> 11] * B[m & 2047]
  double2* bigA64 = nullptr; double2* bigB64 = nullptr;
  float2* bigA32 = nullptr; float2* bigB32 = nullptr;
  double2* bigNA64 = nullptr; double2* bigNB64 = nullptr;  // same for w_N
  float2* bigNA32 = nullptr; float2* bigNB32 = nullptr;
};

}  // namespace az
