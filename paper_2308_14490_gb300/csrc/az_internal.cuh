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

// ---------------------------------------------------------------- FP64 <-> FP32 on the integer pipe
// GB300 runs FP64 arithmetic and FP64 conversions at a small fraction of the
// FP32 rate; the mixed path converts its FP64 inputs/outputs with integer bit
// manipulation instead.  Values outside the FP32 normal range fall back to the
// hardware conversion.
__device__ __forceinline__ float d2f_int(double d) {   // round to nearest even
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(u >> 63);
  const int e = (int)((u >> 52) & 0x7ff);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  if (e == 0) return sign ? -0.0f : 0.0f;
  int fe = e - 1023 + 127;
  if (fe <= 0 || fe >= 254) return (float)d;
  unsigned mant = (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) {
    if (++mant == 0x800000u) { mant = 0; ++fe; }
  }
  return __uint_as_float((sign << 31) | ((unsigned)fe << 23) | mant);
}
__device__ __forceinline__ double f2d_int(float f) {   // exact
  const unsigned u = __float_as_uint(f);
  const unsigned fe = (u >> 23) & 0xff;
  if (fe == 0 || fe == 0xff) return (double)f;   // zero, subnormal, inf, nan
  const unsigned long long e = (unsigned long long)(fe - 127 + 1023);
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | (e << 52) |
                                          ((unsigned long long)(u & 0x7fffff) << 29)));
}
// d = hi + lo with hi = d2f_int(d) and lo = the FP32-rounded remainder (exact
// split up to 2^-48 relative), integer pipe only
__device__ __forceinline__ void d2ff_int(double d, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0 || e - 1023 + 127 <= 52 || e - 1023 + 127 >= 254) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
    return;
  }
  // hi: truncated to 24 significant bits; lo: the remaining 29 bits, rounded
  const unsigned sign = (unsigned)(u >> 63);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const int fe = e - 1023 + 127;
  hi = __uint_as_float((sign << 31) | ((unsigned)fe << 23) | (unsigned)(m >> 29));
  const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);   // value rem * 2^(e - 1023 - 52)
  const float lf = (float)rem;                           // exact up to rounding to 24 bits
  lo = __fmul_rn(sign ? -lf : lf, __uint_as_float((unsigned)(fe - 52) << 23));
}

// The FP64 number nearest to a + b for FP32 a and b (ties to even), which is
// (double)a + (double)b, formed without the FP64 pipe: Knuth's two-sum gives
// s = fl(a + b) and the exact error e (a + b = s + e, |e| <= ulp32(s)/2);
// e in units of ulp64(s), rounded to an integer, is added to the FP64 bit
// pattern of s (the carry can never leave the binade of s, and when s is a
// power of two and e points toward zero the units below s are half as
// large).  The rounding of that integer is the rounding of the sum, and the
// FP64 mantissa of s is even, so ties go to even as in the FP64 add.  Sums
// that are zero, subnormal, below 2^-75 in magnitude, infinite or NaN take
// the FP64 pipe.
__device__ __forceinline__ double f32_sum_f64(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
  const unsigned sb = __float_as_uint(s);
  const unsigned ex = (sb >> 23) & 0xffu;
  if (ex < 52u || ex == 255u) return (double)a + (double)b;
  const bool neg = (sb >> 31) != 0u;
  const unsigned mant = sb & 0x7fffffu;
  float es = __fmul_rn(e, __uint_as_float((306u - ex) << 23));   // e / ulp64(s), |es| <= 2^28
  if (mant == 0u && (neg ? es > 0.f : es < 0.f)) es = __fmul_rn(es, 2.f);
  const long long r = __float2int_rn(es);
  const long long mag = (long long)(((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)mant << 29));
  const long long bits = (mag + (neg ? -r : r)) | (neg ? (long long)0x8000000000000000ull : 0ll);
  return __longlong_as_double(bits);
}

// FP64 -> FP32 without branches (integer pipe): round to nearest with ties
// away from zero on the magnitude; FP32-subnormal inputs flush to a signed
// zero and values beyond the FP32 range become infinities.  Branch-free, so
// a caller's loads can all be in flight before any conversion.
__device__ __forceinline__ float d2f_fast(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sign = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned mag = ((((hi & 0x7fffffffu) - 0x38000000u) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
  const unsigned r = e < 897u ? 0u : (e > 1150u ? 0x7f800000u : mag);
  return __uint_as_float(sign | r);
}

template <typename TO, typename TI> __device__ __forceinline__ TO cvt(TI v) { return (TO)v; }
template <> __device__ __forceinline__ float cvt<float, double>(double v) { return d2f_int(v); }
template <> __device__ __forceinline__ double cvt<double, float>(float v) { return f2d_int(v); }

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
  // kept grid points: when they are the run [run0, run0 + runM) of grid
  // indices (runM > 0), row m of b is grid point run0 + m
  int64_t run0, runM;
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
