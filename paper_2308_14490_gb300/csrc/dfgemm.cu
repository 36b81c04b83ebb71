// Tall products of the wide low-rank step in double-float arithmetic on the
// FP32 pipe (the solve's c = U_tau^T g and x = z + W u of Algorithm 1, step 1
// and the correction of steps 2-3, Sec. 3.2.3).
//
// GB300 runs FP64 at 1/58 of its FP32 rate, so FP64-accurate products are
// formed from FP32 pairs: every FP64 operand a is split into hi + lo (48
// significant bits, on the integer pipe), each product hi*hi is made exact
// with one fma (Dekker's product), the cross terms are added in FP32, and the
// running sum is a renormalised (hi, lo) pair updated with Knuth's two-sum.
// Each output is summed in one fixed order (deterministic).
//
// Tiling: a CTA of 256 threads owns a 64 x 64 output block (256 x 16 for at
// most 16 right-hand sides, 256 x 4 for at most 4); the contraction runs in chunks staged in shared
// memory as FP32 hi and lo planes [kk][row] and [kk][col].  Where a double-float
// product is not accurate enough (FP64 setups at eps h < 0.66, whose symbol
// inverse amplifies rounding by exp((pi / (2 eps h))^2) > 300), the same tiles
// accumulate in FP64 arithmetic instead (f64).
#include <algorithm>
#include <type_traits>

#include "dfgemm.cuh"
#include "profile.cuh"

namespace az {

namespace {

// Plane row padding (keeps 16-byte alignment of the 4-element reads)
constexpr int PADP = 4;

__device__ __forceinline__ void split_in(double v, float& hi, float& lo) { d2ff_int(v, hi, lo); }
__device__ __forceinline__ void split_in(float v, float& hi, float& lo) { hi = v; lo = 0.f; }

// (ch, cl) += (ah + al) (bh + bl), renormalised; LO = false drops the cross
// terms of operands without a low part (FP32 inputs)
template <bool LO>
__device__ __forceinline__ void df_fma(float& ch, float& cl, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  if (LO) {
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
  }
  const float s = ch + p;
  const float v = s - ch;
  const float t = (ch - (s - v)) + (p - v);
  const float w = cl + (t + e);
  ch = s + w;
  cl = w - (ch - s);
}

__device__ __forceinline__ double df_to_double(float hi, float lo) { return f2d_int(hi) + f2d_int(lo); }

// Shared-memory tile of a CTA: TR output rows x TC output columns,
// contraction chunks of KT.  256 threads on a TX x TY grid, each owning a
// 4 x CJ block of outputs.  FP32 hi and lo planes (double-float) or one FP64
// plane (F64).
template <int TR, int TC, int KT, bool F64>
struct Tile {
  static constexpr int TX = TR / 4;           // threads along rows (4 rows each)
  static constexpr int TY = 256 / TX;         // threads along columns
  static constexpr int CJ = TC / TY;          // columns per thread
  static_assert(TX * TY == 256 && CJ * TY == TC && CJ >= 1, "tile shape");
  using E = typename std::conditional<F64, double, float>::type;
  E ah[KT][TR + PADP], al[F64 ? 1 : KT][F64 ? 1 : TR + PADP];
  E bh[KT][TC + PADP], bl[F64 ? 1 : KT][F64 ? 1 : TC + PADP];
};

// Stage a chunk of a column-major matrix X (element (r, q) at X[q * ld + r])
// into plane[kk][c] for kk < KT, c < NC:
//  KROWS: kk indexes rows of X (r = k0 + kk, q = c0 + c): contiguous in kk;
//  else:  kk indexes columns (q = k0 + kk, r = c0 + c): contiguous in c.
template <int KT, int NC, int LD, bool F64, typename TX, typename TE, bool KROWS, typename PL>
__device__ __forceinline__ void stage(const TX* __restrict__ X, int64_t ld, int64_t nr, int64_t nq, int64_t k0, int kn,
                                      int64_t c0, TE (*ph)[LD], PL pl) {
  for (int t = threadIdx.x; t < KT * NC; t += 256) {
    int kk, c;
    if (KROWS) { kk = t % KT; c = t / KT; }
    else { c = t % NC; kk = t / NC; }
    const int64_t r = KROWS ? k0 + kk : c0 + c;
    const int64_t q = KROWS ? c0 + c : k0 + kk;
    const bool in = kk < kn && r < nr && q < nq;
    if constexpr (F64) {
      ph[kk][c] = in ? (TE)X[q * ld + r] : (TE)0;
    } else {
      float h = 0.f, l = 0.f;
      if (in) split_in(X[q * ld + r], h, l);
      ph[kk][c] = h;
      pl[kk][c] = l;
    }
  }
}

template <int TR, int TC, int KT, bool F64, bool LO>
__device__ __forceinline__ void micro(const Tile<TR, TC, KT, F64>& P, int kn, int tx, int ty,
                                      float (&ch)[4][Tile<TR, TC, KT, F64>::CJ], float (&cl)[4][Tile<TR, TC, KT, F64>::CJ],
                                      double (&cd)[4][Tile<TR, TC, KT, F64>::CJ]) {
  constexpr int CJ = Tile<TR, TC, KT, F64>::CJ;
  for (int kk = 0; kk < kn; ++kk) {
    if constexpr (F64) {
      double a[4], b[CJ];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = P.ah[kk][tx * 4 + i];
#pragma unroll
      for (int j = 0; j < CJ; ++j) b[j] = P.bh[kk][ty * CJ + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) cd[i][j] = fma(a[i], b[j], cd[i][j]);
    } else {
      float ah[4], al[4], bh[CJ], bl[CJ];
#pragma unroll
      for (int i = 0; i < 4; ++i) { ah[i] = P.ah[kk][tx * 4 + i]; al[i] = LO ? P.al[kk][tx * 4 + i] : 0.f; }
#pragma unroll
      for (int j = 0; j < CJ; ++j) { bh[j] = P.bh[kk][ty * CJ + j]; bl[j] = LO ? P.bl[kk][ty * CJ + j] : 0.f; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CJ; ++j) df_fma<LO>(ch[i][j], cl[i][j], ah[i], al[i], bh[j], bl[j]);
    }
  }
}

// part[split][j + col * ka] = sum over rows m of this split of A[m, j] B[m, col]
template <typename TA, typename TB, int TR, int TC, int KT, bool F64>
__global__ void __launch_bounds__(256) k_tn(const TA* __restrict__ A, int64_t lda, int ka, const TB* __restrict__ B,
                                            int64_t ldb, int nb, int64_t M, int64_t rows_per_split,
                                            double* __restrict__ part) {
  using TL = Tile<TR, TC, KT, F64>;
  constexpr int CJ = TL::CJ;
  constexpr bool LO = sizeof(TA) == 8 || sizeof(TB) == 8;
  __shared__ __align__(16) TL P;
  const int tx = threadIdx.x % TL::TX, ty = threadIdx.x / TL::TX;
  const int64_t j0 = (int64_t)blockIdx.x * TR, col0 = (int64_t)blockIdx.y * TC;
  const int64_t m0 = (int64_t)blockIdx.z * rows_per_split;
  const int64_t m1 = M < m0 + rows_per_split ? M : m0 + rows_per_split;
  float ch[4][CJ], cl[4][CJ];
  double cd[4][CJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) { ch[i][j] = 0.f; cl[i][j] = 0.f; cd[i][j] = 0.0; }
  for (int64_t k0 = m0; k0 < m1; k0 += KT) {
    const int kn = m1 - k0 < KT ? (int)(m1 - k0) : KT;
    __syncthreads();
    stage<KT, TR, TR + PADP, F64, TA, typename TL::E, true>(A, lda, M, ka, k0, kn, j0, P.ah, P.al);
    stage<KT, TC, TC + PADP, F64, TB, typename TL::E, true>(B, ldb, M, nb, k0, kn, col0, P.bh, P.bl);
    __syncthreads();
    micro<TR, TC, KT, F64, LO>(P, kn, tx, ty, ch, cl, cd);
  }
  double* out = part + (int64_t)blockIdx.z * ka * nb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      const int64_t r = j0 + tx * 4 + i, c = col0 + ty * CJ + j;
      if (r < ka && c < nb) out[r + c * ka] = F64 ? cd[i][j] : df_to_double(ch[i][j], cl[i][j]);
    }
}

__global__ void k_df_reduce(const double* __restrict__ part, int nsplit, int64_t n, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s = 0.0;
  for (int q = 0; q < nsplit; ++q) s += part[(int64_t)q * n + t];
  out[t] = s;
}

// x[i, col] = (acc ? x : 0) + z[i, col] + sum_j W[i, j] u[j, col].
// zf (FP32 z only, may alias z): the result is rounded to FP32, written
// there, and x receives exactly that FP32 value (the mixed path's first pass,
// whose residual is formed from the FP32 solution).
template <typename TW, typename TZ, int TR, int TC, int KT, bool F64>
__global__ void __launch_bounds__(256) k_nn(const TW* __restrict__ Wm, int64_t ldw, int k, const double* __restrict__ u,
                                            int64_t ldu, int nb, const TZ* z, int64_t ldz, int64_t N,
                                            double* __restrict__ x, int64_t ldx, int acc, float* zf) {
  using TL = Tile<TR, TC, KT, F64>;
  constexpr int CJ = TL::CJ;
  __shared__ __align__(16) TL P;
  const int tx = threadIdx.x % TL::TX, ty = threadIdx.x / TL::TX;
  const int64_t i0 = (int64_t)blockIdx.x * TR, col0 = (int64_t)blockIdx.y * TC;
  float ch[4][CJ], cl[4][CJ];
  double cd[4][CJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) { ch[i][j] = 0.f; cl[i][j] = 0.f; cd[i][j] = 0.0; }
  for (int k0 = 0; k0 < k; k0 += KT) {
    const int kn = k - k0 < KT ? k - k0 : KT;
    __syncthreads();
    stage<KT, TR, TR + PADP, F64, TW, typename TL::E, false>(Wm, ldw, N, k, k0, kn, i0, P.ah, P.al);
    stage<KT, TC, TC + PADP, F64, double, typename TL::E, true>(u, ldu, k, nb, k0, kn, col0, P.bh, P.bl);
    __syncthreads();
    micro<TR, TC, KT, F64, true>(P, kn, tx, ty, ch, cl, cd);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      const int64_t r = i0 + tx * 4 + i, c = col0 + ty * CJ + j;
      if (r < N && c < nb) {
        double* xp = x + c * ldx + r;
        double v = (z ? cvt<double>(z[c * ldz + r]) : 0.0) + (F64 ? cd[i][j] : df_to_double(ch[i][j], cl[i][j]));
        if (zf) {
          const float f = d2f_int(v);
          zf[c * ldz + r] = f;
          v = f2d_int(f);
        }
        *xp = acc ? *xp + v : v;
      }
    }
}

int sm_count_df() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    }
  }
  return n;
}

// column tile by the number of right-hand sides: 256 x 4 (nb <= 4),
// 256 x 16 (nb <= 16), else 64 x 64
int col_tile(int nb) { return nb <= 4 ? 4 : (nb <= 16 ? 16 : 64); }

}  // namespace

int df_tn_splits(int64_t M, int ka, int nb) {
  const int TC = col_tile(nb), TR = TC == 64 ? 64 : 256;
  const int64_t tiles = (int64_t)((ka + TR - 1) / TR) * ((nb + TC - 1) / TC);
  const int64_t want = 3 * (int64_t)sm_count_df();
  int64_t s = std::max<int64_t>(1, (want + tiles - 1) / tiles);
  s = std::min<int64_t>(s, std::max<int64_t>(1, M / 512));   // at least 512 rows per split
  return (int)std::min<int64_t>(s, 64);
}

template <typename TA, typename TB>
az_status launch_df_tn(const TA* A, int64_t lda, int ka, const TB* B, int64_t ldb, int nb, int64_t M, double* part,
                       double* C, cudaStream_t st, bool f64) {
  if (ka < 1 || nb < 1 || M < 1) { set_error("df_tn: empty shape"); return AZ_ERR_ARG; }
  const int ns = df_tn_splits(M, ka, nb);
  const int64_t rps = ((M + ns - 1) / ns + 31) / 32 * 32;
  const int nsplit = (int)((M + rps - 1) / rps);
  ProfScope ps(f64 ? "wide_proj_f64" : "wide_proj_df", (double)M * (ka * sizeof(TA) + nb * sizeof(TB)) + 8.0 * ka * nb, st);
  if (col_tile(nb) == 4) {
    dim3 grid((unsigned)((ka + 255) / 256), (unsigned)((nb + 3) / 4), (unsigned)nsplit);
    if (f64) k_tn<TA, TB, 256, 4, 16, true><<<grid, 256, 0, st>>>(A, lda, ka, B, ldb, nb, M, rps, part);
    else k_tn<TA, TB, 256, 4, 16, false><<<grid, 256, 0, st>>>(A, lda, ka, B, ldb, nb, M, rps, part);
  } else if (col_tile(nb) == 16) {
    dim3 grid((unsigned)((ka + 255) / 256), (unsigned)((nb + 15) / 16), (unsigned)nsplit);
    if (f64) k_tn<TA, TB, 256, 16, 16, true><<<grid, 256, 0, st>>>(A, lda, ka, B, ldb, nb, M, rps, part);
    else k_tn<TA, TB, 256, 16, 16, false><<<grid, 256, 0, st>>>(A, lda, ka, B, ldb, nb, M, rps, part);
  } else {
    dim3 grid((unsigned)((ka + 63) / 64), (unsigned)((nb + 63) / 64), (unsigned)nsplit);
    if (f64) k_tn<TA, TB, 64, 64, 32, true><<<grid, 256, 0, st>>>(A, lda, ka, B, ldb, nb, M, rps, part);
    else k_tn<TA, TB, 64, 64, 32, false><<<grid, 256, 0, st>>>(A, lda, ka, B, ldb, nb, M, rps, part);
  }
  AZ_CUDA(cudaGetLastError());
  const int64_t n = (int64_t)ka * nb;
  k_df_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, nsplit, n, C);
  AZ_CUDA(cudaGetLastError());
  return AZ_OK;
}

template <typename TW, typename TZ>
az_status launch_df_update(const TW* Wm, int64_t ldw, int k, const double* u, int nb, const TZ* z, int64_t ldz,
                           int64_t N, double* x, int64_t ldx, bool accumulate, cudaStream_t st, float* zf, bool f64) {
  if (k < 1 || nb < 1 || N < 1) { set_error("df_update: empty shape"); return AZ_ERR_ARG; }
  ProfScope ps(f64 ? "wide_update_f64" : "wide_update_df",
               (double)N * k * sizeof(TW) + (double)N * nb * (sizeof(TZ) + 8.0 * (accumulate ? 2 : 1)), st);
  const int acc = accumulate ? 1 : 0;
  if (col_tile(nb) == 4) {
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)((nb + 3) / 4));
    if (f64) k_nn<TW, TZ, 256, 4, 16, true><<<grid, 256, 0, st>>>(Wm, ldw, k, u, k, nb, z, ldz, N, x, ldx, acc, zf);
    else k_nn<TW, TZ, 256, 4, 16, false><<<grid, 256, 0, st>>>(Wm, ldw, k, u, k, nb, z, ldz, N, x, ldx, acc, zf);
  } else if (col_tile(nb) == 16) {
    dim3 grid((unsigned)((N + 255) / 256), (unsigned)((nb + 15) / 16));
    if (f64) k_nn<TW, TZ, 256, 16, 16, true><<<grid, 256, 0, st>>>(Wm, ldw, k, u, k, nb, z, ldz, N, x, ldx, acc, zf);
    else k_nn<TW, TZ, 256, 16, 16, false><<<grid, 256, 0, st>>>(Wm, ldw, k, u, k, nb, z, ldz, N, x, ldx, acc, zf);
  } else {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((nb + 63) / 64));
    if (f64) k_nn<TW, TZ, 64, 64, 32, true><<<grid, 256, 0, st>>>(Wm, ldw, k, u, k, nb, z, ldz, N, x, ldx, acc, zf);
    else k_nn<TW, TZ, 64, 64, 32, false><<<grid, 256, 0, st>>>(Wm, ldw, k, u, k, nb, z, ldz, N, x, ldx, acc, zf);
  }
  AZ_CUDA(cudaGetLastError());
  return AZ_OK;
}

template az_status launch_df_tn<double, double>(const double*, int64_t, int, const double*, int64_t, int, int64_t,
                                                double*, double*, cudaStream_t, bool);
template az_status launch_df_tn<float, float>(const float*, int64_t, int, const float*, int64_t, int, int64_t,
                                              double*, double*, cudaStream_t, bool);
template az_status launch_df_update<double, double>(const double*, int64_t, int, const double*, int, const double*,
                                                    int64_t, int64_t, double*, int64_t, bool, cudaStream_t, float*, bool);
template az_status launch_df_update<double, float>(const double*, int64_t, int, const double*, int, const float*,
                                                   int64_t, int64_t, double*, int64_t, bool, cudaStream_t, float*, bool);
template az_status launch_df_update<float, float>(const float*, int64_t, int, const double*, int, const float*,
                                                  int64_t, int64_t, double*, int64_t, bool, cudaStream_t, float*, bool);

}  // namespace az
