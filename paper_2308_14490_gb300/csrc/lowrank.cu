// Low-rank factorisation and projections (S6, S7, S9).
//
// The paper's step 1 (Sec. 3.2.3) takes an SVD of the sketch Y = (A - A Z* A) R.
// Here Y is tall (M rows) and narrow (k columns), and numerically rank
// deficient (its trailing singular values are rounding noise).  The
// factorisation is the CholeskyQR2 pattern with a rank-revealing first pass:
//   pass 1 (SVQB): G1 = Y^T Y, G1 = V Lambda V^T, Q1 = Y V_r1 Lambda_r1^{-1/2}
//   pass 2 (Cholesky): G2 = Q1^T Q1 = R2^T R2, Q = Q1 R2^{-1}
// so Y V_r1 = Q R2 Lambda^{1/2}; the small factor Rs = R2 Lambda^{1/2} is
// decomposed by a one-sided Jacobi SVD, Rs = U_R Sigma V_R^T, and the
// truncated solve keeps sigma_i > tau sigma_1.  Stored: U_tau = Q U_R[:, :r]
// (formed as Q1 T with T = R2^{-1} U_R[:, :r]) and VS = V_r1 V_R[:, :r]
// Sigma^{-1}, so that u = VS U_tau^T g.
#include <cmath>
#include <type_traits>
#include "lowrank.cuh"
#include "profile.cuh"
#include <mutex>
#include <unordered_map>

namespace az {
// once per (kernel, size): keeps steady-state launches free of attribute calls
template <typename K> static void smem_once(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done;
  std::lock_guard<std::mutex> g(mu);
  auto it = done.find((const void*)kernel);
  if (it != done.end() && it->second >= bytes) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    done[(const void*)kernel] = bytes;
}
}  // namespace az

namespace az {

#define AZ_LCHECK()                                                                                  \
  do {                                                                                               \
    cudaError_t _e = cudaGetLastError();                                                             \
    if (_e != cudaSuccess) { set_error(std::string("kernel launch: ") + cudaGetErrorString(_e)); return AZ_ERR_CUDA; } \
  } while (0)

static constexpr int GRAM_ROWS = 1024;  // rows per CTA of the Gram partials
static constexpr int GRAM_TILE = 64;    // rows staged per step

int gram_blocks(int64_t M) { return (int)std::max<int64_t>(1, (M + GRAM_ROWS - 1) / GRAM_ROWS); }

// Each CTA: rows [b*GRAM_ROWS, ...); each thread owns an RA x RB block of the
// ka x kb output; tiles of GRAM_TILE rows are staged in shared memory in the
// staging type TS.  Products within a tile are summed in TS, tiles are summed
// in FP64 (TS = double gives FP64 products throughout).
// Exact FP32 product a*b = p + e (e from one fma) and two-sum accumulation into
// a (hi, lo) pair: the "double-float" arithmetic used where FP32 inputs need an
// FP64-accurate sum (about 48 significant bits) at FP32 throughput.
struct DF { float hi, lo; };
__device__ __forceinline__ void df_add_prod(DF& s, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += err + e;
}
__device__ __forceinline__ void df_add_prod_split(DF& s, float a, float bh, float bl) {
  df_add_prod(s, a, bh);
  s.lo = fmaf(a, bl, s.lo);
}

// Asynchronous global->shared copy of one element (zero-filled when !valid).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* sdst, const void* gsrc, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(sdst);
  const int srcsize = valid ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(saddr), "l"(gsrc), "n"(BYTES), "r"(srcsize));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Staged tiles are double-buffered with cp.async so the next tile's loads are
// in flight while the current one is multiplied.  TS is the input type (no
// conversion on the copy).
template <typename TA, typename TB, typename TS, int RA, int RB, bool DFMODE>
__global__ void __launch_bounds__(512) k_gram_partial(const TA* __restrict__ A, int64_t lda, int ka, const TB* __restrict__ B,
                                                      int64_t ldb, int kb, int64_t M, double* __restrict__ partial, int sym) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TS* sbuf = (TS*)smem_raw;                       // 2 x GRAM_TILE x (ka + kb)
  const int tile_elems = GRAM_TILE * (ka + kb);
  double* red = (double*)smem_raw;                 // nsplit x nblk x RA*RB (reduction; aliases the tiles)
  const int nta = (ka + RA - 1) / RA, ntb = (kb + RB - 1) / RB;
  // symmetric product (B == A): threads only for the blocks on or above the
  // block diagonal, enumerated column by column (bt = tb (tb + 1) / 2 + ta)
  const int nblkt = sym ? nta * (nta + 1) / 2 : nta * ntb;
  const int nsplit = blockDim.x / nblkt;        // thread groups splitting each tile's rows
  const int bt = threadIdx.x % nblkt, sp = threadIdx.x / nblkt;
  int ta = bt % nta, tb = bt / nta;
  if (sym) {
    tb = 0;
    while ((tb + 1) * (tb + 2) / 2 <= bt) ++tb;
    ta = bt - tb * (tb + 1) / 2;
  }
  const bool active = sp < nsplit;
  const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS;
  const int64_t r1 = (M < r0 + GRAM_ROWS) ? M : r0 + GRAM_ROWS;
  const int ntiles = (int)((r1 - r0 + GRAM_TILE - 1) / GRAM_TILE);
  auto issue = [&](int tix) {
    TS* sA = sbuf + (tix & 1) * tile_elems;
    TS* sB = sA + GRAM_TILE * ka;
    const int64_t rb = r0 + (int64_t)tix * GRAM_TILE;
    const int nr = (int)((r1 - rb) < GRAM_TILE ? (r1 - rb) : GRAM_TILE);
    for (int t = threadIdx.x; t < GRAM_TILE * ka; t += blockDim.x) {
      const int a = t / GRAM_TILE, rr = t % GRAM_TILE;
      const bool v = rr < nr;
      cp_async_elem<sizeof(TS)>(sA + rr * ka + a, A + (int64_t)a * lda + (v ? rb + rr : r0), v);
    }
    for (int t = threadIdx.x; t < GRAM_TILE * kb; t += blockDim.x) {
      const int c = t / GRAM_TILE, rr = t % GRAM_TILE;
      const bool v = rr < nr;
      cp_async_elem<sizeof(TS)>(sB + rr * kb + c, B + (int64_t)c * ldb + (v ? rb + rr : r0), v);
    }
    cp_async_commit();
  };
  // accumulators live across all tiles of this CTA (FP64, FP32 or
  // double-float); converted to FP64 once at the end
  TS sacc[RA][RB];
  DF dacc[RA][RB];
#pragma unroll
  for (int i = 0; i < RA; ++i)
#pragma unroll
    for (int j = 0; j < RB; ++j) { sacc[i][j] = (TS)0; dacc[i][j].hi = 0.f; dacc[i][j].lo = 0.f; }
  if (ntiles > 0) issue(0);
  for (int tix = 0; tix < ntiles; ++tix) {
    if (tix + 1 < ntiles) { issue(tix + 1); cp_async_wait<1>(); }
    else cp_async_wait<0>();
    __syncthreads();
    const TS* sA = sbuf + (tix & 1) * tile_elems;
    const TS* sB = sA + GRAM_TILE * ka;
    const int64_t rb = r0 + (int64_t)tix * GRAM_TILE;
    const int nr = (int)((r1 - rb) < GRAM_TILE ? (r1 - rb) : GRAM_TILE);
    if (active) {
      for (int rr = sp; rr < nr; rr += nsplit) {
        TS av[RA], bv[RB];
#pragma unroll
        for (int i = 0; i < RA; ++i) { int a = ta * RA + i; av[i] = a < ka ? sA[rr * ka + a] : (TS)0; }
#pragma unroll
        for (int j = 0; j < RB; ++j) { int c = tb * RB + j; bv[j] = c < kb ? sB[rr * kb + c] : (TS)0; }
        if (DFMODE) {
#pragma unroll
          for (int i = 0; i < RA; ++i)
#pragma unroll
            for (int j = 0; j < RB; ++j) df_add_prod(dacc[i][j], (float)av[i], (float)bv[j]);
        } else {
#pragma unroll
          for (int i = 0; i < RA; ++i)
#pragma unroll
            for (int j = 0; j < RB; ++j) sacc[i][j] = fma(av[i], bv[j], sacc[i][j]);
        }
      }
    }
    __syncthreads();   // buffer (tix & 1) is refilled by the issue of tile tix + 2
  }
  double acc[RA][RB];
#pragma unroll
  for (int i = 0; i < RA; ++i)
#pragma unroll
    for (int j = 0; j < RB; ++j)
      acc[i][j] = DFMODE ? (double)dacc[i][j].hi + (double)dacc[i][j].lo : (double)sacc[i][j];
  // reduce the split groups in a fixed order
  __syncthreads();
  if (active) {
#pragma unroll
    for (int i = 0; i < RA; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) red[((size_t)sp * nblkt + bt) * (RA * RB) + i * RB + j] = acc[i][j];
  }
  __syncthreads();
  const int npair = ka * kb;
  for (int t = threadIdx.x; t < nblkt * RA * RB; t += blockDim.x) {
    const int b2 = t / (RA * RB), e = t % (RA * RB);
    const int i = e / RB, j = e % RB;
    int ta2 = b2 % nta, tb2 = b2 / nta;
    if (sym) {
      tb2 = 0;
      while ((tb2 + 1) * (tb2 + 2) / 2 <= b2) ++tb2;
      ta2 = b2 - tb2 * (tb2 + 1) / 2;
    }
    const int a = ta2 * RA + i, c = tb2 * RB + j;
    if (a >= ka || c >= kb) continue;
    double sacc2 = 0.0;
    for (int q = 0; q < nsplit; ++q) sacc2 += red[((size_t)q * nblkt + b2) * (RA * RB) + e];
    partial[(int64_t)blockIdx.x * npair + a + (int64_t)c * ka] = sacc2;
  }
}
// One warp per output entry: lanes stride over the per-block partial sums,
// then a shuffle tree (fixed order, so the result is deterministic).
__global__ void k_gram_reduce(const double* __restrict__ partial, int nblk, int npair, int ka, int sym, int RA,
                              double* __restrict__ G) {
  const int p = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= npair) return;
  const int a = p % ka, c = p / ka;
  // symmetric case: entries in blocks below the block diagonal were not
  // computed; read the mirrored entry
  int src = p;
  if (sym && (a / RA) > (c / RA)) src = c + a * ka;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[(int64_t)b * npair + src];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) G[p] = s;  // column-major ka x kb: p = a + c*ka
}
az_status launch_gram_reduce(const double* partial, int nblk, int ka, int kb, double* G, cudaStream_t st) {
  const int npair = ka * kb;
  k_gram_reduce<<<(unsigned)(((int64_t)npair * 32 + 255) / 256), 256, 0, st>>>(partial, nblk, npair, ka, 0, 1, G);
  AZ_LCHECK();
  return AZ_OK;
}
// mode: products summed in FP32 within a tile ("fast", FP32 inputs only),
// else double-float for FP32 inputs, else FP64.
template <typename TA, typename TB>
az_status launch_gram(const TA* A, int64_t lda, int ka, const TB* B, int64_t ldb, int kb, int64_t M,
                      double* partial, double* G, cudaStream_t st, bool fast) {
  constexpr int RA = 4, RB = 4;
  const int npair = ka * kb;
  const int sym = ((const void*)A == (const void*)B && ka == kb && lda == ldb) ? 1 : 0;
  const int nta = (ka + RA - 1) / RA, ntb = (kb + RB - 1) / RB;
  const int nthr = sym ? nta * (nta + 1) / 2 : nta * ntb;   // one thread per (upper) 4 x 4 block
  if (nthr > 1024) { set_error("gram: too many columns for this kernel"); return AZ_ERR_ARG; }
  const int nsplit = std::max(1, 512 / nthr);
  const int threads = nsplit * nthr;
  const int nblk = gram_blocks(M);
  const bool in32 = sizeof(TA) == 4 && sizeof(TB) == 4;
  const size_t ts = in32 ? sizeof(float) : sizeof(double);
  size_t sm = 2 * (size_t)GRAM_TILE * (ka + kb) * ts;
  sm = std::max(sm, (size_t)nsplit * nthr * RA * RB * sizeof(double));
  ProfScope ps(in32 ? (fast ? "proj_f32" : "gram_df32") : "gram_f64", (double)M * (ka * sizeof(TA) + kb * sizeof(TB)), st, 2);
  if (in32 && fast) {
    auto k = k_gram_partial<TA, TB, float, RA, RB, false>;
    smem_once(k, sm);
    k<<<nblk, threads, sm, st>>>(A, lda, ka, B, ldb, kb, M, partial, sym);
  } else if (in32) {
    auto k = k_gram_partial<TA, TB, float, RA, RB, true>;
    smem_once(k, sm);
    k<<<nblk, threads, sm, st>>>(A, lda, ka, B, ldb, kb, M, partial, sym);
  } else {
    auto k = k_gram_partial<TA, TB, double, RA, RB, false>;
    smem_once(k, sm);
    k<<<nblk, threads, sm, st>>>(A, lda, ka, B, ldb, kb, M, partial, sym);
  }
  k_gram_reduce<<<(unsigned)(((int64_t)npair * 32 + 255) / 256), 256, 0, st>>>(partial, nblk, npair, ka, sym, RA, G);
  AZ_LCHECK();
  return AZ_OK;
}

// out[M x r] = A[M x k] * S[k x r] with A FP32 and S FP64 split into FP32
// (hi, lo): each product a*S = a*hi (exact, two-product) + a*lo, summed in
// double-float; the result is rounded to TO.  Used for Q1 = Y B1, whose small
// directions cancel by up to sigma_1/sigma_r.
template <typename TO, int KB>
__global__ void __launch_bounds__(128) k_tsprod_df(const float* __restrict__ A, int64_t lda, int k,
                                                   const double* __restrict__ S, int r, int64_t M, TO* __restrict__ out,
                                                   int64_t ldo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sh = (float*)smem_raw;      // [a*KB + c]
  float* sl = sh + k * KB;
  for (int t = threadIdx.x; t < k * KB; t += blockDim.x) {
    const int a = t / KB, c = t % KB;
    const double v = c < r ? S[a + (int64_t)c * k] : 0.0;
    const float h = (float)v;
    sh[t] = h;
    sl[t] = (float)(v - (double)h);
  }
  __syncthreads();
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  DF acc[KB];
#pragma unroll
  for (int c = 0; c < KB; ++c) { acc[c].hi = 0.f; acc[c].lo = 0.f; }
  for (int a = 0; a < k; ++a) {
    const float v = A[(int64_t)a * lda + m];
#pragma unroll
    for (int c = 0; c < KB; ++c) df_add_prod_split(acc[c], v, sh[a * KB + c], sl[a * KB + c]);
  }
#pragma unroll
  for (int c = 0; c < KB; ++c)
    if (c < r) out[(int64_t)c * ldo + m] = (TO)((double)acc[c].hi + (double)acc[c].lo);
}
template <typename TO>
az_status launch_tsprod_df(const float* A, int64_t lda, int k, const double* S, int r, int64_t M, TO* out, int64_t ldo,
                           cudaStream_t st) {
  ProfScope ps("tsprod_df32", (double)M * (k * 4 + r * sizeof(TO)), st);
  const unsigned grid = (unsigned)((M + 127) / 128);
  // output columns in chunks of at most 32 (double-float accumulators in registers)
  for (int c0 = 0; c0 < r; c0 += 32) {
    const int rc = std::min(32, r - c0);
    const double* Sc = S + (int64_t)c0 * k;
    TO* oc = out + (int64_t)c0 * ldo;
    if (rc <= 16) {
      k_tsprod_df<TO, 16><<<grid, 128, 2 * (size_t)k * 16 * sizeof(float), st>>>(A, lda, k, Sc, rc, M, oc, ldo);
    } else if (rc <= 24) {
      k_tsprod_df<TO, 24><<<grid, 128, 2 * (size_t)k * 24 * sizeof(float), st>>>(A, lda, k, Sc, rc, M, oc, ldo);
    } else {
      k_tsprod_df<TO, 32><<<grid, 128, 2 * (size_t)k * 32 * sizeof(float), st>>>(A, lda, k, Sc, rc, M, oc, ldo);
    }
  }
  AZ_LCHECK();
  return AZ_OK;
}
template az_status launch_tsprod_df<float>(const float*, int64_t, int, const double*, int, int64_t, float*, int64_t, cudaStream_t);

// out = A * S : thread per row, S (k x r) in shared memory, r <= KB outputs
// accumulated in registers (FP64 for FP64 inputs, else FP32).
template <typename TA, typename TO, int KB>
__global__ void __launch_bounds__(128) k_tsprod(const TA* __restrict__ A, int64_t lda, int k, const double* __restrict__ S,
                                                int r, int64_t M, TO* __restrict__ out, int64_t ldo) {
  using TC = typename std::conditional<sizeof(TA) == 8, double, float>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TC* sS = (TC*)smem_raw;   // sS[a*KB + c] = S[a, c]
  for (int t = threadIdx.x; t < k * KB; t += blockDim.x) {
    const int a = t / KB, c = t % KB;
    sS[t] = c < r ? (TC)S[a + (int64_t)c * k] : (TC)0;
  }
  __syncthreads();
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  TC acc[KB];
#pragma unroll
  for (int c = 0; c < KB; ++c) acc[c] = 0;
  for (int a = 0; a < k; ++a) {
    const TC v = (TC)A[(int64_t)a * lda + m];
#pragma unroll
    for (int c = 0; c < KB; ++c) acc[c] = fma(v, sS[a * KB + c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < KB; ++c)
    if (c < r) out[(int64_t)c * ldo + m] = (TO)acc[c];
}
template <typename TA, typename TO>
az_status launch_tsprod(const TA* A, int64_t lda, int k, const double* S, int r, int64_t M, TO* out, int64_t ldo,
                        cudaStream_t st) {
  using TC = typename std::conditional<sizeof(TA) == 8, double, float>::type;
  ProfScope ps("tsprod", (double)M * (k * sizeof(TA) + r * sizeof(TO)), st);
  const unsigned grid = (unsigned)((M + 127) / 128);
  if (r <= 16) k_tsprod<TA, TO, 16><<<grid, 128, (size_t)k * 16 * sizeof(TC), st>>>(A, lda, k, S, r, M, out, ldo);
  else if (r <= 32) k_tsprod<TA, TO, 32><<<grid, 128, (size_t)k * 32 * sizeof(TC), st>>>(A, lda, k, S, r, M, out, ldo);
  else if (r <= 64) {
    size_t sm = (size_t)k * 64 * sizeof(TC);
    smem_once(k_tsprod<TA, TO, 64>, sm);
    k_tsprod<TA, TO, 64><<<grid, 128, sm, st>>>(A, lda, k, S, r, M, out, ldo);
  } else { set_error("tsprod: r > 64 not supported by this kernel"); return AZ_ERR_ARG; }
  AZ_LCHECK();
  return AZ_OK;
}

// ---------------------------------------------------------------- one-CTA small dense work
// One-sided (Hestenes) Jacobi on the columns of a (m x n, column-major in
// shared memory, ld m): rotates column pairs until they are mutually
// orthogonal; V (n x n) accumulates the rotations.  Round-robin pair order, one
// warp per pair.  After convergence column j has norm sigma_j and
// a[:, j] / sigma_j is the left singular vector.
template <typename TJ>
__device__ int jacobi_onesided(TJ* a, int m, int n, TJ* V, int* flag, double floor_rel) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ TJ fro2;
  // identity V; ||a||_F^2 is invariant under the rotations and sets the level
  // below which column pairs are rounding noise and are left alone
  for (int c = warp; c < n; c += nwarps)
    for (int r = lane; r < n; r += 32) V[c * n + r] = (r == c) ? (TJ)1 : (TJ)0;
  if (threadIdx.x == 0) fro2 = 0;
  __syncthreads();
  {
    TJ f = 0;
    for (int t = threadIdx.x; t < m * n; t += blockDim.x) f += a[t] * a[t];
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) atomicAdd(&fro2, f);
  }
  __syncthreads();
  // a pair is orthogonal to working precision once |gamma| is below the
  // rounding level of the larger column against the whole matrix (floor_rel;
  // 0 = plain relative criterion)
  // relative orthogonality reachable by an m-term dot product in TJ; the
  // tests below compare squares (|g| > f sqrt(x)  <=>  g^2 > f^2 x)
  const TJ ueps = sizeof(TJ) == 8 ? (TJ)1.1e-16 : (TJ)6e-8;
  const TJ reltol = fmax((TJ)(10 * ueps), (TJ)(2 * m) * ueps);
  const TJ rel2 = reltol * reltol;
  const TJ flr2 = (TJ)floor_rel * (TJ)floor_rel * fro2;
  const int nn = (n + 1) & ~1;  // even count for round-robin (a dummy column if n odd)
  int sweeps = 0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    sweeps = sweep + 1;
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int step = 0; step < nn - 1; ++step) {
      for (int pr = warp; pr < nn / 2; pr += nwarps) {
        // round-robin pairing: positions 0..nn-1, position 0 fixed
        int p0 = pr, p1 = nn - 1 - pr;
        auto idx = [&](int pos) {   // 1 + (pos - 1 + step) mod (nn - 1), both terms < nn - 1
          int v = pos - 1 + step;
          if (v >= nn - 1) v -= nn - 1;
          return pos == 0 ? 0 : 1 + v;
        };
        int i = idx(p0), j = idx(p1);
        if (i > j) { int tt = i; i = j; j = tt; }
        if (j >= n) continue;
        TJ al = 0, be = 0, ga = 0;
        for (int r = lane; r < m; r += 32) {
          TJ x = a[i * m + r], y = a[j * m + r];
          al += x * x; be += y * y; ga += x * y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        const TJ ga2 = ga * ga;
        if (ga2 > flr2 * fmax(al, be) && ga2 > rel2 * (al * be)) {
          TJ c, s;
          if constexpr (sizeof(TJ) == 4) {
            // the rotation angle only steers convergence (fast divides); the
            // cosine is normalised to working precision (rsqrt and one Newton
            // step), so that c^2 + s^2 = 1 and V stays orthogonal
            const float zeta = __fdividef(be - al, 2.f * ga);
            const float t = __fdividef(zeta >= 0.f ? 1.f : -1.f, fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
            const float x = fmaf(t, t, 1.f);
            float r = rsqrtf(x);
            r = r * fmaf(-0.5f * x, r * r, 1.5f);
            c = r;
            s = r * t;
          } else {
            TJ zeta = (be - al) / ((TJ)2 * ga);
            TJ t = (zeta >= 0 ? (TJ)1 : (TJ)-1) / (fabs(zeta) + sqrt((TJ)1 + zeta * zeta));
            c = (TJ)1 / sqrt((TJ)1 + t * t);
            s = c * t;
          }
          for (int r = lane; r < m; r += 32) {
            TJ x = a[i * m + r], y = a[j * m + r];
            a[i * m + r] = c * x - s * y;
            a[j * m + r] = s * x + c * y;
          }
          for (int r = lane; r < n; r += 32) {
            TJ x = V[i * n + r], y = V[j * n + r];
            V[i * n + r] = c * x - s * y;
            V[j * n + r] = s * x + c * y;
          }
          if (lane == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (*flag == 0) break;
    __syncthreads();
  }
  return sweeps;
}

// Pass 1 (rank-revealing): Cholesky of G1 = Y^T Y with symmetric diagonal
// pivoting, stopped when the largest remaining pivot is <= tol * the largest
// initial diagonal.  Y P = Q1 R1 with R1 = [R11 R12] (r1 x k, upper
// trapezoidal in pivoted order).  Writes B1 = P[:, :r1] R11^{-1} (k x k, zero
// columns beyond r1), R1P = R1 P^T (r1 x k, ld k; the small factor of Y in the
// original column order) and r1.
__global__ void k_factor1(const double* __restrict__ G1, int k, double tol, double floor2, double* R1P, double* lam,
                          double* B1, FactorInfo* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* G = (double*)smem_raw;   // k x k working copy, column-major
  double* R = G + k * k;           // r1 x k rows (ld k): R[i*k + c]
  __shared__ int perm[64];
  __shared__ int piv, r1s, stop;
  __shared__ double dmax, dpiv, rdpiv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) { G[t] = G1[t]; R[t] = 0.0; }
  for (int t = threadIdx.x; t < k; t += blockDim.x) perm[t] = t;
  if (threadIdx.x == 0) { r1s = 0; stop = 0; }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x < 32) {
      // pivot: the first largest remaining diagonal entry (warp arg-max, k <= 64)
      const int lane = threadIdx.x;
      double best = -INFINITY;
      int p = k;
      for (int i = j + lane; i < k; i += 32) {
        const double v = G[i * k + i];
        if (v > best || (p == k && !(v == v))) { best = v == v ? v : -INFINITY; p = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (lane == 0) {
        const double gjj = G[j * k + j];
        if (!(gjj == gjj)) { best = gjj; p = j; }   // a NaN pivot candidate stops the pass
        if (p >= k) p = j;
        if (j == 0) dmax = best;
        if (!(best > tol * dmax) || !(best > floor2) || !isfinite(best)) stop = 1;
        piv = p;
        // the pivot's square root and its reciprocal, once
        if (!stop) { dpiv = sqrt(best); rdpiv = 1.0 / dpiv; }
      }
    }
    __syncthreads();
    if (stop) break;
    const int p = piv;
    if (p != j) {  // symmetric swap of rows/columns j and p, and of R's columns
      for (int t = threadIdx.x; t < k; t += blockDim.x) {
        double u = G[t * k + j]; G[t * k + j] = G[t * k + p]; G[t * k + p] = u;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < k; t += blockDim.x) {
        double u = G[j * k + t]; G[j * k + t] = G[p * k + t]; G[p * k + t] = u;
      }
      for (int t = threadIdx.x; t < j; t += blockDim.x) {
        double u = R[t * k + j]; R[t * k + j] = R[t * k + p]; R[t * k + p] = u;
      }
      if (threadIdx.x == 0) { int u = perm[j]; perm[j] = perm[p]; perm[p] = u; }
      __syncthreads();
    }
    const double d = dpiv, rd = rdpiv;
    for (int c = j + threadIdx.x; c < k; c += blockDim.x) R[j * k + c] = (c == j) ? d : G[c * k + j] * rd;
    __syncthreads();
    for (int c = j + 1 + warp; c < k; c += nwarps)
      for (int i = j + 1 + lane; i < k; i += 32) G[c * k + i] -= R[j * k + i] * R[j * k + c];
    if (threadIdx.x == 0) r1s = j + 1;
    __syncthreads();
  }
  const int r1 = r1s;
  if (threadIdx.x == 0) { info->r1 = r1; info->status = isfinite(dmax) ? 0 : 2; info->pad = 0; }
  // B1 = P[:, :r1] R11^{-1}: column c solves R11 y = e_c by back substitution
  // (the r1 reciprocal pivots are formed once, in parallel)
  __shared__ double rdiag[64];
  for (int i = threadIdx.x; i < r1; i += blockDim.x) rdiag[i] = 1.0 / R[i * k + i];
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) B1[(int64_t)c * k + i] = 0.0;
    if (c < r1) {
      double* y = G + (size_t)c * k;   // G is free after the Cholesky; column c is this thread's
      for (int i = r1 - 1; i >= 0; --i) {
        double sacc = (i == c) ? 1.0 : 0.0;
        for (int l = i + 1; l < r1; ++l) sacc -= R[i * k + l] * y[l];
        y[i] = sacc * rdiag[i];
      }
      for (int i = 0; i < r1; ++i) B1[(int64_t)c * k + perm[i]] = y[i];
    }
  }
  // R1P = R1 P^T (rows i < r1, original column order), ld k
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t % k, c = t / k;
    R1P[(int64_t)c * k + i] = 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < r1 * k; t += blockDim.x) {
    const int i = t % r1, c = t / r1;   // pivoted column c
    R1P[(int64_t)perm[c] * k + i] = c >= i ? R[i * k + c] : 0.0;
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) lam[t] = t < r1 ? R[t * k + t] : 0.0;
}
az_status launch_factor1(const double* G1, int k, double taug, double floor2, double* V, double* lam, double* B1,
                         FactorInfo* info, cudaStream_t st) {
  if (k > 64) { set_error("factor: k > 64 not supported by the one-CTA factorisation"); return AZ_ERR_ARG; }
  size_t sm = (2 * (size_t)k * k) * sizeof(double);
  smem_once(k_factor1, sm);
  ProfScope ps("factor1", 0.0, st);
  const double tol = fmax(taug * taug, 1e-15);
  k_factor1<<<1, 256, sm, st>>>(G1, k, tol, floor2, V, lam, B1, info);
  AZ_LCHECK();
  return AZ_OK;
}

// Pass 2: R2 = chol(G2[:r1, :r1]) with G2 = Q1^T Q1, Q1 = Y B1; the small
// factor of Y is Rs = R2 R1P (r1 x k), so Y = (Q1 R2^{-1}) Rs.  One-sided
// Jacobi on Rs^T (k x r1) gives Rs^T = V_R Sigma U_R^T; rank r = #(sigma >
// tau sigma_1, > floor); T = R2^{-1} U_R[:, :r] (so U_tau = Q1 T) and
// VS = V_R[:, :r] Sigma^{-1}; both k x k with zero columns beyond r.
__global__ void k_factor2(const double* __restrict__ G2, int k, const double* __restrict__ R1P,
                          double tau, double floor, double* T, double* VS, double* sig, FactorInfo* info, int f32jac) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* R = (double*)smem_raw;   // r1 x r1 Cholesky factor (upper), column-major ld k
  double* A = R + k * k;           // Rs^T: k x r1, column-major ld k
  double* VR = A + k * k;          // r1 x r1 rotations
  double* sg = VR + k * k;
  __shared__ int flag;
  __shared__ int fail;
  const int r1 = info->r1;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) { R[t] = 0.0; A[t] = 0.0; }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < r1 * r1; t += blockDim.x) {
    int i = t % r1, j = t / r1;
    if (i <= j) R[j * k + i] = G2[(int64_t)j * k + i];
  }
  __syncthreads();
  __shared__ double rdj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int j = 0; j < r1; ++j) {
    if (threadIdx.x == 0) {
      double d = R[j * k + j];
      if (!(d > 0.0) || !isfinite(d)) { fail = 1; d = 1.0; }
      const double sd = sqrt(d);
      R[j * k + j] = sd;
      rdj = 1.0 / sd;
    }
    __syncthreads();
    const double rd = rdj;
    for (int c = j + 1 + threadIdx.x; c < r1; c += blockDim.x) R[c * k + j] *= rd;
    __syncthreads();
    // trailing update of the upper triangle, j < i <= c < r1
    for (int c = j + 1 + warp; c < r1; c += nwarps)
      for (int i = j + 1 + lane; i <= c; i += 32) R[c * k + i] -= R[i * k + j] * R[c * k + j];
    __syncthreads();
  }
  // A = Rs^T = R1P^T R2^T : A[c, i] = sum_{l >= i} R1P[l, c] R2[i, l]  (R2 upper)
  for (int t = threadIdx.x; t < k * r1; t += blockDim.x) {
    const int c = t % k, i = t / k;
    double sacc = 0.0;
    for (int l = i; l < r1; ++l) sacc += R1P[(int64_t)c * k + l] * R[l * k + i];
    A[i * k + c] = sacc;
  }
  __syncthreads();
  int sw;
  if (f32jac) {
    // mixed path: Rs is only FP32-accurate (its inputs are), so its SVD is
    // taken in FP32 and widened back
    float* Af = (float*)(sg + k);
    float* Vf = Af + k * k;
    for (int t = threadIdx.x; t < k * r1; t += blockDim.x) Af[t] = (float)A[t];
    __syncthreads();
    sw = jacobi_onesided<float>(Af, k, r1, Vf, &flag, 0.0);
    for (int t = threadIdx.x; t < k * r1; t += blockDim.x) A[t] = (double)Af[t];
    for (int t = threadIdx.x; t < r1 * r1; t += blockDim.x) VR[t] = (double)Vf[t];
    __syncthreads();
  } else {
    sw = jacobi_onesided<double>(A, k, r1, VR, &flag, 0.0);
  }
  if (threadIdx.x == 0) info->pad = sw;
  // sort by decreasing norm (columns of A of length k, rotations VR of length r1)
  for (int j = threadIdx.x; j < r1; j += blockDim.x) {
    double sacc = 0;
    for (int rr = 0; rr < k; ++rr) sacc += A[j * k + rr] * A[j * k + rr];
    sg[j] = sqrt(sacc);
  }
  __syncthreads();
  // stable rank of each column (larger norm first, ties by index), then a
  // parallel permutation through the scratch above sg
  {
    int* rank = (int*)(sg + k);
    double* tmp = (double*)(rank + k + (k & 1));
    for (int j = threadIdx.x; j < r1; j += blockDim.x) {
      int rj = 0;
      for (int i = 0; i < r1; ++i) rj += (sg[i] > sg[j]) || (sg[i] == sg[j] && i < j);
      rank[j] = rj;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < r1 * k; t += blockDim.x) tmp[rank[t / k] * k + t % k] = A[t];
    __syncthreads();
    for (int t = threadIdx.x; t < r1 * k; t += blockDim.x) A[t] = tmp[t];
    __syncthreads();
    for (int t = threadIdx.x; t < r1 * r1; t += blockDim.x) tmp[rank[t / r1] * r1 + t % r1] = VR[t];
    double sgv = 0.0;
    if (threadIdx.x < r1) sgv = sg[threadIdx.x];
    __syncthreads();
    for (int t = threadIdx.x; t < r1 * r1; t += blockDim.x) VR[t] = tmp[t];
    if (threadIdx.x < r1) sg[rank[threadIdx.x]] = sgv;
    __syncthreads();
  }
  __shared__ int rs;
  if (threadIdx.x == 0) {
    int r = 0;
    const double s1 = r1 > 0 ? sg[0] : 0.0;
    for (int j = 0; j < r1; ++j) if (sg[j] > tau * s1 && sg[j] > floor) ++r;
    rs = r;
    info->r = r;
    info->sigma_max = s1;
    info->sigma_min_kept = r > 0 ? sg[r - 1] : 0.0;
    if (fail) info->status = 1;
  }
  __syncthreads();
  const int r = rs;
  // U_R = VR (r1 x r1, column c); T = R2^{-1} U_R[:, :r] by back substitution,
  // solved in a shared-memory scratch (after the sort buffers) and written out once
  {
    double* Ts = (double*)((int*)(sg + k) + k + (k & 1)) + (size_t)k * k;   // after rank + sort scratch
    __shared__ double rdiag[64], rsg2[64];
    for (int i = threadIdx.x; i < r1; i += blockDim.x) {
      rdiag[i] = 1.0 / R[i * k + i];
      rsg2[i] = i < r ? 1.0 / (sg[i] * sg[i]) : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      double* tc = Ts + (size_t)c * k;
      for (int i = 0; i < k; ++i) tc[i] = 0.0;
      if (c < r) {
        for (int i = r1 - 1; i >= 0; --i) {
          double sacc = VR[c * r1 + i];
          for (int l = i + 1; l < r1; ++l) sacc -= R[l * k + i] * tc[l];
          tc[i] = sacc * rdiag[i];
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) T[t] = Ts[t];
    // VS = V_R[:, :r] Sigma^{-1} = A[:, c] / sigma_c^2
    for (int c = warp; c < k; c += nwarps)
      for (int i = lane; i < k; i += 32) VS[c * k + i] = c < r ? A[c * k + i] * rsg2[c] : 0.0;
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) sig[t] = t < r1 ? sg[t] : 0.0;
}
az_status launch_factor2(const double* G2, int k, const double* V, const double* lam, double tau, double floor,
                         double* T, double* VS, double* sig, FactorInfo* info, cudaStream_t st, bool f32jac) {
  if (k > 64) { set_error("factor: k > 64 not supported by the one-CTA factorisation"); return AZ_ERR_ARG; }
  // R, A, VR, sg, then the FP32 Jacobi copies or the sort's rank + scratch
  // R, A, VR, sg, then the FP32 Jacobi copies or the sort's rank + scratch,
  // then the back-substitution scratch
  size_t sm = (3 * (size_t)k * k + k) * sizeof(double) +
              std::max(2 * (size_t)k * k * sizeof(float), (size_t)(k + 1) * sizeof(int) + sizeof(int) + (size_t)k * k * sizeof(double)) +
              (size_t)k * k * sizeof(double);
  smem_once(k_factor2, sm);
  ProfScope ps("factor2", 0.0, st);
  (void)lam;
  k_factor2<<<1, 32 * std::max(1, std::min(32, (k + 1) / 2)), sm, st>>>(G2, k, V, tau, floor, T, VS, sig, info, f32jac ? 1 : 0);
  AZ_LCHECK();
  return AZ_OK;
}

__global__ void k_small_mm(const double* VS, int k, const double* c, int n, double* u) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * n) return;
  int i = t % k, j = t / k;
  double s = 0;
  for (int l = 0; l < k; ++l) s += VS[(int64_t)l * k + i] * c[(int64_t)j * k + l];
  u[t] = s;
}
az_status launch_small_mm(const double* VS, int k, const double* c, int n, double* u, cudaStream_t st) {
  ProfScope ps("small_mm", 0.0, st);
  k_small_mm<<<(k * n + 255) / 256, 256, 0, st>>>(VS, k, c, n, u);
  AZ_LCHECK();
  return AZ_OK;
}

// x[:, c] = (accumulate ? x : 0) + z[:, c] + W u[:, c]: one thread per
// coefficient j, its W row held in registers, all right-hand sides in a loop;
// arithmetic in the precision of W (FP32 in the mixed path), result stored FP64.
template <typename TW, typename TZ, int KB>
__global__ void __launch_bounds__(256) k_update_x(const TW* __restrict__ W, int64_t ldw, int k, const double* __restrict__ u,
                                                  const TZ* z, int64_t ldz, int64_t N, int nrhs,
                                                  double* __restrict__ x, int64_t ldx, int accumulate, float* xf,
                                                  const float* __restrict__ xbase) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TW* su = (TW*)smem_raw;   // [c*k + a]
  for (int t = threadIdx.x; t < k * nrhs; t += blockDim.x) su[t] = (TW)u[t];
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  TW w[KB];
#pragma unroll
  for (int a = 0; a < KB; ++a) w[a] = a < k ? W[(int64_t)a * ldw + j] : (TW)0;
  for (int c = 0; c < nrhs; ++c) {
    TW s = (TW)z[(int64_t)c * ldz + j];
    const TW* uc = su + c * k;
#pragma unroll
    for (int a = 0; a < KB; ++a) if (a < k) s = fma(w[a], uc[a], s);
    const double sd = cvt<double>(s);
    if (x) {
      double* xp = x + (int64_t)c * ldx + j;
      *xp = xbase ? (double)xbase[(int64_t)c * ldz + j] + sd : (accumulate ? *xp + sd : sd);
    }
    if (xf) xf[(int64_t)c * ldz + j] = (float)s;   // exact FP32 copy
  }
}
// FP32 variant for aligned shapes: a CTA stages its 512-row tile of W and all
// of u in shared memory; each warp then streams whole columns of z and x with
// 16-byte accesses (4 rows per lane), so every global access is a full,
// contiguous 512-byte warp transaction.
constexpr int UPX_ROWS = 512;
__global__ void __launch_bounds__(256) k_update_x_v4(const float* __restrict__ W, int64_t ldw, int k,
                                                     const double* __restrict__ u, const float* z, int64_t ldz,
                                                     int64_t N, int nrhs, double* x, int64_t ldx, int accumulate,
                                                     float* xf, const float* __restrict__ xbase) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sW = (float*)smem_raw;                 // [a][UPX_ROWS]
  float* su = sW + (size_t)k * UPX_ROWS;         // [c][k]
  const int64_t r0 = (int64_t)blockIdx.x * UPX_ROWS;
  const int rows = (int)(N - r0 < UPX_ROWS ? N - r0 : UPX_ROWS);   // multiple of 4
  for (int t = threadIdx.x; t < k * (UPX_ROWS / 4); t += blockDim.x) {
    const int a = t / (UPX_ROWS / 4), q = (t % (UPX_ROWS / 4)) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < rows) v = *(const float4*)(W + (int64_t)a * ldw + r0 + q);
    *(float4*)(sW + a * UPX_ROWS + q) = v;
  }
  for (int t = threadIdx.x; t < k * nrhs; t += blockDim.x) su[t] = (float)u[t];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NQ = UPX_ROWS / 128;   // 16-byte chunks per lane and column, loaded together
  for (int c = warp; c < nrhs; c += 8) {
    const float* uc = su + c * k;
    const float* zc = z + (int64_t)c * ldz + r0;
    double* xc = x ? x + (int64_t)c * ldx + r0 : nullptr;
    float4 s[NQ];
    double2 xa[NQ], xb[NQ];
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      const int q = lane * 4 + t * 128;
      s[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      xa[t] = make_double2(0.0, 0.0);
      xb[t] = make_double2(0.0, 0.0);
      if (q < rows) {
        s[t] = *(const float4*)(zc + q);
        if (xbase) {
          const float4 v = *(const float4*)(xbase + (int64_t)c * ldz + r0 + q);
          xa[t] = make_double2(v.x, v.y);
          xb[t] = make_double2(v.z, v.w);
        } else if (accumulate && xc) {
          xa[t] = *(const double2*)(xc + q);
          xb[t] = *(const double2*)(xc + q + 2);
        }
      }
    }
    for (int a = 0; a < k; ++a) {
      const float ua = uc[a];
#pragma unroll
      for (int t = 0; t < NQ; ++t) {
        const float4 w = *(const float4*)(sW + a * UPX_ROWS + lane * 4 + t * 128);
        s[t].x = fmaf(w.x, ua, s[t].x);
        s[t].y = fmaf(w.y, ua, s[t].y);
        s[t].z = fmaf(w.z, ua, s[t].z);
        s[t].w = fmaf(w.w, ua, s[t].w);
      }
    }
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      const int q = lane * 4 + t * 128;
      if (q >= rows) continue;
      if (xc) {
        xa[t].x += cvt<double>(s[t].x);
        xa[t].y += cvt<double>(s[t].y);
        xb[t].x += cvt<double>(s[t].z);
        xb[t].y += cvt<double>(s[t].w);
        *(double2*)(xc + q) = xa[t];
        *(double2*)(xc + q + 2) = xb[t];
      }
      if (xf) *(float4*)(xf + (int64_t)c * ldz + r0 + q) = s[t];   // exact FP32 copy
    }
  }
}

// FP32 variant with W in registers: a thread owns two consecutive rows (all
// k <= KB values of W for them in registers) and walks the right-hand sides
// in groups of 8, reading u for a group as two 16-byte shared loads per a.
// Every global access is a contiguous warp transaction (8 bytes of z, 16 of x
// per lane).
template <int KB, bool ACC64>
__global__ void __launch_bounds__(256) k_update_x_r2(const float* __restrict__ W, int64_t ldw, int k,
                                                     const double* __restrict__ u, const float* z, int64_t ldz,
                                                     int64_t N, int nrhs, double* x, int64_t ldx, int accumulate,
                                                     float* xf, const float* __restrict__ xbase) {
  constexpr int CG = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* su = (float*)smem_raw;   // [a][c], c padded to a multiple of CG
  const int nc8 = (nrhs + CG - 1) / CG * CG;
  for (int t = threadIdx.x; t < KB * nc8; t += blockDim.x) {
    const int a = t / nc8, c = t % nc8;
    su[t] = (a < k && c < nrhs) ? (float)u[c * k + a] : 0.f;
  }
  __syncthreads();
  const int64_t j = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= N) return;
  float2 w[KB];
#pragma unroll
  for (int a = 0; a < KB; ++a) w[a] = a < k ? *(const float2*)(W + (int64_t)a * ldw + j) : make_float2(0.f, 0.f);
  // x = base + s in FP64: base is the FP32 xbase or zero (ACC64 false: the
  // FP64 pipe is never used), or the FP64 x itself (ACC64: accumulating
  // without xbase)
  for (int c0 = 0; c0 < nrhs; c0 += CG) {
    float2 s[CG];
    float2 xb[CG];
    double2 xo[ACC64 ? CG : 1];
#pragma unroll
    for (int q = 0; q < CG; ++q) {
      const int c = c0 + q;
      s[q] = c < nrhs ? *(const float2*)(z + (int64_t)c * ldz + j) : make_float2(0.f, 0.f);
      if constexpr (ACC64) {
        if (c < nrhs) xo[q] = *(const double2*)(x + (int64_t)c * ldx + j);
      } else {
        xb[q] = (c < nrhs && xbase) ? *(const float2*)(xbase + (int64_t)c * ldz + j) : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      const float4 u0 = *(const float4*)(su + a * nc8 + c0);
      const float4 u1 = *(const float4*)(su + a * nc8 + c0 + 4);
      const float uu[CG] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
      for (int q = 0; q < CG; ++q) {
        s[q].x = fmaf(w[a].x, uu[q], s[q].x);
        s[q].y = fmaf(w[a].y, uu[q], s[q].y);
      }
    }
#pragma unroll
    for (int q = 0; q < CG; ++q) {
      const int c = c0 + q;
      if (c >= nrhs) break;
      if (x) {
        double2 r;
        if constexpr (ACC64) {
          r.x = xo[q].x + cvt<double>(s[q].x);
          r.y = xo[q].y + cvt<double>(s[q].y);
        } else {
          r.x = f32_sum_f64(xb[q].x, s[q].x);
          r.y = f32_sum_f64(xb[q].y, s[q].y);
        }
        *(double2*)(x + (int64_t)c * ldx + j) = r;
      }
      if (xf) *(float2*)(xf + (int64_t)c * ldz + j) = s[q];   // exact FP32 copy
    }
  }
}

template <typename TW, typename TZ>
az_status launch_update_x(const TW* W, int64_t ldw, int k, const double* u, const TZ* z, int64_t ldz, int64_t N,
                          int nrhs, double* x, int64_t ldx, bool accumulate, cudaStream_t st, float* xf,
                          const float* xbase) {
  // algorithmic bytes: W, z, then per column x written (and read when
  // accumulating), the FP32 base read, the FP32 copy written
  const double per_col = sizeof(TZ) + (x ? 8.0 * ((accumulate && !xbase) ? 2 : 1) : 0.0) + (xbase ? 4.0 : 0.0) +
                         (xf ? 4.0 : 0.0);
  ProfScope ps("update_x", (double)N * (k * sizeof(TW) + nrhs * per_col), st);
  if constexpr (sizeof(TW) == 4 && sizeof(TZ) == 4) {
    const bool al2 = N % 2 == 0 && ldw % 2 == 0 && ldz % 2 == 0 && ldx % 2 == 0 && ((uintptr_t)W & 7) == 0 &&
                     ((uintptr_t)z & 7) == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)xf & 7) == 0 &&
                     ((uintptr_t)xbase & 7) == 0;
    if (al2 && k <= 24) {
      const int nc8 = (nrhs + 7) / 8 * 8;
      const unsigned grid2 = (unsigned)((N / 2 + 255) / 256);
      const int acc = accumulate ? 1 : 0;
      const bool a64 = accumulate && x && !xbase;
#define AZ_UPX_R2(KB)                                                                                 \
  {                                                                                                   \
    auto kern = a64 ? k_update_x_r2<KB, true> : k_update_x_r2<KB, false>;                             \
    kern<<<grid2, 256, KB * nc8 * sizeof(float), st>>>(W, ldw, k, u, z, ldz, N, nrhs, x, ldx, acc, xf, xbase); \
  }
      if (k <= 8) AZ_UPX_R2(8)
      else if (k <= 16) AZ_UPX_R2(16)
      else AZ_UPX_R2(24)
#undef AZ_UPX_R2
      AZ_LCHECK();
      return AZ_OK;
    }
    const size_t sm4 = ((size_t)k * UPX_ROWS + (size_t)k * nrhs) * sizeof(float);
    const bool aligned = N % 4 == 0 && ldw % 4 == 0 && ldz % 4 == 0 && ldx % 2 == 0 && ((uintptr_t)W & 15) == 0 &&
                         ((uintptr_t)z & 15) == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)xf & 15) == 0 &&
                         ((uintptr_t)xbase & 15) == 0;
    if (aligned && sm4 <= 160 * 1024) {
      smem_once(k_update_x_v4, sm4);
      k_update_x_v4<<<(unsigned)((N + UPX_ROWS - 1) / UPX_ROWS), 256, sm4, st>>>(W, ldw, k, u, z, ldz, N, nrhs, x, ldx,
                                                                               accumulate ? 1 : 0, xf, xbase);
      AZ_LCHECK();
      return AZ_OK;
    }
  }
  size_t sm = (size_t)k * nrhs * sizeof(TW);
  unsigned grid = (unsigned)((N + 255) / 256);
  if (k <= 8) k_update_x<TW, TZ, 8><<<grid, 256, sm, st>>>(W, ldw, k, u, z, ldz, N, nrhs, x, ldx, accumulate ? 1 : 0, xf, xbase);
  else if (k <= 16) k_update_x<TW, TZ, 16><<<grid, 256, sm, st>>>(W, ldw, k, u, z, ldz, N, nrhs, x, ldx, accumulate ? 1 : 0, xf, xbase);
  else if (k <= 32) k_update_x<TW, TZ, 32><<<grid, 256, sm, st>>>(W, ldw, k, u, z, ldz, N, nrhs, x, ldx, accumulate ? 1 : 0, xf, xbase);
  else k_update_x<TW, TZ, 64><<<grid, 256, sm, st>>>(W, ldw, k, u, z, ldz, N, nrhs, x, ldx, accumulate ? 1 : 0, xf, xbase);
  AZ_LCHECK();
  return AZ_OK;
}

template az_status launch_gram<float, float>(const float*, int64_t, int, const float*, int64_t, int, int64_t, double*, double*, cudaStream_t, bool);
template az_status launch_gram<double, double>(const double*, int64_t, int, const double*, int64_t, int, int64_t, double*, double*, cudaStream_t, bool);
template az_status launch_gram<float, double>(const float*, int64_t, int, const double*, int64_t, int, int64_t, double*, double*, cudaStream_t, bool);
template az_status launch_tsprod<float, double>(const float*, int64_t, int, const double*, int, int64_t, double*, int64_t, cudaStream_t);
template az_status launch_tsprod<double, double>(const double*, int64_t, int, const double*, int, int64_t, double*, int64_t, cudaStream_t);
template az_status launch_tsprod<double, float>(const double*, int64_t, int, const double*, int, int64_t, float*, int64_t, cudaStream_t);
template az_status launch_tsprod<float, float>(const float*, int64_t, int, const double*, int, int64_t, float*, int64_t, cudaStream_t);
template az_status launch_update_x<float, float>(const float*, int64_t, int, const double*, const float*, int64_t, int64_t, int, double*, int64_t, bool, cudaStream_t, float*, const float*);
template az_status launch_update_x<double, double>(const double*, int64_t, int, const double*, const double*, int64_t, int64_t, int, double*, int64_t, bool, cudaStream_t, float*, const float*);
template az_status launch_update_x<double, float>(const double*, int64_t, int, const double*, const float*, int64_t, int64_t, int, double*, int64_t, bool, cudaStream_t, float*, const float*);

}  // namespace az
