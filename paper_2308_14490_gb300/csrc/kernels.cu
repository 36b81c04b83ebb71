// Kernels of the AZ hot path: index map (S1), symbol (S2), Rademacher bits
// (S3), the three FFT passes of the sketch / solve (S4, S5, S8, S10), the
// local A-apply stencils (S4, S8, S11) and boundary rows (Sec. 6.2).
#include <cmath>
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include "kernels.cuh"
#include "profile.cuh"
#include "fft_reg.cuh"

namespace az {

int image_count(double eps, double T) {
  int p = 1;
  while ((eps * (2 * p - 1) * T) * (eps * (2 * p - 1) * T) < 700.0) ++p;
  return p + 1;
}

static constexpr int TW_N = 4096;  // master twiddle table length
static inline size_t padix_host(size_t e, int sh) { return e + (e >> sh); }

// ------------------------------------------------------------------ utilities
// Raise a kernel's dynamic shared-memory limit once per (kernel, size) so that
// steady-state launches issue no attribute calls (solves can be captured into
// CUDA graphs).
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done;
  std::lock_guard<std::mutex> g(mu);
  auto it = done.find((const void*)kernel);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[(const void*)kernel] = bytes;
  return e;
}
#define AZ_LAUNCH_CHECK()                                               \
  do {                                                                  \
    cudaError_t _e = cudaGetLastError();                                \
    if (_e != cudaSuccess) {                                            \
      set_error(std::string("kernel launch: ") + cudaGetErrorString(_e) + " at " + __FILE__ + ":" + std::to_string(__LINE__)); \
      return AZ_ERR_CUDA;                                               \
    }                                                                   \
  } while (0)

// exp(-2 pi i m / n) with the angle reduced to the first octant in exact
// integer arithmetic before calling the FP64 library cos/sin.
static void twiddle_exact(int64_t m, int64_t n, double& re, double& im) {
  m %= n; if (m < 0) m += n;
  // angle = 2 pi m / n = pi * (2m) / n ; work with fraction a/b of pi, a in [0, 2b)
  int64_t a = 2 * m, b = n;
  bool neg_s = false, neg_c = false, swap = false;
  if (2 * a > 2 * b) { a = 2 * b - a; neg_s = true; }            // (pi, 2pi]: sin flips
  if (2 * a > b) { a = b - a; neg_c = true; }                    // (pi/2, pi]: cos flips
  if (4 * a > b) { a = b - 2 * a; b = 2 * b; swap = true; }      // (pi/4, pi/2]: swap via pi/2 - x
  const double x = M_PI * (double)a / (double)b;
  double c = std::cos(x), s = std::sin(x);
  if (swap) std::swap(c, s);
  if (neg_c) c = -c;
  if (neg_s) s = -s;
  re = c; im = -s;  // exp(-i angle)
}

void host_twiddles(int n, std::vector<double>& re, std::vector<double>& im) {
  re.resize(n); im.resize(n);
  for (int m = 0; m < n; ++m) twiddle_exact(m, n, re[m], im[m]);
}

// ------------------------------------------------------------------ S1: index map
__global__ void k_count(const uint8_t* __restrict__ mask, int64_t L, int32_t* __restrict__ blk) {
  __shared__ int s[32];
  int64_t base = (int64_t)blockIdx.x * 4096;
  int cnt = 0;
  for (int t = threadIdx.x; t < 4096; t += blockDim.x) {
    int64_t i = base + t;
    if (i < L && mask[i]) ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s[w];
    blk[blockIdx.x] = tot;
  }
}
__global__ void k_scan_blocks(int32_t* blk, int nb, int64_t* M_dev) {
  // one thread, sequential exclusive scan (nb <= 4096)
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t acc = 0;
    for (int b = 0; b < nb; ++b) { int32_t v = blk[b]; blk[b] = (int32_t)acc; acc += v; }
    *M_dev = acc;
  }
}
__global__ void k_scatter(const uint8_t* __restrict__ mask, int64_t L, const int32_t* __restrict__ blk,
                          int32_t* __restrict__ pos2m, int32_t* __restrict__ idx) {
  // 256 threads, each 16 consecutive elements of the 4096-block
  __shared__ int wsum[8];
  int64_t base = (int64_t)blockIdx.x * 4096 + threadIdx.x * 16;
  int loc[16];
  int cnt = 0;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    int64_t i = base + e;
    int v = (i < L && mask[i]) ? 1 : 0;
    loc[e] = v; cnt += v;
  }
  // block exclusive scan of cnt
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, incl, o); if (lane >= o) incl += y; }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int wpre = 0;
  for (int q = 0; q < w; ++q) wpre += wsum[q];
  int run = blk[blockIdx.x] + wpre + incl - cnt;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    int64_t i = base + e;
    if (i < L) {
      if (loc[e]) { pos2m[i] = run; idx[run] = (int32_t)i; ++run; }
      else pos2m[i] = -1;
    }
  }
}
az_status launch_compact(const uint8_t* mask, int64_t L, int32_t* pos2m, int32_t* idx, int64_t* M_dev,
                         int32_t* scratch, cudaStream_t st) {
  int nb = (int)((L + 4095) / 4096);
  if (nb > 4096) { set_error("grid too large for the index map"); return AZ_ERR_ARG; }
  ProfScope ps("compact", 6.0 * L, st, 3);
  k_count<<<nb, 256, 0, st>>>(mask, L, scratch);
  k_scan_blocks<<<1, 32, 0, st>>>(scratch, nb, M_dev);
  k_scatter<<<nb, 256, 0, st>>>(mask, L, scratch, pos2m, idx);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ S2: samples, taps
// g(m) = sum_p f((m + p L) h_L), f = phi or phi'' (Eq. periodic_rbf on the L-grid)
__device__ double periodised_sample(int64_t m, int64_t L, double hL, double eps, int deriv, int pimg) {
  m = ((m % L) + L) % L;
  const double mm = (double)(m > L / 2 ? m - L : m);
  const double e2 = eps * eps;
  double acc = 0.0;
  for (int p = -pimg; p <= pimg; ++p) {
    const double r = (mm + (double)p * (double)L) * hL;
    const double q = e2 * r * r;
    if (q > 760.0) continue;   // exp(-q) underflows to zero in FP64
    const double ex = exp(-q);
    acc += deriv == 0 ? ex : -2.0 * e2 * ex * (1.0 - 2.0 * e2 * r * r);
  }
  return acc;
}
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}
az_status launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st) {
  ProfScope ps("samples", 24.0 * n, st);
  k_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, y);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_samples(double* g, int64_t L, double hL, double eps, int deriv, int pimg) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  g[m] = periodised_sample(m, L, hL, eps, deriv, pimg);
}
az_status launch_samples(double* g, int64_t L, double hL, double eps, int deriv, int pimg, cudaStream_t st) {
  ProfScope ps("samples", 8.0 * L, st);
  k_samples<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(g, L, hL, eps, deriv, pimg);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
// a window of half-width L/2 sees offset L/2 from both ends: half the sample each
__device__ __forceinline__ double edge_half(int64_t m, int64_t L) { return 2 * (m < 0 ? -m : m) == L ? 0.5 : 1.0; }
__global__ void k_taps(const double* g, int64_t L, int W64, double* t64, int W32, float* t32, float* th, float* tl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= 2 * W64) {
    const int64_t m = (int64_t)i - W64;
    const double v = g[fmod_pos(m, L)] * edge_half(m, L);
    t64[i] = v;
    if (th) { const float h = (float)v; th[i] = h; tl[i] = (float)(v - (double)h); }
  }
  if (i <= 2 * W32) {
    const int64_t m = (int64_t)i - W32;
    t32[i] = (float)(g[fmod_pos(m, L)] * edge_half(m, L));
  }
}
// Taps straight from the image sum (1D: the L samples themselves are not needed)
// (ode != 0: taps of the collocation kernel -(phi'' + k0^2 phi) / (2 eps^2), Example 6.1)
__device__ __forceinline__ double tap_value(int64_t m, int64_t L, double hL, double eps, int pimg, int ode, double k0) {
  const double g0 = periodised_sample(m, L, hL, eps, 0, pimg);
  if (!ode) return g0;
  const double g2 = periodised_sample(m, L, hL, eps, 2, pimg);
  return -(g2 + k0 * k0 * g0) / (2.0 * eps * eps);
}
__global__ void k_taps_direct(int64_t L, double hL, double eps, int pimg, int W64, double* t64, int W32, float* t32,
                              float* th, float* tl, int ode, double k0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= 2 * W64) {
    const int64_t m = (int64_t)i - W64;
    const double v = tap_value(m, L, hL, eps, pimg, ode, k0) * edge_half(m, L);
    t64[i] = v;
    if (th) { const float h = (float)v; th[i] = h; tl[i] = (float)(v - (double)h); }
  }
  if (i <= 2 * W32) {
    const int64_t m = (int64_t)i - W32;
    t32[i] = (float)(tap_value(m, L, hL, eps, pimg, ode, k0) * edge_half(m, L));
  }
}
az_status launch_taps_direct(int64_t L, double hL, double eps, int pimg, int W64, double* t64, int W32, float* t32,
                             cudaStream_t st, float* th, float* tl, int ode, double k0) {
  const int W = W64 > W32 ? W64 : W32;
  ProfScope ps("taps", 12.0 * (2 * W + 1), st);
  k_taps_direct<<<(2 * W + 1 + 127) / 128, 128, 0, st>>>(L, hL, eps, pimg, W64, t64, W32, t32, th, tl, ode, k0);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// 1D symbol from the Poisson-summation form of DFT_L(g) (proof of Lemma 4.3):
// with a = eps h_L and t = k/L taken in [-1/2, 1/2],
//   Ghat_k = sqrt(pi)/a * sum_p exp(-(pi/a)^2 (t + p)^2),
// which equals the DFT of the periodised samples to rounding (the oracle pins
// both forms against each other).  A thread takes J consecutive k (never
// across k = L/2, where t jumps) and, per image p, evaluates the Gaussian by
// the exact recurrence E_{j+1} = E_j F_j, F_{j+1} = F_j Q (u_j = t_j + p,
// F_j = exp(-c d (2 u_j + d)), Q = exp(-2 c d^2), d = 1/L): three FP64
// exponentials per image and J outputs instead of one per output (FP64 exp is
// slow on this part), at a cost of about 2J rounding units.
constexpr int SYM_J = 16;
// (ode != 0: the symbol of -(phi'' + k0^2 phi) / (2 eps^2); the Fourier
// transform of phi'' is -(2 pi nu)^2 times that of phi, nu = (t + p) / h_L)
__global__ void k_symbol_closed_1d(int64_t L, double a, int Q, int J, double* Ghat, int ode, double hL, double kw,
                                   double eps) {
  const int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * J;
  if (k0 >= L) return;
  const double c = (M_PI / a) * (M_PI / a);
  const double d = 1.0 / (double)L;
  const double t0 = (double)(k0 > L / 2 ? k0 - L : k0) * d;
  double acc[SYM_J], acc2[SYM_J];
#pragma unroll
  for (int j = 0; j < SYM_J; ++j) { acc[j] = 0.0; acc2[j] = 0.0; }
  const double q = exp(-2.0 * c * d * d);
  // the largest image over the run has exponent at most c * emax^2, with
  // emax the largest |t| of the run reduced to [-1/2, 1/2]; images whose
  // exponent exceeds that by 40 everywhere on the run add below 2^-57 of
  // the sum and are skipped
  const double te = fmin(fmax(fabs(t0), fabs(t0 + (J - 1) * d)), 0.5);
  const double ecut = c * te * te + 40.0;
  for (int p = -Q; p <= Q; ++p) {
    const double u0 = t0 + (double)p;
    const double umin = fmin(fabs(u0), fabs(u0 + (J - 1) * d));
    if (u0 * (u0 + (J - 1) * d) > 0.0 && c * umin * umin > fmin(ecut, 745.0)) continue;
    double e = exp(-c * u0 * u0);
    double f = exp(-c * d * (2.0 * u0 + d));
#pragma unroll
    for (int j = 0; j < SYM_J; ++j) {
      if (j < J) {
        acc[j] += e;
        if (ode) {
          const double u = u0 + j * d;
          acc2[j] += e * u * u;
        }
      }
      e *= f;
      f *= q;
    }
  }
  const double sc = sqrt(M_PI) / a;
  const double w2 = (2.0 * M_PI / hL) * (2.0 * M_PI / hL);
#pragma unroll
  for (int j = 0; j < SYM_J; ++j)
    if (j < J) Ghat[k0 + j] = ode ? sc * (w2 * acc2[j] - kw * kw * acc[j]) / (2.0 * eps * eps) : sc * acc[j];
}
az_status launch_symbol_closed_1d(int64_t L, double a, double* Ghat, cudaStream_t st, int ode, double hL, double k0,
                                  double eps) {
  const int Q = (int)std::ceil(0.5 + a * std::sqrt(745.0) / M_PI);
  const int J = (L % (2 * SYM_J) == 0) ? SYM_J : 1;   // runs end at k = L/2
  const int64_t nth = L / J;
  ProfScope ps("symbol", 8.0 * L, st);
  k_symbol_closed_1d<<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(L, a, Q, J, Ghat, ode, hL, k0, eps);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

az_status launch_taps(const double* g, int64_t L, int W64, double* t64, int W32, float* t32, cudaStream_t st,
                      float* th, float* tl) {
  const int W = W64 > W32 ? W64 : W32;
  ProfScope ps("taps", 12.0 * (2 * W + 1), st);
  k_taps<<<(2 * W + 1 + 127) / 128, 128, 0, st>>>(g, L, W64, t64, W32, t32, th, tl);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ S3: Philox bits
__global__ void k_philox_bits(uint32_t* bits, int64_t N, int k, uint32_t k0, uint32_t k1) {
  // one thread per (column, 128-row block) -> 4 words
  int64_t nblk = (N + 127) / 128;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int col = blockIdx.y;
  if (t >= nblk || col >= k) return;
  uint4 o = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)col, 0u, 0u), k0, k1);
  int64_t nw = (N + 31) / 32;
  uint32_t w[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int64_t wi = t * 4 + q;
    if (wi < nw) bits[(int64_t)col * nw + wi] = w[q];
  }
}
az_status launch_philox_bits(uint32_t* bits, int64_t N, int k, uint64_t seed, cudaStream_t st) {
  int64_t nblk = (N + 127) / 128;
  dim3 grid((unsigned)((nblk + 127) / 128), (unsigned)k);
  ProfScope ps("philox_bits", 4.0 * ((N + 31) / 32) * k, st);
  k_philox_bits<<<grid, 128, 0, st>>>(bits, N, k, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_bits_to_R(const uint32_t* bits, int64_t N, int k, double* R) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int col = blockIdx.y;
  if (j >= N) return;
  R[(int64_t)col * N + j] = (double)rad_bit(bits, (N + 31) / 32, j, col);
}
az_status launch_bits_to_R(const uint32_t* bits, int64_t N, int k, double* R, cudaStream_t st) {
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)k);
  ProfScope ps("bits_to_R", 8.25 * N * k, st);
  k_bits_to_R<<<grid, 256, 0, st>>>(bits, N, k, R);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ FFT pass helpers
template <typename V>
__device__ __forceinline__ V big_tw(const V* __restrict__ A, const V* __restrict__ B, int m, bool inv) {
  V w = cmul(__ldg(A + (m >> 12)), __ldg(B + (m & 4095)));
  if (inv) w.y = -w.y;
  return w;
}
// w^(c * o) for the outputs o = o0 + u * Ns of one butterfly of a last FFT
// stage: w^(c * o0) is gathered once per butterfly and w^(c * Ns * 2^b) once per
// thread, so an output costs at most four complex products (u < 16) instead of
// two table gathers; the result is within a few rounding units of the table.
template <typename V>
struct BigTwPow {
  V p[4];
  V base;
  __device__ __forceinline__ void init(const V* A, const V* B, int c, int Ns, int R, bool inv) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if ((1 << b) < R) p[b] = big_tw<V>(A, B, c * (Ns << b), inv);
  }
  __device__ __forceinline__ V at(const V* A, const V* B, int c, int u, int o0, bool inv) {
    if (u == 0) base = big_tw<V>(A, B, c * o0, inv);
    V w = base;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (u & (1 << b)) w = cmul(w, p[b]);
    return w;
  }
};
// stride Ns and radix R of the last stage of fft_reg for a line of 2^logn with E per thread
__device__ __forceinline__ void last_stage_shape(int logn, int logE, int& Ns, int& R) {
  if (logn >= logE) { Ns = 1 << (logn - logE); R = 1 << logE; }
  else { Ns = 1; R = 1 << logn; }
}

// ceil(a / 2^l) and floor(a / 2^l) for signed a (arithmetic shift floors)
__device__ __forceinline__ int cdiv_p2(int a, int l) { return -((-a) >> l); }
__device__ __forceinline__ int fdiv_p2(int a, int l) { return a >> l; }

static int ilog2i(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

// Column tile width for a column pass of FFT length n (ping-pong buffers <= 128 KB).
template <typename V> static int col_tile(int n, int ncols) {
  int c = (int)(65536 / ((size_t)n * sizeof(V)));
  int p = 1;
  while (p * 2 <= c && p * 2 <= 16) p *= 2;
  return std::max(1, std::min(p, ncols));
}

// Forward column FFT of the tile held in s0 (layout [i*C + c]) then store with
// the four-step twiddle (1D) into X1[pair][k0*D1 + n1].
template <typename T>
__device__ void colfwd_finish(const Geom& g, typename C2<T>::t* s0, typename C2<T>::t* s1, int logC, int c0,
                              typename C2<T>::t* __restrict__ X1, const PassTabs& tb) {
  using V = typename C2<T>::t;
  __syncthreads();
  int cur = fft_lines<V, false>(s0, s1, g.logD0, logC, 1, 1 << logC, (const V*)tb.tw, TW_N >> g.logD0);
  V* res = cur ? s1 : s0;
  const int total = g.D0 << logC;
  const int Cm = (1 << logC) - 1;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int c = t & Cm, k0 = t >> logC;
    const int n1 = c0 + c;
    V v = res[t];
    if (g.dim == 1 && k0 != 0 && n1 != 0) v = cmul(v, big_tw<V>((const V*)tb.bigA, (const V*)tb.bigB, n1 * k0, false));
    X1[(k0 << g.logD1) + n1] = v;
  }
}

// Sketch prologue: v = mask * (A^c R) at the tile's grid points, two Rademacher
// columns packed as (real, imag).
template <typename T>
__global__ void __launch_bounds__(256) k_colfwd_stencil(Geom g, SketchIn<T> in, int pair0, int logC,
                                                        typename C2<T>::t* X1base, PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = 1 << logC, Cm = C - 1;
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)g.D0 * C;
  const int c0 = blockIdx.x * C;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  const bool hasB = colB < in.k;
  V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  if (g.dim == 1) {
    const int ls = g.logs[0], s = g.s[0];
    const int Nm = (int)g.N - 1;
    const int W = in.Wx;
    const int total = g.D0 << logC;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int c = t & Cm, n0 = t >> logC;
      const int pos = (n0 << g.logD1) + c0 + c;
      T re = 0, im = 0;
      if (__ldg(in.pos2m + pos) >= 0) {
        const int jlo = cdiv_p2(pos - W, ls), jhi = fdiv_p2(pos + W, ls);
        for (int j = jlo; j <= jhi; ++j) {
          const T tap = __ldg(in.tapx + (pos - s * j + W));
          const int jj = j & Nm;
          re += tap * (T)rad_bit(in.bits, in.nw, jj, colA);
          if (hasB) im += tap * (T)rad_bit(in.bits, in.nw, jj, colB);
        }
      }
      V v; v.x = re; v.y = im;
      s0[t] = v;
    }
  } else {
    // separable: t[jx][c] = sum_jy gy(iy - sy jy) R[jx, jy]  (into s1), then
    // v[ix][c] = mask * sum_jx gx(ix - sx jx) t[jx][c]      (into s0)
    const int sx = g.s[0], sy = g.s[1];
    const int Nxm = (int)g.n[0] - 1, Nym = (int)g.n[1] - 1, lNy = g.logn[1];
    const int tot1 = (int)g.n[0] << logC;
    for (int t = threadIdx.x; t < tot1; t += blockDim.x) {
      const int c = t & Cm, jx = t >> logC;
      const int iy = c0 + c;
      const int jlo = cdiv_p2(iy - in.Wy, g.logs[1]), jhi = fdiv_p2(iy + in.Wy, g.logs[1]);
      T re = 0, im = 0;
      for (int jy = jlo; jy <= jhi; ++jy) {
        const T tap = __ldg(in.tapy + (iy - sy * jy + in.Wy));
        const int j = (jx << lNy) + (jy & Nym);
        re += tap * (T)rad_bit(in.bits, in.nw, j, colA);
        if (hasB) im += tap * (T)rad_bit(in.bits, in.nw, j, colB);
      }
      V v; v.x = re; v.y = im;
      s1[t] = v;
    }
    __syncthreads();
    const int tot0 = g.D0 << logC;
    for (int t = threadIdx.x; t < tot0; t += blockDim.x) {
      const int c = t & Cm, ix = t >> logC;
      const int pos = (ix << g.logD1) + c0 + c;
      V v; v.x = 0; v.y = 0;
      if (__ldg(in.pos2m + pos) >= 0) {
        const int jlo = cdiv_p2(ix - in.Wx, g.logs[0]), jhi = fdiv_p2(ix + in.Wx, g.logs[0]);
        for (int jx = jlo; jx <= jhi; ++jx) {
          const T tap = __ldg(in.tapx + (ix - sx * jx + in.Wx));
          const V u = s1[((jx & Nxm) << logC) + c];
          v.x += tap * u.x; v.y += tap * u.y;
        }
      }
      s0[t] = v;
    }
    __syncthreads();  // s1 is reused by the FFT
  }
  colfwd_finish<T>(g, s0, s1, logC, c0, X1, tb);
}

template <typename T, typename TB>
__global__ void __launch_bounds__(256) k_colfwd_gather(Geom g, const int32_t* __restrict__ pos2m, const TB* __restrict__ b,
                                                       int64_t ldb, int ncols, int pair0, int logC,
                                                       typename C2<T>::t* X1base, PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = 1 << logC, Cm = C - 1;
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)g.D0 * C;
  const int c0 = blockIdx.x * C;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  const TB* bA = b + (int64_t)colA * ldb;
  const TB* bB = b + (int64_t)colB * ldb;
  const bool hasB = colB < ncols;
  V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  const int total = g.D0 << logC;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int c = t & Cm, n0 = t >> logC;
    const int pos = (n0 << g.logD1) + c0 + c;
    const int m = __ldg(pos2m + pos);
    V v; v.x = 0; v.y = 0;
    if (m >= 0) {
      v.x = (T)bA[m];
      if (hasB) v.y = (T)bB[m];
    }
    s0[t] = v;
  }
  colfwd_finish<T>(g, s0, s1, logC, c0, X1, tb);
}


template <typename T>
az_status launch_colfwd_stencil_v1(const Geom& g, const SketchIn<T>& in, int pair0, int npairs,
                                typename C2<T>::t* X1, const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  int C = col_tile<V>(g.D0, g.D1);
  size_t sm = 2 * (size_t)g.D0 * C * sizeof(V);
  if (set_smem(k_colfwd_stencil<T>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D1 / C, npairs);
  ProfScope ps(sizeof(T) == 4 ? "colfwd_sketch_f32" : "colfwd_sketch_f64", (double)npairs * g.L * sizeof(V) + npairs * 2.0 * g.N / 8 + 4.0 * g.L, st);
  k_colfwd_stencil<T><<<grid, 256, sm, st>>>(g, in, pair0, ilog2i(C), X1, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
template <typename T, typename TB>
az_status launch_colfwd_gather_v1(const Geom& g, const int32_t* pos2m, const TB* b, int64_t ldb, int ncols,
                               int pair0, int npairs, typename C2<T>::t* X1, const PassTabs& tb,
                               cudaStream_t st, int64_t M_rows) {
  using V = typename C2<T>::t;
  int C = col_tile<V>(g.D0, g.D1);
  size_t sm = 2 * (size_t)g.D0 * C * sizeof(V);
  if (set_smem(k_colfwd_gather<T, TB>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D1 / C, npairs);
  ProfScope ps(sizeof(T) == 4 ? "colfwd_gather_f32" : "colfwd_gather_f64", (double)npairs * g.L * sizeof(V) + (double)std::min(ncols - 2 * pair0, 2 * npairs) * M_rows * sizeof(TB) + 4.0 * g.L, st);
  k_colfwd_gather<T, TB><<<grid, 256, sm, st>>>(g, pos2m, b, ldb, ncols, pair0, ilog2i(C), X1, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ row passes
template <typename V> static int row_groups_per_cta(const Geom& g) {
  size_t per = (size_t)g.Rg * g.D1 * sizeof(V) * 2;
  int gp = (int)std::max<size_t>(1, 65536 / per);
  int p = 1;
  while (p * 2 <= gp && p * 2 <= 8) p *= 2;
  int ngroups = g.G0;
  while (p > 1 && ngroups % p) p >>= 1;
  return p;
}


// Row pass of the sketch / solve: forward FFT of each group's rows, fold of the
// alias group with H = Ghat/S (Eq. B_pinv), inverse FFT of length N1, twiddle
// (1D four-step), store on the N-grid layout X3[pair][G*N1 + n1].
template <typename T>
__global__ void __launch_bounds__(256) k_rowfold(Geom g, const typename C2<T>::t* __restrict__ X1base,
                                                 const T* __restrict__ H, int logGPB, typename C2<T>::t* X3base,
                                                 PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int GPB = 1 << logGPB;
  const int lognr = logGPB + g.logRg;
  const int nrows = 1 << lognr;
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)nrows * g.D1;
  const V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  V* X3 = X3base + (int64_t)blockIdx.y * g.N;
  const int G0 = blockIdx.x * GPB;
  const int D1m = g.D1 - 1, Rgm = g.Rg - 1, N1m = g.N1 - 1;
  // load rows: local row lr = gg*Rg + q  <->  global row (G0+gg) + q*Rstride
  const int total = nrows << g.logD1;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int lr = t >> g.logD1, i = t & D1m;
    const int gg = lr >> g.logRg, q = lr & Rgm;
    const int row = G0 + gg + q * g.Rstride;
    s0[t] = X1[(row << g.logD1) + i];
  }
  __syncthreads();
  int cur = fft_lines<V, false>(s0, s1, g.logD1, lognr, g.D1, 1, (const V*)tb.tw, TW_N >> g.logD1);
  V* X = cur ? s1 : s0;
  V* F = cur ? s0 : s1;  // fold output lines [gg][N1]
  const int totF = GPB << g.logN1;
  for (int t = threadIdx.x; t < totF; t += blockDim.x) {
    const int gg = t >> g.logN1, k1 = t & N1m;
    T ar = 0, ai = 0;
    for (int q = 0; q < g.Rg; ++q) {
      const int row = G0 + gg + q * g.Rstride;
      const V* xr = X + ((gg * g.Rg + q) << g.logD1);
      const T* hr = H + ((int64_t)row << g.logD1);
      for (int p = 0; p < g.Fq; ++p) {
        const int kk = k1 + p * g.N1;
        const T hh = __ldg(hr + kk);
        const V xv = xr[kk];
        ar += hh * xv.x; ai += hh * xv.y;
      }
    }
    V o; o.x = ar; o.y = ai;
    F[t] = o;
  }
  __syncthreads();
  int c2 = fft_lines<V, true>(F, X, g.logN1, logGPB, g.N1, 1, (const V*)tb.tw, TW_N >> g.logN1);
  V* Z = c2 ? X : F;
  for (int t = threadIdx.x; t < totF; t += blockDim.x) {
    const int gg = t >> g.logN1, n1 = t & N1m;
    const int k0 = G0 + gg;
    V v = Z[t];
    if (g.dim == 1 && k0 != 0 && n1 != 0) v = cmul(v, big_tw<V>((const V*)tb.bigNA, (const V*)tb.bigNB, n1 * k0, true));
    X3[(k0 << g.logN1) + n1] = v;
  }
}
template <typename T>
az_status launch_rowfold_v1(const Geom& g, const typename C2<T>::t* X1, const T* H, int npairs,
                         typename C2<T>::t* X3, const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  int GPB = row_groups_per_cta<V>(g);
  size_t sm = 2 * (size_t)GPB * g.Rg * g.D1 * sizeof(V);
  if (set_smem(k_rowfold<T>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.G0 / GPB, npairs);
  ProfScope ps(sizeof(T) == 4 ? "rowfold_f32" : "rowfold_f64", (double)npairs * (g.L + g.N) * sizeof(V) + (double)g.L * sizeof(T), st);
  k_rowfold<T><<<grid, 256, sm, st>>>(g, X1, H, ilog2i(GPB), X3, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ inverse column pass
template <typename T, typename TO>
__global__ void __launch_bounds__(256) k_colinv(Geom g, const typename C2<T>::t* __restrict__ X3base, int pair0,
                                                int ncols, int logC, TO* __restrict__ out, int64_t ldo,
                                                const uint32_t* __restrict__ bits, int64_t nw, PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int C = 1 << logC, Cm = C - 1;
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)g.G0 * C;
  const int c0 = blockIdx.x * C;
  const V* X3 = X3base + (int64_t)blockIdx.y * g.N;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  const bool hasB = colB < ncols;
  TO* oA = out + (int64_t)colA * ldo;
  TO* oB = out + (int64_t)colB * ldo;
  const int total = g.G0 << logC;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int c = t & Cm, k0 = t >> logC;
    s0[t] = X3[(k0 << g.logN1) + c0 + c];
  }
  __syncthreads();
  int cur = fft_lines<V, true>(s0, s1, g.logG0, logC, 1, C, (const V*)tb.tw, TW_N >> g.logG0);
  V* res = cur ? s1 : s0;
  const T sc = (T)(1.0 / (double)g.N);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int c = t & Cm, n0 = t >> logC;
    const int j = (n0 << g.logN1) + c0 + c;
    const V v = res[t];
    T za = v.x * sc, zb = v.y * sc;
    if (bits) {
      za = (T)rad_bit(bits, nw, j, colA) - za;
      if (hasB) zb = (T)rad_bit(bits, nw, j, colB) - zb;
    }
    oA[j] = (TO)za;
    if (hasB) oB[j] = (TO)zb;
  }
}
template <typename T, typename TO>
az_status launch_colinv_v1(const Geom& g, const typename C2<T>::t* X3, int pair0, int npairs, int ncols,
                        TO* out, int64_t ldo, const uint32_t* bits, int64_t nw, const PassTabs& tb,
                        cudaStream_t st) {
  using V = typename C2<T>::t;
  int C = col_tile<V>(g.G0, g.N1);
  size_t sm = 2 * (size_t)g.G0 * C * sizeof(V);
  if (set_smem(k_colinv<T, TO>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.N1 / C, npairs);
  ProfScope ps(sizeof(T) == 4 ? "colinv_f32" : "colinv_f64", (double)npairs * g.N * sizeof(V) + (double)std::min(ncols - 2 * pair0, 2 * npairs) * g.N * sizeof(TO), st);
  k_colinv<T, TO><<<grid, 256, sm, st>>>(g, X3, pair0, ncols, ilog2i(C), out, ldo, bits, nw, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ stencils
// Rows of A at the kept grid points: out[m, c] = alpha*b[m, c] + beta*(A z)[m, c].
// One thread per kept point m and a group of CPT columns (index arithmetic and
// taps shared across the group).
constexpr int STENCIL_WIN = 512;   // coefficients staged per block and column (1D)
// b into the arithmetic type of the stencil rows; FP64 -> FP32 branch-free
// (round to nearest, ties away; the loads of all columns stay in flight)
template <typename T, typename TB> __device__ __forceinline__ T cvt_b(TB v) {
  if constexpr (sizeof(T) == 4 && sizeof(TB) == 8) return d2f_fast(v);
  else return cvt<T>(v);
}
// The block's window of coefficients, columns cbase .. cbase + nc - 1 and
// entries wlo .. wlo + nwin - 1 (periodic index), into swin[c * STENCIL_WIN + o]:
// a thread takes entries o = threadIdx.x + q blockDim.x and issues the loads
// of all its columns before any store (no integer division).
template <typename TZ, int CPT>
__device__ __forceinline__ void stage_window(TZ* swin, const TZ* __restrict__ zb, int64_t ldz, int cbase, int nc, int wlo,
                                             int nwin, int Nm) {
  for (int o = threadIdx.x; o < nwin; o += blockDim.x) {
    const int64_t jj = (wlo + o) & Nm;
    TZ v[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) v[c] = c < nc ? zb[(int64_t)(cbase + c) * ldz + jj] : (TZ)0;
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (c < nc) swin[c * STENCIL_WIN + o] = v[c];
  }
  __syncthreads();
}
template <typename T, typename TZ, typename TB, typename TO, int CPT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 5) k_stencil_rows(Geom g, int kind, T inv2e2, const int32_t* __restrict__ idx, int M,
                                                      const T* __restrict__ x0, const T* __restrict__ x2,
                                                      const T* __restrict__ y0, const T* __restrict__ y2, int Wx, int Wy,
                                                      const TZ* __restrict__ zb, int64_t ldz, const TB* __restrict__ bb,
                                                      int64_t ldb, T alpha, T beta, TO* __restrict__ outb, int64_t ldo,
                                                      int ncols) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = m < M;
  const int cbase = blockIdx.y * CPT;
  const int nc = min(CPT, ncols - cbase);
  const int i = act ? __ldg(idx + m) : 0;
  T acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = 0;
  if (g.dim == 1) {
    const int ls = g.logs[0], s = g.s[0], Nm = (int)g.N - 1;
    const int jlo = cdiv_p2(i - Wx, ls), jhi = fdiv_p2(i + Wx, ls);
    // coefficients the block needs: one window when its rows are (nearly)
    // contiguous, staged once in shared memory with coalesced loads
    const int m0 = blockIdx.x * blockDim.x;
    const int m1 = min(M, m0 + (int)blockDim.x) - 1;
    const int wlo = cdiv_p2(__ldg(idx + m0) - Wx, ls), whi = fdiv_p2(__ldg(idx + m1) + Wx, ls);
    const int nwin = whi - wlo + 1;
    __shared__ TZ swin[CPT * STENCIL_WIN];
    if (nwin <= STENCIL_WIN) {
      stage_window<TZ, CPT>(swin, zb, ldz, cbase, nc, wlo, nwin, Nm);
      if (act) {
        for (int j = jlo; j <= jhi; ++j) {
          const T tap = __ldg(x0 + (i - s * j + Wx));
#pragma unroll
          for (int c = 0; c < CPT; ++c)
            if (c < nc) acc[c] += tap * (T)swin[c * STENCIL_WIN + (j - wlo)];
        }
      }
    } else if (act) {
      for (int j = jlo; j <= jhi; ++j) {
        const T tap = __ldg(x0 + (i - s * j + Wx));
        const int jj = j & Nm;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
          if (c < nc) acc[c] += tap * (T)__ldg(zb + (int64_t)(cbase + c) * ldz + jj);
      }
    }
  } else if (act) {
    const int sx = g.s[0], sy = g.s[1];
    const int Nxm = (int)g.n[0] - 1, Nym = (int)g.n[1] - 1, lNy = g.logn[1];
    const int ix = i >> g.logD1, iy = i & (g.D1 - 1);
    const int xlo = cdiv_p2(ix - Wx, g.logs[0]), xhi = fdiv_p2(ix + Wx, g.logs[0]);
    const int ylo = cdiv_p2(iy - Wy, g.logs[1]), yhi = fdiv_p2(iy + Wy, g.logs[1]);
    for (int jx = xlo; jx <= xhi; ++jx) {
      const int rowoff = (jx & Nxm) << lNy;
      const T tx0 = __ldg(x0 + (ix - sx * jx + Wx));
      const T tx2 = kind == 1 ? __ldg(x2 + (ix - sx * jx + Wx)) : (T)0;
      for (int jy = ylo; jy <= yhi; ++jy) {
        const T ty0 = __ldg(y0 + (iy - sy * jy + Wy));
        T w = tx0 * ty0;
        if (kind == 1) w = -(tx2 * ty0 + tx0 * __ldg(y2 + (iy - sy * jy + Wy))) * inv2e2;
        const int jj = rowoff + (jy & Nym);
#pragma unroll
        for (int c = 0; c < CPT; ++c)
          if (c < nc) acc[c] += w * (T)__ldg(zb + (int64_t)(cbase + c) * ldz + jj);
      }
    }
  }
  if (!act) return;
  // b after the stencil: its registers stay free during the window loop
  TB bv[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) bv[c] = (bb && c < nc) ? bb[(int64_t)(cbase + c) * ldb + m] : (TB)0;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    if (c < nc) {
      T r = beta * acc[c];
      if (bb) r += alpha * cvt_b<T>(bv[c]);
      outb[(int64_t)(cbase + c) * ldo + m] = cvt<TO>(r);
    }
  }
}
template <typename T, typename TZ, typename TB, typename TO>
az_status launch_stencil_rows(const Geom& g, int kind, double eps, const int32_t* idx, int64_t M,
                              const StencilTaps& tp, const TZ* z, int64_t ldz, const TB* b, int64_t ldb,
                              T alpha, T beta, TO* out, int64_t ldo, int ncols, cudaStream_t st) {
  if (M == 0 || ncols == 0) return AZ_OK;
  constexpr int CPT = sizeof(T) == 4 ? 8 : 4;
  dim3 grid((unsigned)((M + 255) / 256), (ncols + CPT - 1) / CPT);
  ProfScope ps(sizeof(T) == 4 ? "stencil_rows_f32" : "stencil_rows_f64", (double)g.N * ncols * sizeof(TZ) + (double)M * ncols * ((b ? sizeof(TB) : 0) + sizeof(TO)) + 4.0 * M, st);
  k_stencil_rows<T, TZ, TB, TO, CPT><<<grid, 256, 0, st>>>(g, kind, (T)(1.0 / (2.0 * eps * eps)), idx, (int)M, (const T*)tp.x0,
                                                           (const T*)tp.x2, (const T*)tp.y0, (const T*)tp.y2, tp.Wx,
                                                           tp.Wy, z, ldz, b, ldb, alpha, beta, out, ldo, ncols);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// FP64-accurate residual rows r = b - A x in double-FP32 arithmetic, for
// coefficients x that are exactly representable in FP32 (the mixed path's
// first-pass solution is formed in FP32).  Each FP64 tap is split into FP32
// hi + lo; tap*x = hi*x (exact: product + fma error) + lo*x, accumulated with
// two-sum; the ~48-bit sum is subtracted from b in FP64.
struct DFa { float hi, lo; };
__device__ __forceinline__ void dfa_add(DFa& s, float x, float th, float tl) {
  const float p = th * x;
  const float e = fmaf(th, x, -p);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += err + fmaf(tl, x, e);
}
// (ah + al) * (bh + bl) as a double-float (hi exact product + cross terms)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  ph = ah * bh;
  pl = fmaf(ah, bh, -ph) + fmaf(ah, bl, al * bh);
}
// the staged 1D window: acc[c] += sum_j tap(i - s j) x[j, c] for j in [jlo, jhi]
template <int CPT, bool FULL>
__device__ __forceinline__ void resid_win(DFa (&acc)[CPT], const float* swin, int jlo, int jhi, int wlo, int i, int s,
                                          int Wx, const float* __restrict__ x0h, const float* __restrict__ x0l, int nc) {
  for (int j = jlo; j <= jhi; ++j) {
    const int ti = i - s * j + Wx;
    const float th = __ldg(x0h + ti), tl = __ldg(x0l + ti);
    const float* w = swin + (j - wlo);
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (FULL || c < nc) dfa_add(acc[c], w[c * STENCIL_WIN], th, tl);
  }
}
template <int CPT>
__global__ void __launch_bounds__(256) k_resid_df(Geom g, int kind, double inv2e2, const int32_t* __restrict__ idx, int M,
                                                  const float* __restrict__ x0h, const float* __restrict__ x0l,
                                                  const float* __restrict__ x2h, const float* __restrict__ x2l,
                                                  const float* __restrict__ y0h, const float* __restrict__ y0l,
                                                  const float* __restrict__ y2h, const float* __restrict__ y2l,
                                                  int Wx, int Wy, const float* __restrict__ xf, int64_t ldx,
                                                  const double* __restrict__ bb, int64_t ldb, float* __restrict__ out,
                                                  int64_t ldo, int ncols) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = m < M;
  const int cbase = blockIdx.y * CPT;
  const int nc = min(CPT, ncols - cbase);
  const int i = act ? __ldg(idx + m) : 0;
  DFa acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) { acc[c].hi = 0.f; acc[c].lo = 0.f; }
  if (g.dim == 1) {
    const int ls = g.logs[0], s = g.s[0], Nm = (int)g.N - 1;
    const int jlo = cdiv_p2(i - Wx, ls), jhi = fdiv_p2(i + Wx, ls);
    // the block's window of x staged in shared memory (as in k_stencil_rows)
    const int m0 = blockIdx.x * blockDim.x;
    const int m1 = min(M, m0 + (int)blockDim.x) - 1;
    const int wlo = cdiv_p2(__ldg(idx + m0) - Wx, ls), whi = fdiv_p2(__ldg(idx + m1) + Wx, ls);
    const int nwin = whi - wlo + 1;
    __shared__ float swin[CPT * STENCIL_WIN];
    if (nwin <= STENCIL_WIN) {
      stage_window<float, CPT>(swin, xf, ldx, cbase, nc, wlo, nwin, Nm);
      if (act) {
        // block-uniform: a full group of CPT columns runs without per-column predicates
        if (nc == CPT) resid_win<CPT, true>(acc, swin, jlo, jhi, wlo, i, s, Wx, x0h, x0l, nc);
        else resid_win<CPT, false>(acc, swin, jlo, jhi, wlo, i, s, Wx, x0h, x0l, nc);
      }
    } else if (act) {
      for (int j = jlo; j <= jhi; ++j) {
        const int ti = i - s * j + Wx;
        const float th = __ldg(x0h + ti), tl = __ldg(x0l + ti);
        const int jj = j & Nm;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
          if (c < nc) dfa_add(acc[c], __ldg(xf + (int64_t)(cbase + c) * ldx + jj), th, tl);
      }
    }
  } else if (act) {
    const int sx = g.s[0], sy = g.s[1];
    const int Nxm = (int)g.n[0] - 1, Nym = (int)g.n[1] - 1, lNy = g.logn[1];
    const int ix = i >> g.logD1, iy = i & (g.D1 - 1);
    const int xlo = cdiv_p2(ix - Wx, g.logs[0]), xhi = fdiv_p2(ix + Wx, g.logs[0]);
    const int ylo = cdiv_p2(iy - Wy, g.logs[1]), yhi = fdiv_p2(iy + Wy, g.logs[1]);
    for (int jx = xlo; jx <= xhi; ++jx) {
      const int rowoff = (jx & Nxm) << lNy;
      const int tx = ix - sx * jx + Wx;
      const float ah = __ldg(x0h + tx), al = __ldg(x0l + tx);
      const float a2h = kind == 1 ? __ldg(x2h + tx) : 0.f, a2l = kind == 1 ? __ldg(x2l + tx) : 0.f;
      for (int jy = ylo; jy <= yhi; ++jy) {
        const int ty = iy - sy * jy + Wy;
        const float bh = __ldg(y0h + ty), bl = __ldg(y0l + ty);
        float wh, wl;
        df_mul(ah, al, bh, bl, wh, wl);
        if (kind == 1) {
          float uh, ul, vh, vl;
          df_mul(a2h, a2l, bh, bl, uh, ul);
          df_mul(ah, al, __ldg(y2h + ty), __ldg(y2l + ty), vh, vl);
          // w = -(u + v) * inv2e2 (FP64 scalar applied after the sum below)
          const float sh = uh + vh;
          const float bz = sh - uh;
          const float se = (uh - (sh - bz)) + (vh - bz) + ul + vl;
          wh = sh; wl = se;
        }
        const int jj = rowoff + (jy & Nym);
#pragma unroll
        for (int c = 0; c < CPT; ++c)
          if (c < nc) dfa_add(acc[c], __ldg(xf + (int64_t)(cbase + c) * ldx + jj), wh, wl);
      }
    }
  }
  if (!act) return;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    if (c < nc) {
      const double bv = bb[(int64_t)(cbase + c) * ldb + m];
      if (g.dim == 2 && kind == 1) {
        double ax = -((double)acc[c].hi + (double)acc[c].lo) * inv2e2;
        out[(int64_t)(cbase + c) * ldo + m] = (float)(bv - ax);
      } else {
        // r = (bh + bl) - (hi + lo) with a two-difference on the leading terms
        float bh, bl;
        d2ff_int(bv, bh, bl);
        const float sd = bh - acc[c].hi;
        const float bz = sd - bh;
        const float er = (bh - (sd - bz)) + (-acc[c].hi - bz);
        out[(int64_t)(cbase + c) * ldo + m] = sd + (er + (bl - acc[c].lo));
      }
    }
  }
}
az_status launch_resid_df(const Geom& g, int kind, double eps, const int32_t* idx, int64_t M, const float* const th[4],
                          const float* const tl[4], int Wx, int Wy, const float* xf, int64_t ldx, const double* b,
                          int64_t ldb, float* out, int64_t ldo, int ncols, cudaStream_t st) {
  if (M == 0 || ncols == 0) return AZ_OK;
  constexpr int CPT = 4;
  dim3 grid((unsigned)((M + 255) / 256), (ncols + CPT - 1) / CPT);
  ProfScope ps("resid_df", (double)g.N * ncols * 4 + (double)M * ncols * (8 + 4) + 4.0 * M, st);
  const float* y0h = g.dim == 1 ? th[0] : th[1];
  const float* y0l = g.dim == 1 ? tl[0] : tl[1];
  const float* y2h = g.dim == 1 ? th[2] : th[3];
  const float* y2l = g.dim == 1 ? tl[2] : tl[3];
  k_resid_df<CPT><<<grid, 256, 0, st>>>(g, kind, 1.0 / (2.0 * eps * eps), idx, (int)M, th[0], tl[0], th[2], tl[2], y0h, y0l,
                                        y2h, y2l, Wx, g.dim == 1 ? Wx : Wy, xf, ldx, b, ldb, out, ldo, ncols);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// phi_per at distance d (center window handles the images): plain Gaussian
// and its first derivative, -2 eps^2 d exp(-eps^2 d^2)
template <typename T> __device__ __forceinline__ T gauss(T d, T eps) { T e = eps * d; return exp(-e * e); }
template <typename T> __device__ __forceinline__ T dgauss(T d, T eps) {
  T e = eps * d;
  return (T)-2 * eps * e * exp(-e * e);
}

// Centers within reach of a point, per dimension: the 2 Wc + 2 nearest ones,
// one image each, while the Gaussian falls below exp(-42) inside that window;
// otherwise (small grids, wide kernels) all n_d centers, each with its image
// sum |p| <= P (Eq. periodic_rbf).
struct CenterWin { int W[2]; int P[2]; };
static CenterWin center_window(const Geom& g, double eps) {
  CenterWin cw{};
  for (int d = 0; d < g.dim; ++d) {
    const double h = 2.0 * g.T[d] / (double)g.n[d];
    const int64_t need = (int64_t)std::ceil(std::sqrt(42.0) / (eps * h)) + 1;
    if (2 * need + 2 <= g.n[d]) { cw.W[d] = (int)need; cw.P[d] = 0; }
    else { cw.W[d] = (int)(g.n[d] / 2 - 1); cw.P[d] = image_count(eps, g.T[d]); }
  }
  return cw;
}
template <typename T> __device__ __forceinline__ T gauss_per(T d, T eps, T twoT, int P) {
  T a = gauss<T>(d, eps);
  for (int p = 1; p <= P; ++p) a += gauss<T>(d - (T)p * twoT, eps) + gauss<T>(d + (T)p * twoT, eps);
  return a;
}
template <typename T> __device__ __forceinline__ T dgauss_per(T d, T eps, T twoT, int P) {
  T a = dgauss<T>(d, eps);
  for (int p = 1; p <= P; ++p) a += dgauss<T>(d - (T)p * twoT, eps) + dgauss<T>(d + (T)p * twoT, eps);
  return a;
}

// Boundary rows (Sec. 6.1, 6.2, 6.3): out = alpha b + beta w A^b z.  A point
// with a nonzero normal n (nrm, Mb x dim, may be null) gives the Neumann row
// n . grad phi_j(p) / eps; the others the Dirichlet row phi_j(p).
template <typename T, typename TZ, typename TB, typename TO>
__global__ void k_boundary_rows(Geom g, T eps, T w, CenterWin cw, const double* __restrict__ pts,
                                const double* __restrict__ nrm, int64_t Mb,
                                const TZ* __restrict__ zb, int64_t ldz, const TB* __restrict__ bb, int64_t ldb,
                                T alpha, T beta, TO* __restrict__ outb, int64_t ldo) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Mb) return;
  const int c = blockIdx.y;
  const TZ* z = zb + (int64_t)c * ldz;
  const T ieps = (T)1 / eps;
  if (g.dim == 1) {
    const double px = pts[m], hx = 2.0 * g.T[0] / g.n[0];
    const T nx = nrm ? (T)nrm[m] : (T)0, tx = (T)(2.0 * g.T[0]);
    const int Wc = cw.W[0], P = cw.P[0];
    const int64_t cxi = (int64_t)floor((px + g.T[0]) / hx);
    T acc = 0;
    if (nx != (T)0) {
      for (int64_t jx = cxi - Wc; jx <= cxi + Wc + 1; ++jx)
        acc += dgauss_per<T>((T)(px - (-g.T[0] + (double)jx * hx)), eps, tx, P) * (T)z[fmod_pos(jx, g.n[0])];
      acc *= nx * ieps;
    } else {
      for (int64_t jx = cxi - Wc; jx <= cxi + Wc + 1; ++jx)
        acc += gauss_per<T>((T)(px - (-g.T[0] + (double)jx * hx)), eps, tx, P) * (T)z[fmod_pos(jx, g.n[0])];
    }
    T r = beta * w * acc;
    if (bb) r += alpha * (T)bb[(int64_t)c * ldb + m];
    outb[(int64_t)c * ldo + m] = (TO)r;
    return;
  }
  const double px = pts[2 * m], py = pts[2 * m + 1];
  const T nx = nrm ? (T)nrm[2 * m] : (T)0, ny = nrm ? (T)nrm[2 * m + 1] : (T)0;
  const bool neu = nx != (T)0 || ny != (T)0;
  const double hx = 2.0 * g.T[0] / g.n[0], hy = 2.0 * g.T[1] / g.n[1];
  const T tx = (T)(2.0 * g.T[0]), ty = (T)(2.0 * g.T[1]);
  const int64_t cxi = (int64_t)floor((px + g.T[0]) / hx), cyi = (int64_t)floor((py + g.T[1]) / hy);
  T acc = 0;
  for (int64_t jx = cxi - cw.W[0]; jx <= cxi + cw.W[0] + 1; ++jx) {
    const T dx = (T)(px - (-g.T[0] + (double)jx * hx));
    const T wx = gauss_per<T>(dx, eps, tx, cw.P[0]);
    const TZ* zr = z + fmod_pos(jx, g.n[0]) * g.n[1];
    T a0 = 0, a1 = 0;
    for (int64_t jy = cyi - cw.W[1]; jy <= cyi + cw.W[1] + 1; ++jy) {
      const T dy = (T)(py - (-g.T[1] + (double)jy * hy));
      const T zv = (T)zr[fmod_pos(jy, g.n[1])];
      a0 += gauss_per<T>(dy, eps, ty, cw.P[1]) * zv;
      if (neu) a1 += dgauss_per<T>(dy, eps, ty, cw.P[1]) * zv;
    }
    if (neu) acc += nx * dgauss_per<T>(dx, eps, tx, cw.P[0]) * a0 + ny * wx * a1;
    else acc += wx * a0;
  }
  if (neu) acc *= ieps;
  T r = beta * w * acc;
  if (bb) r += alpha * (T)bb[(int64_t)c * ldb + m];
  outb[(int64_t)c * ldo + m] = (TO)r;
}
template <typename T, typename TZ, typename TB, typename TO>
az_status launch_boundary_rows(const Geom& g, double eps, double w, const double* pts, const double* nrm, int64_t Mb,
                               const TZ* z, int64_t ldz, const TB* b, int64_t ldb, T alpha, T beta,
                               TO* out, int64_t ldo, int ncols, cudaStream_t st) {
  if (Mb == 0 || ncols == 0) return AZ_OK;
  dim3 grid((unsigned)((Mb + 127) / 128), ncols);
  ProfScope ps("boundary_rows", (double)Mb * ncols * ((b ? sizeof(TB) : 0) + sizeof(TO)) + 16.0 * Mb, st);
  k_boundary_rows<T, TZ, TB, TO><<<grid, 128, 0, st>>>(g, (T)eps, (T)w, center_window(g, eps), pts, nrm, Mb, z, ldz,
                                                       b, ldb, alpha, beta, out, ldo);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// Boundary data of a collocation solve: out = w g on Dirichlet points and
// w g / eps on Neumann points (the row scalings of k_boundary_rows).
__global__ void k_boundary_rhs(int dim, const double* __restrict__ g, int64_t ldg, int64_t Mb,
                               const double* __restrict__ nrm, double w, double w_eps, double* __restrict__ out,
                               int64_t ldo) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Mb) return;
  const int c = blockIdx.y;
  bool neu = false;
  if (nrm)
    for (int d = 0; d < dim; ++d) neu |= nrm[(int64_t)dim * m + d] != 0.0;
  out[(int64_t)c * ldo + m] = (neu ? w_eps : w) * g[(int64_t)c * ldg + m];
}
az_status launch_boundary_rhs(int dim, const double* g, int64_t ldg, int64_t Mb, int ncols, const double* nrm,
                              double w, double eps, double* out, int64_t ldo, cudaStream_t st) {
  if (Mb == 0 || ncols == 0) return AZ_OK;
  dim3 grid((unsigned)((Mb + 127) / 128), ncols);
  ProfScope ps("boundary_rhs", 16.0 * Mb * ncols, st);
  k_boundary_rhs<<<grid, 128, 0, st>>>(dim, g, ldg, Mb, nrm, w, w / eps, out, ldo);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// Evaluation on the s_test-refined box grid (FP64)
__global__ void k_evaluate(Geom g, double eps, int st_, CenterWin cw, const double* __restrict__ xb, int64_t ldx,
                           double* __restrict__ outb, int64_t ldo, int64_t npts) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npts) return;
  const int c = blockIdx.y;
  const double* x = xb + (int64_t)c * ldx;
  double acc = 0;
  if (g.dim == 1) {
    const int64_t Lt = g.n[0] * st_;
    const double h = 2.0 * g.T[0] / g.n[0], tx = 2.0 * g.T[0];
    const double px = -g.T[0] + (double)q * (2.0 * g.T[0] / (double)Lt);
    const int64_t ci = (int64_t)floor((px + g.T[0]) / h);
    for (int64_t j = ci - cw.W[0]; j <= ci + cw.W[0] + 1; ++j)
      acc += gauss_per<double>(px - (-g.T[0] + (double)j * h), eps, tx, cw.P[0]) * x[fmod_pos(j, g.n[0])];
  } else {
    const int64_t Lty = g.n[1] * st_;
    const int64_t ix = q / Lty, iy = q % Lty;
    const double hx = 2.0 * g.T[0] / g.n[0], hy = 2.0 * g.T[1] / g.n[1];
    const double tx = 2.0 * g.T[0], ty = 2.0 * g.T[1];
    const double px = -g.T[0] + (double)ix * hx / st_, py = -g.T[1] + (double)iy * hy / st_;
    const int64_t cxi = (int64_t)floor((px + g.T[0]) / hx), cyi = (int64_t)floor((py + g.T[1]) / hy);
    for (int64_t jx = cxi - cw.W[0]; jx <= cxi + cw.W[0] + 1; ++jx) {
      double wx = gauss_per<double>(px - (-g.T[0] + (double)jx * hx), eps, tx, cw.P[0]);
      const double* zr = x + fmod_pos(jx, g.n[0]) * g.n[1];
      double a = 0;
      for (int64_t jy = cyi - cw.W[1]; jy <= cyi + cw.W[1] + 1; ++jy)
        a += gauss_per<double>(py - (-g.T[1] + (double)jy * hy), eps, ty, cw.P[1]) * zr[fmod_pos(jy, g.n[1])];
      acc += wx * a;
    }
  }
  outb[(int64_t)c * ldo + q] = acc;
}
az_status launch_evaluate(const Geom& g, double eps, int s_test, const double* x, int64_t ldx, int nrhs,
                          double* out, int64_t ldo, cudaStream_t st) {
  int64_t npts = g.dim == 1 ? g.n[0] * s_test : g.n[0] * s_test * g.n[1] * s_test;
  dim3 grid((unsigned)((npts + 255) / 256), nrhs);
  ProfScope ps("evaluate", 8.0 * npts * nrhs + 8.0 * g.N * nrhs, st);
  k_evaluate<<<grid, 256, 0, st>>>(g, eps, s_test, center_window(g, eps), x, ldx, out, ldo, npts);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ symbol assembly
__global__ void k_symbol_full(Geom g, int kind, double inv2e2, const double* G0x, const double* G0y,
                              const double* G2x, const double* G2y, double* Ghat) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.L) return;
  if (g.dim == 1) { Ghat[t] = G0x[t]; return; }
  int64_t kx = t / g.D1, ky = t % g.D1;
  if (kind == 0) Ghat[t] = G0x[kx] * G0y[ky];
  else Ghat[t] = -(G2x[kx] * G0y[ky] + G0x[kx] * G2y[ky]) * inv2e2;
}
az_status launch_symbol_full(const Geom& g, int kind, double eps, const double* G0x, const double* G0y,
                             const double* G2x, const double* G2y, double* Ghat, cudaStream_t st) {
  ProfScope ps("symbol", 8.0 * g.L, st);
  k_symbol_full<<<(unsigned)((g.L + 255) / 256), 256, 0, st>>>(g, kind, 1.0 / (2.0 * eps * eps), G0x, G0y, G2x, G2y, Ghat);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_fold_S(Geom g, const double* __restrict__ Gh, double* __restrict__ S) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.N) return;
  double acc = 0;
  if (g.dim == 1) {
    for (int q = 0; q < g.s[0]; ++q) { double v = Gh[k + q * g.N]; acc += v * v; }
  } else {
    int64_t kx = k / g.n[1], ky = k % g.n[1];
    for (int qx = 0; qx < g.s[0]; ++qx)
      for (int qy = 0; qy < g.s[1]; ++qy) { double v = Gh[(kx + qx * g.n[0]) * g.D1 + ky + qy * g.n[1]]; acc += v * v; }
  }
  S[k] = acc;
}
az_status launch_fold_S(const Geom& g, const double* Ghat, double* S, cudaStream_t st) {
  ProfScope ps("symbol", 8.0 * (g.L + g.N), st);
  k_fold_S<<<(unsigned)((g.N + 255) / 256), 256, 0, st>>>(g, Ghat, S);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_H(Geom g, const double* __restrict__ Gh, const double* __restrict__ S, const double* thr_dev,
                    double thr_rel, double* H64, float* H32) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.L) return;
  const double thr = thr_rel * (*thr_dev);
  int64_t row = t / g.D1, col = t % g.D1;
  int64_t fnat, k;
  if (g.dim == 1) { fnat = row + (int64_t)g.D0 * col; k = fnat % g.N; }
  else { fnat = t; k = (row % g.n[0]) * g.n[1] + (col % g.n[1]); }
  double s = S[k];
  double h = (s > thr && s > 0) ? Gh[fnat] / s : 0.0;
  H64[t] = h; H32[t] = (float)h;
}
az_status launch_H(const Geom& g, const double* Ghat, const double* S, double thr, double* H64, float* H32,
                   cudaStream_t st) {
  // thr: relative threshold tau_sym^2; the max of S is expected in H64 scratch? no: S max stored at S[g.N]
  ProfScope ps("symbol", 8.0 * (2 * g.L + g.N) + 4.0 * g.L, st);
  k_H<<<(unsigned)((g.L + 255) / 256), 256, 0, st>>>(g, Ghat, S, S + g.N, thr, H64, H32);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
// max |v_i| over all blocks: block maxima combined by an integer atomicMax on
// the IEEE bit patterns (for non-negative doubles their order is the numeric
// order); *out must hold +0.0 before the launch.
__global__ void k_max_abs(const double* __restrict__ v, int64_t n, unsigned long long* out) {
  __shared__ double sm[32];
  double m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(v[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sm[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong(r));
  }
}
az_status launch_max_abs(const double* v, int64_t n, double* out, cudaStream_t st) {
  ProfScope ps("symbol", 8.0 * n, st);
  AZ_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  const int64_t want = (n + 1023) / 1024;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 4 * 152));
  k_max_abs<<<blocks, 1024, 0, st>>>(v, n, (unsigned long long*)out);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_line_dft_real(const double* in, int logn, double* out, const double2* tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = 1 << logn;
  double2* s0 = (double2*)smem_raw;
  double2* s1 = s0 + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s0[i] = make_double2(in[i], 0.0);
  __syncthreads();
  int cur = fft_lines<double2, false>(s0, s1, logn, 0, n, 1, tw, TW_N >> logn);
  double2* r = cur ? s1 : s0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = r[i].x;
}
az_status launch_line_dft_real(const double* in, int n, double* out, const double2* tw, cudaStream_t st) {
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  size_t sm = 2 * (size_t)n * sizeof(double2);
  if (set_smem(k_line_dft_real, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  ProfScope ps("symbol", 16.0 * n, st);
  k_line_dft_real<<<1, 256, sm, st>>>(in, logn, out, tw);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ elementwise
__global__ void k_scale_rows(const double* in, int64_t ldi, int64_t rows, double sc, double* out, int64_t ldo) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= rows) return;
  int c = blockIdx.y;
  out[(int64_t)c * ldo + m] = sc * in[(int64_t)c * ldi + m];
}
az_status launch_scale_rows(const double* in, int64_t ldi, int64_t rows, int ncols, double sc, double* out,
                            int64_t ldo, cudaStream_t st) {
  if (rows == 0 || ncols == 0) return AZ_OK;
  dim3 grid((unsigned)((rows + 255) / 256), ncols);
  ProfScope ps("scale_rows", 16.0 * rows * ncols, st);
  k_scale_rows<<<grid, 256, 0, st>>>(in, ldi, rows, sc, out, ldo);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_sumsq_cols(const double* v, int64_t ld, int64_t rows, double* out) {
  __shared__ double sm[32];
  int c = blockIdx.x;
  double a = 0;
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) { double x = v[(int64_t)c * ld + i]; a += x * x; }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sm[w];
    out[c] = r;
  }
}
az_status launch_sumsq_cols(const double* v, int64_t ld, int64_t rows, int ncols, double* out, cudaStream_t st) {
  if (ncols == 0) return AZ_OK;
  ProfScope ps("sumsq", 8.0 * rows * ncols, st);
  k_sumsq_cols<<<ncols, 1024, 0, st>>>(v, ld, rows, out);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ================================================================== register-resident passes
// Same three passes as above, with the FFT held in registers (E values per
// thread) and one padded shared buffer; used whenever every FFT length of the
// pass is >= E.  E = 16 (FP32) or 8 (FP64).
// Values per thread (FP32 / FP64) and CTA shape of the register passes:
// 256 threads and 3 CTAs per SM (80 registers) keep the load, compute and
// store phases of different CTAs overlapped without spilling.
#ifndef AZ_REG_E32
#define AZ_REG_E32 16
#endif
#ifndef REG_THREADS
#define REG_THREADS 256
#endif
#ifndef REG_MINB
#define REG_MINB 3
#endif
#define PADC 4   // shared-memory padding: one element every 16 (column and row layouts)
template <typename T> struct EPT {
  static constexpr int E = sizeof(T) == 4 ? AZ_REG_E32 : 8;
  static constexpr int LOGE = E == 16 ? 4 : (E == 8 ? 3 : 2);
};

// Cache hints of the register passes' single-use traffic (the b gather, and the
// X1 / X3 intermediates, each written once and read once by the next pass):
// AZ_STREAM_LD loads them evict-first, AZ_STREAM_ST stores them as streaming.
#ifndef AZ_STREAM_LD
#define AZ_STREAM_LD 0
#endif
#ifndef AZ_STREAM_ST
#define AZ_STREAM_ST 0
#endif
template <typename V> __device__ __forceinline__ V ld1(const V* p) {
  if constexpr (AZ_STREAM_LD) return __ldcs(p);
  else return *p;
}
template <typename V> __device__ __forceinline__ void st1(V* p, V v) {
  if constexpr (AZ_STREAM_ST) __stcs(p, v);
  else *p = v;
}

// Compile-time shapes for the register passes.  ShapeRT leaves every size to
// the Geom at run time; Shape1D<LL, LS, LC> fixes a 1D grid with L = 2^LL,
// s = 2^LS and 2^LC lines per CTA, so that all FFT index arithmetic folds to
// constants (the passes are issue-bound, about half of it integer work).
// THR, MINB: block size and minimum resident blocks of the column passes
// (FP32, 16 values per thread: 2^LC columns of length D0 need 2^LC D0 / 16
// threads).
struct ShapeRT {
  static constexpr bool fixed = false;
  static constexpr int logD1 = 0, logD0 = 0, logN1 = 0, logC = 0;
  static constexpr int THR = REG_THREADS, MINB = REG_MINB;
};
template <int LL, int LS, int LC>
struct Shape1D {
  static constexpr bool fixed = true;
  static constexpr int logD1 = (LL + 1) / 2, logD0 = LL - logD1, logN1 = logD1 - LS, logC = LC;
  static constexpr int THR = (1 << LC) * ((1 << logD0) / 16);
  static constexpr int MINB = THR >= 1024 ? 1 : 1024 / THR;
};
// Columns per CTA of the compile-time column passes (L = 2^21, s = 2):
// 2^AZ_COL_LC columns of 1024, i.e. 8 * 2^AZ_COL_LC bytes of every grid row per
// CTA for the complex FP32 intermediates.
#ifndef AZ_COL_LC
#define AZ_COL_LC 3
#endif
template <class S>
__device__ __forceinline__ Geom fix_geom(const Geom& g) {
  Geom r = g;
  if constexpr (S::fixed) {
    r.dim = 1;
    r.logD0 = S::logD0; r.D0 = 1 << S::logD0;
    r.logD1 = S::logD1; r.D1 = 1 << S::logD1;
    r.logN1 = S::logN1; r.N1 = 1 << S::logN1;
    r.logG0 = S::logD0; r.G0 = 1 << S::logD0;
    r.Rg = 1; r.logRg = 0; r.Rstride = 0; r.Fq = 1 << (S::logD1 - S::logN1);
    r.logs[0] = S::logD1 - S::logN1; r.s[0] = 1 << r.logs[0];
    r.L = (int64_t)1 << (S::logD0 + S::logD1); r.N = r.L >> r.logs[0]; r.logN = S::logD0 + S::logN1;
  }
  return r;
}
// Row of b for grid point pos, or -1 outside Omega: arithmetic when the kept
// points are one run of grid indices, else the index map.
__device__ __forceinline__ int kept_row(const Geom& g, const int32_t* __restrict__ pos2m, int pos) {
  if (g.runM > 0) {
    const int64_t m = (int64_t)pos - g.run0;
    return (m >= 0 && m < g.runM) ? (int)m : -1;
  }
  return __ldg(pos2m + pos);
}
// Host side: the fixed shape a launch may use (config-2 scale: L = 2^21, s = 2)
static bool is_shape_21_1(const Geom& g) { return g.dim == 1 && g.L == ((int64_t)1 << 21) && g.s[0] == 2; }

template <typename T, int MODE, typename TB, class S>
__global__ void __launch_bounds__(S::THR, S::MINB) k_colfwd_r(Geom g_in, const int32_t* __restrict__ pos2m, const TB* __restrict__ b,
                                                  int64_t ldb, int ncols, SketchIn<T> in, int pair0, int logC_in,
                                                  typename C2<T>::t* X1base, PassTabs tb) {
  const Geom g = fix_geom<S>(g_in);
  const int logC = S::fixed ? S::logC : logC_in;
  // MODE 0: gather b (E b on the grid); MODE 1: sketch stencil A^c R with the mask
  using V = typename C2<T>::t;
  constexpr int E = EPT<T>::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = (V*)smem_raw;
  const int C = 1 << logC;
  const int line = threadIdx.x & (C - 1), tl = threadIdx.x >> logC;
  const int c0 = blockIdx.x * C;
  const int n1 = c0 + line;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  const V* twp = (const V*)tb.tw;
  // 2D sketch: y-stencil of R into a staging region after the FFT buffer
  V* stg = sm + padix<PADC>(g.D0 << logC) + 32;
  if (MODE == 1 && g.dim == 2) {
    const int sy = g.s[1];
    const int Nym = (int)g.n[1] - 1, lNy = g.logn[1];
    const int tot1 = (int)g.n[0] << logC;
    const bool hasB = colB < in.k;
    for (int t = threadIdx.x; t < tot1; t += blockDim.x) {
      const int c = t & (C - 1), jx = t >> logC;
      const int iy = c0 + c;
      const int jlo = cdiv_p2(iy - in.Wy, g.logs[1]), jhi = fdiv_p2(iy + in.Wy, g.logs[1]);
      T re = 0, im = 0;
      for (int jy = jlo; jy <= jhi; ++jy) {
        const T tap = __ldg(in.tapy + (iy - sy * jy + in.Wy));
        const int j = (jx << lNy) + (jy & Nym);
        re += tap * (T)rad_bit(in.bits, in.nw, j, colA);
        if (hasB) im += tap * (T)rad_bit(in.bits, in.nw, j, colB);
      }
      V v; v.x = re; v.y = im;
      stg[t] = v;
    }
    __syncthreads();
  }
  if (MODE == 1) {
    // sketch: v = mask * A^c R at every tile point, staged into the FFT
    // buffer (keeps the stencil out of the unrolled first stage)
    const int tot = g.D0 << logC;
    const bool hasB = colB < in.k;
    // FP32 1D windows of at most 16 taps: a point's window starts at tap
    // 2W - ph (ph = its phase mod s), so the signed sum of 8 consecutive taps
    // (+tap for a set Rademacher bit, -tap for a clear one) for a byte of bits
    // is a table entry T[ph][chunk][byte], and v = T[ph][0][b0] + T[ph][1][b1]
    float* tab = (float*)stg;
    const bool use_tab = sizeof(T) == 4 && g.dim == 1 && (2 * in.Wx) / g.s[0] + 1 <= 16;
    if (use_tab) {
      const int s = g.s[0], W = in.Wx;
      for (int e = threadIdx.x; e < s * 512; e += blockDim.x) {
        const int byte = e & 255, ch = (e >> 8) & 1, ph = e >> 9;
        float acc = 0.f;
        for (int u = 0; u < 8; ++u) {
          const int ti = 2 * W - ph - s * (8 * ch + u);
          if (ti >= 0) {
            const float tv = (float)__ldg(in.tapx + ti);
            acc += ((byte >> u) & 1) ? tv : -tv;
          }
        }
        tab[e] = acc;
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int c = t & (C - 1), p = t >> logC;
      const int pos = (p << g.logD1) + c0 + c;
      V v; v.x = 0; v.y = 0;
      if (kept_row(g, pos2m, pos) >= 0) {
        if (g.dim == 1) {
          const int ls = g.logs[0], s = g.s[0], Nm = (int)g.N - 1, W = in.Wx;
          const int jlo = cdiv_p2(pos - W, ls), jhi = fdiv_p2(pos + W, ls);
          if (jlo >= 0 && jhi < (int)g.N && jhi - jlo < 32) {
            // no wrap-around and at most 33 bits: two words per column hold
            // every R entry of the window
            const int w0 = jlo >> 5;
            const int64_t nw = in.nw;
            const uint32_t* ba = in.bits + (int64_t)colA * nw + w0;
            const uint64_t bitsA = (uint64_t)__ldg(ba) | ((int64_t)(w0 + 1) < nw ? (uint64_t)__ldg(ba + 1) << 32 : 0ull);
            uint64_t bitsB = 0;
            if (hasB) {
              const uint32_t* bbp = in.bits + (int64_t)colB * nw + w0;
              bitsB = (uint64_t)__ldg(bbp) | ((int64_t)(w0 + 1) < nw ? (uint64_t)__ldg(bbp + 1) << 32 : 0ull);
            }
            if (use_tab) {
              const int sh = jlo - (w0 << 5);
              const float* tp = tab + (W - pos + s * jlo) * 512;   // phase 2W - (pos + W - s jlo)
              const unsigned bA = (unsigned)(bitsA >> sh) & 0xFFFFu, bB = (unsigned)(bitsB >> sh) & 0xFFFFu;
              v.x = (T)(tp[bA & 255u] + tp[256 + (bA >> 8)]);
              v.y = (T)(tp[bB & 255u] + tp[256 + (bB >> 8)]);
            } else {
              for (int j = jlo; j <= jhi; ++j) {
                const T tap = __ldg(in.tapx + (pos - s * j + W));
                const int sh = j - (w0 << 5);
                v.x += ((bitsA >> sh) & 1ull) ? tap : -tap;
                v.y += ((bitsB >> sh) & 1ull) ? tap : -tap;
              }
            }
            if (!hasB) v.y = 0;
          } else {
            for (int j = jlo; j <= jhi; ++j) {
              const T tap = __ldg(in.tapx + (pos - s * j + W));
              const int jj = j & Nm;
              v.x += tap * (T)rad_bit(in.bits, in.nw, jj, colA);
              if (hasB) v.y += tap * (T)rad_bit(in.bits, in.nw, jj, colB);
            }
          }
        } else {
          const int sx = g.s[0], Nxm = (int)g.n[0] - 1;
          const int jlo = cdiv_p2(p - in.Wx, g.logs[0]), jhi = fdiv_p2(p + in.Wx, g.logs[0]);
          for (int jx = jlo; jx <= jhi; ++jx) {
            const T tap = __ldg(in.tapx + (p - sx * jx + in.Wx));
            const V u = stg[((jx & Nxm) << logC) + c];
            v.x += tap * u.x; v.y += tap * u.y;
          }
        }
      }
      sm[padix<PADC>(t)] = v;
    }
    __syncthreads();
  }
  const TB* bA = b ? b + (int64_t)colA * ldb : nullptr;
  const TB* bB = b ? b + (int64_t)colB * ldb : nullptr;
  const bool hasB = colB < ncols;
  auto pro = [&](int p) -> V {
    if (MODE == 1) return sm[padix<PADC>((p << logC) + line)];
    const int pos = (p << g.logD1) + n1;
    // unconditional loads (row 0 stands in for points outside Omega) and
    // branch-free conversions, so that all of a thread's loads are in flight
    // together; the selects then zero the points outside Omega
    const int m = kept_row(g, pos2m, pos);
    const int mc = m < 0 ? 0 : m;
    const TB a = ld1(bA + mc);
    const TB c = ld1((hasB ? bB : bA) + mc);
    V v;
    if constexpr (sizeof(T) == 4 && sizeof(TB) == 8) {
      v.x = m < 0 ? 0.f : d2f_fast(a);
      v.y = (m < 0 || !hasB) ? 0.f : d2f_fast(c);
    } else {
      v.x = m < 0 ? (T)0 : cvt<T>(a);
      v.y = (m < 0 || !hasB) ? (T)0 : cvt<T>(c);
    }
    return v;
  };
  // four-step twiddle w_L^(n1 k0) (1D), formed from per-butterfly powers
  BigTwPow<V> tw;
  const V* twA = (const V*)tb.bigA;
  const V* twB = (const V*)tb.bigB;
  if (g.dim == 1) {
    int NsL, RL;
    last_stage_shape(g.logD0, EPT<T>::LOGE, NsL, RL);
    tw.init(twA, twB, n1, NsL, RL, false);
  }
  auto epi = [&](int k0, V v, int u, int o0, int Ns) {
    if (g.dim == 1) v = cmul(v, tw.at(twA, twB, n1, u, o0, false));
    st1(X1 + (k0 << g.logD1) + n1, v);
  };
  fft_reg<V, E, false, PADC>(sm, g.logD0, true, line, tl, 1, C, twp + TW_N, pro, epi, MODE == 1);
}

template <typename T, int E2, class S>
__global__ void __launch_bounds__(REG_THREADS, REG_MINB) k_rowfold_r(Geom g_in, const typename C2<T>::t* __restrict__ X1base,
                                                   const T* __restrict__ H, int logGPB_in, typename C2<T>::t* X3base,
                                                   PassTabs tb) {
  const Geom g = fix_geom<S>(g_in);
  const int logGPB = S::fixed ? S::logC : logGPB_in;
  using V = typename C2<T>::t;
  constexpr int E = EPT<T>::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int GPB = 1 << logGPB;
  const int lognr = logGPB + g.logRg;
  V* smX = (V*)smem_raw;                                       // nrows x D1 (padded)
  V* smF = smX + padix<PADC>(g.D1 << lognr) + 16;             // GPB x N1 (padded)
  const V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  V* X3 = X3base + (int64_t)blockIdx.y * g.N;
  const int G0 = blockIdx.x * GPB;
  const V* twp = (const V*)tb.tw;
  if constexpr (S::fixed && E == 16 && E2 == 8 && S::logD1 - S::logN1 == 1 && S::logN1 == 10) {
    // 1D, s = 2, N1 = 1024: the last radix-16 stage of the forward row FFT
    // leaves thread tl with the outputs tl + 128 u (u < 16), which hold both
    // members k1 and k1 + N1 of every alias pair this thread folds, and the
    // first (radix-2) stage of the inverse N1 FFT reads exactly the folded
    // values tl + 128 q (q < 8) of the same thread: the fold runs in
    // registers, without the shared-memory round trip of the row
    constexpr int P = 128;
    const int lr = threadIdx.x >> 7, tl = threadIdx.x & (P - 1);
    const int row = G0 + lr;
    const V* xr = X1 + ((int64_t)row << g.logD1);
    V fwd[16];
    {
      auto pro = [&](int p) -> V { return ld1(xr + p); };
      auto epi = [&](int o, V v, int u, int o0, int Ns) { fwd[u] = v; };
      fft_reg<V, E, false, PADC>(smX, g.logD1, true, lr, tl, g.D1, 1, twp + TW_N, pro, epi);
    }
    const T* hr = H + ((int64_t)row << g.logD1);
    BigTwPow<V> tw;
    const V* nA = (const V*)tb.bigNA;
    const V* nB = (const V*)tb.bigNB;
    {
      int NsL, RL;
      last_stage_shape(g.logN1, 3, NsL, RL);
      tw.init(nA, nB, row, NsL, RL, true);
    }
    // inverse first stage: radix 2, 4 groups, p = tl + 128 (g + 4 u)
    auto pro = [&](int p, int gq, int u) -> V {
      const int q = gq + 4 * u;
      const T h0 = __ldg(hr + tl + P * q), h1 = __ldg(hr + tl + P * (q + 8));
      V o;
      o.x = h0 * fwd[q].x + h1 * fwd[q + 8].x;
      o.y = h0 * fwd[q].y + h1 * fwd[q + 8].y;
      return o;
    };
    auto epi = [&](int n1, V v, int u, int o0, int Ns) {
      v = cmul(v, tw.at(nA, nB, row, u, o0, true));
      st1(X3 + (row << g.logN1) + n1, v);
    };
    fft_reg<V, E2, true, PADC>(smF, g.logN1, true, lr, tl, g.N1, 1, twp + TW_N, pro, epi);
    return;
  }
  // forward FFT of the rows: P1 = D1/E threads per row
  {
    const int logP1 = g.logD1 - (E == 16 ? 4 : (E == 8 ? 3 : 2));
    const int lr = threadIdx.x >> logP1, tl = threadIdx.x & ((1 << logP1) - 1);
    const int gg = lr >> g.logRg, q = lr & (g.Rg - 1);
    const int row = G0 + gg + q * g.Rstride;
    const V* xr = X1 + ((int64_t)row << g.logD1);
    auto pro = [&](int p) -> V { return ld1(xr + p); };
    auto epi = [&](int o, V v) { smX[padix<PADC>((lr << g.logD1) + o)] = v; };
    fft_reg<V, E, false, PADC>(smX, g.logD1, true, lr, tl, g.D1, 1, twp + TW_N, pro, epi);
  }
  __syncthreads();
  // fold (prologue of the inverse FFT of length N1, P2 = N1/E2 threads per line)
  {
    constexpr int LOGE2 = E2 == 16 ? 4 : (E2 == 8 ? 3 : (E2 == 4 ? 2 : 1));
    const int logP2 = g.logN1 - LOGE2;
    const int gg = threadIdx.x >> logP2, tl = threadIdx.x & ((1 << logP2) - 1);
    const int k0 = G0 + gg;
    auto pro = [&](int k1) -> V {
      T ar = 0, ai = 0;
      for (int q = 0; q < g.Rg; ++q) {
        const int row = k0 + q * g.Rstride;
        const int lr = gg * g.Rg + q;
        const T* hr = H + ((int64_t)row << g.logD1);
        for (int p = 0; p < g.Fq; ++p) {
          const int kk = k1 + p * g.N1;
          const T hh = __ldg(hr + kk);
          const V xv = smX[padix<PADC>((lr << g.logD1) + kk)];
          ar += hh * xv.x; ai += hh * xv.y;
        }
      }
      V o; o.x = ar; o.y = ai;
      return o;
    };
    // four-step twiddle conj(w_N^(n1 k0)) (1D), formed from per-butterfly powers
    BigTwPow<V> tw;
    const V* nA = (const V*)tb.bigNA;
    const V* nB = (const V*)tb.bigNB;
    if (g.dim == 1) {
      int NsL, RL;
      last_stage_shape(g.logN1, LOGE2, NsL, RL);
      tw.init(nA, nB, k0, NsL, RL, true);
    }
    auto epi = [&](int n1, V v, int u, int o0, int Ns) {
      if (g.dim == 1) v = cmul(v, tw.at(nA, nB, k0, u, o0, true));
      st1(X3 + (k0 << g.logN1) + n1, v);
    };
    fft_reg<V, E2, true, PADC>(smF, g.logN1, true, gg, tl, g.N1, 1, twp + TW_N, pro, epi);
  }
}

template <typename T, typename TO, bool WMODE, class S>
__global__ void __launch_bounds__(S::THR, S::MINB) k_colinv_r(Geom g_in, const typename C2<T>::t* __restrict__ X3base, int pair0,
                                                  int ncols, int logC_in, TO* __restrict__ out, int64_t ldo,
                                                  const uint32_t* __restrict__ bits, int64_t nw, PassTabs tb) {
  const Geom g = fix_geom<S>(g_in);
  const int logC = S::fixed ? S::logC : logC_in;
  using V = typename C2<T>::t;
  constexpr int E = EPT<T>::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = (V*)smem_raw;
  const int C = 1 << logC;
  const int line = threadIdx.x & (C - 1), tl = threadIdx.x >> logC;
  const int c0 = blockIdx.x * C;
  const int n1 = c0 + line;
  const V* X3 = X3base + (int64_t)blockIdx.y * g.N;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  const bool hasB = colB < ncols;
  TO* oA = out + (int64_t)colA * ldo;
  TO* oB = out + (int64_t)colB * ldo;
  const T sc = (T)(1.0 / (double)g.N);
  auto pro = [&](int k0) -> V { return ld1(X3 + (k0 << g.logN1) + n1); };
  auto epi = [&](int n0, V v) {
    const int j = (n0 << g.logN1) + n1;
    T za = v.x * sc, zb = v.y * sc;
    if (WMODE) {
      za = (T)rad_bit(bits, nw, j, colA) - za;
      if (hasB) zb = (T)rad_bit(bits, nw, j, colB) - zb;
    }
    oA[j] = (TO)za;
    if (hasB) oB[j] = (TO)zb;
  };
  fft_reg<V, E, true, PADC>(sm, g.logG0, true, line, tl, 1, C, (const V*)tb.tw + TW_N, pro, epi);
}

// Column count per CTA for the register passes: C * (n / E) threads <= 512.
template <typename T> static int reg_cols(int n, int ncols) {
  const int P = n / EPT<T>::E;
  int C = std::max(1, REG_THREADS / P);
  C = std::min(C, 16);
  int p = 1;
  while (p * 2 <= C) p *= 2;
  return std::min(p, ncols);
}
template <typename T> static bool reg_ok(const Geom& g) {
  const int E = EPT<T>::E;
  const int E2 = E / (g.Rg * g.Fq);
  return g.D0 >= E && g.D1 >= E && g.G0 >= E && E2 >= 2 && g.N1 >= E2 && (g.D1 / E) * g.Rg <= REG_THREADS &&
         (g.D0 / E) <= REG_THREADS && (g.G0 / E) <= REG_THREADS;
}

template <typename T>
az_status launch_colfwd_stencil(const Geom& g, const SketchIn<T>& in, int pair0, int npairs,
                                typename C2<T>::t* X1, const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  if (!reg_ok<T>(g)) return launch_colfwd_stencil_v1<T>(g, in, pair0, npairs, X1, tb, st);
  const bool fx = sizeof(T) == 4 && is_shape_21_1(g);
  const int C = fx ? 1 << AZ_COL_LC : reg_cols<T>(g.D0, g.D1);
  const int threads = C * (g.D0 / EPT<T>::E);
  // after the FFT buffer: the 2D staging, or the 1D FP32 sign-sum tables (s x 512 floats)
  const size_t extra = g.dim == 2 ? (size_t)g.n[0] * C * sizeof(V) : (sizeof(T) == 4 ? (size_t)g.s[0] * 512 * 4 : 0);
  size_t sm = ((size_t)padix_host(g.D0 * C, PADC) + 32) * sizeof(V) + extra;
  auto kern = k_colfwd_r<T, 1, double, ShapeRT>;
  if (fx) kern = k_colfwd_r<T, 1, double, Shape1D<21, 1, AZ_COL_LC>>;
  if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D1 / C, npairs);
  ProfScope ps(sizeof(T) == 4 ? "colfwd_sketch_f32" : "colfwd_sketch_f64", (double)npairs * g.L * sizeof(V) + npairs * 2.0 * g.N / 8 + 4.0 * g.L, st);
  kern<<<grid, threads, sm, st>>>(g, in.pos2m, nullptr, 0, 0, in, pair0, ilog2i(C), X1, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
template <typename T, typename TB>
az_status launch_colfwd_gather(const Geom& g, const int32_t* pos2m, const TB* b, int64_t ldb, int ncols,
                               int pair0, int npairs, typename C2<T>::t* X1, const PassTabs& tb,
                               cudaStream_t st, int64_t M_rows) {
  using V = typename C2<T>::t;
  if (!reg_ok<T>(g)) return launch_colfwd_gather_v1<T, TB>(g, pos2m, b, ldb, ncols, pair0, npairs, X1, tb, st, M_rows);
  const bool fx = sizeof(T) == 4 && is_shape_21_1(g);
  const int C = fx ? 1 << AZ_COL_LC : reg_cols<T>(g.D0, g.D1);
  const int threads = C * (g.D0 / EPT<T>::E);
  size_t sm = ((size_t)padix_host(g.D0 * C, PADC) + 32) * sizeof(V);
  auto kern = k_colfwd_r<T, 0, TB, ShapeRT>;
  if (fx) kern = k_colfwd_r<T, 0, TB, Shape1D<21, 1, AZ_COL_LC>>;
  if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D1 / C, npairs);
  SketchIn<T> none{};
  ProfScope ps(sizeof(T) == 4 ? "colfwd_gather_f32" : "colfwd_gather_f64", (double)npairs * g.L * sizeof(V) + (double)std::min(ncols - 2 * pair0, 2 * npairs) * M_rows * sizeof(TB) + 4.0 * g.L, st);
  kern<<<grid, threads, sm, st>>>(g, pos2m, b, ldb, ncols, none, pair0, ilog2i(C), X1, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
template <typename T>
az_status launch_rowfold(const Geom& g, const typename C2<T>::t* X1, const T* H, int npairs,
                         typename C2<T>::t* X3, const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  if (!reg_ok<T>(g)) return launch_rowfold_v1<T>(g, X1, H, npairs, X3, tb, st);
  constexpr int E = EPT<T>::E;
  const int P1 = g.D1 / E;
  // groups per CTA: threads = GPB * Rg * P1 <= 512
  int GPB = 1;
  while (GPB * 2 * g.Rg * P1 <= REG_THREADS && g.G0 % (GPB * 2) == 0 && GPB * 2 <= 8) GPB *= 2;
  const int threads = GPB * g.Rg * P1;
  size_t sm = ((size_t)padix_host(g.D1 * GPB * g.Rg, PADC) + 16 + padix_host(g.N1 * GPB, PADC) + 16) * sizeof(V);
  const int E2 = E / (g.Rg * g.Fq);
  dim3 grid(g.G0 / GPB, npairs);
  ProfScope ps(sizeof(T) == 4 ? "rowfold_f32" : "rowfold_f64", (double)npairs * (g.L + g.N) * sizeof(V) + (double)g.L * sizeof(T), st);
  if (E2 == 8) {
    auto kern = k_rowfold_r<T, 8, ShapeRT>;
    if (sizeof(T) == 4 && is_shape_21_1(g) && GPB == 2) kern = k_rowfold_r<T, 8, Shape1D<21, 1, 1>>;
    if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
    kern<<<grid, threads, sm, st>>>(g, X1, H, ilog2i(GPB), X3, tb);
  } else if (E2 == 4) {
    auto kern = k_rowfold_r<T, 4, ShapeRT>;
    if (sizeof(T) == 4 && is_shape_21_1(g) && GPB == 2) kern = k_rowfold_r<T, 4, Shape1D<21, 1, 1>>;
    if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
    kern<<<grid, threads, sm, st>>>(g, X1, H, ilog2i(GPB), X3, tb);
  } else if (E2 == 2) {
    auto kern = k_rowfold_r<T, 2, ShapeRT>;
    if (sizeof(T) == 4 && is_shape_21_1(g) && GPB == 2) kern = k_rowfold_r<T, 2, Shape1D<21, 1, 1>>;
    if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
    kern<<<grid, threads, sm, st>>>(g, X1, H, ilog2i(GPB), X3, tb);
  } else {
    auto kern = k_rowfold_r<T, 16, ShapeRT>;
    if (sizeof(T) == 4 && is_shape_21_1(g) && GPB == 2) kern = k_rowfold_r<T, 16, Shape1D<21, 1, 1>>;
    if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
    kern<<<grid, threads, sm, st>>>(g, X1, H, ilog2i(GPB), X3, tb);
  }
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
template <typename T, typename TO>
az_status launch_colinv(const Geom& g, const typename C2<T>::t* X3, int pair0, int npairs, int ncols,
                        TO* out, int64_t ldo, const uint32_t* bits, int64_t nw, const PassTabs& tb,
                        cudaStream_t st) {
  using V = typename C2<T>::t;
  if (!reg_ok<T>(g)) return launch_colinv_v1<T, TO>(g, X3, pair0, npairs, ncols, out, ldo, bits, nw, tb, st);
  const bool fx = sizeof(T) == 4 && is_shape_21_1(g);
  const int C = fx ? 1 << AZ_COL_LC : reg_cols<T>(g.G0, g.N1);
  const int threads = C * (g.G0 / EPT<T>::E);
  size_t sm = ((size_t)padix_host(g.G0 * C, PADC) + 32) * sizeof(V);
  dim3 grid(g.N1 / C, npairs);
  ProfScope ps(sizeof(T) == 4 ? "colinv_f32" : "colinv_f64", (double)npairs * g.N * sizeof(V) + (double)std::min(ncols - 2 * pair0, 2 * npairs) * g.N * sizeof(TO), st);
  if (bits) {
    auto kern = k_colinv_r<T, TO, true, ShapeRT>;
    if (fx) kern = k_colinv_r<T, TO, true, Shape1D<21, 1, AZ_COL_LC>>;
    if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
    kern<<<grid, threads, sm, st>>>(g, X3, pair0, ncols, ilog2i(C), out, ldo, bits, nw, tb);
  } else {
    auto kern = k_colinv_r<T, TO, false, ShapeRT>;
    if (fx) kern = k_colinv_r<T, TO, false, Shape1D<21, 1, AZ_COL_LC>>;
    if (set_smem(kern, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
    kern<<<grid, threads, sm, st>>>(g, X3, pair0, ncols, ilog2i(C), out, ldo, bits, nw, tb);
  }
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

#define INST_R(T)                                                                                           \
  template az_status launch_colfwd_stencil<T>(const Geom&, const SketchIn<T>&, int, int, C2<T>::t*,          \
                                              const PassTabs&, cudaStream_t);                               \
  template az_status launch_rowfold<T>(const Geom&, const C2<T>::t*, const T*, int, C2<T>::t*,              \
                                       const PassTabs&, cudaStream_t);                                      \
  template az_status launch_colfwd_gather<T, double>(const Geom&, const int32_t*, const double*, int64_t,    \
                                                     int, int, int, C2<T>::t*, const PassTabs&,             \
                                                     cudaStream_t, int64_t);                                \
  template az_status launch_colfwd_gather<T, float>(const Geom&, const int32_t*, const float*, int64_t, int, \
                                                    int, int, C2<T>::t*, const PassTabs&, cudaStream_t,     \
                                                    int64_t);                                               \
  template az_status launch_colinv<T, float>(const Geom&, const C2<T>::t*, int, int, int, float*, int64_t,  \
                                             const uint32_t*, int64_t, const PassTabs&, cudaStream_t);      \
  template az_status launch_colinv<T, double>(const Geom&, const C2<T>::t*, int, int, int, double*,         \
                                              int64_t, const uint32_t*, int64_t, const PassTabs&,           \
                                              cudaStream_t);
INST_R(float)
INST_R(double)

// ------------------------------------------------------------------ explicit instantiations

#define INST_ST(T, TZ, TB, TO)                                                                              \
  template az_status launch_stencil_rows<T, TZ, TB, TO>(const Geom&, int, double, const int32_t*, int64_t,  \
                                                        const StencilTaps&, const TZ*, int64_t, const TB*,  \
                                                        int64_t, T, T, TO*, int64_t, int, cudaStream_t);     \
  template az_status launch_boundary_rows<T, TZ, TB, TO>(const Geom&, double, double, const double*,        \
                                                         const double*,                                     \
                                                         int64_t, const TZ*, int64_t, const TB*, int64_t, T, \
                                                         T, TO*, int64_t, int, cudaStream_t);
INST_ST(float, float, double, float)
INST_ST(float, float, float, float)
INST_ST(double, double, double, double)
INST_ST(double, double, double, float)
INST_ST(double, float, double, float)
INST_ST(double, double, float, float)
INST_ST(float, float, double, double)
INST_ST(float, double, double, float)

}  // namespace az
