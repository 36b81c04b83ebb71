// Kernels of the AZ hot path: index map (S1), symbol (S2), Rademacher bits
// (S3), the three FFT passes of the sketch / solve (S4, S5, S8, S10), the
// local A-apply stencils (S4, S8, S11) and boundary rows (Sec. 6.2).
#include <cmath>
#include <algorithm>
#include "kernels.cuh"

namespace az {

static constexpr int TW_N = 4096;  // master twiddle table length

// ------------------------------------------------------------------ utilities
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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
  k_count<<<nb, 256, 0, st>>>(mask, L, scratch);
  k_scan_blocks<<<1, 32, 0, st>>>(scratch, nb, M_dev);
  k_scatter<<<nb, 256, 0, st>>>(mask, L, scratch, pos2m, idx);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ S2: samples, taps
__global__ void k_samples(double* g, int64_t L, double hL, double eps, int deriv, int pimg) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double mm = (double)(m > L / 2 ? m - L : m);
  double e2 = eps * eps, acc = 0.0;
  for (int p = -pimg; p <= pimg; ++p) {
    double r = (mm + (double)p * (double)L) * hL;
    double ex = exp(-e2 * r * r);
    acc += deriv == 0 ? ex : -2.0 * e2 * ex * (1.0 - 2.0 * e2 * r * r);
  }
  g[m] = acc;
}
az_status launch_samples(double* g, int64_t L, double hL, double eps, int deriv, int pimg, cudaStream_t st) {
  k_samples<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(g, L, hL, eps, deriv, pimg);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_taps(const double* g, int64_t L, int W, double* t64, float* t32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > 2 * W) return;
  int64_t m = fmod_pos((int64_t)i - W, L);
  t64[i] = g[m];
  t32[i] = (float)g[m];
}
az_status launch_taps(const double* g, int64_t L, int W, double* t64, float* t32, cudaStream_t st) {
  k_taps<<<(2 * W + 1 + 127) / 128, 128, 0, st>>>(g, L, W, t64, t32);
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
  k_bits_to_R<<<grid, 256, 0, st>>>(bits, N, k, R);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ FFT pass helpers
template <typename V>
__device__ __forceinline__ V big_tw(const V* __restrict__ A, const V* __restrict__ B, int64_t m, bool inv) {
  V w = cmul(__ldg(A + (m >> 12)), __ldg(B + (m & 4095)));
  if (inv) w.y = -w.y;
  return w;
}

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
__device__ void colfwd_finish(const Geom& g, typename C2<T>::t* s0, typename C2<T>::t* s1, int C, int c0,
                              typename C2<T>::t* __restrict__ X1, const PassTabs& tb) {
  using V = typename C2<T>::t;
  __syncthreads();
  int cur = fft_lines<V, false>(s0, s1, g.logD0, C, 1, C, (const V*)tb.tw, TW_N >> g.logD0);
  V* res = cur ? s1 : s0;
  const int64_t total = (int64_t)g.D0 * C;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    int c = (int)(t % C), k0 = (int)(t / C);
    int n1 = c0 + c;
    V v = res[t];
    if (g.dim == 1 && k0 != 0 && n1 != 0) v = cmul(v, big_tw<V>((const V*)tb.bigA, (const V*)tb.bigB, (int64_t)n1 * k0, false));
    X1[(int64_t)k0 * g.D1 + n1] = v;
  }
}

// Sketch prologue: v = mask * (A^c R) at the tile's grid points, two Rademacher
// columns packed as (real, imag).
template <typename T>
__global__ void k_colfwd_stencil(Geom g, SketchIn<T> in, int pair0, int C, typename C2<T>::t* X1base,
                                 PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)g.D0 * C;
  const int c0 = blockIdx.x * C;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  const bool hasB = colB < in.k;
  V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  if (g.dim == 1) {
    const int s = g.s[0];
    const int64_t N = g.N;
    const int64_t total = (int64_t)g.D0 * C;
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      int c = (int)(t % C), n0 = (int)(t / C);
      int64_t pos = (int64_t)n0 * g.D1 + c0 + c;
      T re = 0, im = 0;
      if (__ldg(in.pos2m + pos) >= 0) {
        int64_t jlo = fdiv(pos - in.Wx + s - 1, s), jhi = fdiv(pos + in.Wx, s);
        for (int64_t j = jlo; j <= jhi; ++j) {
          T tap = __ldg(in.tapx + (pos - s * j + in.Wx));
          int64_t jj = fmod_pos(j, N);
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
    const int64_t Nx = g.n[0], Ny = g.n[1];
    const int64_t tot1 = Nx * C;
    for (int64_t t = threadIdx.x; t < tot1; t += blockDim.x) {
      int c = (int)(t % C);
      int64_t jx = t / C;
      int64_t iy = c0 + c;
      int64_t jlo = fdiv(iy - in.Wy + sy - 1, sy), jhi = fdiv(iy + in.Wy, sy);
      T re = 0, im = 0;
      for (int64_t jy = jlo; jy <= jhi; ++jy) {
        T tap = __ldg(in.tapy + (iy - sy * jy + in.Wy));
        int64_t j = jx * Ny + fmod_pos(jy, Ny);
        re += tap * (T)rad_bit(in.bits, in.nw, j, colA);
        if (hasB) im += tap * (T)rad_bit(in.bits, in.nw, j, colB);
      }
      V v; v.x = re; v.y = im;
      s1[t] = v;
    }
    __syncthreads();
    const int64_t tot0 = (int64_t)g.D0 * C;
    for (int64_t t = threadIdx.x; t < tot0; t += blockDim.x) {
      int c = (int)(t % C);
      int64_t ix = t / C;
      int64_t pos = ix * g.D1 + c0 + c;
      V v; v.x = 0; v.y = 0;
      if (__ldg(in.pos2m + pos) >= 0) {
        int64_t jlo = fdiv(ix - in.Wx + sx - 1, sx), jhi = fdiv(ix + in.Wx, sx);
        for (int64_t jx = jlo; jx <= jhi; ++jx) {
          T tap = __ldg(in.tapx + (ix - sx * jx + in.Wx));
          V u = s1[fmod_pos(jx, Nx) * C + c];
          v.x += tap * u.x; v.y += tap * u.y;
        }
      }
      s0[t] = v;
    }
    __syncthreads();  // s1 is reused by the FFT
  }
  colfwd_finish<T>(g, s0, s1, C, c0, X1, tb);
}

template <typename T, typename TB>
__global__ void k_colfwd_gather(Geom g, const int32_t* __restrict__ pos2m, const TB* __restrict__ b, int64_t ldb,
                                int ncols, int pair0, int C, typename C2<T>::t* X1base, PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)g.D0 * C;
  const int c0 = blockIdx.x * C;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  const int64_t total = (int64_t)g.D0 * C;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    int c = (int)(t % C), n0 = (int)(t / C);
    int64_t pos = (int64_t)n0 * g.D1 + c0 + c;
    int m = __ldg(pos2m + pos);
    V v; v.x = 0; v.y = 0;
    if (m >= 0) {
      v.x = (T)b[(int64_t)colA * ldb + m];
      if (colB < ncols) v.y = (T)b[(int64_t)colB * ldb + m];
    }
    s0[t] = v;
  }
  colfwd_finish<T>(g, s0, s1, C, c0, X1, tb);
}

template <typename T>
__global__ void k_colfwd_load(Geom g, const typename C2<T>::t* __restrict__ inbase, int C,
                              typename C2<T>::t* X1base, PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)g.D0 * C;
  const int c0 = blockIdx.x * C;
  const V* in = inbase + (int64_t)blockIdx.y * g.L;
  V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  const int64_t total = (int64_t)g.D0 * C;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    int c = (int)(t % C), n0 = (int)(t / C);
    s0[t] = in[(int64_t)n0 * g.D1 + c0 + c];
  }
  colfwd_finish<T>(g, s0, s1, C, c0, X1, tb);
}

template <typename T>
az_status launch_colfwd_stencil(const Geom& g, const SketchIn<T>& in, int pair0, int npairs,
                                typename C2<T>::t* X1, const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  int C = col_tile<V>(g.D0, g.D1);
  size_t sm = 2 * (size_t)g.D0 * C * sizeof(V);
  if (g.dim == 2 && (size_t)g.n[0] * C > (size_t)g.D0 * C) return AZ_ERR_ARG;
  if (set_smem(k_colfwd_stencil<T>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D1 / C, npairs);
  k_colfwd_stencil<T><<<grid, 256, sm, st>>>(g, in, pair0, C, X1, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
template <typename T, typename TB>
az_status launch_colfwd_gather(const Geom& g, const int32_t* pos2m, const TB* b, int64_t ldb, int ncols,
                               int pair0, int npairs, typename C2<T>::t* X1, const PassTabs& tb,
                               cudaStream_t st) {
  using V = typename C2<T>::t;
  int C = col_tile<V>(g.D0, g.D1);
  size_t sm = 2 * (size_t)g.D0 * C * sizeof(V);
  if (set_smem(k_colfwd_gather<T, TB>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D1 / C, npairs);
  k_colfwd_gather<T, TB><<<grid, 256, sm, st>>>(g, pos2m, b, ldb, ncols, pair0, C, X1, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
template <typename T>
az_status launch_colfwd_load(const Geom& g, const typename C2<T>::t* in, int npairs,
                             typename C2<T>::t* X1, const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  int C = col_tile<V>(g.D0, g.D1);
  size_t sm = 2 * (size_t)g.D0 * C * sizeof(V);
  if (set_smem(k_colfwd_load<T>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D1 / C, npairs);
  k_colfwd_load<T><<<grid, 256, sm, st>>>(g, in, C, X1, tb);
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

template <typename T>
__global__ void k_rowfft(Geom g, const typename C2<T>::t* __restrict__ X1base, int GPB,
                         typename C2<T>::t* X2base, PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)GPB * g.D1;
  const V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  V* X2 = X2base + (int64_t)blockIdx.y * g.L;
  const int r0 = blockIdx.x * GPB;
  const int64_t total = (int64_t)GPB * g.D1;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) s0[t] = X1[(int64_t)r0 * g.D1 + t];
  __syncthreads();
  int cur = fft_lines<V, false>(s0, s1, g.logD1, GPB, g.D1, 1, (const V*)tb.tw, TW_N >> g.logD1);
  V* res = cur ? s1 : s0;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) X2[(int64_t)r0 * g.D1 + t] = res[t];
}
template <typename T>
az_status launch_rowfft(const Geom& g, const typename C2<T>::t* X1, int npairs, typename C2<T>::t* X2,
                        const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  if (g.dim != 1) return AZ_ERR_ARG;
  int GPB = 1;
  while (GPB * 2 * 2 * (size_t)g.D1 * sizeof(V) <= 65536 && GPB * 2 <= 8 && g.D0 % (GPB * 2) == 0) GPB *= 2;
  size_t sm = 2 * (size_t)GPB * g.D1 * sizeof(V);
  if (set_smem(k_rowfft<T>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.D0 / GPB, npairs);
  k_rowfft<T><<<grid, 256, sm, st>>>(g, X1, GPB, X2, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// Row pass of the sketch / solve: forward FFT of each group's rows, fold of the
// alias group with H = Ghat/S (Eq. B_pinv), inverse FFT of length N1, twiddle
// (1D four-step), store on the N-grid layout X3[pair][G*N1 + n1].
template <typename T>
__global__ void k_rowfold(Geom g, const typename C2<T>::t* __restrict__ X1base, const T* __restrict__ H, int GPB,
                          typename C2<T>::t* X3base, PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrows = GPB * g.Rg;
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)nrows * g.D1;
  const V* X1 = X1base + (int64_t)blockIdx.y * g.L;
  V* X3 = X3base + (int64_t)blockIdx.y * g.N;
  const int G0 = blockIdx.x * GPB;
  // load rows: local row lr = gg*Rg + q  <->  global row (G0+gg) + q*Rstride
  const int64_t total = (int64_t)nrows * g.D1;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    int lr = (int)(t / g.D1), i = (int)(t % g.D1);
    int gg = lr / g.Rg, q = lr % g.Rg;
    int64_t row = (int64_t)(G0 + gg) + (int64_t)q * g.Rstride;
    s0[t] = X1[row * g.D1 + i];
  }
  __syncthreads();
  int cur = fft_lines<V, false>(s0, s1, g.logD1, nrows, g.D1, 1, (const V*)tb.tw, TW_N >> g.logD1);
  V* X = cur ? s1 : s0;
  V* F = cur ? s0 : s1;  // fold output lines [gg][N1]
  const int64_t totF = (int64_t)GPB * g.N1;
  for (int64_t t = threadIdx.x; t < totF; t += blockDim.x) {
    int gg = (int)(t / g.N1), k1 = (int)(t % g.N1);
    T ar = 0, ai = 0;
    for (int q = 0; q < g.Rg; ++q) {
      int64_t row = (int64_t)(G0 + gg) + (int64_t)q * g.Rstride;
      const V* xr = X + (int64_t)(gg * g.Rg + q) * g.D1;
      for (int p = 0; p < g.Fq; ++p) {
        int kk = k1 + p * g.N1;
        T hh = __ldg(H + row * g.D1 + kk);
        V xv = xr[kk];
        ar += hh * xv.x; ai += hh * xv.y;
      }
    }
    V o; o.x = ar; o.y = ai;
    F[t] = o;
  }
  __syncthreads();
  V* Fo = F;
  V* Fs = X;
  int c2 = fft_lines<V, true>(Fo, Fs, g.logN1, GPB, g.N1, 1, (const V*)tb.tw, TW_N >> g.logN1);
  V* Z = c2 ? Fs : Fo;
  for (int64_t t = threadIdx.x; t < totF; t += blockDim.x) {
    int gg = (int)(t / g.N1), n1 = (int)(t % g.N1);
    int k0 = G0 + gg;
    V v = Z[t];
    if (g.dim == 1 && k0 != 0 && n1 != 0) v = cmul(v, big_tw<V>((const V*)tb.bigNA, (const V*)tb.bigNB, (int64_t)n1 * k0, true));
    X3[(int64_t)k0 * g.N1 + n1] = v;
  }
}
template <typename T>
az_status launch_rowfold(const Geom& g, const typename C2<T>::t* X1, const T* H, int npairs,
                         typename C2<T>::t* X3, const PassTabs& tb, cudaStream_t st) {
  using V = typename C2<T>::t;
  int GPB = row_groups_per_cta<V>(g);
  size_t sm = 2 * (size_t)GPB * g.Rg * g.D1 * sizeof(V);
  if (set_smem(k_rowfold<T>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.G0 / GPB, npairs);
  k_rowfold<T><<<grid, 256, sm, st>>>(g, X1, H, GPB, X3, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ inverse column pass
template <typename T, typename TO>
__global__ void k_colinv(Geom g, const typename C2<T>::t* __restrict__ X3base, int pair0, int ncols, int C,
                         TO* __restrict__ out, int64_t ldo, const uint32_t* __restrict__ bits, int64_t nw,
                         PassTabs tb) {
  using V = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* s0 = (V*)smem_raw;
  V* s1 = s0 + (size_t)g.G0 * C;
  const int c0 = blockIdx.x * C;
  const V* X3 = X3base + (int64_t)blockIdx.y * g.N;
  const int pair = pair0 + blockIdx.y;
  const int colA = 2 * pair, colB = 2 * pair + 1;
  const int64_t total = (int64_t)g.G0 * C;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    int c = (int)(t % C), k0 = (int)(t / C);
    s0[t] = X3[(int64_t)k0 * g.N1 + c0 + c];
  }
  __syncthreads();
  int cur = fft_lines<V, true>(s0, s1, g.logG0, C, 1, C, (const V*)tb.tw, TW_N >> g.logG0);
  V* res = cur ? s1 : s0;
  const T sc = (T)(1.0 / (double)g.N);
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    int c = (int)(t % C), n0 = (int)(t / C);
    int64_t j = (int64_t)n0 * g.N1 + c0 + c;
    V v = res[t];
    T za = v.x * sc, zb = v.y * sc;
    if (bits) {
      za = (T)rad_bit(bits, nw, j, colA) - za;
      if (colB < ncols) zb = (T)rad_bit(bits, nw, j, colB) - zb;
    }
    out[(int64_t)colA * ldo + j] = (TO)za;
    if (colB < ncols) out[(int64_t)colB * ldo + j] = (TO)zb;
  }
}
template <typename T, typename TO>
az_status launch_colinv(const Geom& g, const typename C2<T>::t* X3, int pair0, int npairs, int ncols,
                        TO* out, int64_t ldo, const uint32_t* bits, int64_t nw, const PassTabs& tb,
                        cudaStream_t st) {
  using V = typename C2<T>::t;
  int C = col_tile<V>(g.G0, g.N1);
  size_t sm = 2 * (size_t)g.G0 * C * sizeof(V);
  if (set_smem(k_colinv<T, TO>, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
  dim3 grid(g.N1 / C, npairs);
  k_colinv<T, TO><<<grid, 256, sm, st>>>(g, X3, pair0, ncols, C, out, ldo, bits, nw, tb);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ stencils
template <typename T, typename TZ>
__device__ __forceinline__ T stencil_1d(const Geom& g, const T* __restrict__ tp, int W, int64_t i,
                                        const TZ* __restrict__ z) {
  const int s = g.s[0];
  int64_t jlo = fdiv(i - W + s - 1, s), jhi = fdiv(i + W, s);
  T acc = 0;
  for (int64_t j = jlo; j <= jhi; ++j) acc += __ldg(tp + (i - s * j + W)) * (T)z[fmod_pos(j, g.N)];
  return acc;
}

template <typename T, typename TZ, typename TB, typename TO>
__global__ void k_stencil_rows(Geom g, int kind, T inv2e2, const int32_t* __restrict__ idx, int64_t M,
                               const T* __restrict__ x0, const T* __restrict__ x2, const T* __restrict__ y0,
                               const T* __restrict__ y2, int Wx, int Wy, const TZ* __restrict__ zb, int64_t ldz,
                               const TB* __restrict__ bb, int64_t ldb, T alpha, T beta, TO* __restrict__ outb,
                               int64_t ldo) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int c = blockIdx.y;
  const TZ* z = zb + (int64_t)c * ldz;
  const int64_t i = idx[m];
  T az;
  if (g.dim == 1) {
    az = stencil_1d<T, TZ>(g, x0, Wx, i, z);
  } else {
    const int sx = g.s[0], sy = g.s[1];
    const int64_t Nx = g.n[0], Ny = g.n[1];
    const int64_t ix = i / g.D1, iy = i % g.D1;
    int64_t xlo = fdiv(ix - Wx + sx - 1, sx), xhi = fdiv(ix + Wx, sx);
    int64_t ylo = fdiv(iy - Wy + sy - 1, sy), yhi = fdiv(iy + Wy, sy);
    T acc = 0;
    for (int64_t jx = xlo; jx <= xhi; ++jx) {
      const TZ* zr = z + fmod_pos(jx, Nx) * Ny;
      T a0 = 0, a2 = 0;
      for (int64_t jy = ylo; jy <= yhi; ++jy) {
        T zv = (T)zr[fmod_pos(jy, Ny)];
        a0 += __ldg(y0 + (iy - sy * jy + Wy)) * zv;
        if (kind == 1) a2 += __ldg(y2 + (iy - sy * jy + Wy)) * zv;
      }
      T tx0 = __ldg(x0 + (ix - sx * jx + Wx));
      if (kind == 1) acc += __ldg(x2 + (ix - sx * jx + Wx)) * a0 + tx0 * a2;
      else acc += tx0 * a0;
    }
    az = kind == 1 ? -acc * inv2e2 : acc;
  }
  T r = beta * az;
  if (bb) r += alpha * (T)bb[(int64_t)c * ldb + m];
  outb[(int64_t)c * ldo + m] = (TO)r;
}
template <typename T, typename TZ, typename TB, typename TO>
az_status launch_stencil_rows(const Geom& g, int kind, double eps, const int32_t* idx, int64_t M,
                              const StencilTaps& tp, const TZ* z, int64_t ldz, const TB* b, int64_t ldb,
                              T alpha, T beta, TO* out, int64_t ldo, int ncols, cudaStream_t st) {
  if (M == 0 || ncols == 0) return AZ_OK;
  dim3 grid((unsigned)((M + 255) / 256), ncols);
  k_stencil_rows<T, TZ, TB, TO><<<grid, 256, 0, st>>>(g, kind, (T)(1.0 / (2.0 * eps * eps)), idx, M, (const T*)tp.x0,
                                                      (const T*)tp.x2, (const T*)tp.y0, (const T*)tp.y2, tp.Wx,
                                                      tp.Wy, z, ldz, b, ldb, alpha, beta, out, ldo);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// phi_per at distance d (center window handles the images): plain Gaussian here
template <typename T> __device__ __forceinline__ T gauss(T d, T eps) { T e = eps * d; return exp(-e * e); }

template <typename T, typename TZ, typename TB, typename TO>
__global__ void k_boundary_rows(Geom g, T eps, T w, int Wc, const double* __restrict__ pts, int64_t Mb,
                                const TZ* __restrict__ zb, int64_t ldz, const TB* __restrict__ bb, int64_t ldb,
                                T alpha, T beta, TO* __restrict__ outb, int64_t ldo) {
  int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Mb) return;
  const int c = blockIdx.y;
  const TZ* z = zb + (int64_t)c * ldz;
  const double px = pts[2 * m], py = pts[2 * m + 1];
  const double hx = 2.0 * g.T[0] / g.n[0], hy = 2.0 * g.T[1] / g.n[1];
  const int64_t cxi = (int64_t)floor((px + g.T[0]) / hx), cyi = (int64_t)floor((py + g.T[1]) / hy);
  T acc = 0;
  for (int64_t jx = cxi - Wc; jx <= cxi + Wc + 1; ++jx) {
    T wx = gauss<T>((T)(px - (-g.T[0] + (double)jx * hx)), eps);
    const TZ* zr = z + fmod_pos(jx, g.n[0]) * g.n[1];
    T a = 0;
    for (int64_t jy = cyi - Wc; jy <= cyi + Wc + 1; ++jy) {
      T wy = gauss<T>((T)(py - (-g.T[1] + (double)jy * hy)), eps);
      a += wy * (T)zr[fmod_pos(jy, g.n[1])];
    }
    acc += wx * a;
  }
  T r = beta * w * acc;
  if (bb) r += alpha * (T)bb[(int64_t)c * ldb + m];
  outb[(int64_t)c * ldo + m] = (TO)r;
}
static int center_window(const Geom& g, double eps) {
  double h = 2.0 * g.T[0] / (double)g.n[0];
  int Wc = (int)std::ceil(std::sqrt(42.0) / (eps * h)) + 1;
  int lim = (int)std::min<int64_t>(g.n[0], g.n[1]) / 2 - 1;
  return std::max(0, std::min(Wc, lim));
}
template <typename T, typename TZ, typename TB, typename TO>
az_status launch_boundary_rows(const Geom& g, double eps, double w, const double* pts, int64_t Mb,
                               const TZ* z, int64_t ldz, const TB* b, int64_t ldb, T alpha, T beta,
                               TO* out, int64_t ldo, int ncols, cudaStream_t st) {
  if (Mb == 0 || ncols == 0) return AZ_OK;
  dim3 grid((unsigned)((Mb + 127) / 128), ncols);
  k_boundary_rows<T, TZ, TB, TO><<<grid, 128, 0, st>>>(g, (T)eps, (T)w, center_window(g, eps), pts, Mb, z, ldz, b,
                                                       ldb, alpha, beta, out, ldo);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// Evaluation on the s_test-refined box grid (FP64)
__global__ void k_evaluate(Geom g, double eps, int st_, int Wc, const double* __restrict__ xb, int64_t ldx,
                           double* __restrict__ outb, int64_t ldo, int64_t npts) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npts) return;
  const int c = blockIdx.y;
  const double* x = xb + (int64_t)c * ldx;
  double acc = 0;
  if (g.dim == 1) {
    const int64_t Lt = g.n[0] * st_;
    const double h = 2.0 * g.T[0] / g.n[0];
    const double px = -g.T[0] + (double)q * (2.0 * g.T[0] / (double)Lt);
    const int64_t ci = (int64_t)floor((px + g.T[0]) / h);
    for (int64_t j = ci - Wc; j <= ci + Wc + 1; ++j) acc += gauss<double>(px - (-g.T[0] + (double)j * h), eps) * x[fmod_pos(j, g.n[0])];
  } else {
    const int64_t Lty = g.n[1] * st_;
    const int64_t ix = q / Lty, iy = q % Lty;
    const double hx = 2.0 * g.T[0] / g.n[0], hy = 2.0 * g.T[1] / g.n[1];
    const double px = -g.T[0] + (double)ix * hx / st_, py = -g.T[1] + (double)iy * hy / st_;
    const int64_t cxi = (int64_t)floor((px + g.T[0]) / hx), cyi = (int64_t)floor((py + g.T[1]) / hy);
    for (int64_t jx = cxi - Wc; jx <= cxi + Wc + 1; ++jx) {
      double wx = gauss<double>(px - (-g.T[0] + (double)jx * hx), eps);
      const double* zr = x + fmod_pos(jx, g.n[0]) * g.n[1];
      double a = 0;
      for (int64_t jy = cyi - Wc; jy <= cyi + Wc + 1; ++jy) a += gauss<double>(py - (-g.T[1] + (double)jy * hy), eps) * zr[fmod_pos(jy, g.n[1])];
      acc += wx * a;
    }
  }
  outb[(int64_t)c * ldo + q] = acc;
}
az_status launch_evaluate(const Geom& g, double eps, int s_test, const double* x, int64_t ldx, int nrhs,
                          double* out, int64_t ldo, cudaStream_t st) {
  int64_t npts = g.dim == 1 ? g.n[0] * s_test : g.n[0] * s_test * g.n[1] * s_test;
  int Wc;
  {
    double h = 2.0 * g.T[0] / (double)g.n[0];
    Wc = (int)std::ceil(std::sqrt(42.0) / (eps * h)) + 1;
    int64_t lim = (g.dim == 1 ? g.n[0] : std::min(g.n[0], g.n[1])) / 2 - 1;
    Wc = (int)std::max<int64_t>(0, std::min<int64_t>(Wc, lim));
  }
  dim3 grid((unsigned)((npts + 255) / 256), nrhs);
  k_evaluate<<<grid, 256, 0, st>>>(g, eps, s_test, Wc, x, ldx, out, ldo, npts);
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
  k_H<<<(unsigned)((g.L + 255) / 256), 256, 0, st>>>(g, Ghat, S, S + g.N, thr, H64, H32);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_max_abs(const double* v, int64_t n, double* out) {
  __shared__ double sm[32];
  double m = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sm[w]);
    *out = r;
  }
}
az_status launch_max_abs(const double* v, int64_t n, double* out, cudaStream_t st) {
  k_max_abs<<<1, 1024, 0, st>>>(v, n, out);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}
__global__ void k_spec_to_natural(Geom g, const double2* X, double* out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.L) return;
  int64_t k0 = t / g.D1, k1 = t % g.D1;
  out[k0 + (int64_t)g.D0 * k1] = X[t].x;
}
az_status launch_spec_to_natural(const Geom& g, const double2* X, double* out, cudaStream_t st) {
  k_spec_to_natural<<<(unsigned)((g.L + 255) / 256), 256, 0, st>>>(g, X, out);
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
  int cur = fft_lines<double2, false>(s0, s1, logn, 1, n, 1, tw, TW_N >> logn);
  double2* r = cur ? s1 : s0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = r[i].x;
}
az_status launch_line_dft_real(const double* in, int n, double* out, const double2* tw, cudaStream_t st) {
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  size_t sm = 2 * (size_t)n * sizeof(double2);
  if (set_smem(k_line_dft_real, sm) != cudaSuccess) { set_error("smem attribute"); return AZ_ERR_CUDA; }
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
  k_sumsq_cols<<<ncols, 1024, 0, st>>>(v, ld, rows, out);
  AZ_LAUNCH_CHECK();
  return AZ_OK;
}

// ------------------------------------------------------------------ explicit instantiations
#define INST_T(T)                                                                                           \
  template az_status launch_colfwd_stencil<T>(const Geom&, const SketchIn<T>&, int, int, C2<T>::t*,          \
                                              const PassTabs&, cudaStream_t);                               \
  template az_status launch_colfwd_load<T>(const Geom&, const C2<T>::t*, int, C2<T>::t*, const PassTabs&,    \
                                           cudaStream_t);                                                   \
  template az_status launch_rowfft<T>(const Geom&, const C2<T>::t*, int, C2<T>::t*, const PassTabs&,        \
                                      cudaStream_t);                                                        \
  template az_status launch_rowfold<T>(const Geom&, const C2<T>::t*, const T*, int, C2<T>::t*,              \
                                       const PassTabs&, cudaStream_t);                                      \
  template az_status launch_colfwd_gather<T, double>(const Geom&, const int32_t*, const double*, int64_t,    \
                                                     int, int, int, C2<T>::t*, const PassTabs&,             \
                                                     cudaStream_t);                                         \
  template az_status launch_colfwd_gather<T, float>(const Geom&, const int32_t*, const float*, int64_t, int, \
                                                    int, int, C2<T>::t*, const PassTabs&, cudaStream_t);    \
  template az_status launch_colinv<T, float>(const Geom&, const C2<T>::t*, int, int, int, float*, int64_t,  \
                                             const uint32_t*, int64_t, const PassTabs&, cudaStream_t);      \
  template az_status launch_colinv<T, double>(const Geom&, const C2<T>::t*, int, int, int, double*,         \
                                              int64_t, const uint32_t*, int64_t, const PassTabs&,           \
                                              cudaStream_t);
INST_T(float)
INST_T(double)

#define INST_ST(T, TZ, TB, TO)                                                                              \
  template az_status launch_stencil_rows<T, TZ, TB, TO>(const Geom&, int, double, const int32_t*, int64_t,  \
                                                        const StencilTaps&, const TZ*, int64_t, const TB*,  \
                                                        int64_t, T, T, TO*, int64_t, int, cudaStream_t);     \
  template az_status launch_boundary_rows<T, TZ, TB, TO>(const Geom&, double, double, const double*,        \
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
