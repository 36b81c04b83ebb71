// C ABI of the AZ solver (include/az.h): handle lifecycle and the host-side
// orchestration of the kernels, all stream-ordered.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "cluster_sketch.cuh"
#include "dfgemm.cuh"
#include "kernels.cuh"
#include "lowrank.cuh"
#include "lowrank_large.cuh"
#include "tc_tsgram.cuh"
#include "profile.cuh"

namespace az {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace az

using namespace az;

// Sketch widths up to this use the one-CTA factorisation and register-blocked
// tall products; wider sketches use the Householder QR + GEMM path.
static constexpr int kNarrowK = 64;
static constexpr double kGramTau = 1e-8;   // smallest sigma / sigma_1 the FP64 Gram route resolves

struct az_setup_t {
  Geom g{};
  int kind = 0, precision = AZ_MIXED, k = 0, refine = 1;
  double eps = 0, tau_svd = 1e-8, tau_sym = 0, bweight = 1.0, floor = 0;
  double k0 = 0;            // Helmholtz wavenumber of the collocation operator (0 = Poisson)
  uint64_t seed = 0;
  int64_t M = 0, Mb = 0, Mtot = 0;
  int64_t ldm = 0;        // leading dimension of Ut and gb: Mtot rounded up to 32 (16-byte TMA strides)
  std::vector<void*> allocs;
  size_t bytes = 0;
  int32_t* pos2m = nullptr;
  int32_t* idx = nullptr;
  double* bpts = nullptr;
  double* bnrm = nullptr;   // Mb x dim outward normals (null: all Dirichlet)
  double* Ghat = nullptr;
  double* S = nullptr;
  double* H64 = nullptr;
  float* H32 = nullptr;
  double* taps64[4] = {nullptr, nullptr, nullptr, nullptr};  // x0, y0, x2, y2
  float* taps32[4] = {nullptr, nullptr, nullptr, nullptr};
  float* tapsH[4] = {nullptr, nullptr, nullptr, nullptr};   // FP64 taps split into FP32 hi + lo
  float* tapsL[4] = {nullptr, nullptr, nullptr, nullptr};
  int W32[2] = {0, 0}, W64[2] = {0, 0};
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  double2* big64[4] = {nullptr, nullptr, nullptr, nullptr};  // A_L, B_L, A_N, B_N
  float2* big32[4] = {nullptr, nullptr, nullptr, nullptr};
  uint32_t* bits = nullptr;
  int64_t nw = 0;
  void* W = nullptr;    // N x k   (T)
  void* Y = nullptr;    // Mtot x k (T)
  void* Ut = nullptr;   // Mtot x k (T, ld ldm), zero beyond rank
  // 2D mixed precision: the sketch, its factorisation, W and Ut are FP64 (an
  // FP32 sketch misplaces the fitted subspace by ~1e-4 sigma_1 in 2D), while
  // the solve's transforms, stencils and projection run in FP32 on Ut32 and
  // the update x = z + W u reads the FP64 W
  bool sk64 = false;
  float* Ut32 = nullptr; // Mtot x k (FP32 copy of Ut, ld ldm)
  bool prod64 = false;   // FP64-accurate tall products in FP64 arithmetic (eps h < 0.66), else double-float
  // 2D FP64 Z* chains (sketch, FP64 solves) as one cluster-resident kernel
  // where the grid allows it (square, L = 64..256, s = 2) and it is enabled
  bool use_cluster = false;
  float* xsh = nullptr;  // 2D mixed: x split into FP32 hi + lo for the residual (N x 2 pairs_max each)
  float* xsl = nullptr;
  double *G = nullptr, *V = nullptr, *lam = nullptr, *B1 = nullptr, *Tm = nullptr, *VS = nullptr, *sig = nullptr;
  double* partial = nullptr;
  FactorInfo* info = nullptr;
  // workspace (precision T)
  int pairs_max = 0;
  void* X1 = nullptr;   // pairs_max x L complex
  void* X3 = nullptr;   // pairs_max x N complex
  void* zb = nullptr;   // N x 2 pairs_max (T)
  void* gb = nullptr;   // Mtot x 2 pairs_max (T, ld ldm)
  void* rb = nullptr;   // Mtot x 2 pairs_max (T) residual
  float* xfb = nullptr; // N x 2 pairs_max: the mixed path's first-pass solution (exactly FP32)
  double* cb = nullptr; // k x 2 pairs_max
  double* ub = nullptr;
  double* normb = nullptr;  // 2 x 2 pairs_max
  // FP64 scratch for az_apply_Zstar in mixed mode
  void* X1d = nullptr;
  void* X3d = nullptr;
  // persistent setup scratch (so that az_refactor neither allocates nor syncs)
  uint8_t* mask = nullptr;
  int64_t* Md = nullptr;
  int32_t* scan = nullptr;
  double* samp[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [dim][phi, phi'']
  double* Gd[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  double* Q1 = nullptr;     // Mtot x k
  double* Rd = nullptr;     // N x k (collocation sketch)
  double* r64 = nullptr;    // Mtot x cols (relres residual), lazily
  double* bcoll = nullptr;  // Mtot x 2 pairs_max (scaled collocation data of az_collocate)
  LargeK* wide = nullptr;   // k > 64: Householder QR + FP64 SVD + GEMM path
  // Omega = the whole box, no boundary rows, exact pseudo-inverse: Z* A = I,
  // so the perturbation is exactly zero (Sec. 3.1) and the sketch is skipped
  bool periodic = false;
  // leading sketch columns (of W and Y) already valid, copied from a
  // narrower setup with the same seed by the adaptive width; the next
  // sketch computes only the columns after them
  int k_done = 0;
  int* tc_err = nullptr;    // set by a tensor-core pipeline wait that timed out
  cudaEvent_t info_ev = nullptr;  // recorded after each factorisation (az_get_info waits on it)
  // az_refactor runs the sketch and factorisation (S3-S7) on fst, after the
  // index map and symbol on the caller's stream (ev_sym), so that the next
  // solve's first Z* pass overlaps it; the solve waits on ev_fac before it
  // uses the factors.  X1s/X3s: the sketch chain's own FFT workspace.
  cudaStream_t fst = nullptr;
  cudaEvent_t ev_sym = nullptr, ev_fac = nullptr;
  bool fac_pending = false;
  void* X1s = nullptr;
  void* X3s = nullptr;
  int pairs_s = 0;
};

namespace {

template <typename T> struct Prec;
template <> struct Prec<float> { static constexpr bool fp64 = false; };
template <> struct Prec<double> { static constexpr bool fp64 = true; };

az_status dalloc(az_setup_t* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    return AZ_ERR_OOM;
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  return AZ_OK;
}
template <typename P> az_status dalloc_t(az_setup_t* h, P** p, size_t count) {
  return dalloc(h, (void**)p, count * sizeof(P));
}

// per-CTA partial sums of the tall products: the SIMT Gram kernel or the
// tensor-core kernel, whichever launches more CTAs
int partial_blocks(int64_t M) {
  return std::max(gram_blocks(M), (int)std::min<int64_t>(tc_tsgram_blocks(), (M + 31) / 32));
}

std::string tc_wait_message(int code) {
  return "tensor-core tall product: pipeline wait timed out (role " + std::to_string(code) + "); results invalid";
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) { int l = 0; while ((int64_t(1) << l) < v) ++l; return l; }

// Half-width W (grid units) such that the periodised samples beyond W are below
// delta * g(0): the Gaussian exp(-(eps m h_L)^2) decays below delta past
// m = sqrt(ln(1/delta)) / (eps h_L); for phi'' the polynomial factor is covered by
// two extra points.
// A width that reaches half the period stops at W = Ld/2: the window then
// covers the whole period, and the taps at m = +-Ld/2 (one grid offset seen
// from both ends) carry half the sample each.
int stencil_halfwidth(double eps, double hL, double delta, int64_t Ld, bool deriv) {
  int W = (int)std::ceil(std::sqrt(std::log(1.0 / delta)) / (eps * hL)) + (deriv ? 2 : 0);
  int64_t lim = Ld / 2;
  return (int)std::min<int64_t>(W, lim);
}

az_status make_geom(const az_grid* gr, Geom& g) {
  std::memset(&g, 0, sizeof(g));
  if (!gr || (gr->dim != 1 && gr->dim != 2)) { set_error("dim must be 1 or 2"); return AZ_ERR_ARG; }
  g.dim = gr->dim;
  for (int d = 0; d < 2; ++d) {
    bool used = d < g.dim;
    g.n[d] = used ? gr->n[d] : 1;
    g.s[d] = used ? gr->s[d] : 1;
    g.T[d] = used ? gr->T[d] : 1.0;
    if (used && (!is_pow2(g.n[d]) || !is_pow2(g.s[d]) || g.s[d] > 8 || !(g.T[d] > 0))) {
      set_error("n and s must be powers of two (s <= 8) and T > 0");
      return AZ_ERR_ARG;
    }
    g.Ld[d] = g.n[d] * g.s[d];
  }
  g.N = g.n[0] * g.n[1];
  g.L = g.Ld[0] * g.Ld[1];
  if (g.dim == 1) {
    if (g.L < 4 || g.L > (int64_t(1) << 24) || g.N < 2) { set_error("1D grid size out of range (4 <= L <= 2^24)"); return AZ_ERR_ARG; }
    int lL = ilog2(g.L);
    g.logD1 = (lL + 1) / 2;
    g.logD0 = lL - g.logD1;
    g.D1 = 1 << g.logD1;
    g.D0 = 1 << g.logD0;
    if (g.D1 < g.s[0]) { set_error("grid too small for the oversampling factor"); return AZ_ERR_ARG; }
    g.N1 = g.D1 / g.s[0];
    g.G0 = g.D0;
    g.Rg = 1; g.Rstride = 0; g.Fq = g.s[0];
  } else {
    if (g.Ld[0] > 4096 || g.Ld[1] > 4096 || g.Ld[0] < 2 || g.Ld[1] < 2) { set_error("2D grid: L per dimension must be in [2, 4096]"); return AZ_ERR_ARG; }
    g.D0 = (int)g.Ld[0]; g.D1 = (int)g.Ld[1];
    g.logD0 = ilog2(g.D0); g.logD1 = ilog2(g.D1);
    g.G0 = (int)g.n[0]; g.N1 = (int)g.n[1];
    g.Rg = g.s[0]; g.Rstride = (int)g.n[0]; g.Fq = g.s[1];
  }
  g.logN1 = ilog2(g.N1);
  g.logG0 = ilog2(g.G0);
  g.logN = ilog2(g.N);
  for (int d = 0; d < 2; ++d) { g.logs[d] = ilog2(g.s[d]); g.logn[d] = ilog2(g.n[d]); g.logLd[d] = ilog2(g.Ld[d]); }
  g.logRg = ilog2(g.Rg);
  return AZ_OK;
}


template <typename T> PassTabs tabs(az_setup_t* h) {
  PassTabs t;
  if (Prec<T>::fp64) { t.tw = h->tw64; t.bigA = h->big64[0]; t.bigB = h->big64[1]; t.bigNA = h->big64[2]; t.bigNB = h->big64[3]; }
  else { t.tw = h->tw32; t.bigA = h->big32[0]; t.bigB = h->big32[1]; t.bigNA = h->big32[2]; t.bigNB = h->big32[3]; }
  return t;
}
template <typename T> const T* Hsym(az_setup_t* h);
template <> const double* Hsym<double>(az_setup_t* h) { return h->H64; }
template <> const float* Hsym<float>(az_setup_t* h) { return h->H32; }

template <typename T> StencilTaps taps(az_setup_t* h) {
  StencilTaps t;
  if (Prec<T>::fp64) { t.x0 = h->taps64[0]; t.y0 = h->taps64[1]; t.x2 = h->taps64[2]; t.y2 = h->taps64[3]; t.Wx = h->W64[0]; t.Wy = h->W64[1]; }
  else { t.x0 = h->taps32[0]; t.y0 = h->taps32[1]; t.x2 = h->taps32[2]; t.y2 = h->taps32[3]; t.Wx = h->W32[0]; t.Wy = h->W32[1]; }
  if (h->g.dim == 1) { t.y0 = t.x0; t.y2 = t.x2; t.Wy = t.Wx; }
  return t;
}

// Tables for the four-step twiddles: w_n^m = A[m >> 12] * B[m & 4095], m < n.
az_status big_tables(az_setup_t* h, int64_t n, double2** A64, double2** B64, float2** A32, float2** B32,
                     cudaStream_t st) {
  int64_t na = std::max<int64_t>(1, (n + 4095) / 4096);
  std::vector<double2> a(na), b(4096);
  std::vector<float2> af(na), bf(4096);
  std::vector<double> re, im;
  // exact-reduced twiddles via the 4096 table builder generalised to length n
  for (int64_t q = 0; q < na; ++q) {
    // angle of w_n^(4096 q)
    int64_t m = (4096 * q) % n;
    std::vector<double> r1, i1;
    // reuse host_twiddles semantics through a tiny local computation
    double ang = 2.0 * M_PI * (double)m / (double)n;
    (void)ang;
    r1.resize(1); i1.resize(1);
    {
      // exp(-2 pi i m / n) with octant reduction
      int64_t aa = 2 * m, bb = n;
      bool ns = false, nc = false, sw = false;
      if (aa > bb) { aa = 2 * bb - aa; ns = true; }
      if (2 * aa > bb) { aa = bb - aa; nc = true; }
      if (4 * aa > bb) { aa = bb - 2 * aa; bb = 2 * bb; sw = true; }
      double x = M_PI * (double)aa / (double)bb, c = std::cos(x), s = std::sin(x);
      if (sw) std::swap(c, s);
      if (nc) c = -c;
      if (ns) s = -s;
      a[q] = make_double2(c, -s);
    }
  }
  for (int64_t r = 0; r < 4096; ++r) {
    int64_t m = r % n;
    int64_t aa = 2 * m, bb = n;
    bool ns = false, nc = false, sw = false;
    if (aa > bb) { aa = 2 * bb - aa; ns = true; }
    if (2 * aa > bb) { aa = bb - aa; nc = true; }
    if (4 * aa > bb) { aa = bb - 2 * aa; bb = 2 * bb; sw = true; }
    double x = M_PI * (double)aa / (double)bb, c = std::cos(x), s = std::sin(x);
    if (sw) std::swap(c, s);
    if (nc) c = -c;
    if (ns) s = -s;
    b[r] = make_double2(c, -s);
  }
  for (int64_t q = 0; q < na; ++q) af[q] = make_float2((float)a[q].x, (float)a[q].y);
  for (int r = 0; r < 4096; ++r) bf[r] = make_float2((float)b[r].x, (float)b[r].y);
  AZ_TRY(dalloc_t(h, A64, na)); AZ_TRY(dalloc_t(h, B64, 4096));
  AZ_TRY(dalloc_t(h, A32, na)); AZ_TRY(dalloc_t(h, B32, 4096));
  AZ_CUDA(cudaMemcpyAsync(*A64, a.data(), na * sizeof(double2), cudaMemcpyHostToDevice, st));
  AZ_CUDA(cudaMemcpyAsync(*B64, b.data(), 4096 * sizeof(double2), cudaMemcpyHostToDevice, st));
  AZ_CUDA(cudaMemcpyAsync(*A32, af.data(), na * sizeof(float2), cudaMemcpyHostToDevice, st));
  AZ_CUDA(cudaMemcpyAsync(*B32, bf.data(), 4096 * sizeof(float2), cudaMemcpyHostToDevice, st));
  // host vectors must outlive the async copies: synchronise (setup only)
  AZ_CUDA(cudaStreamSynchronize(st));
  return AZ_OK;
}

template <typename TI>
__global__ void k_to_double(const TI* in, int64_t ldi, int64_t rows, int ncols, double* out, int64_t ldo) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < rows && c < ncols) out[(int64_t)c * ldo + i] = (double)in[(int64_t)c * ldi + i];
}
template <typename TI>
az_status to_double(const TI* in, int64_t ldi, int64_t rows, int ncols, double* out, int64_t ldo, cudaStream_t st) {
  if (rows == 0 || ncols == 0) return AZ_OK;
  dim3 grid((unsigned)((rows + 255) / 256), ncols);
  k_to_double<TI><<<grid, 256, 0, st>>>(in, ldi, rows, ncols, out, ldo);
  AZ_CUDA(cudaGetLastError());
  return AZ_OK;
}

// FP64 matrix -> FP32 copy (same leading dimension)
__global__ void k_to_float(const double* in, int64_t ld, int64_t rows, int ncols, float* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < rows && c < ncols) out[(int64_t)c * ld + i] = (float)in[(int64_t)c * ld + i];
}

// x = hi + lo (FP32 pair, 48 bits), column by column
__global__ void k_split_x(const double* x, int64_t ldx, int64_t N, int ncols, float* hi, float* lo, int64_t ldo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= N || c >= ncols) return;
  float h, l;
  d2ff_int(x[(int64_t)c * ldx + i], h, l);
  hi[(int64_t)c * ldo + i] = h;
  lo[(int64_t)c * ldo + i] = l;
}

// precision of the stored sketch, W, Y and Ut (FP64 also for the 2D mixed path)
bool store64(const az_setup_t* h) { return h->precision == AZ_FP64 || h->sk64; }

// ------------------------------------------------------------------ setup pieces
// Host-side stencil widths (phi and phi'' taps of one dimension share a width).
void stencil_widths(az_setup_t* h) {
  const Geom& g = h->g;
  for (int d = 0; d < g.dim; ++d) {
    const double hL = 2.0 * g.T[d] / (double)g.Ld[d];
    const bool der = h->kind == 1;
    h->W64[d] = stencil_halfwidth(h->eps, hL, 1e-18, g.Ld[d], der);
    h->W32[d] = stencil_halfwidth(h->eps, hL, 1e-9, g.Ld[d], der);
  }
}

az_status alloc_symbol(az_setup_t* h) {
  const Geom& g = h->g;
  const int nder = h->kind == 1 ? 2 : 1;
  for (int d = 0; d < g.dim; ++d)
    for (int q = 0; q < nder; ++q) {
      if (g.dim == 2) AZ_TRY(dalloc_t(h, &h->samp[d][q], g.Ld[d]));
      if (g.dim == 2) AZ_TRY(dalloc_t(h, &h->Gd[d][q], g.Ld[d]));
      AZ_TRY(dalloc_t(h, &h->taps64[d + 2 * q], 2 * h->W64[d] + 1));
      AZ_TRY(dalloc_t(h, &h->taps32[d + 2 * q], 2 * h->W32[d] + 1));
      AZ_TRY(dalloc_t(h, &h->tapsH[d + 2 * q], 2 * h->W64[d] + 1));
      AZ_TRY(dalloc_t(h, &h->tapsL[d + 2 * q], 2 * h->W64[d] + 1));
    }
  AZ_TRY(dalloc_t(h, &h->Ghat, g.L));
  AZ_TRY(dalloc_t(h, &h->S, g.N + 1));
  AZ_TRY(dalloc_t(h, &h->H64, g.L));
  AZ_TRY(dalloc_t(h, &h->H32, g.L));
  return AZ_OK;
}

// S2: stencil taps of the periodised kernel (Eq. periodic_rbf), Ghat =
// DFT_L(g) (Lemma 4.2; 1D in its Poisson-summation form, 2D as line DFTs of
// the samples), S_k = sum over the alias group of Ghat^2 and H = Ghat / S
// (Eq. B_pinv), stored in the row-pass layout.  Launches only.
az_status build_symbol(az_setup_t* h, cudaStream_t st) {
  Geom& g = h->g;
  const double eps = h->eps;
  const int nder = h->kind == 1 ? 2 : 1;
  if (g.dim == 1) {
    // taps from the image sum; Ghat = DFT_L(g) in its Poisson-summation form
    const double hL = 2.0 * g.T[0] / (double)g.Ld[0];
    // (collocation, Example 6.1: the interior kernel -(phi'' + k0^2 phi) / (2 eps^2)
    // takes the place of phi in the taps and the symbol; boundary rows use phi)
    AZ_TRY(launch_taps_direct(g.Ld[0], hL, eps, image_count(eps, g.T[0]), h->W64[0], h->taps64[0], h->W32[0],
                              h->taps32[0], st, h->tapsH[0], h->tapsL[0], h->kind, h->k0));
    AZ_TRY(launch_symbol_closed_1d(g.L, eps * hL, h->Ghat, st, h->kind, hL, h->k0, eps));
  } else {
    for (int d = 0; d < g.dim; ++d)
      for (int q = 0; q < nder; ++q) {
        const double hL = 2.0 * g.T[d] / (double)g.Ld[d];
        AZ_TRY(launch_samples(h->samp[d][q], g.Ld[d], hL, eps, q == 0 ? 0 : 2, image_count(eps, g.T[d]), st));
        // Helmholtz (Sec. 6.2): -(phi''_x phi_y + phi_x phi''_y + k0^2 phi_x phi_y) =
        // -(phi''_x phi_y + phi_x (phi''_y + k0^2 phi_y)): the k0 term joins the y
        // second-derivative samples, and taps, symbol, stencils and residual follow
        if (d == 1 && q == 1 && h->k0 != 0.0)
          AZ_TRY(launch_axpy(g.Ld[1], h->k0 * h->k0, h->samp[1][0], h->samp[1][1], st));
        AZ_TRY(launch_taps(h->samp[d][q], g.Ld[d], h->W64[d], h->taps64[d + 2 * q], h->W32[d], h->taps32[d + 2 * q],
                           st, h->tapsH[d + 2 * q], h->tapsL[d + 2 * q]));
      }
    for (int d = 0; d < 2; ++d)
      for (int q = 0; q < nder; ++q) AZ_TRY(launch_line_dft_real(h->samp[d][q], (int)g.Ld[d], h->Gd[d][q], h->tw64, st));
    AZ_TRY(launch_symbol_full(g, h->kind, eps, h->Gd[0][0], h->Gd[1][0], h->Gd[0][1], h->Gd[1][1], h->Ghat, st));
  }
  AZ_TRY(launch_fold_S(g, h->Ghat, h->S, st));
  AZ_TRY(launch_max_abs(h->S, g.N, h->S + g.N, st));
  AZ_TRY(launch_H(g, h->Ghat, h->S, h->tau_sym * h->tau_sym, h->H64, h->H32, st));
  return AZ_OK;
}

// The chain Z* applied to pairs of columns of b (or of the sketch), T precision.
//  mode 0: b is a compact vector (TB) -> z = Z* b (N x ncols, T) in zout
//  mode 1: sketch: R columns via stencil, -> W = R - Z* A R (N x k, T)
//  mode 2: b = A R given as a compact vector -> W = R - Z* b
template <typename T, typename TB>
az_status zstar_chain(az_setup_t* h, int mode, const TB* b, int64_t ldb, int ncols, T* zout, int64_t ldz,
                      cudaStream_t st, int first_col = 0) {
  using V = typename C2<T>::t;
  const Geom& g = h->g;
  PassTabs tb = tabs<T>(h);
  const int npairs_total = (ncols + 1) / 2;
  const bool own = mode == 1 && h->X1s;   // the sketch chain on its own workspace
  const int step = own ? h->pairs_s : h->pairs_max;
  if (first_col & 1) { set_error("zstar_chain: odd first column"); return AZ_ERR_ARG; }
  if constexpr (Prec<T>::fp64 && sizeof(TB) == 8) {
    if (h->use_cluster && mode != 1) {
      // the whole chain in one cluster-resident launch per column pair
      const int p0 = first_col / 2;
      if (p0 >= npairs_total) return AZ_OK;
      return launch_zstar_cluster(g, (const double*)b, ldb, ncols, h->pos2m, h->H64, mode != 0 ? h->bits : nullptr,
                                  h->nw, (double*)zout, ldz, h->tw64, p0, npairs_total - p0, h->tc_err, st);
    }
  }
  for (int p0 = first_col / 2; p0 < npairs_total; p0 += step) {
    const int np = std::min(step, npairs_total - p0);
    V* X1 = (V*)(own ? h->X1s : h->X1);
    V* X3 = (V*)(own ? h->X3s : h->X3);
    if (mode == 1) {
      SketchIn<T> in;
      in.bits = h->bits; in.nw = h->nw; in.k = h->k; in.pos2m = h->pos2m;
      StencilTaps tp = taps<T>(h);
      in.tapx = (const T*)tp.x0; in.tapy = (const T*)tp.y0; in.Wx = tp.Wx; in.Wy = tp.Wy;
      AZ_TRY(launch_colfwd_stencil<T>(g, in, p0, np, X1, tb, st));
    } else {
      AZ_TRY((launch_colfwd_gather<T, TB>(g, h->pos2m, b, ldb, ncols, p0, np, X1, tb, st, h->M)));
    }
    AZ_TRY(launch_rowfold<T>(g, X1, Hsym<T>(h), np, X3, tb, st));
    AZ_TRY((launch_colinv<T, T>(g, X3, p0, np, ncols, zout, ldz, mode != 0 ? h->bits : nullptr, h->nw, tb, st)));
  }
  return AZ_OK;
}

// rows of A applied to coefficient columns: out = alpha*b + beta*A z over all Mtot rows
template <typename T, typename TZ, typename TB, typename TO>
az_status apply_rows(az_setup_t* h, const TZ* z, int64_t ldz, const TB* b, int64_t ldb, T alpha, T beta, TO* out,
                     int64_t ldo, int ncols, cudaStream_t st) {
  StencilTaps tp = taps<T>(h);
  AZ_TRY((launch_stencil_rows<T, TZ, TB, TO>(h->g, h->kind, h->eps, h->idx, h->M, tp, z, ldz, b, ldb, alpha, beta,
                                             out, ldo, ncols, st)));
  if (h->Mb) {
    AZ_TRY((launch_boundary_rows<T, TZ, TB, TO>(h->g, h->eps, h->bweight, h->bpts, h->bnrm, h->Mb, z, ldz,
                                                b ? b + h->M : nullptr, ldb, alpha, beta, out + h->M, ldo, ncols, st)));
  }
  return AZ_OK;
}

// S3-S7: Rademacher bits, sketch W = (I - Z* A) R and Y = A W, then the
// SVQB + Cholesky factorisation and truncated SVD.  Launches only.
template <typename T>
az_status sketch_and_factor(az_setup_t* h, cudaStream_t st) {
  const Geom& g = h->g;
  const int k = h->k;
  T* W = (T*)h->W;
  T* Y = (T*)h->Y;
  const int k0 = h->k_done < k ? h->k_done : 0;   // columns [0, k0) of W and Y are current
  h->k_done = 0;
  AZ_TRY(launch_philox_bits(h->bits, g.N, k, h->seed, st));
  if (h->periodic) {
    // rank 0: W = (I - Z* A) R = 0 and Y = 0 exactly; nothing to factorise
    AZ_CUDA(cudaMemsetAsync(W, 0, (size_t)g.N * k * sizeof(T), st));
    AZ_CUDA(cudaMemsetAsync(Y, 0, (size_t)h->Mtot * k * sizeof(T), st));
    AZ_CUDA(cudaMemsetAsync(h->Ut, 0, (size_t)h->ldm * k * sizeof(T), st));
    AZ_CUDA(cudaMemsetAsync(h->VS, 0, (size_t)k * k * sizeof(double), st));
    AZ_CUDA(cudaMemsetAsync(h->sig, 0, (size_t)k * sizeof(double), st));
    AZ_CUDA(cudaMemsetAsync(h->info, 0, sizeof(FactorInfo), st));
    return AZ_OK;
  }
  if (h->kind == 0 && !h->use_cluster) {
    // W = (I - Z* A) R through the fused FFT chain (A R by the local stencil)
    AZ_TRY((zstar_chain<T, double>(h, 1, nullptr, 0, k, W, g.N, st, k0)));
  } else {
    // Collocation (and the cluster-resident chain): v = A R on all rows by the
    // stencil rows (R materialised in FP64), then W = R - Z* v through the
    // gather chain (Z* has zero columns for the boundary rows).
    T* v = (T*)h->gb;    // Mtot x k scratch (gb holds >= k columns)
    AZ_TRY(launch_bits_to_R(h->bits, g.N, k, h->Rd, st));
    AZ_TRY((apply_rows<T, double, double, T>(h, h->Rd + (size_t)k0 * g.N, g.N, nullptr, 0, (T)0, (T)1,
                                              v + (size_t)k0 * h->ldm, h->ldm, k - k0, st)));
    AZ_TRY((zstar_chain<T, T>(h, 2, v, h->ldm, k, W, g.N, st, k0)));
  }
  // Y = A W on all rows (kept grid rows, then weighted boundary rows)
  AZ_TRY((apply_rows<T, T, double, T>(h, W + (size_t)k0 * g.N, g.N, nullptr, 0, (T)0, (T)1,
                                      Y + (size_t)k0 * h->Mtot, h->Mtot, k - k0, st)));
  if (h->wide) {
    // wide sketch: Householder QR of Y (Q into the Q1 scratch), SVD of R
    return large_factor(h->wide, Y, h->Mtot, h->Q1, h->Ut, h->ldm, h->tau_svd, h->floor, h->VS, h->sig, h->info, st);
  }
  // pass 1: G1 = Y^T Y, SVQB; an FP32 sketch takes the exact tensor-core
  // Gram (BF16 slices, FP64 fold) where its shape allows, else double-float
  if (!Prec<T>::fp64 && tc_gram_oz_ok(Y, h->Mtot, k, h->Mtot)) {
    AZ_TRY(launch_tc_gram_oz((const float*)Y, h->Mtot, k, h->Mtot, h->partial, h->G, h->tc_err, st));
  } else {
    AZ_TRY((launch_gram<T, T>(Y, h->Mtot, k, Y, h->Mtot, k, h->Mtot, h->partial, h->G, st)));
  }
  const double taug = Prec<T>::fp64 ? kGramTau : 1e-7;
  AZ_TRY(launch_factor1(h->G, k, taug, h->floor * h->floor, h->V, h->lam, h->B1, h->info, st));
  // pass 2: Q1 = Y B1, G2 = Q1^T Q1, Cholesky, SVD of the small factor, Ut = Q1 T
  if (Prec<T>::fp64) {
    AZ_TRY((launch_tsprod<T, double>(Y, h->Mtot, k, h->B1, k, h->Mtot, h->Q1, h->Mtot, st)));
    AZ_TRY((launch_gram<double, double>(h->Q1, h->Mtot, k, h->Q1, h->Mtot, k, h->Mtot, h->partial, h->G, st)));
    AZ_TRY(launch_factor2(h->G, k, h->V, h->lam, h->tau_svd, h->floor, h->Tm, h->VS, h->sig, h->info, st));
    AZ_TRY((launch_tsprod<double, T>(h->Q1, h->Mtot, k, h->Tm, k, h->Mtot, (T*)h->Ut, h->ldm, st)));
  } else {
    // mixed: Q1 = Y B1 needs extended precision (its small directions cancel
    // by up to sigma_1 / sigma_r1), computed in double-float and rounded to
    // FP32; Q1 is then well conditioned, so G2 and Ut = Q1 T run in FP32.
    // (FP32 Q1 in the FP64 Q1 buffer, leading dimension ldm: 16-byte rows for TMA)
    float* Q1f = (float*)h->Q1;
    AZ_TRY(launch_tsprod_df<float>((const float*)Y, h->Mtot, k, h->B1, k, h->Mtot, Q1f, h->ldm, st));
    if (tc_tsgram_ok(Q1f, h->ldm, k, Q1f, h->ldm, k)) {
      AZ_TRY(launch_tc_tsgram(Q1f, h->ldm, k, Q1f, h->ldm, k, h->Mtot, h->partial, h->G, h->tc_err, st));
    } else {
      AZ_TRY((launch_gram<float, float>(Q1f, h->ldm, k, Q1f, h->ldm, k, h->Mtot, h->partial, h->G, st, true)));
    }
    AZ_TRY(launch_factor2(h->G, k, h->V, h->lam, h->tau_svd, h->floor, h->Tm, h->VS, h->sig, h->info, st, true));
    AZ_TRY((launch_tsprod<float, float>(Q1f, h->ldm, k, h->Tm, k, h->Mtot, (float*)h->Ut, h->ldm, st)));
  }
  return AZ_OK;
}

// S3-S7 in the storage precision; the 2D mixed path then rounds Ut to FP32
// for the solve's projection.
az_status sketch_factor_any(az_setup_t* h, cudaStream_t st) {
  if (!store64(h)) return sketch_and_factor<float>(h, st);
  AZ_TRY(sketch_and_factor<double>(h, st));
  if (h->sk64) {
    dim3 grid((unsigned)((h->ldm + 255) / 256), h->k);
    k_to_float<<<grid, 256, 0, st>>>((const double*)h->Ut, h->ldm, h->ldm, h->k, h->Ut32);
    AZ_CUDA(cudaGetLastError());
  }
  return AZ_OK;
}

az_status compute_setup(az_setup_t* h, cudaStream_t st, bool with_index_map) {
  if (with_index_map) AZ_TRY(launch_compact(h->mask, h->g.L, h->pos2m, h->idx, h->Md, h->scan, st));
  AZ_TRY(build_symbol(h, st));
  AZ_TRY(sketch_factor_any(h, st));
  if (h->info_ev) AZ_CUDA(cudaEventRecord(h->info_ev, st));
  return AZ_OK;
}

// One AZ solve of ncols columns (T precision): x (=|+=) Z* b + W VS U^T (b - A Z* b).
// Mixed path: xf_out receives the (exactly FP32) result, x may then be null;
// xbase (FP32, ld N) makes the update x = xbase + (...).
// last: the solve's final pass (its projection error is not refined away):
// the wide path then projects with exact products instead of split TF32.
template <typename T, typename TB>
az_status az_once(az_setup_t* h, const TB* b, int64_t ldb, int ncols, double* x, int64_t ldx, bool accumulate,
                  cudaStream_t st, float* xf_out = nullptr, const float* xbase = nullptr, bool last = true) {
  const Geom& g = h->g;
  T* z = (T*)h->zb;
  T* gg = (T*)h->gb;
  AZ_TRY((zstar_chain<T, TB>(h, 0, b, ldb, ncols, z, g.N, st)));
  if (h->periodic) {
    // rank 0: x = Z* b (the update with no low-rank columns)
    return launch_update_x<T, T>((const T*)h->W, g.N, 0, h->ub, z, g.N, g.N, ncols, x, ldx, accumulate, st,
                                 Prec<T>::fp64 ? nullptr : xf_out, Prec<T>::fp64 ? nullptr : xbase);
  }
  AZ_TRY((apply_rows<T, T, TB, T>(h, z, g.N, b, ldb, (T)1, (T)-1, gg, h->ldm, ncols, st)));
  if (h->fac_pending) {
    // the factors of an az_refactor still running on the setup's own stream
    AZ_CUDA(cudaStreamWaitEvent(st, h->ev_fac, 0));
    h->fac_pending = false;
  }
  // the FP32 projection basis: Ut itself, or the FP32 copy of the FP64 Ut
  const T* Ub = h->sk64 ? (const T*)h->Ut32 : (const T*)h->Ut;
  const bool w64 = h->sk64 || Prec<T>::fp64;
  if (h->wide) {
    AZ_TRY(large_project(h->wide, Ub, h->ldm, gg, h->ldm, ncols, h->cb, st, !Prec<T>::fp64,
                         last ? nullptr : h->tc_err));
    AZ_TRY(launch_small_mm(h->VS, h->k, h->cb, ncols, h->ub, st));
    AZ_TRY(large_update(h->wide, h->W, g.N, h->ub, z, g.N, g.N, ncols, x, ldx, accumulate, st, w64,
                        !Prec<T>::fp64));
    return AZ_OK;
  }
  if (!Prec<T>::fp64 && tc_tsgram_ok(Ub, h->ldm, h->k, gg, h->ldm, ncols)) {
    // c = U_tau^T g on the tensor cores (split TF32, FP32-level accuracy)
    AZ_TRY(launch_tc_tsgram((const float*)Ub, h->ldm, h->k, (const float*)gg, h->ldm, ncols, h->Mtot, h->partial,
                            h->cb, h->tc_err, st));
  } else {
    AZ_TRY((launch_gram<T, T>(Ub, h->ldm, h->k, gg, h->ldm, ncols, h->Mtot, h->partial, h->cb, st, true)));
  }
  AZ_TRY(launch_small_mm(h->VS, h->k, h->cb, ncols, h->ub, st));
  if (h->sk64 && !Prec<T>::fp64) {
    // x = z + W u with the FP64 W (the sketch's own precision), FP32 z, in
    // double-float (FP64 arithmetic where eps h < 0.66)
    return launch_df_update<double, float>((const double*)h->W, g.N, h->k, h->ub, ncols, (const float*)z, g.N, g.N,
                                           x, ldx, accumulate, st, nullptr, h->prod64);
  }
  AZ_TRY((launch_update_x<T, T>((const T*)h->W, g.N, h->k, h->ub, z, g.N, g.N, ncols, x, ldx, accumulate, st,
                                Prec<T>::fp64 ? nullptr : xf_out, Prec<T>::fp64 ? nullptr : xbase)));
  return AZ_OK;
}

template <typename T>
az_status solve_impl(az_setup_t* h, const double* b, int64_t ldb, int64_t nrhs, double* x, int64_t ldx,
                     cudaStream_t st, double* relres) {
  const int chunk = 2 * h->pairs_max;
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int nc = (int)std::min<int64_t>(chunk, nrhs - c0);
    const double* bc = b + c0 * ldb;
    double* xc = x + c0 * ldx;
    // mixed path with refinement and no boundary rows: the first pass keeps
    // its result only as the exact FP32 copy, and the second forms
    // x = x1 + dx directly (one FP64 write of x instead of a write, a read
    // and a write)
    // (the 2D mixed path updates x with the FP64 W: x is not FP32 after the
    // first pass, and its residual is the plain FP64 one below)
    const bool mixed = !Prec<T>::fp64 && !h->sk64;
    // (the wide path leaves the FP32 first-pass result in the z buffer instead)
    const bool defer = mixed && h->refine > 0 && h->Mb == 0 && !h->wide;
    AZ_TRY((az_once<T, double>(h, bc, ldb, nc, defer ? nullptr : xc, ldx, false, st,
                               mixed && h->refine > 0 && !h->wide ? h->xfb : nullptr, nullptr, h->refine == 0)));
    const float* x1f = h->wide ? (const float*)h->zb : h->xfb;
    for (int it = 0; it < h->refine; ++it) {
      T* res = (T*)h->rb;
      if (mixed && it == 0) {
        // r = b - A x, FP64-accurate: x is exactly FP32 after the first pass, so
        // double-FP32 arithmetic on the split FP64 taps reproduces the FP64
        // residual (about 48 significant bits) at FP32 throughput
        const float* th[4] = {h->tapsH[0], h->tapsH[1], h->tapsH[2], h->tapsH[3]};
        const float* tl[4] = {h->tapsL[0], h->tapsL[1], h->tapsL[2], h->tapsL[3]};
        AZ_TRY(launch_resid_df(h->g, h->kind, h->eps, h->idx, h->M, th, tl, h->W64[0], h->W64[1], x1f,
                               h->g.N, bc, ldb, (float*)res, h->Mtot, nc, st));
        if (h->Mb) {
          AZ_TRY((launch_boundary_rows<double, double, double, T>(h->g, h->eps, h->bweight, h->bpts, h->bnrm, h->Mb, xc, ldx,
                                                                  bc + h->M, ldb, 1.0, -1.0, res + h->M, h->Mtot, nc, st)));
        }
      } else if (h->sk64 && it == 0) {
        // 2D mixed: x = x_hi + x_lo (FP32 pair); r = b - A x_hi to about 48
        // bits on the FP32 pipe (as above), then - A x_lo in FP32 (x_lo is
        // 2^-24 of x, so its FP32 product is FP64-accurate in the sum)
        dim3 sg((unsigned)((h->g.N + 255) / 256), nc);
        k_split_x<<<sg, 256, 0, st>>>(xc, ldx, h->g.N, nc, h->xsh, h->xsl, h->g.N);
        AZ_CUDA(cudaGetLastError());
        const float* th[4] = {h->tapsH[0], h->tapsH[1], h->tapsH[2], h->tapsH[3]};
        const float* tl[4] = {h->tapsL[0], h->tapsL[1], h->tapsL[2], h->tapsL[3]};
        float* rhi = (float*)h->gb;   // b - A x_hi (the g workspace is free between passes)
        AZ_TRY(launch_resid_df(h->g, h->kind, h->eps, h->idx, h->M, th, tl, h->W64[0], h->W64[1], h->xsh, h->g.N, bc,
                               ldb, rhi, h->ldm, nc, st));
        StencilTaps tp = taps<float>(h);
        AZ_TRY((launch_stencil_rows<float, float, float, float>(h->g, h->kind, h->eps, h->idx, h->M, tp, h->xsl, h->g.N,
                                                                rhi, h->ldm, 1.0f, -1.0f, (float*)res, h->Mtot, nc,
                                                                st)));
        if (h->Mb) {
          AZ_TRY((launch_boundary_rows<double, double, double, T>(h->g, h->eps, h->bweight, h->bpts, h->bnrm, h->Mb, xc, ldx,
                                                                  bc + h->M, ldb, 1.0, -1.0, res + h->M, h->Mtot, nc, st)));
        }
      } else {
        // r = b - A x with the residual computed in FP64
        AZ_TRY((apply_rows<double, double, double, T>(h, xc, ldx, bc, ldb, 1.0, -1.0, res, h->Mtot, nc, st)));
      }
      const bool last = it + 1 == h->refine;
      if (defer && it == 0) AZ_TRY((az_once<T, T>(h, res, h->Mtot, nc, xc, ldx, false, st, nullptr, h->xfb, last)));
      else AZ_TRY((az_once<T, T>(h, res, h->Mtot, nc, xc, ldx, true, st, nullptr, nullptr, last)));
    }
    if (relres) {
      if (!h->r64) {
        cudaError_t e0 = cudaMalloc((void**)&h->r64, (size_t)h->Mtot * chunk * sizeof(double));
        if (e0 != cudaSuccess) { cudaGetLastError(); h->r64 = nullptr; set_error("relres buffer"); return AZ_ERR_OOM; }
      }
      double* r64 = h->r64;
      az_status rc = apply_rows<double, double, double, double>(h, xc, ldx, bc, ldb, 1.0, -1.0, r64, h->Mtot, nc, st);
      if (rc == AZ_OK) rc = launch_sumsq_cols(r64, h->Mtot, h->Mtot, nc, h->normb, st);
      if (rc == AZ_OK) rc = launch_sumsq_cols(bc, ldb, h->Mtot, nc, h->normb + nc, st);
      std::vector<double> hv(2 * nc);
      int tcerr = 0;
      cudaError_t e = cudaMemcpyAsync(hv.data(), h->normb, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, st);
      cudaError_t e1 = cudaMemcpyAsync(&tcerr, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st);
      cudaError_t e2 = cudaStreamSynchronize(st);
      if (rc) return rc;
      if (e != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess) { set_error("relres readback failed"); return AZ_ERR_CUDA; }
      if (tcerr) {
        // reported once: the flag is cleared so that later calls start clean
        cudaMemsetAsync(h->tc_err, 0, sizeof(int), st);
        set_error(tc_wait_message(tcerr));
        return AZ_ERR_TIMEOUT;
      }
      for (int c = 0; c < nc; ++c) relres[c0 + c] = hv[nc + c] > 0 ? std::sqrt(hv[c] / hv[nc + c]) : 0.0;
    }
  }
  return AZ_OK;
}

az_status alloc_workspace(az_setup_t* h) {
  const Geom& g = h->g;
  // (sized for the storage precision: the 2D mixed path runs its sketch chain
  // in FP64 on the same workspace as its FP32 solves)
  const size_t vsz = store64(h) ? 16 : 8, tsz = vsz / 2;
  const size_t per_pair = (size_t)(g.L + g.N) * vsz;
  int pm = std::max(32, (h->k + 1) / 2);
  while (pm > 1 && per_pair * pm > (size_t)3 << 30) pm /= 2;
  h->pairs_max = pm;
  const int cols = std::max(2 * pm, h->k);
  AZ_TRY(dalloc(h, &h->X1, per_pair * pm / (g.L + g.N) * g.L));
  AZ_TRY(dalloc(h, &h->X3, per_pair * pm / (g.L + g.N) * g.N));
  AZ_TRY(dalloc(h, &h->zb, (size_t)g.N * cols * tsz));
  AZ_TRY(dalloc(h, &h->gb, (size_t)h->ldm * cols * tsz));
  AZ_TRY(dalloc(h, &h->rb, (size_t)h->Mtot * cols * tsz));
  if (h->precision == AZ_MIXED && !h->sk64) AZ_TRY(dalloc_t(h, &h->xfb, (size_t)g.N * cols));
  if (h->sk64) {
    AZ_TRY(dalloc_t(h, &h->xsh, (size_t)g.N * cols));
    AZ_TRY(dalloc_t(h, &h->xsl, (size_t)g.N * cols));
  }
  AZ_TRY(dalloc_t(h, &h->cb, (size_t)h->k * cols));
  AZ_TRY(dalloc_t(h, &h->ub, (size_t)h->k * cols));
  AZ_TRY(dalloc_t(h, &h->normb, (size_t)2 * cols));
  return AZ_OK;
}

void destroy(az_setup_t* h) {
  if (!h) return;
  if (h->fst) cudaStreamSynchronize(h->fst);
  for (void* p : h->allocs) cudaFree(p);
  if (h->X1d) cudaFree(h->X1d);
  if (h->X3d) cudaFree(h->X3d);
  if (h->r64) cudaFree(h->r64);
  if (h->wide) large_destroy(h->wide);
  if (h->info_ev) cudaEventDestroy(h->info_ev);
  if (h->ev_sym) cudaEventDestroy(h->ev_sym);
  if (h->ev_fac) cudaEventDestroy(h->ev_fac);
  if (h->fst) cudaStreamDestroy(h->fst);
  delete h;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* az_last_error(void) { return g_last_error.c_str(); }

void az_destroy(az_handle h) { destroy(h); }

az_status az_rademacher(int64_t N, int32_t k, uint64_t seed, double* R_dev, void* stream) {
  if (N <= 0 || k <= 0 || !R_dev) { set_error("az_rademacher: bad arguments"); return AZ_ERR_ARG; }
  if (k > 65535) { set_error("az_rademacher: k exceeds 65535 columns"); return AZ_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* bits;
  int64_t nw = (N + 31) / 32;
  AZ_CUDA(cudaMalloc((void**)&bits, (size_t)nw * k * 4 + 16));
  az_status rc = launch_philox_bits(bits, N, k, seed, st);
  if (rc == AZ_OK) rc = launch_bits_to_R(bits, N, k, R_dev, st);
  cudaStreamSynchronize(st);
  cudaFree(bits);
  return rc;
}

az_status az_debug_tc_withhold(int32_t iteration, int64_t wait_ns) {
  if (iteration < 0 || wait_ns <= 0) { set_error("az_debug_tc_withhold: bad arguments"); return AZ_ERR_ARG; }
  tc_tsgram_debug_withhold(iteration, (uint64_t)wait_ns);
  return AZ_OK;
}

__global__ void k_debug_f32_sum(const float* __restrict__ a, const float* __restrict__ b, double* __restrict__ out,
                                int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = f32_sum_f64(a[i], b[i]);
}

az_status az_debug_f32_sum_f64(const float* a, const float* b, double* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!a || !b || !out))) { set_error("az_debug_f32_sum_f64: bad arguments"); return AZ_ERR_ARG; }
  if (n == 0) return AZ_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  k_debug_f32_sum<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a, b, out, n);
  AZ_CUDA(cudaGetLastError());
  return AZ_OK;
}

az_status az_debug_gram(const float* Y, int64_t ldy, int32_t k, int64_t M, double* G, int32_t route, void* stream) {
  if (!Y || !G || k < 1 || k > 64 || M < 1 || ldy < M || (route != 0 && route != 1)) {
    set_error("az_debug_gram: bad arguments");
    return AZ_ERR_ARG;
  }
  if (route == 1 && !tc_gram_oz_ok(Y, ldy, k, M)) {
    set_error("az_debug_gram: the tensor-core route needs k <= 24, ldy a multiple of 4 and 16-byte aligned Y");
    return AZ_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nb = (size_t)std::max(gram_blocks(M), tc_gram_oz_blocks(M));
  double* partial = nullptr;
  int* err = nullptr;
  AZ_CUDA(cudaMalloc((void**)&partial, nb * k * k * sizeof(double)));
  az_status rc = AZ_OK;
  if (cudaMalloc((void**)&err, sizeof(int)) != cudaSuccess || cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) {
    set_error("az_debug_gram: scratch");
    rc = AZ_ERR_CUDA;
  }
  if (rc == AZ_OK) {
    rc = route == 1 ? launch_tc_gram_oz(Y, ldy, k, M, partial, G, err, st)
                    : launch_gram<float, float>(Y, ldy, k, Y, ldy, k, M, partial, G, st);
  }
  int e = 0;
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = AZ_ERR_CUDA;
  if (err && cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && e != 0 && rc == AZ_OK) {
    set_error(tc_wait_message(e));
    rc = AZ_ERR_TIMEOUT;
  }
  cudaFree(partial);
  if (err) cudaFree(err);
  return rc;
}

az_status az_query_footprint(const az_grid* gr, int64_t M, int64_t n_boundary, const az_options* opt, int64_t nrhs_max,
                             size_t* bytes) {
  if (!bytes) { set_error("az_query_footprint: null output"); return AZ_ERR_ARG; }
  Geom g;
  AZ_TRY(make_geom(gr, g));
  const int prec = opt ? opt->precision : AZ_MIXED;
  const int k = opt ? opt->k : 24;
  // (2D mixed setups store the sketch and factors in FP64 and add an FP32 Ut)
  const bool s64 = prec == AZ_FP64 || g.dim == 2;
  const size_t vsz = s64 ? 16 : 8, tsz = vsz / 2;
  const int64_t Mt = M + n_boundary;
  int pm = (int)std::max<int64_t>(std::max<int64_t>(1, (nrhs_max + 1) / 2), (k + 1) / 2);
  size_t b = 0;
  b += (size_t)g.L * (4 + 8 + 8 + 4);              // pos2m, Ghat, H64, H32
  b += (size_t)M * 4 + (size_t)g.N * 8;             // idx, S
  b += (size_t)((g.N + 31) / 32) * 4 * k;           // bits
  const int64_t ldm = (Mt + 31) / 32 * 32;
  b += (size_t)g.N * k * tsz + (size_t)(Mt + ldm) * k * tsz;  // W, Y, Ut
  if (prec == AZ_MIXED && g.dim == 2) b += (size_t)ldm * k * 4;  // Ut FP32 copy
  b += (size_t)pm * (g.L + g.N) * vsz;              // X1, X3
  const int cols = std::max(2 * pm, k);
  b += (size_t)g.N * cols * tsz + (size_t)(Mt + ldm) * cols * tsz;
  if (k <= 64) b += (size_t)partial_blocks(Mt) * k * std::max(k, cols) * 8;
  else b += (size_t)k * k * 8 * 5 + (size_t)Mt * k * 4 + (32u << 20);   // small FP64 factors, QR workspace, cuBLAS workspace
  b += (size_t)Mt * k * 8;                          // transient Q1 during setup
  if (n_boundary == 0 && k <= 64 && M < g.L)        // the sketch chain's own X1, X3 (approximation)
    b += (size_t)std::min<int64_t>(pm, (k + 1) / 2) * (g.L + g.N) * vsz;
  *bytes = b;
  return AZ_OK;
}

static az_status setup_fixed(const az_grid* gr, const uint8_t* mask, const double* bpts, int64_t n_boundary,
                             double eps, int32_t kernel, double boundary_weight, const az_options* opt, void* stream,
                             az_handle* out, const az_setup_t* reuse = nullptr);

// The mixed path inverts the symbol in FP32.  Within one alias group of the
// Gaussian symbol (Eq. periodic_rbf, Poisson summation) the largest member
// lies at most half a coarse period from the origin, where Ghat has fallen
// by exp(-(pi / (2 eps h))^2) from its peak; Z* scales FP32 rounding by that
// range.  The sketch stays usable while the amplified rounding,
// 2^-24 exp((pi / (2 eps h))^2), is below 1e-3, i.e. eps h >= 0.504 (the
// eps h = 1 regime of the large workloads passes; the tau0 = 1e-10 regime of
// Eq. constant_shapeparam, eps h = 0.33, does not and needs AZ_FP64).
// The wide path's double-float (48-bit) tall products see the same
// amplification: FP64 setups use them while 2^-48 exp((pi / (2 eps h))^2)
// stays near 1e-12 (eps h >= 0.66, amplification <= 300), else FP64 arithmetic.
static bool df_resolves(const Geom& g, double eps) {
  double epsh = 1e300;
  for (int d = 0; d < g.dim; ++d) epsh = std::min(epsh, eps * 2.0 * g.T[d] / (double)(g.Ld[d] / g.s[d]));
  const double a = M_PI / (2.0 * epsh);
  return a * a <= std::log(300.0);
}

static bool mixed_resolves(const Geom& g, double eps) {
  double epsh = 1e300;
  for (int d = 0; d < g.dim; ++d) epsh = std::min(epsh, eps * 2.0 * g.T[d] / (double)(g.Ld[d] / g.s[d]));
  const double a = M_PI / (2.0 * epsh);
  return a * a <= std::log(1e-3 * 16777216.0);
}

// k = 0: the sketch width grows (64, 128, ... up to 4096 and N) until the
// k-th singular value of the sketch falls below tau_sat sigma_1, i.e. the
// sketch holds every direction of the perturbation above the level that
// precision resolves (FP64: 1e-7; mixed: 1e-4, the FP32 sketch's noise
// floor).  Each attempt is a complete setup; a saturated one is discarded.
az_status az_setup(const az_grid* gr, const uint8_t* mask, const double* bpts, int64_t n_boundary, double eps,
                   int32_t kernel, double boundary_weight, const az_options* opt, void* stream, az_handle* out) {
  if (!opt || opt->k != 0) return setup_fixed(gr, mask, bpts, n_boundary, eps, kernel, boundary_weight, opt, stream, out);
  if (!out || !gr) { set_error("az_setup: null argument"); return AZ_ERR_ARG; }
  *out = nullptr;
  int64_t N = 1;
  for (int d = 0; d < gr->dim && d < 2; ++d) N *= gr->n[d];
  // (2D mixed setups sketch in FP64, so they take the FP64 level)
  const double tsat = (opt->precision == AZ_FP64 || (gr->dim == 2)) ? 1e-7 : 1e-4;
  az_options o = *opt;
  az_handle prev = nullptr;   // the narrower setup, whose sketch columns are reused
  for (int k = 64;; k *= 2) {
    o.k = (int)std::min<int64_t>(std::min<int64_t>(k, 4096), std::max<int64_t>(1, N));
    az_handle h = nullptr;
    const az_status rs = setup_fixed(gr, mask, bpts, n_boundary, eps, kernel, boundary_weight, &o, stream, &h, prev);
    if (prev) az_destroy(prev);
    prev = nullptr;
    if (rs) return rs;
    az_info_t info;
    const az_status rc = az_get_info(h, &info);
    if (rc) { az_destroy(h); return rc; }
    const bool saturated = info.rank >= o.k && info.sigma_max > 0 && info.sigma_min_kept > tsat * info.sigma_max;
    if (!saturated || o.k >= 4096 || o.k >= N) { *out = h; return AZ_OK; }
    prev = h;
  }
}

static az_status setup_fixed(const az_grid* gr, const uint8_t* mask, const double* bpts, int64_t n_boundary,
                             double eps, int32_t kernel, double boundary_weight, const az_options* opt, void* stream,
                             az_handle* out, const az_setup_t* reuse) {
  if (!out) { set_error("az_setup: null output handle"); return AZ_ERR_ARG; }
  *out = nullptr;
  if (!mask) { set_error("az_setup: Omega mask is required"); return AZ_ERR_ARG; }
  if (!(eps > 0) || !std::isfinite(eps)) { set_error("az_setup: eps must be positive"); return AZ_ERR_ARG; }
  if (kernel != AZ_GAUSS && kernel != AZ_NEG_LAPLACE_GAUSS) { set_error("az_setup: unknown kernel"); return AZ_ERR_ARG; }
  if (n_boundary < 0 || (n_boundary > 0 && !bpts)) { set_error("az_setup: boundary points"); return AZ_ERR_ARG; }
  az_options o;
  if (opt) o = *opt;
  else { o.precision = AZ_MIXED; o.k = 24; o.tau_svd = 0; o.tau_sym = 0; o.seed = 1; o.refine_steps = -1; o.k0 = 0; o.bnormal = nullptr; }
  if (!std::isfinite(o.k0)) { set_error("az_setup: k0 must be finite"); return AZ_ERR_ARG; }
  if (o.precision != AZ_FP64 && o.precision != AZ_MIXED) { set_error("az_setup: precision"); return AZ_ERR_ARG; }
  if (o.k < 1 || o.k > 4096) { set_error("az_setup: k must be in [1, 4096]"); return AZ_ERR_ARG; }
  if (!gr) { set_error("az_setup: grid"); return AZ_ERR_ARG; }
  az_setup_t* h = new az_setup_t();
  az_status rc = make_geom(gr, h->g);
  if (rc) { delete h; return rc; }
  if (o.precision == AZ_MIXED && !mixed_resolves(h->g, eps)) {
    delete h;
    set_error("az_setup: eps h is too small for the FP32 sketch (mixed precision needs eps h >= 0.504); use AZ_FP64");
    return AZ_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  h->kind = kernel == AZ_NEG_LAPLACE_GAUSS ? 1 : 0;
  h->precision = o.precision;
  h->sk64 = o.precision == AZ_MIXED && h->g.dim == 2;
  h->prod64 = !df_resolves(h->g, eps);
  h->k = o.k;
  h->eps = eps;
  h->tau_svd = o.tau_svd > 0 ? o.tau_svd : 1e-8;
  h->tau_sym = o.tau_sym > 0 ? o.tau_sym : 0.0;
  h->k0 = h->kind == 1 ? o.k0 : 0.0;
  h->seed = o.seed;
  h->refine = o.refine_steps >= 0 ? o.refine_steps : (o.precision == AZ_MIXED ? 1 : 0);
  h->bweight = boundary_weight;
  h->Mb = h->kind == 1 ? n_boundary : 0;
  Geom& g = h->g;
  do {
    // S1: index map (the count M fixes the remaining allocations: one sync)
    rc = dalloc_t(h, &h->mask, g.L); if (rc) break;
    if (cudaMemcpyAsync(h->mask, mask, g.L, cudaMemcpyDeviceToDevice, st) != cudaSuccess) { set_error("az_setup: mask copy"); rc = AZ_ERR_CUDA; break; }
    rc = dalloc_t(h, &h->pos2m, g.L); if (rc) break;
    rc = dalloc_t(h, &h->idx, g.L); if (rc) break;
    rc = dalloc_t(h, &h->scan, 4096); if (rc) break;
    rc = dalloc_t(h, &h->Md, 1); if (rc) break;
    rc = launch_compact(h->mask, g.L, h->pos2m, h->idx, h->Md, h->scan, st); if (rc) break;
    int64_t M = 0;
    if (cudaMemcpyAsync(&M, h->Md, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { set_error("az_setup: reading M failed"); rc = AZ_ERR_CUDA; break; }
    h->M = M;
    h->Mtot = M + h->Mb;
    h->ldm = (h->Mtot + 31) / 32 * 32;
    if (h->Mtot < 1) { set_error("az_setup: Omega contains no grid point"); rc = AZ_ERR_ARG; break; }
    // Y = A W (Mtot x k) has rank <= Mtot: a wider sketch adds no direction,
    // and the Householder route needs k <= Mtot; the first columns of R are kept
    h->k = (int)std::min<int64_t>(h->k, h->Mtot);
    h->periodic = M == g.L && h->Mb == 0 && h->kind == 0 && h->tau_sym == 0.0;
    if (M > 0) {
      // kept points forming one run of consecutive grid indices (a 1D
      // interval): the gather then needs no index-map lookups
      int32_t ends[2] = {0, 0};
      if (cudaMemcpy(&ends[0], h->idx, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(&ends[1], h->idx + (M - 1), sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("az_setup: reading the index map failed"); rc = AZ_ERR_CUDA; break;
      }
      if ((int64_t)ends[1] - ends[0] + 1 == M) { h->g.run0 = ends[0]; h->g.runM = M; }
    }
    if (h->Mb) {
      rc = dalloc_t(h, &h->bpts, (size_t)g.dim * h->Mb); if (rc) break;   // Mb x dim
      if (cudaMemcpyAsync(h->bpts, bpts, (size_t)g.dim * h->Mb * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) { rc = AZ_ERR_CUDA; break; }
      if (o.bnormal) {
        rc = dalloc_t(h, &h->bnrm, (size_t)g.dim * h->Mb); if (rc) break;
        if (cudaMemcpyAsync(h->bnrm, o.bnormal, (size_t)g.dim * h->Mb * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) { rc = AZ_ERR_CUDA; break; }
      }
    }
    // twiddle tables (host-built constants)
    {
      std::vector<double> re, im;
      host_twiddles(4096, re, im);
      // master table w_4096^j (j < 4096), then the stage table of the
      // register FFTs: w_m^(b k) = w_4096^(b k 4096/m) at 4096 + 2m - m/b + k
      // for each span m <= 4096, power of two b <= m/2 and k < m/(2b)
      constexpr int NT = 4096 + 8192;
      std::vector<double2> t64(NT);
      std::vector<float2> t32(NT);
      for (int m = 0; m < 4096; ++m) { t64[m] = make_double2(re[m], im[m]); t32[m] = make_float2((float)re[m], (float)im[m]); }
      for (int m = 2; m <= 4096; m *= 2)
        for (int b = 1; 2 * b <= m; b *= 2)
          for (int k = 0; k < m / (2 * b); ++k) {
            const int dst = 4096 + 2 * m - m / b + k, src = b * k * (4096 / m);
            t64[dst] = t64[src];
            t32[dst] = t32[src];
          }
      rc = dalloc_t(h, &h->tw64, NT); if (rc) break;
      rc = dalloc_t(h, &h->tw32, NT); if (rc) break;
      if (cudaMemcpy(h->tw64, t64.data(), NT * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(h->tw32, t32.data(), NT * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) { rc = AZ_ERR_CUDA; break; }
      rc = big_tables(h, g.L, &h->big64[0], &h->big64[1], &h->big32[0], &h->big32[1], st); if (rc) break;
      rc = big_tables(h, g.N, &h->big64[2], &h->big64[3], &h->big32[2], &h->big32[3], st); if (rc) break;
    }
    stencil_widths(h);
    rc = alloc_symbol(h); if (rc) break;
    h->nw = (g.N + 31) / 32;
    rc = dalloc_t(h, &h->bits, (size_t)h->nw * h->k + 4); if (rc) break;
    const size_t tsz = store64(h) ? 8 : 4;
    rc = dalloc(h, &h->W, (size_t)g.N * h->k * tsz); if (rc) break;
    rc = dalloc(h, &h->Y, (size_t)h->Mtot * h->k * tsz); if (rc) break;
    rc = dalloc(h, &h->Ut, (size_t)h->ldm * h->k * tsz); if (rc) break;
    if (h->sk64) { rc = dalloc_t(h, &h->Ut32, (size_t)h->ldm * h->k); if (rc) break; }
    rc = dalloc_t(h, &h->tc_err, 1); if (rc) break;
    if (cudaEventCreateWithFlags(&h->info_ev, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); set_error("event"); rc = AZ_ERR_CUDA; break; }
    if (cudaMemsetAsync(h->tc_err, 0, sizeof(int), st) != cudaSuccess) { cudaGetLastError(); set_error("memset"); rc = AZ_ERR_CUDA; break; }
    rc = dalloc_t(h, &h->Q1, (size_t)std::max<int64_t>(h->Mtot, (h->ldm + 1) / 2) * h->k); if (rc) break;   // also holds FP32 Q1 with ld ldm
    {
      // opt-in: AZ_SKETCH_CLUSTER=1 (the chain is FP64-arithmetic bound on
      // this GPU, where the three-pass chain spreads over every SM and is
      // faster; both are tested against each other and the oracle)
      const char* ev = std::getenv("AZ_SKETCH_CLUSTER");
      h->use_cluster = store64(h) && ev && ev[0] == '1' && zstar_cluster_ok(g, st);
    }
    if (h->kind == 1 || h->use_cluster) { rc = dalloc_t(h, &h->Rd, (size_t)g.N * h->k); if (rc) break; }
    for (double** p : {&h->G, &h->V, &h->B1, &h->Tm, &h->VS}) { rc = dalloc_t(h, p, (size_t)h->k * h->k); if (rc) break; }
    if (rc) break;
    rc = dalloc_t(h, &h->lam, h->k); if (rc) break;
    rc = dalloc_t(h, &h->sig, h->k); if (rc) break;
    rc = dalloc_t(h, &h->info, 1); if (rc) break;
    rc = alloc_workspace(h); if (rc) break;
    if (h->kind == 1) { rc = dalloc_t(h, &h->bcoll, (size_t)h->Mtot * 2 * h->pairs_max); if (rc) break; }
    if (h->kind == 0 && !h->periodic && h->k <= kNarrowK && !(store64(h) && h->tau_svd < kGramTau)) {
      // overlap of az_refactor's sketch with the next solve: own stream,
      // events and FFT workspace for the sketch chain
      h->pairs_s = std::min(h->pairs_max, (h->k + 1) / 2);
      const size_t vsz = store64(h) ? 16 : 8;
      rc = dalloc(h, &h->X1s, (size_t)h->pairs_s * g.L * vsz); if (rc) break;
      rc = dalloc(h, &h->X3s, (size_t)h->pairs_s * g.N * vsz); if (rc) break;
      // higher priority: the sketch-to-factor chain is the critical path, and
      // the solve's passes fill the SMs it leaves idle (the one-CTA factor
      // kernels)
      int prio_lo = 0, prio_hi = 0;
      cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
      if (cudaStreamCreateWithPriority(&h->fst, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_sym, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_fac, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError(); set_error("az_setup: stream or event"); rc = AZ_ERR_CUDA; break;
      }
    }
    // The Gram route squares the sketch's condition number, so in FP64 it
    // resolves singular values down to about 1e-8 sigma_1; a tighter tau
    // takes the Householder route whatever the width.
    if (h->k > kNarrowK || (store64(h) && h->tau_svd < kGramTau)) {
      size_t wb = 0;
      rc = large_create(&h->wide, h->Mtot, h->k, store64(h), h->Q1, &wb, 2 * h->pairs_max, h->prod64);
      h->bytes += wb;
      if (rc) break;
    } else {
      rc = dalloc_t(h, &h->partial, (size_t)partial_blocks(h->Mtot) * h->k * std::max(h->k, 2 * h->pairs_max)); if (rc) break;
    }
    // rounding floor of the sketch's singular values: 1e-13 * ||A R||_F, with
    // ||A R||_F^2 ~ k (Mtot/L) sum_k S_k / s (estimate from the symbol's peak)
    rc = build_symbol(h, st); if (rc) break;
    {
      double smax = 0;
      if (cudaMemcpyAsync(&smax, h->S + g.N, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) { set_error("az_setup: symbol readback"); rc = AZ_ERR_CUDA; break; }
      double est = std::sqrt((double)h->k * (double)h->Mtot / (double)g.L * (double)g.N * smax / (double)(g.s[0] * g.s[1]));
      h->floor = 1e-13 * est;
    }
    // S3-S7
    if (reuse && reuse->k < h->k && reuse->k % 2 == 0 && reuse->precision == h->precision && reuse->seed == h->seed &&
        reuse->g.N == g.N && reuse->Mtot == h->Mtot && !h->periodic) {
      // adaptive growth: the first reuse->k columns of R, hence of W and Y,
      // are those of the narrower setup (same seed, same geometry)
      const size_t tsz = store64(h) ? 8 : 4;
      if (cudaMemcpyAsync(h->W, reuse->W, (size_t)g.N * reuse->k * tsz, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(h->Y, reuse->Y, (size_t)h->Mtot * reuse->k * tsz, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError(); set_error("az_setup: sketch column copy"); rc = AZ_ERR_CUDA; break;
      }
      h->k_done = reuse->k;
    }
    rc = sketch_factor_any(h, st);
    if (rc) break;
    FactorInfo fi;
    if (cudaMemcpyAsync(&fi, h->info, sizeof(fi), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) { set_error("az_setup: factorisation readback"); rc = AZ_ERR_CUDA; break; }
    if (fi.status != 0) {
      set_error(fi.status == 1 ? "factorisation: Cholesky breakdown in the second pass" : "factorisation: non-finite sketch");
      rc = AZ_ERR_NUMERIC;
      break;
    }
  } while (0);
  if (rc) { destroy(h); return rc; }
  *out = h;
  return AZ_OK;
}

az_status az_refactor(az_handle h, uint64_t seed, void* stream) {
  if (!h) { set_error("az_refactor: null handle"); return AZ_ERR_ARG; }
  h->seed = seed;
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->fst) return compute_setup(h, st, true);
  // index map and symbol on the caller's stream (after any earlier
  // factorisation); sketch and factorisation on the setup's stream
  if (h->fac_pending) AZ_CUDA(cudaStreamWaitEvent(st, h->ev_fac, 0));
  AZ_TRY(launch_compact(h->mask, h->g.L, h->pos2m, h->idx, h->Md, h->scan, st));
  AZ_TRY(build_symbol(h, st));
  AZ_CUDA(cudaEventRecord(h->ev_sym, st));
  AZ_CUDA(cudaStreamWaitEvent(h->fst, h->ev_sym, 0));
  const az_status rc = sketch_factor_any(h, h->fst);
  // recorded whatever happened, so that later calls wait for whatever was
  // enqueued before an error
  AZ_CUDA(cudaEventRecord(h->info_ev, h->fst));
  AZ_CUDA(cudaEventRecord(h->ev_fac, h->fst));
  h->fac_pending = true;
  return rc;
}

az_status az_solve(az_handle h, const double* b, int64_t ldb, int64_t nrhs, double* x, int64_t ldx, void* stream,
                   double* relres) {
  if (!h || !b || !x || nrhs < 0 || ldb < h->Mtot || ldx < h->g.N) { set_error("az_solve: bad arguments"); return AZ_ERR_ARG; }
  if (nrhs == 0) return AZ_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return h->precision == AZ_FP64 ? solve_impl<double>(h, b, ldb, nrhs, x, ldx, st, relres)
                                 : solve_impl<float>(h, b, ldb, nrhs, x, ldx, st, relres);
}

az_status az_collocate(az_handle h, const double* f, int64_t ldf, const double* gb, int64_t ldg, int64_t nrhs,
                       double* x, int64_t ldx, void* stream, double* relres) {
  if (!h || h->kind != 1) { set_error("az_collocate: needs a collocation setup"); return AZ_ERR_ARG; }
  if (!f || !gb || !x || nrhs < 0 || ldf < h->M || ldg < h->Mb || ldx < h->g.N) { set_error("az_collocate: bad arguments"); return AZ_ERR_ARG; }
  if (nrhs == 0) return AZ_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // the scaled data [f / (2 eps^2); w g] in the handle's buffer, one solve
  // chunk at a time (stream-ordered: no allocation, no synchronisation)
  const int chunk = 2 * h->pairs_max;
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int nc = (int)std::min<int64_t>(chunk, nrhs - c0);
    double* b = h->bcoll;
    AZ_TRY(launch_scale_rows(f + c0 * ldf, ldf, h->M, nc, 1.0 / (2.0 * h->eps * h->eps), b, h->Mtot, st));
    AZ_TRY(launch_boundary_rhs(h->g.dim, gb + c0 * ldg, ldg, h->Mb, nc, h->bnrm, h->bweight, h->eps, b + h->M,
                               h->Mtot, st));
    AZ_TRY(az_solve(h, b, h->Mtot, nc, x + c0 * ldx, ldx, stream, relres ? relres + c0 : nullptr));
  }
  return AZ_OK;
}

az_status az_evaluate(az_handle h, const double* x, int64_t ldx, int64_t nrhs, int32_t s_test, double* out, int64_t ldo,
                      void* stream) {
  if (!h || !x || !out || s_test < 1 || nrhs < 0) { set_error("az_evaluate: bad arguments"); return AZ_ERR_ARG; }
  int64_t npts = h->g.dim == 1 ? h->g.n[0] * s_test : h->g.n[0] * s_test * h->g.n[1] * s_test;
  if (ldo < npts || ldx < h->g.N) { set_error("az_evaluate: leading dimension"); return AZ_ERR_ARG; }
  if (nrhs == 0) return AZ_OK;
  return launch_evaluate(h->g, h->eps, s_test, x, ldx, (int)nrhs, out, ldo, (cudaStream_t)stream);
}

az_status az_apply_A(az_handle h, const double* x, int64_t ldx, int64_t nrhs, double* y, int64_t ldy, void* stream) {
  if (!h || !x || !y || ldx < h->g.N || ldy < h->Mtot || nrhs < 0) { set_error("az_apply_A: bad arguments"); return AZ_ERR_ARG; }
  if (nrhs == 0) return AZ_OK;
  return apply_rows<double, double, double, double>(h, x, ldx, nullptr, 0, 0.0, 1.0, y, ldy, (int)nrhs,
                                                    (cudaStream_t)stream);
}

az_status az_apply_Zstar(az_handle h, const double* y, int64_t ldy, int64_t nrhs, double* x, int64_t ldx, void* stream) {
  if (!h || !x || !y || ldx < h->g.N || ldy < h->Mtot || nrhs < 0) { set_error("az_apply_Zstar: bad arguments"); return AZ_ERR_ARG; }
  if (nrhs == 0) return AZ_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // FP64 chain on a private workspace (one pair at a time in mixed handles)
  void* sX1 = h->X1; void* sX3 = h->X3; int spm = h->pairs_max;
  if (h->precision != AZ_FP64) {
    if (!h->X1d) {
      if (cudaMalloc(&h->X1d, (size_t)h->g.L * 16) != cudaSuccess || cudaMalloc(&h->X3d, (size_t)h->g.N * 16) != cudaSuccess) {
        cudaGetLastError(); set_error("az_apply_Zstar: workspace"); return AZ_ERR_OOM;
      }
    }
    h->X1 = h->X1d; h->X3 = h->X3d; h->pairs_max = 1;
  }
  az_status rc = zstar_chain<double, double>(h, 0, y, ldy, (int)nrhs, x, ldx, st);
  h->X1 = sX1; h->X3 = sX3; h->pairs_max = spm;
  return rc;
}

az_status az_get_info(az_handle h, az_info_t* info) {
  if (!h || !info) { set_error("az_get_info: bad arguments"); return AZ_ERR_ARG; }
  FactorInfo fi;
  int tcerr = 0;
  // waits for the latest factorisation only, not for other streams' work
  AZ_CUDA(cudaEventSynchronize(h->info_ev));
  AZ_CUDA(cudaMemcpy(&fi, h->info, sizeof(fi), cudaMemcpyDeviceToHost));
  AZ_CUDA(cudaMemcpy(&tcerr, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (tcerr) {
    // reported once: the flag is cleared so that later calls start clean
    AZ_CUDA(cudaMemset(h->tc_err, 0, sizeof(int)));
    set_error(tc_wait_message(tcerr));
    return AZ_ERR_TIMEOUT;
  }
  info->N = h->g.N; info->L = h->g.L; info->M = h->M; info->Mb = h->Mb; info->k = h->k;
  info->rank = fi.r; info->rank_gram = fi.r1; info->precision = h->precision;
  info->sigma_max = fi.sigma_max; info->sigma_min_kept = fi.sigma_min_kept;
  info->device_bytes = h->bytes;
  info->jacobi_sweeps = fi.pad;
  return AZ_OK;
}

az_status az_get_array(az_handle h, int32_t which, double* dst, void* stream) {
  if (!h || !dst) { set_error("az_get_array: bad arguments"); return AZ_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (h->fac_pending) AZ_CUDA(cudaStreamWaitEvent(st, h->ev_fac, 0));
  const bool f64 = store64(h);
  switch (which) {
    case AZ_ARRAY_SYMBOL:
      AZ_CUDA(cudaMemcpyAsync(dst, h->Ghat, h->g.L * sizeof(double), cudaMemcpyDeviceToDevice, st));
      return AZ_OK;
    case AZ_ARRAY_SKETCH:
      return f64 ? to_double<double>((double*)h->Y, h->Mtot, h->Mtot, h->k, dst, h->Mtot, st)
                 : to_double<float>((float*)h->Y, h->Mtot, h->Mtot, h->k, dst, h->Mtot, st);
    case AZ_ARRAY_W:
      return f64 ? to_double<double>((double*)h->W, h->g.N, h->g.N, h->k, dst, h->g.N, st)
                 : to_double<float>((float*)h->W, h->g.N, h->g.N, h->k, dst, h->g.N, st);
    case AZ_ARRAY_R:
      return launch_bits_to_R(h->bits, h->g.N, h->k, dst, st);
    case AZ_ARRAY_UT: {
      FactorInfo fi;
      AZ_CUDA(cudaStreamSynchronize(st));
      AZ_CUDA(cudaMemcpy(&fi, h->info, sizeof(fi), cudaMemcpyDeviceToHost));
      return f64 ? to_double<double>((double*)h->Ut, h->ldm, h->Mtot, fi.r, dst, h->Mtot, st)
                 : to_double<float>((float*)h->Ut, h->ldm, h->Mtot, fi.r, dst, h->Mtot, st);
    }
    case AZ_ARRAY_SIGMA: {
      FactorInfo fi;
      AZ_CUDA(cudaStreamSynchronize(st));
      AZ_CUDA(cudaMemcpy(&fi, h->info, sizeof(fi), cudaMemcpyDeviceToHost));
      AZ_CUDA(cudaMemcpyAsync(dst, h->sig, std::max(fi.r, 0) * sizeof(double), cudaMemcpyDeviceToDevice, st));
      return AZ_OK;
    }
    case AZ_ARRAY_KEPT:
      return to_double<int32_t>(h->idx, h->M, h->M, 1, dst, h->M, st);
    default:
      set_error("az_get_array: unknown array");
      return AZ_ERR_ARG;
  }
}

}  // extern "C"
