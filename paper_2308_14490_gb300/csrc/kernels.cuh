// Host-side launchers of the kernels in kernels.cu (all stream-ordered).
#pragma once
#include "az_internal.cuh"

namespace az {

// Images |p| <= P of Eq. periodic_rbf needed in a box of half-width T: the
// first omitted image is below exp(-700) of the peak everywhere in the box.
int image_count(double eps, double T);

// S1: compact index map of the kept grid points.  pos2m[L] (-1 if not kept),
// idx[M]; the count M is written to *M_dev.
az_status launch_compact(const uint8_t* mask, int64_t L, int32_t* pos2m, int32_t* idx, int64_t* M_dev,
                         int32_t* scratch_blocks, cudaStream_t st);

// S2: periodised samples g(m) = sum_p f((m + p L) h_L) on one dimension
// (f = phi or phi''), FP64, m = 0..L-1.
az_status launch_samples(double* g, int64_t L, double hL, double eps, int deriv, int pimg, cudaStream_t st);
az_status launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st);   // y += a x
// 1D: stencil taps from the image sum, and Ghat from its Poisson-summation form
// (ode != 0: of the collocation kernel -(phi'' + k0^2 phi) / (2 eps^2) instead of phi)
az_status launch_taps_direct(int64_t L, double hL, double eps, int pimg, int W64, double* t64, int W32, float* t32,
                             cudaStream_t st, float* th, float* tl, int ode = 0, double k0 = 0.0);
az_status launch_symbol_closed_1d(int64_t L, double a, double* Ghat, cudaStream_t st, int ode = 0, double hL = 0.0,
                                  double k0 = 0.0, double eps = 1.0);
// stencil taps t[m + W] = g(m mod L) for |m| <= W, FP64 and FP32 copies
az_status launch_taps(const double* g, int64_t L, int W64, double* t64, int W32, float* t32, cudaStream_t st,
                      float* th = nullptr, float* tl = nullptr);
// FP64-accurate residual rows (kept grid rows only): out = b - A x for x exactly
// representable in FP32 (given as floats), taps split into FP32 hi/lo.
az_status launch_resid_df(const Geom& g, int kind, double eps, const int32_t* idx, int64_t M, const float* const th[4],
                          const float* const tl[4], int Wx, int Wy, const float* xf, int64_t ldx, const double* b,
                          int64_t ldb, float* out, int64_t ldo, int ncols, cudaStream_t st);

// Twiddle tables (host-built, copied): master table of 4096 entries w_4096^m.
void host_twiddles(int n, std::vector<double>& re, std::vector<double>& im);

// S3: packed Rademacher bits, nw = ceil(N/32) words per column.
az_status launch_philox_bits(uint32_t* bits, int64_t N, int k, uint64_t seed, cudaStream_t st);
az_status launch_bits_to_R(const uint32_t* bits, int64_t N, int k, double* R, cudaStream_t st);

struct PassTabs {
  const void* tw;        // master twiddle table (4096 entries) then the stage table (8192), float2 or double2
  const void* bigA;      // four-step twiddles for L (1D): w_L^m = bigA[m>>12]*bigB[m&4095]
  const void* bigB;
  const void* bigNA;     // same for N (fold inverse twiddle)
  const void* bigNB;
};

template <typename T> struct SketchIn {
  const uint32_t* bits; int64_t nw; int k;       // Rademacher bits
  const int32_t* pos2m;                          // mask via index map
  const T* tapx; const T* tapy; int Wx, Wy;      // phi taps per dim
};

// Forward column pass, prologue variants.  Output: X1 (npairs x L complex, spectrum/column layout)
template <typename T>
az_status launch_colfwd_stencil(const Geom& g, const SketchIn<T>& in, int pair0, int npairs,
                                typename C2<T>::t* X1, const PassTabs& tb, cudaStream_t st);
template <typename T, typename TB>
az_status launch_colfwd_gather(const Geom& g, const int32_t* pos2m, const TB* b, int64_t ldb, int ncols,
                               int pair0, int npairs, typename C2<T>::t* X1, const PassTabs& tb,
                               cudaStream_t st, int64_t M_rows);
// Row pass with the alias-group fold by H = Ghat * S^{-1}: output on the N-grid (npairs x N complex)
template <typename T>
az_status launch_rowfold(const Geom& g, const typename C2<T>::t* X1, const T* H, int npairs,
                         typename C2<T>::t* X3, const PassTabs& tb, cudaStream_t st);
// Inverse column pass on the N-grid; epilogue writes z = IDFT_N(.) into real
// columns (pair p -> columns 2p, 2p+1 of out, ld), or W = R - z when bits != null.
template <typename T, typename TO>
az_status launch_colinv(const Geom& g, const typename C2<T>::t* X3, int pair0, int npairs, int ncols,
                        TO* out, int64_t ldo, const uint32_t* bits, int64_t nw, const PassTabs& tb,
                        cudaStream_t st);

// Rows of A applied to coefficients: out[m,c] = alpha*b[m,c] + beta*(A z)[m,c],
// m < M (kept grid rows; kind 0 Gaussian, 1 -Lap/(2 eps^2)), computed in T.
struct StencilTaps {
  const void* x0; const void* x2; const void* y0; const void* y2; int Wx, Wy;
};
template <typename T, typename TZ, typename TB, typename TO>
az_status launch_stencil_rows(const Geom& g, int kind, double eps, const int32_t* idx, int64_t M,
                              const StencilTaps& tp, const TZ* z, int64_t ldz, const TB* b, int64_t ldb,
                              T alpha, T beta, TO* out, int64_t ldo, int ncols, cudaStream_t st);
// Boundary rows: out[m,c] = alpha*b[m,c] + beta*w*sum_j r_j(p_m) z[j,c], m < Mb, with
// r_j = phi_j (Dirichlet) or n_m . grad phi_j / eps where the normal n_m (nrm, Mb x dim,
// may be null) is nonzero (Neumann)
template <typename T, typename TZ, typename TB, typename TO>
az_status launch_boundary_rows(const Geom& g, double eps, double w, const double* pts, const double* nrm, int64_t Mb,
                               const TZ* z, int64_t ldz, const TB* b, int64_t ldb, T alpha, T beta,
                               TO* out, int64_t ldo, int ncols, cudaStream_t st);
// Boundary data: out = w g (Dirichlet points), w g / eps (Neumann points)
az_status launch_boundary_rhs(int dim, const double* g, int64_t ldg, int64_t Mb, int ncols, const double* nrm,
                              double w, double eps, double* out, int64_t ldo, cudaStream_t st);
// Values of sum_j x_j phi_j on the s_test-refined full grid (FP64)
az_status launch_evaluate(const Geom& g, double eps, int s_test, const double* x, int64_t ldx, int nrhs,
                          double* out, int64_t ldo, cudaStream_t st);

// Symbol assembly: Ghat on the L-grid in natural frequency order (FP64, from per-dim
// FFTs), S on the N-grid, H = Ghat*Sinv stored in the row-pass layout (FP64+FP32).
az_status launch_symbol_full(const Geom& g, int kind, double eps, const double* G0x, const double* G0y,
                             const double* G2x, const double* G2y, double* Ghat, cudaStream_t st);
az_status launch_fold_S(const Geom& g, const double* Ghat, double* S, cudaStream_t st);
az_status launch_H(const Geom& g, const double* Ghat, const double* S, double thr, double* H64, float* H32,
                   cudaStream_t st);
az_status launch_max_abs(const double* v, int64_t n, double* out, cudaStream_t st);
// Take the real part of a spectrum (1D four-step layout -> natural frequency order)
// One-line FFT (length n <= 4096) of a real FP64 array: out = Re(DFT(in))
az_status launch_line_dft_real(const double* in, int n, double* out, const double2* tw, cudaStream_t st);

// Elementwise helpers
az_status launch_scale_rows(const double* in, int64_t ldi, int64_t rows, int ncols, double sc, double* out,
                            int64_t ldo, cudaStream_t st);
az_status launch_sumsq_cols(const double* v, int64_t ld, int64_t rows, int ncols, double* out, cudaStream_t st);

}  // namespace az
