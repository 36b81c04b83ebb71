// In-shared-memory Stockham FFT stages for batches of lines (FP32 / FP64).
//
// A batch of `nlines` lines of length n (a power of two, 2..4096) lives in
// shared memory; element i of line c sits at base[c*cs + i*is].  The transform
// runs as a sequence of radix-R Stockham autosort stages (R in {2,4,8,16}),
// ping-ponging between two buffers, so input and output are both in natural
// order.  One stage, for butterfly j in [0, n/R) with current span Ns:
//   k = j mod Ns;  a_t = in[j + t n/R] * w_{Ns R}^{t k};  b = DFT_R(a);
//   out[(j - k) R + k + u Ns] = b_u.
// The forward transform uses w_m = exp(-2 pi i / m), the inverse its conjugate
// (no 1/n scaling here).  Twiddles come from a master table
// tw[m] = exp(-2 pi i m / 4096) built on the host in FP64 from exact rationals of
// pi; a transform of length n reads it with stride tws = 4096 / n.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace az {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <typename V> __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) { return cmk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); } // a*conj(b)
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return cmk<V>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename V, bool INV> __device__ __forceinline__ V mul_mi(V a) { return INV ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x); }

template <typename V, bool INV> __device__ __forceinline__ void dft2(V& a, V& b) { V t = a; a = cadd(t, b); b = csub(t, b); }

template <typename V, bool INV> __device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
  V s0 = cadd(a0, a2), d0 = csub(a0, a2), s1 = cadd(a1, a3), d1 = mul_mi<V, INV>(csub(a1, a3));
  a0 = cadd(s0, s1); a2 = csub(s0, s1); a1 = cadd(d0, d1); a3 = csub(d0, d1);
}

// exp(-+ 2 pi i m / 8) for m = 1, 3 (forward sign; INV conjugates)
template <typename V, bool INV> __device__ __forceinline__ V w8(V a, int m) {
  using T = decltype(V::x);
  const T h = (T)0.70710678118654752440;
  // m=1: (h, -h) ; m=2: (0,-1) ; m=3: (-h, -h)
  V w = m == 1 ? cmk<V>(h, -h) : (m == 2 ? cmk<V>((T)0, (T)-1) : cmk<V>(-h, -h));
  if (INV) w.y = -w.y;
  return cmul(a, w);
}

template <typename V, bool INV> __device__ __forceinline__ void dft8(V* a) {
  // n = 2 n1 + n2, k = k1 + 4 k2 : inner DFT4 over n1, twiddle w8^{n2 k1}, DFT2 over n2
  dft4<V, INV>(a[0], a[2], a[4], a[6]);
  dft4<V, INV>(a[1], a[3], a[5], a[7]);
  a[3] = w8<V, INV>(a[3], 1); a[5] = w8<V, INV>(a[5], 2); a[7] = w8<V, INV>(a[7], 3);
  V o[8];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    V x0 = a[2 * k1], x1 = a[2 * k1 + 1];
    o[k1] = cadd(x0, x1); o[k1 + 4] = csub(x0, x1);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = o[i];
}

template <typename V, bool INV> __device__ __forceinline__ V w16(V a, int m) {
  using T = decltype(V::x);
  // exp(-2 pi i m/16), m in [0, 9]
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, h = (T)0.70710678118654752440;
  T wr, wi;
  switch (m) {
    case 0: return a;
    case 1: wr = c1; wi = -s1; break;
    case 2: wr = h; wi = -h; break;
    case 3: wr = s1; wi = -c1; break;
    case 4: wr = 0; wi = -1; break;
    case 6: wr = -h; wi = -h; break;
    case 9: wr = -c1; wi = s1; break;
    default: wr = 1; wi = 0; break;
  }
  if (INV) wi = -wi;
  return cmul(a, cmk<V>(wr, wi));
}

template <typename V, bool INV> __device__ __forceinline__ void dft16(V* a) {
  // n = 4 n1 + n2, k = k1 + 4 k2
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<V, INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
  // now a[4 k1 + n2] holds Y[n2][k1]; twiddle by w16^{n2 k1}
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) a[4 * k1 + n2] = w16<V, INV>(a[4 * k1 + n2], n2 * k1);
  V o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    V x0 = a[4 * k1], x1 = a[4 * k1 + 1], x2 = a[4 * k1 + 2], x3 = a[4 * k1 + 3];
    dft4<V, INV>(x0, x1, x2, x3);
    o[k1] = x0; o[k1 + 4] = x1; o[k1 + 8] = x2; o[k1 + 12] = x3;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = o[i];
}

template <typename V, int R, bool INV> __device__ __forceinline__ void dftR(V* a) {
  if constexpr (R == 2) dft2<V, INV>(a[0], a[1]);
  else if constexpr (R == 4) dft4<V, INV>(a[0], a[1], a[2], a[3]);
  else if constexpr (R == 8) dft8<V, INV>(a);
  else dft16<V, INV>(a);
}

// One Stockham stage over all lines (nlines = 2^lognl, n = 2^logn).
template <typename V, int R, int LOGR, bool INV>
__device__ __forceinline__ void stockham_stage(const V* __restrict__ in, V* __restrict__ out, int logn, int Ns,
                                               int lognl, int cs, int is, const V* __restrict__ tw, int tws) {
  const int n = 1 << logn;
  const int lognbf = logn - LOGR;
  const int nbf = 1 << lognbf;
  const int total = nbf << lognl;
  const int step = n / (Ns * R);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int c, j;
    if (cs == 1) { c = t & ((1 << lognl) - 1); j = t >> lognl; } else { j = t & (nbf - 1); c = t >> lognbf; }
    const int k = j & (Ns - 1);
    V a[R];
#pragma unroll
    for (int u = 0; u < R; ++u) a[u] = in[c * cs + (j + u * nbf) * is];
    if (Ns > 1) {
#pragma unroll
      for (int u = 1; u < R; ++u) {
        V w = __ldg(tw + ((u * k * step) & (n - 1)) * tws);
        if (INV) w.y = -w.y;
        a[u] = cmul(a[u], w);
      }
    }
    dftR<V, R, INV>(a);
    const int ob = (j - k) * R + k;
#pragma unroll
    for (int u = 0; u < R; ++u) out[c * cs + (ob + u * Ns) * is] = a[u];
  }
}

// Full FFT of length n = 2^logn on 2^lognl lines.  Data starts in buf0; the
// result ends in buf[return value] (0 or 1).  Contains __syncthreads().
template <typename V, bool INV>
__device__ int fft_lines(V* buf0, V* buf1, int logn, int lognl, int cs, int is, const V* __restrict__ tw, int tws) {
  V* b[2] = {buf0, buf1};
  int cur = 0, Ns = 1, rem = logn;
  while (rem > 0) {
    // radix plan: 16 while >= 4 bits remain (but avoid leaving 1 bit: use 8 then)
    if (rem >= 4 && rem != 5) { stockham_stage<V, 16, 4, INV>(b[cur], b[cur ^ 1], logn, Ns, lognl, cs, is, tw, tws); Ns <<= 4; rem -= 4; }
    else if (rem >= 3) { stockham_stage<V, 8, 3, INV>(b[cur], b[cur ^ 1], logn, Ns, lognl, cs, is, tw, tws); Ns <<= 3; rem -= 3; }
    else if (rem == 2) { stockham_stage<V, 4, 2, INV>(b[cur], b[cur ^ 1], logn, Ns, lognl, cs, is, tw, tws); Ns <<= 2; rem -= 2; }
    else { stockham_stage<V, 2, 1, INV>(b[cur], b[cur ^ 1], logn, Ns, lognl, cs, is, tw, tws); Ns <<= 1; rem -= 1; }
    cur ^= 1;
    __syncthreads();
  }
  return cur;
}

}  // namespace az
