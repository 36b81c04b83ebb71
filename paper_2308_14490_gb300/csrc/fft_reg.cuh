// Register-resident Stockham FFT of one line distributed over P threads.
//
// A line of length n = 2^logn (n >= E) is held by P = n / E threads, E
// elements each.  Each Stockham stage of radix R = 2^LR (R <= E) gives every
// thread E/R butterflies j = tl + g P (g < E/R); butterfly j reads positions
// j + u n/R, applies the twiddles w_{Ns R}^{u k} (k = j mod Ns), does a radix-R
// DFT and writes positions (j - k) R + k + u Ns.  The first stage takes its
// inputs from a caller-supplied prologue, the last stage hands its outputs to
// an epilogue, and the stages in between exchange data through one
// shared-memory buffer, padded by one element every 2^PADSH elements to spread
// strided accesses over the banks.  Stage radices are compile-time (one stage
// of radix 2^(logn mod log E) first, then radix-E stages) so the E values stay
// in registers.  Every thread of the block must call this (it contains
// __syncthreads()); threads with active == false only take part in barriers.
//
// Twiddles come from the stage table stw: for a span m = Ns R <= 4096 and a
// power of two b < R, the values w_m^(b k) for k < m / (2b) sit contiguously
// at stw[2m - m/b + k], so the gathers of a warp's consecutive k read
// consecutive entries (a strided read of one master table of w_4096 would
// touch up to one cache line per thread).
#pragma once
#include <type_traits>

#include "fft.cuh"

namespace az {

// The last stage hands each output to the epilogue as epi(o, v), or, when the
// epilogue accepts them, as epi(o, v, u, o0, Ns) with o = o0 + u * Ns and u
// the (compile-time, after unrolling) output slot of the butterfly: an
// epilogue that multiplies by w^(c * o) can then form it from w^(c * o0) and
// the powers w^(c * Ns * 2^b) instead of one table gather per output.
// The first stage reads input p through pro(p), or, when the prologue accepts
// them, pro(p, g, u) with the butterfly group g and slot u of this thread
// (compile-time after unrolling; p = tl + g P + u n/R).
template <typename V, typename Pro>
__device__ __forceinline__ V pro_call(Pro& pro, int p, int g, int u) {
  if constexpr (std::is_invocable_v<Pro&, int, int, int>) return pro(p, g, u);
  else return pro(p);
}

template <typename Epi, typename V>
__device__ __forceinline__ void epi_call(Epi& epi, int o, const V& v, int u, int o0, int Ns) {
  if constexpr (std::is_invocable_v<Epi&, int, V, int, int, int>) epi(o, v, u, o0, Ns);
  else epi(o, v);
}

template <int PADSH> __device__ __forceinline__ int padix(int e) { return e + (e >> PADSH); }

template <typename V, int E, int LR, bool INV, int PADSH, class Pro, class Epi>
__device__ __forceinline__ void fft_stage(V (&v)[E], V* __restrict__ sm, int logn, int Ns, bool first, bool last,
                                          bool active, int line, int tl, int cs, int is, const V* __restrict__ stw,
                                          Pro& pro, Epi& epi, bool sync_first) {
  constexpr int R = 1 << LR;
  constexpr int NG = E / R;
  const int n = 1 << logn;
  const int nbf = n >> LR;
  const int P = n / E;
  const int m = Ns * R;   // span of this stage: its twiddles are w_m^(u k), k < Ns
  if (active) {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int j = tl + g * P;
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const int p = j + u * nbf;
        if (first) v[g * R + u] = pro_call<V>(pro, p, g, u);
        else v[g * R + u] = sm[padix<PADSH>(line * cs + p * is)];
      }
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int j = tl + g * P;
      const int k = j & (Ns - 1);
      if (Ns > 1) {
        // w^u for u < R: the power-of-two exponents come from the table (one
        // gather each), the rest are products of those (at most LR - 1
        // products, so a few rounding units), which keeps the scattered
        // table reads per butterfly at LR instead of R - 1.
        V w[R];
#pragma unroll
        for (int b = 1; b < R; b <<= 1) {
          w[b] = __ldg(stw + 2 * m - m / b + k);
          if (INV) w[b].y = -w[b].y;
        }
#pragma unroll
        for (int u = 3; u < R; ++u) {
          if (u & (u - 1)) {
            const int hb = u >= 8 ? 8 : (u >= 4 ? 4 : 2);
            w[u] = cmul(w[hb], w[u - hb]);
          }
        }
#pragma unroll
        for (int u = 1; u < R; ++u) v[g * R + u] = cmul(v[g * R + u], w[u]);
      }
      dftR<V, R, INV>(v + g * R);
    }
  }
  if (!first || sync_first) __syncthreads();  // everyone has read the previous stage's buffer
  if (active) {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int j = tl + g * P;
      const int k = j & (Ns - 1);
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const int o = (j - k) * R + k + u * Ns;
        if (last) epi_call(epi, o, v[g * R + u], u, (j - k) * R + k, Ns);
        else sm[padix<PADSH>(line * cs + o * is)] = v[g * R + u];
      }
    }
  }
  if (!last) __syncthreads();   // stage output visible
}

// sync_first: the prologue reads the shared buffer itself, so the first
// stage must also wait for every thread's reads before storing.
template <typename V, int E, bool INV, int PADSH, class Pro, class Epi>
__device__ __forceinline__ void fft_reg(V* __restrict__ sm, int logn, bool active, int line, int tl, int cs, int is,
                                        const V* __restrict__ stw, Pro pro, Epi epi, bool sync_first = false) {
  constexpr int LOGE = E == 16 ? 4 : (E == 8 ? 3 : (E == 4 ? 2 : 1));
  V v[E];
  const int r0 = logn % LOGE;
  const int nfull = logn / LOGE;
  int Ns = 1;
  bool first = true;
  if (r0 != 0) {
    const bool last = nfull == 0;
    if (r0 == 1) fft_stage<V, E, 1, INV, PADSH>(v, sm, logn, Ns, true, last, active, line, tl, cs, is, stw, pro, epi, sync_first);
    if constexpr (LOGE > 2) {
      if (r0 == 2) fft_stage<V, E, 2, INV, PADSH>(v, sm, logn, Ns, true, last, active, line, tl, cs, is, stw, pro, epi, sync_first);
    }
    if constexpr (LOGE > 3) {
      if (r0 == 3) fft_stage<V, E, 3, INV, PADSH>(v, sm, logn, Ns, true, last, active, line, tl, cs, is, stw, pro, epi, sync_first);
    }
    Ns <<= r0;
    first = false;
  }
  for (int st = 0; st < nfull; ++st) {
    fft_stage<V, E, LOGE, INV, PADSH>(v, sm, logn, Ns, first, st == nfull - 1, active, line, tl, cs, is, stw, pro, epi,
                                      first && sync_first);
    Ns <<= LOGE;
    first = false;
  }
}

}  // namespace az
