// The Z* chain of a 2D sketch (W = R - Z* v, or z = Z* v) fused into one
// cluster-resident kernel: Sec. 5.1, the tensor-product periodic solver
// (Eq. B_pinv_2d) applied to the extended data, Z* y = IDFT_N(sum over the
// alias group of Ghat DFT_L(E y) / S) (Sec. 3.2.2).
//
// One cluster of CL = 16 CTAs takes one pair of columns (two real columns in
// one complex FP64 array) of a square L x L grid (L = 2^LOGL <= 256, s = 2).
// CTA c holds 1/CL of the grid in shared memory, so the whole chain runs
// without an HBM round trip:
//   A  v on its L/CL x-rows (gathered from the compact input), y-FFT per row;
//   B  x-FFT of its L/CL y-columns, inputs read from the other CTAs' shared
//      memory (distributed shared memory) into registers first;
//   C  (CTAs holding ky < L/2) alias fold with H = Ghat / S over the four
//      members (kx + qx N1, ky + qy N1), the qy = 1 members read from the
//      partner CTA c + CL/2;
//   D  inverse x-FFT of length N1 = L/2 on the folded columns;
//   E  inverse y-FFT of length N1 on L/2/CL rows per CTA, inputs read from the
//      CTAs of phase D, and W = R - z / N (or z / N) written to global memory.
// Between phases the CTAs meet at cluster barriers built from mbarriers: each
// CTA arrives on every CTA's barrier (remote arrive, release at cluster
// scope) and waits on its own with a bounded try_wait (1 s of %globaltimer);
// a wait that runs out records its phase in *err (the host reports
// AZ_ERR_TIMEOUT) and the CTA skips its remaining work.  The only unbounded
// wait is the hardware cluster barrier that publishes the mbarrier
// initialisation at the start (the CTAs of a cluster are co-scheduled).
// FP64 throughout (the 2D sketch runs in FP64, see the 2D mixed path).
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "cluster_sketch.cuh"
#include "fft_reg.cuh"
#include "profile.cuh"

namespace cg = cooperative_groups;

namespace az {

namespace {

constexpr int CL = 16;                     // CTAs per cluster
constexpr int PADS = 4;                    // shared-memory padding: one element every 16
constexpr int TWN = 4096;                  // length of the master twiddle table
constexpr uint64_t CWAIT_NS = 1000000000ull;

using V = double2;

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gclock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded cluster barrier on the CTAs' own mbarriers (count CL each): the
// calling CTA's thread 0 arrives (release, cluster scope) on every CTA's
// barrier, then every thread waits (acquire, cluster scope) for the phase of
// this episode on its own.  false: the wait ran out (or an earlier one did).
__device__ bool cluster_sync_bounded(uint64_t* bar, int episode, volatile int* failed, int* err, int code) {
  __syncthreads();
  if (threadIdx.x == 0 && !*failed) {
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    const uint32_t local = s_addr(bar);
    for (int r = 0; r < CL; ++r) {
      uint32_t remote;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
      asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
    }
  }
  bool ok = !*failed;
  if (ok) {
    const uint32_t a = s_addr(bar), parity = (uint32_t)(episode & 1);
    const uint64_t t0 = gclock();
    while (true) {
      uint32_t done;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(a), "r"(parity)
          : "memory");
      if (done) break;
      if (gclock() - t0 > CWAIT_NS) { ok = false; break; }
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(err, code);
    *failed = 1;
  }
  __syncthreads();
  return !*failed;
}

// The register FFT's first stage reads inputs p = tl + g P + u nbf (g < E/R0,
// u < R0, R0 the radix of that stage); Pre holds them in that order.
template <int LOGN>
struct FirstStage {
  static constexpr int R0 = (LOGN % 3) == 0 ? 8 : (1 << (LOGN % 3));
  static constexpr int NG = 8 / R0;
  static constexpr int P = (1 << LOGN) / 8;
  static constexpr int NBF = (1 << LOGN) / R0;
  __device__ static int pos(int tl, int g, int u) { return tl + g * P + u * NBF; }
};

template <int LOGL>
__global__ void __launch_bounds__((1 << (2 * LOGL)) / 128)
    k_zstar_cluster(const double* __restrict__ vin, int64_t ldv, int ncols, const int32_t* __restrict__ pos2m,
                    const double* __restrict__ H, const uint32_t* __restrict__ bits, int64_t nw, double* __restrict__ out,
                    int64_t ldo, const V* __restrict__ tw, int pair0, int* __restrict__ err) {
  constexpr int L = 1 << LOGL, N1 = L / 2, LOGN1 = LOGL - 1;
  constexpr int RX = L / CL;                 // x-rows per CTA (phase A), y-columns per CTA (phases B-D)
  constexpr int NT = L * L / 128;            // threads
  constexpr int RE = N1 / CL;                // N-grid rows per CTA (phase E)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = (V*)smem_raw;                                         // padix(L * L / CL) elements
  uint64_t* cbar = (uint64_t*)(smem_raw + (size_t)padix<PADS>(L * RX) * sizeof(V));
  volatile int* failed = (volatile int*)(cbar + 1);

  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const int pair = pair0 + (int)(blockIdx.x / CL);
  const int colA = 2 * pair, colB = 2 * pair + 1;
  const bool hasB = colB < ncols;
  const int tid = threadIdx.x;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(cbar)), "r"(CL) : "memory");
    *failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // publish the initialisation before any remote arrive (the one hardware
  // cluster barrier; the cluster's CTAs are co-scheduled)
  cluster.sync();
  int ep = 0;

  // ---- A: gather v on the x-rows [c RX, c RX + RX), y-FFT of each row (natural ky)
  {
    constexpr int P = L / 8;
    const int line = tid / P, tl = tid % P;
    const int x = c * RX + line;
    const double* va = vin + (int64_t)colA * ldv;
    const double* vb = vin + (int64_t)(hasB ? colB : colA) * ldv;
    auto pro = [&](int p) -> V {
      const int m = __ldg(pos2m + x * L + p);
      const int mc = m < 0 ? 0 : m;
      const double a = va[mc], b = vb[mc];
      V v;
      v.x = m < 0 ? 0.0 : a;
      v.y = (m < 0 || !hasB) ? 0.0 : b;
      return v;
    };
    auto epi = [&](int o, V v) { buf[padix<PADS>(line * L + o)] = v; };
    fft_reg<V, 8, false, PADS>(buf, LOGL, true, line, tl, L, 1, tw + TWN, pro, epi);
  }
  if (!cluster_sync_bounded(cbar, ep++, failed, err, 11)) return;

  // ---- B: x-FFT of the y-columns [c RX, c RX + RX); inputs from the row owners
  {
    using FS = FirstStage<LOGL>;
    constexpr int P = L / 8;
    const int line = tid / P, tl = tid % P;
    const int ky = c * RX + line;
    V pre[8];
#pragma unroll
    for (int g = 0; g < FS::NG; ++g)
#pragma unroll
      for (int u = 0; u < FS::R0; ++u) {
        const int x = FS::pos(tl, g, u);
        const V* rb = cluster.map_shared_rank(buf, x / RX);
        pre[g * FS::R0 + u] = rb[padix<PADS>((x % RX) * L + ky)];
      }
    // every CTA has read what it needs from the others' row data
    if (!cluster_sync_bounded(cbar, ep++, failed, err, 12)) return;
    auto pro = [&](int p, int g, int u) -> V { return pre[g * FS::R0 + u]; };
    auto epi = [&](int o, V v) { buf[padix<PADS>(line * L + o)] = v; };   // [ky local][kx]
    fft_reg<V, 8, false, PADS>(buf, LOGL, true, line, tl, L, 1, tw + TWN, pro, epi);
  }
  if (!cluster_sync_bounded(cbar, ep++, failed, err, 13)) return;

  // ---- C, D: the CTAs holding ky < N1 fold the alias group and run the inverse x-FFT
  if (c < CL / 2) {
    const V* partner = cluster.map_shared_rank(buf, c + CL / 2);
    for (int t = tid; t < RX * N1; t += NT) {
      const int jl = t / N1, jx = t % N1;           // column jy = c RX + jl
      const int jy = c * RX + jl;
      double ar = 0.0, ai = 0.0;
#pragma unroll
      for (int qy = 0; qy < 2; ++qy) {
        const V* src = qy == 0 ? buf : partner;
        const int ky = jy + qy * N1;
#pragma unroll
        for (int qx = 0; qx < 2; ++qx) {
          const int kx = jx + qx * N1;
          const double h = __ldg(H + (int64_t)kx * L + ky);
          const V v = src[padix<PADS>(jl * L + kx)];
          ar = fma(h, v.x, ar);
          ai = fma(h, v.y, ai);
        }
      }
      V o;
      o.x = ar;
      o.y = ai;
      buf[padix<PADS>(jl * L + jx)] = o;             // read above by this thread only
    }
    __syncthreads();
    constexpr int P = N1 / 8;
    const int line = tid / P, tl = tid % P;
    const bool act = line < RX;
    auto pro = [&](int p) -> V { return buf[padix<PADS>(line * L + p)]; };
    auto epi = [&](int o, V v) { buf[padix<PADS>(line * L + o)] = v; };   // [jy local][nx]
    fft_reg<V, 8, true, PADS>(buf, LOGN1, act, act ? line : 0, tl, L, 1, tw + TWN, pro, epi, true);
  }
  if (!cluster_sync_bounded(cbar, ep++, failed, err, 14)) return;

  // ---- E: inverse y-FFT of the N-grid rows [c RE, c RE + RE); output W = R - z / N
  {
    using FS = FirstStage<LOGN1>;
    constexpr int P = N1 / 8;
    const int line = tid / P, tl = tid % P;
    const bool act = line < RE;
    const int nxr = c * RE + (act ? line : 0);
    V pre[8];
#pragma unroll
    for (int g = 0; g < FS::NG; ++g)
#pragma unroll
      for (int u = 0; u < FS::R0; ++u) {
        const int jy = FS::pos(tl, g, u);
        V v;
        v.x = 0.0;
        v.y = 0.0;
        if (act) {
          const V* rb = cluster.map_shared_rank(buf, jy / RX);
          v = rb[padix<PADS>((jy % RX) * L + nxr)];
        }
        pre[g * FS::R0 + u] = v;
      }
    if (!cluster_sync_bounded(cbar, ep++, failed, err, 15)) return;
    const double sc = 1.0 / ((double)N1 * (double)N1);
    double* oA = out + (int64_t)colA * ldo;
    double* oB = out + (int64_t)colB * ldo;
    auto pro = [&](int p, int g, int u) -> V { return pre[g * FS::R0 + u]; };
    auto epi = [&](int ny, V v) {
      if (!act) return;
      const int j = nxr * N1 + ny;
      double za = v.x * sc, zb = v.y * sc;
      if (bits) {
        za = (double)rad_bit(bits, nw, j, colA) - za;
        if (hasB) zb = (double)rad_bit(bits, nw, j, colB) - zb;
      }
      oA[j] = za;
      if (hasB) oB[j] = zb;
    };
    fft_reg<V, 8, true, PADS>(buf, LOGN1, act, act ? line : 0, tl, N1, 1, tw + TWN, pro, epi);
  }
}

}  // namespace

namespace {

size_t smem_of(int logl) {
  const int L = 1 << logl, RX = L / CL;
  const size_t e = (size_t)L * RX;
  return (e + (e >> PADS)) * sizeof(V) + 16;
}

template <int LOGL>
void* kernel_of() { return (void*)k_zstar_cluster<LOGL>; }

// 16-CTA clusters with this kernel's shared memory fit on the device: set the
// function attributes once and ask the occupancy calculator.
template <int LOGL>
bool prepare(cudaStream_t st) {
  static std::mutex mu;
  static int state[3] = {0, 0, 0};   // per device ordinal is not needed: one GPU per process
  std::lock_guard<std::mutex> g(mu);
  int& s = state[LOGL - 6];
  if (s != 0) return s > 0;
  auto kern = k_zstar_cluster<LOGL>;
  const size_t sm = smem_of(LOGL);
  bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3((1u << (2 * LOGL)) / 128, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    ok = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0;
  }
  if (!ok) cudaGetLastError();
  s = ok ? 1 : -1;
  return ok;
}

}  // namespace

bool zstar_cluster_ok(const Geom& g, cudaStream_t st) {
  if (g.dim != 2 || g.s[0] != 2 || g.s[1] != 2 || g.Ld[0] != g.Ld[1]) return false;
  switch (g.Ld[0]) {
    case 64: return prepare<6>(st);
    case 128: return prepare<7>(st);
    case 256: return prepare<8>(st);
    default: return false;
  }
}

template <int LOGL>
static az_status launch_t(const double* v, int64_t ldv, int ncols, const int32_t* pos2m, const double* H,
                          const uint32_t* bits, int64_t nw, double* out, int64_t ldo, const double2* tw, int pair0,
                          int npairs, int* err, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(CL * npairs), 1, 1);
  cfg.blockDim = dim3((1u << (2 * LOGL)) / 128, 1, 1);
  cfg.dynamicSmemBytes = smem_of(LOGL);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AZ_CUDA(cudaLaunchKernelEx(&cfg, k_zstar_cluster<LOGL>, v, ldv, ncols, pos2m, H, bits, nw, out, ldo, tw, pair0, err));
  return AZ_OK;
}

az_status launch_zstar_cluster(const Geom& g, const double* v, int64_t ldv, int ncols, const int32_t* pos2m,
                               const double* H, const uint32_t* bits, int64_t nw, double* out, int64_t ldo,
                               const double2* tw, int pair0, int npairs, int* err, cudaStream_t st) {
  if (!zstar_cluster_ok(g, st) || npairs < 1) { set_error("cluster Z* chain: unsupported grid"); return AZ_ERR_ARG; }
  const double L = (double)g.L, N = (double)g.N;
  // algorithmic bytes: the compact input read once, the index map, H, the output
  ProfScope ps("zstar_cluster_f64", npairs * (2.0 * 8.0 * L / 2 + 2.0 * 8.0 * N) + 4.0 * L + 8.0 * L, st);
  switch (g.Ld[0]) {
    case 64: return launch_t<6>(v, ldv, ncols, pos2m, H, bits, nw, out, ldo, tw, pair0, npairs, err, st);
    case 128: return launch_t<7>(v, ldv, ncols, pos2m, H, bits, nw, out, ldo, tw, pair0, npairs, err, st);
    default: return launch_t<8>(v, ldv, ncols, pos2m, H, bits, nw, out, ldo, tw, pair0, npairs, err, st);
  }
}

}  // namespace az
