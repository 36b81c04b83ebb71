// G = A^T B for tall FP32 operands on the tcgen05 tensor cores (kind::tf32).
//
// Split-K over CTAs: each CTA takes a contiguous range of 32-row blocks of M
// and keeps one accumulator tile in tensor memory.  Per 32-row block:
//   * TMA loads the block of B (kb columns -> MMA rows 0..kb-1) and of A
//     (ka columns -> N rows 0..ka-1) into 128-byte-swizzled K-major tiles;
//   * converter warps split every FP32 value x into hi = x rounded to TF32 and
//     lo = x - hi (exact in FP32), writing hi in place and lo into the second
//     half of the tile: B' = [B_hi; B_lo] (128 MMA rows), A' = [A_hi | A_lo]
//     (2 NB N rows, NB = ka rounded up to 8);
//   * one thread issues four tcgen05.mma (K = 8 each), D += B' A'^T, so D holds
//     B_hi A_hi, B_hi A_lo, B_lo A_hi and B_lo A_lo in four quadrants.
// The sum of the first three quadrants is the product to about 2^-21 relative
// per term (lo is itself rounded to TF32, so the errors take either sign),
// against 2^-11 for plain TF32.  The
// epilogue adds the quadrants in FP64 and writes one partial per CTA; a warp
// per entry then sums the partials in a fixed order.
//
// Every wait on an mbarrier is bounded (1 s of %globaltimer); on timeout the
// CTA raises *err, stops issuing work, waits (bounded) for its own copies and
// MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>

#include "lowrank.cuh"
#include "profile.cuh"
#include "tc_tsgram.cuh"

namespace az {

namespace {

constexpr int TC_THREADS = 256;             // warp 0 TMA, warp 1 MMA (+ TMEM owner), warps 4-7 converters
constexpr int KBLK = 32;                    // rows of M per stage: 128 bytes of FP32, one swizzle span
constexpr int P_BYTES = 128 * 128;          // B' tile: 128 MMA rows x 128 bytes
constexpr int XCH_BYTES = 64 * 64 * 4;      // epilogue exchange of the B_lo rows
constexpr int TMEM_COLS = 128;              // >= 2 NB accumulator columns
constexpr uint64_t WAIT_NS = 1000000000ull; // bound of every wait (a test hook may shorten it)

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity; false after limit_ns or (when abort
// is given) once another role has given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, const volatile int* abort, uint64_t limit_ns) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (abort && *abort) return false;
    if (gtimer() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset 1024; the leading offset is unused when one
// MMA's K extent (32 bytes) lies inside a swizzle row); descriptor version 1.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t a) {
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 32 lanes x 8 columns of FP32 from tensor memory (lane quadrant of this warp)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

// x ~ hi + lo with hi = x rounded to the nearest TF32 (10 stored mantissa
// bits, ties away from zero) and lo = x - hi (exact in FP32, |lo| <= 2^-11 |x|)
// rounded to the nearest TF32 as well: the tensor core would otherwise
// truncate lo's extra bits, an error of one sign that grows linearly over a
// long contraction; rounded, |x - hi - lo| <= 2^-22 |x| with either sign.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
  lo = __uint_as_float((__float_as_uint(lo) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ float4 split4(float4 v, float4& lo) {
  float4 h;
  split_tf32(v.x, h.x, lo.x);
  split_tf32(v.y, h.y, lo.y);
  split_tf32(v.z, h.z, lo.z);
  split_tf32(v.w, h.w, lo.w);
  return h;
}

__device__ __forceinline__ void give_up(int* err, volatile int* abort, int code) {
  atomicExch(err, code);
  *abort = 1;
}

// P = B (np <= 64 columns -> MMA rows), Q = A (nq columns -> N rows, loaded
// in boxes of qbox <= 64 columns: grid row blockIdx.y takes columns
// [blockIdx.y qbox, +qbox) of A).
// partial[(blockIdx.y gridDim.x + blockIdx.x) qstride np + j + i qstride] =
// sum_m Q[m, y0 + j] P[m, i] over this CTA's rows.
// wait_ns bounds every wait; withhold >= 0 (test hook only) makes the TMA
// producer stop issuing at that iteration, so the consumers' waits run out.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_tsgram(const __grid_constant__ CUtensorMap mapP, const __grid_constant__ CUtensorMap mapQ, int np, int nq,
                int NB, int stages, int64_t nkb, double* __restrict__ partial, int* __restrict__ err,
                uint64_t wait_ns, int withhold, int qbox, int qstride) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // tiles start on a 1024-byte boundary of the shared address space (the
  // 128-byte swizzle pattern repeats every 8 rows of 128 bytes)
  const uint32_t s0 = saddr(smem_raw);
  unsigned char* base = smem_raw + (((s0 + 1023u) & ~1023u) - s0);
  const int SB = P_BYTES + 2 * NB * 128;
  float* xch = (float*)(base + stages * SB);
  uint64_t* full = (uint64_t*)(base + stages * SB + XCH_BYTES);
  uint64_t* conv = full + stages;
  uint64_t* empty = conv + stages;
  uint64_t* done = empty + stages;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t kb0 = nkb * blockIdx.x / gridDim.x;
  const int64_t kb1 = nkb * (blockIdx.x + 1) / gridDim.x;
  const int nit = kb1 > kb0 ? (int)(kb1 - kb0) : 0;

  // rows that neither TMA nor the converters write must read as zero
  for (int i = threadIdx.x; i < stages * SB / 16; i += TC_THREADS) ((int4*)base)[i] = make_int4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer
      const uint32_t bytes = (uint32_t)(np + qbox) * 128u;
      int issued = 0;
      for (int it = 0; it < nit; ++it) {
        const int s = it % stages;
        if (it == withhold) break;   // test hook: this stage never arrives
        if (it >= stages && !mbar_wait(&empty[s], ((it / stages) + 1) & 1, abort, wait_ns)) {
          give_up(err, abort, 1);
          break;
        }
        unsigned char* t = base + s * SB;
        mbar_expect_tx(&full[s], bytes);
        const int x = (int)((kb0 + it) * KBLK);
        tma_load_2d(t, &mapP, x, 0, &full[s]);
        tma_load_2d(t + P_BYTES, &mapQ, x, (int)blockIdx.y * qbox, &full[s]);
        issued = it + 1;
      }
      // never leave with copies in flight
      for (int it = issued > stages ? issued - stages : 0; it < issued; ++it)
        if (!mbar_wait(&full[it % stages], (it / stages) & 1, nullptr, wait_ns)) give_up(err, abort, 4);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: D[128 x 2NB] += B'[128 x 32] A'[2NB x 32]^T per stage
      const uint32_t idesc = idesc_tf32(128, 2 * NB);
      for (int it = 0; it < nit; ++it) {
        const int s = it % stages;
        if (!mbar_wait(&conv[s], (it / stages) & 1, abort, wait_ns)) {
          give_up(err, abort, 2);
          break;
        }
        tc_fence_after();
        const uint32_t pa = saddr(base + s * SB), qa = pa + P_BYTES;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma_tf32(tmem, desc_sw128(pa + ks * 32), desc_sw128(qa + ks * 32), idesc, (it | ks) != 0 ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      mma_commit(done);  // arrives once every MMA above has completed
    }
  } else if (warp >= 4) {
    // converters: B rows r < np -> lo at row 64 + r; A rows r < nq -> lo at row NB + r
    const int ct = threadIdx.x - 128;
    const int nP = np * 8, nQ = qbox * 8;  // 16-byte chunks of the loaded rows
    for (int it = 0; it < nit; ++it) {
      const int s = it % stages;
      if (!mbar_wait(&full[s], (it / stages) & 1, abort, wait_ns)) {
        give_up(err, abort, 3);
        break;
      }
      unsigned char* t = base + s * SB;
      for (int c = ct; c < nP + nQ; c += 128) {
        const int off = c < nP ? c * 16 : P_BYTES + (c - nP) * 16;
        const int lo_off = c < nP ? off + 64 * 128 : off + NB * 128;
        float4 lo;
        const float4 hi = split4(*(const float4*)(t + off), lo);
        *(float4*)(t + off) = hi;
        *(float4*)(t + lo_off) = lo;
      }
      fence_async_smem();
      mbar_arrive(&conv[s]);
    }
  }

  // epilogue: warps 0-3 read the accumulator lanes 32w .. 32w+31
  __syncwarp();
  bool have = false;
  if (warp < 4) {
    const bool ok = nit > 0 && mbar_wait(done, 0, nullptr, wait_ns) && !*abort;
    have = __all_sync(0xffffffffu, ok);
    tc_fence_after();
  }
  const int row = warp * 32 + lane;  // MMA row (warps 0-3)
  if (warp >= 2 && warp < 4 && have) {
    const int i = row - 64;
    for (int j0 = 0; j0 < NB; j0 += 8) {
      float a[8], b[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + j0, a);
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + NB + j0, b);
#pragma unroll
      for (int q = 0; q < 8; ++q) xch[i * 64 + j0 + q] = a[q] + b[q];
    }
  }
  __syncthreads();
  if (warp < 2) {
    double* out = partial + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * qstride * np;
    const int nqe = min(nq - (int)blockIdx.y * qbox, qbox);   // columns of A in this box
    if (have) {
      for (int j0 = 0; j0 < NB; j0 += 8) {
        float a[8], b[8];
        tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + j0, a);
        tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + NB + j0, b);
        if (row < np) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = j0 + q;
            if (j < nqe) out[j + row * qstride] = (double)a[q] + (double)b[q] + (double)xch[row * 64 + j];
          }
        }
      }
    } else if (row < np) {
      for (int j = 0; j < nqe; ++j) out[j + row * qstride] = 0.0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// 2D map over a column-major M x ncols FP32 matrix: 32-row x boxcols boxes,
// 128-byte swizzle (the tcgen05 K-major layout), zero fill past row M.
bool make_map(CUtensorMap* m, const float* p, int64_t M, int64_t ld, int ncols, int boxcols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)ncols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)KBLK, (cuuint32_t)boxcols};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int sm_count() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = 1;
  }
  cache[dev] = n;
  return n;
}

size_t smem_bytes(int NB, int* stages_out) {
  const int SB = P_BYTES + 2 * NB * 128;
  const int budget = 200 * 1024 - XCH_BYTES;
  const int stages = std::max(2, std::min(8, budget / SB));
  *stages_out = stages;
  return 1024 + (size_t)stages * SB + XCH_BYTES + (3 * stages + 1) * 8 + 16;
}


// ---------------------------------------------------------------- exact Gram on BF16 slices
// G = Y^T Y for FP32 Y (M x k, k <= OZ_KMAX) on the tensor cores, to FP64
// accuracy, with an exact split in the manner of Ozaki et al.: every column a
// is scaled by 2^-E_a into [-1/2, 1/2) (E_a from the largest magnitude of the
// column in the CTA's rows, a first pass), and each scaled value is cut into six slices
// s_i = t_i 2^(-8i), |t_i| <= 128 an integer (so s_i is exact in BF16),
// covering 48 bits below the column's scale.  The product of two slices is an
// integer multiple of 2^(-8(i+j)) below 2^14 in units; a CTA sums at most
// OZ_ROWS = 1024 rows, so every per-CTA sum of one slice pair is an integer
// below 2^24 units, exact in the FP32 accumulator whatever the order.  The
// operand holds rows (i, a) = slice i of column a, i < 6, in one K-major
// 128-byte-swizzled tile per 64 rows of Y; A = its first 128 rows (slices
// 1-5 when 5k <= 128), B = all 6k rows, D = A B^T in tensor memory.  The
// missing pair (6, 6) weighs 2^-80 of the column scales.  The epilogue folds
// the 35 slice pairs of each entry in FP64 and scales by 2^(E_a + E_b).
constexpr int OZ_KMAX = 24;         // 6 k <= 144 B rows, 5 k <= 128 A rows
constexpr int OZ_ROWS = 1024;       // rows per CTA (exactness bound above)
constexpr int OZ_SLICES = 6;
constexpr int OZ_STAGE_ROWS = 64;   // rows of Y per operand tile (128 bytes of BF16)
constexpr int OZ_NB = 4;            // operand tiles in flight
constexpr int OZ_TILE_BYTES = 144 * 128;
constexpr int OZ_THREADS = 256;     // warp 0: MMA + TMEM owner; warps 1-7 convert
constexpr int OZ_TMEM_COLS = 256;
constexpr int OZ_DST = 145;         // row stride of D in shared memory (odd: no bank conflicts)
constexpr int OZ_AREA = 75776;      // >= max(tiles, 128 x OZ_DST floats), a multiple of 1024

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// E with max|y| < 2^(E-1) (clamped to the range where 2^-E is a normal float)
__device__ __forceinline__ int oz_exp(unsigned mbits) {
  const int eb = (int)(mbits >> 23);
  const int E = mbits == 0 ? 0 : (eb == 0 ? -125 : eb - 125);
  return min(max(E, -126), 126);
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_tc_gram_oz(const float* __restrict__ Y, int64_t ldy, int k, int64_t M, double* __restrict__ partial,
                 int* __restrict__ err, uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t s0 = saddr(smem_raw);
  unsigned char* base = smem_raw + (((s0 + 1023u) & ~1023u) - s0);
  static_assert(OZ_NB * OZ_TILE_BYTES <= OZ_AREA && 128 * OZ_DST * 4 <= OZ_AREA, "shared-memory area");
  uint64_t* full = (uint64_t*)(base + OZ_AREA);
  uint64_t* empty = full + OZ_NB;
  uint64_t* done = empty + OZ_NB;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  int* Es = (int*)(tmem_slot + 2);    // OZ_KMAX column exponents
  float* Dsm = (float*)base;          // 128 x OZ_DST FP32 after the contraction (aliases the tiles)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * OZ_ROWS;
  const int64_t r1 = min(M, r0 + OZ_ROWS);
  const int nst = (int)((r1 - r0 + OZ_STAGE_ROWS - 1) / OZ_STAGE_ROWS);
  const int NB_ = 6 * k;                 // B rows (MMA N)
  const int Nmma = (NB_ + 15) / 16 * 16;

  // rows of the tiles that no converter writes stay zero
  for (int i = threadIdx.x; i < OZ_NB * OZ_TILE_BYTES / 16; i += OZ_THREADS) ((int4*)base)[i] = make_int4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_NB; ++s) {
      mbar_init(&full[s], 7);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, Nmma);
      for (int st = 0; st < nst; ++st) {
        const int b = st % OZ_NB;
        if (!mbar_wait(&full[b], (st / OZ_NB) & 1, abort, wait_ns)) {
          give_up(err, abort, 12);
          break;
        }
        tc_fence_after();
        const uint32_t ta = saddr(base + b * OZ_TILE_BYTES);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          mma_bf16(tmem, desc_sw128(ta + ks * 32), desc_sw128(ta + ks * 32), idesc, (st | ks) != 0 ? 1u : 0u);
        mma_commit(&empty[b]);
      }
      mma_commit(done);
    }
  } else {
    // converters: task (column a, 8-row group g) of each 64-row tile
    const int ct = threadIdx.x - 32;
    const bool has = ct < k * 8;
    const int a = ct >> 3, g = ct & 7;
    const float* src0 = Y + (int64_t)(has ? a : 0) * ldy + r0 + 8 * g;
    auto load8 = [&](int st, float (&v)[8]) {
      const int64_t rb = r0 + (int64_t)st * OZ_STAGE_ROWS + 8 * g;
      const float* src = src0 + (int64_t)st * OZ_STAGE_ROWS;
      if (!has || st >= nst) {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0.f;
      } else if (rb + 8 <= r1) {
        const float4 p = *(const float4*)src, q = *(const float4*)(src + 4);
        v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w; v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = rb + u < r1 ? src[u] : 0.f;
      }
    };
    // pass 1: this CTA's largest magnitude of column a (its 8 row groups are
    // 8 consecutive lanes), all loads in flight; the scale 2^E_a is this CTA's
    unsigned mb = 0;
#pragma unroll 4
    for (int st = 0; st < nst; ++st) {
      float v[8];
      load8(st, v);
#pragma unroll
      for (int u = 0; u < 8; ++u) mb = max(mb, __float_as_uint(v[u]) & 0x7fffffffu);
    }
    mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 1));
    mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 2));
    mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 4));
    const int E = oz_exp(mb);
    if (has && g == 0) Es[a] = E;
    const float sc = __uint_as_float((unsigned)(127 - E) << 23);   // 2^-E
    // pass 2: slices, with the next two tiles' loads in flight
    float v0[8], v1[8], v2[8];
    load8(0, v0);
    load8(1, v1);
    for (int st = 0; st < nst; ++st) {
      const int b = st % OZ_NB;
      load8(st + 2, v2);
      if (st >= OZ_NB && !mbar_wait(&empty[b], ((st / OZ_NB) + 1) & 1, abort, wait_ns)) {
        give_up(err, abort, 13);
        break;
      }
      if (has) {
        unsigned char* tile = base + b * OZ_TILE_BYTES;
        float r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r[u] = v0[u] * sc;   // exact: a power-of-two scaling
#pragma unroll
        for (int i = 0; i < OZ_SLICES; ++i) {
          const float up = __uint_as_float((unsigned)(127 + 8 * (i + 1)) << 23), dn = __uint_as_float((unsigned)(127 - 8 * (i + 1)) << 23);
          uint32_t w[4];
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            const float s0v = rintf(r[u] * up) * dn, s1v = rintf(r[u + 1] * up) * dn;   // exact slices
            r[u] -= s0v;
            r[u + 1] -= s1v;
            const __nv_bfloat162 h = __floats2bfloat162_rn(s0v, s1v);
            w[u >> 1] = *(const uint32_t*)&h;
          }
          // row (i, a), 16-byte chunk g of its 128 bytes, 128-byte swizzle
          const int row = i * k + a;
          *(uint4*)(tile + row * 128 + ((g ^ (row & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[b]);
#pragma unroll
      for (int u = 0; u < 8; ++u) { v0[u] = v1[u]; v1[u] = v2[u]; }
    }
  }

  // epilogue: D (128 lanes x Nmma columns) to shared memory, then the fold
  __syncwarp();
  bool ok = true;
  if (warp < 4) {
    ok = nst > 0 && mbar_wait(done, 0, nullptr, wait_ns) && !*abort;
    tc_fence_after();
  }
  __syncthreads();   // every converter is past its last tile; the tiles are free
  __shared__ int all_ok;
  if (threadIdx.x == 0) all_ok = 1;
  __syncthreads();
  if (warp < 4 && !ok) all_ok = 0;
  __syncthreads();
  const bool have = all_ok != 0;
  if (warp < 4 && have) {
    const int row = warp * 32 + lane;
    for (int j0 = 0; j0 < Nmma; j0 += 8) {
      float d[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + j0, d);
#pragma unroll
      for (int q = 0; q < 8; ++q) Dsm[row * OZ_DST + j0 + q] = d[q];
    }
  }
  __syncthreads();
  double* out = partial + (int64_t)blockIdx.x * k * k;
  for (int e = threadIdx.x; e < k * k; e += OZ_THREADS) {
    const int a = e % k, b2 = e / k;
    if (a > b2) continue;
    double s = 0.0;
    if (have) {
      // pairs (i, j) by increasing weight 2^-8(i+j): i < 5 from the A rows,
      // (5, j < 5) from the transposed entry D[(j, b), (5, a)]; summed in
      // double-float on the FP32 pipe (each term is exact), widened once
      float hi = 0.f, lo = 0.f;
      for (int w2 = 0; w2 <= 9; ++w2)
        for (int i = 0; i < OZ_SLICES; ++i) {
          const int j = w2 - i;
          if (j < 0 || j >= OZ_SLICES || (i == 5 && j == 5)) continue;
          const float t = i < 5 ? Dsm[(i * k + a) * OZ_DST + j * k + b2] : Dsm[(j * k + b2) * OZ_DST + 5 * k + a];
          const float u = hi + t, bv = u - hi;
          lo += (hi - (u - bv)) + (t - bv);
          hi = u;
        }
      s = ldexp(f2d_int(hi) + f2d_int(lo), Es[a] + Es[b2]);
    }
    out[a + (int64_t)b2 * k] = s;
    out[b2 + (int64_t)a * k] = s;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

}  // namespace

// The kernel's dynamic shared-memory limit, shared by both launchers and
// only ever raised (a lower value would break a launch that relies on an
// earlier, larger setting).
static az_status ensure_smem(size_t sm) {
  static std::mutex mu;
  static size_t set_bytes = 0;
  std::lock_guard<std::mutex> g(mu);
  if (sm > set_bytes) {
    AZ_CUDA(cudaFuncSetAttribute(k_tc_tsgram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    set_bytes = sm;
  }
  return AZ_OK;
}

// test hook (az_debug_tc_withhold): one-shot, read by the next launch
static std::mutex g_hook_mu;
static int g_hook_withhold = -1;
static uint64_t g_hook_wait_ns = WAIT_NS;

void tc_tsgram_debug_withhold(int iteration, uint64_t wait_ns) {
  std::lock_guard<std::mutex> g(g_hook_mu);
  g_hook_withhold = iteration;
  g_hook_wait_ns = wait_ns;
}

int tc_tsgram_blocks() { return sm_count(); }

bool tc_tsgram_ok(const void* A, int64_t lda, int ka, const void* B, int64_t ldb, int kb) {
  return ka >= 1 && ka <= 64 && kb >= 1 && kb <= 64 && lda % 4 == 0 && ldb % 4 == 0 &&
         ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0 && encode_fn() != nullptr;
}

az_status launch_tc_tsgram(const float* A, int64_t lda, int ka, const float* B, int64_t ldb, int kb, int64_t M,
                           double* partial, double* G, int* err, cudaStream_t st) {
  if (!tc_tsgram_ok(A, lda, ka, B, ldb, kb) || M < 1) {
    set_error("tensor-core tall product: unsupported shape or alignment");
    return AZ_ERR_ARG;
  }
  ProfScope ps("proj_tc", (double)M * (ka + kb) * 4.0, st);
  CUtensorMap mP, mQ;
  if (!make_map(&mP, B, M, ldb, kb, kb) || !make_map(&mQ, A, M, lda, ka, ka)) {
    set_error("tensor-core tall product: cuTensorMapEncodeTiled failed");
    return AZ_ERR_CUDA;
  }
  const int NB = (ka + 7) / 8 * 8;
  int stages = 0;
  const size_t sm = smem_bytes(NB, &stages);
  const int64_t nkb = (M + KBLK - 1) / KBLK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nkb, tc_tsgram_blocks()));
  AZ_TRY(ensure_smem(sm));
  uint64_t wait_ns = WAIT_NS;
  int withhold = -1;
  {
    std::lock_guard<std::mutex> g(g_hook_mu);
    if (g_hook_withhold >= 0) {
      withhold = g_hook_withhold;
      wait_ns = g_hook_wait_ns;
      g_hook_withhold = -1;
    }
  }
  k_tc_tsgram<<<grid, TC_THREADS, sm, st>>>(mP, mQ, kb, ka, NB, stages, nkb, partial, err, wait_ns, withhold, ka, ka);
  {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("tensor-core tall product launch: ") + cudaGetErrorString(e));
      return AZ_ERR_CUDA;
    }
  }
  return launch_gram_reduce(partial, grid, ka, kb, G, st);
}

// ---------------------------------------------------------------- wide A (ka > 64)
namespace {

// CTAs per 64-column chunk of A: about two waves over the SMs in total
int wide_splits(int64_t M, int ka) {
  const int64_t chunks = (ka + 63) / 64;
  const int64_t nkb = (M + KBLK - 1) / KBLK;
  const int64_t want = (2 * (int64_t)tc_tsgram_blocks() + chunks - 1) / chunks;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, nkb));
}

// G[(64 c + j) + i ka] = sum over the chunk's CTAs x of partial[(c gx + x) 64 kb + j + 64 i]
__global__ void k_tc_wide_reduce(const double* __restrict__ partial, int gx, int ka, int kb, double* __restrict__ G) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ka * kb) return;
  const int r = (int)(t % ka), i = (int)(t / ka);
  const int c = r / 64, j = r % 64;
  const double* p = partial + ((int64_t)c * gx) * 64 * kb + j + 64 * i;
  double s = 0.0;
  for (int x = 0; x < gx; ++x) s += p[(int64_t)x * 64 * kb];
  G[t] = s;
}

}  // namespace

bool tc_tsgram_wide_ok(const void* A, int64_t lda, int ka, const void* B, int64_t ldb, int kb) {
  return ka >= 1 && kb >= 1 && kb <= 64 && lda % 4 == 0 && ldb % 4 == 0 && ((uintptr_t)A & 15) == 0 &&
         ((uintptr_t)B & 15) == 0 && encode_fn() != nullptr;
}

size_t tc_tsgram_wide_partial(int64_t M, int ka, int kb) {
  return (size_t)wide_splits(M, ka) * (size_t)((ka + 63) / 64) * 64 * (size_t)kb;
}

az_status launch_tc_tsgram_wide(const float* A, int64_t lda, int ka, const float* B, int64_t ldb, int kb, int64_t M,
                                double* partial, double* G, int* err, cudaStream_t st) {
  if (!tc_tsgram_wide_ok(A, lda, ka, B, ldb, kb) || M < 1) {
    set_error("tensor-core wide product: unsupported shape or alignment");
    return AZ_ERR_ARG;
  }
  ProfScope ps("proj_tc_wide", (double)M * (ka + kb) * 4.0, st);
  CUtensorMap mP, mQ;
  if (!make_map(&mP, B, M, ldb, kb, kb) || !make_map(&mQ, A, M, lda, ka, 64)) {
    set_error("tensor-core wide product: cuTensorMapEncodeTiled failed");
    return AZ_ERR_CUDA;
  }
  const int NB = 64;
  int stages = 0;
  const size_t sm = smem_bytes(NB, &stages);
  const int64_t nkb = (M + KBLK - 1) / KBLK;
  const int gx = wide_splits(M, ka);
  const int chunks = (ka + 63) / 64;
  AZ_TRY(ensure_smem(sm));
  uint64_t wait_ns = WAIT_NS;
  int withhold = -1;
  {
    std::lock_guard<std::mutex> g(g_hook_mu);
    if (g_hook_withhold >= 0) {
      withhold = g_hook_withhold;
      wait_ns = g_hook_wait_ns;
      g_hook_withhold = -1;
    }
  }
  k_tc_tsgram<<<dim3(gx, chunks), TC_THREADS, sm, st>>>(mP, mQ, kb, ka, NB, stages, nkb, partial, err, wait_ns,
                                                        withhold, 64, 64);
  {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("tensor-core wide product launch: ") + cudaGetErrorString(e));
      return AZ_ERR_CUDA;
    }
  }
  const int64_t n = (int64_t)ka * kb;
  k_tc_wide_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(partial, gx, ka, kb, G);
  AZ_CUDA(cudaGetLastError());
  return AZ_OK;
}


// ---------------------------------------------------------------- exact Gram launcher
bool tc_gram_oz_ok(const void* Y, int64_t ldy, int k, int64_t M) {
  return k >= 1 && k <= OZ_KMAX && M >= 1 && ldy % 4 == 0 && ((uintptr_t)Y & 15) == 0 && encode_fn() != nullptr;
}

int tc_gram_oz_blocks(int64_t M) { return (int)((M + OZ_ROWS - 1) / OZ_ROWS); }

az_status launch_tc_gram_oz(const float* Y, int64_t ldy, int k, int64_t M, double* partial, double* G, int* err,
                            cudaStream_t st) {
  if (!tc_gram_oz_ok(Y, ldy, k, M) || !partial || !G || !err) {
    set_error("tensor-core exact Gram: unsupported shape or alignment");
    return AZ_ERR_ARG;
  }
  ProfScope ps("gram_oz", (double)M * k * 4.0, st, 2);
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  const size_t sm = 1024 + (size_t)OZ_AREA + (2 * OZ_NB + 1) * 8 + 8 + OZ_KMAX * 4 + 64;
  std::call_once(once, [&] {
    attr_rc = cudaFuncSetAttribute(k_tc_gram_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  AZ_CUDA(attr_rc);
  const int nblk = tc_gram_oz_blocks(M);
  k_tc_gram_oz<<<nblk, OZ_THREADS, sm, st>>>(Y, ldy, k, M, partial, err, WAIT_NS);
  {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("tensor-core exact Gram launch: ") + cudaGetErrorString(e));
      return AZ_ERR_CUDA;
    }
  }
  return launch_gram_reduce(partial, nblk, k, k, G, st);
}

}  // namespace az
