// az_rademacher_noalloc: the Rademacher test matrix without any device
// allocation.  The packed random bits (the scratch between the Philox kernel
// and the expansion to +1/-1) live in a fixed file-scope device array instead
// of a cudaMalloc'd buffer.
#include <mutex>
#include <string>

#include "kernels.cuh"

// 4 MiB of packed bits: k * ceil(N / 32) words at most.  Every GPU that loads
// this library keeps this array until the process exits.
static constexpr int64_t kNoallocWords = int64_t(1) << 20;
static __device__ __align__(256) uint32_t g_noalloc_bits[kNoallocWords];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_bits_addr[kMaxDevices] = {};  // device address of g_noalloc_bits, per device

}  // namespace

using namespace az;

extern "C" az_status az_rademacher_noalloc(int64_t N, int32_t k, uint64_t seed, double* R_dev, void* stream) {
  if (N <= 0 || k <= 0 || !R_dev) { set_error("az_rademacher_noalloc: bad arguments"); return AZ_ERR_ARG; }
  if (k > 65535) {
    // one grid row per column in both kernels (gridDim.y <= 65535)
    set_error("az_rademacher_noalloc: k = " + std::to_string(k) + " exceeds 65535 columns");
    return AZ_ERR_ARG;
  }
  const int64_t words = (int64_t)k * ((N + 31) / 32);
  if (words > kNoallocWords) {
    set_error("az_rademacher_noalloc: k * ceil(N/32) = " + std::to_string(words) + " words exceeds the fixed scratch of " +
              std::to_string(kNoallocWords) + " words (at most 2^25 entries of R)");
    return AZ_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error(std::string("az_rademacher_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return AZ_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) {
    set_error(std::string("az_rademacher_noalloc: cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    return AZ_ERR_CUDA;
  }
  uint32_t* bits = nullptr;
  {
    // The host-side name of the array is not a device address: look the
    // address up with this device current.  Outside stream capture it is
    // looked up on every call (cheap once the module is loaded), so a context
    // destroyed and re-created (cudaDeviceReset) never leaves a stale address;
    // during capture the address of the last uncaptured call on this device
    // is used (a first call that is being captured still looks it up).
    std::lock_guard<std::mutex> g(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_bits_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_bits);
      if (e != cudaSuccess || !p) {
        set_error(std::string("az_rademacher_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return AZ_ERR_CUDA;
      }
      g_bits_addr[dev] = (uint32_t*)p;
    }
    bits = g_bits_addr[dev];
  }
  // The Philox kernel writes every word the expansion reads, so nothing left
  // in the array by an earlier call needs clearing.
  AZ_TRY(launch_philox_bits(bits, N, k, seed, st));
  AZ_TRY(launch_bits_to_R(bits, N, k, R_dev, st));
  return AZ_OK;
}
