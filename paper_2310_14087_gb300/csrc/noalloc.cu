// Allocation-free entry point: the embedding-norm pair sum ||w||^2 = (1/n^2) sum_ij k(s_i, s_j)
// with its per-tile partial sums kept in a fixed device array instead of memory from cudaMalloc.
//
// Who needs it: code that may not allocate device memory at the time it runs, e.g. a caller
// inside a framework's custom memory allocator or pool (where a nested cudaMalloc would
// re-enter or fragment it), a memory-capped serving process that reserved all device memory up
// front, or a plugin whose host forbids driver allocations after start-up.  Such a caller owns
// its inputs and output; this entry point adds no allocation of its own.
#include <cmath>
#include <mutex>

#include "kot_internal.cuh"

namespace {

// 64 x 64-sample tiles: (n / 64)^2 partial sums, so n <= 4096 samples fit.
constexpr int kMaxTiles = 4096;
__device__ __align__(256) double g_pair_partials[kMaxTiles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {};

// Device address of g_pair_partials on the current device, looked up once per device (the name
// itself is only a host-side stand-in in host code).  The address is that of the device's
// primary context at the first call; a cudaDeviceReset invalidates it (see kot.h).
kot_status partials_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return KOT_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return KOT_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pair_partials);
    if (e != cudaSuccess || !p) return KOT_ERR_CUDA;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return KOT_OK;
}

}  // namespace

extern "C" kot_status kot_embedding_sqnorm_noalloc(int n, int d, const double* S, double sigma,
                                                   double* out, void* stream) {
  if (n < 1 || d < 1 || !S || !out || !std::isfinite(sigma) || !(sigma > 0.0))
    return KOT_ERR_INVALID;
  if (kot::pair_blocks(n) > kMaxTiles) return KOT_ERR_TOO_LARGE;
  double* partials = nullptr;
  kot_status s = partials_on_current_device(&partials);
  if (s != KOT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  try {
    // every tile slot that the sum reads is rewritten by this call, so nothing is cleared
    kot::pair_mean_f64(st, n, d, S, 1.0 / (2.0 * sigma * sigma), out, partials, kMaxTiles);
  } catch (const kot::Error& e) {
    return e.status;
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? KOT_OK : KOT_ERR_CUDA;
}
