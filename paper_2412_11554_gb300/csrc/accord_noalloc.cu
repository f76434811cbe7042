// accord_loss_f64_noalloc: the FP64 objective evaluation of accord_loss for
// callers that must not allocate device memory -- for example code running
// inside a custom allocator's callback, a latency-bound loop where the
// allocator's implicit synchronisation is not acceptable, or a process whose
// device memory is already fully reserved by another caching allocator.
//
// Its only scratch (per-tile partial sums of ||Omega X^T||^2 and per-row
// statistics of Omega) lives in the file-scope array below, which every GPU
// that loads the library keeps until the process exits.  Every call uses the
// same array: calls whose kernels overlap on the GPU (different streams, or
// different host threads without ordering) race on it.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "accord.h"
#include "internal.h"

namespace accord {
namespace {

constexpr size_t kScratchBytes = ACCORD_NOALLOC_SCRATCH_BYTES;
constexpr int64_t kMaxExtent = 2147483647LL;  // n and p; larger sizes are rejected with ACCORD_EINVAL

// Device scratch.  In host code this name is only a stand-in for the symbol:
// the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
cudaError_t scratch_address(int dev, void** out) {
  try {  // std::mutex::lock may throw; no exception leaves the C ABI
    std::lock_guard<std::mutex> guard(g_lock);
    if (g_scratch_addr[dev] == nullptr) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return e;
      g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
  } catch (...) {
    return cudaErrorUnknown;
  }
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace accord

using namespace accord;

extern "C" int accord_loss_f64_noalloc(const double* X, int64_t n, int64_t p, const double* Omega, double lambda,
                                       int penalize_diag, void* stream, double* fg_out) {
  clear_last_error();
  if (X == nullptr || Omega == nullptr || fg_out == nullptr || n < 1 || p < 1 || !(lambda >= 0.0) ||
      !std::isfinite(lambda))
    return kEinval;
  // index limits first, so that the size arithmetic below cannot wrap
  if (n > kMaxExtent || p > kMaxExtent) {
    set_last_error(__FILE__, __LINE__, "n and p must not exceed 2^31 - 1");
    return kEinval;
  }
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return kEcuda;
  if (dev < 0 || dev >= kMaxDevices) return kEunsupported;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return kEunsupported;

  // scratch layout: [Y-GEMM partials: tiles x kYSlots][Omega stats: p x kProxSlots]
  const int64_t tiles = gemm_f64_tiles(p, n);
  const size_t part_bytes = align_up((size_t)tiles * kYSlots * sizeof(double));
  const size_t stats_bytes = align_up((size_t)p * kProxSlots * sizeof(double));
  if (part_bytes + stats_bytes > kScratchBytes) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "needs %zu bytes of scratch, the static array holds %zu",
                  part_bytes + stats_bytes, kScratchBytes);
    set_last_error(__FILE__, __LINE__, msg);
    return kEnomem;
  }
  void* base = nullptr;
  cudaError_t e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    set_last_error(__FILE__, __LINE__, cudaGetErrorString(e));
    return kEcuda;
  }
  double* part = static_cast<double*>(base);
  double* stats = reinterpret_cast<double*>(static_cast<char*>(base) + part_bytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // Every partial row read below is written first by this call (one row per
  // GEMM tile, one per row of Omega), so nothing has to start at zero.
  GemmF64Params g{};
  g.A[0] = g.A[1] = Omega;
  g.lda = p;
  g.B = X;
  g.ldb = p;
  g.M = p;
  g.N = n;
  g.K = p;
  g.out[0] = g.out[1] = nullptr;
  g.part = part;
  g.scale = 1.0;
  e = launch_gemm_f64(kModeY, g, st);
  int64_t nstats = 0;
  if (e == cudaSuccess) e = launch_omega_stats(Omega, 1, p, p, stats, &nstats, st);
  const double lam_d = penalize_diag ? lambda : 0.0;
  if (e == cudaSuccess) e = launch_loss_finish(stats, nstats, part, tiles, lambda, lam_d, 1.0 / (double)n, fg_out, st);
  if (e != cudaSuccess) {
    set_last_error(__FILE__, __LINE__, cudaGetErrorString(e));
    return kEcuda;
  }
  return kOk;
}
