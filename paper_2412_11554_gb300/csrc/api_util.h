// Host helpers shared by the C-ABI translation units: workspace carving,
// error capture, device and option checks.
#pragma once

#include <cmath>
#include <cstdint>
#include <new>
#include <stdexcept>
#include <cuda_runtime.h>

#include "accord.h"
#include "internal.h"

namespace accord {
namespace {

constexpr size_t kAlign = 1024;

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

size_t take(size_t& cursor, size_t bytes) {
  const size_t at = cursor;
  cursor += (bytes + kAlign - 1) / kAlign * kAlign;
  return at;
}

constexpr int kBucketCap = 4096;  // Delta entries a 32-row group can hold

template <class T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

struct Guard {  // frees an internally allocated workspace on every exit path
  void* ptr = nullptr;
  cudaStream_t st = nullptr;
  ~Guard() {
    if (ptr) cudaFreeAsync(ptr, st);
  }
};

#define ACCORD_CK(call)                                            \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      set_last_error(__FILE__, __LINE__, cudaGetErrorString(e_));  \
      return kEcuda;                                               \
    }                                                              \
  } while (0)

// Runs an entry point's body so that no C++ exception leaves the C ABI: a
// failed host allocation (std::vector, std::map) becomes ACCORD_ENOMEM, any
// other exception ACCORD_EINVAL, each with a line in accord_last_error.
template <class F>
int abi_call(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    set_last_error(__FILE__, __LINE__, "host memory allocation failed");
    return kEnomem;
  } catch (const std::length_error&) {
    set_last_error(__FILE__, __LINE__, "host buffer size out of range");
    return kEnomem;
  } catch (...) {
    set_last_error(__FILE__, __LINE__, "unexpected host exception");
    return kEinval;
  }
}

int check_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return kEcuda;
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return kEcuda;
  if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return kEcuda;
  if (major != 10 || minor != 3) return kEunsupported;
  return kOk;
}

// Operand-plane type of a mixed precision mode (unused in FP64 mode).
int plane_type(int precision) { return precision == ACCORD_MIXED_TF32X3 ? kPlaneTf32 : kPlaneBf16; }

bool known_precision(int precision) {
  return precision == ACCORD_FP64 || precision == ACCORD_MIXED_BF16X3 || precision == ACCORD_MIXED_TF32X3;
}

int check_opts(const accord_opts& o) {
  if (!known_precision(o.precision)) return kEinval;
  if (!(o.beta > 0.0 && o.beta <= 1.0)) return kEinval;
  if (!std::isfinite(o.tau0)) return kEinval;
  if (!(o.kkt_tol >= 0.0)) return kEinval;
  if (o.max_iter < 0 || o.max_backtracks < 0) return kEinval;
  if (!(o.lipschitz >= 0.0) || !std::isfinite(o.lipschitz)) return kEinval;
  if (o.lipschitz_max_iter < 1) return kEinval;
  if (!(o.lipschitz_tol >= 0.0)) return kEinval;
  if (!(o.epbic_gamma >= 0.0)) return kEinval;
  if (o.trace_cap < 0) return kEinval;
  if (o.y_refresh < 0) return kEinval;
  if (!(o.coarse_kkt >= 0.0) || !std::isfinite(o.coarse_kkt)) return kEinval;
  return kOk;
}

}  // namespace
}  // namespace accord
