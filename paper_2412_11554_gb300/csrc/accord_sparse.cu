// Compressed sparse rows of an ACCORD estimate.  The estimated graph is the
// nonzero pattern of Omega-hat (Sec 3.1), which is sparse by construction of
// the l1 penalty of Eq. 3.2; this export moves only its nonzero entries, so a
// caller reads back O(nnz) bytes instead of the dense p x p array.
//
// Three launches on the caller's stream:
//   row_count_kernel  one warp per row counts the row's nonzero entries into
//                     row_ptr[i + 1] (an HBM pass over Omega);
//   scan_kernel       one block turns the counts into row offsets in place;
//   fill_kernel       one warp per row walks its columns in order, 32 at a
//                     time: a ballot marks the nonzero lanes and their rank
//                     in the ballot gives each one its slot (a second pass).
// The count is read back once (one stream synchronisation) to check the
// caller's capacity before the fill.
#include <cmath>
#include <cstring>

#include "api_util.h"
#include "internal.h"

namespace accord {
namespace {

constexpr int kRowsPerBlock = 8;   // warps a block, one row each
constexpr int kUnroll = 8;         // 32-column chunks in flight per lane
constexpr int kScanThreads = 1024;

// Entries that count as nonzero: everything but +0 and -0 (a NaN counts, so
// that a broken estimate shows up in the export instead of vanishing).
template <class T>
__device__ __forceinline__ bool nz(T v) {
  return !(v == T(0));
}

template <class T>
__global__ void __launch_bounds__(kRowsPerBlock * 32) row_count_kernel(const T* __restrict__ Om, int64_t p,
                                                                        int64_t ld, int64_t* __restrict__ row_ptr) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5);
  if (i >= p) return;
  const T* row = Om + i * ld;
  int cnt = 0;
  for (int64_t c0 = 0; c0 < p; c0 += 32 * kUnroll) {
    T v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t c = c0 + 32 * u + lane;
      v[u] = c < p ? __ldg(row + c) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) cnt += nz(v[u]) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) row_ptr[i + 1] = cnt;
}

// row_ptr[0] = 0 and row_ptr[1..p] hold the counts on entry; on exit
// row_ptr[k] = sum of the counts of rows < k.  One block: each thread sums a
// contiguous run of rows, the block scans the run totals in shared memory,
// and each thread then writes the offsets of its run.
__global__ void __launch_bounds__(kScanThreads) scan_kernel(int64_t* __restrict__ row_ptr, int64_t p) {
  __shared__ int64_t part[kScanThreads];
  const int t = threadIdx.x;
  const int64_t per = (p + kScanThreads - 1) / kScanThreads;
  const int64_t lo = 1 + t * per, hi = min(p + 1, lo + per);
  int64_t s = 0;
  for (int64_t k = lo; k < hi; ++k) s += row_ptr[k];
  part[t] = s;
  __syncthreads();
  // inclusive Hillis-Steele scan of the run totals
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int64_t add = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  int64_t run = part[t] - s;  // offset of this thread's first row
  for (int64_t k = lo; k < hi; ++k) {
    run += row_ptr[k];
    row_ptr[k] = run;
  }
  if (t == 0) row_ptr[0] = 0;
}

template <class T>
__global__ void __launch_bounds__(kRowsPerBlock * 32) fill_kernel(const T* __restrict__ Om, int64_t p, int64_t ld,
                                                                   const int64_t* __restrict__ row_ptr,
                                                                   int32_t* __restrict__ col_idx,
                                                                   T* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5);
  if (i >= p) return;
  const T* row = Om + i * ld;
  const uint32_t below = (1u << lane) - 1u;  // lanes before this one
  int64_t pos = row_ptr[i];
  for (int64_t c0 = 0; c0 < p; c0 += 32 * kUnroll) {
    T v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t c = c0 + 32 * u + lane;
      v[u] = c < p ? __ldg(row + c) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool on = nz(v[u]);
      const uint32_t m = __ballot_sync(0xffffffffu, on);
      if (on) {
        const int64_t at = pos + __popc(m & below);
        col_idx[at] = (int32_t)(c0 + 32 * u + lane);
        vals[at] = v[u];
      }
      pos += __popc(m);
    }
  }
}

}  // namespace
}  // namespace accord

using namespace accord;

extern "C" int accord_to_csr(int64_t p, const void* Omega, const accord_opts* optp, int64_t* row_ptr,
                             int32_t* col_idx, void* vals, int64_t cap, int64_t* nnz) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (nnz) *nnz = 0;
  if (Omega == nullptr || row_ptr == nullptr || nnz == nullptr || p < 1 || p > 2147483647LL || cap < 0)
    return kEinval;
  if (cap > 0 && (col_idx == nullptr || vals == nullptr)) return kEinval;
  if (!known_precision(o.precision)) return kEinval;
  if (int e = check_device()) return e;
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const bool f64 = o.precision == ACCORD_FP64;
  const int64_t blocks = (p + kRowsPerBlock - 1) / kRowsPerBlock;
  if (blocks > 2147483647LL) return kEinval;
  ACCORD_CK(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
  if (f64)
    row_count_kernel<double><<<(unsigned)blocks, kRowsPerBlock * 32, 0, st>>>(static_cast<const double*>(Omega),
                                                                              p, p, row_ptr);
  else
    row_count_kernel<float><<<(unsigned)blocks, kRowsPerBlock * 32, 0, st>>>(static_cast<const float*>(Omega), p,
                                                                             p, row_ptr);
  ACCORD_CK(cudaGetLastError());
  scan_kernel<<<1, kScanThreads, 0, st>>>(row_ptr, p);
  ACCORD_CK(cudaGetLastError());
  int64_t total = 0;
  ACCORD_CK(cudaMemcpyAsync(&total, row_ptr + p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaStreamSynchronize(st));
  *nnz = total;
  if (total > cap) return kEnomem;
  if (total == 0) return kOk;
  if (f64)
    fill_kernel<double><<<(unsigned)blocks, kRowsPerBlock * 32, 0, st>>>(
        static_cast<const double*>(Omega), p, p, row_ptr, col_idx, static_cast<double*>(vals));
  else
    fill_kernel<float><<<(unsigned)blocks, kRowsPerBlock * 32, 0, st>>>(
        static_cast<const float*>(Omega), p, p, row_ptr, col_idx, static_cast<float*>(vals));
  ACCORD_CK(cudaGetLastError());
  return kOk;
}
