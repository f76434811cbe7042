// Post-processing of an ACCORD estimate (Sec 3.1): the precision matrix
// Theta-hat = T^-1(Omega-hat) = Omega_D Omega and the partial correlations
// rho_ij = -(1/2)(omega_ij / omega_jj + omega_ji / omega_ii).  One pass over
// Omega in 32 x 32 tiles: each block stages its tile and the mirrored tile
// (for omega_ji) in shared memory, so both reads and writes are coalesced.
#include <cmath>
#include <cstring>

#include "api_util.h"
#include "internal.h"

namespace accord {
namespace {

template <class T>
__global__ void post_kernel(const T* __restrict__ Om, int64_t p, T* __restrict__ theta, T* __restrict__ rho,
                            int* bad) {
  __shared__ T a[32][33], b[32][33];
  __shared__ T di[32], dj[32];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x;
  if (threadIdx.y == 0) {
    di[tx] = (i0 + tx < p) ? Om[(i0 + tx) * p + i0 + tx] : T(1);
    dj[tx] = (j0 + tx < p) ? Om[(j0 + tx) * p + j0 + tx] : T(1);
  }
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    a[r][tx] = (i0 + r < p && j0 + tx < p) ? Om[(i0 + r) * p + j0 + tx] : T(0);  // omega_ij
    b[r][tx] = (j0 + r < p && i0 + tx < p) ? Om[(j0 + r) * p + i0 + tx] : T(0);  // omega_ji, stored [j][i]
  }
  __syncthreads();
  int nbad = 0;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, j = j0 + tx;
    if (i >= p || j >= p) continue;
    const T wij = a[r][tx], wji = b[tx][r], wii = di[r], wjj = dj[tx];
    if (!(wii > T(0)) || !(wjj > T(0))) ++nbad;
    if (theta) theta[i * p + j] = wii * wij;
    if (rho) rho[i * p + j] = (i == j) ? T(1) : T(-0.5) * (wij / wjj + wji / wii);
  }
  if (nbad) atomicAdd(bad, nbad);
}

}  // namespace
}  // namespace accord

using namespace accord;

extern "C" int accord_postprocess(int64_t p, const void* Omega, const accord_opts* optp, void* Theta_out,
                                  void* Rho_out) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (Omega == nullptr || p < 1 || (Theta_out == nullptr && Rho_out == nullptr)) return kEinval;
  if (!known_precision(o.precision)) return kEinval;
  if (int e = check_device()) return e;
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const int64_t nb = (p + 31) / 32;
  if (nb > 65535) return kEinval;
  Guard g;
  if (cudaMallocAsync(&g.ptr, 64, st) != cudaSuccess) return kEnomem;
  g.st = st;
  int* bad = static_cast<int*>(g.ptr);
  ACCORD_CK(cudaMemsetAsync(bad, 0, 64, st));
  const dim3 grid((unsigned)nb, (unsigned)nb), block(32, 8);
  if (o.precision == ACCORD_FP64)
    post_kernel<double><<<grid, block, 0, st>>>(static_cast<const double*>(Omega), p, static_cast<double*>(Theta_out),
                                                static_cast<double*>(Rho_out), bad);
  else
    post_kernel<float><<<grid, block, 0, st>>>(static_cast<const float*>(Omega), p, static_cast<float*>(Theta_out),
                                               static_cast<float*>(Rho_out), bad);
  ACCORD_CK(cudaGetLastError());
  int h = 0;
  ACCORD_CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaStreamSynchronize(st));
  return h ? kEdomain : kOk;
}
