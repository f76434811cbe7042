// FP64 SIMT GEMM C = A * B^T with the fused epilogues of the ACCORD-FBS
// iteration (FP64 precision mode).  GB300 executes FP64 on the CUDA cores at
// a small fraction of its tensor rate, so a plain register-blocked tile is
// enough to reach the FP64 pipe's limit; the epilogue carries Eq. 3.5, the
// line-search reductions of Algorithm 1 and the KKT residual of Eq. 3.3.
#include "internal.h"

namespace accord {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct Red {  // per-thread epilogue accumulators
  double s[kProxSlots];
};

template <int MODE>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(const GemmF64Params prm) {
  const bool batch = prm.nprob > 1 || prm.active != nullptr;
  int b = blockIdx.z;
  if (prm.active != nullptr) {
    if (b >= *prm.nactive) return;
    b = prm.active[b];
  }
  const Ctrl* ctrl = prm.ctrl ? prm.ctrl + b : nullptr;
  if (ctrl && ctrl->done) return;
  const int cur = ctrl ? ctrl->cur : 0;
  const int nxt = cur ^ 1;
  const double* __restrict__ A = prm.A[prm.a_nxt ? nxt : cur] + b * prm.s_a;
  const double* __restrict__ B = prm.B + b * prm.s_b;

  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ double red[NT / 32][kProxSlots];

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const int lk = tid % BK, lr = tid / BK;  // loader: 16 k x 16 rows per pass
  for (int64_t k0 = 0; k0 < prm.K; k0 += BK) {
    const int64_t kk = k0 + lk;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = m0 + lr + 16 * i;
      As[lk][lr + 16 * i] = (r < prm.M && kk < prm.K) ? A[r * prm.lda + kk] : 0.0;
      const int64_t c = n0 + lr + 16 * i;
      Bs[lk][lr + 16 * i] = (c < prm.N && kk < prm.K) ? B[c * prm.ldb + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  // ------------------------------------------------------------ epilogue --
  Red r;
#pragma unroll
  for (int q = 0; q < kProxSlots; ++q) r.s[q] = 0.0;
  const double tau = ctrl ? ctrl->tau : 0.0;
  const bool pp = batch && ctrl != nullptr;
  const double lam = pp ? ctrl->lam : prm.lam, lam_d = pp ? ctrl->lam_d : prm.lam_d;
  const double scale = (pp && (MODE == kModeProx || MODE == kModeGram)) ? ctrl->inv_n : prm.scale;
  double* __restrict__ out = prm.out[nxt] ? prm.out[nxt] + b * prm.s_out : nullptr;
  const double* __restrict__ aux = prm.aux[cur] ? prm.aux[cur] + b * prm.s_aux : nullptr;

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = m0 + ty + 16 * i;
    if (row >= prm.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t col = n0 + tx + 16 * j;
      if (col >= prm.N) continue;
      const double v = acc[i][j] * scale;
      if (MODE == kModeY) {
        // Y+ entry; the old Y (aux) gives ||Y+ - Y||^2 = ||Delta X^T||^2.
        const double yo = aux ? aux[row * prm.ldaux + col] : 0.0;
        if (out) out[row * prm.ldout + col] = v;
        const double d = v - yo;
        r.s[kYDiff2] += d * d;
        r.s[kYNorm2] += v * v;
        if (!isfinite(v)) r.s[kYBad] += 1.0;
      } else if (MODE == kModeProx) {
        // v = [Omega S]_ij; A = Omega - tau G; Eq. 3.5.
        const double om = aux[row * prm.ldaux + col];
        const bool dg = (row + prm.row_off == col);
        const double a = om - tau * v;
        double lam_e = lam;  // Eq. 3.8 refit: infinite weight off the support
        if (prm.mask != nullptr && !dg && !((prm.mask[row * prm.mask_ld + (col >> 5)] >> (col & 31)) & 1u))
          lam_e = INFINITY;
        const double w = dg ? diag_prox(a, tau, lam_d) : soft_threshold(a, tau * lam_e);
        out[row * prm.ldout + col] = w;
        const double d = w - om;
        r.s[kPDelta2] += d * d;
        if (dg) {
          r.s[kPLogDiag] += log(w);
          r.s[kPDiagSum] += w;
        } else {
          r.s[kPL1Off] += fabs(w);
          r.s[kPNnz] += (w != 0.0) ? 1.0 : 0.0;
        }
        r.s[kPKkt] = fmax(r.s[kPKkt], kkt_entry(om, v, dg, lam_e, lam_d));
        if (!isfinite(w) || !isfinite(v)) r.s[kPBad] += 1.0;
      } else if (MODE == kModeGrad) {
        double gv = v;
        if (prm.smooth && row + prm.row_off == col) gv -= 1.0 / aux[row * prm.ldaux + col];
        out[row * prm.ldout + col] = gv;
      } else {  // kModeGram
        out[row * prm.ldout + col] = v;
      }
    }
  }
  if (prm.part == nullptr) return;

  // deterministic block reduction -> one partial row per tile
  const int warp = tid / 32, lane = tid % 32;
#pragma unroll
  for (int q = 0; q < kProxSlots; ++q) {
    const double t = (MODE == kModeProx && q == kPKkt) ? warp_max(r.s[q]) : warp_sum(r.s[q]);
    if (lane == 0) red[warp][q] = t;
  }
  __syncthreads();
  if (tid < kProxSlots) {
    double t = red[0][tid];
    for (int w = 1; w < NT / 32; ++w)
      t = (MODE == kModeProx && tid == kPKkt) ? fmax(t, red[w][tid]) : t + red[w][tid];
    const int slots = (MODE == kModeProx) ? kProxSlots : kYSlots;
    if (tid < slots) {
      const int64_t tile = b * prm.s_part + (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      prm.part[tile * slots + tid] = t;
    }
  }
}

}  // namespace

int64_t gemm_f64_tiles(int64_t M, int64_t N) { return ((M + BM - 1) / BM) * ((N + BN - 1) / BN); }

cudaError_t launch_gemm_f64(int mode, const GemmF64Params& prm, cudaStream_t st) {
  if (prm.M <= 0 || prm.N <= 0) return cudaSuccess;
  dim3 grid((unsigned)((prm.N + BN - 1) / BN), (unsigned)((prm.M + BM - 1) / BM),
            (unsigned)(prm.nprob > 1 ? prm.nprob : 1));
  if ((prm.N + BN - 1) / BN > 2147483647LL || grid.y > 65535u || grid.z > 65535u)
    return cudaErrorInvalidConfiguration;
  switch (mode) {
    case kModeY: gemm_f64_kernel<kModeY><<<grid, NT, 0, st>>>(prm); break;
    case kModeProx: gemm_f64_kernel<kModeProx><<<grid, NT, 0, st>>>(prm); break;
    case kModeGrad: gemm_f64_kernel<kModeGrad><<<grid, NT, 0, st>>>(prm); break;
    case kModeGram: gemm_f64_kernel<kModeGram><<<grid, NT, 0, st>>>(prm); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace accord
