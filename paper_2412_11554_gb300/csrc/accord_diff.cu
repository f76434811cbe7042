// Differentiation of the ACCORD objective.
//
// accord_grad_x: the adjoint of the smooth loss L = -sum log omega_ii +
//   1/2 tr(Omega^T Omega S) in the data, dL/dX = (1/n) X Omega^T Omega, formed
//   as Y^T = X Omega^T followed by (1/n) Y^T Omega (two GEMMs, no p x p x p
//   product).
// accord_dloss_dloglam: d L(Omega-hat(lambda); X_val) / d log(lambda) by
//   implicit differentiation of the stationarity conditions of Eq. 3.3 on the
//   active set.  The objective separates over the rows of Omega (proof of
//   Thm 3.2), so each row i with active set A (its nonzeros, i included) and
//   signs s solves its own system
//       (S_AA + omega_ii^-2 e_i e_i^T) dw = -lambda v,
//   v_j = s_j off the diagonal, v_i = 1 when the diagonal is penalised (else 0);
//   one CTA per row builds the system from S, factors it (Cholesky) and dots
//   the solution with the held-out gradient -diag(1/omega) + Omega S_val.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "api_util.h"
#include "internal.h"
#include "tc_gemm.h"

namespace accord {
namespace {

constexpr int kMaxActive = 128;  // active sets up to this size are solved in shared memory
constexpr int kRowThreads = 256;
constexpr size_t kRowSmem = (size_t)kMaxActive * kMaxActive * 8 + kMaxActive * 8;
constexpr int kBigActive = 1024;  // larger ones (up to this size) in a global-memory scratch
constexpr int kBigBlocks = 4;     // blocks of the large-row pass, one scratch slot each
constexpr int kBigThreads = 512;

template <class T>
__global__ void to_f64_kernel(const T* __restrict__ src, int64_t count, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

// The active set of row i (its nonzero columns, the diagonal included) in
// increasing column order into idx[0 .. cap); returns its size, which may
// exceed cap (then only the first cap columns are stored), and sets *pos to
// the diagonal's place (-1 if it lies past cap).  All threads of the block
// call it; wcnt holds one int per warp.
__device__ int active_set(const double* __restrict__ orow, int64_t i, int64_t p, int* idx, int cap, int* wcnt,
                          int* m_sh, int* pos_sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) {
    *m_sh = 0;
    *pos_sh = -1;
  }
  __syncthreads();
  for (int64_t base = 0; base < p; base += blockDim.x) {
    const int64_t j = base + tid;
    const bool nz = j < p && (j == i || orow[j] != 0.0);
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    int off = *m_sh;
    for (int w = 0; w < warp; ++w) off += wcnt[w];
    off += __popc(bal & ((1u << lane) - 1u));
    if (nz && off < cap) {
      idx[off] = (int)j;
      if (j == i) *pos_sh = off;
    }
    __syncthreads();
    if (tid == 0) {
      int t = *m_sh;
      for (int w = 0; w < nw; ++w) t += wcnt[w];
      *m_sh = t;
    }
    __syncthreads();
  }
  return *m_sh;
}

// Row i's system (S_AA + omega_ii^-2 e_i e_i^T) x = v on its active set A =
// idx[0 .. m) (the diagonal at pos), factored by Cholesky in H (leading
// dimension ldh, shared or global memory) and solved in v; then this row's
// share of the derivative into contrib[i] and, if dOm, its row of
// dOmega / dlog(lambda) = -lambda x.  All threads of the block call it.
template <class TO>
__device__ void solve_row(const double* __restrict__ S, const double* __restrict__ orow, const double* __restrict__ Gv,
                          int64_t p, double lam, int pen_diag, int64_t i, const int* idx, int m, int pos, double* H,
                          int ldh, double* v, double* red, int* bad_sh, double* __restrict__ contrib,
                          TO* __restrict__ dOm, int* err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  if (tid == 0) *bad_sh = 0;
  for (int t = tid; t < m * m; t += nt) {
    const int a = t / m, b = t % m;
    double h = S[(int64_t)idx[a] * p + idx[b]];
    if (a == pos && b == pos) h += 1.0 / (orow[i] * orow[i]);
    H[(int64_t)a * ldh + b] = h;
  }
  for (int a = tid; a < m; a += nt) {
    const double w = orow[idx[a]];
    v[a] = (a == pos) ? (pen_diag ? 1.0 : 0.0) : (w > 0.0 ? 1.0 : -1.0);
  }
  __syncthreads();
  // Cholesky factor H = L L^T in place (lower triangle)
  for (int k = 0; k < m; ++k) {
    if (tid == 0) {
      const double d = H[(int64_t)k * ldh + k];
      if (!(d > 0.0)) {
        *bad_sh = 1;
        H[(int64_t)k * ldh + k] = 1.0;
      } else {
        H[(int64_t)k * ldh + k] = sqrt(d);
      }
    }
    __syncthreads();
    const double lkk = H[(int64_t)k * ldh + k];
    for (int r = k + 1 + tid; r < m; r += nt) H[(int64_t)r * ldh + k] /= lkk;
    __syncthreads();
    const int t = m - k - 1;
    for (int q = tid; q < t * t; q += nt) {
      const int r = k + 1 + q / t, c = k + 1 + q % t;
      if (c <= r) H[(int64_t)r * ldh + c] -= H[(int64_t)r * ldh + k] * H[(int64_t)c * ldh + k];
    }
    __syncthreads();
  }
  // L y = v, then L^T x = y
  for (int k = 0; k < m; ++k) {
    if (tid == 0) v[k] /= H[(int64_t)k * ldh + k];
    __syncthreads();
    for (int r = k + 1 + tid; r < m; r += nt) v[r] -= H[(int64_t)r * ldh + k] * v[k];
    __syncthreads();
  }
  for (int k = m - 1; k >= 0; --k) {
    if (tid == 0) v[k] /= H[(int64_t)k * ldh + k];
    __syncthreads();
    for (int r = tid; r < k; r += nt) v[r] -= H[(int64_t)k * ldh + r] * v[k];
    __syncthreads();
  }
  // d omega_iA / d log(lambda) = -lambda x; this row's share of the derivative
  double s = 0.0;
  for (int a = tid; a < m; a += nt) s += Gv[i * p + idx[a]] * (-lam * v[a]);
  s = warp_sum(s);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (tid == 0) {
    double tsum = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) tsum += red[w];
    contrib[i] = *bad_sh ? NAN : tsum;
    if (*bad_sh) atomicOr(err, 2);
  }
  if (dOm != nullptr) {
    for (int64_t j = tid; j < p; j += nt) dOm[i * p + j] = TO(0);
    __syncthreads();
    for (int a = tid; a < m; a += nt) dOm[i * p + idx[a]] = (TO)(-lam * v[a]);
  }
  __syncthreads();
}

// One CTA per row; a row whose active set exceeds kMaxActive is listed in
// big_rows for implicit_big_kernel instead.
template <class TO>
__global__ void __launch_bounds__(kRowThreads) implicit_row_kernel(const double* __restrict__ S,
                                                                   const double* __restrict__ Om,
                                                                   const double* __restrict__ Gv, int64_t p,
                                                                   double lam, int pen_diag,
                                                                   double* __restrict__ contrib, TO* __restrict__ dOm,
                                                                   int* err, int* big_rows, int* n_big) {
  extern __shared__ double smem[];
  double* H = smem;                         // kMaxActive x kMaxActive (row-major, lower part used)
  double* v = H + kMaxActive * kMaxActive;  // right-hand side, then the solution
  __shared__ int idx[kMaxActive];
  __shared__ int wcnt[kRowThreads / 32];
  __shared__ double red[kRowThreads / 32];
  __shared__ int m_sh, pos_sh, bad_sh;
  const int64_t i = blockIdx.x;
  const double* orow = Om + i * p;
  const int m = active_set(orow, i, p, idx, kMaxActive, wcnt, &m_sh, &pos_sh);
  if (m > kMaxActive) {
    if (threadIdx.x == 0) big_rows[atomicAdd(n_big, 1)] = (int)i;
    return;
  }
  const int pos = pos_sh;
  solve_row<TO>(S, orow, Gv, p, lam, pen_diag, i, idx, m, pos, H, kMaxActive, v, red, &bad_sh, contrib, dOm, err);
}

// The listed rows, kBigBlocks CTAs each taking every kBigBlocks-th one, with
// the system in the CTA's slot of a global scratch (max_m x max_m FP64,
// L2-resident at these sizes).  A row over max_m entries sets error bit 1.
template <class TO>
__global__ void __launch_bounds__(kBigThreads) implicit_big_kernel(const double* __restrict__ S,
                                                                   const double* __restrict__ Om,
                                                                   const double* __restrict__ Gv, int64_t p,
                                                                   double lam, int pen_diag,
                                                                   double* __restrict__ contrib, TO* __restrict__ dOm,
                                                                   int* err, const int* big_rows, const int* n_big,
                                                                   double* scratch, int* scratch_idx, int max_m) {
  __shared__ int wcnt[kBigThreads / 32];
  __shared__ double red[kBigThreads / 32];
  __shared__ int m_sh, pos_sh, bad_sh;
  double* H = scratch + (int64_t)blockIdx.x * ((int64_t)max_m * max_m + max_m);
  double* v = H + (int64_t)max_m * max_m;
  int* idx = scratch_idx + (int64_t)blockIdx.x * max_m;
  const int nb = *n_big;
  for (int r = blockIdx.x; r < nb; r += gridDim.x) {
    const int64_t i = big_rows[r];
    const double* orow = Om + i * p;
    const int m = active_set(orow, i, p, idx, max_m, wcnt, &m_sh, &pos_sh);
    const int pos = pos_sh;
    if (m > max_m || pos < 0) {
      if (threadIdx.x == 0) {
        atomicOr(err, 1);
        contrib[i] = NAN;
      }
      __syncthreads();
      continue;
    }
    solve_row<TO>(S, orow, Gv, p, lam, pen_diag, i, idx, m, pos, H, max_m, v, red, &bad_sh, contrib, dOm, err);
  }
}

// Fixed-order sum of n doubles into out[0] (one block).
__global__ void sum_kernel(const double* __restrict__ x, int64_t n, double* out) {
  __shared__ double red[512 / 32];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += x[k];
  s = warp_sum(s);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    out[0] = t;
  }
}

unsigned blocks_for(int64_t count) {
  int64_t b = (count + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

int check_x_omega(const float* X, int64_t n, int64_t p, const void* Omega, const accord_opts& o) {
  if (X == nullptr || Omega == nullptr || n < 1 || p < 1) return kEinval;
  if (!known_precision(o.precision)) return kEinval;
  return check_device();
}

int read_err(const int* err, cudaStream_t st, int* host) {
  ACCORD_CK(cudaMemcpyAsync(host, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaStreamSynchronize(st));
  return kOk;
}

int grad_x_impl(const float* X, int64_t n, int64_t p, const void* Omega, const accord_opts& o, void* GX) {
  const bool f64 = o.precision == ACCORD_FP64;
  const int pt = plane_type(o.precision);
  const size_t pe = plane_bytes(pt);
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const int64_t ldk = round_up(p, 8), ldn = round_up(n, 8);
  size_t c = 0;
  const size_t err_off = take(c, 64);
  size_t x_a = 0, x_b = 0, yt_a = 0, yt_b = 0, om_a = 0, om_b = 0, omt_a = 0, omt_b = 0, tmp = 0;
  if (f64) {
    x_a = take(c, (size_t)n * ldk * 8);          // X (FP64)
    x_b = take(c, (size_t)p * ldn * 8);          // X^T (unused, written by the conversion)
    yt_a = take(c, (size_t)n * ldk * 8);         // Y^T = X Omega^T
    om_a = take(c, (size_t)p * ldk * 8);         // Omega copy
    omt_a = take(c, (size_t)p * ldk * 8);        // Omega^T
  } else {
    x_a = take(c, (size_t)n * ldk * pe);         // X planes
    x_b = take(c, (size_t)n * ldk * pe);
    tmp = take(c, (size_t)p * ldn * pe * 2);     // X^T planes (written by the conversion)
    yt_a = take(c, (size_t)n * ldk * pe);        // Y^T planes
    yt_b = take(c, (size_t)n * ldk * pe);
    om_a = take(c, (size_t)p * ldk * pe);        // Omega planes
    om_b = take(c, (size_t)p * ldk * pe);
    omt_a = take(c, (size_t)p * ldk * pe);       // Omega^T planes
    omt_b = take(c, (size_t)p * ldk * pe);
  }
  const size_t f32t = take(c, f64 ? 0 : (size_t)p * ldk * 4);  // Omega^T in FP32
  Guard g;
  if (cudaMallocAsync(&g.ptr, c, st) != cudaSuccess) return kEnomem;
  g.st = st;
  void* ws = g.ptr;
  int* err = at<int>(ws, err_off);
  ACCORD_CK(cudaMemsetAsync(err, 0, 64, st));
  if (f64) {
    ACCORD_CK(launch_convert_x_f64(X, nullptr, n, p, at<double>(ws, x_a), ldk, at<double>(ws, x_b), ldn, err, st));
    ACCORD_CK(launch_convert_x_f64(nullptr, static_cast<const double*>(Omega), p, p, at<double>(ws, om_a), ldk,
                                   at<double>(ws, omt_a), ldk, err + 1, st));
    GemmF64Params a{};  // Y^T = X Omega^T
    a.A[0] = a.A[1] = at<double>(ws, x_a);
    a.lda = ldk;
    a.B = at<double>(ws, om_a);
    a.ldb = ldk;
    a.M = n; a.N = p; a.K = p;
    a.out[0] = a.out[1] = at<double>(ws, yt_a);
    a.ldout = ldk;
    a.scale = 1.0;
    ACCORD_CK(launch_gemm_f64(kModeGram, a, st));
    GemmF64Params b{};  // dL/dX = (1/n) Y^T Omega
    b.A[0] = b.A[1] = at<double>(ws, yt_a);
    b.lda = ldk;
    b.B = at<double>(ws, omt_a);
    b.ldb = ldk;
    b.M = n; b.N = p; b.K = p;
    b.out[0] = b.out[1] = static_cast<double*>(GX);
    b.ldout = p;
    b.scale = 1.0 / (double)n;
    ACCORD_CK(launch_gemm_f64(kModeGram, b, st));
  } else {
    void* xh = at<void>(ws, x_a);
    void* xl = at<void>(ws, x_b);
    void* xth = at<void>(ws, tmp);
    void* xtl = at<char>(ws, tmp) + (size_t)p * ldn * pe;
    ACCORD_CK(launch_convert_x_planes(X, n, p, xh, xl, ldk, xth, xtl, ldn, err, pt, st));
    const float* Om = static_cast<const float*>(Omega);
    ACCORD_CK(launch_split_planes(Om, p, p, p, at<void>(ws, om_a), at<void>(ws, om_b), ldk, pt, st));
    ACCORD_CK(launch_transpose_x_f32(Om, p, p, at<float>(ws, f32t), ldk, st));
    ACCORD_CK(launch_split_planes(at<float>(ws, f32t), p, p, ldk, at<void>(ws, omt_a), at<void>(ws, omt_b), ldk, pt,
                                  st));
    TcParams a{};  // Y^T = X Omega^T, stored as planes
    if (!encode_plane_map(&a.a_hi[0], xh, pt, n, p, ldk, 128) ||
        !encode_plane_map(&a.a_lo[0], xl, pt, n, p, ldk, 128) ||
        !encode_plane_map(&a.b_hi, at<void>(ws, om_a), pt, p, p, ldk, tc_box_n()) ||
        !encode_plane_map(&a.b_lo, at<void>(ws, om_b), pt, p, p, ldk, tc_box_n()))
      return kEcuda;
    a.a_hi[1] = a.a_hi[0];
    a.a_lo[1] = a.a_lo[0];
    a.err = err + 1;
    tc_shape(a, n, p, p, pt);
    a.out_hi[0] = a.out_hi[1] = at<void>(ws, yt_a);
    a.out_lo[0] = a.out_lo[1] = at<void>(ws, yt_b);
    a.ldplane = ldk;
    a.scale = 1.f;
    ACCORD_CK(launch_tc_gemm(kModeY, a, st));
    TcParams b{};  // dL/dX = (1/n) Y^T Omega
    if (!encode_plane_map(&b.a_hi[0], at<void>(ws, yt_a), pt, n, p, ldk, 128) ||
        !encode_plane_map(&b.a_lo[0], at<void>(ws, yt_b), pt, n, p, ldk, 128) ||
        !encode_plane_map(&b.b_hi, at<void>(ws, omt_a), pt, p, p, ldk, tc_box_n()) ||
        !encode_plane_map(&b.b_lo, at<void>(ws, omt_b), pt, p, p, ldk, tc_box_n()))
      return kEcuda;
    b.a_hi[1] = b.a_hi[0];
    b.a_lo[1] = b.a_lo[0];
    b.err = err + 1;
    tc_shape(b, n, p, p, pt);
    b.out[0] = b.out[1] = static_cast<float*>(GX);
    b.ldout = p;
    b.scale = (float)(1.0 / (double)n);
    ACCORD_CK(launch_tc_gemm(kModeGrad, b, st));
  }
  int h[2] = {0, 0};
  if (int e = read_err(err, st, h)) return e;
  if (h[0] != 0) return kEdomain;
  if (h[1] != 0) {
    set_last_error(__FILE__, __LINE__, f64 ? "non-finite Omega" : "device error bits (an mbarrier wait timed out)");
    return f64 ? kEdomain : kEcuda;
  }
  return kOk;
}

int dloss_impl(const float* Xt, int64_t n, const float* Xv, int64_t n_val, int64_t p, const void* Omega_hat,
               double lambda, const accord_opts& o, double* dloss, double* loss_val, void* dOmega) {
  const bool f64 = o.precision == ACCORD_FP64;
  const int pt = plane_type(o.precision);
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const int64_t ldk = round_up(p, 8), ldn = round_up(n, 8);
  size_t c = 0;
  // error words: [0] non-finite training rows, [1] row-system bits (1: an
  // active set over 1024 entries, 2: not positive definite), [2] non-finite
  // held-out rows, [3] device error bits of the GEMMs
  // results: res[0] = dloss, res[1..2] = f, g of the held-out loss
  const size_t err_off = take(c, 64), res_off = take(c, 64), contrib_off = take(c, (size_t)p * 8);
  const size_t S_off = take(c, (size_t)p * p * 8), Gv_off = take(c, (size_t)p * p * 8);
  const size_t om_off = take(c, (size_t)p * p * 8);
  const size_t x_off = take(c, (size_t)n * ldk * 8), xt_off = take(c, (size_t)p * ldn * 8);
  const size_t g32_off = take(c, f64 ? 0 : (size_t)p * p * 4);  // mixed modes: FP32 held-out gradient
  // rows whose active set exceeds kMaxActive: their list and the large-row
  // pass's scratch (kBigBlocks systems of up to max_m entries)
  const int max_m = (int)(p < kBigActive ? p : kBigActive);
  const size_t big_off = take(c, (size_t)p * 4 + 64);
  const size_t bigs_off = take(c, (size_t)kBigBlocks * ((size_t)max_m * max_m + max_m) * 8);
  const size_t bigi_off = take(c, (size_t)kBigBlocks * max_m * 4);
  Guard g;
  if (cudaMallocAsync(&g.ptr, c, st) != cudaSuccess) return kEnomem;
  g.st = st;
  void* ws = g.ptr;
  int* err = at<int>(ws, err_off);
  double* Om64 = at<double>(ws, om_off);
  ACCORD_CK(cudaMemsetAsync(err, 0, 64, st));
  int* big_rows = at<int>(ws, big_off);
  int* n_big = big_rows + p;
  ACCORD_CK(cudaMemsetAsync(n_big, 0, sizeof(int), st));
  if (f64) ACCORD_CK(cudaMemcpyAsync(Om64, Omega_hat, (size_t)p * p * 8, cudaMemcpyDeviceToDevice, st));
  else to_f64_kernel<float><<<blocks_for(p * p), 256, 0, st>>>(static_cast<const float*>(Omega_hat), p * p, Om64);
  ACCORD_CK(cudaGetLastError());
  double* res = at<double>(ws, res_off);
  if (f64) {
    // S = X^T X / n of the training rows and the held-out loss and gradient
    // -diag(1/omega) + Omega S_val, all in FP64
    ACCORD_CK(launch_convert_x_f64(Xt, nullptr, n, p, at<double>(ws, x_off), ldk, at<double>(ws, xt_off), ldn, err,
                                   st));
    GemmF64Params gs{};
    gs.A[0] = gs.A[1] = at<double>(ws, xt_off);
    gs.lda = ldn;
    gs.B = at<double>(ws, xt_off);
    gs.ldb = ldn;
    gs.M = p; gs.N = p; gs.K = n;
    gs.out[0] = gs.out[1] = at<double>(ws, S_off);
    gs.ldout = p;
    gs.scale = 1.0 / (double)n;
    ACCORD_CK(launch_gemm_f64(kModeGram, gs, st));
    accord_opts o64 = o;
    o64.precision = ACCORD_FP64;
    o64.penalize_diag = 0;
    if (int e = eval_loss_grad_async(Xv, n_val, p, Om64, o64, 0.0, res + 1, 1, at<double>(ws, Gv_off), err + 2))
      return e;
  } else {
    // mixed modes: the same products on the split-operand tensor-core path
    // (FP32 accumulation, FP64 output of S and FP64 reductions), the row
    // systems in FP64.  Both planes of X (and of X^T) fit in the FP64 buffer.
    const size_t pe = plane_bytes(pt);
    void* xh = at<void>(ws, x_off);
    void* xl = at<char>(ws, x_off) + (size_t)n * ldk * pe;
    void* xth = at<void>(ws, xt_off);
    void* xtl = at<char>(ws, xt_off) + (size_t)p * ldn * pe;
    ACCORD_CK(launch_convert_x_planes(Xt, n, p, xh, xl, ldk, xth, xtl, ldn, err, pt, st));
    TcParams t{};
    if (!encode_plane_map(&t.a_hi[0], xth, pt, p, n, ldn, 128) ||
        !encode_plane_map(&t.a_lo[0], xtl, pt, p, n, ldn, 128) ||
        !encode_plane_map(&t.b_hi, xth, pt, p, n, ldn, tc_box_n()) ||
        !encode_plane_map(&t.b_lo, xtl, pt, p, n, ldn, tc_box_n()))
      return kEcuda;
    t.a_hi[1] = t.a_hi[0];
    t.a_lo[1] = t.a_lo[0];
    t.err = err + 3;
    tc_shape(t, p, p, n, pt);
    t.out64 = at<double>(ws, S_off);
    t.ldout64 = p;
    t.scale = (float)(1.0 / (double)n);
    ACCORD_CK(launch_tc_gemm(kModeGram, t, st));
    accord_opts om = o;
    om.penalize_diag = 0;
    float* G32 = at<float>(ws, g32_off);
    if (int e = eval_loss_grad_async(Xv, n_val, p, Omega_hat, om, 0.0, res + 1, 1, G32, err + 2)) return e;
    to_f64_kernel<float><<<blocks_for(p * p), 256, 0, st>>>(G32, p * p, at<double>(ws, Gv_off));
    ACCORD_CK(cudaGetLastError());
  }
  // per-row implicit solves
  static std::mutex mu;
  static int configured = -1;
  int dev = 0;
  ACCORD_CK(cudaGetDevice(&dev));
  std::unique_lock<std::mutex> lock(mu);
  if (configured != dev) {
    ACCORD_CK(cudaFuncSetAttribute(implicit_row_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kRowSmem));
    ACCORD_CK(cudaFuncSetAttribute(implicit_row_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kRowSmem));
    configured = dev;
  }
  lock.unlock();
  if (p > 2147483647LL) return kEinval;
  const int pen = o.penalize_diag ? 1 : 0;
  double* bigs = at<double>(ws, bigs_off);
  int* bigi = at<int>(ws, bigi_off);
  if (f64) {
    implicit_row_kernel<double><<<(unsigned)p, kRowThreads, kRowSmem, st>>>(
        at<double>(ws, S_off), Om64, at<double>(ws, Gv_off), p, lambda, pen, at<double>(ws, contrib_off),
        static_cast<double*>(dOmega), err + 1, big_rows, n_big);
    ACCORD_CK(cudaGetLastError());
    implicit_big_kernel<double><<<kBigBlocks, kBigThreads, 0, st>>>(
        at<double>(ws, S_off), Om64, at<double>(ws, Gv_off), p, lambda, pen, at<double>(ws, contrib_off),
        static_cast<double*>(dOmega), err + 1, big_rows, n_big, bigs, bigi, max_m);
  } else {
    implicit_row_kernel<float><<<(unsigned)p, kRowThreads, kRowSmem, st>>>(
        at<double>(ws, S_off), Om64, at<double>(ws, Gv_off), p, lambda, pen, at<double>(ws, contrib_off),
        static_cast<float*>(dOmega), err + 1, big_rows, n_big);
    ACCORD_CK(cudaGetLastError());
    implicit_big_kernel<float><<<kBigBlocks, kBigThreads, 0, st>>>(
        at<double>(ws, S_off), Om64, at<double>(ws, Gv_off), p, lambda, pen, at<double>(ws, contrib_off),
        static_cast<float*>(dOmega), err + 1, big_rows, n_big, bigs, bigi, max_m);
  }
  ACCORD_CK(cudaGetLastError());
  sum_kernel<<<1, 512, 0, st>>>(at<double>(ws, contrib_off), p, res);
  ACCORD_CK(cudaGetLastError());
  // one readback for the whole call
  double hres[3] = {0.0, 0.0, 0.0};
  int h[4] = {0, 0, 0, 0};
  ACCORD_CK(cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaMemcpyAsync(h, err, sizeof(h), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaStreamSynchronize(st));
  if (h[0] != 0 || h[2] != 0) return kEdomain;
  if (h[3] != 0) {
    set_last_error(__FILE__, __LINE__, "device error bits (an mbarrier wait timed out)");
    return kEcuda;
  }
  if (h[1] & 1) {
    set_last_error(__FILE__, __LINE__, "a row's active set exceeds 1024 entries");
    return kEunsupported;
  }
  if (h[1] & 2) {
    set_last_error(__FILE__, __LINE__, "a row's active-set system is not positive definite");
    return kEdomain;
  }
  if (dloss) *dloss = hres[0];
  if (loss_val) *loss_val = hres[1];
  return kOk;
}

}  // namespace
}  // namespace accord

using namespace accord;

extern "C" {

int accord_grad_x(const float* X, int64_t n, int64_t p, const void* Omega, const accord_opts* optp, void* GX_out) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (GX_out == nullptr) return kEinval;
  if (int e = check_x_omega(X, n, p, Omega, o)) return e;
  return grad_x_impl(X, n, p, Omega, o, GX_out);
}

int accord_dloss_dloglam(const float* X_train, int64_t n, const float* X_val, int64_t n_val, int64_t p,
                         const void* Omega_hat, double lambda, const accord_opts* optp, double* dloss,
                         double* loss_val, void* dOmega) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (X_val == nullptr || n_val < 1 || !(lambda >= 0.0) || !std::isfinite(lambda)) return kEinval;
  if (int e = check_x_omega(X_train, n, p, Omega_hat, o)) return e;
  return dloss_impl(X_train, n, X_val, n_val, p, Omega_hat, lambda, o, dloss, loss_val, dOmega);
}

}  // extern "C"
