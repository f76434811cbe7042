// Setup, statistics and control kernels of the ACCORD-FBS solver: data
// conversion, Omega^0, Omega statistics, a Lanczos estimate of
// L = sigma_max(S) (Sec 3.2) and the device-side accept / backtrack logic of
// Algorithm 1.  All reductions of partial sums run in one block in a fixed
// order, so every result is reproducible run to run.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace accord {
namespace {

constexpr int kRedThreads = 512;

// Deterministic single-block fold of `rows` partial rows of width W.  Slots
// whose bit is set in max_mask are folded with max, the others with +.
template <int W>
__device__ void fold_partials(const double* __restrict__ part, int64_t rows, unsigned max_mask,
                              double (&out)[W]) {
  __shared__ double sh[kRedThreads / 32][W];
  double acc[W];
#pragma unroll
  for (int q = 0; q < W; ++q) acc[q] = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const double v = part[r * W + q];
      acc[q] = ((max_mask >> q) & 1u) ? fmax(acc[q], v) : acc[q] + v;
    }
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    const double t = ((max_mask >> q) & 1u) ? warp_max(acc[q]) : warp_sum(acc[q]);
    if (lane == 0) sh[warp][q] = t;
  }
  __syncthreads();
  // lane q of warp 0 folds slot q over the warps (FP64 is a slow pipe on this
  // part: one thread a slot, not every thread every slot), then all read it
  __shared__ double tot[W];
  if (threadIdx.x < W) {
    const int q = threadIdx.x;
    double t = sh[0][q];
    for (int w = 1; w < (int)(blockDim.x / 32); ++w)
      t = ((max_mask >> q) & 1u) ? fmax(t, sh[w][q]) : t + sh[w][q];
    tot[q] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < W; ++q) out[q] = tot[q];
  __syncthreads();
}

__device__ __forceinline__ void trace_put(double* trace, int64_t cap, int t, int field, double v) {
  if (trace && t >= 0 && t < cap) trace[(int64_t)t * kTraceFields + field] = v;
}

// ------------------------------------------------------------ conversion --
template <class Tin>
__global__ void convert_x_f64_kernel(const Tin* __restrict__ X, int64_t n, int64_t p,
                                     double* __restrict__ X64, int64_t ldx,
                                     double* __restrict__ XT64, int64_t ldxt, int* bad) {
  __shared__ double tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  int nbad = 0;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    double v = 0.0;
    if (r < n && c < p) {
      v = (double)X[r * p + c];
      if (!isfinite(v)) ++nbad;
      X64[r * ldx + c] = v;
    }
    tile[i][threadIdx.x] = v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;  // XT[c][r] = X[r][c]
    if (c < p && r < n) XT64[c * ldxt + r] = tile[threadIdx.x][i];
  }
  if (nbad) atomicAdd(bad, nbad);
}

// Operand planes (type pt) of X (n x ldx) and of X^T (p x ldxt), plus a count
// of the non-finite entries of X.
__global__ void convert_x_planes_kernel(const float* __restrict__ X, int64_t n, int64_t p, void* Xhi, void* Xlo,
                                        int64_t ldx, void* XThi, void* XTlo, int64_t ldxt, int* bad, int pt) {
  __shared__ float tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  int nbad = 0;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < n && c < p) {
      v = X[r * p + c];
      if (!isfinite(v)) ++nbad;
      store_split(Xhi, Xlo, r * ldx + c, v, pt);
    }
    tile[i][threadIdx.x] = v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < p && r < n) store_split(XThi, XTlo, c * ldxt + r, tile[threadIdx.x][i], pt);
  }
  if (nbad) atomicAdd(bad, nbad);
}

// X^T in FP32 (the rows of X^T are read by the sparse Y update).
__global__ void transpose_x_f32_kernel(const float* __restrict__ X, int64_t n, int64_t p, float* __restrict__ XT,
                                       int64_t ldxt) {
  __shared__ float tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < n && c < p) ? X[r * p + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < p && r < n) XT[c * ldxt + r] = tile[threadIdx.x][i];
  }
}

// Row-parallel: a block takes rows r, r + gridDim.x, ..., its threads sweep
// the row's columns contiguously (no index division per element).
template <class T>
__global__ void set_identity_kernel(T* __restrict__ Om, int64_t rows, int64_t ld, int64_t row0) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    T* row = Om + r * ld;
    for (int64_t c = threadIdx.x; c < ld; c += blockDim.x) row[c] = (r + row0 == c) ? T(1) : T(0);
  }
}

// Occupancy bitmap of Omega = I (rows row0 .. row0 + rows of it): word
// (c, i) = c * ldbm + i holds the bit of the diagonal entry (i, i + row0)
// when column i + row0 falls in chunk c.
__global__ void identity_bitmap_kernel(uint32_t* __restrict__ bm, int64_t rows, int64_t row0, int64_t ldbm,
                                       int64_t nwords) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nwords; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / ldbm, i = k - c * ldbm, j = i + row0;
    bm[k] = (i < rows && (j >> 5) == c) ? (1u << (j & 31)) : 0u;
  }
}

// Occupancy bitmap of a dense FP32 rows x cols matrix: one warp per 32 x 32
// block, one ballot per row, and lane r stores the word of row r.
__global__ void bitmap_from_dense_kernel(const float* __restrict__ Om, int64_t rows, int64_t cols, int64_t ld,
                                         uint32_t* __restrict__ bm, int64_t ldbm) {
  const int lane = threadIdx.x & 31;
  const int64_t nch = (cols + 31) / 32, nrb = (rows + 31) / 32, nblk = nch * nrb;
  const int64_t wpb = blockDim.x / 32;
  for (int64_t blk = blockIdx.x * wpb + threadIdx.x / 32; blk < nblk; blk += (int64_t)gridDim.x * wpb) {
    const int64_t rb = blk / nch, c = blk - rb * nch;
    const int64_t col = c * 32 + lane;
    uint32_t mine = 0u;
    for (int r = 0; r < 32; ++r) {
      const int64_t row = rb * 32 + r;
      const bool nz = row < rows && col < cols && Om[row * ld + col] != 0.f;
      const uint32_t w = __ballot_sync(0xffffffffu, nz);
      if (lane == r) mine = w;
    }
    bm[c * ldbm + rb * 32 + lane] = mine;
  }
}

// Dense copy of a mixed-mode iterate buffer: its value where its occupancy
// bitmap has a bit, 0 elsewhere (the buffer's other entries are not read).
__global__ void copy_omega_masked_kernel(const float* __restrict__ src, int64_t lds, const uint32_t* __restrict__ bm,
                                         int64_t ldbm, float* __restrict__ dst, int64_t ldd, int64_t rows, int64_t p) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const float* s = src + r * lds;
    float* d = dst + r * ldd;
    for (int64_t c = threadIdx.x; c < p; c += blockDim.x) {
      const uint32_t w = __ldg(bm + (c >> 5) * ldbm + r);
      d[c] = ((w >> (c & 31)) & 1u) ? s[c] : 0.f;
    }
  }
}

template <class T>
__global__ void copy_omega_kernel(const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                                  int64_t ldd, int64_t rows, int64_t p) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const T* s = src + r * lds;
    T* d = dst + r * ldd;
    for (int64_t c = threadIdx.x; c < p; c += blockDim.x) d[c] = s[c];
  }
}

// One block per row: log-diag, diag sum, off-diagonal l1, nnz, and a bad
// count (non-finite entry, or omega_ii <= 0).
template <class T>
__global__ void omega_stats_kernel(const T* __restrict__ Om, int64_t p, int64_t ld,
                                   double* __restrict__ part, int64_t row0) {
  const int64_t r = blockIdx.x, rd = r + row0;  // rd: this row's diagonal column
  double l1 = 0.0, nnz = 0.0, bad = 0.0;
  for (int64_t c = threadIdx.x; c < p; c += blockDim.x) {
    const double v = (double)Om[r * ld + c];
    if (!isfinite(v)) bad += 1.0;
    if (c != rd) {
      l1 += fabs(v);
      nnz += (v != 0.0) ? 1.0 : 0.0;
    }
  }
  __shared__ double sh[3][8];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  l1 = warp_sum(l1);
  nnz = warp_sum(nnz);
  bad = warp_sum(bad);
  if (lane == 0) { sh[0][warp] = l1; sh[1][warp] = nnz; sh[2][warp] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) { a += sh[0][w]; b += sh[1][w]; c += sh[2][w]; }
    const double d = (double)Om[r * ld + rd];
    if (!(d > 0.0)) c += 1.0;
    double* o = part + r * kProxSlots;
    o[kPDelta2] = 0.0;
    o[kPLogDiag] = d > 0.0 ? log(d) : 0.0;
    o[kPDiagSum] = d;
    o[kPL1Off] = a;
    o[kPNnz] = b;
    o[kPKkt] = 0.0;
    o[kPBad] = c;
    o[7] = 0.0;
  }
}

__global__ void split_planes_kernel(const float* __restrict__ src, int64_t rows, int64_t cols,
                                    int64_t lds, void* hi, void* lo, int64_t ldd, int pt) {
  const int64_t total = rows * ldd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ldd, c = i % ldd;
    store_split(hi, lo, i, c < cols ? src[r * lds + c] : 0.f, pt);
  }
}

// ------------------------------------------------- Lanczos for sigma_max --
// L = sigma_max(S) = lambda_max(K), K = X X^T / n (n x n, symmetric PSD).
// Lanczos with full (two-pass classical Gram-Schmidt) reorthogonalisation;
// after step j the largest eigenvalue of the tridiagonal T_{j+1} is found by
// Sturm-count multisection.  Ritz values increase to lambda_max from below.

// Lanczos kernels serve one problem or a batch: problem b (block x of init
// and step, block y of matvec) uses ctrl[b] and its slices of K, V, w, alpha
// and beta at the strides in LzStrides.  They run in FP64 (FP64 mode, where
// L must match a dense eigensolver to rounding) or in FP32 (mixed modes,
// where the Gram itself carries FP32 accumulation error and L only sets the
// tau <= 1/L floor): FP64 is a slow pipe on this part, and the Sturm
// multisection's divisions dominate an FP64 step.
struct LzStrides {
  int64_t K, V, w, ab;
};

template <class T> struct LzEps;
template <> struct LzEps<double> {
  static constexpr double section = 4e-16, breakdown = 1e-13, tiny = 1e-300, huge = 1e300;
};
template <> struct LzEps<float> {
  static constexpr float section = 2e-7f, breakdown = 1e-6f, tiny = 1e-30f, huge = 1e30f;
};

template <class T>
__global__ void lanczos_init_kernel(Ctrl* ctrl, T* V, int64_t n, LzStrides s) {
  const int b = blockIdx.x;
  ctrl += b;
  V += b * s.V;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) V[i] = T(1) / sqrt(T(n));
  if (threadIdx.x == 0) {
    ctrl->power_done = 0;
    ctrl->pw_iter = 0;
    ctrl->pw_est = 0.0;
    ctrl->pw_prev = 0.0;
  }
}

// w = K V[j], one warp per row (K is the FP64 Gram in both precisions).
template <class T>
__global__ void lanczos_matvec_kernel(const Ctrl* ctrl, const double* __restrict__ K, int64_t ldk,
                                      const T* __restrict__ V, T* __restrict__ w, int64_t n, LzStrides st) {
  const int b = blockIdx.y;
  ctrl += b;
  K += b * st.K;
  V += b * st.V;
  w += b * st.w;
  if (ctrl->power_done) return;
  const T* v = V + (int64_t)ctrl->pw_iter * n;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= n) return;
  T s = T(0);
  for (int64_t c = lane; c < n; c += 32) s = fma(T(K[row * ldk + c]), v[c], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) w[row] = s;
}

template <class T>
__device__ T block_sum(T v, T* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  T t = T(0);
  for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += sh[q];
  return t;
}

// number of eigenvalues of the m x m tridiagonal (a, b) below x
template <class T>
__device__ int sturm_count(const T* a, const T* b, int m, T x) {
  int c = 0;
  T d = a[0] - x;
  if (d < T(0)) ++c;
  for (int i = 1; i < m; ++i) {
    const T dd = (d == T(0)) ? LzEps<T>::tiny : d;
    d = a[i] - x - b[i - 1] * b[i - 1] / dd;
    if (d < T(0)) ++c;
  }
  return c;
}

// One Lanczos step on w = K v_j (block of kLanczosThreads threads).
constexpr int kLanczosThreads = 1024;
template <class T>
__global__ void __launch_bounds__(kLanczosThreads) lanczos_step_kernel(Ctrl* ctrl, T* V, T* w, T* alpha, T* beta,
                                                                       int64_t n, int kmax, double tol, LzStrides st) {
  {
    const int b = blockIdx.x;
    ctrl += b;
    V += b * st.V;
    w += b * st.w;
    alpha += b * st.ab;
    beta += b * st.ab;
  }
  if (ctrl->power_done) return;
  __shared__ T sh[kLanczosThreads / 32];
  __shared__ T h[256];
  __shared__ T lohi[2];
  const int j = ctrl->pw_iter;
  const T* vj = V + (int64_t)j * n;
  T a = T(0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a = fma(vj[i], w[i], a);
  a = block_sum(a, sh);
  const T bprev = j > 0 ? beta[j - 1] : T(0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    w[i] -= a * vj[i] + (j > 0 ? bprev * V[(int64_t)(j - 1) * n + i] : T(0));
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int pass = 0; pass < 2; ++pass) {  // w -= V_{0..j} (V_{0..j}^T w), twice
    for (int q = warp; q <= j; q += nw) {
      const T* vq = V + (int64_t)q * n;
      T s = T(0);
      for (int64_t i = lane; i < n; i += 32) s = fma(vq[i], w[i], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) h[q] = s;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      T s = T(0);
      for (int q = 0; q <= j; ++q) s = fma(h[q], V[(int64_t)q * n + i], s);
      w[i] -= s;
    }
    if (threadIdx.x == 0) a += h[j];
    __syncthreads();
  }
  T bb = T(0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) bb = fma(w[i], w[i], bb);
  const T b = sqrt(block_sum(bb, sh));
  if (threadIdx.x == 0) {
    alpha[j] = a;
    beta[j] = b;
  }
  __syncthreads();
  // largest eigenvalue of T_{j+1} by multisection (warp 0: 32 probes a round)
  const int m = j + 1;
  if (warp == 0) {
    T lo = LzEps<T>::huge, hi = -LzEps<T>::huge;
    for (int i = lane; i < m; i += 32) {
      const T r = (i > 0 ? fabs(beta[i - 1]) : T(0)) + (i + 1 < m ? fabs(beta[i]) : T(0));
      lo = fmin(lo, alpha[i] - r);
      hi = fmax(hi, alpha[i] + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    for (int round = 0; round < 16 && hi - lo > LzEps<T>::section * fmax(fabs(hi), LzEps<T>::tiny); ++round) {
      const T x = lo + (hi - lo) * T(lane + 1) / T(33);
      const bool above = sturm_count(alpha, beta, m, x) == m;  // lambda_max < x
      const unsigned mask = __ballot_sync(0xffffffffu, above);
      const int first = mask ? __ffs(mask) - 1 : 32;  // lowest probe above lambda_max
      const T nlo = first == 0 ? lo : lo + (hi - lo) * T(first) / T(33);
      const T nhi = first == 32 ? hi : lo + (hi - lo) * T(first + 1) / T(33);
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) {
      lohi[0] = lo;
      lohi[1] = hi;
    }
  }
  __syncthreads();
  const double theta = 0.5 * ((double)lohi[0] + (double)lohi[1]);
  const bool stop = ((double)b <= (double)LzEps<T>::breakdown * fmax(fabs(theta), 1e-300)) || (m >= kmax) ||
                    (m >= n) || (j >= 3 && fabs(theta - ctrl->pw_est) <= tol * theta);
  if (!stop)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) V[(int64_t)(j + 1) * n + i] = w[i] / b;
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl->pw_prev = ctrl->pw_est;
    ctrl->pw_est = theta;
    ctrl->pw_iter = j + 1;
    if (stop) ctrl->power_done = 1;
  }
}

// First stage of a two-stage fold: block b folds the contiguous rows
// [b * chunk, (b + 1) * chunk) into row b of out (same slot semantics).
template <int W>
__global__ void fold_stage1_kernel(const Ctrl* ctrl, const double* __restrict__ part, int64_t rows, int64_t chunk,
                                   unsigned max_mask, double* __restrict__ out) {
  if (ctrl != nullptr && ctrl->done) return;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = r0 + chunk < rows ? r0 + chunk : rows;
  double s[W];
  fold_partials<W>(part + r0 * W, r1 > r0 ? r1 - r0 : 0, max_mask, s);
  if (threadIdx.x < W) out[(int64_t)blockIdx.x * W + threadIdx.x] = s[threadIdx.x];
}

// ||Y||^2 partials of Y = X^T (Omega^0 = I): one kYSlots row per block of 64
// rows (slot kYDiff2 = slot kYNorm2, since Y - 0 = Y).
template <class T>
__global__ void rows_norm2_kernel(const T* __restrict__ A, int64_t rows, int64_t cols, int64_t ld,
                                  double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  double s = 0.0, bad = 0.0;
  for (int64_t r = r0; r < r0 + 64 && r < rows; ++r)
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
      const double v = (double)A[r * ld + c];
      s = fma(v, v, s);
      if (!isfinite(v)) bad += 1.0;
    }
  __shared__ double sh[2][kRedThreads / 32];
  s = warp_sum(s);
  bad = warp_sum(bad);
  if (threadIdx.x % 32 == 0) {
    sh[0][threadIdx.x / 32] = s;
    sh[1][threadIdx.x / 32] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      a += sh[0][w];
      b += sh[1][w];
    }
    double* o = part + (int64_t)blockIdx.x * kYSlots;
    o[kYDiff2] = a;
    o[kYNorm2] = a;
    o[kYBad] = b;
    o[3] = 0.0;
  }
}

template <class T>
__global__ void support_mask_kernel(const T* __restrict__ Om, int64_t p, int64_t ld, uint32_t* __restrict__ mask,
                                    int64_t mask_ld) {
  const int64_t total = p * mask_ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / mask_ld, w = i % mask_ld;
    uint32_t bits = 0u;
    for (int b = 0; b < 32; ++b) {
      const int64_t c = 32 * w + b;
      if (c < p && (c == r || Om[r * ld + c] != T(0))) bits |= 1u << b;
    }
    mask[i] = bits;
  }
}

// Statistics of Omega^0 = I in one partial row: log-diag 0, diag sum p.
__global__ void identity_stats_kernel(double* part, int64_t p) {
  if (threadIdx.x < kProxSlots) part[threadIdx.x] = (threadIdx.x == kPDiagSum) ? (double)p : 0.0;
}

// ------------------------------------------------------ Algorithm 1 loop --
__global__ void ctrl_init_kernel(Ctrl* ctrl, const double* ompart, int64_t nomp, const double* ypart,
                                 int64_t nyp, SolveParams sp, double L_given, double* trace) {
  double om[kProxSlots], y[kYSlots];
  fold_partials<kProxSlots>(ompart, nomp, 0u, om);
  fold_partials<kYSlots>(ypart, nyp, 0u, y);
  if (threadIdx.x != 0) return;
  Ctrl& c = *ctrl;
  c.t = 0;
  c.k = 0;
  c.trials = 0;
  c.cur = 0;
  c.done = 0;
  c.refresh = 0;
  c.since_refresh = 0;
  c.n_refresh = 0;
  c.cut_trials = 0;
  c.y_drift = 0.0;
  c.kkt_prev = INFINITY;
  c.coarse = sp.coarse_kkt > 0.0 ? 1 : 0;
  c.n_coarse = 0;
  c.predicted = 0;
  c.no_predict = 0;
  c.status = kNotConverged;
  c.lam = sp.lam;
  c.lam_d = sp.lam_d;
  c.inv_n = sp.inv_n;
  c.L = L_given > 0.0 ? L_given : c.pw_est;
  c.inv_L = c.L > 0.0 ? 1.0 / c.L : INFINITY;
  c.tau0 = sp.tau0 > 0.0 ? sp.tau0 : c.inv_L;
  c.tau = c.tau0;
  c.tau_prev = c.tau0;
  c.g = 0.5 * y[kYNorm2] * c.inv_n;
  c.logdiag = om[kPLogDiag];
  c.diagsum = om[kPDiagSum];
  c.l1off = om[kPL1Off];
  c.nnz = om[kPNnz];
  c.f = c.g - c.logdiag + c.lam * c.l1off + c.lam_d * c.diagsum;
  c.kkt = INFINITY;
  if (om[kPBad] > 0.0) {
    c.done = 1;
    c.status = kEdomain;
  } else if (y[kYBad] > 0.0 || !isfinite(c.f) || !(c.L > 0.0) || !isfinite(c.tau0)) {
    c.done = 1;
    c.status = kEnonfinite;
  }
  trace_put(trace, sp.trace_cap, 0, 0, c.f);
  trace_put(trace, sp.trace_cap, 0, 4, c.nnz);
  trace_put(trace, sp.trace_cap, 0, 6, c.g);
}

// After the prox GEMM, with its folded partials s: on the first trial of a
// step the KKT residual of Omega^t decides convergence (it needs G(Omega^t),
// which this GEMM has just formed); otherwise record the trial's sums.
__device__ void post_prox_update(Ctrl& c, const double (&s)[kProxSlots], const SolveParams& sp, double* trace) {
  const bool coarse = c.coarse != 0;
  if (coarse) c.n_coarse += 1;
  if (c.k == 0) {
    c.kkt_prev = c.kkt;
    c.kkt = s[kPKkt];
    trace_put(trace, sp.trace_cap, c.t, 1, c.kkt);
    // a refresh taken for a predicted pass that did not come: predict no more
    if (c.predicted && c.since_refresh == 0 && !(c.kkt <= sp.kkt_tol)) c.no_predict = 1;
    c.predicted = 0;
    // a residual from the one-product gradient never ends the fit: under the
    // threshold (or the tolerance), or once it stops falling (the one
    // product's own error floor), the next launches form G with the three
    // split products
    if (coarse && (c.kkt <= sp.coarse_kkt || c.kkt <= sp.kkt_tol || !(c.kkt < c.kkt_prev))) c.coarse = 0;
    if (!coarse && c.kkt <= sp.kkt_tol) {
      if (sp.y_refresh > 0 && c.since_refresh > 0) {
        // the residual came from a Y carried forward by updates: form Y
        // afresh from Omega^t and test again, cutting this trial short
        c.refresh = 1;
        c.cut_trials += 1;
        return;
      }
      c.done = 1;
      c.status = kOk;
      return;
    }
    if (!isfinite(c.kkt)) {
      c.done = 1;
      c.status = kEnonfinite;
      return;
    }
    if (c.t >= sp.max_iter) {
      c.done = 1;
      c.status = kNotConverged;
      return;
    }
  }
  if (s[kPBad] > 0.0) {
    c.done = 1;
    c.status = kEnonfinite;
    return;
  }
  c.t_d2 = s[kPDelta2];
  c.t_logdiag = s[kPLogDiag];
  c.t_diagsum = s[kPDiagSum];
  c.t_l1off = s[kPL1Off];
  c.t_nnz = s[kPNnz];
}

// After the Y update of the trial, with its folded partials s: the
// sufficient-decrease test of Algorithm 1 in the form
// ||Y+ - Y||^2 / n <= ||Delta||^2 / tau (identical to the printed test because
// g is quadratic), or the tau <= 1/L floor; accept or backtrack.
__device__ void decide_update(Ctrl& c, const double (&s)[kYSlots], const SolveParams& sp, double* trace) {
  c.dense = 0;
  if (c.refresh) return;  // a trial cut short for a refresh of Y decides nothing
  c.trials += 1;
  if (s[kYBad] > 0.0) {
    c.done = 1;
    c.status = kEnonfinite;
    return;
  }
  c.t_dy2 = s[kYDiff2];
  c.t_y2 = s[kYNorm2];
  const double lhs = c.t_dy2 * c.inv_n;
  const double rhs = c.t_d2 / c.tau;
  const bool accept = (lhs <= rhs) || (c.tau <= c.inv_L) || sp.fixed_step;
  if (accept) {
    trace_put(trace, sp.trace_cap, c.t, 2, c.tau);
    trace_put(trace, sp.trace_cap, c.t, 3, (double)(c.k + 1));
    trace_put(trace, sp.trace_cap, c.t, 5, sqrt(c.t_d2));
    c.t += 1;
    c.cur ^= 1;
    c.g = 0.5 * c.t_y2 * c.inv_n;
    c.logdiag = c.t_logdiag;
    c.diagsum = c.t_diagsum;
    c.l1off = c.t_l1off;
    c.nnz = c.t_nnz;
    c.f = c.g - c.logdiag + c.lam * c.l1off + c.lam_d * c.diagsum;
    trace_put(trace, sp.trace_cap, c.t, 0, c.f);
    trace_put(trace, sp.trace_cap, c.t, 4, c.nnz);
    trace_put(trace, sp.trace_cap, c.t, 6, c.g);
    c.tau_prev = c.tau;
    c.k = 0;
    c.tau = sp.tau_warm ? fmin(c.tau0, c.tau / sp.beta) : c.tau0;
    c.since_refresh += 1;
    if (sp.y_refresh > 0) {
      // due, or ahead of a step whose KKT test is expected to pass (the last
      // ratio of residuals carried one step on): a refresh then saves the
      // trial that a passing test on a carried Y would have to cut short
      const double rate = (isfinite(c.kkt_prev) && c.kkt_prev > c.kkt) ? c.kkt / c.kkt_prev : 1.0;
      const bool due = c.since_refresh >= sp.y_refresh;
      const bool predict = !c.no_predict && c.kkt * rate <= sp.kkt_tol;
      if (due || predict) c.refresh = 1;
      c.predicted = (!due && predict) ? 1 : 0;
    }
  } else {
    c.k += 1;
    if (c.k > sp.max_backtracks) {
      c.done = 1;
      c.status = kEbacktrack;
      return;
    }
    c.tau *= sp.beta;
  }
}

__global__ void post_prox_kernel(Ctrl* ctrl, const double* part, int64_t ntiles, SolveParams sp,
                                 double* trace) {
  if (ctrl->done) return;
  double s[kProxSlots];
  fold_partials<kProxSlots>(part, ntiles, 1u << kPKkt, s);
  if (threadIdx.x == 0) post_prox_update(*ctrl, s, sp, trace);
}

// ----------------------------------------------- row blocks of one fit --
// The objective separates over the rows of Omega (the row-wise form in the
// proof of Thm 3.2), so a fit can be split into blocks of rows that share
// only Algorithm 1's scalars.  A block folds its own trial sums here (out:
// the kProxSlots prox sums, then the kYSlots sums of whichever Y update ran)
// for the caller's exchange over all blocks; decide_global_kernel then takes
// the decisions of post_prox_update and decide_update on the sums over all
// blocks, so every block takes the same ones.
__global__ void fold_block_kernel(const Ctrl* ctrl, const double* prox_part, int64_t nprox, const double* y_part,
                                  int64_t ny, int* bucket_counts, int nbuckets, const double* part_sparse,
                                  unsigned long long* delta_entries, double* out) {
  if (ctrl->done) return;
  double s[kProxSlots], y[kYSlots];
  fold_partials<kProxSlots>(prox_part, nprox, 1u << kPKkt, s);
  const bool sparse_ran = part_sparse != nullptr && !ctrl->dense;
  fold_partials<kYSlots>(sparse_ran ? part_sparse : y_part, sparse_ran ? nbuckets : ny, 0u, y);
  unsigned long long cnt = 0;
  for (int i = threadIdx.x; bucket_counts != nullptr && i < nbuckets; i += blockDim.x) {
    if (sparse_ran) cnt += (unsigned long long)bucket_counts[i];
    bucket_counts[i] = 0;
  }
  if (delta_entries != nullptr && sparse_ran) {
    __shared__ unsigned long long red[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
      *delta_entries += t;
    }
  }
  if (threadIdx.x < kProxSlots) out[threadIdx.x] = s[threadIdx.x];
  if (threadIdx.x < kYSlots) out[kProxSlots + threadIdx.x] = y[threadIdx.x];
}

__global__ void decide_global_kernel(Ctrl* ctrl, const double* g, SolveParams sp, double* trace) {
  if (threadIdx.x != 0 || ctrl->done) return;
  double s[kProxSlots], y[kYSlots];
#pragma unroll
  for (int q = 0; q < kProxSlots; ++q) s[q] = g[q];
#pragma unroll
  for (int q = 0; q < kYSlots; ++q) y[q] = g[kProxSlots + q];
  post_prox_update(*ctrl, s, sp, trace);
  if (!ctrl->done) decide_update(*ctrl, y, sp, trace);
}

__global__ void decide_kernel(Ctrl* ctrl, const double* part, int64_t ntiles, SolveParams sp,
                              double* trace, int* bucket_counts, int nbuckets, const double* part_sparse,
                              unsigned long long* delta_entries) {
  if (ctrl->done) return;
  double s[kYSlots];
  // partial sums of whichever Y update ran: the sparse one (one row per
  // bucket) unless a bucket overflowed and the dense product ran instead
  const bool sparse_ran = part_sparse != nullptr && !ctrl->dense;
  fold_partials<kYSlots>(sparse_ran ? part_sparse : part, sparse_ran ? nbuckets : ntiles, 0u, s);
  // Delta entries the sparse update applied in this trial (none overflowed
  // when it ran), then empty buckets for the next trial's prox epilogue
  unsigned long long cnt = 0;
  for (int i = threadIdx.x; bucket_counts != nullptr && i < nbuckets; i += blockDim.x) {
    if (sparse_ran) cnt += (unsigned long long)bucket_counts[i];
    bucket_counts[i] = 0;
  }
  if (delta_entries != nullptr && sparse_ran) {
    __shared__ unsigned long long red[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
      *delta_entries += t;
    }
  }
  if (threadIdx.x == 0) decide_update(*ctrl, s, sp, trace);
}

// After y_refresh_kernel: the drift it found and, for a whole fit, g and f
// of the iterate from the Y formed afresh (a row block leaves them: its
// ||Y||^2 covers its own rows only).  Then the trial that follows tests the
// KKT residual on the new Y.
__global__ void y_refresh_fold_kernel(Ctrl* ctrl, const int32_t* active, const int32_t* nactive, const double* part,
                                      int64_t ngroups, int64_t s_part, int update_g) {
  int b = blockIdx.x;
  if (active != nullptr) {
    if (b >= *nactive) return;
    b = active[b];
  }
  Ctrl& c = ctrl[b];
  if (c.done || !c.refresh) return;
  double s[kYSlots];
  fold_partials<kYSlots>(part + b * s_part, ngroups, 0u, s);
  if (threadIdx.x != 0) return;
  const double y2 = s[kYNorm2];
  const double drift = y2 > 0.0 ? sqrt(s[kYDiff2] / y2) : (s[kYDiff2] > 0.0 ? INFINITY : 0.0);
  c.y_drift = fmax(c.y_drift, drift);
  if (s[kYBad] > 0.0) {
    c.done = 1;
    c.status = kEnonfinite;
    return;
  }
  if (update_g) {
    c.g = 0.5 * y2 * c.inv_n;
    c.f = c.g - c.logdiag + c.lam * c.l1off + c.lam_d * c.diagsum;
  }
  c.refresh = 0;
  c.since_refresh = 0;
  c.n_refresh += 1;
}

// ------------------------------------------------------- batched control --
constexpr int kBucketRowsDev = kBucketRows;
__device__ __forceinline__ int slot_problem(const int32_t* active, const int32_t* nactive, int slot) {
  if (active == nullptr) return slot;
  return slot < *nactive ? active[slot] : -1;
}

__global__ void post_prox_batch_kernel(Ctrl* ctrl, const int32_t* active, const int32_t* nactive,
                                       const double* part, int64_t ntiles, SolveParams sp) {
  const int b = slot_problem(active, nactive, blockIdx.x);
  if (b < 0 || ctrl[b].done) return;
  double s[kProxSlots];
  fold_partials<kProxSlots>(part + b * ntiles * kProxSlots, ntiles, 1u << kPKkt, s);
  if (threadIdx.x == 0) post_prox_update(ctrl[b], s, sp, nullptr);
}

__global__ void decide_batch_kernel(Ctrl* ctrl, const int32_t* active, const int32_t* nactive, const double* part,
                                    int64_t ntiles, SolveParams sp, int* bucket_counts, int nbuckets,
                                    const double* part_sparse) {
  const int b = slot_problem(active, nactive, blockIdx.x);
  if (b < 0) return;
  Ctrl& c = ctrl[b];
  // every problem of the trial starts the next one with empty Delta buckets,
  // including one whose fit ended in this trial (its prox already filled them)
  for (int i = threadIdx.x; bucket_counts != nullptr && i < nbuckets; i += blockDim.x)
    bucket_counts[(int64_t)b * nbuckets + i] = 0;
  if (c.done) {
    if (threadIdx.x == 0) c.dense = 0;
    return;
  }
  double s[kYSlots];
  const bool sparse_ran = part_sparse != nullptr && !c.dense && !c.ymode;
  if (sparse_ran) fold_partials<kYSlots>(part_sparse + (int64_t)b * nbuckets * kYSlots, nbuckets, 0u, s);
  else fold_partials<kYSlots>(part + b * ntiles * kYSlots, ntiles, 0u, s);
  if (threadIdx.x == 0) {
    // Y update of the next trial: dense (the prox writes Delta planes) after a
    // bucket overflowed; back to the buckets once Omega+ has so few nonzeros
    // (under 16 a row off the diagonal) that Delta fits them with room to spare
    if (part_sparse != nullptr) {
      if (c.dense) c.ymode = 1;
      else if (c.ymode && c.t_nnz < 16.0 * (double)(nbuckets * kBucketRowsDev)) c.ymode = 0;
    }
    decide_update(c, s, sp, nullptr);
  }
}

// One block per chain: g of Y^0 = X^T, then the state of Omega^0 = I.
template <class T>
__global__ void batch_ctrl_init_kernel(PathDev pd, const T* __restrict__ yt0, int64_t p, int64_t ldy, int64_t s_y,
                                       SolveParams sp, double L_given) {
  const int c = blockIdx.x;
  const T* y = yt0 + c * s_y;
  double s = 0.0, bad = 0.0;
  for (int64_t i = threadIdx.x; i < p * ldy; i += blockDim.x) {
    const double v = (double)y[i];
    s = fma(v, v, s);
    if (!isfinite(v)) bad += 1.0;
  }
  __shared__ double sh[2][kRedThreads / 32];
  s = warp_sum(s);
  bad = warp_sum(bad);
  if (threadIdx.x % 32 == 0) {
    sh[0][threadIdx.x / 32] = s;
    sh[1][threadIdx.x / 32] = bad;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double ys = 0.0, yb = 0.0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
    ys += sh[0][w];
    yb += sh[1][w];
  }
  Ctrl& C = pd.ctrl[c];
  C.refresh = 0;
  C.since_refresh = 0;
  C.n_refresh = 0;
  C.cut_trials = 0;
  C.y_drift = 0.0;
  C.kkt_prev = INFINITY;
  C.coarse = sp.coarse_kkt > 0.0 ? 1 : 0;
  C.n_coarse = 0;
  C.predicted = 0;
  C.no_predict = 0;
  C.L = L_given > 0.0 ? L_given : C.pw_est;
  C.inv_L = C.L > 0.0 ? 1.0 / C.L : INFINITY;
  C.tau0 = sp.tau0 > 0.0 ? sp.tau0 : C.inv_L;
  C.tau = C.tau0;
  C.tau_prev = C.tau0;
  C.g = 0.5 * ys * C.inv_n;
  C.logdiag = 0.0;
  C.diagsum = (double)p;
  C.l1off = 0.0;
  C.nnz = 0.0;
  C.f = C.g + C.lam_d * C.diagsum;
  C.kkt = INFINITY;
  if (yb > 0.0 || !isfinite(C.f) || !(C.L > 0.0) || !isfinite(C.tau0)) {
    C.done = 1;
    C.status = kEnonfinite;
  }
  if (c == 0) {
    // every chain starts active
    for (int q = 0; q < pd.nchains; ++q) pd.active[q] = q;
    *pd.nactive = pd.nchains;
  }
}

__global__ void path_advance_kernel(PathDev pd) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < pd.nchains; c += blockDim.x) {
    Ctrl& C = pd.ctrl[c];
    C.emit = 0;
    if (C.finished || !C.done) continue;
    const int k = C.lam_idx;
    PathRec& r = pd.rec[(int64_t)k * pd.nchains + c];
    const double n = pd.n_obs[c];
    r.status = C.status;
    r.iters = C.t;
    r.trials = C.trials;
    r.y_refreshes = C.n_refresh;
    r.y_drift = C.y_drift;
    r.lambda = pd.lambdas[k];
    r.f = C.f;
    r.g = C.g;
    r.kkt = C.kkt;
    r.logdet_d = C.logdiag;
    r.tau_last = C.tau_prev;
    r.nnz_offdiag = (int64_t)C.nnz;
    // Eq. 3.7: 2n(-log det Omega_D + g) + ||Omega||_0 (log n + 4 gamma log p)
    r.epbic = 2.0 * n * (-C.logdiag + C.g) + C.nnz * (log(n) + 4.0 * pd.gamma * pd.log_p);
    C.iters_tot += C.t;
    C.trials_tot += C.trials;
    C.emit = 1;
    C.emit_lam = k;
    if (C.status >= 0 && r.epbic < pd.best_epbic[c]) {
      pd.best_epbic[c] = r.epbic;
      pd.best_idx[c] = k;
      C.emit |= 2;
    }
    if (C.status >= 0 && k + 1 < pd.n_lambda) {
      // warm start: the next penalty begins at this estimate
      const double lam = pd.lambdas[k + 1];
      C.lam_idx = k + 1;
      C.lam = lam;
      C.lam_d = pd.penalize_diag ? lam : 0.0;
      C.f = C.g - C.logdiag + C.lam * C.l1off + C.lam_d * C.diagsum;
      C.t = 0;
      C.k = 0;
      C.trials = 0;
      C.tau = C.tau0;
      C.tau_prev = C.tau0;
      C.kkt = INFINITY;
      C.status = kNotConverged;
      C.done = 0;
      C.n_refresh = 0;
      C.cut_trials = 0;
      C.y_drift = 0.0;
      C.kkt_prev = INFINITY;
      C.coarse = pd.coarse;
      C.predicted = 0;
      C.no_predict = 0;
    } else {
      // the chain ends here; an error also ends the penalties after it
      for (int q = k + 1; q < pd.n_lambda; ++q) {
        PathRec& z = pd.rec[(int64_t)q * pd.nchains + c];
        z = PathRec{};
        z.status = C.status;
        z.lambda = pd.lambdas[q];
        z.epbic = INFINITY;
      }
      C.finished = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int c = 0; c < pd.nchains; ++c)
      if (!pd.ctrl[c].finished) {
        pd.active[m++] = c;
        any |= pd.ctrl[c].ymode;
      }
    *pd.nactive = m;
    // the dense Y kernels of the next trial run only if some chain needs them
    // (a bucket overflow during the trial sets the flag too)
    if (pd.any_dense != nullptr) *pd.any_dense = any;
  }
}

template <class T>
// bm0 / bm1 (mixed modes): the occupancy bitmaps of the two buffers, whose
// values count only where a bit is set; null in FP64 mode (dense buffers).
__global__ void path_emit_kernel(PathDev pd, const T* __restrict__ om0, const T* __restrict__ om1, int64_t p,
                                 int64_t ldo, int64_t s_om, uint32_t* __restrict__ support, int64_t mask_ld,
                                 T* __restrict__ best, const uint32_t* __restrict__ bm0, const uint32_t* __restrict__ bm1,
                                 int64_t ldbm, int64_t s_bm) {
  const int c = blockIdx.y;
  const Ctrl& C = pd.ctrl[c];
  if (C.emit == 0) return;
  const T* Om = (C.cur ? om1 : om0) + c * s_om;
  const uint32_t* bm = bm0 != nullptr ? (C.cur ? bm1 : bm0) + c * s_bm : nullptr;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  if (support != nullptr) {
    uint32_t* out = support + ((int64_t)C.emit_lam * pd.nchains + c) * p * mask_ld;
    for (int64_t i = tid; i < p * mask_ld; i += stride) {
      const int64_t r = i / mask_ld, w = i % mask_ld;
      uint32_t bits = 0u;
      if (bm != nullptr) {
        bits = bm[w * ldbm + r];  // the diagonal bit is always set (omega_ii > 0)
      } else {
        for (int q = 0; q < 32; ++q) {
          const int64_t col = 32 * w + q;
          if (col < p && (col == r || Om[r * ldo + col] != T(0))) bits |= 1u << q;
        }
      }
      out[i] = bits;
    }
  }
  if ((C.emit & 2) && best != nullptr) {
    T* dst = best + c * p * p;
    for (int64_t i = tid; i < p * p; i += stride) {
      const int64_t r = i / p, col = i % p;
      const bool nz = bm == nullptr || ((bm[(col >> 5) * ldbm + r] >> (col & 31)) & 1u);
      dst[i] = nz ? Om[r * ldo + col] : T(0);
    }
  }
}

__global__ void loss_finish_kernel(const double* ompart, int64_t nomp, const double* ypart, int64_t nyp,
                                   double lam, double lam_d, double inv_n, double* out) {
  double om[kProxSlots], y[kYSlots];
  fold_partials<kProxSlots>(ompart, nomp, 0u, om);
  fold_partials<kYSlots>(ypart, nyp, 0u, y);
  if (threadIdx.x != 0) return;
  double g = 0.5 * y[kYNorm2] * inv_n;
  double f = g - om[kPLogDiag] + lam * om[kPL1Off] + lam_d * om[kPDiagSum];
  if (om[kPBad] > 0.0) f = INFINITY;  // a diagonal entry outside the domain of -log
  if (y[kYBad] > 0.0) f = g = NAN;    // non-finite data: Omega X^T has no finite value
  out[0] = f;
  out[1] = g;
}

unsigned grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_convert_x_f64(const float* X32, const double* X64in, int64_t n, int64_t p,
                                 double* X64, int64_t ldx, double* XT64, int64_t ldxt, int* bad,
                                 cudaStream_t st) {
  dim3 grid((unsigned)((p + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  if (X64in)
    convert_x_f64_kernel<double><<<grid, block, 0, st>>>(X64in, n, p, X64, ldx, XT64, ldxt, bad);
  else
    convert_x_f64_kernel<float><<<grid, block, 0, st>>>(X32, n, p, X64, ldx, XT64, ldxt, bad);
  return cudaGetLastError();
}

cudaError_t launch_convert_x_planes(const float* X32, int64_t n, int64_t p, void* Xhi, void* Xlo, int64_t ldx,
                                    void* XThi, void* XTlo, int64_t ldxt, int* bad, int pt, cudaStream_t st) {
  dim3 grid((unsigned)((p + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  convert_x_planes_kernel<<<grid, block, 0, st>>>(X32, n, p, Xhi, Xlo, ldx, XThi, XTlo, ldxt, bad, pt);
  return cudaGetLastError();
}

cudaError_t launch_set_identity(void* Om, int is_f64, int64_t p, int64_t ld, cudaStream_t st, int64_t rows,
                                int64_t row0) {
  if (rows < 0) rows = p;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, 152 * 16));
  if (is_f64) set_identity_kernel<double><<<g, 512, 0, st>>>((double*)Om, rows, ld, row0);
  else set_identity_kernel<float><<<g, 512, 0, st>>>((float*)Om, rows, ld, row0);
  return cudaGetLastError();
}

int64_t bitmap_ld(int64_t rows) { return (rows + 31) / 32 * 32; }
int64_t bitmap_words(int64_t rows, int64_t cols) { return (cols + 31) / 32 * bitmap_ld(rows); }
int64_t bitmap_words(int64_t p) { return bitmap_words(p, p); }

cudaError_t launch_identity_bitmap(uint32_t* bm, int64_t p, cudaStream_t st, int64_t rows, int64_t row0) {
  if (rows < 0) rows = p;
  const int64_t nw = bitmap_words(rows, p);
  identity_bitmap_kernel<<<grid_for(nw, 256), 256, 0, st>>>(bm, rows, row0, bitmap_ld(rows), nw);
  return cudaGetLastError();
}

cudaError_t launch_bitmap_from_dense(const float* Om, int64_t p, int64_t ld, uint32_t* bm, cudaStream_t st,
                                     int64_t rows) {
  if (rows < 0) rows = p;
  const int64_t blocks = ((p + 31) / 32 * ((rows + 31) / 32) + 7) / 8;
  bitmap_from_dense_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, 152 * 32)), 256, 0, st>>>(
      Om, rows, p, ld, bm, bitmap_ld(rows));
  return cudaGetLastError();
}

cudaError_t launch_copy_omega_masked(const float* src, int64_t lds, const uint32_t* bm, float* dst, int64_t ldd,
                                     int64_t p, cudaStream_t st, int64_t rows) {
  if (rows < 0) rows = p;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, 152 * 16));
  copy_omega_masked_kernel<<<g, 512, 0, st>>>(src, lds, bm, bitmap_ld(rows), dst, ldd, rows, p);
  return cudaGetLastError();
}

cudaError_t launch_copy_omega(const void* src, int64_t lds, void* dst, int64_t ldd, int is_f64,
                              int64_t p, cudaStream_t st, int64_t rows) {
  if (rows < 0) rows = p;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, 152 * 16));
  if (is_f64) copy_omega_kernel<double><<<g, 512, 0, st>>>((const double*)src, lds, (double*)dst, ldd, rows, p);
  else copy_omega_kernel<float><<<g, 512, 0, st>>>((const float*)src, lds, (float*)dst, ldd, rows, p);
  return cudaGetLastError();
}

cudaError_t launch_omega_stats(const void* Om, int is_f64, int64_t p, int64_t ld, double* part,
                               int64_t* nparts, cudaStream_t st, int64_t rows, int64_t row0) {
  if (rows < 0) rows = p;
  if (rows > 2147483647LL || rows < 1) return cudaErrorInvalidValue;
  if (is_f64) omega_stats_kernel<double><<<(unsigned)rows, 256, 0, st>>>((const double*)Om, p, ld, part, row0);
  else omega_stats_kernel<float><<<(unsigned)rows, 256, 0, st>>>((const float*)Om, p, ld, part, row0);
  *nparts = rows;
  return cudaGetLastError();
}

cudaError_t launch_split_planes(const float* src, int64_t rows, int64_t cols, int64_t lds, void* hi, void* lo,
                                int64_t ldd, int pt, cudaStream_t st) {
  split_planes_kernel<<<grid_for(rows * ldd, 256), 256, 0, st>>>(src, rows, cols, lds, hi, lo, ldd, pt);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_init(Ctrl* ctrl, void* V, int64_t n, cudaStream_t st, int nprob, int64_t sV, int f32) {
  if (nprob < 1 || nprob > 65535) return cudaErrorInvalidValue;
  if (f32) lanczos_init_kernel<float><<<(unsigned)nprob, 256, 0, st>>>(ctrl, (float*)V, n, LzStrides{0, sV, 0, 0});
  else lanczos_init_kernel<double><<<(unsigned)nprob, 256, 0, st>>>(ctrl, (double*)V, n, LzStrides{0, sV, 0, 0});
  return cudaGetLastError();
}

cudaError_t launch_lanczos_steps(Ctrl* ctrl, const double* K, int64_t ldk, void* V, void* w, void* alpha, void* beta,
                                 int64_t n, int kmax, int nsteps, double tol, cudaStream_t st, int nprob, int64_t sK,
                                 int64_t sV, int64_t sW, int64_t sAB, int f32) {
  if (kmax > 256 || nprob < 1 || nprob > 65535) return cudaErrorInvalidValue;
  const LzStrides s{sK, sV, sW, sAB};
  const dim3 g((unsigned)((n + 7) / 8), (unsigned)nprob);
  for (int q = 0; q < nsteps; ++q) {
    if (f32) {
      lanczos_matvec_kernel<float><<<g, 256, 0, st>>>(ctrl, K, ldk, (const float*)V, (float*)w, n, s);
      lanczos_step_kernel<float><<<(unsigned)nprob, kLanczosThreads, 0, st>>>(ctrl, (float*)V, (float*)w,
                                                                              (float*)alpha, (float*)beta, n, kmax,
                                                                              tol, s);
    } else {
      lanczos_matvec_kernel<double><<<g, 256, 0, st>>>(ctrl, K, ldk, (const double*)V, (double*)w, n, s);
      lanczos_step_kernel<double><<<(unsigned)nprob, kLanczosThreads, 0, st>>>(ctrl, (double*)V, (double*)w,
                                                                               (double*)alpha, (double*)beta, n, kmax,
                                                                               tol, s);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_ctrl_init(Ctrl* ctrl, const double* ompart, int64_t nomp, const double* ypart,
                             int64_t nyp, const SolveParams& sp, double L_given, double* trace,
                             cudaStream_t st) {
  ctrl_init_kernel<<<1, kRedThreads, 0, st>>>(ctrl, ompart, nomp, ypart, nyp, sp, L_given, trace);
  return cudaGetLastError();
}

cudaError_t launch_y_refresh_fold(Ctrl* ctrl, int32_t nprob, const int32_t* active, const int32_t* nactive,
                                  const double* part, int64_t ngroups, int64_t s_part, int update_g,
                                  cudaStream_t st) {
  if (nprob < 1 || nprob > 65535) return cudaErrorInvalidConfiguration;
  y_refresh_fold_kernel<<<(unsigned)nprob, kRedThreads, 0, st>>>(ctrl, active, nactive, part, ngroups, s_part,
                                                                 update_g);
  return cudaGetLastError();
}

cudaError_t launch_post_prox(Ctrl* ctrl, const double* part, int64_t ntiles, const SolveParams& sp,
                             double* trace, double* fold_scratch, cudaStream_t st) {
  if (fold_scratch != nullptr && ntiles > 4 * kFoldChunks) {
    // two-stage fixed-order fold: kFoldChunks blocks, then one
    const int64_t chunk = (ntiles + kFoldChunks - 1) / kFoldChunks;
    fold_stage1_kernel<kProxSlots><<<kFoldChunks, kRedThreads, 0, st>>>(ctrl, part, ntiles, chunk, 1u << kPKkt,
                                                                         fold_scratch);
    post_prox_kernel<<<1, kRedThreads, 0, st>>>(ctrl, fold_scratch, kFoldChunks, sp, trace);
  } else {
    post_prox_kernel<<<1, kRedThreads, 0, st>>>(ctrl, part, ntiles, sp, trace);
  }
  return cudaGetLastError();
}

cudaError_t launch_fold_block(Ctrl* ctrl, const double* prox_part, int64_t ntiles_prox, double* fold_scratch,
                              const double* y_part, int64_t ntiles_y, int* bucket_counts, int nbuckets,
                              const double* part_sparse, unsigned long long* delta_entries, double* out,
                              cudaStream_t st) {
  const double* pp = prox_part;
  int64_t np = ntiles_prox;
  if (fold_scratch != nullptr && ntiles_prox > 4 * kFoldChunks) {
    const int64_t chunk = (ntiles_prox + kFoldChunks - 1) / kFoldChunks;
    fold_stage1_kernel<kProxSlots><<<kFoldChunks, kRedThreads, 0, st>>>(ctrl, prox_part, ntiles_prox, chunk,
                                                                         1u << kPKkt, fold_scratch);
    pp = fold_scratch;
    np = kFoldChunks;
  }
  fold_block_kernel<<<1, kRedThreads, 0, st>>>(ctrl, pp, np, y_part, ntiles_y, bucket_counts, nbuckets, part_sparse,
                                               delta_entries, out);
  return cudaGetLastError();
}

cudaError_t launch_decide_global(Ctrl* ctrl, const double* sums, const SolveParams& sp, double* trace,
                                 cudaStream_t st) {
  decide_global_kernel<<<1, 32, 0, st>>>(ctrl, sums, sp, trace);
  return cudaGetLastError();
}

cudaError_t launch_rows_norm2(const void* A, int is_f64, int64_t rows, int64_t cols, int64_t ld, double* part,
                              int64_t* nparts, cudaStream_t st) {
  const unsigned g = (unsigned)((rows + 63) / 64);
  if (is_f64) rows_norm2_kernel<double><<<g, kRedThreads, 0, st>>>((const double*)A, rows, cols, ld, part);
  else rows_norm2_kernel<float><<<g, kRedThreads, 0, st>>>((const float*)A, rows, cols, ld, part);
  *nparts = g;
  return cudaGetLastError();
}

cudaError_t launch_support_mask(const void* Om, int is_f64, int64_t p, int64_t ld, uint32_t* mask, int64_t mask_ld,
                                cudaStream_t st) {
  const unsigned g = grid_for(p * mask_ld, 256);
  if (is_f64) support_mask_kernel<double><<<g, 256, 0, st>>>((const double*)Om, p, ld, mask, mask_ld);
  else support_mask_kernel<float><<<g, 256, 0, st>>>((const float*)Om, p, ld, mask, mask_ld);
  return cudaGetLastError();
}

cudaError_t launch_identity_stats(double* part, int64_t p, cudaStream_t st) {
  identity_stats_kernel<<<1, 32, 0, st>>>(part, p);
  return cudaGetLastError();
}

cudaError_t launch_decide(Ctrl* ctrl, const double* part, int64_t ntiles, const SolveParams& sp,
                          double* trace, int* bucket_counts, int nbuckets, const double* part_sparse,
                          cudaStream_t st, unsigned long long* delta_entries) {
  decide_kernel<<<1, kRedThreads, 0, st>>>(ctrl, part, ntiles, sp, trace, bucket_counts, nbuckets, part_sparse,
                                           delta_entries);
  return cudaGetLastError();
}

cudaError_t launch_transpose_x_f32(const float* X, int64_t n, int64_t p, float* XT, int64_t ldxt, cudaStream_t st) {
  dim3 grid((unsigned)((p + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  transpose_x_f32_kernel<<<grid, block, 0, st>>>(X, n, p, XT, ldxt);
  return cudaGetLastError();
}

cudaError_t launch_loss_finish(const double* ompart, int64_t nomp, const double* ypart, int64_t nyp,
                               double lam, double lam_d, double inv_n, double* out, cudaStream_t st) {
  loss_finish_kernel<<<1, kRedThreads, 0, st>>>(ompart, nomp, ypart, nyp, lam, lam_d, inv_n, out);
  return cudaGetLastError();
}

cudaError_t launch_batch_ctrl_init(const PathDev& pd, const void* yt0, int is_f64, int64_t p, int64_t ldy,
                                   int64_t s_y, const SolveParams& sp, double L_given, cudaStream_t st) {
  if (pd.nchains < 1 || pd.nchains > 65535) return cudaErrorInvalidValue;
  if (is_f64)
    batch_ctrl_init_kernel<double><<<(unsigned)pd.nchains, kRedThreads, 0, st>>>(pd, (const double*)yt0, p, ldy,
                                                                                   s_y, sp, L_given);
  else
    batch_ctrl_init_kernel<float><<<(unsigned)pd.nchains, kRedThreads, 0, st>>>(pd, (const float*)yt0, p, ldy, s_y,
                                                                                  sp, L_given);
  return cudaGetLastError();
}

cudaError_t launch_post_prox_batch(Ctrl* ctrl, int32_t nprob, const int32_t* active, const int32_t* nactive,
                                   const double* part, int64_t ntiles, const SolveParams& sp, cudaStream_t st) {
  if (nprob < 1 || nprob > 65535) return cudaErrorInvalidValue;
  post_prox_batch_kernel<<<(unsigned)nprob, kRedThreads, 0, st>>>(ctrl, active, nactive, part, ntiles, sp);
  return cudaGetLastError();
}

cudaError_t launch_decide_batch(Ctrl* ctrl, int32_t nprob, const int32_t* active, const int32_t* nactive,
                                const double* part, int64_t ntiles, const SolveParams& sp, int* bucket_counts,
                                int nbuckets, const double* part_sparse, cudaStream_t st) {
  if (nprob < 1 || nprob > 65535) return cudaErrorInvalidValue;
  decide_batch_kernel<<<(unsigned)nprob, kRedThreads, 0, st>>>(ctrl, active, nactive, part, ntiles, sp,
                                                              bucket_counts, nbuckets, part_sparse);
  return cudaGetLastError();
}

cudaError_t launch_path_advance(const PathDev& pd, cudaStream_t st) {
  path_advance_kernel<<<1, 256, 0, st>>>(pd);
  return cudaGetLastError();
}

cudaError_t launch_path_emit(const PathDev& pd, const void* om0, const void* om1, int is_f64, int64_t p,
                             int64_t ldo, int64_t s_om, uint32_t* support, int64_t mask_ld, void* omega_best,
                             cudaStream_t st, const uint32_t* bm0, const uint32_t* bm1, int64_t s_bm) {
  if (pd.nchains < 1 || pd.nchains > 65535) return cudaErrorInvalidValue;
  const dim3 g(64, (unsigned)pd.nchains);
  if (is_f64)
    path_emit_kernel<double><<<g, 256, 0, st>>>(pd, (const double*)om0, (const double*)om1, p, ldo, s_om, support,
                                                mask_ld, (double*)omega_best, nullptr, nullptr, 0, 0);
  else
    path_emit_kernel<float><<<g, 256, 0, st>>>(pd, (const float*)om0, (const float*)om1, p, ldo, s_om, support,
                                               mask_ld, (float*)omega_best, bm0, bm1, bitmap_ld(p), s_bm);
  return cudaGetLastError();
}

}  // namespace accord
