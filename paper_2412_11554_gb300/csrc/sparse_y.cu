// Sparse update of Y = Omega X^T after a prox step (mixed precision modes):
// Y+ = Y + Delta X^T with Delta = Omega+ - Omega.  The iterate is sparse by
// construction (Sec 3.3; the Remark after Thm 3.3 notes that sparsity cuts
// the work of the product), and so is each step Delta, so instead of a dense
// p x p x n product the prox epilogue records the nonzero entries of Delta in
// one bucket per 32-row group and this kernel applies them row by row:
//
//     Y+[i, :] = Y[i, :] + sum_{j : Delta_ij != 0} Delta_ij X^T[j, :]     (FP32)
//
// Entries arrive in any order from many CTAs; each block sorts its bucket by
// (row, column) first, so the sums are formed in a fixed order and the result
// is the same on every run.  The kernel also writes the hi/lo operand planes
// of Y+ (BF16 or TF32: the A operand of the next gradient GEMM) and the
// per-block partial sums
// ||Delta X^T||^2 and ||Y+||^2 for the line search of Algorithm 1.
#include <atomic>
#include <mutex>

#include "internal.h"

namespace accord {
namespace {

constexpr int kThreads = 512;
constexpr int kRowsPerBlock = kBucketRows;
constexpr int kColsPerPass = 256;  // 8 columns a lane per pass

__device__ __forceinline__ void bitonic_sort(uint32_t* key, float* val, int m) {
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int ij = i ^ j;
        if (ij > i) {
          const bool up = (i & k) == 0;
          const uint32_t a = key[i], b = key[ij];
          if ((a > b) == up) {
            key[i] = b;
            key[ij] = a;
            const float t = val[i];
            val[i] = val[ij];
            val[ij] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

// first index in [0, m) whose key >= target (keys sorted ascending)
__device__ __forceinline__ int lower_bound(const uint32_t* key, int m, uint32_t target) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (key[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <int PT>
__global__ void __launch_bounds__(kThreads) sparse_y_kernel(SparseYParams prm) {
  using E = typename Plane<PT>::E;
  int b = blockIdx.y;  // problem slot of a batch (0 for one fit)
  if (prm.active != nullptr) {
    if (b >= *prm.nactive) return;
    b = prm.active[b];
  }
  const Ctrl* ctrl = prm.ctrl + b;
  if (ctrl->done || ctrl->dense || ctrl->ymode || ctrl->refresh) return;
  extern __shared__ uint8_t smem_raw[];
  const int mb = blockIdx.x;  // bucket = 32-row group
  const int cur = ctrl->cur, nxt = cur ^ 1;
  const float* __restrict__ Y = prm.y[cur] + b * prm.s_y;
  float* __restrict__ Yp = prm.yw[nxt] + b * prm.s_y;
  E* __restrict__ Yh = static_cast<E*>(prm.y_hi[nxt]) + b * prm.s_yk;
  E* __restrict__ Yl = static_cast<E*>(prm.y_lo[nxt]) + b * prm.s_yk;
  const float* __restrict__ XT = prm.xt + b * prm.s_xt;
  const int64_t bk = b * prm.s_bkt + mb;  // this problem's bucket

  int cnt = prm.counts[bk];
  if (cnt > prm.cap) cnt = prm.cap;  // overflow is handled by the dense path
  int m = 1;
  while (m < cnt) m <<= 1;
  uint32_t* key = reinterpret_cast<uint32_t*>(smem_raw);
  float* val = reinterpret_cast<float*>(smem_raw + (size_t)prm.cap * sizeof(uint32_t));
  const uint32_t* gk = prm.keys + (size_t)bk * prm.cap;
  const float* gv = prm.vals + (size_t)bk * prm.cap;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    key[i] = i < cnt ? gk[i] : 0xFFFFFFFFu;
    val[i] = i < cnt ? gv[i] : 0.f;
  }
  __syncthreads();
  if (cnt > 1) bitonic_sort(key, val, m);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
  float s_d = 0.f, s_n = 0.f, chk = 0.f;
  for (int rl = warp; rl < kRowsPerBlock; rl += nwarps) {
    const int64_t row = (int64_t)mb * kRowsPerBlock + rl;
    if (row >= prm.p) break;
    const int lo = lower_bound(key, cnt, (uint32_t)rl << 25);
    const int hi = (rl + 1 < kRowsPerBlock) ? lower_bound(key, cnt, (uint32_t)(rl + 1) << 25) : cnt;
    const float* yr = Y + row * prm.ldy;
    float* ypr = Yp + row * prm.ldy;
    E* hr = Yh + row * prm.ldyk;
    E* lr = Yl + row * prm.ldyk;
    for (int64_t c0 = 0; c0 < prm.n; c0 += kColsPerPass) {
      float acc[kColsPerPass / 32];
#pragma unroll
      for (int u = 0; u < kColsPerPass / 32; ++u) acc[u] = 0.f;
      int k = lo;
      if (c0 + kColsPerPass <= prm.n) {
        // four Delta entries at a time: their X^T rows are independent loads,
        // so 32 of them are in flight per lane (the walk is latency-bound)
        for (; k + 4 <= hi; k += 4) {
          float d[4], x[4][kColsPerPass / 32];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int64_t j = key[k + q] & 0x1FFFFFFu;
            d[q] = val[k + q];
            const float* xr = XT + j * prm.ldy + c0 + lane;
#pragma unroll
            for (int u = 0; u < kColsPerPass / 32; ++u) x[q][u] = __ldg(xr + 32 * u);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int u = 0; u < kColsPerPass / 32; ++u) acc[u] = fmaf(d[q], x[q][u], acc[u]);
        }
      }
      for (; k < hi; ++k) {
        const int64_t j = key[k] & 0x1FFFFFFu;
        const float d = val[k];
        const float* xr = XT + j * prm.ldy + c0 + lane;
#pragma unroll
        for (int u = 0; u < kColsPerPass / 32; ++u)
          if (c0 + lane + 32 * u < prm.n) acc[u] = fmaf(d, __ldg(xr + 32 * u), acc[u]);
      }
#pragma unroll
      for (int u = 0; u < kColsPerPass / 32; ++u) {
        const int64_t c = c0 + lane + 32 * u;
        if (c < prm.n) {
          const float yn = yr[c] + acc[u];
          s_d = fmaf(acc[u], acc[u], s_d);
          s_n = fmaf(yn, yn, s_n);
          chk = fmaf(yn, 0.f, chk);
          ypr[c] = yn;
          E h, l;
          Plane<PT>::split(yn, h, l);
          hr[c] = h;
          lr[c] = l;
        }
      }
    }
  }
  // block partial sums: FP32 warp trees, FP64 across warps (fixed order)
  __shared__ double red[kThreads / 32][3];
  s_d = warp_sum_f(s_d);
  s_n = warp_sum_f(s_n);
  const float bad = __ballot_sync(0xffffffffu, chk != 0.f) ? 1.f : 0.f;
  if (lane == 0) {
    red[warp][0] = (double)s_d;
    red[warp][1] = (double)s_n;
    red[warp][2] = (double)bad;
  }
  __syncthreads();
  // one partial row per bucket (the fold reads nbuckets rows)
  if (threadIdx.x < kYSlots) {
    const int q = threadIdx.x;
    double v = 0.0;
    if (q < 3)
      for (int w = 0; w < nwarps; ++w) v += red[w][q];
    prm.part[bk * kYSlots + q] = v;
  }
}

// Dense fallback when a bucket overflowed: planes (type pt) of Delta = Omega+ - Omega.
__global__ void delta_planes_kernel(const Ctrl* ctrl, const float* om0, const float* om1, const uint32_t* bm0,
                                    const uint32_t* bm1, int64_t ldbm, int64_t s_bm, int64_t rows, int64_t p, int64_t ld,
                                    void* hi, void* lo, int64_t ldk, int pt, const int32_t* active,
                                    const int32_t* nactive, int64_t s_om, int64_t s_pl, const int* any_dense) {
  if (any_dense != nullptr && *any_dense == 0) return;
  int b = blockIdx.y;
  if (active != nullptr) {
    if (b >= *nactive) return;
    b = active[b];
  }
  ctrl += b;
  // overflow in bucket mode only: in dense mode the prox epilogue wrote the planes
  if (ctrl->done || !ctrl->dense || ctrl->ymode) return;
  const float* Om = (ctrl->cur ? om1 : om0) + b * s_om;
  const float* Op = (ctrl->cur ? om0 : om1) + b * s_om;
  const uint32_t* Bm = (ctrl->cur ? bm1 : bm0) + b * s_bm;
  const uint32_t* Bp = (ctrl->cur ? bm0 : bm1) + b * s_bm;
  const int64_t total = rows * p;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / p, c = i % p;
    const int64_t wi = (c >> 5) * ldbm + r;
    const uint32_t bit = 1u << (c & 31);
    const float op = (Bp[wi] & bit) ? Op[r * ld + c] : 0.f;
    const float om = (Bm[wi] & bit) ? Om[r * ld + c] : 0.f;
    store_split(hi, lo, b * s_pl + r * ldk + c, op - om, pt);
  }
}

// Y of the current iterate formed afresh (mixed modes).  The sparse and
// dense updates carry Y = Omega X^T forward as Y + Delta X^T in FP32, so
// rounding accumulates over the steps of a fit (and over the penalties of a
// path chain); every few steps, and before a KKT residual under the tolerance
// may end the fit, this kernel recomputes
//
//     Y[i, :] = sum_{j : omega_ij != 0} omega_ij X^T[j, :]               (FP32)
//
// from the nonzeros of Omega^t (its occupancy bitmap), in ascending j, in
// place of Y[cur] and its hi/lo operand planes.  One CTA per 32-row group.
// Its warps first list the group's nonzero columns in shared memory, row by
// row in ascending order: each warp takes a slice of the chunks, and a warp
// load fetches the group's 32 words of a chunk (lane = row, consecutive
// words); the rows' bit counts give each row's start and each slice's start
// within it, and a second read of the words places the columns.  All threads
// then read the values omega_ij of the listed columns.  Then one warp a row:
// the gathers take the row's list four entries at a time (four X^T rows in
// flight per lane) into its output columns held in registers (16 a lane, 512
// a pass).  A group with more nonzeros than the list holds is worked row by
// row instead: the warp lists its row's columns from the row's words (32
// chunks a warp load, eight loads in flight), 512 at a time, and a longer
// row in segments of whole words, in order.  Per 32-row group it writes
// ||Y_old - Y_new||^2 and ||Y_new||^2 for the drift statistic and g.
constexpr int kRfThreads = 256;
constexpr int kRfWarps = kRfThreads / 32;
constexpr int kRfColsPerLane = 16;
constexpr int kRfGroupCap = 4096;                   // nonzeros of a 32-row group listed together
constexpr int kRfListCap = kRfGroupCap / kRfWarps;  // nonzeros of a row listed at once by the row walk
constexpr int kRfGroups = 8;                        // 32-word groups of a row read together by the row walk
constexpr int kRfBatch = 16;                        // chunks of the group's words in flight per warp
constexpr int kRdMaxThreads = 512;

// A dense iterate makes the walk gather one X^T row per entry of Omega;
// from this many nonzeros on (YRefreshParams::dense_nnz, a tenth of the
// entries) the refresh runs as a blocked product instead.  A testing hook
// may fix the form (form 1: the walk, 2: the blocked product).
__device__ __forceinline__ bool refresh_is_dense(const YRefreshParams& prm, const Ctrl& c) {
  if (prm.form == 1) return false;
  if (prm.form == 2) return true;
  return c.nnz >= prm.dense_nnz;
}

// Lists the columns of the row's nonzeros from occupancy word w0 on, in
// ascending order, into col[0 .. len).  Stops before the first word whose
// bits do not all fit in cap entries and returns that word; returns nchunks
// when the row's words ran out.  bmr[c * ldbm] is the row's word of chunk c;
// bits of columns at or past p are not listed.  Warp-uniform; cap >= 32, so
// a segment always takes at least one word.
__device__ __forceinline__ int64_t rf_list(const uint32_t* __restrict__ bmr, int64_t ldbm, int64_t p,
                                           int64_t nchunks, int64_t w0, int cap, uint32_t* col, int& len,
                                           int lane) {
  const uint32_t last_mask = (p & 31) ? (1u << (p & 31)) - 1u : 0xFFFFFFFFu;
  len = 0;
  for (int64_t w = w0; w < nchunks; w += 32 * kRfGroups) {
    uint32_t wd[kRfGroups];
#pragma unroll
    for (int g = 0; g < kRfGroups; ++g) {
      const int64_t c = w + 32 * g + lane;
      wd[g] = c < nchunks ? bmr[c * ldbm] : 0u;
      if (c == nchunks - 1) wd[g] &= last_mask;
    }
#pragma unroll
    for (int g = 0; g < kRfGroups; ++g) {
      const int pc = __popc(wd[g]);
      int incl = pc;  // inclusive scan of the bit counts over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const bool fits = len + incl <= cap;  // true for a prefix of the lanes
      const uint32_t over = __ballot_sync(0xffffffffu, !fits);
      if (fits) {
        uint32_t bits = wd[g];
        int pos = len + incl - pc;
        const uint32_t base = (uint32_t)((w + 32 * g + lane) * 32);
        while (bits != 0u) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1u;
          col[pos++] = base + (uint32_t)b;
        }
      }
      if (over != 0u) {
        const int f = __ffs(over) - 1;
        len += __shfl_sync(0xffffffffu, incl - pc, f);
        return w + 32 * g + f;
      }
      len += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  return nchunks;
}

// val[k] = omega[row, col[k]] for the listed entries, four loads a lane in
// flight; the warp's list writes are visible on entry (__syncwarp).
__device__ __forceinline__ void rf_values(const float* __restrict__ om_row, const uint32_t* col, float* val, int len,
                                          int lane) {
  for (int k0 = 0; k0 < len; k0 += 128) {
    float t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + 32 * q + lane;
      t[q] = k < len ? __ldg(om_row + col[k]) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + 32 * q + lane;
      if (k < len) val[k] = t[q];
    }
  }
}

// acc += v_k X^T[j_k, c0 + lane + 32 u] for the K entries k in order (K <= 4);
// columns at or past n are neither read nor used.
template <int K>
__device__ __forceinline__ void rf_apply(float (&acc)[kRfColsPerLane], const float* __restrict__ XT, int64_t ldx,
                                         int64_t c0, int64_t n, int lane, const uint32_t* col, const float* val) {
  float x[K][kRfColsPerLane];
  float v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    v[k] = val[k];
    const float* xr = XT + (int64_t)col[k] * ldx + c0 + lane;
#pragma unroll
    for (int u = 0; u < kRfColsPerLane; ++u) x[k][u] = (c0 + lane + 32 * u < n) ? __ldg(xr + 32 * u) : 0.f;
  }
#pragma unroll
  for (int u = 0; u < kRfColsPerLane; ++u)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[u] = fmaf(v[k], x[k][u], acc[u]);
}

// acc += the listed entries' terms, in list order
__device__ __forceinline__ void rf_gather(float (&acc)[kRfColsPerLane], const float* __restrict__ XT, int64_t ldx,
                                          int64_t c0, int64_t n, int lane, const uint32_t* col, const float* val,
                                          int len) {
  int k = 0;
  for (; k + 4 <= len; k += 4) rf_apply<4>(acc, XT, ldx, c0, n, lane, col + k, val + k);
  const int r = len - k;
  if (r == 3) rf_apply<3>(acc, XT, ldx, c0, n, lane, col + k, val + k);
  else if (r == 2) rf_apply<2>(acc, XT, ldx, c0, n, lane, col + k, val + k);
  else if (r == 1) rf_apply<1>(acc, XT, ldx, c0, n, lane, col + k, val + k);
}

// Y[row, c0 + lane + 32 u] = acc[u] with its planes, for the columns below n,
// and the drift and norm sums of the group's partial row.
template <int PT>
__device__ __forceinline__ void rf_store(const float (&acc)[kRfColsPerLane], float* __restrict__ yr,
                                         typename Plane<PT>::E* __restrict__ hr, typename Plane<PT>::E* __restrict__ lr,
                                         int64_t c0, int64_t n, int lane, float& s_d, float& s_n, float& chk) {
  using E = typename Plane<PT>::E;
#pragma unroll
  for (int u = 0; u < kRfColsPerLane; ++u) {
    const int64_t c = c0 + lane + 32 * u;
    if (c < n) {
      const float yn = acc[u];
      const float d = yn - yr[c];
      s_d = fmaf(d, d, s_d);
      s_n = fmaf(yn, yn, s_n);
      chk = fmaf(yn, 0.f, chk);
      yr[c] = yn;
      E h, l;
      Plane<PT>::split(yn, h, l);
      hr[c] = h;
      lr[c] = l;
    }
  }
}

// The words of chunks c .. c + kRfBatch (below ce) of one row, lane = row of
// the group: one 128-byte load per chunk for the warp.
__device__ __forceinline__ void rf_group_words(const uint32_t* __restrict__ Bm, int64_t ldbm, int64_t row, bool rok,
                                               int64_t c, int64_t ce, int64_t nchunks, uint32_t last_mask,
                                               uint32_t (&wd)[kRfBatch]) {
#pragma unroll
  for (int q = 0; q < kRfBatch; ++q) {
    const int64_t cc = c + q;
    wd[q] = (rok && cc < ce) ? Bm[cc * ldbm + row] : 0u;
    if (cc == nchunks - 1) wd[q] &= last_mask;
  }
}

template <int PT>
__global__ void __launch_bounds__(kRfThreads, 2) y_refresh_kernel(YRefreshParams prm) {
  using E = typename Plane<PT>::E;
  __shared__ uint32_t s_col[kRfGroupCap];
  __shared__ float s_val[kRfGroupCap];
  __shared__ int s_cnt[kRfWarps][32];
  __shared__ int s_start[33];
  __shared__ double red[kRfWarps][3];
  int b = blockIdx.y;
  if (prm.active != nullptr) {
    if (b >= *prm.nactive) return;
    b = prm.active[b];
  }
  const Ctrl* ctrl = prm.ctrl + b;
  if (ctrl->done || !ctrl->refresh || refresh_is_dense(prm, *ctrl)) return;
  const int cur = ctrl->cur;
  const float* __restrict__ Om = prm.om[cur] + b * prm.s_om;
  const uint32_t* __restrict__ Bm = prm.bm[cur] + b * prm.s_bm;
  float* __restrict__ Y = prm.y[cur] + b * prm.s_y;
  E* __restrict__ Yh = static_cast<E*>(prm.y_hi[cur]) + b * prm.s_yk;
  E* __restrict__ Yl = static_cast<E*>(prm.y_lo[cur]) + b * prm.s_yk;
  const float* __restrict__ XT = prm.xt + b * prm.s_xt;
  const int mb = blockIdx.x;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t nchunks = (prm.p + 31) / 32;
  const int64_t r0 = (int64_t)mb * kBucketRows;
  const uint32_t last_mask = (prm.p & 31) ? (1u << (prm.p & 31)) - 1u : 0xFFFFFFFFu;
  constexpr int kPass = 32 * kRfColsPerLane;
  float s_d = 0.f, s_n = 0.f, chk = 0.f;

  // The group's nonzeros, counted per row (lane) in this warp's slice of the
  // chunks; then each row's start in the group list and each slice's start
  // within the row.
  const int64_t slice = (nchunks + kRfWarps - 1) / kRfWarps;
  const int64_t cb = min(nchunks, (int64_t)warp * slice), ce = min(nchunks, cb + slice);
  const int64_t grow = r0 + lane;
  const bool rok = grow < prm.rows;
  int cnt = 0;
  for (int64_t c = cb; c < ce; c += kRfBatch) {
    uint32_t wd[kRfBatch];
    rf_group_words(Bm, prm.ldbm, grow, rok, c, ce, nchunks, last_mask, wd);
#pragma unroll
    for (int q = 0; q < kRfBatch; ++q) cnt += __popc(wd[q]);
  }
  s_cnt[warp][lane] = cnt;
  __syncthreads();
  if (warp == 0) {
    int run = 0;
    for (int w = 0; w < kRfWarps; ++w) {
      const int t = s_cnt[w][lane];
      s_cnt[w][lane] = run;
      run += t;
    }
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    s_start[lane] = incl - run;
    if (lane == 31) s_start[32] = incl;
  }
  __syncthreads();
  const int total = s_start[32];

  if (total <= kRfGroupCap && prm.list_cap == 0) {
    // The group list: each row's columns in ascending order (the slices are
    // in chunk order, the words in a slice too, the bits of a word too).
    int pos = s_start[lane] + s_cnt[warp][lane];
    for (int64_t c = cb; c < ce; c += kRfBatch) {
      uint32_t wd[kRfBatch];
      rf_group_words(Bm, prm.ldbm, grow, rok, c, ce, nchunks, last_mask, wd);
#pragma unroll
      for (int q = 0; q < kRfBatch; ++q) {
        uint32_t bits = wd[q];
        const uint32_t base = (uint32_t)((c + q) * 32);
        while (bits != 0u) {
          const int bit = __ffs(bits) - 1;
          bits &= bits - 1u;
          s_col[pos++] = base + (uint32_t)bit;
        }
      }
    }
    __syncthreads();
    // the values: entry k belongs to the row r with s_start[r] <= k < s_start[r + 1]
    for (int k = threadIdx.x; k < total; k += kRfThreads) {
      int lo = 0, hi = 32;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_start[mid] <= k) lo = mid;
        else hi = mid;
      }
      s_val[k] = __ldg(Om + (r0 + lo) * prm.ldo + s_col[k]);
    }
    __syncthreads();
    for (int rl = warp; rl < kBucketRows; rl += kRfWarps) {
      const int64_t row = r0 + rl;
      if (row >= prm.rows) break;
      const int k0 = s_start[rl], len = s_start[rl + 1] - k0;
      for (int64_t c0 = 0; c0 < prm.n; c0 += kPass) {
        float acc[kRfColsPerLane];
#pragma unroll
        for (int u = 0; u < kRfColsPerLane; ++u) acc[u] = 0.f;
        rf_gather(acc, XT, prm.ldx, c0, prm.n, lane, s_col + k0, s_val + k0, len);
        rf_store<PT>(acc, Y + row * prm.ldy, Yh + row * prm.ldyk, Yl + row * prm.ldyk, c0, prm.n, lane, s_d, s_n,
                     chk);
      }
    }
  } else {
    // Too many for the group list (or the testing hook asks for it): one
    // warp a row, each with a list of its own in the warp's share of the
    // buffers, worked in segments of whole words when the row does not fit.
    const int cap = (prm.list_cap >= 32 && prm.list_cap <= kRfListCap) ? prm.list_cap : kRfListCap;
    uint32_t* lcol = s_col + warp * kRfListCap;
    float* lval = s_val + warp * kRfListCap;
    for (int rl = warp; rl < kBucketRows; rl += kRfWarps) {
      const int64_t row = r0 + rl;
      if (row >= prm.rows) break;
      const uint32_t* bmr = Bm + row;
      const float* om_row = Om + row * prm.ldo;
      int len = 0;
      __syncwarp();  // the previous row's list has been read
      int64_t wn = rf_list(bmr, prm.ldbm, prm.p, nchunks, 0, cap, lcol, len, lane);
      __syncwarp();
      rf_values(om_row, lcol, lval, len, lane);
      __syncwarp();
      const bool whole = wn >= nchunks;  // the list holds the whole row
      for (int64_t c0 = 0; c0 < prm.n; c0 += kPass) {
        float acc[kRfColsPerLane];
#pragma unroll
        for (int u = 0; u < kRfColsPerLane; ++u) acc[u] = 0.f;
        for (;;) {
          rf_gather(acc, XT, prm.ldx, c0, prm.n, lane, lcol, lval, len);
          if (wn >= nchunks) break;
          // the next segment of the row, from the first word not listed
          __syncwarp();
          wn = rf_list(bmr, prm.ldbm, prm.p, nchunks, wn, cap, lcol, len, lane);
          __syncwarp();
          rf_values(om_row, lcol, lval, len, lane);
          __syncwarp();
        }
        rf_store<PT>(acc, Y + row * prm.ldy, Yh + row * prm.ldyk, Yl + row * prm.ldyk, c0, prm.n, lane, s_d, s_n,
                     chk);
        if (!whole && c0 + kPass < prm.n) {
          // a row worked in segments is listed again from its first word
          __syncwarp();
          wn = rf_list(bmr, prm.ldbm, prm.p, nchunks, 0, cap, lcol, len, lane);
          __syncwarp();
          rf_values(om_row, lcol, lval, len, lane);
          __syncwarp();
        }
      }
    }
  }
  s_d = warp_sum_f(s_d);
  s_n = warp_sum_f(s_n);
  const float bad = __ballot_sync(0xffffffffu, chk != 0.f) ? 1.f : 0.f;
  if (lane == 0) {
    red[warp][0] = (double)s_d;
    red[warp][1] = (double)s_n;
    red[warp][2] = (double)bad;
  }
  __syncthreads();
  if (threadIdx.x < kYSlots) {
    const int q = threadIdx.x;
    double vs = 0.0;
    if (q < 3)
      for (int w = 0; w < kRfWarps; ++w) vs += red[w][q];
    prm.part[b * prm.s_part + (int64_t)mb * kYSlots + q] = vs;
  }
}

// The refresh for a dense iterate: one CTA per 32-row group, thread t owning
// output column c0 + t with the 32 rows' accumulators in registers.  Each
// 32-column chunk of Omega (zeros where its bitmap has no bit) is staged in
// shared memory, XOR-swizzled in 4-float granules, and every thread reads
// its X^T entry of each of the chunk's columns once for all 32 rows.  The
// sums run in ascending column order with zero terms adding exactly 0, so
// the result is bit for bit that of y_refresh_kernel.
template <int PT>
__global__ void __launch_bounds__(kRdMaxThreads) y_refresh_dense_kernel(YRefreshParams prm) {
  using E = typename Plane<PT>::E;
  int b = blockIdx.y;
  if (prm.active != nullptr) {
    if (b >= *prm.nactive) return;
    b = prm.active[b];
  }
  const Ctrl* ctrl = prm.ctrl + b;
  if (ctrl->done || !ctrl->refresh || !refresh_is_dense(prm, *ctrl)) return;
  const int cur = ctrl->cur;
  const float* __restrict__ Om = prm.om[cur] + b * prm.s_om;
  const uint32_t* __restrict__ Bm = prm.bm[cur] + b * prm.s_bm;
  float* __restrict__ Y = prm.y[cur] + b * prm.s_y;
  E* __restrict__ Yh = static_cast<E*>(prm.y_hi[cur]) + b * prm.s_yk;
  E* __restrict__ Yl = static_cast<E*>(prm.y_lo[cur]) + b * prm.s_yk;
  const float* __restrict__ XT = prm.xt + b * prm.s_xt;
  __shared__ __align__(16) float W[32 * 32];  // W[j][r]: Omega[r0 + r][32 c + j]
  __shared__ double red[kRdMaxThreads / 32][3];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int64_t nchunks = (prm.p + 31) / 32;
  float s_d = 0.f, s_n = 0.f, chk = 0.f;
  for (int64_t c0 = 0; c0 < prm.n; c0 += nt) {
    const int64_t col = c0 + tid;
    const bool cok = col < prm.n;
    float acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = 0.f;
    for (int64_t c = 0; c < nchunks; ++c) {
      __syncthreads();  // the last chunk's reads of W are done
      for (int t = tid; t < 1024; t += nt) {
        const int r = t >> 5, j = t & 31;
        const int64_t row = r0 + r, cj = c * 32 + j;
        float v = 0.f;
        if (row < prm.rows && cj < prm.p && ((Bm[c * prm.ldbm + row] >> j) & 1u)) v = Om[row * prm.ldo + cj];
        W[j * 32 + ((((r >> 2) ^ (j & 7))) << 2) + (r & 3)] = v;
      }
      __syncthreads();
      if (cok) {
        const int jn = (int)(prm.p - c * 32 < 32 ? prm.p - c * 32 : 32);
        for (int j = 0; j < jn; ++j) {
          const float x = __ldg(XT + (c * 32 + j) * prm.ldx + col);
          const float4* wj = reinterpret_cast<const float4*>(W + j * 32);
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const float4 w4 = wj[g ^ (j & 7)];
            acc[4 * g + 0] = fmaf(w4.x, x, acc[4 * g + 0]);
            acc[4 * g + 1] = fmaf(w4.y, x, acc[4 * g + 1]);
            acc[4 * g + 2] = fmaf(w4.z, x, acc[4 * g + 2]);
            acc[4 * g + 3] = fmaf(w4.w, x, acc[4 * g + 3]);
          }
        }
      }
    }
    if (cok) {
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const int64_t row = r0 + r;
        if (row < prm.rows) {
          float* yp = Y + row * prm.ldy + col;
          const float yn = acc[r];
          const float d = yn - *yp;
          s_d = fmaf(d, d, s_d);
          s_n = fmaf(yn, yn, s_n);
          chk = fmaf(yn, 0.f, chk);
          *yp = yn;
          E h, l;
          Plane<PT>::split(yn, h, l);
          Yh[row * prm.ldyk + col] = h;
          Yl[row * prm.ldyk + col] = l;
        }
      }
    }
  }
  s_d = warp_sum_f(s_d);
  s_n = warp_sum_f(s_n);
  const float bad = __ballot_sync(0xffffffffu, chk != 0.f) ? 1.f : 0.f;
  if (lane == 0) {
    red[warp][0] = (double)s_d;
    red[warp][1] = (double)s_n;
    red[warp][2] = (double)bad;
  }
  __syncthreads();
  if (tid < kYSlots) {
    double v = 0.0;
    if (tid < 3)
      for (int w = 0; w < (nt >> 5); ++w) v += red[w][tid];
    prm.part[b * prm.s_part + (int64_t)blockIdx.x * kYSlots + tid] = v;
  }
}

}  // namespace

size_t sparse_y_smem_bytes(int cap) { return (size_t)cap * (sizeof(uint32_t) + sizeof(float)); }

cudaError_t sparse_y_prepare() {
  static std::mutex mu;
  static int configured = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (configured != dev) {
    e = cudaFuncSetAttribute(sparse_y_kernel<kPlaneBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sparse_y_kernel<kPlaneTf32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  return cudaSuccess;
}

cudaError_t launch_sparse_y(const SparseYParams& prm, cudaStream_t st) {
  const size_t smem = sparse_y_smem_bytes(prm.cap);
  cudaError_t e = sparse_y_prepare();
  if (e != cudaSuccess) return e;
  if (smem > 64 * 1024) return cudaErrorInvalidValue;
  const unsigned nb = (unsigned)(prm.nprob > 1 ? prm.nprob : 1);
  if (nb > 65535u) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)prm.tiles_m, nb);
  if (prm.ptype == kPlaneTf32) sparse_y_kernel<kPlaneTf32><<<grid, kThreads, smem, st>>>(prm);
  else sparse_y_kernel<kPlaneBf16><<<grid, kThreads, smem, st>>>(prm);
  return cudaGetLastError();
}

static std::atomic<int> g_rf_list_cap{0};
static std::atomic<int> g_rf_form{0};

void y_refresh_set_test(int list_cap, int form) {
  g_rf_list_cap.store(list_cap);
  g_rf_form.store(form);
}

cudaError_t launch_y_refresh(const YRefreshParams& prm_in, cudaStream_t st) {
  YRefreshParams prm = prm_in;
  prm.list_cap = g_rf_list_cap.load();
  prm.form = g_rf_form.load();
  const unsigned nb = (unsigned)(prm.nprob > 1 ? prm.nprob : 1);
  if (nb > 65535u) return cudaErrorInvalidConfiguration;
  const int64_t groups = (prm.rows + kBucketRows - 1) / kBucketRows;
  if (groups < 1 || groups > 2147483647LL) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)groups, nb);
  // both forms are launched; each problem's nonzero count picks the one that works
  const int64_t nd = (prm.n + 31) / 32 * 32;
  const unsigned td = (unsigned)(nd < kRdMaxThreads ? nd : kRdMaxThreads);
  if (prm.ptype == kPlaneTf32) {
    y_refresh_kernel<kPlaneTf32><<<grid, kRfThreads, 0, st>>>(prm);
    y_refresh_dense_kernel<kPlaneTf32><<<grid, td, 0, st>>>(prm);
  } else {
    y_refresh_kernel<kPlaneBf16><<<grid, kRfThreads, 0, st>>>(prm);
    y_refresh_dense_kernel<kPlaneBf16><<<grid, td, 0, st>>>(prm);
  }
  return cudaGetLastError();
}

cudaError_t launch_delta_planes(const Ctrl* ctrl, const float* om0, const float* om1, const uint32_t* bm0,
                                const uint32_t* bm1, int64_t p, int64_t ld, void* hi, void* lo, int64_t ldk, int pt,
                                cudaStream_t st, int32_t nprob, const int32_t* active, const int32_t* nactive,
                                int64_t s_om, int64_t s_pl, const int* any_dense, int64_t s_bm, int64_t rows) {
  const unsigned nb = (unsigned)(nprob > 1 ? nprob : 1);
  if (nb > 65535u) return cudaErrorInvalidConfiguration;
  if (rows < 0) rows = p;
  const unsigned gx = nb > 1 ? 152u * 16u / nb + 1u : 152u * 16u;
  delta_planes_kernel<<<dim3(gx, nb), 256, 0, st>>>(ctrl, om0, om1, bm0, bm1, bitmap_ld(rows), s_bm, rows, p, ld, hi,
                                                    lo, ldk, pt, active, nactive, s_om, s_pl, any_dense);
  return cudaGetLastError();
}

}  // namespace accord
