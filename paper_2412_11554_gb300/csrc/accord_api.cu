// C ABI of libaccord (include/accord.h): argument checks, workspace layout,
// setup (conversions, Omega^0, Y^0 = Omega^0 X^T, L = sigma_max(S)) and the
// launch loop of Algorithm 1.  All arithmetic happens in the kernels; the host
// only queues launches and reads the device control block to learn when the
// fit has finished.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "accord.h"
#include "api_util.h"
#include "internal.h"
#include "tc_gemm.h"

namespace accord {

static thread_local char g_last_error[256] = "";

void set_last_error(const char* where, int line, const char* what) {
  if (g_last_error[0] != 0) return;  // keep the first failure
  const char* base = where;
  for (const char* c = where; *c; ++c)
    if (*c == '/') base = c + 1;
  std::snprintf(g_last_error, sizeof(g_last_error), "%s:%d: %s", base, line, what);
}

void clear_last_error() { g_last_error[0] = 0; }

namespace {

// Byte offsets of every sub-buffer of the fit workspace.
struct Layout {
  bool f64 = true;
  int64_t n = 0, p = 0;
  int64_t rows = 0, row0 = 0;  // the block of rows of Omega this fit owns (all p rows: 0, p)
  int64_t ldo = 0;   // Omega (elements)
  int64_t ldy = 0;   // Y (elements)
  int pt = kPlaneBf16;  // operand-plane type of the mixed modes
  int64_t ldk = 0;   // operand planes whose columns run over p
  int64_t ldyk = 0;  // operand planes whose columns run over n
  int64_t tiles_prox = 0, tiles_y = 0, trace_rows = 0;
  size_t ctrl = 0, trace = 0, part_prox = 0, part_y = 0, part_om = 0, bad = 0, part_fold = 0, dent = 0;
  size_t xsum = 0;  // row blocks: this block's trial sums, then the sums over all blocks
  size_t om[2] = {0, 0}, y[2] = {0, 0};
  size_t x64 = 0, xt64 = 0;                        // FP64 mode
  size_t om_hi = 0, om_lo = 0, y_hi[2] = {0, 0}, y_lo[2] = {0, 0};
  size_t bm[2] = {0, 0};                           // occupancy bitmaps of the iterate buffers
  size_t x_hi = 0, x_lo = 0, xt_hi = 0, xt_lo = 0;  // mixed modes
  size_t gram = 0, lz_v = 0, lz_w = 0, lz_a = 0, lz_b = 0;
  size_t mask = 0;
  int64_t mask_ld = 0;  // 32-bit words per row of the refit support mask
  int lz_k = 0;
  // sparse Delta update (mixed modes)
  bool sparse = false;
  int64_t nbuckets = 0;
  size_t xt32 = 0, bkt_keys = 0, bkt_vals = 0, bkt_cnt = 0, part_sy = 0;
  size_t total = 0;
};


// rows < 0: the whole matrix (rows = p, row0 = 0); else the block of rows
// row0 .. row0 + rows of Omega.  X and X^T are always whole.
Layout make_layout(int64_t n, int64_t p, int precision, int max_iter, int lanczos_max, bool sparse,
                   int64_t rows = -1, int64_t row0 = 0) {
  Layout L;
  const bool f64 = precision == ACCORD_FP64;
  L.f64 = f64;
  L.pt = plane_type(precision);
  const size_t pe = plane_bytes(L.pt);
  L.n = n;
  L.p = p;
  L.rows = rows < 0 ? p : rows;
  L.row0 = rows < 0 ? 0 : row0;
  const int64_t m = L.rows;
  L.ldo = round_up(p, 8);
  L.ldy = round_up(n, 8);
  L.ldk = round_up(p, 8);
  L.ldyk = round_up(n, 8);
  L.tiles_prox = f64 ? gemm_f64_tiles(m, p) : tc_tiles(m, p);
  const int64_t ty = f64 ? gemm_f64_tiles(m, n) : tc_tiles(m, n);
  const int64_t tg = f64 ? gemm_f64_tiles(n, n) : tc_tiles(n, n);
  L.tiles_y = ty > tg ? ty : tg;
  L.trace_rows = (int64_t)max_iter + 2;
  const size_t es = f64 ? 8 : 4;
  size_t c = 0;
  L.ctrl = take(c, sizeof(Ctrl));
  L.bad = take(c, 64);
  L.dent = take(c, 64);  // Delta entries applied by the sparse Y update (a counter)
  L.trace = take(c, (size_t)L.trace_rows * kTraceFields * 8);
  L.part_prox = take(c, (size_t)L.tiles_prox * kProxSlots * 8);
  L.part_y = take(c, (size_t)L.tiles_y * kProxSlots * 8);
  L.part_om = take(c, (size_t)m * kProxSlots * 8);
  L.part_fold = take(c, (size_t)kFoldChunks * kProxSlots * 8);
  L.xsum = take(c, (size_t)2 * (kProxSlots + kYSlots) * 8);
  for (int b = 0; b < 2; ++b) L.om[b] = take(c, (size_t)m * L.ldo * es);
  if (f64) {
    for (int b = 0; b < 2; ++b) L.y[b] = take(c, (size_t)m * L.ldy * 8);
    L.x64 = take(c, (size_t)n * L.ldo * 8);
    L.xt64 = take(c, (size_t)p * L.ldy * 8);
  } else {
    for (int b = 0; b < 2; ++b) L.y[b] = take(c, (size_t)m * L.ldy * 4);
    for (int b = 0; b < 2; ++b) L.bm[b] = take(c, (size_t)bitmap_words(m, p) * 4);
    L.om_hi = take(c, (size_t)m * L.ldk * pe);
    L.om_lo = take(c, (size_t)m * L.ldk * pe);
    for (int b = 0; b < 2; ++b) {
      L.y_hi[b] = take(c, (size_t)m * L.ldyk * pe);
      L.y_lo[b] = take(c, (size_t)m * L.ldyk * pe);
    }
    L.x_hi = take(c, (size_t)n * L.ldk * pe);
    L.x_lo = take(c, (size_t)n * L.ldk * pe);
    L.xt_hi = take(c, (size_t)p * L.ldyk * pe);
    L.xt_lo = take(c, (size_t)p * L.ldyk * pe);
    L.sparse = sparse;
    // X^T in FP32 and one partial row per 32-row group: the sparse update and
    // the refresh of Y (both Y update forms carry Y forward in FP32)
    L.nbuckets = (m + kBucketRows - 1) / kBucketRows;
    L.xt32 = take(c, (size_t)p * L.ldy * 4);
    L.part_sy = take(c, (size_t)L.nbuckets * kYSlots * 8);
    if (sparse) {
      L.bkt_keys = take(c, (size_t)L.nbuckets * kBucketCap * 4);
      L.bkt_vals = take(c, (size_t)L.nbuckets * kBucketCap * 4);
      L.bkt_cnt = take(c, (size_t)L.nbuckets * 4);
    }
  }
  L.mask_ld = (p + 31) / 32;
  L.mask = take(c, (size_t)m * L.mask_ld * 4);
  L.gram = take(c, (size_t)n * n * 8);
  int64_t k = lanczos_max < kLanczosMax ? lanczos_max : kLanczosMax;
  if (k > n) k = n;
  if (k < 1) k = 1;
  L.lz_k = (int)k;
  L.lz_v = take(c, (size_t)(k + 1) * n * 8);
  L.lz_w = take(c, (size_t)n * 8);
  L.lz_a = take(c, (size_t)k * 8);
  L.lz_b = take(c, (size_t)k * 8);
  L.total = c;
  return L;
}

// The sparse Delta update runs in the mixed modes; bucket keys hold a column index
// in 25 bits.
bool use_sparse(const accord_opts& o, int64_t p) {
  return o.precision != ACCORD_FP64 && o.sparse_update != 0 && p < (1 << 25) - 1;
}

// Device GEMM wrappers that pick the precision's kernel family.
struct Plan {
  Layout L;
  void* ws;
  cudaStream_t st;
  Ctrl* ctrl;
  int* err;
};

// Y^(b) = Omega^(src) X^T for setup (no control block).  Partials -> part_y.
int setup_y(const Plan& P, int src, int dst) {
  const Layout& L = P.L;
  void* ws = P.ws;
  if (L.f64) {
    GemmF64Params g{};
    g.ctrl = nullptr;
    g.A[0] = g.A[1] = at<double>(ws, L.om[src]);
    g.lda = L.ldo;
    g.B = at<double>(ws, L.x64);
    g.ldb = L.ldo;
    g.M = L.rows; g.N = L.n; g.K = L.p;
    g.out[0] = g.out[1] = at<double>(ws, L.y[dst]);
    g.ldout = L.ldy;
    g.aux[0] = g.aux[1] = nullptr;
    g.part = at<double>(ws, L.part_y);
    g.scale = 1.0;
    ACCORD_CK(launch_gemm_f64(kModeY, g, P.st));
    return kOk;
  }
  ACCORD_CK(launch_split_planes(at<float>(ws, L.om[src]), L.rows, L.p, L.ldo, at<void>(ws, L.om_hi),
                                at<void>(ws, L.om_lo), L.ldk, L.pt, P.st));
  TcParams t{};
  if (!encode_plane_map(&t.a_hi[0], at<void>(ws, L.om_hi), L.pt, L.rows, L.p, L.ldk, 128) ||
      !encode_plane_map(&t.a_lo[0], at<void>(ws, L.om_lo), L.pt, L.rows, L.p, L.ldk, 128) ||
      !encode_plane_map(&t.b_hi, at<void>(ws, L.x_hi), L.pt, L.n, L.p, L.ldk, tc_box_n()) ||
      !encode_plane_map(&t.b_lo, at<void>(ws, L.x_lo), L.pt, L.n, L.p, L.ldk, tc_box_n()))
    return kEcuda;
  t.a_hi[1] = t.a_hi[0];
  t.a_lo[1] = t.a_lo[0];
  t.ctrl = nullptr;
  t.err = P.err;
  tc_shape(t, L.rows, L.n, L.p, L.pt);
  t.out[0] = t.out[1] = at<float>(ws, L.y[dst]);
  t.ldout = L.ldy;
  t.out_hi[0] = t.out_hi[1] = at<void>(ws, L.y_hi[dst]);
  t.out_lo[0] = t.out_lo[1] = at<void>(ws, L.y_lo[dst]);
  t.ldplane = L.ldyk;
  t.aux[0] = t.aux[1] = nullptr;
  t.part = at<double>(ws, L.part_y);
  t.scale = 1.f;
  ACCORD_CK(launch_tc_gemm(kModeY, t, P.st));
  return kOk;
}

// K = X X^T / n into the FP64 Gram buffer.
int setup_gram(const Plan& P) {
  const Layout& L = P.L;
  void* ws = P.ws;
  if (L.f64) {
    GemmF64Params g{};
    g.A[0] = g.A[1] = at<double>(ws, L.x64);
    g.lda = L.ldo;
    g.B = at<double>(ws, L.x64);
    g.ldb = L.ldo;
    g.M = L.n; g.N = L.n; g.K = L.p;
    g.out[0] = g.out[1] = at<double>(ws, L.gram);
    g.ldout = L.n;
    g.scale = 1.0 / (double)L.n;
    ACCORD_CK(launch_gemm_f64(kModeGram, g, P.st));
    return kOk;
  }
  TcParams t{};
  if (!encode_plane_map(&t.a_hi[0], at<void>(ws, L.x_hi), L.pt, L.n, L.p, L.ldk, 128) ||
      !encode_plane_map(&t.a_lo[0], at<void>(ws, L.x_lo), L.pt, L.n, L.p, L.ldk, 128) ||
      !encode_plane_map(&t.b_hi, at<void>(ws, L.x_hi), L.pt, L.n, L.p, L.ldk, tc_box_n()) ||
      !encode_plane_map(&t.b_lo, at<void>(ws, L.x_lo), L.pt, L.n, L.p, L.ldk, tc_box_n()))
    return kEcuda;
  t.a_hi[1] = t.a_hi[0];
  t.a_lo[1] = t.a_lo[0];
  t.err = P.err;
  tc_shape(t, L.n, L.n, L.p, L.pt);
  t.out64 = at<double>(ws, L.gram);
  t.ldout64 = L.n;
  t.scale = 1.f / (float)L.n;
  ACCORD_CK(launch_tc_gemm(kModeGram, t, P.st));
  return kOk;
}

// Per-trial launch parameters, fixed for the whole fit (buffer choice is made
// on the device from ctrl->cur).
struct TrialPlan {
  GemmF64Params g2{}, g1{};
  TcParams t2{}, t1{};
  SparseYParams sy{};
  SolveParams sp{};
  YRefreshParams rf{};
  bool refresh = false;  // mixed modes with sp.y_refresh > 0: the refresh kernels open every trial
  int update_g = 1;      // a whole fit (0 for a row block: its ||Y||^2 covers its rows only)
};

int make_trial_plan(const Plan& P, TrialPlan& T, double lam, double lam_d) {
  const Layout& L = P.L;
  void* ws = P.ws;
  if (L.f64) {
    // prox GEMM: G = Y[cur] XT^T / n, Omega[cur] -> Omega[nxt]
    GemmF64Params& g2 = T.g2;
    g2.ctrl = P.ctrl;
    g2.A[0] = at<double>(ws, L.y[0]);
    g2.A[1] = at<double>(ws, L.y[1]);
    g2.a_nxt = 0;
    g2.lda = L.ldy;
    g2.B = at<double>(ws, L.xt64);
    g2.ldb = L.ldy;
    g2.M = L.rows; g2.N = L.p; g2.K = L.n;
    g2.row_off = L.row0;
    g2.out[0] = at<double>(ws, L.om[0]);
    g2.out[1] = at<double>(ws, L.om[1]);
    g2.ldout = L.ldo;
    g2.aux[0] = at<double>(ws, L.om[0]);
    g2.aux[1] = at<double>(ws, L.om[1]);
    g2.ldaux = L.ldo;
    g2.part = at<double>(ws, L.part_prox);
    g2.lam = lam; g2.lam_d = lam_d;
    g2.scale = 1.0 / (double)L.n;
    // GEMM1: Y[nxt] = Omega[nxt] X^T, old Y[cur] for the difference
    GemmF64Params& g1 = T.g1;
    g1.ctrl = P.ctrl;
    g1.A[0] = at<double>(ws, L.om[0]);
    g1.A[1] = at<double>(ws, L.om[1]);
    g1.a_nxt = 1;
    g1.lda = L.ldo;
    g1.B = at<double>(ws, L.x64);
    g1.ldb = L.ldo;
    g1.M = L.rows; g1.N = L.n; g1.K = L.p;
    g1.out[0] = at<double>(ws, L.y[0]);
    g1.out[1] = at<double>(ws, L.y[1]);
    g1.ldout = L.ldy;
    g1.aux[0] = at<double>(ws, L.y[0]);
    g1.aux[1] = at<double>(ws, L.y[1]);
    g1.ldaux = L.ldy;
    g1.part = at<double>(ws, L.part_y);
    g1.scale = 1.0;
    return kOk;
  }
  TcParams& t2 = T.t2;
  for (int b = 0; b < 2; ++b) {
    if (!encode_plane_map(&t2.a_hi[b], at<void>(ws, L.y_hi[b]), L.pt, L.rows, L.n, L.ldyk, 128) ||
        !encode_plane_map(&t2.a_lo[b], at<void>(ws, L.y_lo[b]), L.pt, L.rows, L.n, L.ldyk, 128))
      return kEcuda;
  }
  if (!encode_plane_map(&t2.b_hi, at<void>(ws, L.xt_hi), L.pt, L.p, L.n, L.ldyk, tc_box_n()) ||
      !encode_plane_map(&t2.b_lo, at<void>(ws, L.xt_lo), L.pt, L.p, L.n, L.ldyk, tc_box_n()))
    return kEcuda;
  t2.ctrl = P.ctrl;
  t2.err = P.err;
  t2.a_nxt = 0;
  tc_shape(t2, L.rows, L.p, L.n, L.pt);
  t2.row_off = L.row0;
  t2.out[0] = at<float>(ws, L.om[0]);
  t2.out[1] = at<float>(ws, L.om[1]);
  t2.ldout = L.ldo;
  t2.out_hi[0] = t2.out_hi[1] = at<void>(ws, L.om_hi);
  t2.out_lo[0] = t2.out_lo[1] = at<void>(ws, L.om_lo);
  t2.ldplane = L.ldk;
  t2.aux[0] = at<float>(ws, L.om[0]);
  t2.aux[1] = at<float>(ws, L.om[1]);
  t2.ldaux = L.ldo;
  t2.part = at<double>(ws, L.part_prox);
  t2.lam = (float)lam;
  t2.lam_d = (float)lam_d;
  t2.scale = (float)(1.0 / (double)L.n);
  t2.bm[0] = at<uint32_t>(ws, L.bm[0]);
  t2.bm[1] = at<uint32_t>(ws, L.bm[1]);
  t2.ldbm = bitmap_ld(L.rows);
  t2.s_bm = 0;

  TcParams& t1 = T.t1;
  if (!encode_plane_map(&t1.a_hi[0], at<void>(ws, L.om_hi), L.pt, L.rows, L.p, L.ldk, 128) ||
      !encode_plane_map(&t1.a_lo[0], at<void>(ws, L.om_lo), L.pt, L.rows, L.p, L.ldk, 128) ||
      !encode_plane_map(&t1.b_hi, at<void>(ws, L.x_hi), L.pt, L.n, L.p, L.ldk, tc_box_n()) ||
      !encode_plane_map(&t1.b_lo, at<void>(ws, L.x_lo), L.pt, L.n, L.p, L.ldk, tc_box_n()))
    return kEcuda;
  t1.a_hi[1] = t1.a_hi[0];
  t1.a_lo[1] = t1.a_lo[0];
  t1.ctrl = P.ctrl;
  t1.err = P.err;
  t1.a_nxt = 1;
  tc_shape(t1, L.rows, L.n, L.p, L.pt);
  t1.out[0] = at<float>(ws, L.y[0]);
  t1.out[1] = at<float>(ws, L.y[1]);
  t1.ldout = L.ldy;
  for (int b = 0; b < 2; ++b) {
    t1.out_hi[b] = at<void>(ws, L.y_hi[b]);
    t1.out_lo[b] = at<void>(ws, L.y_lo[b]);
  }
  t1.ldplane = L.ldyk;
  t1.aux[0] = at<float>(ws, L.y[0]);
  t1.aux[1] = at<float>(ws, L.y[1]);
  t1.ldaux = L.ldy;
  t1.part = at<double>(ws, L.part_y);
  t1.scale = 1.f;
  if (L.sparse) {
    // prox epilogue fills the Delta buckets; the dense Y GEMM only runs when
    // one of them overflowed (its Delta planes then come from delta_planes)
    t2.keys = at<uint32_t>(ws, L.bkt_keys);
    t2.vals = at<float>(ws, L.bkt_vals);
    t2.counts = at<int>(ws, L.bkt_cnt);
    t2.dense_flag = &P.ctrl->dense;
    t2.cap = kBucketCap;
    t1.gate_dense = 1;
    SparseYParams& sy = T.sy;
    sy.ctrl = P.ctrl;
    for (int b = 0; b < 2; ++b) {
      sy.y[b] = at<float>(ws, L.y[b]);
      sy.yw[b] = at<float>(ws, L.y[b]);
      sy.y_hi[b] = at<void>(ws, L.y_hi[b]);
      sy.y_lo[b] = at<void>(ws, L.y_lo[b]);
    }
    sy.xt = at<float>(ws, L.xt32);
    sy.keys = at<uint32_t>(ws, L.bkt_keys);
    sy.vals = at<float>(ws, L.bkt_vals);
    sy.counts = at<int>(ws, L.bkt_cnt);
    sy.cap = kBucketCap;
    sy.tiles_m = (int32_t)L.nbuckets;
    sy.tiles_n = t1.tiles_n;
    sy.p = L.rows;
    sy.n = L.n;
    sy.ldy = L.ldy;
    sy.ldyk = L.ldyk;
    sy.part = at<double>(ws, L.part_sy);
    sy.ptype = L.pt;
  }
  YRefreshParams& rf = T.rf;
  rf.ctrl = P.ctrl;
  for (int b = 0; b < 2; ++b) {
    rf.om[b] = at<float>(ws, L.om[b]);
    rf.bm[b] = at<uint32_t>(ws, L.bm[b]);
    rf.y[b] = at<float>(ws, L.y[b]);
    rf.y_hi[b] = at<void>(ws, L.y_hi[b]);
    rf.y_lo[b] = at<void>(ws, L.y_lo[b]);
  }
  rf.xt = at<float>(ws, L.xt32);
  rf.rows = L.rows;
  rf.p = L.p;
  rf.n = L.n;
  rf.ldo = L.ldo;
  rf.ldbm = bitmap_ld(L.rows);
  rf.ldy = L.ldy;
  rf.ldyk = L.ldyk;
  rf.ldx = L.ldy;
  rf.part = at<double>(ws, L.part_sy);
  rf.ptype = L.pt;
  rf.nprob = 1;
  // the blocked form from a tenth of the entries on: there its FP32 FMAs
  // (~3e13/s) beat one 4n-byte gather per nonzero (~6e12 B/s)
  rf.dense_nnz = 0.1 * (double)L.p * (double)L.p;
  return kOk;
}

// Optional per-launch CUDA events around the two GEMMs of every trial.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> prox, y;  // start/stop pairs in launch order
  ~Profiler() {
    for (auto e : prox) cudaEventDestroy(e);
    for (auto e : y) cudaEventDestroy(e);
  }
  cudaError_t mark(std::vector<cudaEvent_t>& v, cudaStream_t st) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    v.push_back(e);
    return cudaEventRecord(e, st);
  }
  // summed duration of the first `count` launches
  double total_ms(const std::vector<cudaEvent_t>& v, int64_t count) const {
    double t = 0.0;
    for (int64_t i = 0; i < count && 2 * i + 1 < (int64_t)v.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, v[2 * i], v[2 * i + 1]) == cudaSuccess) t += ms;
    }
    return t;
  }
};

// One trial of Algorithm 1.  exchange (a row block of the fit): the
// decisions wait for the sums over all blocks, so the trial ends with this
// block's sums folded into the exchange buffer (the caller exchanges them and
// launches launch_decide_global) instead of with post_prox and decide.
int launch_trial(const Plan& P, const TrialPlan& T, Profiler& prof, int64_t& nlaunch, bool exchange = false) {
  const Layout& L = P.L;
  double* trace = at<double>(P.ws, L.trace);
  if (T.refresh) {
    // Y of Omega^t formed afresh when the last decision asked for it (both
    // kernels return at once otherwise)
    ACCORD_CK(launch_y_refresh(T.rf, P.st));
    ACCORD_CK(launch_y_refresh_fold(P.ctrl, 1, nullptr, nullptr, at<double>(P.ws, L.part_sy), L.nbuckets, 0,
                                    T.update_g, P.st));
    nlaunch += 3;
  }
  if (prof.on) ACCORD_CK(prof.mark(prof.prox, P.st));
  if (L.f64) ACCORD_CK(launch_gemm_f64(kModeProx, T.g2, P.st));
  else ACCORD_CK(launch_tc_gemm(kModeProx, T.t2, P.st));
  if (prof.on) ACCORD_CK(prof.mark(prof.prox, P.st));
  if (!exchange)
    ACCORD_CK(launch_post_prox(P.ctrl, at<double>(P.ws, L.part_prox), L.tiles_prox, T.sp, trace,
                               at<double>(P.ws, L.part_fold), P.st));
  const int64_t ty = L.f64 ? gemm_f64_tiles(L.rows, L.n) : tc_tiles(L.rows, L.n);
  if (prof.on) ACCORD_CK(prof.mark(prof.y, P.st));
  if (L.f64) {
    ACCORD_CK(launch_gemm_f64(kModeY, T.g1, P.st));
  } else if (L.sparse) {
    // Y+ = Y + Delta X^T: sparse update, or the dense fallback when a bucket
    // overflowed (each kernel checks ctrl->dense and exits when not its turn)
    ACCORD_CK(launch_delta_planes(P.ctrl, at<float>(P.ws, L.om[0]), at<float>(P.ws, L.om[1]),
                                  at<uint32_t>(P.ws, L.bm[0]), at<uint32_t>(P.ws, L.bm[1]), L.p, L.ldo,
                                  at<void>(P.ws, L.om_hi), at<void>(P.ws, L.om_lo), L.ldk, L.pt, P.st, 1,
                                  nullptr, nullptr, 0, 0, nullptr, 0, L.rows));
    ACCORD_CK(launch_tc_gemm(kModeY, T.t1, P.st));
    ACCORD_CK(launch_sparse_y(T.sy, P.st));
    nlaunch += 2;
  } else {
    ACCORD_CK(launch_tc_gemm(kModeY, T.t1, P.st));
  }
  if (prof.on) ACCORD_CK(prof.mark(prof.y, P.st));
  if (exchange) {
    ACCORD_CK(launch_fold_block(P.ctrl, at<double>(P.ws, L.part_prox), L.tiles_prox, at<double>(P.ws, L.part_fold),
                                at<double>(P.ws, L.part_y), ty, L.sparse ? at<int>(P.ws, L.bkt_cnt) : nullptr,
                                L.sparse ? (int)L.nbuckets : 0, L.sparse ? at<double>(P.ws, L.part_sy) : nullptr,
                                L.sparse ? at<unsigned long long>(P.ws, L.dent) : nullptr,
                                at<double>(P.ws, L.xsum), P.st));
  } else {
    ACCORD_CK(launch_decide(P.ctrl, at<double>(P.ws, L.part_y), ty, T.sp, trace,
                            L.sparse ? at<int>(P.ws, L.bkt_cnt) : nullptr, L.sparse ? (int)L.nbuckets : 0,
                            L.sparse ? at<double>(P.ws, L.part_sy) : nullptr, P.st,
                            L.sparse ? at<unsigned long long>(P.ws, L.dent) : nullptr));
  }
  nlaunch += 4;
  return kOk;
}

int read_ctrl(const Plan& P, Ctrl* host) {
  ACCORD_CK(cudaMemcpyAsync(host, P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, P.st));
  ACCORD_CK(cudaStreamSynchronize(P.st));
  return kOk;
}

// A row block of a fit: rows row0 .. row0 + rows of Omega, and the caller's
// exchange of Algorithm 1's sums over all blocks of the partition.
struct RowBlock {
  int64_t row0, rows;
  accord_exchange_fn fn;
  void* ctx;
};

// The exchange of one block: its folded sums (xsum[0 .. 11]: the kProxSlots
// prox slots, then the kYSlots Y slots) go to the caller as 9 sums and one
// maximum (the KKT residual); the sums over all blocks come back into
// xsum[12 .. 23] in the same layout.  A block whose own kernels reported a
// device error adds one to the exchanged bad count, so that every block
// stops at the same trial.
int exchange_sums(const Plan& P, const RowBlock& rb, int dev_error) {
  double h[2 * (kProxSlots + kYSlots)];
  double* xs = at<double>(P.ws, P.L.xsum);
  ACCORD_CK(cudaMemcpyAsync(h, xs, (kProxSlots + kYSlots) * sizeof(double), cudaMemcpyDeviceToHost, P.st));
  ACCORD_CK(cudaStreamSynchronize(P.st));
  double sums[9] = {h[kPDelta2], h[kPLogDiag], h[kPDiagSum], h[kPL1Off], h[kPNnz], h[kPBad] + (dev_error ? 1.0 : 0.0),
                    h[kProxSlots + kYDiff2], h[kProxSlots + kYNorm2], h[kProxSlots + kYBad]};
  double maxes[1] = {h[kPKkt]};
  if (rb.fn(sums, 9, maxes, 1, rb.ctx) != 0) {
    set_last_error(__FILE__, __LINE__, "the exchange callback failed");
    return kEcuda;
  }
  double* g = h + kProxSlots + kYSlots;
  for (int q = 0; q < kProxSlots + kYSlots; ++q) g[q] = 0.0;
  g[kPDelta2] = sums[0];
  g[kPLogDiag] = sums[1];
  g[kPDiagSum] = sums[2];
  g[kPL1Off] = sums[3];
  g[kPNnz] = sums[4];
  g[kPBad] = sums[5];
  g[kPKkt] = maxes[0];
  g[kProxSlots + kYDiff2] = sums[6];
  g[kProxSlots + kYNorm2] = sums[7];
  g[kProxSlots + kYBad] = sums[8];
  ACCORD_CK(cudaMemcpyAsync(xs + kProxSlots + kYSlots, g, (kProxSlots + kYSlots) * sizeof(double),
                            cudaMemcpyHostToDevice, P.st));
  ACCORD_CK(cudaStreamSynchronize(P.st));
  return kOk;
}

int fit_impl(const float* X32, const double* X64in, int64_t n, int64_t p, double lam, const accord_opts* optp,
             void* Omega, void* workspace, size_t ws_bytes, accord_stats* out, const void* support = nullptr,
             double phi = 1.0, const RowBlock* rb = nullptr) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (out) std::memset(out, 0, sizeof(*out));
  if ((X32 == nullptr && X64in == nullptr) || Omega == nullptr || n < 1 || p < 1 || !(lam >= 0.0) ||
      !std::isfinite(lam))
    return kEinval;
  if (int e = check_opts(o)) return e;
  if (X64in && o.precision != ACCORD_FP64) return kEunsupported;
  if (int e = check_device()) return e;
  const bool f64 = o.precision == ACCORD_FP64;
  if (!f64 && (n > 2147483647LL / 2 || p > 2147483647LL / 2)) return kEinval;
  if (rb != nullptr && (rb->fn == nullptr || rb->rows < 1 || rb->row0 < 0 || rb->row0 % 32 != 0 ||
                        rb->row0 > p - rb->rows || support != nullptr))
    return kEinval;

  Plan P;
  P.L = make_layout(n, p, o.precision, o.max_iter, o.lipschitz_max_iter, use_sparse(o, p), rb ? rb->rows : -1,
                    rb ? rb->row0 : 0);
  P.st = static_cast<cudaStream_t>(o.stream);
  Guard guard;
  if (workspace == nullptr) {
    if (cudaMallocAsync(&guard.ptr, P.L.total, P.st) != cudaSuccess) return kEnomem;
    guard.st = P.st;
    workspace = guard.ptr;
  } else if (ws_bytes < P.L.total || ((uintptr_t)workspace & 255u) != 0) {
    return ws_bytes < P.L.total ? kEnomem : kEinval;
  }
  P.ws = workspace;
  P.ctrl = at<Ctrl>(workspace, P.L.ctrl);
  P.err = &P.ctrl->dev_error;
  const Layout& L = P.L;
  void* ws = workspace;
  // Eq. 3.8 refit: weight phi * lambda on the support of `support`, infinite
  // off it (the epilogues read the bitmask built below)
  if (support != nullptr) lam = phi * lam;
  const double lam_d = o.penalize_diag ? lam : 0.0;

  cudaEvent_t ev[3];
  for (auto& e : ev) ACCORD_CK(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() { for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]); }
  } evg{ev};
  ACCORD_CK(cudaEventRecord(ev[0], P.st));

  // ---------------------------------------------------------------- setup --
  int64_t nlaunch = 0;
  ACCORD_CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), P.st));
  ACCORD_CK(cudaMemsetAsync(at<int>(ws, L.bad), 0, 64, P.st));
  ACCORD_CK(cudaMemsetAsync(at<int>(ws, L.dent), 0, 64, P.st));
  ACCORD_CK(cudaMemsetAsync(at<double>(ws, L.trace), 0xff, (size_t)L.trace_rows * kTraceFields * 8, P.st));
  if (f64) {
    ACCORD_CK(launch_convert_x_f64(X32, X64in, n, p, at<double>(ws, L.x64), L.ldo, at<double>(ws, L.xt64), L.ldy,
                                   at<int>(ws, L.bad), P.st));
  } else {
    ACCORD_CK(launch_convert_x_planes(X32, n, p, at<void>(ws, L.x_hi), at<void>(ws, L.x_lo), L.ldk,
                                      at<void>(ws, L.xt_hi), at<void>(ws, L.xt_lo), L.ldyk, at<int>(ws, L.bad), L.pt,
                                      P.st));
    ACCORD_CK(launch_transpose_x_f32(X32, n, p, at<float>(ws, L.xt32), L.ldy, P.st));
    nlaunch += 1;
    if (L.sparse) ACCORD_CK(cudaMemsetAsync(at<int>(ws, L.bkt_cnt), 0, (size_t)L.nbuckets * 4, P.st));
  }
  int64_t nomp = 0, nyp = 0;
  // Mixed modes: a buffer's values count only where its occupancy bitmap has
  // a bit, and every prox launch writes the whole bitmap of the buffer it
  // fills, so only buffer 0 (the starting iterate) needs one here.
  // a row block holds rows row0 .. row0 + m of Omega (and of Y = Omega X^T)
  const int64_t m = L.rows, row0 = L.row0;
  if (o.init_from_omega) {
    ACCORD_CK(launch_copy_omega(Omega, p, at<void>(ws, L.om[0]), L.ldo, f64, p, P.st, m));
    if (!f64) {
      ACCORD_CK(launch_bitmap_from_dense(at<float>(ws, L.om[0]), p, L.ldo, at<uint32_t>(ws, L.bm[0]), P.st, m));
      nlaunch += 1;
    }
    ACCORD_CK(launch_omega_stats(at<void>(ws, L.om[0]), f64, p, L.ldo, at<double>(ws, L.part_om), &nomp, P.st, m,
                                 row0));
    if (int e = setup_y(P, 0, 0)) return e;
    nyp = f64 ? gemm_f64_tiles(m, n) : tc_tiles(m, n);
    nlaunch += f64 ? 3 : 4;
  } else {
    // Omega^0 = I: its statistics are known and Y^0 = I X^T = X^T exactly
    ACCORD_CK(launch_set_identity(at<void>(ws, L.om[0]), f64, p, L.ldo, P.st, m, row0));
    if (!f64) {
      ACCORD_CK(launch_identity_bitmap(at<uint32_t>(ws, L.bm[0]), p, P.st, m, row0));
      nlaunch += 1;
    }
    ACCORD_CK(launch_identity_stats(at<double>(ws, L.part_om), m, P.st));
    nomp = 1;
    nlaunch += 2;
    if (f64) {
      ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.y[0]), at<double>(ws, L.xt64) + row0 * L.ldy, (size_t)m * L.ldy * 8,
                                cudaMemcpyDeviceToDevice, P.st));
      ACCORD_CK(launch_rows_norm2(at<double>(ws, L.y[0]), 1, m, n, L.ldy, at<double>(ws, L.part_y), &nyp, P.st));
      nlaunch += 1;
    } else if (L.sparse) {
      const size_t pe = plane_bytes(L.pt);
      ACCORD_CK(cudaMemcpyAsync(at<float>(ws, L.y[0]), at<float>(ws, L.xt32) + row0 * L.ldy, (size_t)m * L.ldy * 4,
                                cudaMemcpyDeviceToDevice, P.st));
      ACCORD_CK(cudaMemcpyAsync(at<void>(ws, L.y_hi[0]), at<char>(ws, L.xt_hi) + row0 * L.ldyk * pe,
                                (size_t)m * L.ldyk * pe, cudaMemcpyDeviceToDevice, P.st));
      ACCORD_CK(cudaMemcpyAsync(at<void>(ws, L.y_lo[0]), at<char>(ws, L.xt_lo) + row0 * L.ldyk * pe,
                                (size_t)m * L.ldyk * pe, cudaMemcpyDeviceToDevice, P.st));
      ACCORD_CK(launch_rows_norm2(at<float>(ws, L.y[0]), 0, m, n, L.ldy, at<double>(ws, L.part_y), &nyp, P.st));
      nlaunch += 1;
    } else {
      if (int e = setup_y(P, 0, 0)) return e;
      nyp = tc_tiles(m, n);
      nlaunch += 2;
    }
  }
  if (rb != nullptr) {
    // the starting sums over all blocks: one exchange, then one partial row each
    ACCORD_CK(launch_fold_block(P.ctrl, at<double>(ws, L.part_om), nomp, nullptr, at<double>(ws, L.part_y), nyp,
                                nullptr, 0, nullptr, nullptr, at<double>(ws, L.xsum), P.st));
    if (int e = exchange_sums(P, *rb, 0)) return e;
    ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.part_om), at<double>(ws, L.xsum) + kProxSlots + kYSlots,
                              kProxSlots * sizeof(double), cudaMemcpyDeviceToDevice, P.st));
    ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.part_y), at<double>(ws, L.xsum) + 2 * kProxSlots + kYSlots,
                              kYSlots * sizeof(double), cudaMemcpyDeviceToDevice, P.st));
    nomp = 1;
    nyp = 1;
    nlaunch += 1;
  }
  const int64_t ty = nyp;

  Ctrl hc;
  double L_given = o.lipschitz;
  if (!(L_given > 0.0)) {
    if (int e = setup_gram(P)) return e;
    // 0 = automatic: FP64 mode matches a dense eigensolver to rounding; the
    // mixed modes need L only to set the tau <= 1/L floor, and run the
    // process in FP32 on a Gram that carries FP32 accumulation error anyway
    const double lz_tol = o.lipschitz_tol > 0.0 ? o.lipschitz_tol : (f64 ? 1e-14 : 1e-6);
    ACCORD_CK(launch_lanczos_init(P.ctrl, at<double>(ws, L.lz_v), n, P.st, 1, 0, f64 ? 0 : 1));
    nlaunch += 2;
    const int chunk = 8;
    for (int steps = 0; steps < L.lz_k + chunk; steps += chunk) {
      ACCORD_CK(launch_lanczos_steps(P.ctrl, at<double>(ws, L.gram), n, at<double>(ws, L.lz_v),
                                     at<double>(ws, L.lz_w), at<double>(ws, L.lz_a), at<double>(ws, L.lz_b), n,
                                     L.lz_k, chunk, lz_tol, P.st, 1, 0, 0, 0, 0, f64 ? 0 : 1));
      nlaunch += 2 * chunk;
      if (int e = read_ctrl(P, &hc)) return e;
      if (hc.power_done) break;
    }
  }
  int hbad = 0;
  ACCORD_CK(cudaMemcpyAsync(&hbad, at<int>(ws, L.bad), sizeof(int), cudaMemcpyDeviceToHost, P.st));
  ACCORD_CK(cudaStreamSynchronize(P.st));
  if (hbad != 0) return kEdomain;

  TrialPlan T;
  if (int e = make_trial_plan(P, T, lam, lam_d)) return e;
  if (support != nullptr) {
    ACCORD_CK(launch_support_mask(support, f64, p, p, at<uint32_t>(ws, L.mask), L.mask_ld, P.st));
    nlaunch += 1;
    T.g2.mask = at<uint32_t>(ws, L.mask);
    T.g2.mask_ld = L.mask_ld;
    T.t2.mask = at<uint32_t>(ws, L.mask);
    T.t2.mask_ld = L.mask_ld;
  }
  SolveParams& sp = T.sp;
  sp.lam = lam;
  sp.lam_d = lam_d;
  sp.tau0 = o.tau0;
  sp.beta = o.beta;
  sp.kkt_tol = o.kkt_tol;
  sp.inv_n = 1.0 / (double)n;
  sp.max_iter = o.max_iter;
  sp.max_backtracks = o.max_backtracks;
  sp.tau_warm = o.tau_warm;
  sp.fixed_step = o.beta >= 1.0 ? 1 : 0;
  sp.trace_cap = L.trace_rows;
  sp.y_refresh = f64 ? 0 : o.y_refresh;
  sp.coarse_kkt = f64 ? 0.0 : o.coarse_kkt;
  T.t2.coarse_ok = sp.coarse_kkt > 0.0 ? 1 : 0;
  T.refresh = sp.y_refresh > 0;
  T.update_g = rb == nullptr ? 1 : 0;
  ACCORD_CK(launch_ctrl_init(P.ctrl, at<double>(ws, L.part_om), nomp, at<double>(ws, L.part_y), ty, sp, L_given,
                             at<double>(ws, L.trace), P.st));
  nlaunch += 1;
  ACCORD_CK(cudaEventRecord(ev[1], P.st));
  Profiler prof;
  prof.on = o.profile != 0;

  // ---------------------------------------------------------- iterations --
  const int64_t max_trials = ((int64_t)o.max_iter + 1) * ((int64_t)o.max_backtracks + 1) + 2;
  int64_t queued = 0;
  int chunk = 2;
  int32_t last_trials = -1;
  bool stalled = false;
  while (rb != nullptr) {
    // a row block: one trial at a time, each ended by the exchange of its sums
    // over all blocks; every block sees the same sums and so stops at the
    // same trial (a block's own device error travels as a bad count)
    if (int e = read_ctrl(P, &hc)) return e;
    if (hc.done || queued >= max_trials) break;
    if (int e = launch_trial(P, T, prof, nlaunch, true)) return e;
    if (int e = exchange_sums(P, *rb, hc.dev_error)) return e;
    ACCORD_CK(launch_decide_global(P.ctrl, at<double>(ws, L.xsum) + kProxSlots + kYSlots, sp,
                                   at<double>(ws, L.trace), P.st));
    nlaunch += 1;
    queued += 1;
  }
  for (; rb == nullptr;) {
    if (int e = read_ctrl(P, &hc)) return e;
    if (hc.done || queued >= max_trials || hc.dev_error != 0) break;
    // every live trial advances ctrl->trials; a chunk without progress means
    // the kernels are not doing their work, so stop queueing more
    if (hc.trials == last_trials) {
      stalled = true;
      break;
    }
    last_trials = hc.trials;
    for (int c = 0; c < chunk; ++c)
      if (int e = launch_trial(P, T, prof, nlaunch)) return e;
    queued += chunk;
    if (chunk < 16) chunk *= 2;
  }
  if (!hc.done) hc.status = kNotConverged;
  if (hc.dev_error != 0) {
    char msg[96];
    std::snprintf(msg, sizeof(msg), "device error bits 0x%x (1: an mbarrier wait timed out)", hc.dev_error);
    set_last_error(__FILE__, __LINE__, msg);
    hc.status = kEcuda;
  } else if (stalled) {
    set_last_error(__FILE__, __LINE__, "trial kernels made no progress");
    hc.status = kEcuda;
  }

  // copy the returned iterate (this block's rows) to the caller (mixed modes:
  // zeros wherever its bitmap has no bit)
  if (f64)
    ACCORD_CK(launch_copy_omega(at<void>(ws, L.om[hc.cur]), L.ldo, Omega, p, f64, p, P.st, m));
  else
    ACCORD_CK(launch_copy_omega_masked(at<float>(ws, L.om[hc.cur]), L.ldo, at<uint32_t>(ws, L.bm[hc.cur]),
                                       static_cast<float*>(Omega), p, p, P.st, m));
  nlaunch += 1;
  ACCORD_CK(cudaEventRecord(ev[2], P.st));
  if (o.trace && o.trace_cap > 0) {
    const int64_t rows = o.trace_cap < L.trace_rows ? o.trace_cap : L.trace_rows;
    ACCORD_CK(cudaMemcpyAsync(o.trace, at<double>(ws, L.trace), (size_t)rows * kTraceFields * 8,
                              cudaMemcpyDeviceToHost, P.st));
  }
  unsigned long long dent = 0;
  if (L.sparse)
    ACCORD_CK(cudaMemcpyAsync(&dent, at<unsigned long long>(ws, L.dent), sizeof(dent), cudaMemcpyDeviceToHost,
                              P.st));
  ACCORD_CK(cudaStreamSynchronize(P.st));
  if (out) {
    out->delta_entries = (int64_t)dent;
    out->y_refreshes = hc.n_refresh;
    out->coarse_prox = hc.n_coarse;
    out->y_drift = hc.y_drift;
    out->iters = hc.t;
    out->trials = hc.trials;
    out->status = hc.status;
    out->f = hc.f;
    out->g = hc.g;
    out->kkt = hc.kkt;
    out->tau_last = hc.tau_prev;
    out->L = hc.L;
    out->nnz_offdiag = (int64_t)hc.nnz;
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    out->t_setup_ms = a;
    out->t_solve_ms = b;
    // prox GEMMs that did work: one per trial, one per trial cut short for a
    // refresh of Y, plus the launch whose KKT check ended the fit (OK, or
    // NOT_CONVERGED at max_iter)
    const int64_t live_prox =
        hc.trials + hc.cut_trials + ((hc.status == kOk || hc.status == kNotConverged) ? 1 : 0);
    out->n_prox_gemm = (int32_t)live_prox;
    out->n_y_gemm = hc.trials;
    out->t_prox_gemm_ms = prof.on ? prof.total_ms(prof.prox, live_prox) : 0.0;
    out->t_y_gemm_ms = prof.on ? prof.total_ms(prof.y, hc.trials) : 0.0;
    out->n_launches = nlaunch;
    // Eq. 3.7 from the returned iterate's sums
    out->logdet_d = hc.logdiag;
    out->epbic = 2.0 * (double)n * (-hc.logdiag + hc.g) +
                 hc.nnz * (std::log((double)n) + 4.0 * o.epbic_gamma * std::log((double)p));
  }
  return hc.status;
}

}  // namespace
}  // namespace accord

using namespace accord;

extern "C" {

void accord_default_opts(accord_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = ACCORD_MIXED_BF16X3;
  o->tau_warm = 0;
  o->max_iter = 500;
  o->max_backtracks = 60;
  o->penalize_diag = 1;
  o->init_from_omega = 0;
  o->lipschitz_max_iter = 128;
  o->profile = 0;
  o->sparse_update = 1;
  o->autotune = 1;
  o->tau0 = 1.0;
  o->beta = 0.5;
  o->kkt_tol = 1e-8;
  o->lipschitz = 0.0;
  o->lipschitz_tol = 0.0;
  o->epbic_gamma = 0.5;
  o->stream = nullptr;
  o->trace = nullptr;
  o->trace_cap = 0;
  o->y_refresh = 32;
  o->coarse_kkt = 5e-3;
}

size_t accord_workspace_bytes(int64_t n, int64_t p, const accord_opts* optp) {
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (n < 1 || p < 1 || check_opts(o) != kOk) return 0;
  return make_layout(n, p, o.precision, o.max_iter, o.lipschitz_max_iter, use_sparse(o, p)).total;
}

int accord_fit(const float* X, int64_t n, int64_t p, double lambda, const accord_opts* opts, void* Omega,
               void* workspace, size_t ws_bytes, accord_stats* out) {
  const int s = abi_call([&] { return fit_impl(X, nullptr, n, p, lambda, opts, Omega, workspace, ws_bytes, out); });
  if (out) out->status = s;
  return s;
}

size_t accord_fit_rows_workspace_bytes(int64_t n, int64_t p, int64_t rows, const accord_opts* optp) {
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (n < 1 || p < 1 || rows < 1 || rows > p || check_opts(o) != kOk) return 0;
  return make_layout(n, p, o.precision, o.max_iter, o.lipschitz_max_iter, use_sparse(o, p), rows, 0).total;
}

int accord_fit_rows(const float* X, int64_t n, int64_t p, int64_t row0, int64_t rows, double lambda,
                    const accord_opts* opts, accord_exchange_fn exchange, void* ctx, void* Omega_rows,
                    void* workspace, size_t ws_bytes, accord_stats* out) {
  const RowBlock rb{row0, rows, exchange, ctx};
  const int s = abi_call([&] {
    return fit_impl(X, nullptr, n, p, lambda, opts, Omega_rows, workspace, ws_bytes, out, nullptr, 1.0, &rb);
  });
  if (out) out->status = s;
  return s;
}

int accord_refit(const float* X, int64_t n, int64_t p, double lambda, double phi, const void* Omega_hat,
                 const accord_opts* opts, void* Omega, void* workspace, size_t ws_bytes, accord_stats* out) {
  if (Omega_hat == nullptr || !(phi >= 0.0 && phi <= 1.0)) {
    if (out) std::memset(out, 0, sizeof(*out));
    if (out) out->status = ACCORD_EINVAL;
    return ACCORD_EINVAL;
  }
  const int s =
      abi_call([&] { return fit_impl(X, nullptr, n, p, lambda, opts, Omega, workspace, ws_bytes, out, Omega_hat, phi); });
  if (out) out->status = s;
  return s;
}

int accord_fit_f64(const double* X, int64_t n, int64_t p, double lambda, const accord_opts* opts, double* Omega,
                   void* workspace, size_t ws_bytes, accord_stats* out) {
  const int s = abi_call([&] { return fit_impl(nullptr, X, n, p, lambda, opts, Omega, workspace, ws_bytes, out); });
  if (out) out->status = s;
  return s;
}

const char* accord_status_string(int s) {
  switch (s) {
    case ACCORD_OK: return "converged (KKT residual <= tolerance)";
    case ACCORD_NOT_CONVERGED: return "not converged within max_iter";
    case ACCORD_EINVAL: return "invalid argument";
    case ACCORD_EDOMAIN: return "input outside the domain (omega_ii <= 0 or non-finite data)";
    case ACCORD_ENONFINITE: return "non-finite value during the iteration";
    case ACCORD_EBACKTRACK: return "line search exhausted max_backtracks";
    case ACCORD_ENOMEM: return "workspace too small or allocation failed";
    case ACCORD_ECUDA: return "CUDA error or a device wait timed out";
    case ACCORD_EUNSUPPORTED: return "unsupported device or option";
    default: return "unknown status";
  }
}

int accord_device_check(void) { return check_device(); }

int accord_test_wait_limit(int64_t wait_limit_ns, int32_t withhold_next_prox) {
  if (wait_limit_ns < 0 || (withhold_next_prox != 0 && withhold_next_prox != 1)) return ACCORD_EINVAL;
  tc_set_wait_test((uint64_t)wait_limit_ns, withhold_next_prox);
  return ACCORD_OK;
}

int accord_test_refresh(int32_t list_cap, int32_t form) {
  if ((list_cap != 0 && (list_cap < 32 || list_cap > 512)) || form < 0 || form > 2) return ACCORD_EINVAL;
  y_refresh_set_test(list_cap, form);
  return ACCORD_OK;
}

const char* accord_last_error(void) { return g_last_error; }

}  // extern "C"
