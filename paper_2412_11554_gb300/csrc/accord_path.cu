// accord_path: the lambda path of Sec 3.4 on many subsamples at once.
//
// Each subsample s is a chain: it walks the penalties in the given order and
// starts every fit from the previous penalty's estimate (warm start).  All
// chains run as one batch: every trial is one batched prox GEMM over the
// chains still running, the batched control kernels of Algorithm 1, and a
// path kernel that records each finished estimate (with its epBIC, Eq. 3.7)
// and moves its chain on.  The trial sequence is captured once into a CUDA
// graph and replayed until every chain has finished.
//
// The objective sees the data only through S, so a subsample with repeated
// rows (a bootstrap sample of n_s rows, K distinct) is run on the K x p matrix
// of its distinct rows, row j scaled by sqrt(K c_j / n_s) with c_j its
// multiplicity: that matrix has the same S = X^T X / n.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "api_util.h"
#include "internal.h"
#include "subsamples.h"
#include "tc_gemm.h"

namespace accord {
namespace {

constexpr int kTrialsPerGraph = 8;

// ------------------------------------------------------------ gather ------
struct GatherParams {
  const float* X;
  int64_t p;
  const int32_t* rows;   // device: distinct rows of every chain, concatenated
  const double* scale;   // device: their scales sqrt(K c_j / n_s)
  const int64_t* off;    // device: nchains + 1 offsets
  int64_t kpad;          // rows of every chain's matrix (zero beyond its K)
  double* x64;           // K x p rows (FP64), ld ldx, chain stride sx
  double* xt64;          // p x K (FP64, FP64 mode), ld ldt, chain stride st
  float* xt32;           // p x K (FP32, mixed modes)
  void *x_hi, *x_lo;    // K x p planes (mixed modes, type pt), ld ldx
  void *xt_hi, *xt_lo;  // p x K planes (mixed modes, type pt), ld ldt
  int64_t ldx, sx, ldt, st, sxp, stp;
  int pt;
  int* bad;
};

__global__ void gather_kernel(GatherParams g) {
  __shared__ double tile[32][33];
  const int c = blockIdx.z;
  const int64_t j0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int64_t o0 = g.off[c], K = g.off[c + 1] - o0;
  int nbad = 0;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t j = j0 + i, col = c0 + threadIdx.x;
    double v = 0.0;
    if (j < K && col < g.p) {
      v = g.scale[o0 + j] * (double)g.X[(int64_t)g.rows[o0 + j] * g.p + col];
      if (!isfinite(v)) ++nbad;
    }
    tile[i][threadIdx.x] = v;
    if (col < g.p) {
      if (g.x64) g.x64[c * g.sx + j * g.ldx + col] = v;
      if (g.x_hi) store_split(g.x_hi, g.x_lo, c * g.sxp + j * g.ldx + col, (float)v, g.pt);
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t col = c0 + i, j = j0 + threadIdx.x;
    if (col >= g.p) continue;
    const double v = tile[threadIdx.x][i];
    if (g.xt64) g.xt64[c * g.st + col * g.ldt + j] = v;
    if (g.xt32) g.xt32[c * g.st + col * g.ldt + j] = (float)v;
    if (g.xt_hi) store_split(g.xt_hi, g.xt_lo, c * g.stp + col * g.ldt + j, (float)v, g.pt);
  }
  if (nbad) atomicAdd(g.bad, nbad);
}

// ------------------------------------------------------------ layout ------
struct PathLayout {
  bool f64 = true;
  int pt = kPlaneBf16;  // operand-plane type of the mixed modes
  int64_t p = 0, nchains = 0, n_lambda = 0, kmax = 0, kpad = 0, ldo = 0;
  int64_t tiles_prox = 0, tiles_y = 0, nbuckets = 0, sum_k = 0;
  int lz_k = 0;
  size_t ctrl = 0, rec = 0, lambdas = 0, n_obs = 0, best_epbic = 0, best_idx = 0, active = 0, nactive = 0, bad = 0;
  size_t any_dense = 0;
  size_t kb_of = 0, g_rows = 0, g_scale = 0, g_off = 0;
  size_t part_prox = 0, part_y = 0;
  size_t om[2] = {0, 0}, y[2] = {0, 0};
  size_t bm[2] = {0, 0};  // occupancy bitmaps of the iterate buffers (mixed modes), one per chain
  size_t x64 = 0, xt64 = 0;
  size_t y_hi[2] = {0, 0}, y_lo[2] = {0, 0}, x_hi = 0, x_lo = 0, xt_hi = 0, xt_lo = 0, dp_hi = 0, dp_lo = 0;
  size_t xt32 = 0, bkt_keys = 0, bkt_vals = 0, bkt_cnt = 0, part_sy = 0;
  size_t gram = 0, lz_v = 0, lz_w = 0, lz_a = 0, lz_b = 0;
  size_t total = 0;
};

PathLayout make_path_layout(int64_t p, int64_t nchains, int64_t n_lambda, int64_t kmax, int64_t sum_k, int precision,
                            int lanczos_max) {
  PathLayout L;
  const bool f64 = precision == ACCORD_FP64;
  L.f64 = f64;
  L.pt = plane_type(precision);
  const size_t pe = plane_bytes(L.pt);
  L.p = p;
  L.nchains = nchains;
  L.n_lambda = n_lambda;
  L.kmax = kmax;
  L.sum_k = sum_k;
  L.kpad = round_up(kmax, 32);
  L.ldo = round_up(p, 32);
  L.tiles_prox = f64 ? gemm_f64_tiles(p, p) : tc_tiles(p, p);
  L.tiles_y = f64 ? gemm_f64_tiles(p, L.kpad) : tc_tiles(p, L.kpad);
  L.nbuckets = (p + kBucketRows - 1) / kBucketRows;
  const int64_t B = nchains, K = L.kpad;
  const size_t es = f64 ? 8 : 4;
  size_t c = 0;
  L.ctrl = take(c, (size_t)B * sizeof(Ctrl));
  L.rec = take(c, (size_t)n_lambda * B * sizeof(PathRec));
  L.lambdas = take(c, (size_t)n_lambda * 8);
  L.n_obs = take(c, (size_t)B * 8);
  L.best_epbic = take(c, (size_t)B * 8);
  L.best_idx = take(c, (size_t)B * 4);
  L.active = take(c, (size_t)B * 4);
  L.nactive = take(c, 64);
  L.bad = take(c, 64);
  L.any_dense = take(c, 64);
  L.kb_of = take(c, (size_t)B * 4);
  L.g_rows = take(c, (size_t)sum_k * 4);
  L.g_scale = take(c, (size_t)sum_k * 8);
  L.g_off = take(c, (size_t)(B + 1) * 8);
  L.part_prox = take(c, (size_t)B * L.tiles_prox * kProxSlots * 8);
  L.part_y = take(c, (size_t)B * L.tiles_y * kYSlots * 8);
  for (int q = 0; q < 2; ++q) L.om[q] = take(c, (size_t)B * p * L.ldo * es);
  for (int q = 0; q < 2; ++q) L.y[q] = take(c, (size_t)B * p * K * es);
  L.x64 = take(c, (size_t)B * K * L.ldo * 8);  // FP64 rows: the Gram (both modes), B of the FP64 Y GEMM
  if (f64) {
    L.xt64 = take(c, (size_t)B * p * K * 8);
  } else {
    for (int q = 0; q < 2; ++q) {
      L.y_hi[q] = take(c, (size_t)B * p * K * pe);
      L.y_lo[q] = take(c, (size_t)B * p * K * pe);
    }
    L.x_hi = take(c, (size_t)B * K * L.ldo * pe);
    L.x_lo = take(c, (size_t)B * K * L.ldo * pe);
    L.xt_hi = take(c, (size_t)B * p * K * pe);
    L.xt_lo = take(c, (size_t)B * p * K * pe);
    for (int q = 0; q < 2; ++q) L.bm[q] = take(c, (size_t)B * bitmap_words(p) * 4);
    L.dp_hi = take(c, (size_t)B * p * L.ldo * pe);
    L.dp_lo = take(c, (size_t)B * p * L.ldo * pe);
    L.xt32 = take(c, (size_t)B * p * K * 4);
    L.bkt_keys = take(c, (size_t)B * L.nbuckets * kBucketCap * 4);
    L.bkt_vals = take(c, (size_t)B * L.nbuckets * kBucketCap * 4);
    L.bkt_cnt = take(c, (size_t)B * L.nbuckets * 4);
    L.part_sy = take(c, (size_t)B * L.nbuckets * kYSlots * 8);
  }
  L.gram = take(c, (size_t)B * K * K * 8);
  int64_t k = lanczos_max < kLanczosMax ? lanczos_max : kLanczosMax;
  if (k > K) k = K;
  if (k < 1) k = 1;
  L.lz_k = (int)k;
  L.lz_v = take(c, (size_t)B * (k + 1) * K * 8);
  L.lz_w = take(c, (size_t)B * K * 8);
  L.lz_a = take(c, (size_t)B * k * 8);
  L.lz_b = take(c, (size_t)B * k * 8);
  L.total = c;
  return L;
}

int check_path_args(const float* X, int64_t n, int64_t p, const int32_t* rows, const int64_t* row_offsets,
                    int64_t n_sub, const double* lambdas, int64_t n_lambda, const accord_opts& o) {
  if (X == nullptr || rows == nullptr || row_offsets == nullptr || lambdas == nullptr) return kEinval;
  if (n < 1 || p < 1 || n_sub < 1 || n_sub > 65535 || n_lambda < 1) return kEinval;
  if (row_offsets[0] != 0) return kEinval;
  for (int64_t k = 0; k < n_lambda; ++k)
    if (!(lambdas[k] >= 0.0) || !std::isfinite(lambdas[k])) return kEinval;
  if (int e = check_opts(o)) return e;
  if (p > (1 << 25) - 2 || p > 2147483647LL / 2) return kEinval;
  return kOk;
}

struct PathPlan {
  PathLayout L;
  void* ws = nullptr;
  PathDev pd{};
  SolveParams sp{};
  GemmF64Params g2{}, g1{};
  TcParams t2{}, t1{};
  SparseYParams sy{};
  YRefreshParams rf{};
  bool refresh = false;  // mixed modes with sp.y_refresh > 0
};

// One trial of every running chain: the batched prox GEMM, then the rest of
// Algorithm 1's trial and the path bookkeeping.
int launch_path_prox(const PathPlan& P, cudaStream_t st) {
  if (P.refresh) {
    // Y formed afresh for the chains whose last decision asked for it
    ACCORD_CK(launch_y_refresh(P.rf, st));
    ACCORD_CK(launch_y_refresh_fold(P.pd.ctrl, (int32_t)P.L.nchains, P.pd.active, P.pd.nactive,
                                    at<double>(P.ws, P.L.part_sy), P.L.nbuckets, P.L.nbuckets * kYSlots, 1, st));
  }
  if (P.L.f64) ACCORD_CK(launch_gemm_f64(kModeProx, P.g2, st));
  else ACCORD_CK(launch_tc_gemm(kModeProx, P.t2, st));
  return kOk;
}

int launch_path_rest(const PathPlan& P, cudaStream_t st) {
  const PathLayout& L = P.L;
  void* ws = P.ws;
  Ctrl* ctrl = P.pd.ctrl;
  const int32_t B = (int32_t)L.nchains;
  ACCORD_CK(launch_post_prox_batch(ctrl, B, P.pd.active, P.pd.nactive, at<double>(ws, L.part_prox), L.tiles_prox,
                                   P.sp, st));
  if (L.f64) {
    ACCORD_CK(launch_gemm_f64(kModeY, P.g1, st));
  } else {
    // sparse Y+ = Y + Delta X^T, or the dense product for a chain whose Delta
    // bucket overflowed (each kernel checks its chain's flag)
    ACCORD_CK(launch_delta_planes(ctrl, at<float>(ws, L.om[0]), at<float>(ws, L.om[1]), at<uint32_t>(ws, L.bm[0]),
                                  at<uint32_t>(ws, L.bm[1]), L.p, L.ldo, at<void>(ws, L.dp_hi), at<void>(ws, L.dp_lo),
                                  L.ldo, L.pt, st, B, P.pd.active, P.pd.nactive, L.p * L.ldo, L.p * L.ldo,
                                  at<int>(ws, L.any_dense), bitmap_words(L.p)));
    ACCORD_CK(launch_tc_gemm(kModeY, P.t1, st));
    ACCORD_CK(launch_sparse_y(P.sy, st));
  }
  ACCORD_CK(launch_decide_batch(ctrl, B, P.pd.active, P.pd.nactive, at<double>(ws, L.part_y), L.tiles_y, P.sp,
                                L.f64 ? nullptr : at<int>(ws, L.bkt_cnt), L.f64 ? 0 : (int)L.nbuckets,
                                L.f64 ? nullptr : at<double>(ws, L.part_sy), st));
  ACCORD_CK(launch_path_advance(P.pd, st));
  return kOk;
}

int launches_per_trial(bool f64, bool refresh) { return f64 ? 5 : (refresh ? 10 : 7); }

// ------------------------------------------------------------ autotuner ---
// The batched prox GEMM's tile raster (pair rows of 256 per group) and its
// persistent grid (CTA pairs) are picked by timing each candidate on the call's own
// operands, once per (device, p, K, chains) in the process.  The runs happen
// before the control blocks are initialised: with tau = 0 the prox returns
// Omega unchanged, so Delta is empty and no state needs restoring.
struct TuneChoice {
  int group_m = 0, pairs = 0;
};
std::mutex g_tune_mu;
std::map<std::array<int64_t, 5>, TuneChoice> g_tune;

int tune_prox(PathPlan& P, cudaStream_t st, TuneChoice& best) {
  int dev = 0;
  ACCORD_CK(cudaGetDevice(&dev));
  const std::array<int64_t, 5> key{dev, P.L.p, P.L.kpad, P.L.nchains, P.L.pt};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      best = it->second;
      P.t2.group_m = best.group_m;
      P.t2.max_pairs = best.pairs;
      return kOk;
    }
  }
  const int maxc = tc_max_pairs(kModeProx, P.L.pt);
  std::vector<int> grids{maxc};
  for (int c : {maxc * 3 / 4, maxc / 2})
    if (c > 0 && c != grids.back()) grids.push_back(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ACCORD_CK(cudaEventCreate(&e0));
  struct EvPair {
    cudaEvent_t a, b;
    ~EvPair() { cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
  } evp{e0, nullptr};
  ACCORD_CK(cudaEventCreate(&e1));
  evp.b = e1;
  float best_ms = 1e30f;
  for (int g : {1, 2, 4, 8, 16}) {
    if (g > P.t2.tiles_mp && g != 1) continue;
    for (int c : grids) {
      P.t2.group_m = g;
      P.t2.max_pairs = c;
      ACCORD_CK(launch_tc_gemm(kModeProx, P.t2, st));  // warm
      ACCORD_CK(cudaEventRecord(e0, st));
      for (int r = 0; r < 2; ++r) ACCORD_CK(launch_tc_gemm(kModeProx, P.t2, st));
      ACCORD_CK(cudaEventRecord(e1, st));
      ACCORD_CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      ACCORD_CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best.group_m = g;
        best.pairs = c;
      }
    }
  }
  P.t2.group_m = best.group_m;
  P.t2.max_pairs = best.pairs;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return kOk;
}

int path_impl(const float* X, int64_t n, int64_t p, const int32_t* rows, const int64_t* row_offsets, int64_t n_sub,
              const double* lambdas, int64_t n_lambda, const accord_opts* optp, accord_path_entry* entries,
              uint32_t* support, void* omega_best, int32_t* best_index, void* workspace, size_t ws_bytes,
              accord_stats* out) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (out) std::memset(out, 0, sizeof(*out));
  if (entries == nullptr) return kEinval;
  if (int e = check_path_args(X, n, p, rows, row_offsets, n_sub, lambdas, n_lambda, o)) return e;
  Subsamples S;
  if (int e = compress_subsamples(rows, row_offsets, n_sub, n, S)) return e;
  if (int e = check_device()) return e;
  const bool f64 = o.precision == ACCORD_FP64;

  PathPlan P;
  P.L = make_path_layout(p, n_sub, n_lambda, S.kmax, (int64_t)S.rows.size(), o.precision, o.lipschitz_max_iter);
  const PathLayout& L = P.L;
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  Guard guard;
  if (workspace == nullptr) {
    if (cudaMallocAsync(&guard.ptr, L.total, st) != cudaSuccess) return kEnomem;
    guard.st = st;
    workspace = guard.ptr;
  } else if (ws_bytes < L.total || ((uintptr_t)workspace & 255u) != 0) {
    return ws_bytes < L.total ? kEnomem : kEinval;
  }
  P.ws = workspace;
  void* ws = workspace;
  const int64_t B = n_sub, K = L.kpad;

  cudaEvent_t ev[3];
  for (auto& e : ev) ACCORD_CK(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() { for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]); }
  } evg{ev};
  ACCORD_CK(cudaEventRecord(ev[0], st));
  int64_t nlaunch = 0;

  // ------------------------------------------------ host-built state -----
  std::vector<Ctrl> hctrl(B);
  std::vector<int32_t> hkb(B);
  for (int64_t c = 0; c < B; ++c) {
    Ctrl& C = hctrl[c];
    std::memset(&C, 0, sizeof(C));
    const int64_t Kc = S.off[c + 1] - S.off[c];
    C.status = kNotConverged;
    C.kdim = (int32_t)Kc;
    C.inv_n = 1.0 / (double)Kc;
    C.lam = lambdas[0];
    C.lam_d = o.penalize_diag ? lambdas[0] : 0.0;
    C.kkt = INFINITY;
    const int64_t bk = tc_bk(P.L.pt);  // K blocks of the mixed prox GEMM (unused in FP64 mode)
    hkb[c] = (int32_t)((Kc + bk - 1) / bk);
  }
  std::vector<double> hbest(B, INFINITY);
  std::vector<int32_t> hbidx(B, -1);
  std::vector<int32_t> hact(B);
  for (int64_t c = 0; c < B; ++c) hact[c] = (int32_t)c;
  const int32_t hnact = (int32_t)B;
  ACCORD_CK(cudaMemcpyAsync(at<Ctrl>(ws, L.ctrl), hctrl.data(), B * sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<int32_t>(ws, L.kb_of), hkb.data(), B * 4, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.lambdas), lambdas, n_lambda * 8, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.n_obs), S.n_obs.data(), B * 8, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.best_epbic), hbest.data(), B * 8, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<int32_t>(ws, L.best_idx), hbidx.data(), B * 4, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<int32_t>(ws, L.active), hact.data(), B * 4, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<int32_t>(ws, L.nactive), &hnact, 4, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<int32_t>(ws, L.g_rows), S.rows.data(), S.rows.size() * 4, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.g_scale), S.scale.data(), S.scale.size() * 8, cudaMemcpyHostToDevice,
                            st));
  ACCORD_CK(cudaMemcpyAsync(at<int64_t>(ws, L.g_off), S.off.data(), (B + 1) * 8, cudaMemcpyHostToDevice, st));
  ACCORD_CK(cudaMemsetAsync(at<int>(ws, L.bad), 0, 64, st));
  ACCORD_CK(cudaMemsetAsync(at<int>(ws, L.any_dense), 0, 64, st));
  ACCORD_CK(cudaMemsetAsync(at<PathRec>(ws, L.rec), 0, (size_t)n_lambda * B * sizeof(PathRec), st));

  // --------------------------------------------- data of every chain -----
  GatherParams g{};
  g.X = X;
  g.p = p;
  g.rows = at<int32_t>(ws, L.g_rows);
  g.scale = at<double>(ws, L.g_scale);
  g.off = at<int64_t>(ws, L.g_off);
  g.kpad = K;
  g.x64 = at<double>(ws, L.x64);
  g.ldx = L.ldo;
  g.sx = K * L.ldo;
  g.sxp = K * L.ldo;
  g.ldt = K;
  g.st = p * K;
  g.stp = p * K;
  if (f64) {
    g.xt64 = at<double>(ws, L.xt64);
  } else {
    g.xt32 = at<float>(ws, L.xt32);
    g.x_hi = at<void>(ws, L.x_hi);
    g.x_lo = at<void>(ws, L.x_lo);
    g.xt_hi = at<void>(ws, L.xt_hi);
    g.xt_lo = at<void>(ws, L.xt_lo);
  }
  g.pt = L.pt;
  g.bad = at<int>(ws, L.bad);
  {
    const dim3 grid((unsigned)((p + 31) / 32), (unsigned)(K / 32), (unsigned)B), block(32, 8);
    gather_kernel<<<grid, block, 0, st>>>(g);
    ACCORD_CK(cudaGetLastError());
    nlaunch += 1;
  }
  // Omega^0 = I and Y^0 = X^T for every chain.  In the mixed modes a buffer's
  // values count only where its occupancy bitmap has a bit, and every prox
  // launch writes the whole bitmap of the buffer it fills, so only buffer 0
  // needs one here.
  const size_t es = f64 ? 8 : 4;
  for (int64_t c = 0; c < B; ++c) {
    ACCORD_CK(launch_set_identity(at<char>(ws, L.om[0]) + (size_t)c * p * L.ldo * es, f64, p, L.ldo, st));
    nlaunch += 1;
    if (!f64) {
      ACCORD_CK(launch_identity_bitmap(at<uint32_t>(ws, L.bm[0]) + c * bitmap_words(p), p, st));
      nlaunch += 1;
    }
  }
  if (f64) {
    ACCORD_CK(cudaMemcpyAsync(at<double>(ws, L.y[0]), at<double>(ws, L.xt64), (size_t)B * p * K * 8,
                              cudaMemcpyDeviceToDevice, st));
  } else {
    ACCORD_CK(cudaMemcpyAsync(at<float>(ws, L.y[0]), at<float>(ws, L.xt32), (size_t)B * p * K * 4,
                              cudaMemcpyDeviceToDevice, st));
    const size_t pbytes = (size_t)B * p * K * plane_bytes(L.pt);
    ACCORD_CK(cudaMemcpyAsync(at<void>(ws, L.y_hi[0]), at<void>(ws, L.xt_hi), pbytes, cudaMemcpyDeviceToDevice, st));
    ACCORD_CK(cudaMemcpyAsync(at<void>(ws, L.y_lo[0]), at<void>(ws, L.xt_lo), pbytes, cudaMemcpyDeviceToDevice, st));
    // the other Y buffer's K padding must read as zero too
    ACCORD_CK(cudaMemsetAsync(at<float>(ws, L.y[1]), 0, (size_t)B * p * K * 4, st));
    ACCORD_CK(cudaMemsetAsync(at<void>(ws, L.y_hi[1]), 0, pbytes, st));
    ACCORD_CK(cudaMemsetAsync(at<void>(ws, L.y_lo[1]), 0, pbytes, st));
    ACCORD_CK(cudaMemsetAsync(at<int>(ws, L.bkt_cnt), 0, (size_t)B * L.nbuckets * 4, st));
  }

  // ------------------------------------------- L of every subsample ------
  Ctrl* ctrl = at<Ctrl>(ws, L.ctrl);
  double L_given = o.lipschitz;
  if (!(L_given > 0.0)) {
    GemmF64Params gg{};
    gg.ctrl = ctrl;  // per-chain 1/n
    gg.A[0] = gg.A[1] = at<double>(ws, L.x64);
    gg.lda = L.ldo;
    gg.B = at<double>(ws, L.x64);
    gg.ldb = L.ldo;
    gg.M = K;
    gg.N = K;
    gg.K = p;
    gg.out[0] = gg.out[1] = at<double>(ws, L.gram);
    gg.ldout = K;
    gg.nprob = (int32_t)B;
    gg.active = at<int32_t>(ws, L.active);  // every chain (per-chain 1/n also for a single chain)
    gg.nactive = at<int32_t>(ws, L.nactive);
    gg.s_a = gg.s_b = K * L.ldo;
    gg.s_out = K * K;
    ACCORD_CK(launch_gemm_f64(kModeGram, gg, st));
    const double lz_tol = o.lipschitz_tol > 0.0 ? o.lipschitz_tol : (f64 ? 1e-14 : 1e-6);
    ACCORD_CK(launch_lanczos_init(ctrl, at<double>(ws, L.lz_v), K, st, (int)B, (int64_t)(L.lz_k + 1) * K,
                                  f64 ? 0 : 1));
    nlaunch += 2;
    const int chunk = 8;
    for (int steps = 0; steps < L.lz_k + chunk; steps += chunk) {
      ACCORD_CK(launch_lanczos_steps(ctrl, at<double>(ws, L.gram), K, at<double>(ws, L.lz_v), at<double>(ws, L.lz_w),
                                     at<double>(ws, L.lz_a), at<double>(ws, L.lz_b), K, L.lz_k, chunk, lz_tol, st,
                                     (int)B, K * K, (int64_t)(L.lz_k + 1) * K, K, L.lz_k, f64 ? 0 : 1));
      nlaunch += 2 * chunk;
      ACCORD_CK(cudaMemcpyAsync(hctrl.data(), ctrl, B * sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
      ACCORD_CK(cudaStreamSynchronize(st));
      bool all = true;
      for (int64_t c = 0; c < B; ++c) all = all && hctrl[c].power_done;
      if (all) break;
    }
  }
  int hbad = 0;
  ACCORD_CK(cudaMemcpyAsync(&hbad, at<int>(ws, L.bad), sizeof(int), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaStreamSynchronize(st));
  if (hbad != 0) return kEdomain;

  // ------------------------------------------------ trial plan -----------
  PathDev& pd = P.pd;
  pd.ctrl = ctrl;
  pd.nchains = (int32_t)B;
  pd.n_lambda = (int32_t)n_lambda;
  pd.lambdas = at<double>(ws, L.lambdas);
  pd.n_obs = at<double>(ws, L.n_obs);
  pd.gamma = o.epbic_gamma;
  pd.log_p = std::log((double)p);
  pd.penalize_diag = o.penalize_diag ? 1 : 0;
  pd.rec = at<PathRec>(ws, L.rec);
  pd.best_epbic = at<double>(ws, L.best_epbic);
  pd.best_idx = at<int32_t>(ws, L.best_idx);
  pd.active = at<int32_t>(ws, L.active);
  pd.nactive = at<int32_t>(ws, L.nactive);
  pd.any_dense = f64 ? nullptr : at<int>(ws, L.any_dense);
  SolveParams& sp = P.sp;
  sp.tau0 = o.tau0;
  sp.beta = o.beta;
  sp.kkt_tol = o.kkt_tol;
  sp.max_iter = o.max_iter;
  sp.max_backtracks = o.max_backtracks;
  sp.tau_warm = o.tau_warm;
  sp.fixed_step = o.beta >= 1.0 ? 1 : 0;
  sp.trace_cap = 0;
  sp.y_refresh = f64 ? 0 : o.y_refresh;
  sp.coarse_kkt = f64 ? 0.0 : o.coarse_kkt;
  pd.coarse = sp.coarse_kkt > 0.0 ? 1 : 0;
  if (f64) {
    GemmF64Params& g2 = P.g2;  // G = Y X / n, prox, Omega[cur] -> Omega[nxt]
    g2.ctrl = ctrl;
    g2.A[0] = at<double>(ws, L.y[0]);
    g2.A[1] = at<double>(ws, L.y[1]);
    g2.lda = K;
    g2.B = at<double>(ws, L.xt64);
    g2.ldb = K;
    g2.M = p; g2.N = p; g2.K = K;
    g2.out[0] = at<double>(ws, L.om[0]);
    g2.out[1] = at<double>(ws, L.om[1]);
    g2.ldout = L.ldo;
    g2.aux[0] = at<double>(ws, L.om[0]);
    g2.aux[1] = at<double>(ws, L.om[1]);
    g2.ldaux = L.ldo;
    g2.part = at<double>(ws, L.part_prox);
    g2.nprob = (int32_t)B;
    g2.active = pd.active;
    g2.nactive = pd.nactive;
    g2.s_a = p * K; g2.s_b = p * K; g2.s_out = p * L.ldo; g2.s_aux = p * L.ldo; g2.s_part = L.tiles_prox;
    GemmF64Params& g1 = P.g1;  // Y[nxt] = Omega[nxt] X^T, old Y[cur] for the difference
    g1.ctrl = ctrl;
    g1.A[0] = at<double>(ws, L.om[0]);
    g1.A[1] = at<double>(ws, L.om[1]);
    g1.a_nxt = 1;
    g1.lda = L.ldo;
    g1.B = at<double>(ws, L.x64);
    g1.ldb = L.ldo;
    g1.M = p; g1.N = K; g1.K = p;
    g1.out[0] = at<double>(ws, L.y[0]);
    g1.out[1] = at<double>(ws, L.y[1]);
    g1.ldout = K;
    g1.aux[0] = at<double>(ws, L.y[0]);
    g1.aux[1] = at<double>(ws, L.y[1]);
    g1.ldaux = K;
    g1.part = at<double>(ws, L.part_y);
    g1.scale = 1.0;
    g1.nprob = (int32_t)B;
    g1.active = pd.active;
    g1.nactive = pd.nactive;
    g1.s_a = p * L.ldo; g1.s_b = K * L.ldo; g1.s_out = p * K; g1.s_aux = p * K; g1.s_part = L.tiles_y;
  } else {
    ACCORD_CK(tc_prepare());
    ACCORD_CK(sparse_y_prepare());
    TcParams& t2 = P.t2;  // prox GEMM over the chains still running
    for (int q = 0; q < 2; ++q)
      if (!encode_plane_map(&t2.a_hi[q], at<void>(ws, L.y_hi[q]), L.pt, p, K, K, 128, B, p * K) ||
          !encode_plane_map(&t2.a_lo[q], at<void>(ws, L.y_lo[q]), L.pt, p, K, K, 128, B, p * K))
        return kEcuda;
    if (!encode_plane_map(&t2.b_hi, at<void>(ws, L.xt_hi), L.pt, p, K, K, tc_box_n(), B, p * K) ||
        !encode_plane_map(&t2.b_lo, at<void>(ws, L.xt_lo), L.pt, p, K, K, tc_box_n(), B, p * K))
      return kEcuda;
    t2.ctrl = ctrl;
    t2.coarse_ok = sp.coarse_kkt > 0.0 ? 1 : 0;
    t2.err = &ctrl[0].dev_error;
    tc_shape(t2, p, p, K, L.pt);
    t2.out[0] = at<float>(ws, L.om[0]);
    t2.out[1] = at<float>(ws, L.om[1]);
    t2.ldout = L.ldo;
    t2.aux[0] = at<float>(ws, L.om[0]);
    t2.aux[1] = at<float>(ws, L.om[1]);
    t2.ldaux = L.ldo;
    t2.part = at<double>(ws, L.part_prox);
    t2.scale = 1.f;
    t2.keys = at<uint32_t>(ws, L.bkt_keys);
    t2.vals = at<float>(ws, L.bkt_vals);
    t2.counts = at<int>(ws, L.bkt_cnt);
    t2.cap = kBucketCap;
    t2.nprob = (int32_t)B;
    t2.b_batched = 1;
    t2.active = pd.active;
    t2.nactive = pd.nactive;
    t2.kb_of = at<int32_t>(ws, L.kb_of);
    t2.s_out = p * L.ldo; t2.s_aux = p * L.ldo; t2.s_part = L.tiles_prox; t2.s_bkt = L.nbuckets;
    t2.bm[0] = at<uint32_t>(ws, L.bm[0]);
    t2.bm[1] = at<uint32_t>(ws, L.bm[1]);
    t2.ldbm = bitmap_ld(p);
    t2.s_bm = bitmap_words(p);
    t2.any_dense = at<int>(ws, L.any_dense);
    // a chain in dense Y mode gets its Delta planes from this epilogue
    t2.out_hi[0] = t2.out_hi[1] = at<void>(ws, L.dp_hi);
    t2.out_lo[0] = t2.out_lo[1] = at<void>(ws, L.dp_lo);
    t2.ldplane = L.ldo;
    t2.s_plane = p * L.ldo;
    TcParams& t1 = P.t1;  // dense Y+ = Y + Delta X^T, only for chains whose bucket overflowed
    if (!encode_plane_map(&t1.a_hi[0], at<void>(ws, L.dp_hi), L.pt, p, p, L.ldo, 128, B, p * L.ldo) ||
        !encode_plane_map(&t1.a_lo[0], at<void>(ws, L.dp_lo), L.pt, p, p, L.ldo, 128, B, p * L.ldo) ||
        !encode_plane_map(&t1.b_hi, at<void>(ws, L.x_hi), L.pt, K, p, L.ldo, tc_box_n(), B, K * L.ldo) ||
        !encode_plane_map(&t1.b_lo, at<void>(ws, L.x_lo), L.pt, K, p, L.ldo, tc_box_n(), B, K * L.ldo))
      return kEcuda;
    t1.a_hi[1] = t1.a_hi[0];
    t1.a_lo[1] = t1.a_lo[0];
    t1.ctrl = ctrl;
    t1.err = &ctrl[0].dev_error;
    tc_shape(t1, p, K, p, L.pt);
    t1.out[0] = at<float>(ws, L.y[0]);
    t1.out[1] = at<float>(ws, L.y[1]);
    t1.ldout = K;
    for (int q = 0; q < 2; ++q) {
      t1.out_hi[q] = at<void>(ws, L.y_hi[q]);
      t1.out_lo[q] = at<void>(ws, L.y_lo[q]);
    }
    t1.ldplane = K;
    t1.aux[0] = at<float>(ws, L.y[0]);
    t1.aux[1] = at<float>(ws, L.y[1]);
    t1.ldaux = K;
    t1.part = at<double>(ws, L.part_y);
    t1.scale = 1.f;
    t1.gate_dense = 1;
    t1.nprob = (int32_t)B;
    t1.b_batched = 1;
    t1.active = pd.active;
    t1.nactive = pd.nactive;
    t1.s_out = p * K; t1.s_aux = p * K; t1.s_plane = p * K; t1.s_part = L.tiles_y;
    t1.any_dense = at<int>(ws, L.any_dense);
    SparseYParams& sy = P.sy;
    sy.ctrl = ctrl;
    for (int q = 0; q < 2; ++q) {
      sy.y[q] = at<float>(ws, L.y[q]);
      sy.yw[q] = at<float>(ws, L.y[q]);
      sy.y_hi[q] = at<void>(ws, L.y_hi[q]);
      sy.y_lo[q] = at<void>(ws, L.y_lo[q]);
    }
    sy.xt = at<float>(ws, L.xt32);
    sy.keys = at<uint32_t>(ws, L.bkt_keys);
    sy.vals = at<float>(ws, L.bkt_vals);
    sy.counts = at<int>(ws, L.bkt_cnt);
    sy.cap = kBucketCap;
    sy.tiles_m = (int32_t)L.nbuckets;
    sy.p = p;
    sy.n = K;
    sy.ldy = K;
    sy.ldyk = K;
    sy.part = at<double>(ws, L.part_sy);
    sy.active = pd.active;
    sy.nactive = pd.nactive;
    sy.nprob = (int32_t)B;
    sy.s_y = p * K; sy.s_yk = p * K; sy.s_xt = p * K; sy.s_bkt = L.nbuckets;
    sy.ptype = L.pt;
    YRefreshParams& rf = P.rf;
    rf.ctrl = ctrl;
    for (int q = 0; q < 2; ++q) {
      rf.om[q] = at<float>(ws, L.om[q]);
      rf.bm[q] = at<uint32_t>(ws, L.bm[q]);
      rf.y[q] = at<float>(ws, L.y[q]);
      rf.y_hi[q] = at<void>(ws, L.y_hi[q]);
      rf.y_lo[q] = at<void>(ws, L.y_lo[q]);
    }
    rf.xt = at<float>(ws, L.xt32);
    rf.rows = p;
    rf.p = p;
    rf.n = K;
    rf.ldo = L.ldo;
    rf.ldbm = bitmap_ld(p);
    rf.ldy = K;
    rf.ldyk = K;
    rf.ldx = K;
    rf.part = at<double>(ws, L.part_sy);
    rf.ptype = L.pt;
    rf.nprob = (int32_t)B;
    rf.active = pd.active;
    rf.nactive = pd.nactive;
    rf.s_om = p * L.ldo; rf.s_bm = bitmap_words(p); rf.s_y = p * K; rf.s_yk = p * K; rf.s_xt = p * K;
    rf.s_part = L.nbuckets * kYSlots;
    rf.dense_nnz = 0.1 * (double)p * (double)p;
    P.refresh = P.sp.y_refresh > 0;
  }
  TuneChoice tune;
  if (!f64 && o.autotune) {
    if (int e = tune_prox(P, st, tune)) return e;
  }
  ACCORD_CK(launch_batch_ctrl_init(pd, at<void>(ws, L.y[0]), f64, p, K, p * K, sp, L_given, st));
  nlaunch += 1;
  ACCORD_CK(cudaEventRecord(ev[1], st));

  // ------------------------------------------ captured trial sequence ----
  // kTrialsPerGraph trials are captured once on a private stream (the
  // caller's may be the legacy default stream, which cannot capture) and the
  // graph is replayed on the caller's stream.  With opts->profile the trials
  // are launched directly instead, with CUDA events around every batched
  // prox GEMM.
  const bool emit = support != nullptr || omega_best != nullptr;
  auto one_trial = [&](cudaStream_t s, std::vector<cudaEvent_t>* marks) -> int {
    if (marks) {
      cudaEvent_t e;
      ACCORD_CK(cudaEventCreate(&e));
      marks->push_back(e);
      ACCORD_CK(cudaEventRecord(e, s));
    }
    if (int r = launch_path_prox(P, s)) return r;
    if (marks) {
      cudaEvent_t e;
      ACCORD_CK(cudaEventCreate(&e));
      marks->push_back(e);
      ACCORD_CK(cudaEventRecord(e, s));
    }
    if (int r = launch_path_rest(P, s)) return r;
    if (emit)
      ACCORD_CK(launch_path_emit(pd, at<void>(ws, L.om[0]), at<void>(ws, L.om[1]), f64, p, L.ldo, p * L.ldo, support,
                                 (p + 31) / 32, omega_best, s, f64 ? nullptr : at<uint32_t>(ws, L.bm[0]),
                                 f64 ? nullptr : at<uint32_t>(ws, L.bm[1]), bitmap_words(p)));
    return kOk;
  };
  const bool use_graph = o.profile == 0;
  struct Marks {
    std::vector<cudaEvent_t> v;
    ~Marks() { for (auto e : v) cudaEventDestroy(e); }
  } marks;
  cudaStream_t cs = nullptr;
  ACCORD_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } sgd{cs};
  struct ExecGuard {
    cudaGraphExec_t g = nullptr;
    ~ExecGuard() {
      if (g) cudaGraphExecDestroy(g);
    }
  } egd;
  if (use_graph) {
    cudaGraph_t graph = nullptr;
    ACCORD_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int cap_err = kOk;
    for (int t = 0; t < kTrialsPerGraph && cap_err == kOk; ++t) cap_err = one_trial(cs, nullptr);
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (cap_err != kOk) {
      if (graph) cudaGraphDestroy(graph);
      return cap_err;
    }
    ACCORD_CK(ce);
    const cudaError_t ie = cudaGraphInstantiate(&egd.g, graph, 0);
    cudaGraphDestroy(graph);
    ACCORD_CK(ie);
  }
  const int per_trial = launches_per_trial(f64, P.refresh) + (emit ? 1 : 0);

  // every penalty ends by max_iter steps of at most max_backtracks + 1 trials
  const int64_t max_graphs =
      (n_lambda * ((int64_t)o.max_iter + 1) * ((int64_t)o.max_backtracks + 1)) / kTrialsPerGraph + 2;
  int32_t nact = (int32_t)B;
  int64_t graphs = 0;
  int hstatus = kOk;
  while (nact > 0) {
    if (graphs >= max_graphs) {
      set_last_error(__FILE__, __LINE__, "lambda path did not finish within its trial bound");
      hstatus = kEcuda;
      break;
    }
    if (use_graph) {
      ACCORD_CK(cudaGraphLaunch(egd.g, st));
    } else {
      for (int t = 0; t < kTrialsPerGraph; ++t)
        if (int r = one_trial(st, &marks.v)) return r;
    }
    nlaunch += (int64_t)per_trial * kTrialsPerGraph;
    ++graphs;
    ACCORD_CK(cudaMemcpyAsync(&nact, pd.nactive, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    ACCORD_CK(cudaStreamSynchronize(st));
  }
  double prox_ms = 0.0;
  for (size_t i = 0; i + 1 < marks.v.size(); i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, marks.v[i], marks.v[i + 1]) == cudaSuccess) prox_ms += ms;
  }
  ACCORD_CK(cudaEventRecord(ev[2], st));
  // the launch cost of a replay: the same graph once more, now that every
  // chain has finished and each of its kernels returns at once
  double idle_ms = 0.0;
  if (use_graph && hstatus == kOk) {
    cudaEvent_t i0 = nullptr, i1 = nullptr;
    ACCORD_CK(cudaEventCreate(&i0));
    cudaError_t ie = cudaEventCreate(&i1);
    if (ie == cudaSuccess) ie = cudaEventRecord(i0, st);
    if (ie == cudaSuccess) ie = cudaGraphLaunch(egd.g, st);
    if (ie == cudaSuccess) ie = cudaEventRecord(i1, st);
    if (ie == cudaSuccess) ie = cudaEventSynchronize(i1);
    float ms = 0.f;
    if (ie == cudaSuccess) ie = cudaEventElapsedTime(&ms, i0, i1);
    cudaEventDestroy(i0);
    if (i1) cudaEventDestroy(i1);
    ACCORD_CK(ie);
    idle_ms = ms;
    nlaunch += (int64_t)per_trial * kTrialsPerGraph;
  }

  // ------------------------------------------------------- results -------
  static_assert(sizeof(PathRec) == sizeof(accord_path_entry), "path record layout");
  ACCORD_CK(cudaMemcpyAsync(entries, pd.rec, (size_t)n_lambda * B * sizeof(PathRec), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaMemcpyAsync(hbidx.data(), pd.best_idx, B * 4, cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaMemcpyAsync(hctrl.data(), ctrl, B * sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  ACCORD_CK(cudaStreamSynchronize(st));
  if (best_index) std::memcpy(best_index, hbidx.data(), B * 4);
  int dev_err = 0;
  for (int64_t c = 0; c < B; ++c) dev_err |= hctrl[c].dev_error;
  if (dev_err != 0) {
    char msg[96];
    std::snprintf(msg, sizeof(msg), "device error bits 0x%x (1: an mbarrier wait timed out)", dev_err);
    set_last_error(__FILE__, __LINE__, msg);
    hstatus = kEcuda;
  }
  if (hstatus == kOk) {
    for (int64_t i = 0; i < n_lambda * B; ++i) {
      if (entries[i].status < 0) {
        hstatus = entries[i].status;
        break;
      }
      if (entries[i].status == kNotConverged) hstatus = kNotConverged;
    }
  }
  if (out) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    out->t_setup_ms = a;
    out->t_solve_ms = b;
    out->status = hstatus;
    int64_t it = 0, tr = 0;
    for (int64_t c = 0; c < B; ++c) {
      it += hctrl[c].iters_tot;
      tr += hctrl[c].trials_tot;
    }
    out->iters = (int32_t)it;
    out->trials = (int32_t)tr;
    int64_t nrf = 0;
    double drift = 0.0;
    for (int64_t i = 0; i < n_lambda * B; ++i) {
      nrf += entries[i].y_refreshes;
      drift = std::max(drift, entries[i].y_drift);
    }
    out->y_refreshes = (int32_t)nrf;
    int64_t nco = 0;
    for (int64_t c = 0; c < B; ++c) nco += hctrl[c].n_coarse;
    out->coarse_prox = (int32_t)nco;
    out->y_drift = drift;
    out->t_graph_idle_ms = idle_ms;
    out->n_prox_gemm = (int32_t)(graphs * kTrialsPerGraph);
    out->t_prox_gemm_ms = prox_ms;
    out->n_launches = nlaunch;
    out->L = hctrl[0].L;
    out->tile_group_m = f64 ? 0 : P.t2.group_m;
    out->tile_pairs = f64 ? 0 : (P.t2.max_pairs > 0 ? P.t2.max_pairs : tc_max_pairs(kModeProx, L.pt));
  }
  return hstatus;
}

}  // namespace
}  // namespace accord

using namespace accord;

extern "C" {

size_t accord_path_workspace_bytes(int64_t n, int64_t p, const int32_t* rows, const int64_t* row_offsets,
                                   int64_t n_sub, int64_t n_lambda, const accord_opts* optp) {
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  double lam0 = 0.0;
  if (check_path_args(reinterpret_cast<const float*>(16), n, p, rows, row_offsets, n_sub, &lam0, 1, o) != kOk ||
      n_lambda < 1)
    return 0;
  size_t total = 0;
  abi_call([&]() -> int {
    Subsamples S;
    if (int e = compress_subsamples(rows, row_offsets, n_sub, n, S)) return e;
    total = make_path_layout(p, n_sub, n_lambda, S.kmax, (int64_t)S.rows.size(), o.precision,
                             o.lipschitz_max_iter)
                .total;
    return kOk;
  });
  return total;
}

int accord_path(const float* X, int64_t n, int64_t p, const int32_t* rows, const int64_t* row_offsets, int64_t n_sub,
                const double* lambdas, int64_t n_lambda, const accord_opts* opts, accord_path_entry* entries,
                uint32_t* support, void* omega_best, int32_t* best_index, void* workspace, size_t ws_bytes,
                accord_stats* out) {
  const int s = abi_call([&] {
    return path_impl(X, n, p, rows, row_offsets, n_sub, lambdas, n_lambda, opts, entries, support, omega_best,
                     best_index, workspace, ws_bytes, out);
  });
  if (out) out->status = s;
  return s;
}

}  // extern "C"
