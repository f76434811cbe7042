// Host-side launchers exported by each CUDA translation unit of libaccord.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace accord {

// Records the first failure of the current call (thread-local): where it
// happened and the CUDA error or device error bits.  Read through
// accord_last_error().
void set_last_error(const char* where, int line, const char* what);
void clear_last_error();

// Epilogue roles of the fused GEMMs C = A * B^T (A: M x K, B: N x K, both
// row-major with K contiguous).
enum GemmMode : int {
  kModeY = 0,     // Y+ = Omega+ X^T: store Y+, reduce ||Y+ - Y||^2, ||Y+||^2
  kModeProx = 1,  // G = Y X / n -> Eq. 3.5 prox -> Omega+, reductions, KKT(Omega)
  kModeGrad = 2,  // G = Omega S (minus diag(1/omega) when smooth)
  kModeGram = 3,  // K = X X^T / n (for the Lipschitz constant)
};

// Operand and epilogue pointers.  Arrays of two are the double-buffered
// iterates: the kernel reads ctrl->cur (0 when ctrl is null) and uses
// A[a_nxt ? nxt : cur], aux[cur], out[nxt] with nxt = cur ^ 1.
struct GemmF64Params {
  const Ctrl* ctrl;
  const double* A[2];
  int64_t lda;
  const double* B;
  int64_t ldb;
  int64_t M, N, K;
  double* out[2];
  int64_t ldout;
  const double* aux[2];
  int64_t ldaux;
  double* part;
  double lam, lam_d, scale;
  int32_t a_nxt;
  int32_t smooth;
  const uint32_t* mask;  // Eq. 3.8 refit support bitmask, or null
  int64_t mask_ld;
  // Batch of problems with the same M, N, K (grid z = problem slot): problem
  // b = active[slot] (or slot) uses ctrl[b] for its step, penalty and 1/n and
  // the operands and outputs at + b * stride; finished problems do nothing.
  int32_t nprob;            // problems (1: a single fit)
  const int32_t* active;    // device list of problems, or null (0 .. nprob-1)
  const int32_t* nactive;   // device length of `active`
  int64_t s_a, s_b, s_out, s_aux, s_part;  // strides: elements (s_part: tiles)
  // Row block of Omega (prox / grad modes): output row r is row r + row_off
  // of the full matrix, so its diagonal entry sits in column r + row_off.
  int64_t row_off;
};

int64_t gemm_f64_tiles(int64_t M, int64_t N);
cudaError_t launch_gemm_f64(int mode, const GemmF64Params& prm, cudaStream_t st);

// ---------------------------------------------------------- misc kernels ---
cudaError_t launch_convert_x_f64(const float* X32, const double* X64in, int64_t n, int64_t p,
                                 double* X64, int64_t ldx, double* XT64, int64_t ldxt,
                                 int* bad_flag, cudaStream_t st);
// Operand planes (type pt, kPlaneBf16 or kPlaneTf32) of X and X^T.
cudaError_t launch_convert_x_planes(const float* X32, int64_t n, int64_t p, void* Xhi, void* Xlo, int64_t ldx,
                                    void* XThi, void* XTlo, int64_t ldxt, int* bad_flag, int pt, cudaStream_t st);
// Omega^0 = I in an internal buffer with leading dimension ld (elements); a
// row block (rows >= 0) holds rows row0 .. row0 + rows of it.
cudaError_t launch_set_identity(void* Om, int is_f64, int64_t p, int64_t ld, cudaStream_t st, int64_t rows = -1,
                                int64_t row0 = 0);
// Occupancy bitmaps of the mixed-mode iterate buffers (the prox epilogue's
// sparse reads and writes of Omega): ceil(p / 32) column chunks of
// bitmap_ld(p) words each; word [c * bitmap_ld(p) + i] has bit j - 32 c set
// iff Omega[i][j] != 0.  Rows past p hold 0.
// A row block of `rows` rows keeps ceil(p / 32) chunks of bitmap_ld(rows) words.
int64_t bitmap_ld(int64_t rows);
int64_t bitmap_words(int64_t rows, int64_t cols);
int64_t bitmap_words(int64_t p);
// rows >= 0: a row block holding rows row0 .. row0 + rows of the p x p matrix.
cudaError_t launch_identity_bitmap(uint32_t* bm, int64_t p, cudaStream_t st, int64_t rows = -1, int64_t row0 = 0);
// Dense copy (ld ldd) of an FP32 iterate buffer that counts only where its bitmap has a bit.
cudaError_t launch_copy_omega_masked(const float* src, int64_t lds, const uint32_t* bm, float* dst, int64_t ldd,
                                     int64_t p, cudaStream_t st, int64_t rows = -1);
cudaError_t launch_bitmap_from_dense(const float* Om, int64_t p, int64_t ld, uint32_t* bm, cudaStream_t st,
                                     int64_t rows = -1);
// Copy between a dense p x p user array (ld = p) and an internal buffer
// (rows >= 0: the first `rows` rows only).
cudaError_t launch_copy_omega(const void* src, int64_t lds, void* dst, int64_t ldd, int is_f64,
                              int64_t p, cudaStream_t st, int64_t rows = -1);
// Per-row-block statistics of Omega into kProxSlots partials (log-diag,
// diag sum, off-diagonal l1, nnz, bad count); returns the number of rows of
// partials written through *nparts.
cudaError_t launch_omega_stats(const void* Om, int is_f64, int64_t p, int64_t ld, double* part,
                               int64_t* nparts, cudaStream_t st, int64_t rows = -1, int64_t row0 = 0);
// Support bitmask of the Eq. 3.8 refit: bit (i, j) of word [i][j / 32] is set
// where Om_ij != 0 or i == j.  Om is p x p with leading dimension ld.
cudaError_t launch_support_mask(const void* Om, int is_f64, int64_t p, int64_t ld, uint32_t* mask, int64_t mask_ld,
                                cudaStream_t st);
// hi/lo planes (type pt) of an FP32 matrix (rows x cols, lds) into ldd planes.
cudaError_t launch_split_planes(const float* src, int64_t rows, int64_t cols, int64_t lds, void* hi, void* lo,
                                int64_t ldd, int pt, cudaStream_t st);

// Lanczos estimate of lambda_max of the symmetric n x n matrix K (FP64).
// V holds (kmax + 1) x n doubles, alpha / beta kmax doubles each, w n.
constexpr int kLanczosMax = 128;
// A batch of nprob problems (one Ctrl each) takes its slices of K, V, w and
// alpha / beta at the given strides (doubles).
// f32 = 1 runs the process in FP32 (V, w, alpha, beta are float arrays; the
// mixed modes), else in FP64 (double arrays).  K is FP64 in both.
cudaError_t launch_lanczos_init(Ctrl* ctrl, void* V, int64_t n, cudaStream_t st, int nprob = 1, int64_t sV = 0,
                                int f32 = 0);
cudaError_t launch_lanczos_steps(Ctrl* ctrl, const double* K, int64_t ldk, void* V, void* w, void* alpha, void* beta,
                                 int64_t n, int kmax, int nsteps, double tol, cudaStream_t st, int nprob = 1,
                                 int64_t sK = 0, int64_t sV = 0, int64_t sW = 0, int64_t sAB = 0, int f32 = 0);

// Control kernels of the Algorithm 1 loop.
cudaError_t launch_ctrl_init(Ctrl* ctrl, const double* ompart, int64_t nomp, const double* ypart,
                             int64_t nyp, const SolveParams& sp, double L_given, double* trace,
                             cudaStream_t st);
constexpr int kFoldChunks = 128;  // first-stage blocks of the prox-partials fold
cudaError_t launch_post_prox(Ctrl* ctrl, const double* part, int64_t ntiles, const SolveParams& sp,
                             double* trace, double* fold_scratch, cudaStream_t st);
// ||A||^2 partials (kYSlots rows, one per 64 rows of A); *nparts rows written.
cudaError_t launch_rows_norm2(const void* A, int is_f64, int64_t rows, int64_t cols, int64_t ld, double* part,
                              int64_t* nparts, cudaStream_t st);
// One kProxSlots partial row with the statistics of Omega = I.
cudaError_t launch_identity_stats(double* part, int64_t p, cudaStream_t st);
// delta_entries (or null): adds the number of Delta entries the sparse Y
// update applied in this trial.
cudaError_t launch_decide(Ctrl* ctrl, const double* part, int64_t ntiles, const SolveParams& sp,
                          double* trace, int* bucket_counts, int nbuckets, const double* part_sparse,
                          cudaStream_t st, unsigned long long* delta_entries = nullptr);
// Row blocks of one fit: fold this block's trial sums into out[0 .. 11]
// (kProxSlots prox sums, then the kYSlots sums of the Y update that ran;
// empties the buckets), and, once the caller has exchanged them over all
// blocks, take Algorithm 1's decisions on the global sums.
cudaError_t launch_fold_block(Ctrl* ctrl, const double* prox_part, int64_t ntiles_prox, double* fold_scratch,
                              const double* y_part, int64_t ntiles_y, int* bucket_counts, int nbuckets,
                              const double* part_sparse, unsigned long long* delta_entries, double* out,
                              cudaStream_t st);
cudaError_t launch_decide_global(Ctrl* ctrl, const double* sums, const SolveParams& sp, double* trace,
                                 cudaStream_t st);
// Loss helper: reduce Omega stats and Y partials into out[0] = f, out[1] = g.
cudaError_t launch_loss_finish(const double* ompart, int64_t nomp, const double* ypart, int64_t nyp,
                               double lam, double lam_d, double inv_n, double* out, cudaStream_t st);

// --------------------------------------------------- loss and gradient ---
// The loss parts res[0] = f, res[1] = g (device doubles) and the gradient
// G_out (smooth = 0: Omega S; 1: -diag(1/omega) + Omega S) of X at Omega,
// queued on opts.stream without waiting: one Y = Omega X^T serves both.
// err (device, 2 ints): [0] counts non-finite entries of X, [1] collects
// device error bits.  Scratch memory is freed in stream order.
int eval_loss_grad_async(const float* X, int64_t n, int64_t p, const void* Omega, const struct accord_opts& o,
                         double lambda, double* res, int smooth, void* G_out, int* err);

// ------------------------------------------------------------ lambda path ---
// A path runs one chain per subsample; chain c is problem c of the batch and
// walks the penalties lambdas[0..n_lambda) in order, each fit starting from
// the previous estimate.
struct PathDev {
  Ctrl* ctrl;
  int32_t nchains, n_lambda;
  const double* lambdas;   // device, in solve order
  const double* n_obs;     // device, rows of each chain's subsample (the n of Eq. 3.7)
  double gamma, log_p;
  int32_t penalize_diag;
  int32_t coarse;          // every penalty starts with one-product gradients (SolveParams::coarse_kkt > 0)
  PathRec* rec;            // device, n_lambda x nchains, record [k * nchains + c]
  double* best_epbic;      // device, per chain (initialised to +inf)
  int32_t* best_idx;       // device, per chain
  int32_t* active;         // device list of unfinished chains
  int32_t* nactive;
  int* any_dense;          // device flag: some chain takes the dense Y update next trial (or null)
};
// Finishes the per-chain control blocks after L is known: tau0, f and g of
// Omega^0 = I with Y^0 = X^T (yt0: p x ldy per chain, s_y elements apart).
cudaError_t launch_batch_ctrl_init(const PathDev& pd, const void* yt0, int is_f64, int64_t p, int64_t ldy,
                                   int64_t s_y, const SolveParams& sp, double L_given, cudaStream_t st);
// Batched post_prox / decide: block `slot` serves problem active[slot];
// partial rows of problem b start at part + b * ntiles rows.
cudaError_t launch_post_prox_batch(Ctrl* ctrl, int32_t nprob, const int32_t* active, const int32_t* nactive,
                                   const double* part, int64_t ntiles, const SolveParams& sp, cudaStream_t st);
// With buckets (part_sparse != null) it also picks each problem's Y-update
// mode for the next trial (Ctrl::ymode).
cudaError_t launch_decide_batch(Ctrl* ctrl, int32_t nprob, const int32_t* active, const int32_t* nactive,
                                const double* part, int64_t ntiles, const SolveParams& sp, int* bucket_counts,
                                int nbuckets, const double* part_sparse, cudaStream_t st);
// After each trial: record every estimate completed in it (status, sums,
// epBIC of Eq. 3.7), move its chain to the next penalty (warm start) or
// finish it, and rebuild the active list.
cudaError_t launch_path_advance(const PathDev& pd, cudaStream_t st);
// For each estimate recorded by the last advance: its support bits (if
// support != null; record k * nchains + c, p rows of mask_ld words) and, when
// its epBIC is the chain's best so far, a dense copy into omega_best + c p^2.
// Mixed modes pass the buffers' occupancy bitmaps (bm0, bm1, s_bm words per
// chain): a buffer's values count only where its bitmap has a bit.
cudaError_t launch_path_emit(const PathDev& pd, const void* om0, const void* om1, int is_f64, int64_t p,
                             int64_t ldo, int64_t s_om, uint32_t* support, int64_t mask_ld, void* omega_best,
                             cudaStream_t st, const uint32_t* bm0 = nullptr, const uint32_t* bm1 = nullptr,
                             int64_t s_bm = 0);

// ------------------------------------------------------ sparse Y update ---
// Rows of 32 share one bucket of Delta entries: key = (row - 32 b) << 25 | col,
// value = Delta_ij (FP32), count in counts[b] (may exceed cap: overflow).
constexpr int kBucketRows = 32;
struct SparseYParams {
  const Ctrl* ctrl;           // a batch: one per problem (grid y = problem slot)
  const float* y[2];          // Y (p x ldy FP32), index cur / nxt
  float* yw[2];
  void* y_hi[2];              // planes of Y+ (p x ldyk, type ptype), index nxt
  void* y_lo[2];
  const float* xt;            // X^T, p x ldy FP32
  const uint32_t* keys;
  const float* vals;
  const int* counts;
  int32_t cap, tiles_m, tiles_n, ptype;
  int64_t p, n, ldy, ldyk;
  double* part;               // one row of kYSlots per bucket
  // batch: problem b = active[slot] (or slot), data at + b * stride
  const int32_t* active;
  const int32_t* nactive;
  int32_t nprob;
  int64_t s_y, s_yk, s_xt, s_bkt;  // strides: Y (elements), planes, X^T, buckets
};
// Y of the current iterate formed afresh from Omega^t (mixed modes): for a
// problem whose ctrl->refresh is set, Y[cur] and its operand planes become
// Omega[cur] X^T (FP32, the nonzeros of Omega's occupancy bitmap in
// ascending column order); part gets one row of kYSlots per 32-row group
// (kYDiff2: ||Y_old - Y_new||^2, kYNorm2: ||Y_new||^2, kYBad).  A batch runs
// grid y over problem slots with data at + b * stride.
struct YRefreshParams {
  const Ctrl* ctrl;
  const float* om[2];      // Omega buffers (rows x ldo FP32), index cur
  const uint32_t* bm[2];   // their occupancy bitmaps (chunk-major, ldbm words a chunk)
  float* y[2];             // Y (rows x ldy FP32)
  void* y_hi[2];           // planes of Y (rows x ldyk, type ptype)
  void* y_lo[2];
  const float* xt;         // X^T, p x ldx FP32
  int64_t rows, p, n, ldo, ldbm, ldy, ldyk, ldx;
  double* part;
  int32_t ptype, nprob;
  const int32_t* active;
  const int32_t* nactive;
  int64_t s_om, s_bm, s_y, s_yk, s_xt, s_part;  // per-problem strides (elements / words / doubles)
  double dense_nnz;        // off-diagonal nonzeros of Omega from which the blocked (dense) form runs
  // set by launch_y_refresh from the testing hook: 0 to list a 32-row
  // group's nonzeros together when they fit, else the nonzeros of a row the
  // row-by-row walk lists at once; and the form (0: by dense_nnz, 1: the
  // walk, 2: the blocked product)
  int32_t list_cap, form;
};
// Two kernels per call: the walk over Omega's nonzeros (listed per 32-row
// group, then gathered one warp a row), and a blocked product for a problem
// with at least dense_nnz nonzeros; each problem takes exactly one of them.
cudaError_t launch_y_refresh(const YRefreshParams& prm, cudaStream_t st);
// Testing hook (accord_test_refresh): list_cap and form for later launches.
void y_refresh_set_test(int list_cap, int form);
// Folds the refresh partials (ngroups rows of kYSlots per problem, s_part
// doubles apart): y_drift = max(y_drift, sqrt(||Y_old - Y_new||^2 /
// ||Y_new||^2)); with update_g, g and f of the iterate from ||Y_new||^2; then
// clears refresh and since_refresh.  One block per problem slot.
cudaError_t launch_y_refresh_fold(Ctrl* ctrl, int32_t nprob, const int32_t* active, const int32_t* nactive,
                                  const double* part, int64_t ngroups, int64_t s_part, int update_g,
                                  cudaStream_t st);
size_t sparse_y_smem_bytes(int cap);
cudaError_t launch_sparse_y(const SparseYParams& prm, cudaStream_t st);
cudaError_t sparse_y_prepare();  // one-time shared-memory opt-in (before a graph capture)
// Dense fallback: planes (type pt) of Delta = Omega[nxt] - Omega[cur] when ctrl->dense.
// A batch runs grid y over problem slots (active list or 0 .. nprob-1) with
// Omega at + b * s_om and the planes at + b * s_pl.
// The buffers count only where their occupancy bitmaps (bm0, bm1; s_bm words
// apart in a batch) have a bit.
cudaError_t launch_delta_planes(const Ctrl* ctrl, const float* om0, const float* om1, const uint32_t* bm0,
                                const uint32_t* bm1, int64_t p, int64_t ld, void* hi, void* lo, int64_t ldk, int pt,
                                cudaStream_t st, int32_t nprob = 1, const int32_t* active = nullptr,
                                const int32_t* nactive = nullptr, int64_t s_om = 0, int64_t s_pl = 0,
                                const int* any_dense = nullptr, int64_t s_bm = 0, int64_t rows = -1);
// X^T in FP32 (p x ldxt).
cudaError_t launch_transpose_x_f32(const float* X, int64_t n, int64_t p, float* XT, int64_t ldxt, cudaStream_t st);

}  // namespace accord
