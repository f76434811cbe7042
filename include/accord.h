/*
 * accord.h -- C ABI of the GB300 ACCORD-FBS solver (HP-ACCORD, arXiv 2412.11554).
 *
 * The library fits the ACCORD estimator (Eq. 3.2)
 *
 *     Omega-hat = argmin_Omega  -sum_i log omega_ii + 1/2 tr(Omega^T Omega S) + lambda ||Omega||_1,
 *     S = X^T X / n,
 *
 * with the forward-backward splitting of Eq. 3.4, the elementwise update of
 * Eq. 3.5 and the backtracking line search of Algorithm 1.  The gradient
 * Omega S is formed in two steps, Y = Omega X^T and (1/n) Y X (Sec 3.3), on the
 * GPU; nothing runs on the CPU except argument checks and launch control.
 *
 * Conventions shared by every entry point
 *   - X is n x p, row-major (rows are samples, as in Sec 2), never centred or
 *     scaled by the library, divisor n in S.
 *   - Omega is p x p, row-major, dense, asymmetric.  Its element type follows
 *     opts->precision: double for ACCORD_FP64, float for the mixed modes.
 *   - All array pointers are DEVICE pointers owned by the caller; the library
 *     never frees them and never keeps them after the call returns.
 *   - Work is queued on opts->stream (a cudaStream_t; NULL = legacy default
 *     stream).  Every call returns after synchronising that stream, so
 *     outputs are ready when it returns, with two exceptions that say so
 *     below: accord_to_csr queues its fill after its one synchronisation, and
 *     accord_loss_f64_noalloc does not synchronise at all.
 *   - Return value: ACCORD_OK (0), a positive soft status, or a negative error.
 *     No call aborts, throws or traps the GPU; device loops are bounded.
 *   - Only compute capability 10.3 (GB300, sm_103a) is supported; any other
 *     device gives ACCORD_EUNSUPPORTED.  There is no CPU fallback.
 *   - Host threads: the first call of an entry point on a device sets kernel
 *     attributes (shared memory opt-in, persistent grid size) and caches them
 *     in unsynchronised process-wide variables.  Make that first call from one
 *     thread; after it, calls from several threads on their own streams and
 *     workspaces are independent (the tile autotuner's table is locked),
 *     except accord_loss_f64_noalloc, whose scratch array all calls share.
 */
#ifndef ACCORD_H_
#define ACCORD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define ACCORD_OK             0   /* converged: KKT residual <= kkt_tol                */
#define ACCORD_NOT_CONVERGED  1   /* max_iter accepted steps; Omega = last iterate      */
#define ACCORD_EINVAL        -1   /* NULL pointer, n < 1, p < 1, lambda < 0, bad opts   */
#define ACCORD_EDOMAIN       -2   /* warm start with omega_ii <= 0 or non-finite entry  */
#define ACCORD_ENONFINITE    -3   /* NaN/Inf appeared in an iterate or a reduction      */
#define ACCORD_EBACKTRACK    -4   /* max_backtracks step reductions without acceptance  */
#define ACCORD_ENOMEM        -5   /* workspace too small, or allocation failed          */
#define ACCORD_ECUDA         -6   /* CUDA runtime/driver error, or a device wait gave up */
#define ACCORD_EUNSUPPORTED  -7   /* device is not sm_103, or option not supported      */

/* ---- precision modes --------------------------------------------------- */
#define ACCORD_FP64          0    /* FP64 GEMMs, FP64 iterate                           */
#define ACCORD_MIXED_BF16X3  1    /* tcgen05 BF16 hi+lo split GEMMs (3 products),
                                     FP32 accumulation, FP32 iterate, FP64 reductions   */
#define ACCORD_MIXED_TF32X3  2    /* as BF16X3 with TF32 hi+lo planes (kind::tf32 MMAs):
                                     hi+lo carry an operand to 2^-24 instead of 2^-18,
                                     so a product's error is that of its FP32
                                     accumulation: more accurate than BF16X3 when n is
                                     small (tens of samples), about as accurate from n
                                     of a few hundred.  Half the tensor rate and twice
                                     the plane bytes of BF16X3; same API data types.    */

/* Columns of one trace row (one row per iterate Omega^t, t = 0..iters). */
#define ACCORD_TRACE_FIELDS  8
#define ACCORD_TRACE_F       0    /* f(Omega^t)                                         */
#define ACCORD_TRACE_KKT     1    /* KKT residual r(Omega^t)                             */
#define ACCORD_TRACE_TAU     2    /* accepted step tau_t (Omega^t -> Omega^t+1)          */
#define ACCORD_TRACE_NTRIALS 3    /* prox evaluations spent on step t                    */
#define ACCORD_TRACE_NNZ     4    /* off-diagonal nonzeros of Omega^t                    */
#define ACCORD_TRACE_DELTA   5    /* ||Omega^t+1 - Omega^t||_F                           */
#define ACCORD_TRACE_G       6    /* g(Omega^t) = ||Omega^t X^T||_F^2 / (2n)             */

typedef struct accord_opts {
    int32_t precision;       /* ACCORD_FP64, ACCORD_MIXED_BF16X3 (default) or ACCORD_MIXED_TF32X3 */
    int32_t tau_warm;        /* 0: every outer step starts at tau0 (Algorithm 1 as printed);
                                1: starts at min(tau0, tau_{t-1}/beta)                         */
    int32_t max_iter;        /* accepted steps allowed (default 500)                           */
    int32_t max_backtracks;  /* step reductions allowed per outer step (default 60)            */
    int32_t penalize_diag;   /* 1: lambda on the diagonal too (Eq. 3.2, default); 0: off only  */
    int32_t init_from_omega; /* 1: Omega holds the starting iterate on entry; 0: Omega^0 = I   */
    int32_t lipschitz_max_iter; /* Lanczos steps allowed for L, at most 128 (default 128)    */
    int32_t profile;         /* 1: time every GEMM launch with CUDA events (stats t_*_gemm_ms)  */
    int32_t sparse_update;   /* mixed modes: 1 (default) forms Y+ = Y + Delta X^T from the nonzero
                                entries of Delta (the iterate is sparse); 0: dense tensor-core
                                product every trial.  Ignored in FP64 mode (always dense).    */
    int32_t autotune;        /* accord_path, mixed modes: 1 (default) times the batched prox GEMM's
                                tile raster and persistent grid on the first call for a shape
                                and keeps the fastest; 0: fixed defaults                         */
    double  tau0;            /* initial step (default 1); <= 0 means 1/L                        */
    double  beta;            /* backtracking factor in (0, 1]; 1 = fixed step (default 0.5)     */
    double  kkt_tol;         /* stop when r(Omega^t) <= kkt_tol (default 1e-8)                  */
    double  lipschitz;       /* > 0: use this L = sigma_max(S); 0: estimate it by Lanczos on
                                X X^T / n (default 0)                                            */
    double  lipschitz_tol;   /* relative change of the Ritz value that ends Lanczos; 0 (default)
                                = 1e-14 in FP64 mode (FP64 process), 1e-6 in the mixed modes
                                (FP32 process: there L only sets the tau <= 1/L floor)           */
    double  epbic_gamma;     /* gamma of the extended pseudo-BIC, Eq. 3.7 (default 0.5)         */
    void*   stream;          /* cudaStream_t for all work (default NULL)                        */
    double* trace;           /* optional HOST array, trace_cap x ACCORD_TRACE_FIELDS doubles    */
    int64_t trace_cap;       /* rows available in trace (rows beyond are dropped)               */
    int32_t y_refresh;       /* mixed modes: Y = Omega X^T is carried from step to step as
                                Y + Delta X^T in FP32, which accumulates rounding; every
                                y_refresh accepted steps (default 32), ahead of a step whose KKT
                                test the last ratio of residuals predicts to pass (once per fit
                                or path penalty if the prediction misses), and before a KKT
                                residual under kkt_tol may end a fit (that trial is then cut
                                short), Y is formed afresh from the iterate.  0: never (the
                                residual test then uses the carried Y).  Ignored in FP64 mode,
                                where every trial forms Y+ = Omega+ X^T.                        */
    int32_t reserved1;
    double  coarse_kkt;      /* mixed modes: while the KKT residual is above this (default 5e-3),
                                the prox GEMM forms G with the one product hi x hi instead of the
                                three split products (G then carries the error of one BF16 or TF32
                                product, about 1e-4 of |G| at n = 1000); the first residual under it
                                switches to the three products for the rest of the fit (and a
                                path's penalty), and no fit ends on a one-product residual.
                                0: three products throughout.  Ignored in FP64 mode.           */
} accord_opts;

typedef struct accord_stats {
    int32_t iters;           /* accepted steps taken                                            */
    int32_t trials;          /* prox evaluations (accepted + rejected; a trial whose KKT test
                                asked for a refresh of Y is not one)                             */
    int32_t status;          /* same value as the call's return                                  */
    int32_t y_refreshes;     /* mixed modes: times Y was formed afresh (opts->y_refresh)         */
    double  f;               /* objective of the returned Omega (Eq. 3.2)                        */
    double  g;               /* its smooth part g = 1/2 tr(Omega^T Omega S)                      */
    double  kkt;             /* its KKT residual                                                 */
    double  tau_last;        /* last accepted step                                               */
    double  L;               /* Lipschitz constant used (estimated or given)                     */
    int64_t nnz_offdiag;     /* off-diagonal nonzeros of the returned Omega                     */
    double  t_setup_ms;      /* device time: conversions, L estimate, Omega^0, Y^0              */
    double  t_solve_ms;      /* device time: the iteration loop and the copy-out                 */
    int32_t n_prox_gemm;     /* prox GEMM launches that did work (trials, trials cut short by a
                                refresh of Y, and the final KKT check)                           */
    int32_t n_y_gemm;        /* Y GEMM launches that did work (one per trial)                    */
    double  t_prox_gemm_ms;  /* their summed device time when opts->profile, else 0              */
    double  t_y_gemm_ms;
    int64_t n_launches;      /* kernels this call launched (setup + every queued trial)          */
    double  logdet_d;        /* sum_i log omega_ii of the returned Omega                         */
    double  epbic;           /* extended pseudo-BIC of Eq. 3.7 with opts->epbic_gamma:
                                2n(-log det Omega_D + g) + nnz (log n + 4 gamma log p)           */
    int32_t tile_group_m;    /* accord_path, mixed modes: raster group (rows of 256-row pair
                                tiles) of the batched prox GEMM in use (0 elsewhere)             */
    int32_t tile_pairs;      /* ... and its persistent grid in CTA pairs (2 SMs each)            */
    int64_t delta_entries;   /* mixed modes, single fit: nonzero Delta entries the sparse Y
                                update applied, summed over the trials (0 elsewhere)             */
    double  y_drift;         /* mixed modes: the largest ||Y - Omega X^T||_F / ||Omega X^T||_F
                                that a refresh of Y found (the rounding the carried Y had
                                gathered since the one before); accord_path: the largest over
                                every chain and penalty.  0 in FP64 mode.                        */
    double  t_graph_idle_ms; /* accord_path: device time of one replay of its captured trial
                                graph after every chain has finished, when each of its kernels
                                returns at once: what launching a replay costs (0 elsewhere)     */
    int32_t coarse_prox;     /* mixed modes: prox launches that formed G with one product
                                (opts->coarse_kkt); accord_path: summed over the chains          */
    int32_t reserved2;
} accord_stats;

/* Fills *opts with the defaults listed above. */
void accord_default_opts(accord_opts* opts);

/* Device workspace, in bytes, that accord_fit (Algorithm 1) needs for an
 * n x p problem under opts (precision and max_iter matter).  Returns 0 for
 * invalid sizes.
 * It grows as about 12.6 p^2 bytes in BF16X3 mode, 16.8 p^2 in TF32X3 mode
 * and 16.4 p^2 in FP64 mode.  With the caller's Omega on the same GPU, a
 * 284 GB GB300 holds at n = 1000 a fit of p up to about 131000 (BF16X3),
 * 117000 (TF32X3) or 108000 (FP64). */
size_t accord_workspace_bytes(int64_t n, int64_t p, const accord_opts* opts);

/* ACCORD-FBS fit (Algorithm 1 with Eq. 3.5; stopping rule r(Omega^t) <= kkt_tol
 * with r the max-abs minimum-norm subgradient of Eq. 3.3).
 *   X          device, n x p float, row-major.
 *   lambda     >= 0, penalty weight of Eq. 3.2.
 *   opts       may be NULL (defaults).
 *   Omega      device, p x p, double (FP64) or float (mixed).  Read on entry
 *              only when opts->init_from_omega; always overwritten with the
 *              returned iterate (also on NOT_CONVERGED / EBACKTRACK /
 *              ENONFINITE, where it is the last accepted iterate).
 *   workspace  device buffer of at least accord_workspace_bytes(n, p, opts)
 *              bytes, 256-byte aligned; NULL makes the call allocate and free
 *              its own on the stream.
 *   out        optional host stats.
 * Errors: EINVAL (arguments), ENOMEM (ws_bytes too small), EDOMAIN (bad warm
 * start or non-finite X), ENONFINITE, EBACKTRACK, ECUDA, EUNSUPPORTED. */
int accord_fit(const float* X, int64_t n, int64_t p, double lambda, const accord_opts* opts,
               void* Omega, void* workspace, size_t ws_bytes, accord_stats* out);

/* Bias-corrected refit (Eq. 3.8): Algorithm 1 on
 *   -log det Omega_D + 1/2 tr(Omega^T Omega S) + phi lambda ||Omega||_1
 * over the Omega whose entries vanish off the support of Omega_hat (device,
 * p x p, element type per precision; its nonzero pattern plus the diagonal is
 * the support).  Off the support the weight is infinite, so those entries
 * stay 0 and do not enter the KKT residual.  0 <= phi <= 1 (else EINVAL).
 * Other arguments, workspace and errors as accord_fit; opts->init_from_omega
 * may start from Omega_hat copied into Omega. */
int accord_refit(const float* X, int64_t n, int64_t p, double lambda, double phi, const void* Omega_hat,
                 const accord_opts* opts, void* Omega, void* workspace, size_t ws_bytes, accord_stats* out);

/* Same as accord_fit (Algorithm 1 with Eq. 3.5) for FP64 data; requires
 * opts->precision == ACCORD_FP64 (else EUNSUPPORTED).  Omega is double.
 * Errors as accord_fit. */
int accord_fit_f64(const double* X, int64_t n, int64_t p, double lambda, const accord_opts* opts,
                   double* Omega, void* workspace, size_t ws_bytes, accord_stats* out);

/* Objective of Eq. 3.2 at Omega (device, p x p, element type per precision):
 *   *g_out = 1/2 tr(Omega^T Omega S) = ||Omega X^T||_F^2 / (2n)   (Eq. 3.4)
 *   *f_out = *g_out - sum_i log omega_ii + lambda sum_{i!=j} |omega_ij|
 *            + lambda_d sum_i omega_ii, lambda_d = lambda or 0 per penalize_diag;
 *            +Inf when some omega_ii <= 0.
 * f_out, g_out are HOST doubles (either may be NULL).  Allocates its scratch
 * on opts->stream (stream-ordered) and frees it before returning.
 * Errors: EINVAL (NULL X or Omega, n < 1, p < 1, lambda < 0 or not finite,
 * unknown precision), EDOMAIN (non-finite X), ENOMEM (scratch), ECUDA,
 * EUNSUPPORTED (not sm_103). */
int accord_loss(const float* X, int64_t n, int64_t p, const void* Omega, double lambda,
                const accord_opts* opts, double* f_out, double* g_out);

/* Gradient of the smooth part (Sec 3.2):
 *   smooth = 0:  G_out = Omega S = (1/n)(Omega X^T) X                 (grad g, Eq. 3.4)
 *   smooth = 1:  G_out = -Omega_D^{-1} + Omega S  (gradient of Eq. 3.1's sample loss;
 *                the first two terms of the KKT condition Eq. 3.3)
 * G_out: device p x p, same element type as Omega, row-major, may not alias Omega.
 * Allocates its scratch on opts->stream and frees it before returning.
 * Errors: EINVAL (NULL X, Omega or G_out, G_out == Omega, n < 1, p < 1,
 * unknown precision), EDOMAIN (non-finite X), ENOMEM, ECUDA, EUNSUPPORTED. */
int accord_grad(const float* X, int64_t n, int64_t p, const void* Omega, int smooth,
                const accord_opts* opts, void* G_out);

/* Static description of a status code. */
const char* accord_status_string(int status);

/* ACCORD_OK when the current device is sm_103 and the kernels load, else
 * ACCORD_EUNSUPPORTED / ACCORD_ECUDA. */
int accord_device_check(void);

/* Size of the static device scratch array used by accord_loss_f64_noalloc. */
#define ACCORD_NOALLOC_SCRATCH_BYTES (8u << 20)

/* accord_loss without any device allocation, for callers that must not
 * allocate: code inside a custom allocator's callback, latency-bound loops
 * that cannot afford the allocator's implicit synchronisation, or processes
 * whose device memory another caching allocator has already reserved.  The
 * paper has no counterpart; it is an interface convenience.
 *   X        device, n x p double, row-major (FP64 data: no conversion buffer).
 *   Omega    device, p x p double, row-major.
 *   fg_out   device, 2 doubles: fg_out[0] = f, fg_out[1] = g, as accord_loss.
 *   stream   cudaStream_t (NULL = legacy default stream); the call does not
 *            synchronise it -- read fg_out after the stream's work completes.
 * Domain errors: the call never reads its results back, so its status cannot
 * report them (accord_loss returns ACCORD_EDOMAIN instead).  Check fg_out:
 * f = +inf when a diagonal entry of Omega is non-positive or non-finite, and
 * f = g = NaN when X holds a non-finite value.  n or p above 2^31 - 1 gives
 * ACCORD_EINVAL before anything is sized or launched.
 * Scratch: a file-scope __device__ array of ACCORD_NOALLOC_SCRATCH_BYTES bytes
 * per GPU, held until the process exits; the call needs
 * 32 * ceil(p/64) * ceil(n/64) + 64 * p bytes of it (each part rounded up to
 * 256) and returns ACCORD_ENOMEM when that exceeds the array (for n = 1000 this
 * allows p up to about 116000).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current: make
 * that first call before any stream capture.  All calls share the array, so
 * calls whose work overlaps on the GPU (other streams, unordered host threads)
 * race on it; the array's previous contents are never read. */
int accord_loss_f64_noalloc(const double* X, int64_t n, int64_t p, const double* Omega, double lambda,
                            int penalize_diag, void* stream, double* fg_out);

/* Testing hook for the bounded device waits (the paper has no counterpart).
 * Every mbarrier wait of the tensor-core kernels gives up after a time limit,
 * sets a device error bit, lets the copies it issued land, frees its TMEM and
 * returns; the call then reports ACCORD_ECUDA and accord_last_error() names
 * the timeout.  This sets that limit for every later launch in the process
 * (wait_limit_ns = 0 restores the default of 4 s) and, with
 * withhold_next_prox = 1, makes the producers of the next prox GEMM launch
 * (mixed modes) skip the copies of their first pipeline stage, so that the
 * MMA issuer's first wait runs out with no copy in flight for that stage.
 * Returns ACCORD_OK, or ACCORD_EINVAL for a negative limit or a flag other
 * than 0 / 1.  Not for production use: a short limit can end correct work. */
int accord_test_wait_limit(int64_t wait_limit_ns, int32_t withhold_next_prox);

/* Testing hook for the refresh of Y = Omega X^T in the mixed modes (the paper
 * has no counterpart; Y is re-formed from the iterate so that the FP32
 * rounding of the carried Y + Delta X^T does not build up).  The refresh has
 * two forms that give the same bits: a walk over the nonzeros of Omega, and a
 * blocked product used from p^2 / 10 nonzeros on.  The walk lists the
 * nonzero columns of a group of 32 rows together when they number at most
 * 4096, and otherwise row by row, up to 512 of a row at a time, working a
 * longer row in segments.  For every later launch in the process,
 *   list_cap: 0 for that choice, or 32 .. 512 to walk every group row by row
 *             with at most that many of a row's nonzeros listed at a time;
 *   form:     0 to choose by the nonzero count, 1 the walk, 2 the blocked form.
 * Returns ACCORD_OK, or ACCORD_EINVAL for values outside those ranges.  The
 * results do not depend on either setting, only the time does. */
int accord_test_refresh(int32_t list_cap, int32_t form);

/* Row blocks of one fit.  The objective of Eq. 3.2 separates over the rows
 * of Omega (the row-wise form in the proof of Thm 3.2), as the paper's
 * distributed solver uses when it spreads Omega over nodes by rows (Sec 3.3):
 * a fit can be split into blocks of rows that keep X whole and share only
 * the scalars of Algorithm 1.  Each block calls accord_fit_rows (on its own
 * GPU, or its own stream); once per trial every block passes its sums to
 * `exchange`, which must return the sums over all blocks of the partition,
 * so that every block takes the same decisions and the blocks together
 * follow the iterate sequence of one accord_fit.
 *
 *   exchange(sums, 9, maxes, 1, ctx): on entry this block's values; on
 *            return, element by element, the sums (sums) and the maxima
 *            (maxes) over all blocks.  sums: ||Delta||_F^2, sum log
 *            omega+_ii, sum omega+_ii, sum |omega+_ij| off the diagonal,
 *            off-diagonal nonzeros, non-finite count, ||Delta X^T||_F^2,
 *            ||Y+||_F^2, non-finite count of Y+; maxes: the KKT residual of
 *            Eq. 3.3.  It is called once before the first trial (the sums
 *            of Omega^0 and Y^0 = Omega^0 X^T, the KKT maximum 0) and once
 *            per trial, the same number of times in every block; a nonzero
 *            return ends the fit with ACCORD_ECUDA.  It runs on the calling
 *            thread, which waits for it.
 *   X        device, n x p row-major FP32, the whole data matrix on every
 *            block.
 *   row0, rows  this block holds rows row0 .. row0 + rows - 1 of Omega;
 *            row0 must be a multiple of 32 (the diagonal then crosses whole
 *            32 x 32 blocks of the kernels), rows >= 1, row0 + rows <= p.
 *   Omega_rows  device, rows x p row-major (FP32 in the mixed modes, FP64 in
 *            FP64 mode): the block's rows of Omega-hat on return, its rows of
 *            the starting iterate on entry when opts->init_from_omega.
 *   opts, lambda, n, p: the same in every block (the stream and workspace
 *            may differ).  The support-restricted refit is not offered here.
 *   out      the stats of the whole fit: f, g, the KKT residual, nnz and the
 *            counts are global and the same in every block.
 * Returns as accord_fit; ACCORD_EINVAL for a bad row range or a null
 * exchange.  One fit of the whole matrix is the case row0 = 0, rows = p. */
typedef int (*accord_exchange_fn)(double* sums, int32_t nsums, double* maxes, int32_t nmaxes, void* ctx);
int accord_fit_rows(const float* X, int64_t n, int64_t p, int64_t row0, int64_t rows, double lambda,
                    const accord_opts* opts, accord_exchange_fn exchange, void* ctx, void* Omega_rows,
                    void* workspace, size_t ws_bytes, accord_stats* out);
/* Device workspace, in bytes, of accord_fit_rows for a block of `rows` rows
 * (0 for invalid sizes). */
size_t accord_fit_rows_workspace_bytes(int64_t n, int64_t p, int64_t rows, const accord_opts* opts);

/* Description of the first failure of the calling thread's most recent call
 * of an entry point that queues GPU work (fit, refit, path, loss, gradients,
 * derivative, post-processing, CSR export; "" when it succeeded): the
 * source location and the CUDA error string or the device error bits.  The
 * pointer stays valid until the thread's next call. */
const char* accord_last_error(void);

/* ---- post-processing (Sec 3.1) ----------------------------------------------- */

/* The post-processing of Sec 3.1.  From an estimate Omega (device p x p,
 * element type per opts->precision):
 *   Theta_out = T^-1(Omega) = Omega_D Omega, theta_ij = omega_ii omega_ij (the
 *               precision-matrix estimate), and/or
 *   Rho_out   = partial correlations rho_ij = -(1/2)(omega_ij / omega_jj + omega_ji / omega_ii),
 *               rho_ii = 1.
 * Either output may be NULL (not both); both are device p x p, same element
 * type, and must not alias Omega.  Errors: EINVAL (NULL Omega, both outputs
 * NULL, p < 1 or p > 2097120 (65535 row tiles of 32), unknown precision),
 * EDOMAIN when a diagonal entry is not positive (the outputs are still
 * written), ENOMEM, ECUDA, EUNSUPPORTED. */
int accord_postprocess(int64_t p, const void* Omega, const accord_opts* opts, void* Theta_out, void* Rho_out);

/* Compressed sparse rows of an estimate (Sec 3.1: the estimated graph is the
 * nonzero pattern of Omega-hat): the entries of Omega (device p x p,
 * row-major, element type per opts->precision) that are not +-0, row by row
 * in increasing column order; a NaN counts as nonzero.
 *   row_ptr  device int64_t[p + 1]: row i's entries are [row_ptr[i], row_ptr[i+1]);
 *   col_idx  device int32_t[cap]: their columns;
 *   vals     device [cap], Omega's element type: their values;
 *   cap      entries col_idx and vals can hold;
 *   *nnz     host: the number of nonzeros (written on every return after the
 *            argument checks).
 * When *nnz exceeds cap the call returns ACCORD_ENOMEM having written row_ptr
 * only: call again with cap >= *nnz.  p must be below 2^31.  Synchronises the
 * stream once, to read the count; the fill is queued after it. */
int accord_to_csr(int64_t p, const void* Omega, const accord_opts* opts, int64_t* row_ptr, int32_t* col_idx,
                  void* vals, int64_t cap, int64_t* nnz);

/* ---- differentiation ------------------------------------------------------ */

/* Adjoint in the data of the smooth loss, the unpenalised part of Eq. 3.2,
 * L(Omega; X) = -sum_i log omega_ii + 1/2 tr(Omega^T Omega S): only g (Eq. 3.4)
 * depends on X, so GX_out = dL/dX = (1/n) X Omega^T Omega (n x p, device,
 * element type per precision: double for ACCORD_FP64, float for the mixed
 * modes), formed as Y^T = X Omega^T and (1/n) Y^T Omega.  dL/dOmega =
 * -diag(1/omega_ii) + Omega S is accord_grad with smooth = 1.  X: device n x p
 * FP32; Omega: device p x p, element type per precision.  The call allocates
 * its scratch on opts->stream and frees it before returning.
 * Errors: EINVAL (NULL X, Omega or GX_out, n < 1, p < 1, unknown precision),
 * EDOMAIN (non-finite X; non-finite Omega in FP64 mode), ENOMEM, ECUDA,
 * EUNSUPPORTED. */
int accord_grad_x(const float* X, int64_t n, int64_t p, const void* Omega, const accord_opts* opts,
                  void* GX_out);

/* Derivative of a held-out loss along the regularisation path:
 *   dloss = d L(Omega-hat(lambda); X_val) / d log(lambda),
 * L as in accord_grad_x, Omega-hat = the ACCORD estimate of X_train at lambda,
 * by implicit differentiation of the stationarity conditions (Eq. 3.3) on the
 * active set of Omega_hat: row i with active set A (nonzeros of row i, i
 * included) and signs s solves (S_AA + omega_ii^-2 e_i e_i^T) dw = -lambda v,
 * v = s off the diagonal and v_i = 1 when opts->penalize_diag (else 0), with
 * S = X_train^T X_train / n.  Valid where the active set is locally constant.
 *   X_train   device, n x p FP32;  X_val  device, n_val x p FP32
 *   Omega_hat device, p x p, element type per opts->precision (a converged estimate)
 *   dloss, loss_val  host (either may be NULL): the derivative and L(Omega_hat; X_val)
 *   dOmega    device or NULL: p x p dOmega-hat / dlog(lambda), element type per precision
 * FP64 mode forms S and the held-out products with FP64 GEMMs; the mixed modes
 * use their split-operand tensor-core products (FP32 accumulation, S written
 * in FP64, FP64 reductions).  The row systems are FP64 in all modes: one
 * CTA a row in shared memory up to 128 active entries, larger ones in a
 * second pass with the system in the workspace (up to 1024 entries).
 * Errors: EINVAL; EUNSUPPORTED when a row's active set has more
 * than 1024 entries; EDOMAIN when a row system is not positive definite (an
 * active set larger than the training rows can support) or Omega_hat has a
 * non-positive diagonal. */
int accord_dloss_dloglam(const float* X_train, int64_t n, const float* X_val, int64_t n_val, int64_t p,
                         const void* Omega_hat, double lambda, const accord_opts* opts, double* dloss,
                         double* loss_val, void* dOmega);

/* ---- lambda path over subsamples (Sec 3.4) ------------------------------ */

/* One estimate of a path: record [k * n_sub + s] for penalty k, subsample s. */
typedef struct {
    int32_t status;          /* ACCORD_OK, ACCORD_NOT_CONVERGED (max_iter steps at this
                                penalty; the chain still moves on), or an error, which also
                                ends the chain (its later records carry the same status)   */
    int32_t iters;           /* accepted steps at this penalty                              */
    int32_t trials;          /* prox evaluations at this penalty                            */
    int32_t y_refreshes;     /* mixed modes: refreshes of Y at this penalty                 */
    double  lambda;          /* the penalty                                                 */
    double  f, g, kkt;       /* objective (Eq. 3.2), smooth part, KKT residual (Eq. 3.3)    */
    double  logdet_d;        /* sum_i log omega_ii                                          */
    double  epbic;           /* Eq. 3.7 with n = the subsample's row count and
                                opts->epbic_gamma (+inf after an error)                     */
    double  tau_last;        /* last accepted step                                          */
    int64_t nnz_offdiag;     /* ||Omega||_0 off the diagonal                                */
    double  y_drift;         /* mixed modes: the largest relative drift of Y a refresh found
                                at this penalty (accord_stats.y_drift)                      */
} accord_path_entry;

/* Tuning by epBIC over a penalty grid (Sec 3.4) on subsamples of one data set.
 * Subsample s is the data matrix X[rows[row_offsets[s] .. row_offsets[s+1])]
 * (rows may repeat, as in a bootstrap sample).  For every subsample the
 * penalties lambdas[0 .. n_lambda) are solved in the given order, each fit
 * starting from the previous penalty's estimate of that subsample (warm start;
 * the first starts at Omega = I), with Algorithm 1 and opts as in accord_fit.
 * All subsamples run together as one batch on the GPU.
 *   X            device, n x p row-major FP32 (the whole data set)
 *   rows         host, int32 row indices in [0, n)
 *   row_offsets  host, n_sub + 1 offsets into rows, row_offsets[0] = 0, each
 *                subsample non-empty; 1 <= n_sub <= 65535
 *   lambdas      host, n_lambda >= 1 finite penalties >= 0 (decreasing is the usual path)
 *   entries      host, n_lambda * n_sub records (required)
 *   support      device or NULL: n_lambda * n_sub support bitmasks, record
 *                [k * n_sub + s], each p rows of ceil(p / 32) uint32 words;
 *                bit j % 32 of word [i][j / 32] is set where omega_ij != 0 or i == j
 *   omega_best   device or NULL: n_sub dense p x p matrices (element type per
 *                precision), subsample s's estimate of smallest epBIC
 *   best_index   host or NULL: n_sub penalty indices of those estimates (-1: none)
 *   workspace    device, accord_path_workspace_bytes(...) bytes, 256-byte
 *                aligned, or NULL to allocate (and free) one internally
 *   out          host or NULL: totals (iters, trials over all estimates; setup
 *                and solve time; launches)
 * Returns ACCORD_OK when every estimate converged, ACCORD_NOT_CONVERGED when
 * some reached max_iter, else the first error among the records (or the
 * call's own error: EINVAL, EDOMAIN for non-finite data, ENOMEM, ECUDA).
 * opts->trace, init_from_omega and sparse_update are ignored (the mixed modes
 * always use the sparse Delta update with its dense fallback). */
int accord_path(const float* X, int64_t n, int64_t p, const int32_t* rows, const int64_t* row_offsets,
                int64_t n_sub, const double* lambdas, int64_t n_lambda, const accord_opts* opts,
                accord_path_entry* entries, uint32_t* support, void* omega_best, int32_t* best_index,
                void* workspace, size_t ws_bytes, accord_stats* out);

/* Workspace bytes of accord_path (Sec 3.4) for these subsamples and n_lambda
 * penalties under opts (precision matters); 0 on invalid arguments (the checks
 * of accord_path) or when the host bookkeeping cannot be allocated.  It
 * depends on the subsamples only through their distinct-row counts. */
size_t accord_path_workspace_bytes(int64_t n, int64_t p, const int32_t* rows, const int64_t* row_offsets,
                                   int64_t n_sub, int64_t n_lambda, const accord_opts* opts);

#ifdef __cplusplus
}
#endif
#endif /* ACCORD_H_ */
