// Internal declarations shared by the CUDA translation units of libaccord.
// Elementwise update of Eq. 3.5, KKT residual entries of Eq. 3.3, the device
// control block of the Algorithm 1 line search and the per-tile partial-sum
// layouts.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace accord {

// ---------------------------------------------------------------- status ---
enum : int {
  kOk = 0, kNotConverged = 1, kEinval = -1, kEdomain = -2, kEnonfinite = -3,
  kEbacktrack = -4, kEnomem = -5, kEcuda = -6, kEunsupported = -7,
};

// Device error bits (ctrl->dev_error): a bounded wait gave up, or a kernel
// found an impossible configuration and skipped its work.
enum : int { kErrWaitTimeout = 1, kErrBadConfig = 2 };

// ------------------------------------------------ partial-sum slot layout ---
// Prox epilogue (GEMM2), one row of kProxSlots doubles per output tile.
enum : int {
  kPDelta2 = 0,   // ||Omega+ - Omega||_F^2
  kPLogDiag = 1,  // sum log omega+_ii
  kPDiagSum = 2,  // sum omega+_ii
  kPL1Off = 3,    // sum_{i != j} |omega+_ij|
  kPNnz = 4,      // off-diagonal nonzeros of Omega+
  kPKkt = 5,      // max KKT residual entry of Omega (input iterate)  [max]
  kPBad = 6,      // non-finite values seen / non-positive diagonal
  kProxSlots = 8,
};
// Y epilogue (GEMM1), one row of kYSlots doubles per output tile.
enum : int { kYDiff2 = 0, kYNorm2 = 1, kYBad = 2, kYSlots = 4 };

// ----------------------------------------------------- control block ------
// Lives in device memory; every per-trial kernel reads it first and returns
// immediately once `done` is set, so a fixed launch sequence can run past
// convergence harmlessly.
struct Ctrl {
  int32_t t;          // accepted steps so far (index of the current iterate)
  int32_t k;          // trial index within the current outer step
  int32_t trials;     // total prox evaluations
  int32_t done;       // 1 once the fit has finished
  int32_t status;     // final status when done
  int32_t cur;        // which of the two iterate buffers holds Omega^t
  int32_t dev_error;  // kErr* bits
  int32_t power_done; // power iteration converged
  double tau;         // step of the pending trial
  double tau_prev;    // last accepted step
  double tau0;        // restart step (opts tau0, or 1/L when that is <= 0)
  double L, inv_L;
  // current iterate Omega^t
  double g, logdiag, diagsum, l1off, f, nnz, kkt;
  // pending trial Omega+ (filled after the prox kernel)
  double t_d2, t_logdiag, t_diagsum, t_l1off, t_nnz;
  // pending trial Y+ (filled after GEMM1)
  double t_dy2, t_y2;
  // power iteration state
  double pw_est, pw_prev;
  int32_t pw_iter;
  int32_t dense;      // a Delta bucket overflowed: this trial takes the dense Y GEMM
  // penalty weights and 1/n of this problem (a batch holds one Ctrl per problem)
  double lam, lam_d, inv_n;
  int32_t kdim;       // rows of this problem's data matrix
  int32_t lam_idx;    // lambda path: index of the current penalty
  int32_t finished;   // lambda path: every penalty of the chain is done
  int32_t emit;       // lambda path: 1 = an estimate was completed in this trial, 2 = it is the best so far
  int32_t emit_lam;   // lambda path: penalty index of that estimate
  int32_t iters_tot;  // lambda path: accepted steps over the whole chain
  int32_t trials_tot; // lambda path: prox evaluations over the whole chain
  int32_t ymode;      // batch: 1 = the prox epilogue writes dense Delta planes (Delta too dense for
                      // the buckets), 0 = it fills the sparse buckets
  // mixed modes: Y = Omega X^T is carried forward by Y+ = Y + Delta X^T in
  // FP32, which accumulates rounding; it is formed afresh from Omega^t every
  // SolveParams::y_refresh accepted steps and before a KKT residual under
  // the tolerance may end the fit
  int32_t refresh;        // 1: Y of Omega^t is formed afresh before the next trial
  int32_t since_refresh;  // accepted steps since Y was last formed from Omega
  int32_t n_refresh;      // refreshes so far
  int32_t cut_trials;     // trials cut short because their KKT test asked for a refresh
  double y_drift;         // largest ||Y - Omega X^T||_F / ||Omega X^T||_F found by a refresh
  double kkt_prev;        // KKT residual of the iterate before Omega^t (INFINITY if none)
  // mixed modes: 1 while the prox GEMM forms G with the one product hi x hi
  // (SolveParams::coarse_kkt); the first KKT residual under that threshold
  // switches to the three split products for the rest of the fit
  int32_t coarse;
  int32_t n_coarse;       // prox launches that ran with the one product
  int32_t predicted;      // the pending or last refresh was taken ahead of a predicted passing KKT test
  int32_t no_predict;     // such a prediction missed: until the fit (or penalty) ends, refresh only when due
};

// One estimate of a lambda path (same layout as accord_path_entry).
struct PathRec {
  int32_t status, iters, trials, y_refreshes;
  double lambda, f, g, kkt, logdet_d, epbic, tau_last;
  int64_t nnz_offdiag;
  double y_drift;
};

struct SolveParams {
  double lam, lam_d, tau0, beta, kkt_tol;
  double inv_n;
  int32_t max_iter, max_backtracks, tau_warm, fixed_step;
  int64_t trace_cap;
  int32_t y_refresh;  // mixed modes: accepted steps between refreshes of Y (0: none)
  int32_t pad0;
  double coarse_kkt;  // mixed modes: one-product gradients while the KKT residual is above this (0: never)
};

constexpr int kTraceFields = 8;

// --------------------------------------------------------- Eq. 3.5 math ---
template <class T>
__device__ __forceinline__ T soft_threshold(T x, T a) {
  // S_a(x) = (|x| - a)_+ sign(x); |x| == a and x == 0 both give exactly 0.
  T m = fabs(x) - a;
  return m > T(0) ? copysign(m, x) : T(0);
}

template <class T>
__device__ __forceinline__ T diag_prox(T y, T tau, T lam_d) {
  // positive root of w^2 - b w - tau = 0, b = y - tau lambda_d; the b < 0
  // branch uses 2 tau / (sqrt(b^2 + 4 tau) - b), the same value without
  // cancellation.
  T b = y - tau * lam_d;
  T root = sqrt(b * b + T(4) * tau);
  return b >= T(0) ? T(0.5) * (b + root) : (T(2) * tau) / (root - b);
}

// One entry of the minimum-norm subgradient of Eq. 3.3 (absolute value).
template <class T>
__device__ __forceinline__ T kkt_entry(T omega, T G, bool diag, T lam, T lam_d) {
  if (diag) {
    if (!(omega > T(0))) return T(INFINITY);
    return fabs(G - T(1) / omega + lam_d);
  }
  if (omega != T(0)) return fabs(G + copysign(lam, omega));
  T m = fabs(G) - lam;
  return m > T(0) ? m : T(0);
}

// ----------------------------------------------------- warp reductions ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// BF16 hi/lo split: x ~= hi + lo with hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// ------------------------------------------------------- operand planes ---
// The mixed modes carry each FP32 tensor-core operand x as two planes with
// x ~= hi + lo:
//   kPlaneBf16  hi = bf16(x), lo = bf16(x - hi); 2 bytes an element, hi + lo
//               within 2^-18 |x| of x (8 significant bits each);
//   kPlaneTf32  hi = tf32(x), lo = tf32(x - hi), each in an FP32 word whose
//               13 low mantissa bits are zero; 4 bytes an element, within
//               2^-24 |x| (11 significant bits each).
// x - hi is exact in FP32 in both cases (hi is x rounded to fewer bits).
enum : int { kPlaneBf16 = 0, kPlaneTf32 = 1 };
__host__ __device__ constexpr size_t plane_bytes(int pt) { return pt == kPlaneTf32 ? 4 : 2; }

// x rounded to TF32 (11 significant bits, nearest, ties away from zero),
// returned as an FP32 value with the low 13 mantissa bits cleared.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r & 0xFFFFE000u);
}
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - hi);
}

template <int PT> struct Plane;
template <> struct Plane<kPlaneBf16> {
  using E = __nv_bfloat16;
  __device__ static __forceinline__ void split(float x, E& hi, E& lo) { split_bf16(x, hi, lo); }
};
template <> struct Plane<kPlaneTf32> {
  using E = float;
  __device__ static __forceinline__ void split(float x, E& hi, E& lo) { split_tf32(x, hi, lo); }
};

// Writes the split of x to element idx of the planes hi / lo (type pt).
__device__ __forceinline__ void store_split(void* hi, void* lo, int64_t idx, float x, int pt) {
  if (pt == kPlaneTf32) {
    float h, l;
    split_tf32(x, h, l);
    static_cast<float*>(hi)[idx] = h;
    static_cast<float*>(lo)[idx] = l;
  } else {
    __nv_bfloat16 h, l;
    split_bf16(x, h, l);
    static_cast<__nv_bfloat16*>(hi)[idx] = h;
    static_cast<__nv_bfloat16*>(lo)[idx] = l;
  }
}

}  // namespace accord
