// accord_loss and accord_grad: the objective of Eq. 3.2 and the gradients of
// Sec 3.2 at a given Omega, through the same fused GEMM kernels as the fit.
// Scratch memory comes from one stream-ordered allocation per call.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "accord.h"
#include "internal.h"
#include "tc_gemm.h"

namespace accord {
namespace {

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct Bump {
  char* base = nullptr;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + used);
    used += (count * sizeof(T) + 1023) / 1024 * 1024;
    return p;
  }
};

struct Scratch {
  void* ptr = nullptr;
  cudaStream_t st = nullptr;
  ~Scratch() {
    if (ptr) cudaFreeAsync(ptr, st);
  }
};

#define EVAL_CK(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      set_last_error(__FILE__, __LINE__, cudaGetErrorString(e_));  \
      return kEcuda;                                               \
    }                                                              \
  } while (0)

int check_common(const float* X, int64_t n, int64_t p, const void* Omega, const accord_opts& o) {
  if (X == nullptr || Omega == nullptr || n < 1 || p < 1) return kEinval;
  if (o.precision != ACCORD_FP64 && o.precision != ACCORD_MIXED_BF16X3 && o.precision != ACCORD_MIXED_TF32X3)
    return kEinval;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return kEcuda;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return kEunsupported;
  return kOk;
}

// Sizes of one scratch allocation (two passes: measure, then carve).
struct EvalBuffers {
  double *x64 = nullptr, *xt64 = nullptr, *y64 = nullptr;
  int pt = kPlaneBf16;  // operand-plane type (mixed modes)
  void *om_hi = nullptr, *om_lo = nullptr, *x_hi = nullptr, *x_lo = nullptr;
  void *xt_hi = nullptr, *xt_lo = nullptr, *y_hi = nullptr, *y_lo = nullptr;
  double *part_y = nullptr, *part_om = nullptr, *res = nullptr;
  int* err = nullptr;
};

void carve(Bump& b, EvalBuffers& B, bool f64, bool need_y, int64_t n, int64_t p, int64_t tiles) {
  const int64_t ldk = round_up(p, 8), ldyk = round_up(n, 8);
  B.err = b.take<int>(16);
  B.res = b.take<double>(8);
  B.part_y = b.take<double>((size_t)tiles * kProxSlots);
  B.part_om = b.take<double>((size_t)p * kProxSlots);
  if (f64) {
    B.x64 = b.take<double>((size_t)n * ldk);
    B.xt64 = b.take<double>((size_t)p * ldyk);
    if (need_y) B.y64 = b.take<double>((size_t)p * ldyk);
  } else {
    const size_t pe = plane_bytes(B.pt);
    B.om_hi = b.take<char>((size_t)p * ldk * pe);
    B.om_lo = b.take<char>((size_t)p * ldk * pe);
    B.x_hi = b.take<char>((size_t)n * ldk * pe);
    B.x_lo = b.take<char>((size_t)n * ldk * pe);
    B.xt_hi = b.take<char>((size_t)p * ldyk * pe);
    B.xt_lo = b.take<char>((size_t)p * ldyk * pe);
    if (need_y) {
      B.y_hi = b.take<char>((size_t)p * ldyk * pe);
      B.y_lo = b.take<char>((size_t)p * ldyk * pe);
    }
  }
}

// Y = Omega X^T with reductions (and optionally stored as FP64 / planes).
int eval_y(const EvalBuffers& B, bool f64, const float* X, const void* Omega, int64_t n, int64_t p, bool store_y,
           cudaStream_t st) {
  const int64_t ldk = round_up(p, 8), ldyk = round_up(n, 8);
  if (f64) {
    EVAL_CK(launch_convert_x_f64(X, nullptr, n, p, B.x64, ldk, B.xt64, ldyk, B.err, st));
    GemmF64Params g{};
    g.A[0] = g.A[1] = static_cast<const double*>(Omega);
    g.lda = p;
    g.B = B.x64;
    g.ldb = ldk;
    g.M = p; g.N = n; g.K = p;
    g.out[0] = g.out[1] = store_y ? B.y64 : nullptr;
    g.ldout = ldyk;
    g.part = B.part_y;
    g.scale = 1.0;
    EVAL_CK(launch_gemm_f64(kModeY, g, st));
    return kOk;
  }
  EVAL_CK(launch_convert_x_planes(X, n, p, B.x_hi, B.x_lo, ldk, B.xt_hi, B.xt_lo, ldyk, B.err, B.pt, st));
  EVAL_CK(launch_split_planes(static_cast<const float*>(Omega), p, p, p, B.om_hi, B.om_lo, ldk, B.pt, st));
  TcParams t{};
  if (!encode_plane_map(&t.a_hi[0], B.om_hi, B.pt, p, p, ldk, 128) ||
      !encode_plane_map(&t.a_lo[0], B.om_lo, B.pt, p, p, ldk, 128) ||
      !encode_plane_map(&t.b_hi, B.x_hi, B.pt, n, p, ldk, tc_box_n()) ||
      !encode_plane_map(&t.b_lo, B.x_lo, B.pt, n, p, ldk, tc_box_n()))
  {
    set_last_error(__FILE__, __LINE__, "cuTensorMapEncodeTiled rejected an operand");
    return kEcuda;
  }
  t.a_hi[1] = t.a_hi[0];
  t.a_lo[1] = t.a_lo[0];
  t.err = B.err + 1;
  tc_shape(t, p, n, p, B.pt);
  t.out_hi[0] = t.out_hi[1] = store_y ? B.y_hi : nullptr;
  t.out_lo[0] = t.out_lo[1] = store_y ? B.y_lo : nullptr;
  t.ldplane = ldyk;
  t.part = B.part_y;
  t.scale = 1.f;
  EVAL_CK(launch_tc_gemm(kModeY, t, st));
  return kOk;
}

int finish_errors(const EvalBuffers& B, cudaStream_t st) {
  int h[2] = {0, 0};
  EVAL_CK(cudaMemcpyAsync(h, B.err, sizeof(h), cudaMemcpyDeviceToHost, st));
  EVAL_CK(cudaStreamSynchronize(st));
  if (h[0] != 0) return kEdomain;
  if (h[1] != 0) {
    char msg[96];
    std::snprintf(msg, sizeof(msg), "device error bits 0x%x (1: an mbarrier wait timed out)", h[1]);
    set_last_error(__FILE__, __LINE__, msg);
    return kEcuda;
  }
  return kOk;
}

// f and g of Eq. 3.2 / Eq. 3.4 into res[0], res[1] (device) from the Y
// partials of eval_y and the statistics of Omega.
int loss_into(const EvalBuffers& B, const void* Omega, bool f64, int64_t n, int64_t p, int64_t tiles,
              double lambda, double lam_d, double* res, cudaStream_t st) {
  int64_t nomp = 0;
  EVAL_CK(launch_omega_stats(Omega, f64, p, p, B.part_om, &nomp, st));
  EVAL_CK(launch_loss_finish(B.part_om, nomp, B.part_y, tiles, lambda, lam_d, 1.0 / (double)n, res, st));
  return kOk;
}

// G_out = Omega S (smooth = 0) or -diag(1/omega) + Omega S (smooth = 1) from
// the Y stored by eval_y: the second product (1/n) Y X.
int grad_into(const EvalBuffers& B, const void* Omega, bool f64, int64_t n, int64_t p, int smooth, void* G_out,
              cudaStream_t st) {
  const int64_t ldyk = round_up(n, 8);
  if (f64) {
    GemmF64Params g{};
    g.A[0] = g.A[1] = B.y64;
    g.lda = ldyk;
    g.B = B.xt64;
    g.ldb = ldyk;
    g.M = p; g.N = p; g.K = n;
    g.out[0] = g.out[1] = static_cast<double*>(G_out);
    g.ldout = p;
    g.aux[0] = g.aux[1] = static_cast<const double*>(Omega);
    g.ldaux = p;
    g.scale = 1.0 / (double)n;
    g.smooth = smooth ? 1 : 0;
    EVAL_CK(launch_gemm_f64(kModeGrad, g, st));
    return kOk;
  }
  TcParams t{};
  if (!encode_plane_map(&t.a_hi[0], B.y_hi, B.pt, p, n, ldyk, 128) ||
      !encode_plane_map(&t.a_lo[0], B.y_lo, B.pt, p, n, ldyk, 128) ||
      !encode_plane_map(&t.b_hi, B.xt_hi, B.pt, p, n, ldyk, tc_box_n()) ||
      !encode_plane_map(&t.b_lo, B.xt_lo, B.pt, p, n, ldyk, tc_box_n()))
    return kEcuda;
  t.a_hi[1] = t.a_hi[0];
  t.a_lo[1] = t.a_lo[0];
  t.err = B.err + 1;
  tc_shape(t, p, p, n, B.pt);
  t.out[0] = t.out[1] = static_cast<float*>(G_out);
  t.ldout = p;
  t.aux[0] = t.aux[1] = static_cast<const float*>(Omega);
  t.ldaux = p;
  t.scale = (float)(1.0 / (double)n);
  t.smooth = smooth ? 1 : 0;
  EVAL_CK(launch_tc_gemm(kModeGrad, t, st));
  return kOk;
}

}  // namespace

int eval_loss_grad_async(const float* X, int64_t n, int64_t p, const void* Omega, const accord_opts& o,
                         double lambda, double* res, int smooth, void* G_out, int* err) {
  const bool f64 = o.precision == ACCORD_FP64;
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const int64_t tiles = f64 ? gemm_f64_tiles(p, n) : tc_tiles(p, n);
  Bump meas;
  EvalBuffers B;
  B.pt = o.precision == ACCORD_MIXED_TF32X3 ? kPlaneTf32 : kPlaneBf16;
  carve(meas, B, f64, true, n, p, tiles);
  Scratch s;
  if (cudaMallocAsync(&s.ptr, meas.used, st) != cudaSuccess) return kEnomem;
  s.st = st;  // freed in stream order after the work queued below
  Bump b;
  b.base = static_cast<char*>(s.ptr);
  carve(b, B, f64, true, n, p, tiles);
  B.err = err;  // the caller's error words
  if (int e = eval_y(B, f64, X, Omega, n, p, true, st)) return e;
  if (int e = loss_into(B, Omega, f64, n, p, tiles, lambda, o.penalize_diag ? lambda : 0.0, res, st)) return e;
  return grad_into(B, Omega, f64, n, p, smooth, G_out, st);
}

}  // namespace accord

using namespace accord;

extern "C" {

int accord_loss(const float* X, int64_t n, int64_t p, const void* Omega, double lambda, const accord_opts* optp,
                double* f_out, double* g_out) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (int e = check_common(X, n, p, Omega, o)) return e;
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return kEinval;
  const bool f64 = o.precision == ACCORD_FP64;
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const int64_t tiles = f64 ? gemm_f64_tiles(p, n) : tc_tiles(p, n);
  Bump meas;
  EvalBuffers B;
  B.pt = o.precision == ACCORD_MIXED_TF32X3 ? kPlaneTf32 : kPlaneBf16;
  carve(meas, B, f64, false, n, p, tiles);
  Scratch s;
  if (cudaMallocAsync(&s.ptr, meas.used, st) != cudaSuccess) return kEnomem;
  s.st = st;
  Bump b;
  b.base = static_cast<char*>(s.ptr);
  carve(b, B, f64, false, n, p, tiles);
  EVAL_CK(cudaMemsetAsync(B.err, 0, 64, st));
  if (int e = eval_y(B, f64, X, Omega, n, p, false, st)) return e;
  if (int e = loss_into(B, Omega, f64, n, p, tiles, lambda, o.penalize_diag ? lambda : 0.0, B.res, st)) return e;
  double h[2] = {0, 0};
  EVAL_CK(cudaMemcpyAsync(h, B.res, sizeof(h), cudaMemcpyDeviceToHost, st));
  if (int e = finish_errors(B, st)) return e;
  if (f_out) *f_out = h[0];
  if (g_out) *g_out = h[1];
  return kOk;
}

int accord_grad(const float* X, int64_t n, int64_t p, const void* Omega, int smooth, const accord_opts* optp,
                void* G_out) {
  clear_last_error();
  accord_opts o;
  accord_default_opts(&o);
  if (optp) o = *optp;
  if (int e = check_common(X, n, p, Omega, o)) return e;
  if (G_out == nullptr || G_out == Omega) return kEinval;
  const bool f64 = o.precision == ACCORD_FP64;
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const int64_t tiles = f64 ? gemm_f64_tiles(p, n) : tc_tiles(p, n);
  const int64_t ldyk = round_up(n, 8);
  Bump meas;
  EvalBuffers B;
  B.pt = o.precision == ACCORD_MIXED_TF32X3 ? kPlaneTf32 : kPlaneBf16;
  carve(meas, B, f64, true, n, p, tiles);
  Scratch s;
  if (cudaMallocAsync(&s.ptr, meas.used, st) != cudaSuccess) return kEnomem;
  s.st = st;
  Bump b;
  b.base = static_cast<char*>(s.ptr);
  carve(b, B, f64, true, n, p, tiles);
  EVAL_CK(cudaMemsetAsync(B.err, 0, 64, st));
  if (int e = eval_y(B, f64, X, Omega, n, p, true, st)) return e;
  if (int e = grad_into(B, Omega, f64, n, p, smooth, G_out, st)) return e;
  return finish_errors(B, st);
}

}  // extern "C"
