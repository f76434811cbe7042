// Persistent tcgen05 GEMM C = A * B^T on split-BF16 operands, with the fused
// epilogues of ACCORD-FBS (mixed precision mode).
//
// Each FP32 operand x is carried as two BF16 planes, hi = bf16(x) and
// lo = bf16(x - hi); every 128 x BN x 16 slice issues three MMAs into one FP32
// TMEM accumulator, A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term is below
// FP32 resolution of the sum), which recovers ~16 significant bits per operand.
//
// Warp roles (one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer: A_hi, A_lo, B_hi, B_lo tiles into a STAGES-deep
//               shared-memory ring (128-byte swizzle), one mbarrier per stage.
//   warp 1      TMEM allocator and single-thread MMA issuer (tcgen05.mma).
//   warps 2..9  epilogue: tcgen05.ld from a double-buffered TMEM accumulator,
//               so the epilogue of tile i overlaps the main loop of tile i+1.
//
// Epilogues: Y+ = Y + Delta X^T with ||Delta X^T||^2 and ||Y+||^2 (Algorithm
// 1's test), G = Y X / n fused with the prox of Eq. 3.5, the Delta planes and
// the trial / KKT reductions, the gradient of Sec 3.2, and X X^T / n.
#include <cstdio>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace accord {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;               // BF16 elements per 128-byte swizzle row
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = 64 + kEpiThreads;
constexpr int kBN = 256;
constexpr int kStages = 2;
constexpr uint32_t kABytes = BM * BK * 2;
constexpr uint32_t kBBytes = kBN * BK * 2;
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr uint32_t kTmemCols = 2 * kBN;  // two accumulators
constexpr uint32_t kEpiBufBytes = kEpiWarps * 32 * 32 * 4;  // one 32x32 FP32 block per epilogue warp
constexpr size_t kSmemBytes = 1024 + (size_t)kStages * kStageBytes + kEpiBufBytes + 1024;

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group_m, int& mb, int& nb) {
  const int per_group = group_m * tiles_n;
  const int g = t / per_group;
  const int first_m = g * group_m;
  const int gm = min(tiles_m - first_m, group_m);
  const int r = t - g * per_group;
  mb = first_m + r % gm;
  nb = r / gm;
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory"); }

struct EpiArgs {
  float tau, lam, lam_d, scale;
  float* out;
  __nv_bfloat16* out_hi;
  __nv_bfloat16* out_lo;
  const float* aux;
  int64_t M, N;
};

struct Sums {  // per-thread tile partials (FP64 across chunks, FP32 within)
  double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0, bad = 0.0;
  float kkt = 0.f;
};

// Transpose a 32x32 accumulator block: on entry thread `lane` holds TMEM row
// `lane` (32 consecutive columns); on exit it holds column `lane` of the 32
// rows.  16-byte groups are XOR-swizzled by row, so both the row writes and
// the column reads are free of bank conflicts.
__device__ __forceinline__ void transpose32(float* buf, const uint32_t (&rr)[32], int lane, float (&v)[32]) {
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const float4 x = make_float4(__uint_as_float(rr[4 * g]), __uint_as_float(rr[4 * g + 1]),
                                 __uint_as_float(rr[4 * g + 2]), __uint_as_float(rr[4 * g + 3]));
    *reinterpret_cast<float4*>(buf + lane * 32 + ((g ^ (lane & 7)) << 2)) = x;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = buf[r * 32 + ((((lane >> 2) ^ (r & 7))) << 2) + (lane & 3)];
  __syncwarp();
}

// pre[r] = src[row_base + r][colt] (zero outside the matrix).
__device__ __forceinline__ void load_column(const float* __restrict__ src, int64_t ld, int64_t row_base,
                                            int64_t colt, bool full, const EpiArgs& ea, float (&pre)[32]) {
  const float* p = src + row_base * ld + colt;
  if (full) {
#pragma unroll
    for (int r = 0; r < 32; ++r) pre[r] = __ldg(p + r * ld);
  } else {
    const bool cok = colt < ea.N;
#pragma unroll
    for (int r = 0; r < 32; ++r) pre[r] = (cok && row_base + r < ea.M) ? __ldg(p + r * ld) : 0.f;
  }
}

__device__ __forceinline__ void store_split(__nv_bfloat16* hi, __nv_bfloat16* lo, float x) {
  __nv_bfloat16 h, l;
  split_bf16(x, h, l);
  *hi = h;
  *lo = l;
}

// Y+ = Y + Delta X^T (aux = Y) or Y = Omega X^T (aux = null) for column colt.
template <bool CHECK>
__device__ __forceinline__ void y_chunk(const EpiArgs& ea, const TcParams& prm, int64_t row_base, int64_t colt,
                                        const float (&v)[32], const float (&pre)[32], Sums& sm) {
  float sd = 0.f, sn = 0.f, chk = 0.f;
  const bool cok = !CHECK || colt < ea.N;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int64_t row = row_base + r;
    if (CHECK && !(cok && row < ea.M)) continue;
    const float dv = v[r] * ea.scale;
    const float yn = (ea.aux ? pre[r] : 0.f) + dv;
    sd = fmaf(dv, dv, sd);
    sn = fmaf(yn, yn, sn);
    chk = fmaf(yn, 0.f, chk);
    if (ea.out) ea.out[row * prm.ldout + colt] = yn;
    if (ea.out_hi) store_split(ea.out_hi + row * prm.ldplane + colt, ea.out_lo + row * prm.ldplane + colt, yn);
  }
  sm.r0 += (double)sd;
  sm.r1 += (double)sn;
  if (chk != 0.f) sm.bad += 1.0;
}

// G = acc / n, Eq. 3.5 on A = Omega - tau G, Omega+ and Delta planes, and the
// trial / KKT partial sums for column colt.  CHECK handles the matrix edge
// and the diagonal (row == colt).
template <bool CHECK>
__device__ __forceinline__ void prox_chunk(const EpiArgs& ea, const TcParams& prm, int64_t row_base,
                                           int64_t colt, const float (&v)[32], const float (&pre)[32], Sums& sm) {
  float sd = 0.f, sl1 = 0.f, kk = 0.f, chk = 0.f;
  int nnz = 0;
  const float tau = ea.tau, tlam = ea.tau * ea.lam;
  const bool cok = !CHECK || colt < ea.N;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int64_t row = row_base + r;
    if (CHECK && !(cok && row < ea.M)) continue;
    const float g = v[r] * ea.scale;
    const float om = pre[r];
    const float a = fmaf(-tau, g, om);
    float w;
    if (CHECK && row == colt) {
      w = diag_prox(a, tau, ea.lam_d);
      sm.r2 += log((double)w);
      sm.r3 += (double)w;
      kk = fmaxf(kk, kkt_entry(om, g, true, ea.lam, ea.lam_d));
    } else {
      w = soft_threshold(a, tlam);
      sl1 += fabsf(w);
      nnz += (w != 0.f) ? 1 : 0;
      kk = fmaxf(kk, kkt_entry(om, g, false, ea.lam, ea.lam_d));
    }
    chk = fmaf(g, 0.f, chk);
    const float d = w - om;
    sd = fmaf(d, d, sd);
    ea.out[row * prm.ldout + colt] = w;
    store_split(ea.out_hi + row * prm.ldplane + colt, ea.out_lo + row * prm.ldplane + colt, d);
  }
  sm.r0 += (double)sd;
  sm.r1 += (double)sl1;
  sm.r4 += (double)nnz;
  sm.kkt = fmaxf(sm.kkt, kk);
  if (chk != 0.f || !(sd == sd)) sm.bad += 1.0;
}

__device__ __forceinline__ void grad_chunk(const EpiArgs& ea, const TcParams& prm, int64_t row_base, int64_t colt,
                                           bool check, const float (&v)[32]) {
  const bool cok = colt < ea.N;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int64_t row = row_base + r;
    if (check && !(cok && row < ea.M)) continue;
    float g = v[r] * ea.scale;
    if (prm.smooth && check && row == colt) g -= 1.f / ea.aux[row * prm.ldaux + row];
    ea.out[row * prm.ldout + colt] = g;
  }
}

__device__ __forceinline__ void gram_chunk(const TcParams& prm, int64_t row_base, int64_t colt, const float (&v)[32],
                                           const EpiArgs& ea) {
  const bool cok = colt < ea.N;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int64_t row = row_base + r;
    if (!(cok && row < ea.M)) continue;
    prm.out64[row * prm.ldout64 + colt] = (double)(v[r] * ea.scale);
  }
}

// 320 threads = 10 warps; two SM sub-partitions hold 3 of them, so at most
// 16384 / (3 * 32) = 170 registers a thread (168 after allocation rounding).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const __grid_constant__ TcParams prm) {
  const Ctrl* ctrl = prm.ctrl;
  if (ctrl != nullptr && ctrl->done) return;
  const int cur = ctrl ? ctrl->cur : 0;
  const int nxt = cur ^ 1;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* epi_buf = reinterpret_cast<float*>(smem + kStages * kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + kEpiBufBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* stop_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);
  double* red = reinterpret_cast<double*>(smem + kStages * kStageBytes + kEpiBufBytes + 128);  // [kEpiWarps][8]

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], kEpiThreads);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    *stop_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int asel = prm.a_nxt ? nxt : cur;
  const CUtensorMap* mA_hi = &prm.a_hi[asel];
  const CUtensorMap* mA_lo = &prm.a_lo[asel];
  const CUtensorMap* mB_hi = &prm.b_hi;
  const CUtensorMap* mB_lo = &prm.b_lo;
  const uint32_t smem_base = ptx::smem_u32(smem);

  if (warp == 0) {
    // ------------------------------------------------------ TMA producer --
    if (lane == 0) {
      ptx::tma_prefetch_desc(mA_hi);
      ptx::tma_prefetch_desc(mA_lo);
      ptx::tma_prefetch_desc(mB_hi);
      ptx::tma_prefetch_desc(mB_lo);
      uint32_t s = 0, ph = 0;
      uint32_t fill_ph[kStages];
      bool filled[kStages];
      for (int q = 0; q < kStages; ++q) { filled[q] = false; fill_ph[q] = 0; }
      bool ok = true;
      for (int t = blockIdx.x; t < prm.ntiles && ok; t += gridDim.x) {
        int mb, nb;
        tile_coords(t, prm.tiles_m, prm.tiles_n, prm.group_m, mb, nb);
        for (int kb = 0; kb < prm.num_kb; ++kb) {
          if (!ptx::mbar_wait(&empty[s], ph ^ 1u, abort_flag)) { ok = false; break; }
          ptx::mbar_arrive_expect_tx(&full[s], kStageBytes);
          const uint32_t st = smem_base + s * kStageBytes;
          ptx::tma_load_2d(st, mA_hi, &full[s], kb * BK, mb * BM);
          ptx::tma_load_2d(st + kABytes, mA_lo, &full[s], kb * BK, mb * BM);
          ptx::tma_load_2d(st + 2 * kABytes, mB_hi, &full[s], kb * BK, nb * kBN);
          ptx::tma_load_2d(st + 2 * kABytes + kBBytes, mB_lo, &full[s], kb * BK, nb * kBN);
          filled[s] = true;
          fill_ph[s] = ph;
          if (++s == kStages) { s = 0; ph ^= 1u; }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.err, kErrWaitTimeout);
        // let the copies already issued land before the CTA can exit
        for (int q = 0; q < kStages; ++q)
          if (filled[q]) (void)ptx::mbar_wait(&full[q], fill_ph[q], nullptr);
      }
    }
  } else if (warp == 1) {
    // -------------------------------------------------------- MMA issuer --
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, kBN);
      uint32_t s = 0, ph = 0;
      bool ok = true;
      int i = 0;
      for (int t = blockIdx.x; t < prm.ntiles && ok; t += gridDim.x, ++i) {
        const uint32_t acc = i & 1, aph = (i >> 1) & 1;
        if (!ptx::mbar_wait(&tempty[acc], aph ^ 1u, abort_flag)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t d = tmem_base + acc * kBN;
        for (int kb = 0; kb < prm.num_kb; ++kb) {
          if (!ptx::mbar_wait(&full[s], ph, abort_flag)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t st = smem_base + s * kStageBytes;
          const uint64_t a_hi = ptx::sdesc_k128(st);
          const uint64_t a_lo = ptx::sdesc_k128(st + kABytes);
          const uint64_t b_hi = ptx::sdesc_k128(st + 2 * kABytes);
          const uint64_t b_lo = ptx::sdesc_k128(st + 2 * kABytes + kBBytes);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t off = (uint64_t)(kk * 2);  // 32 bytes >> 4
            ptx::mma_f16(d, a_lo + off, b_hi + off, idesc, (kb | kk) != 0);
            ptx::mma_f16(d, a_hi + off, b_lo + off, idesc, 1u);
            ptx::mma_f16(d, a_hi + off, b_hi + off, idesc, 1u);
          }
          ptx::mma_commit(&empty[s]);
          if (++s == kStages) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;
        ptx::mma_commit(&tfull[acc]);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.err, kErrWaitTimeout);
        ptx::mma_commit(drain);
        (void)ptx::mbar_wait(drain, 0, nullptr);
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue --
    // Warp e reads TMEM lane quarter q (rows row_base .. +31 of the tile) and
    // column half h.  Each 32x32 accumulator block is transposed through a
    // per-warp shared buffer so that thread `lane` owns one column: every
    // global load / store below is then one full 128-byte line per warp.
    const int e = warp - 2;
    const int q = warp & 3;
    const int h = e >> 2;
    constexpr int kColsPerWarp = kBN / (kEpiWarps / 4);
    float* tbuf = epi_buf + e * 1024;
    const double tau_d = ctrl ? ctrl->tau : 0.0;
    EpiArgs ea;
    ea.tau = (float)tau_d;
    ea.lam = prm.lam;
    ea.lam_d = prm.lam_d;
    ea.scale = prm.scale;
    ea.out = prm.out[nxt];
    ea.out_hi = prm.out_hi[nxt];
    ea.out_lo = prm.out_lo[nxt];
    ea.aux = prm.aux[cur];
    ea.M = prm.M;
    ea.N = prm.N;
    constexpr bool kNeedAux = (MODE == kModeProx || MODE == kModeY);
    int i = 0;
    for (int t = blockIdx.x; t < prm.ntiles; t += gridDim.x, ++i) {
      int mb, nb;
      tile_coords(t, prm.tiles_m, prm.tiles_n, prm.group_m, mb, nb);
      const uint32_t acc = i & 1, aph = (i >> 1) & 1;
      const int64_t row_base = (int64_t)mb * BM + 32 * q;
      const int64_t col_base = (int64_t)nb * kBN + h * kColsPerWarp;
      const bool rows_full = row_base + 32 <= prm.M;
      Sums sm;
      float pre[32];
      // the first chunk's operand does not depend on the MMA: fetch it before waiting
      if (kNeedAux && ea.aux != nullptr)
        load_column(ea.aux, prm.ldaux, row_base, col_base + lane, rows_full && col_base + 32 <= prm.N, ea, pre);
      const bool ok = ptx::mbar_wait(&tfull[acc], aph, abort_flag);
      if (!ok) {
        *abort_flag = 1;
        if (lane == 0) atomicOr(prm.err, kErrWaitTimeout);
      }
      ptx::tc_fence_after();
      if (ok) {
#pragma unroll 1
        for (int c = 0; c < kColsPerWarp; c += 32) {
          const int64_t col0 = col_base + c;
          const int64_t colt = col0 + lane;
          const bool full = rows_full && col0 + 32 <= prm.N;
          if (kNeedAux && ea.aux != nullptr && c > 0)
            load_column(ea.aux, prm.ldaux, row_base, colt, full, ea, pre);
          uint32_t rr[32];
          ptx::tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(32 * q) << 16) + acc * kBN + h * kColsPerWarp + c, rr);
          ptx::tmem_ld_wait();
          float v[32];
          transpose32(tbuf, rr, lane, v);
          if (row_base >= prm.M || col0 >= prm.N) continue;  // warp-uniform
          const bool diag = (row_base == col0);
          if (MODE == kModeY) {
            if (full) y_chunk<false>(ea, prm, row_base, colt, v, pre, sm);
            else y_chunk<true>(ea, prm, row_base, colt, v, pre, sm);
          } else if (MODE == kModeProx) {
            if (full && !diag) prox_chunk<false>(ea, prm, row_base, colt, v, pre, sm);
            else prox_chunk<true>(ea, prm, row_base, colt, v, pre, sm);
          } else if (MODE == kModeGrad) {
            grad_chunk(ea, prm, row_base, colt, diag || !full, v);
          } else {
            gram_chunk(prm, row_base, colt, v, ea);
          }
        }
      }
      const double r0 = sm.r0, r1 = sm.r1, r2 = sm.r2, r3 = sm.r3, r4 = sm.r4, rbad = sm.bad;
      const float rkkt = sm.kkt;
      ptx::tc_fence_before();
      ptx::mbar_arrive(&tempty[acc]);
      // Partial sums of this tile, folded in a fixed order.  Both named
      // barriers run on every tile so that all epilogue warps leave the loop
      // together (the stop decision is taken by one thread between them).
      constexpr int W = (MODE == kModeY) ? kYSlots : kProxSlots;
      if (MODE == kModeY || MODE == kModeProx) {
        double vals[8];
        if (MODE == kModeY) {
          vals[kYDiff2] = r0; vals[kYNorm2] = r1; vals[kYBad] = rbad; vals[3] = 0.0;
        } else {
          vals[kPDelta2] = r0; vals[kPLogDiag] = r2; vals[kPDiagSum] = r3; vals[kPL1Off] = r1;
          vals[kPNnz] = r4; vals[kPKkt] = (double)rkkt; vals[kPBad] = rbad; vals[7] = 0.0;
        }
#pragma unroll
        for (int s = 0; s < W; ++s) {
          const double x = (MODE == kModeProx && s == kPKkt) ? warp_max(vals[s]) : warp_sum(vals[s]);
          if (lane == 0) red[e * 8 + s] = x;
        }
      }
      epi_bar();
      if (e == 0) {
        if ((MODE == kModeY || MODE == kModeProx) && prm.part != nullptr && lane < W) {
          double x = red[lane];
          for (int w = 1; w < kEpiWarps; ++w)
            x = (MODE == kModeProx && lane == kPKkt) ? fmax(x, red[w * 8 + lane]) : x + red[w * 8 + lane];
          const int bad_slot = (MODE == kModeProx) ? (int)kPBad : (int)kYBad;
          if (*abort_flag && lane == bad_slot) x += 1.0;
          prm.part[(int64_t)t * W + lane] = x;
        }
        if (lane == 0) *stop_flag = *abort_flag;
      }
      epi_bar();
      if (*stop_flag) break;
    }
  }

  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, kTmemCols);
  }
}

template <int MODE>
cudaError_t launch_mode(const TcParams& prm, cudaStream_t st) {
  static int configured = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured != dev) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    configured = dev;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(prm.ntiles, sms > 0 ? sms : 1);
  tc_gemm_kernel<MODE><<<grid, kThreads, kSmemBytes, st>>>(prm);
  return cudaGetLastError();
}

}  // namespace

int tc_box_n() { return kBN; }

int64_t tc_tiles(int64_t M, int64_t N) { return ((M + BM - 1) / BM) * ((N + kBN - 1) / kBN); }

void tc_shape(TcParams& prm, int64_t M, int64_t N, int64_t K) {
  prm.M = M;
  prm.N = N;
  prm.K = K;
  prm.num_kb = (int32_t)((K + BK - 1) / BK);
  prm.tiles_m = (int32_t)((M + BM - 1) / BM);
  prm.tiles_n = (int32_t)((N + kBN - 1) / kBN);
  prm.ntiles = prm.tiles_m * prm.tiles_n;
  prm.group_m = 8;
  prm.bn = kBN;
}

cudaError_t launch_tc_gemm(int mode, const TcParams& prm, cudaStream_t st) {
  if (prm.ntiles <= 0) return cudaSuccess;
  switch (mode) {
    case kModeY: return launch_mode<kModeY>(prm, st);
    case kModeProx: return launch_mode<kModeProx>(prm, st);
    case kModeGrad: return launch_mode<kModeGrad>(prm, st);
    case kModeGram: return launch_mode<kModeGram>(prm, st);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------ tensor maps --
bool encode_plane_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t cols, int64_t ld,
                      int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (encode == nullptr) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if (((uintptr_t)base & 15u) != 0 || (ld * 2) % 16 != 0 || rows < 1 || cols < 1) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides,
                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace accord
