// Persistent tcgen05 GEMM C = A * B^T on split operands, with the fused
// epilogues of ACCORD-FBS (mixed precision modes).
//
// Each FP32 operand x is carried as two planes x ~= hi + lo, BF16 (kind::f16
// MMAs; hi + lo within 2^-18 of x) or TF32 (kind::tf32 MMAs; within 2^-24).
// Every 32-byte K slice of a 128 x BN tile issues three MMAs into one FP32
// TMEM accumulator, A_hi B_hi + A_hi B_lo + A_lo B_hi; the lo*lo term is
// below the resolution of the split.  A plane row of a pipeline stage is 64
// bytes (32 BF16 or 16 TF32 of K), so the shared-memory layout, descriptors
// and stage sizes are the same for both types.
//
// CTA pairs (tcgen05 cta_group::2): two CTAs of a 2-CTA cluster, one per SM,
// compute one 256 x 256 output tile with M = 256 MMAs.  Each CTA loads its own
// 128 rows of A and its half (128 rows) of the B tile into its own shared
// memory; the MMA reads both CTAs' halves, so no operand byte is fetched
// twice for a pair, and each CTA's 128 accumulator rows land in its own TMEM.
//
// Warp roles (one CTA per SM, persistent over pair tiles):
//   warp 0      TMA producer of each CTA: its A_hi, A_lo, B_hi, B_lo halves
//               (64 bytes of K a row) into a 6-deep shared-memory ring (64-byte
//               swizzle).  The copies of both CTAs complete on the even
//               (leader) CTA's stage barrier.
//   warp 1      TMEM allocator of each CTA; in the leader, the single-thread
//               MMA issuer (tcgen05.mma.cta_group::2), whose commits release
//               each CTA's stage and signal each CTA's accumulator barrier.
//   warps 2..9  epilogue of each CTA: tcgen05.ld from a double-buffered TMEM
//               accumulator, so the epilogue of tile i overlaps the main loop
//               of tile i+1; its release goes to the leader.
//
// Epilogues: Y+ = Y + Delta X^T with ||Delta X^T||^2 and ||Y+||^2 (Algorithm
// 1's test), G = Y X / n fused with the prox of Eq. 3.5, the Delta planes and
// the trial / KKT reductions, the gradient of Sec 3.2, and X X^T / n.
#include <atomic>
#include <cstdio>
#include <mutex>

#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace accord {
namespace {

constexpr int BM = 128;           // accumulator rows of one CTA (one TMEM lane each)
constexpr int kRowBytes = 64;        // K bytes of a plane row per stage (one 64-byte swizzle row)
template <int PT>
constexpr int kBK = kRowBytes / (int)plane_bytes(PT);  // K elements per stage: 32 BF16 or 16 TF32
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = 64 + kEpiThreads;
constexpr int kBN = 256;          // output columns of a tile (MMA N)
constexpr int kBHalf = kBN / 2;   // B rows each CTA of the pair holds
constexpr int kStages = 4;
constexpr uint32_t kABytes = BM * kRowBytes;
constexpr uint32_t kBBytes = kBHalf * kRowBytes;
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;  // one CTA's share of a stage
constexpr uint32_t kTmemCols = 2 * kBN;  // two accumulators
// two 32x32 FP32 blocks per epilogue warp (prox mode stages the iterate two
// chunks ahead; the other modes use the first as their transpose buffer)
constexpr uint32_t kEpiBufBytes = kEpiWarps * 2 * 32 * 32 * 4;
// Prox mode: occupancy words of two tiles per epilogue warp (the current one
// and the next): the current iterate's words of the warp's four chunks, 32
// words (rows) each.
constexpr uint32_t kWordSlotWords = 4 * 32;
constexpr uint32_t kWordBytes = kEpiWarps * 2 * kWordSlotWords * 4;
constexpr size_t kTailBytes = 2048;
constexpr size_t kSmemBytes = 1024 + (size_t)kStages * kStageBytes + kEpiBufBytes + kWordBytes + kTailBytes;
// Tail after the epilogue buffers: 2 kStages + 5 mbarriers, the TMEM slot, two
// flags and two tile counters, then the epilogue's FP64 partials
// [2][kEpiWarps][8] (by tile parity) from kRedOffset.
constexpr size_t kRedOffset = 256;
static_assert((2 * kStages + 5) * 8 + 20 <= kRedOffset, "barriers overlap the epilogue partials");
static_assert(kRedOffset + 2 * kEpiWarps * 8 * 8 <= kTailBytes, "epilogue partials overflow the shared-memory tail");
static_assert(kSmemBytes <= 232448, "more dynamic shared memory than one CTA may use");

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group_m, int& mb, int& nb) {
  const int per_group = group_m * tiles_n;
  const int g = t / per_group;
  const int first_m = g * group_m;
  const int gm = min(tiles_m - first_m, group_m);
  const int r = t - g * per_group;
  mb = first_m + r % gm;
  nb = r / gm;
}

// Pair tile T (256 rows, scheduled per pair) -> this CTA's 128-row M block
// and the N block.
__device__ __forceinline__ void pair_tile(int T, const TcParams& prm, int rank, int& mb, int& nb) {
  int mp;
  tile_coords(T, prm.tiles_mp, prm.tiles_n, prm.group_m, mp, nb);
  mb = 2 * mp + rank;
}

// Flat pair-tile index T of a batch -> problem b and its pair tile Tl.
__device__ __forceinline__ int tile_problem(const TcParams& prm, int T, int& Tl) {
  const int slot = T / prm.ntiles_p;
  Tl = T - slot * prm.ntiles_p;
  return prm.active ? prm.active[slot] : slot;
}

// Problems whose fit has finished (or, for the gated dense fallback, that
// need no dense product in this trial) contribute no tiles.  The control
// block does not change while the kernel runs, so every warp role skips the
// same tiles.
__device__ __forceinline__ bool skip_problem(const TcParams& prm, int b) {
  if (prm.ctrl == nullptr) return false;
  const Ctrl& c = prm.ctrl[b];
  return c.done || (prm.gate_dense && !c.dense && !c.ymode);
}

// Prox mode, a problem whose control block asks for the coarse gradient:
// G from the one product hi x hi (the lo planes are neither loaded nor
// multiplied).  The producer and the MMA issuer read the same flag, which
// does not change while the kernel runs.
__device__ __forceinline__ bool coarse_tile(const TcParams& prm, int b) {
  return prm.coarse_ok && prm.ctrl != nullptr && prm.ctrl[b].coarse != 0;
}

// First flat tile >= T (stepping by `stride`) that is not skipped; ntot if none.
__device__ __forceinline__ int next_tile(const TcParams& prm, int T, int ntot, int stride, int& b, int& Tl) {
  for (; T < ntot; T += stride) {
    b = tile_problem(prm, T, Tl);
    if (!skip_problem(prm, b)) return T;
  }
  return ntot;
}

struct EpiArgs {
  float tau, lam, lam_d, scale;
  float* out;
  void* out_hi;
  void* out_lo;
  const float* aux;
  int64_t M, N;
  uint64_t pol_stream;  // L2 evict-first policy for the iterate stream
  // sparse Delta bucket of the current 32-row group (null: dense planes)
  uint32_t* bkey;
  float* bval;
  int* bcnt;
  int* dense_flag;
  int cap;
  int64_t row0;         // first row of the group
  // support bitmask of the Eq. 3.8 refit (null: plain fit): bit (i, j) set
  // where omega_ij may be nonzero; elsewhere the weight is infinite
  const uint32_t* mask;
  int64_t mask_ld;      // 32-bit words per row
};

// Per-thread tile partials.  The dense sums run in FP32 over the thread's
// share of one tile (at most 128 terms) and are folded across warps and tiles
// in FP64: FP64 is a slow pipe on this part, so it is kept out of the
// per-element path.  The diagonal terms (one per row) are FP64 throughout.
struct Sums {
  float r0 = 0.f, r1 = 0.f, r4 = 0.f, bad = 0.f, kkt = 0.f;
  double r2 = 0.0, r3 = 0.0;
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

// Asynchronous copy of the 32 x 32 FP32 block src[row_base .. +31][col0 .. +31]
// (row-major, 16-byte aligned rows) into buf, row-major: 8 x 16 bytes a thread,
// four full 128-byte rows per warp instruction.
__device__ __forceinline__ void prefetch_block(float* buf, const float* __restrict__ src, int64_t ld,
                                               int64_t row_base, int64_t col0, int lane, uint64_t pol) {
  const uint32_t sbase = ptx::smem_u32(buf);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int idx = k * 32 + lane, r = idx >> 3, seg = idx & 7;
    const float* g = src + (row_base + r) * ld + col0 + 4 * seg;
    ptx::cp_async16_hint(sbase + (uint32_t)(r * 128 + seg * 16), g, pol);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}


// Rows with at most this many nonempty rows in a 32 x 32 block are fetched
// entry by entry, denser blocks row by row.
constexpr int kGatherRows = 8;

// The nonzero entries of the 32 x 32 block src[row_base .. +31][col0 .. +31]
// into buf, row-major with each row's 16-byte slots XOR-swizzled by row
// (columns 4s .. 4s + 3 of row r at slot s ^ (r & 7)), so that the copies and
// the column reads below are free of bank conflicts.  rbits holds, in lane r,
// the occupancy word of row r (bit c: column col0 + c nonzero).  A block with
// few nonempty rows is gathered one row per instruction, lane c copying entry
// c when its bit is set (only the sectors that hold nonzeros are read); a
// denser one is copied by lane r as its row's eight 16-byte segments (eight
// instructions whatever the block holds).  Entries whose bit is clear are not
// defined in buf; read_block_masked reads them as 0.  Nothing past column
// ld - 1 is read.
__device__ __forceinline__ void prefetch_rows(float* buf, const float* __restrict__ src, int64_t ld,
                                              int64_t row_base, int64_t col0, uint32_t rbits, int lane,
                                              uint64_t pol) {
  const uint32_t sbuf = ptx::smem_u32(buf);
  uint32_t rows = __ballot_sync(0xffffffffu, rbits != 0u);
  if (__popc(rows) <= kGatherRows) {
    while (rows != 0u) {
      const int r = __ffs(rows) - 1;
      rows &= rows - 1u;
      const uint32_t m = __shfl_sync(0xffffffffu, rbits, r);
      if ((m >> lane) & 1u)
        ptx::cp_async4_hint(sbuf + (uint32_t)((r * 32 + ((((lane >> 2) ^ (r & 7))) << 2) + (lane & 3)) * 4),
                            src + (row_base + r) * ld + col0 + lane, pol);
    }
  } else if (rbits != 0u) {
    const uint32_t sbase = sbuf + (uint32_t)lane * 128u;
    const float* g = src + (row_base + lane) * ld + col0;
#pragma unroll
    for (int seg = 0; seg < 8; ++seg)
      if (col0 + 4 * seg + 4 <= ld) ptx::cp_async16_hint(sbase + (uint32_t)((seg ^ (lane & 7)) << 4), g + 4 * seg, pol);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}


// Asynchronous copy of one tile's occupancy words into a word slot (prox
// mode): row k is the current iterate's word of chunk ch0 + k; lane r of a
// row is the word of matrix row row_base + r.  Chunks past nch, or a tile
// whose rows lie past the matrix, read as zero words (no global read).  One
// 16-byte copy a lane.
__device__ __forceinline__ void load_words(uint32_t* slot, const uint32_t* bmc, int64_t ldbm, int64_t ch0, int64_t nch,
                                           int64_t row_base, bool rows_in, int lane, bool commit = true) {
  const uint32_t sbase = ptx::smem_u32(slot);
  const int k = lane >> 3, seg = lane & 7;
  const bool in = rows_in && ch0 + k < nch;
  const uint32_t* src = bmc + (in ? (ch0 + k) * ldbm + row_base + 4 * seg : 0);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sbase + (uint32_t)((k * 32 + 4 * seg) * 4)),
               "l"(src), "r"(in ? 16 : 0)
               : "memory");
  if (commit) asm volatile("cp.async.commit_group;" ::: "memory");
}

// Column `lane` of a block written by prefetch_block (conflict-free reads).
__device__ __forceinline__ void read_block_column(const float* buf, int lane, float (&pre)[32]) {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) pre[r] = buf[r * 32 + lane];
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

// Split of x to the operand planes at ph / pl (L2 policy pol).
template <int PT>
__device__ __forceinline__ void st_split_hint(typename Plane<PT>::E* ph, typename Plane<PT>::E* pl, float x,
                                              uint64_t pol) {
  typename Plane<PT>::E h, l;
  Plane<PT>::split(x, h, l);
  if constexpr (PT == kPlaneTf32) {
    ptx::st_f32_hint(ph, h, pol);
    ptx::st_f32_hint(pl, l, pol);
  } else {
    ptx::st_b16_hint(ph, __bfloat16_as_ushort(h), pol);
    ptx::st_b16_hint(pl, __bfloat16_as_ushort(l), pol);
  }
}

// Y+ = Y + Delta X^T (aux = Y) or Y = Omega X^T (aux = null) for column colt.
template <int PT, bool CHECK>
__device__ __forceinline__ void y_chunk(const EpiArgs& ea, const TcParams& prm, int64_t row_base, int64_t colt,
                                        const float (&v)[32], const float (&pre)[32], Sums& sm) {
  float sd = 0.f, sn = 0.f, chk = 0.f;
  const bool cok = !CHECK || colt < ea.N;
  const bool has_aux = ea.aux != nullptr;
  using E = typename Plane<PT>::E;
  float* po = ea.out ? ea.out + row_base * prm.ldout + colt : nullptr;
  E* ph = ea.out_hi ? static_cast<E*>(ea.out_hi) + row_base * prm.ldplane + colt : nullptr;
  E* pl = ea.out_lo ? static_cast<E*>(ea.out_lo) + row_base * prm.ldplane + colt : nullptr;
  const uint32_t ldo = (uint32_t)prm.ldout, ldp = (uint32_t)prm.ldplane;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    if (CHECK && !(cok && row_base + r < ea.M)) continue;
    const float dv = v[r] * ea.scale;
    const float yn = (has_aux ? pre[r] : 0.f) + dv;
    sd = fmaf(dv, dv, sd);
    sn = fmaf(yn, yn, sn);
    chk = fmaf(yn, 0.f, chk);
    if (po) ptx::st_f32_hint(po + r * ldo, yn, ea.pol_stream);
    if (ph) st_split_hint<PT>(ph + r * ldp, pl + r * ldp, yn, ea.pol_stream);
  }
  sm.r0 += sd;
  sm.r1 += sn;
  if (chk != 0.f) sm.bad += 1.f;
}

// Row `lane` of a block written by prefetch_rows, as eight 16-byte reads
// (conflict-free: each quarter-warp reads eight distinct slots): entry c
// where bit c of word is set (word: this row's occupancy word), else 0.
__device__ __forceinline__ void read_row_masked(const float* buf, int lane, uint32_t word, float (&pre)[32]) {
  asm volatile("cp.async.wait_group 1;" ::: "memory");  // the newest group (the next chunk) may still fly
  __syncwarp();
  const float4* row = reinterpret_cast<const float4*>(buf + lane * 32);
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const float4 x = row[g ^ (lane & 7)];
    pre[4 * g + 0] = ((word >> (4 * g + 0)) & 1u) ? x.x : 0.f;
    pre[4 * g + 1] = ((word >> (4 * g + 1)) & 1u) ? x.y : 0.f;
    pre[4 * g + 2] = ((word >> (4 * g + 2)) & 1u) ? x.z : 0.f;
    pre[4 * g + 3] = ((word >> (4 * g + 3)) & 1u) ? x.w : 0.f;
  }
  __syncwarp();
}

// G = acc / n, Eq. 3.5 on A = Omega - tau G, Omega+ and Delta (to the
// buckets, or to operand planes), and the trial / KKT partial sums for one
// 32 x 32 chunk, in TMEM order: lane `lane` owns row row_base + lane, and
// v[c], pre[c] are its columns col0 + c.  CHECK handles the matrix edge and
// the diagonal; the unchecked form is the hot path.  Omega+ is stored only
// where it is nonzero (the receiving buffer's values count only where its
// bitmap has a bit), as 16-byte stores in a whole chunk.  Returns this row's
// occupancy word of Omega+ (bit c: column col0 + c nonzero), with no
// transpose of the accumulator or of the words.
template <int PT, bool CHECK, bool MASK, bool SPARSE>
__device__ __forceinline__ uint32_t prox_row_chunk(const EpiArgs& ea, const TcParams& prm, int64_t row_base,
                                                   int64_t col0, float (&v)[32], float (&pre)[32], Sums& sm,
                                                   int lane) {
  float sd = 0.f, sl1 = 0.f, kk = 0.f;
  const float tau = ea.tau, tlam = ea.tau * ea.lam, lam = ea.lam, scale = ea.scale;
  const int64_t row = row_base + lane;
  const bool rok = !CHECK || row < ea.M;
  constexpr bool sparse = SPARSE;
  using E = typename Plane<PT>::E;
  float* po = ea.out + row * prm.ldout + col0;
  E* ph = sparse ? nullptr : static_cast<E*>(ea.out_hi) + row * prm.ldplane + col0;
  E* pl = sparse ? nullptr : static_cast<E*>(ea.out_lo) + row * prm.ldplane + col0;
  const int64_t dcol = row + prm.row_off - col0;  // this row's diagonal column in the chunk
  uint32_t mw = 0xffffffffu;
  if (MASK && rok) mw = __ldg(ea.mask + row * ea.mask_ld + (col0 >> 5));
  uint32_t nzmask = 0u, newrow = 0u;
  float wdiag = 1.f;
  bool has_diag = false;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    float d = 0.f;
    if (!CHECK || (rok && col0 + c < ea.N)) {
      const float g = v[c] * scale;
      const float om = pre[c];
      const float a = fmaf(-tau, g, om);
      float w;
      if (CHECK && dcol == c) {
        w = diag_prox(a, tau, ea.lam_d);
        wdiag = w;
        has_diag = true;
        kk = fmaxf(kk, kkt_entry(om, g, true, lam, ea.lam_d));
      } else {
        float lam_e = lam, tlam_e = tlam;
        if (MASK && !((mw >> c) & 1u)) {
          lam_e = INFINITY;
          tlam_e = INFINITY;
        }
        const float m = fabsf(a) - tlam_e;
        w = m <= 0.f ? 0.f : copysignf(m, a);
        sl1 += fabsf(w);
        const float kz = fabsf(g) - lam_e;
        const float knz = fabsf(g + copysignf(lam_e, om));
        kk = fmaxf(kk, om != 0.f ? knz : kz);
      }
      d = w - om;
      sd = fmaf(d, d, sd);
      const bool nzw = w != 0.f;
      newrow |= nzw ? (1u << c) : 0u;
      if (CHECK) {
        ptx::st_f32_hint_if(po + c, w, ea.pol_stream, nzw);
        if (!sparse) st_split_hint<PT>(ph + c, pl + c, d, ea.pol_stream);
      } else {
        pre[c] = w;
      }
    }
    v[c] = d;
    nzmask |= (d != 0.f) ? (1u << c) : 0u;
  }
  if (!CHECK) {
#pragma unroll
    for (int g = 0; g < 8; ++g)
      ptx::st_v4_hint_if(po + 4 * g, __float_as_uint(pre[4 * g]), __float_as_uint(pre[4 * g + 1]),
                         __float_as_uint(pre[4 * g + 2]), __float_as_uint(pre[4 * g + 3]), ea.pol_stream,
                         ((newrow >> (4 * g)) & 0xFu) != 0u);
    if (!sparse) {
      if constexpr (PT == kPlaneTf32) {
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          float hi[4], lo[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) split_tf32(v[4 * g + t], hi[t], lo[t]);
          ptx::st_v4_hint_if(ph + 4 * g, __float_as_uint(hi[0]), __float_as_uint(hi[1]), __float_as_uint(hi[2]),
                             __float_as_uint(hi[3]), ea.pol_stream, true);
          ptx::st_v4_hint_if(pl + 4 * g, __float_as_uint(lo[0]), __float_as_uint(lo[1]), __float_as_uint(lo[2]),
                             __float_as_uint(lo[3]), ea.pol_stream, true);
        }
      } else {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(v[8 * g + 2 * t], h0, l0);
            split_bf16(v[8 * g + 2 * t + 1], h1, l1);
            hw[t] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lw[t] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
          }
          ptx::st_v4_hint_if(ph + 8 * g, hw[0], hw[1], hw[2], hw[3], ea.pol_stream, true);
          ptx::st_v4_hint_if(pl + 8 * g, lw[0], lw[1], lw[2], lw[3], ea.pol_stream, true);
        }
      }
    }
  }
  if (CHECK && has_diag) {
    sm.r2 += log((double)wdiag);
    sm.r3 += (double)wdiag;
  }
  if (sparse) {
    const int cnt = __popc(nzmask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total > 0) {
      int base = 0;
      if (lane == 31) base = atomicAdd(ea.bcnt, total);
      base = __shfl_sync(0xffffffffu, base, 31);
      int pos = base + incl - cnt;
      uint32_t m = nzmask;
      while (m != 0u) {
        const int c = __ffs(m) - 1;
        m &= m - 1u;
        float dc = 0.f;
#pragma unroll
        for (int u = 0; u < 32; ++u)
          if (u == c) dc = v[u];
        if (pos < ea.cap) {
          ea.bkey[pos] = ((uint32_t)lane << 25) | (uint32_t)(col0 + c);
          ea.bval[pos] = dc;
        }
        ++pos;
      }
      if (lane == 31 && base + total > ea.cap) {
        atomicOr(ea.dense_flag, 1);
        if (prm.any_dense != nullptr) atomicOr(prm.any_dense, 1);
      }
    }
  }
  int nnz = __popc(newrow);
  if (CHECK && dcol >= 0 && dcol < 32 && ((newrow >> dcol) & 1u)) nnz -= 1;
  sm.r0 += sd;
  sm.r1 += sl1;
  sm.r4 += (float)nnz;
  sm.kkt = fmaxf(sm.kkt, kk);
  if (!(sd <= 3.4e38f)) sm.bad += 1.f;
  return newrow;
}

__device__ __forceinline__ void grad_chunk(const EpiArgs& ea, const TcParams& prm, int64_t row_base, int64_t colt,
                                           bool check, const float (&v)[32]) {
  const bool cok = colt < ea.N;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int64_t row = row_base + r;
    if (check && !(cok && row < ea.M)) continue;
    float g = v[r] * ea.scale;
    if (prm.smooth && check && row + prm.row_off == colt) g -= 1.f / ea.aux[row * prm.ldaux + colt];
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
template <int MODE, int PT>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const __grid_constant__ TcParams prm) {
  constexpr int BK = kBK<PT>;
  Ctrl* ctrl = prm.ctrl;
  const bool batch = prm.nprob > 1 || prm.active != nullptr;
  if (!batch && ctrl != nullptr && (ctrl->done || (prm.gate_dense && !ctrl->dense))) return;
  if (prm.gate_dense && prm.any_dense != nullptr && *prm.any_dense == 0) return;
  const int ntot = (prm.active ? *prm.nactive : (prm.nprob > 1 ? prm.nprob : 1)) * prm.ntiles_p;
  if (ntot <= 0) return;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* epi_buf = reinterpret_cast<float*>(smem + kStages * kStageBytes);
  uint32_t* word_area = reinterpret_cast<uint32_t*>(smem + kStages * kStageBytes + kEpiBufBytes);
  uint8_t* tail = smem + kStages * kStageBytes + kEpiBufBytes + kWordBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(tail);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* tile_count = reinterpret_cast<int*>(tmem_slot + 3);  // [2], by tile parity
  double* red = reinterpret_cast<double*>(tail + kRedOffset);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rank = (int)ptx::cluster_ctarank();  // 0: leader (issues the MMAs), 1: peer
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&full[s], 1);   // leader: its expect_tx; both CTAs' copies complete on it
      ptx::mbar_init(&empty[s], 1);  // released by the leader's MMA commit
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], 2 * kEpiWarps);  // leader: one arrival per epilogue warp of the pair
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    tile_count[0] = 0;
    tile_count[1] = 0;
    ptx::fence_mbar_init();
  }
  // the peer's barriers must be live before any copy, commit or arrival reaches them
  ptx::cluster_sync();
  if (warp == 1) {
    ptx::tmem_alloc_pair(tmem_slot, kTmemCols);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int cta = blockIdx.x / 2;     // pair index
  const int nctas = gridDim.x / 2;    // pairs

  const CUtensorMap* mB_hi = &prm.b_hi;
  const CUtensorMap* mB_lo = &prm.b_lo;
  const uint32_t smem_base = ptx::smem_u32(smem);

  if (warp == 0) {
    // ------------------------------------------------------ TMA producer --
    if (lane == 0) {
      for (int q = 0; q < 2; ++q) {
        ptx::tma_prefetch_desc(&prm.a_hi[q]);
        ptx::tma_prefetch_desc(&prm.a_lo[q]);
      }
      ptx::tma_prefetch_desc(mB_hi);
      ptx::tma_prefetch_desc(mB_lo);
      // operand tiles are shared by many CTAs: keep them in L2 (the A operand
      // of the Y GEMM is the Delta stream, read once: let it leave first)
      const uint64_t pol_a = (MODE == kModeY && prm.ctrl != nullptr) ? ptx::policy_evict_first()
                                                                       : ptx::policy_evict_last();
      const uint64_t pol_keep = ptx::policy_evict_last();
      uint32_t s = 0, ph = 0;
      uint32_t fill_ph[kStages];
      bool filled[kStages];
      for (int q = 0; q < kStages; ++q) { filled[q] = false; fill_ph[q] = 0; }
      bool ok = true;
      bool withhold = prm.withhold_first != 0;  // test of the timeout path: skip the first stage's copies
      int b = 0, Tl = 0;
      for (int T = next_tile(prm, cta, ntot, nctas, b, Tl); T < ntot && ok;
           T = next_tile(prm, T + nctas, ntot, nctas, b, Tl)) {
        int mb, nb;
        pair_tile(Tl, prm, rank, mb, nb);
        const int cb = ctrl ? ctrl[b].cur : 0;
        const int asel = prm.a_nxt ? (cb ^ 1) : cb;
        const CUtensorMap* mA_hi = &prm.a_hi[asel];
        const CUtensorMap* mA_lo = &prm.a_lo[asel];
        const int nkb = prm.kb_of ? prm.kb_of[b] : prm.num_kb;
        const int32_t zb = prm.b_batched ? b : 0;
        const bool one = coarse_tile(prm, b);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!ptx::mbar_wait_cluster(&empty[s], ph ^ 1u, abort_flag, prm.wait_ns)) { ok = false; break; }
          if (!withhold) {
            // the leader expects the bytes of both CTAs' copies of this stage
            if (rank == 0) ptx::mbar_arrive_expect_tx(&full[s], one ? 2 * (kABytes + kBBytes) : 2 * kStageBytes);
            const uint32_t st = smem_base + s * kStageBytes;
            const uint32_t fb = ptx::map_to_cta(&full[s], 0);
            const int32_t by = nb * kBN + rank * kBHalf;
            ptx::tma_load_3d_pair(st, mA_hi, fb, kb * BK, mb * BM, b, pol_a);
            if (!one) ptx::tma_load_3d_pair(st + kABytes, mA_lo, fb, kb * BK, mb * BM, b, pol_a);
            ptx::tma_load_3d_pair(st + 2 * kABytes, mB_hi, fb, kb * BK, by, zb, pol_keep);
            if (!one) ptx::tma_load_3d_pair(st + 2 * kABytes + kBBytes, mB_lo, fb, kb * BK, by, zb, pol_keep);
            filled[s] = true;
            fill_ph[s] = ph;
          }
          withhold = false;
          if (++s == kStages) { s = 0; ph ^= 1u; }
        }
      }
      if (ok) {
        // wait for the last release of every slot, so that no commit can
        // still be on its way to this CTA's barriers when it leaves
        for (int q = 0; q < kStages; ++q)
          if (filled[q] && !ptx::mbar_wait_cluster(&empty[q], fill_ph[q], abort_flag, prm.wait_ns)) ok = false;
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.err, kErrWaitTimeout);
        // let the leader's copies already issued land before the CTA can exit
        // (the peer's copies complete on the leader's barriers; the exit
        // barrier of the pair below keeps the leader alive meanwhile)
        if (rank == 0)
          for (int q = 0; q < kStages; ++q)
            if (filled[q]) (void)ptx::mbar_wait_cluster(&full[q], fill_ph[q], nullptr, prm.wait_ns);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------- MMA issuer (leader only) --
    if (lane == 0 && rank == 0) {
      constexpr uint32_t idesc =
          PT == kPlaneTf32 ? ptx::idesc_tf32_f32(2 * BM, kBN) : ptx::idesc_bf16_f32(2 * BM, kBN);
      uint32_t s = 0, ph = 0;
      bool ok = true;
      int i = 0;
      int b = 0, Tl = 0;
      for (int T = next_tile(prm, cta, ntot, nctas, b, Tl); T < ntot && ok;
           T = next_tile(prm, T + nctas, ntot, nctas, b, Tl), ++i) {
        const uint32_t acc = i & 1, aph = (i >> 1) & 1;
        if (!ptx::mbar_wait_cluster(&tempty[acc], aph ^ 1u, abort_flag, prm.wait_ns)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t d = tmem_base + acc * kBN;
        const int nkb = prm.kb_of ? prm.kb_of[b] : prm.num_kb;
        const bool one = coarse_tile(prm, b);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!ptx::mbar_wait_cluster(&full[s], ph, abort_flag, prm.wait_ns)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t st = smem_base + s * kStageBytes;
          const uint64_t a_hi = ptx::sdesc_k64(st);
          const uint64_t a_lo = ptx::sdesc_k64(st + kABytes);
          const uint64_t b_hi = ptx::sdesc_k64(st + 2 * kABytes);
          const uint64_t b_lo = ptx::sdesc_k64(st + 2 * kABytes + kBBytes);
          if (one) {
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk) {
              const uint64_t off = (uint64_t)(kk * 2);
              if constexpr (PT == kPlaneTf32) ptx::mma_tf32_pair(d, a_hi + off, b_hi + off, idesc, (kb | kk) != 0);
              else ptx::mma_f16_pair(d, a_hi + off, b_hi + off, idesc, (kb | kk) != 0);
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk) {
              const uint64_t off = (uint64_t)(kk * 2);  // 32 bytes >> 4: K = 16 BF16 or 8 TF32
              if constexpr (PT == kPlaneTf32) {
                ptx::mma_tf32_pair(d, a_lo + off, b_hi + off, idesc, (kb | kk) != 0);
                ptx::mma_tf32_pair(d, a_hi + off, b_lo + off, idesc, 1u);
                ptx::mma_tf32_pair(d, a_hi + off, b_hi + off, idesc, 1u);
              } else {
                ptx::mma_f16_pair(d, a_lo + off, b_hi + off, idesc, (kb | kk) != 0);
                ptx::mma_f16_pair(d, a_hi + off, b_lo + off, idesc, 1u);
                ptx::mma_f16_pair(d, a_hi + off, b_hi + off, idesc, 1u);
              }
            }
          }
          // release the slot in both CTAs once these MMAs have read it
          ptx::mma_commit_pair(ptx::map_to_cta(&empty[s], 0));
          ptx::mma_commit_pair(ptx::map_to_cta(&empty[s], 1));
          if (++s == kStages) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;
        ptx::mma_commit_pair(ptx::map_to_cta(&tfull[acc], 0));
        ptx::mma_commit_pair(ptx::map_to_cta(&tfull[acc], 1));
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.err, kErrWaitTimeout);
        ptx::mma_commit_pair(ptx::map_to_cta(drain, 0));
        (void)ptx::mbar_wait(drain, 0, nullptr, prm.wait_ns);
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
    float* tbuf = epi_buf + e * 2048;
    float* const pbuf[2] = {tbuf, tbuf + 1024};  // prox mode: chunk k's block in pbuf[k & 1]
    EpiArgs ea;
    ea.lam = prm.lam;
    ea.lam_d = prm.lam_d;
    ea.scale = prm.scale;
    ea.M = prm.M;
    ea.N = prm.N;
    ea.pol_stream = ptx::policy_evict_first();
    ea.bkey = nullptr;
    ea.bval = nullptr;
    ea.bcnt = nullptr;
    ea.dense_flag = prm.dense_flag;
    ea.cap = prm.cap;
    ea.row0 = 0;
    ea.mask = prm.mask;
    ea.mask_ld = prm.mask_ld;
    constexpr bool kNeedAux = (MODE == kModeProx || MODE == kModeY);
    constexpr bool kProx = MODE == kModeProx;
    // Prox mode keeps one tile of lookahead: the next tile's occupancy words
    // are copied during this tile's first chunk, and the iterate's blocks are
    // staged two chunks ahead (the next tile's first two during this tile's
    // last two), so that no chunk starts on a memory round trip.  One
    // cp.async group per chunk (empty when there is nothing to fetch), so
    // that waiting for all but the newest group finds chunk k's block.
    uint32_t* wslots = word_area + e * 2 * kWordSlotWords;
    const int64_t nch = (prm.N + 31) >> 5;
    int slot = 0;
    bool pending = false;
    int i = 0;
    int b = 0, Tl = 0;
    int T = next_tile(prm, cta, ntot, nctas, b, Tl);
    if (kProx && T < ntot) {
      int mb0, nb0;
      pair_tile(Tl, prm, rank, mb0, nb0);
      const int cb0 = ctrl ? ctrl[b].cur : 0;
      const int64_t rb0 = (int64_t)mb0 * BM + 32 * q, cbase0 = (int64_t)nb0 * kBN + h * kColsPerWarp;
      load_words(wslots, prm.bm[cb0] + b * prm.s_bm, prm.ldbm, cbase0 >> 5, nch, rb0, rb0 < prm.M, lane);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp();
      prefetch_rows(pbuf[0], prm.aux[cb0] + b * prm.s_aux, prm.ldaux, rb0, cbase0, wslots[lane], lane, ea.pol_stream);
      prefetch_rows(pbuf[1], prm.aux[cb0] + b * prm.s_aux, prm.ldaux, rb0, cbase0 + 32, wslots[32 + lane], lane,
                    ea.pol_stream);
      pending = true;
    }
    for (; T < ntot; ++i) {
      int bN = 0, TlN = 0;
      const int TN = next_tile(prm, T + nctas, ntot, nctas, bN, TlN);
      int mb, nb;
      pair_tile(Tl, prm, rank, mb, nb);
      // this tile's problem: its iterate buffers, step and penalty
      const int cb = ctrl ? ctrl[b].cur : 0, nx = cb ^ 1;
      ea.out = prm.out[nx] ? prm.out[nx] + b * prm.s_out : nullptr;
      using PE = typename Plane<PT>::E;  // s_plane counts plane elements
      ea.out_hi = prm.out_hi[nx] ? static_cast<PE*>(prm.out_hi[nx]) + b * prm.s_plane : nullptr;
      ea.out_lo = prm.out_lo[nx] ? static_cast<PE*>(prm.out_lo[nx]) + b * prm.s_plane : nullptr;
      ea.aux = prm.aux[cb] ? prm.aux[cb] + b * prm.s_aux : nullptr;
      ea.tau = ctrl ? (float)ctrl[b].tau : 0.f;
      if (batch && ctrl != nullptr) {
        ea.lam = (float)ctrl[b].lam;
        ea.lam_d = (float)ctrl[b].lam_d;
        if (MODE == kModeProx) ea.scale = (float)ctrl[b].inv_n;
        ea.dense_flag = &ctrl[b].dense;
      }
      double* part_b = prm.part ? prm.part + b * prm.s_part * ((MODE == kModeY) ? kYSlots : kProxSlots) : nullptr;
      // cp.async needs 16-byte aligned rows
      const bool aux_async = ea.aux != nullptr && (prm.ldaux % 4) == 0 && ((uintptr_t)ea.aux & 15u) == 0;
      const uint32_t acc = i & 1, aph = (i >> 1) & 1;
      const int64_t row_base = (int64_t)mb * BM + 32 * q;
      const int64_t col_base = (int64_t)nb * kBN + h * kColsPerWarp;
      const bool rows_full = row_base + 32 <= prm.M;
      // sparse Delta buckets, or (a batch problem in dense mode) Delta planes
      if (MODE == kModeProx && prm.keys != nullptr && !(batch && ctrl != nullptr && ctrl[b].ymode)) {
        const int64_t bkt = b * prm.s_bkt + row_base / 32;  // one bucket per warp row quarter
        ea.bkey = prm.keys + bkt * prm.cap;
        ea.bval = prm.vals + bkt * prm.cap;
        ea.bcnt = prm.counts + bkt;
        ea.row0 = row_base;
      } else {
        ea.bkey = nullptr;
      }
      Sums sm;
      float pre[32];
      // Prox mode: this tile's occupancy words (slot `slot`, lane r: row
      // row_base + r) of the current iterate (which entries of Omega exist);
      // the next tile's go to the other slot.
      const uint32_t* wcur = wslots + slot * kWordSlotWords;
      uint32_t* wnext = wslots + (slot ^ 1) * kWordSlotWords;
      uint32_t* bmn = kProx ? prm.bm[nx] + b * prm.s_bm : nullptr;
      const int64_t ch0 = col_base >> 5;
      int cbN = 0;
      int64_t rbN = 0, cbaseN = 0;
      if (kProx && TN < ntot) {
        int mbN, nbN;
        pair_tile(TlN, prm, rank, mbN, nbN);
        cbN = ctrl ? ctrl[bN].cur : 0;
        rbN = (int64_t)mbN * BM + 32 * q;
        cbaseN = (int64_t)nbN * kBN + h * kColsPerWarp;
      }
      // the first chunk's operand does not depend on the MMA: start fetching it
      // before waiting for the accumulator (prox mode: fetched during the
      // previous tile)
      if (!kProx && kNeedAux && ea.aux != nullptr && aux_async && rows_full && col_base + 32 <= prm.N) {
        prefetch_block(tbuf, ea.aux, prm.ldaux, row_base, col_base, lane, ea.pol_stream);
        pending = true;
      }
      const bool ok = ptx::mbar_wait_cluster(&tfull[acc], aph, abort_flag, prm.wait_ns);
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
          const int k = c >> 5;
          if (kProx) {
            read_row_masked(pbuf[k & 1], lane, wcur[k * 32 + lane], pre);
            // the next tile's words join the group of chunk k + 2's block
            if (k == 0 && TN < ntot)
              load_words(wnext, prm.bm[cbN] + bN * prm.s_bm, prm.ldbm, cbaseN >> 5, nch, rbN, rbN < prm.M, lane,
                         false);
            // the buffer just read takes the block two chunks ahead: this
            // tile's, or (chunks 2 and 3) the next tile's first two, whose
            // words arrived with chunk 2's block
            if (c + 64 < kColsPerWarp) {
              prefetch_rows(pbuf[k & 1], ea.aux, prm.ldaux, row_base, col0 + 64, wcur[(k + 2) * 32 + lane], lane,
                            ea.pol_stream);
            } else if (TN < ntot) {
              const int kn = k + 2 - kColsPerWarp / 32;
              prefetch_rows(pbuf[k & 1], prm.aux[cbN] + bN * prm.s_aux, prm.ldaux, rbN, cbaseN + 32 * kn,
                            wnext[kn * 32 + lane], lane, ea.pol_stream);
            } else {
              asm volatile("cp.async.commit_group;" ::: "memory");
            }
          } else if (kNeedAux && ea.aux != nullptr) {
            if (pending) read_block_column(tbuf, lane, pre);
            else load_column(ea.aux, prm.ldaux, row_base, colt, full, ea, pre);
            pending = false;
          }
          uint32_t rr[32];
          ptx::tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(32 * q) << 16) + acc * kBN + h * kColsPerWarp + c, rr);
          ptx::tmem_ld_wait();
          float v[32];
          if (kProx) {
#pragma unroll
            for (int u = 0; u < 32; ++u) v[u] = __uint_as_float(rr[u]);
          } else {
            transpose32(tbuf, rr, lane, v);
          }
          // the buffer is free again: fetch the next chunk's operand while this one computes
          if (!kProx && kNeedAux && ea.aux != nullptr && aux_async && c + 32 < kColsPerWarp && rows_full &&
                     col0 + 64 <= prm.N) {
            prefetch_block(tbuf, ea.aux, prm.ldaux, row_base, col0 + 32, lane, ea.pol_stream);
            pending = true;
          }
          if (row_base >= prm.M || col0 >= prm.N) continue;  // warp-uniform
          const bool diag = (row_base + prm.row_off == col0);
          if (MODE == kModeY) {
            if (full) y_chunk<PT, false>(ea, prm, row_base, colt, v, pre, sm);
            else y_chunk<PT, true>(ea, prm, row_base, colt, v, pre, sm);
          } else if (MODE == kModeProx) {
            // compile-time variants: full interior chunk, Delta to buckets, no refit mask is the hot one
            const bool fast = full && !diag;
            uint32_t newrow;
            if (ea.mask == nullptr) {
              if (ea.bkey != nullptr) {
                if (fast) newrow = prox_row_chunk<PT, false, false, true>(ea, prm, row_base, col0, v, pre, sm, lane);
                else newrow = prox_row_chunk<PT, true, false, true>(ea, prm, row_base, col0, v, pre, sm, lane);
              } else {
                if (fast) newrow = prox_row_chunk<PT, false, false, false>(ea, prm, row_base, col0, v, pre, sm, lane);
                else newrow = prox_row_chunk<PT, true, false, false>(ea, prm, row_base, col0, v, pre, sm, lane);
              }
            } else if (ea.bkey != nullptr) {
              if (fast) newrow = prox_row_chunk<PT, false, true, true>(ea, prm, row_base, col0, v, pre, sm, lane);
              else newrow = prox_row_chunk<PT, true, true, true>(ea, prm, row_base, col0, v, pre, sm, lane);
            } else {
              if (fast) newrow = prox_row_chunk<PT, false, true, false>(ea, prm, row_base, col0, v, pre, sm, lane);
              else newrow = prox_row_chunk<PT, true, true, false>(ea, prm, row_base, col0, v, pre, sm, lane);
            }
            // the occupancy of Omega+ in this chunk: this lane's row word
            bmn[(ch0 + k) * prm.ldbm + row_base + lane] = newrow;
          } else if (MODE == kModeGrad) {
            grad_chunk(ea, prm, row_base, colt, diag || !full, v);
          } else {
            gram_chunk(prm, row_base, colt, v, ea);
          }
        }
      }
      if (!kProx && pending) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        pending = false;
      }
      // Partial sums of this tile: FP32 warp trees, then FP64 across the warps
      // in a fixed order, by whichever warp finishes the tile last (a counter
      // per tile parity; no warp waits for another).  The TMEM release comes
      // after, so no warp can reach tile i + 2, and reuse this parity's
      // partials and counter, before the fold of tile i is done.
      constexpr int W = (MODE == kModeY) ? kYSlots : kProxSlots;
      double* red_t = red + (i & 1) * kEpiWarps * 8;
      if (MODE == kModeY || MODE == kModeProx) {
        float f0 = sm.r0, f1 = sm.r1, f4 = sm.r4, fb = sm.bad, fk = sm.kkt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          f0 += __shfl_xor_sync(0xffffffffu, f0, o);
          f1 += __shfl_xor_sync(0xffffffffu, f1, o);
          f4 += __shfl_xor_sync(0xffffffffu, f4, o);
          fb += __shfl_xor_sync(0xffffffffu, fb, o);
          fk = fmaxf(fk, __shfl_xor_sync(0xffffffffu, fk, o));
        }
        double d2 = sm.r2, d3 = sm.r3;
        // diagonal entries exist only where the tile's row and column ranges meet
        const int64_t r_lo = (int64_t)mb * BM + prm.row_off, c_lo = (int64_t)nb * kBN;
        if (MODE == kModeProx && r_lo < c_lo + kBN && c_lo < r_lo + BM) {
          d2 = warp_sum(d2);
          d3 = warp_sum(d3);
        }
        if (lane == 0) {
          double* rw = red_t + e * 8;
          if (MODE == kModeY) {
            rw[kYDiff2] = (double)f0; rw[kYNorm2] = (double)f1; rw[kYBad] = (double)fb; rw[3] = 0.0;
          } else {
            rw[kPDelta2] = (double)f0; rw[kPLogDiag] = d2; rw[kPDiagSum] = d3; rw[kPL1Off] = (double)f1;
            rw[kPNnz] = (double)f4; rw[kPKkt] = (double)fk; rw[kPBad] = (double)fb; rw[7] = 0.0;
          }
        }
      }
      if (MODE == kModeY || MODE == kModeProx) {
        int done = 0;
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();  // this warp's partials before its count
          done = atomicAdd(&tile_count[i & 1], 1) + 1;
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done == kEpiWarps) {
          __threadfence_block();  // every warp's partials after the last count
          if (part_b != nullptr && lane < W && mb < prm.tiles_m) {
            const volatile double* rv = red_t;
            double x = rv[lane];
            for (int w = 1; w < kEpiWarps; ++w)
              x = (MODE == kModeProx && lane == kPKkt) ? fmax(x, rv[w * 8 + lane]) : x + rv[w * 8 + lane];
            const int bad_slot = (MODE == kModeProx) ? (int)kPBad : (int)kYBad;
            if (*abort_flag && lane == bad_slot) x += 1.0;
            part_b[((int64_t)mb * prm.tiles_n + nb) * W + lane] = x;
          }
          __syncwarp();
          if (lane == 0) tile_count[i & 1] = 0;
        }
      }
      // this warp's TMEM reads (and its share of the fold) are done: one
      // release per warp, on the leader
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive_cluster(ptx::map_to_cta(&tempty[acc], 0));
      if (*abort_flag) break;
      T = TN;
      b = bN;
      Tl = TlN;
      slot ^= 1;
    }
    // no copy of this warp may still be in flight when the CTA leaves
    if (pending) asm volatile("cp.async.wait_group 0;" ::: "memory");
  }

  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  // neither CTA leaves while its peer may still read its shared memory or
  // signal its barriers
  ptx::cluster_sync();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem_base, kTmemCols);
  }
}

// Shared-memory opt-in and the persistent grid size (CTA pairs that fit at
// once), set up once per device, mode and plane type.  Done outside any
// launch so that a stream capture records launches only.  Host threads that
// fit row blocks side by side call this at once: the lock orders the two
// statics.
template <int MODE, int PT>
cudaError_t configure_mode(int& max_pairs) {
  static std::mutex mu;
  static int configured = -1;
  static int pairs = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (configured != dev) {
    e = cudaFuncSetAttribute(tc_gemm_kernel<MODE, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2, 1, 1);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tc_gemm_kernel<MODE, PT>, &cfg) != cudaSuccess || n < 1) {
      (void)cudaGetLastError();
      int sms = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      n = sms / 2 > 0 ? sms / 2 : 1;
    }
    pairs = n;
    configured = dev;
  }
  max_pairs = pairs;
  return cudaSuccess;
}

template <int MODE, int PT>
cudaError_t launch_mode(const TcParams& prm, cudaStream_t st) {
  int max_pairs = 0;
  cudaError_t e = configure_mode<MODE, PT>(max_pairs);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (prm.max_pairs > 0 && prm.max_pairs < max_pairs) max_pairs = prm.max_pairs;
  const int64_t tiles_total = (int64_t)(prm.nprob > 1 ? prm.nprob : 1) * prm.ntiles_p;
  const int pairs = (int)std::min<int64_t>(tiles_total, max_pairs);
  cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
  return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<MODE, PT>, prm);
}

template <int PT>
int max_pairs_of(int mode) {
  int m = 0;
  switch (mode) {
    case kModeY: configure_mode<kModeY, PT>(m); break;
    case kModeProx: configure_mode<kModeProx, PT>(m); break;
    case kModeGrad: configure_mode<kModeGrad, PT>(m); break;
    default: configure_mode<kModeGram, PT>(m); break;
  }
  return m;
}

template <int PT>
cudaError_t prepare_type() {
  int m = 0;
  cudaError_t e = configure_mode<kModeY, PT>(m);
  if (e == cudaSuccess) e = configure_mode<kModeProx, PT>(m);
  if (e == cudaSuccess) e = configure_mode<kModeGrad, PT>(m);
  if (e == cudaSuccess) e = configure_mode<kModeGram, PT>(m);
  return e;
}

template <int PT>
cudaError_t launch_type(int mode, const TcParams& prm, cudaStream_t st) {
  switch (mode) {
    case kModeY: return launch_mode<kModeY, PT>(prm, st);
    case kModeProx: return launch_mode<kModeProx, PT>(prm, st);
    case kModeGrad: return launch_mode<kModeGrad, PT>(prm, st);
    case kModeGram: return launch_mode<kModeGram, PT>(prm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int tc_box_n() { return kBHalf; }

int tc_bk(int pt) { return pt == kPlaneTf32 ? kBK<kPlaneTf32> : kBK<kPlaneBf16>; }

int tc_max_pairs(int mode, int pt) {
  return pt == kPlaneTf32 ? max_pairs_of<kPlaneTf32>(mode) : max_pairs_of<kPlaneBf16>(mode);
}

cudaError_t tc_prepare() {
  cudaError_t e = prepare_type<kPlaneBf16>();
  if (e == cudaSuccess) e = prepare_type<kPlaneTf32>();
  return e;
}

int64_t tc_tiles(int64_t M, int64_t N) { return ((M + BM - 1) / BM) * ((N + kBN - 1) / kBN); }

void tc_shape(TcParams& prm, int64_t M, int64_t N, int64_t K, int pt) {
  const int bk = tc_bk(pt);
  prm.ptype = pt;
  prm.M = M;
  prm.N = N;
  prm.K = K;
  prm.num_kb = (int32_t)((K + bk - 1) / bk);
  prm.tiles_m = (int32_t)((M + BM - 1) / BM);
  prm.tiles_n = (int32_t)((N + kBN - 1) / kBN);
  prm.ntiles = prm.tiles_m * prm.tiles_n;
  prm.tiles_mp = (prm.tiles_m + 1) / 2;
  prm.ntiles_p = prm.tiles_mp * prm.tiles_n;
  // raster: groups of pair rows (256 rows each), N block by N block; wide
  // groups when there are many N blocks (the B tiles then stream, A tiles
  // stay in L2)
  prm.group_m = prm.tiles_n > 16 ? 32 : 4;
  prm.bn = kBN;
}

// Process-wide wait limit of the tensor-core kernels and the one-shot
// withholding of the timeout test (accord_test_wait_limit).
static std::atomic<uint64_t> g_wait_ns{ptx::kWaitTimeoutNs};
static std::atomic<int> g_withhold_next_prox{0};

void tc_set_wait_test(uint64_t wait_ns, int withhold_next_prox) {
  g_wait_ns.store(wait_ns > 0 ? wait_ns : ptx::kWaitTimeoutNs);
  g_withhold_next_prox.store(withhold_next_prox ? 1 : 0);
}

cudaError_t launch_tc_gemm(int mode, const TcParams& prm_in, cudaStream_t st) {
  if (prm_in.ntiles <= 0) return cudaSuccess;
  TcParams prm = prm_in;
  prm.wait_ns = g_wait_ns.load();
  prm.withhold_first = (mode == kModeProx && g_withhold_next_prox.exchange(0) != 0) ? 1 : 0;
  if (prm.ptype == kPlaneTf32) return launch_type<kPlaneTf32>(mode, prm, st);
  if (prm.ptype == kPlaneBf16) return launch_type<kPlaneBf16>(mode, prm, st);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ tensor maps --
bool encode_plane_map(CUtensorMap* map, const void* base, int pt, int64_t rows, int64_t cols, int64_t ld,
                      int box_rows, int64_t depth, int64_t slice_stride) {
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
  if (pt != kPlaneBf16 && pt != kPlaneTf32) return false;
  const int64_t es = (int64_t)plane_bytes(pt);
  if (depth < 1) depth = 1;
  if (depth == 1 || slice_stride <= 0) slice_stride = rows * ld;
  if (((uintptr_t)base & 15u) != 0 || (ld * es) % 16 != 0 || (slice_stride * es) % 16 != 0 || rows < 1 ||
      cols < 1 || slice_stride < rows * ld)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)depth};
  const cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(slice_stride * es)};
  const cuuint32_t box[3] = {(cuuint32_t)tc_bk(pt), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = pt == kPlaneTf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = encode(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace accord
