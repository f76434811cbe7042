// Parameters of the tcgen05 split-operand GEMM C = A * B^T (A: M x K,
// B: N x K, hi/lo planes of BF16 or TF32, K contiguous) and its host launcher.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace accord {

// Operand planes are 3-D tensor maps (K, rows, slice): the slice is the
// problem of a batch (a lambda path runs one problem per chain), 0 for a
// single fit.
struct TcParams {
  CUtensorMap a_hi[2];  // A planes, index (a_nxt ? nxt : cur)
  CUtensorMap a_lo[2];
  CUtensorMap b_hi;     // B planes
  CUtensorMap b_lo;
  Ctrl* ctrl;           // null: cur = 0, no early exit; a batch: one per problem
  int* err;             // device error word (kErr* bits), never null
  int64_t M, N, K;
  int32_t num_kb, tiles_m, tiles_n, ntiles;  // 128-row M blocks, 256-column N blocks
  int32_t tiles_mp, ntiles_p;                 // pair rows (256 rows), pair tiles per problem
  int32_t a_nxt, smooth, group_m, bn;
  float* out[2];        // FP32 output (Y+, Omega+ or G), index nxt
  int64_t ldout;
  void* out_hi[2];      // operand planes of the output (type ptype), index nxt
  void* out_lo[2];
  int64_t ldplane;
  const float* aux[2];  // old Y (Y mode) or Omega (prox / grad), index cur
  int64_t ldaux;
  double* out64;        // FP64 output (Gram)
  int64_t ldout64;
  double* part;         // per-tile partial sums or null
  float lam, lam_d, scale, pad;
  // Sparse Delta buckets (prox mode): when keys != null the epilogue records
  // the nonzero entries of Delta in the bucket of its 32-row group instead of
  // writing dense Delta planes; an overflow sets *dense_flag.
  uint32_t* keys;
  float* vals;
  int* counts;
  int* dense_flag;
  int32_t cap;
  int32_t gate_dense;   // 1: run only when ctrl->dense is set (dense fallback)
  // Eq. 3.8 refit: support bitmask (bit (i, j) of word [i][j / 32]), or null
  const uint32_t* mask;
  int64_t mask_ld;
  // Batch of problems with the same M and N.  Tile index -> (problem, tile);
  // problem b uses ctrl[b] (its cur, tau, lambda and 1/n), outputs at
  // + b * s_out ..., and skips every tile once ctrl[b].done is set (or, with
  // gate_dense, while ctrl[b].dense is clear).
  int32_t nprob;             // problems (1: a single fit)
  int32_t b_batched;         // B planes: slice b (1) or slice 0 for all (0)
  const int32_t* active;     // device list of the problems to run, or null (0 .. nprob-1)
  const int32_t* nactive;    // device length of `active`
  const int32_t* kb_of;      // device K blocks per problem (ragged K), or null (num_kb)
  int64_t s_out, s_aux, s_plane, s_part, s_bkt;  // strides: elements, elements, elements, tiles, buckets
  // Batch: a prox epilogue whose bucket overflows also sets *any_dense; a
  // gated launch returns at once while *any_dense is clear (no problem needs
  // the dense product), instead of scanning every problem's tiles.
  int* any_dense;
  int32_t coarse_ok;     // prox mode: form G with one product while ctrl[b].coarse is set
  int32_t max_pairs;     // persistent grid limit in CTA pairs (0: as many as fit at once)
  int32_t ptype;         // plane type of the operands and plane outputs: kPlaneBf16 / kPlaneTf32
  // Occupancy bitmaps of the two iterate buffers (prox mode): word
  // [c * ldbm + i] has bit j - 32 c set iff Omega[i][j] != 0 for the 32
  // columns j of chunk c; rows past p read as 0.  A buffer's values count
  // only where its bitmap has a bit (elsewhere the entry is 0, whatever the
  // buffer holds).  The prox epilogue fetches only the nonzero entries of
  // Omega, stores only the nonzero entries of Omega+, and writes the whole
  // bitmap of Omega+.  A batch keeps one pair per problem, s_bm words apart.
  uint32_t* bm[2];
  int64_t ldbm, s_bm;
  // Row block of Omega (prox / grad modes): output row r is row r + row_off
  // of the full matrix, so its diagonal entry sits in column r + row_off
  // (a multiple of 32, so that the diagonal crosses whole 32 x 32 blocks).
  int64_t row_off;
  // Bounded waits: every mbarrier wait of the launch gives up after wait_ns
  // (set from the process-wide limit, 4 s by default).  withhold_first: the
  // producers of both CTAs of the first pair skip the copies of their first
  // stage, so that the MMA issuer's first wait runs out (the test of the
  // timeout path; set only through accord_test_wait_limit).
  uint64_t wait_ns;
  int32_t withhold_first;
  int32_t pad2;
};

// Encodes a 3-D tensor map over `depth` slices of a rows x cols plane of type
// pt with leading dimension ld (elements) and slice_stride elements between
// slices; box (64 bytes of K) x box_rows x 1, 64-byte swizzle.  Returns false
// when the driver rejects the arguments.
bool encode_plane_map(CUtensorMap* map, const void* base, int pt, int64_t rows, int64_t cols, int64_t ld,
                      int box_rows, int64_t depth = 1, int64_t slice_stride = 0);

// K elements one pipeline stage covers (64 bytes of a plane row).
int tc_bk(int pt);
// Fills the shape fields (num_kb, tiles, bn) and the plane type pt of an
// M x N x K problem (the K blocking depends on pt).
void tc_shape(TcParams& prm, int64_t M, int64_t N, int64_t K, int pt);
int64_t tc_tiles(int64_t M, int64_t N);
int tc_box_n();  // rows of the B box a CTA loads (its half of the N tile)
cudaError_t launch_tc_gemm(int mode, const TcParams& prm, cudaStream_t st);
// Wait limit of every later tensor-core launch in the process (0: the default
// 4 s); withhold_next_prox = 1 makes the next prox GEMM launch skip its first
// stage's copies so that its first wait runs out (the timeout path's test).
void tc_set_wait_test(uint64_t wait_ns, int withhold_next_prox);
// One-time per-device setup of every mode (done lazily by the first launch
// otherwise); call before capturing launches into a CUDA graph.
cudaError_t tc_prepare();
// CTA pairs of the persistent grid that fit on the device at once (mode's kernel).
int tc_max_pairs(int mode, int pt = 0);

}  // namespace accord
