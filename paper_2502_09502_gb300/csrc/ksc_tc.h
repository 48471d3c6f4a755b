// ksc_tc.h -- the tensor-core product of the batched solver (k_tcgemm.cu).
//
//   D[m][j] = sum_{q < P} sum_k A_q[m][k] * B[j][k]        (FP32 accumulation)
//
// A_q and B are BF16, K contiguous ("K-major"); A holds P pieces of the same
// M x K matrix stacked as rows [q * Mpad, q * Mpad + M).  The batched FISTA step
// (Algorithm 3 over many nodes) puts the nodes in M: A = the split iterates
// (X beta for all nodes, B = X) or the split residuals (X^T r, B = the column-major
// copy of X).  A vector split into P BF16 pieces whose sum is exact (P = 3 holds
// any FP32 value) accumulates all pieces into one FP32 accumulator, so the product
// is that of the FP32 vector up to the FP32 accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ksc.h"

namespace ksc {

enum : int { kTcStore = 0, kTcAdd = 1, kTcAnchor = 2 };

// E4M3 operands (plan e8 = 1): B is E4M3 X (its power-of-two column scales kept
// apart), A holds kTcE4m3Pieces E4M3 pieces of the vectors, each row scaled by a
// power of two so that its largest entry lies in [128, 256): pieces 0..2 are the
// E4M3 roundings of what the previous ones left, pieces 3..4 those of the
// remainder times 2^kTcE4m3Shift, accumulated in a second TMEM accumulator (the
// epilogue adds hi + 2^-12 lo).  One scale for all pieces would stop every entry
// at the smallest E4M3 subnormal, 2^-18 of the row's largest; the second scale
// takes that floor to 2^-30, below the FP32 accumulation error.  The epilogue
// multiplies row m by rscale[m] (the inverse scale) and, when cscale is given,
// column j by cscale[j] -- both exact in FP32.  Tiles are at most 128 wide (two
// double-buffered accumulators fill the 512 TMEM columns).
constexpr int kTcE4m3Pieces = KSC_E4M3_PIECES;
constexpr int kTcE4m3Hi = 3;       // pieces in the first accumulator
constexpr int kTcE4m3Shift = 12;   // the remainder's scale, 2^12

// Epilogues (row m of the product D, columns j < N):
//   kTcStore   out[m * ldo + j] = D                                   (FP32)
//   kTcAdd     out64[m * ldo + j] = base[m * ldb + j] + D             (FP64)
//   kTcAnchor  u_new = base[m * ldb + j] + D in FP64, written to
//              u64 + m * ldo + slot_out[m] * slot_stride; with u_old read at
//              u64 + m * ldo + slot_in[m] * slot_stride, per row and per 64
//              columns the sums of the loss terms F_j(u_new) (least squares
//              (u - y_j)^2, logistic log(1 + e^{-y_j u})) and of their changes
//              F_j(u_new) - F_j(u_old), evaluated without cancellation, go to
//              part[2 * (m * npart + j / 64) + {0, 1}]  (npart >= ceil(N / 64)).
// The batched solver multiplies differences from an anchor (beta - beta_ref,
// r - r_ref) and adds the anchor's exact product here, so the FP32 accumulation
// error is relative to the difference.
struct TcEpi {
  float* out;
  int64_t ldo;
  const double* base;
  int64_t ldb;
  double* out64;
  double* u64;
  const int* slot_in;
  const int* slot_out;
  int64_t slot_stride;
  const float* y;
  int loss;
  int npart;
  double* part;
  const int* tile_active;   // per 128-row M tile: 0 = every row finished, skip the tile (NULL: none)
  const float* rscale;      // E4M3 plans: per row m, the inverse of its pieces' scale (NULL: 1)
  const float* cscale;      // E4M3 plans: per column j of D (NULL: 1)
  float* skws;              // stream-K partial tiles: 2 * grid * 128 * BN floats (stream-K plans only)
};

struct TcPlan {
  alignas(64) unsigned char tmA[128];   // CUtensorMap of the stacked A pieces
  alignas(64) unsigned char tmB[128];   // CUtensorMap of B
  int P, M, Mpad, N, K, bn;
  int e8;      // 1: E4M3 operands (kind::f8f6f4), K blocks of 128
  int ok;
  int sk;      // 1: stream-K schedule over `grid` persistent CTAs (M <= 1024)
  int grid;
};

// Stream-K schedule (tc_plan_stream_k): the active 128 x BN tiles times their
// K blocks of 128 bytes form one iteration space, split evenly over `grid` CTAs (one per
// SM).  A CTA runs its range tile by tile with a double-buffered TMEM accumulator,
// so the epilogue of one tile overlaps the products of the next; a tile whose
// K blocks span several CTAs leaves FP32 partial tiles in skws, summed in CTA
// order by a second kernel that applies the epilogue.  Every tile of a launch is
// then processed once and every SM works until the end of the launch.
bool tc_plan_stream_k(TcPlan* plan, int grid, const char** why);
size_t tc_skws_floats(int grid, int bn);

// tile widths (columns of B per CTA) the kernel is built for
constexpr int kTcBNs[3] = {64, 128, 256};

// Build the tensor maps.  A: device BF16 (e8: E4M3), (P * Mpad) x lda elements,
// the row stride in bytes a multiple of 16, Mpad (the row stride of the pieces) a
// multiple of 128; rows M .. round_up(M, 128) - 1 of each piece are read (and must
// be finite) but not stored.  B: device BF16 (e8: E4M3), N x ldb.  Returns false
// (with a message in *why) when the shapes or the driver refuse.
bool tc_plan(TcPlan* plan, const void* A, int P, int M, int Mpad, int K, int64_t lda, const void* B,
             int N, int64_t ldb, int bn, const char** why, int e8 = 0);
// enqueue one product; mode kTcStore, kTcAdd or kTcAnchor
void tc_launch(const TcPlan& plan, const TcEpi& epi, int mode, cudaStream_t s);
// device error word of the product kernels (nonzero: a wait gave up); reset by tc_clear_error
int* tc_error_word();
void tc_clear_error(cudaStream_t s);

}  // namespace ksc
