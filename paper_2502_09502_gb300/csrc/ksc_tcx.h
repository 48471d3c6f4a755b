// ksc_tcx.h -- exact products of BF16 X with many FP64 vectors on the tensor
// cores (k_tcexact.cu): the anchors (X beta_ref, X^T r_ref) and the FP64
// certificates (X b^, X^T zeta; Sec. 3.4) of the batched solver.
//
//   D[list[r]][c] = sum_k A[c][k] V[list[r]][k]      (r < R, c < C)
//
// A is BF16 (X itself, c = row, or its column-major copy Xc, c = column of X).
// Fixed-point slicing (the error-free splitting of Ozaki, Ogita, Oishi and
// Rump, Numer. Algorithms 59, 2012): every row c of A is written as
// 2^(e_c - 7) sum_{t<3} xi_t 2^(-8t) with integers |xi_t| <= 255 and one
// exponent e_c per row (entries smaller than 2^(e_c - 16) leave an exact
// residual, kept in a sparse list and added in FP64 afterwards); every vector r
// as 2^(f_r - 7) sum_{s<6} sigma_s 2^(-8s) + tau with |tau| < 2^(f_r - 47).
// A slice product xi_t sigma_s is an integer below 2^16, so a K block of 64
// terms of the three pairs (t, s) with the same t + s sums below 2^24 and the
// tensor cores' FP32 accumulation of it is exact; the eight diagonals t + s of a
// block are drained from TMEM into 64-bit integer accumulators (exact), and the
// result is converted to FP64 once.  Error (rigorous, see tcx_error_factor):
//   |D - exact| <= eps ||A_c||_2 ||V_r||_2,
//   eps = 1.01 [sqrt(K) 2^-47 + 2^-54 (K / 64 + 1) + (4 + res_max) 2^-53].
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ksc {

constexpr int kTcxXSlices = 3;       // slices of A (24 bits below each row's top bit)
constexpr int kTcxVSlices = 6;       // slices of a vector (48 bits below its top bit)
constexpr int kTcxBN = 32;           // vectors per tile (TMEM columns per diagonal)
constexpr int kTcxMaxR = 1024;       // vectors per product

// the slices of one orientation of X (built once per problem)
struct TcxSlices {
  __nv_bfloat16* sl = nullptr;   // kTcxXSlices x Cpad x ld, row c of slice t at (t Cpad + c) ld
  int* ex = nullptr;             // Cpad row exponents
  int C = 0, Cpad = 0, K = 0;
  int64_t ld = 0;
  int* res_rows = nullptr;       // rows with residual entries (nrr of them)
  int* res_ptr = nullptr;        // nrr + 1 offsets into res_k / res_v
  int* res_k = nullptr;
  double* res_v = nullptr;
  int nrr = 0, nres = 0, res_max = 0;
  alignas(64) unsigned char tm[128];   // tensor map of sl (box 64 x 128)
  size_t bytes = 0;
  bool ok = false;
};

// the slices of up to Rcap vectors of length K and the split partials (per
// workspace and orientation)
struct TcxVecs {
  __nv_bfloat16* sl = nullptr;   // kTcxVSlices x Npad x ld
  int* ev = nullptr;             // Npad vector exponents
  long long* part = nullptr;     // split partials: (hi, lo) pairs
  size_t part_pairs = 0;
  int Rcap = 0, Npad = 0, K = 0;
  int64_t ld = 0;
  alignas(64) unsigned char tm[128];   // tensor map of sl (box 64 x kTcxBN)
  size_t bytes = 0;
  bool ok = false;
};

// Build the slices of A (BF16, C x K, row stride lda elements, device).  Allocates;
// synchronises stream s once (the residual count).  false with *why on failure.
bool tcx_slices_build(TcxSlices* x, const void* A, int C, int K, int64_t lda, cudaStream_t s, const char** why);
void tcx_slices_free(TcxSlices* x);
// Allocate the vector slices for up to Rcap vectors of length K.
bool tcx_vecs_alloc(TcxVecs* v, int Rcap, int K, const char** why);
void tcx_vecs_free(TcxVecs* v);
// Enqueue D[list[r]][c] = sum_k A[c][k] V[list[r]][k] (r < R <= Rcap; list NULL:
// the identity), V rows of length K with stride ldv (device), D rows with stride
// ldd (device, written for c < C).  Asynchronous on s; no allocation.
void tcx_product(const TcxSlices& x, TcxVecs& v, const double* V, int64_t ldv, const int* list, int R, double* D,
                 int64_t ldd, cudaStream_t s);
// eps of the error bound above for this orientation
double tcx_error_factor(const TcxSlices& x);
// kernel launches one tcx_product issues for R vectors
int tcx_launches(const TcxSlices& x, int R);
// device error word of the exact products (nonzero: a wait gave up); reset by tcx_clear_error
int* tcx_error_word();
void tcx_clear_error(cudaStream_t s);

}  // namespace ksc
