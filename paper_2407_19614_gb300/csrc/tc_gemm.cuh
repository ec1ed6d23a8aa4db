// Tensor-core GEMM with FP64-class accuracy from BF16 digit planes (tc_gemm.cu).
//
// Each FP64 operand row is written, per block of K, as a fixed-point number
// relative to the block's largest exponent and split into s balanced 8-bit
// digits d_t in [-128, 128] (t = 1..s, weights 2^{48-8(t-1)} on a 2^-55 grid).
// Every digit is exact in BF16.  A product of rows is the sum over digit pairs
// (t, u) of exact integer dot products; pairs on one anti-diagonal g = t + u
// share a weight and accumulate in one FP32 TMEM accumulator, exactly, as long
// as |sum| <= s * K' * 128^2 <= 2^24 over the K' elements accumulated between
// read-outs (K' = 128 for s = 7).  Pairs with t + u > s + 1 are dropped (their
// weight is below 2^{-8s} of the leading term).  Every K' elements the s
// accumulators are read back (tcgen05.ld) and folded into one int64
// fixed-point sum per output element; the final FP64 value is built from the
// integer and the two block exponents.
//
// s = 7 keeps 55 bits relative to max|row| * max|col| of each K block;
// fewer digits trade accuracy for tensor work (s (s + 1) / 2 digit products
// per output tile and K step).  The products of one A digit plane with all
// the B planes it pairs with run as one MMA (or a few, N <= 256): the B planes
// are adjacent in shared memory and form a single operand whose output
// columns fall on the anti-diagonals, so a K step costs about s MMA
// instructions instead of s (s + 1) / 2 small ones.
#pragma once
#include <cstdint>

#include "common.cuh"
#include "linalg.cuh"
#include "tc_gemm_buf.cuh"

namespace rihf {

// Digit planes of one operand.  Layout: for row tile rt (128 rows), K chunk c
// and digit t, a 128 x kOzChunk BF16 block in the no-swizzle K-major
// core-matrix order: element (r, k) at ((r / 8) * (kOzChunk / 8) + k / 8) * 64
// + (r % 8) * 8 + k % 8.
// Block index ((rt * kchunks + c) * smax + t).  exps[r * nkb + kb] is the
// largest biased FP64 exponent in row r over K block kb (0 if all zero).
struct OzOperand {
  const uint16_t* planes = nullptr;
  const int* exps = nullptr;
  int rows = 0, rows_pad = 0;
  int kchunks = 0;
  int smax = 0;
  int nkb = 1, kb_chunks = 0;
};

// Slice X (rows x K, element (r, k) at X[r*s_r + (k % KR)*s_k1 + (k / KR)*s_k2],
// or, with RR > 0, at X[(r % RR)*s_r + (r / RR)*s_r2 + ...]) into smax digit
// planes; K blocks of kb_chunks chunks get their own exponent.  With
// packed_n > 0 the source is pair-packed symmetric packed_n x packed_n
// matrices s_r2 apart: row r is row r % packed_n of matrix r / packed_n, and
// K = packed_n (s_r, s_k1, s_k2, KR and RR unused).  Needs
// oz_plane_elems(rows, K, smax) plane and rows_pad * nkb exponent entries in buf
// (RIHF_ERR_INVALID_ARG otherwise).
OzOperand oz_slice(const LaCtx& la, const double* X, int rows, int K, long long s_r, long long s_k1,
                   long long s_k2, int KR, int smax, int kb_chunks, const OzBuf& buf, int RR = 0,
                   long long s_r2 = 0, int packed_n = 0);

// C(m, n) = alpha * sum_k A(m, k) B(n, k) using s <= min(A.smax, B.smax) digits.
// Output element (m, n) at C[(m % MR) * cs_m1 + (m / MR) * cs_m2 + n * cs_n];
// atomic: added with atomicAdd (C must be initialised); accumulate: C += (one
// writer per element: a single K block); else stored.
// lower_only: only tiles that meet m >= n are computed (symmetric results).
// symcols > 0: column tiles whose every column n has (n % symcols) > (n / symcols)
// (strict upper triangle of a symcols x symcols slice flattened along n) are skipped.
// All CTAs of a K split must share one exponent block: A.kb_chunks == B.kb_chunks
// and the kernel runs one split per exponent block.  Sets la.flag[1] = 1 if a
// bounded wait on the tensor core or the copy engine ran out (la.flag must
// point to at least two ints; la.sched to two zeroed ints owned by the stream).
struct OzGemmArgs {
  OzOperand A, B;
  int M = 0, N = 0;
  int s = kOzMaxDigits;
  double alpha = 1.0;
  double* C = nullptr;
  long long MR = 1LL << 62;
  long long cs_m1 = 0, cs_m2 = 0, cs_n = 1;
  bool atomic = false;
  bool accumulate = false;
  bool lower_only = false;
  int symcols = 0;
  // column tile TN: 0 picks the whole of N when N <= kOzMaxTN, else kOzMaxTN;
  // otherwise a multiple of 16 that is at most kOzMaxTN and, when N > tn,
  // divides 128 (a column tile never straddles a 128-row plane)
  int tn = 0;
};
void oz_gemm(const LaCtx& la, const OzGemmArgs& g);

// Number of BF16 MMA products per output tile and chunk for s digits.
inline int oz_products(int s) { return s * (s + 1) / 2; }

}  // namespace rihf
