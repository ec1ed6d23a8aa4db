// Dense linear algebra of librihf (linalg.cu).  Every FP64 kernel spreads its
// work over all SMs: a GB300 SM retires only ~2 DFMA per clock, so tile sizes
// are small and skinny products are split along K.
#pragma once
#include "common.cuh"
#include "tc_gemm_buf.cuh"

namespace rihf {

struct LaCtx {
  cudaStream_t stream = 0;
  double* work = nullptr;       // split-K workspace
  size_t work_elems = 0;
  long long* launches = nullptr;
  int sms = 152;
  int* flag = nullptr;          // device error flag (non-positive pivot, ...)
  int* sched = nullptr;         // two ints, zero between launches: work counter of the tensor-core GEMM
  // Optional: digit-plane scratch for the two operands.  When set, dgemm runs
  // unbatched products with beta 0 or 1 and at least tc_min_work M N K on the
  // tensor cores with 7 BF16 digits (FP64-class: 55 bits of each row's and
  // column's largest element), as long as K fits one exponent block and the
  // operands fit the scratch; everything else stays FP64 DFMA.
  const OzBuf* tcA = nullptr;
  const OzBuf* tcB = nullptr;
  double tc_min_work = 0.0;
};

// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b] for b < batch.
// op(A) is M x K: A[m*lda + k] (transA = false) or A[k*lda + m] (true);
// op(B) is K x N: B[k*ldb + n] (transB = false) or B[n*ldb + k] (true).
// reduce_batch: all batches accumulate into C[0] (C stride ignored).
// lowerA: A is lower triangular (op(A)[m][k] = 0 for k > m), K-loop is cut.
// symcols: > 0 skips column tiles whose every column j has (j % symcols) > (j / symcols)
//          (strict upper triangle of an N x N slice flattened along columns).
struct GemmArgs {
  int M = 0, N = 0, K = 0;
  double alpha = 1.0, beta = 0.0;
  const double* A = nullptr;
  int lda = 0;
  long long sA = 0;
  bool transA = false;
  const double* B = nullptr;
  int ldb = 0;
  long long sB = 0;
  bool transB = false;
  double* C = nullptr;
  int ldc = 0;
  long long sC = 0;
  int batch = 1;
  bool reduce_batch = false;
  bool lowerA = false;
  int symcols = 0;
  bool lower_only = false;   // symmetric result: compute tiles on/below the diagonal only
};
void dgemm(const LaCtx& la, const GemmArgs& g);

// FP32 operands, FP32 accumulation (CUDA cores, 64 x 64 tiles).  Same
// conventions as GemmArgs; when Cd is set the result goes to the FP64 matrix Cd
// (alpha * sum + beta * Cd, split partial sums added in FP64), else to C (FP32).
struct SGemmArgs {
  int M = 0, N = 0, K = 0;
  double alpha = 1.0, beta = 0.0;
  const float* A = nullptr;
  int lda = 0;
  long long sA = 0;
  bool transA = false;
  const float* B = nullptr;
  int ldb = 0;
  long long sB = 0;
  bool transB = false;
  float* C = nullptr;
  double* Cd = nullptr;
  int ldc = 0;
  long long sC = 0;
  int batch = 1;
  bool reduce_batch = false;
};
void sgemm(const LaCtx& la, const SGemmArgs& g);
// out[i] = (float) in[i]
void to_float(const LaCtx& la, const double* in, long long n, float* out, double scale = 1.0);

// Mirror the lower triangle into the upper one for each of `batch` n x n slices.
void symmetrize_lower(const LaCtx& la, double* X, int n, int batch);

// Forward substitution X <- L^{-1} X (as trsm_lower with trans = false) in two
// levels: inside each kTrsmOuter-row panel, 64-row panels solved in FP64 with
// rank-64 updates of the panel's rows below them; then one rank-kTrsmOuter
// update of all rows below the outer panel.  The updates run on the tensor
// cores as 7-digit BF16 digit-plane GEMMs (FP64-class products, tc_gemm.cuh);
// the outer ones touch the rows below once per 256 rows of L instead of once
// per 64.  Scratch: oz_buf_alloc(n, kTrsmOuter, 7, 1) for L and
// oz_buf_alloc(ncol, kTrsmOuter, 7, 1) for a panel of X.
constexpr int kTrsmPanel = 64;
constexpr int kTrsmOuter = 256;
struct TrsmTcScratch {
  OzBuf L, X;   // kTrsmPanel-column slices of L (n rows) and of the X panel (ncol rows)
};
void trsm_lower_tc(const LaCtx& la, const double* L, int n, double* X, long long ncol, int symcols,
                   const TrsmTcScratch& sc);
// Backward substitution X <- L^{-T} X (as trsm_lower with trans = true), blocked
// the same way from the bottom: the updates of the rows above a panel,
// X[0:k] -= L[k:k+b, 0:k]^T X[k:k+b], run as 7-digit tensor-core GEMMs.
void trsm_lower_t_tc(const LaCtx& la, const double* L, int n, double* X, long long ncol, int symcols,
                     const TrsmTcScratch& sc);

// In-place Cholesky A = L L^T (lower, upper part zeroed) of an n x n matrix;
// sets *flag = 1 on a non-positive pivot.  scratch holds n x 32 doubles.
void cholesky(const LaCtx& la, double* A, int n, double* scratch);

// Blocked triangular solve in place: X <- L^{-1} X (trans = false, forward) or
// X <- L^{-T} X (trans = true, backward), L lower n x n, X n x ncol row-major
// (leading dimension ncol).  Diagonal 32 x 32 blocks are inverted by one warp,
// the off-diagonal updates are FP64 GEMMs over all SMs.  symcols as in GemmArgs.
// tmp must hold 32 * ncol + 32 * 32 doubles.
void trsm_lower(const LaCtx& la, const double* L, int n, double* X, long long ncol, bool trans, int symcols,
                double* tmp);

// Symmetric eigen-decomposition of an n x n FP64 matrix A (row-major):
// W (n, ascending) and V (n x n, column k = eigenvector k).  FP32 parallel
// Jacobi (one CTA up to kBlockJacobiMin, a two-sided block Jacobi over many
// CTAs above), then Ogita-Aishima refinement in FP64 (`refine` steps).
// ws must hold eig_workspace(n) doubles: the FP32 Jacobi copies (A, V, W;
// even order m), then six n x n FP64 refinement matrices and 2n + 8 scalars;
// above kBlockJacobiMin, also the parallel block Jacobi's FP32 matrices (order
// n rounded up to a multiple of 32), rotations and reduction partials.
constexpr int kBlockJacobiMin = 256;
constexpr size_t eig_workspace_base(int n) {
  return ((size_t)(n + (n & 1)) * (n + (n & 1)) + (size_t)n * (n + (n & 1)) + (n + (n & 1)) + 1) / 2 +
         6 * (size_t)n * n + 2 * (size_t)n + 8;
}
constexpr size_t eig_workspace_bj(int n) {   // FP64 matrices, rotations, partials, flag (the FP32 stage fits)
  return n <= kBlockJacobiMin ? 0
                              : 2 * (size_t)((n + 31) / 32 * 32) * ((n + 31) / 32 * 32) +
                                    (size_t)((n + 31) / 32) * 32 * 32 + 2 * 256 + 16;
}
constexpr size_t eig_workspace(int n) { return eig_workspace_base(n) + eig_workspace_bj(n); }
// skip_jacobi: start the refinement from Vguess directly (late SCF iterations).
// max_sweeps caps the FP32 Jacobi sweeps and ns_steps the Newton-Schulz
// re-orthonormalisation steps after the refinement (early SCF iterations need
// the eigenvectors only to the accuracy of the SCF itself).
void eigh(const LaCtx& la, const double* A, int n, double* W, double* V, double* ws, int refine,
          const double* Vguess, bool skip_jacobi = false, int max_sweeps = 20, int ns_steps = 2);

// Elementwise / reductions.
void axpby(const LaCtx& la, int n, double a, const double* x, double b, const double* y, double* out);
void add3(const LaCtx& la, int n, const double* x, const double* y, const double* z, double* out);
// out[0] = sum x*y (deterministic two-level reduction)
void dot(const LaCtx& la, int n, const double* x, const double* y, double* out);
void scale_copy(const LaCtx& la, int n, double a, const double* x, double* out);
// C = A - A^T for square n x n
void antisym(const LaCtx& la, const double* A, double* C, int n);
// Copy columns [0, ncol) of an n_rows x ld matrix into a dense n_rows x ncol one, times s.
void copy_cols(const LaCtx& la, const double* src, int nrows, int ld, int ncol, double s, double* dst);
// Y = diag(v) scaling of columns: out[i][j] = X[i][j] * v[j]
void scale_cols(const LaCtx& la, const double* X, const double* v, int nrows, int ncol, double* out);
// dst (cols x rows) = src^T for a rows x cols matrix.
void transpose(const LaCtx& la, const double* src, int rows, int cols, double* dst);
// Fill dst with the identity (n x n).
void identity(const LaCtx& la, double* dst, int n);

}  // namespace rihf
