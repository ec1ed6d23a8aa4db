// RI-J / RI-K contraction kernels (jk.cu): the HBM-streaming passes over the
// fitted tensor B (Eq. j_ri) and helpers of the gradient's Y formation.
#pragma once
#include "common.cuh"
#include "linalg.cuh"

namespace rihf {

// y[r] = alpha * sum_j A[r*K + j] x[j], r < M (one CTA per row, coalesced).
void gemv_rows(const LaCtx& la, const double* A, int M, long long K, const double* x, double alpha, double* y);
// y[j] = alpha * sum_r x[r] A[r*K + j], j < K (row chunks reduced deterministically).
void gemv_cols(const LaCtx& la, const double* A, int M, long long K, const double* x, double alpha, double* y);
// Symmetric slices: A holds M rows of N x N matrices that are symmetric in
// their two indices, and x (rows pass) / y (columns pass) are symmetric N x N.
// Both passes read only each slice's lower triangle (half of the bytes):
// y[r] = alpha * sum_{mu >= nu} w_{mu nu} A[r][mu][nu] x[mu][nu] with w = 2 off the
// diagonal, and y[mu][nu] = y[nu][mu] = alpha * sum_r x[r] A[r][mu][nu].
void gemv_rows_sym(const LaCtx& la, const double* A, int M, int N, const double* x, double alpha, double* y);
void gemv_cols_sym(const LaCtx& la, const double* A, int M, int N, const double* x, double alpha, double* y);
// FP32 operand versions (mixed-precision SCF iterations): products and
// per-thread partial sums in FP32, cross-thread sums and outputs in FP64.
void gemv_rows_f32(const LaCtx& la, const float* A, int M, long long K, const float* x, double alpha, double* y);
void gemv_cols_f32(const LaCtx& la, const float* A, int M, long long K, const double* x, double alpha, double* y);
// Y[P][e] = c[P] * D[e] for e < n2, P < naux.
void outer_fill(const LaCtx& la, const double* c, int naux, const double* D, long long n2, double* Y);

// Pair-packed symmetric storage: element (mu, nu) of an N x N symmetric
// matrix at tri(max) + min, tri(i) = i (i + 1) / 2; N (N + 1) / 2 entries.
__host__ __device__ inline long long tri_index(int mu, int nu) {
  const long long a = mu > nu ? mu : nu, b = mu > nu ? nu : mu;
  return a * (a + 1) / 2 + b;
}
// Ap = packed A with the off-diagonal entries times w (w = 2 turns a packed
// dot product into the full symmetric one).
void pack_sym(const LaCtx& la, const double* A, int N, double w, double* Ap);
// A (N x N) from packed Ap, both triangles.
void unpack_sym(const LaCtx& la, const double* Ap, int N, double* A);
// nmat matrices: A[m][mu][nu] = Ap[m * ldp + tri_index(mu, nu)], and back
// (pack_sym_batch reads the lower triangle of each A[m]).
void unpack_sym_batch(const LaCtx& la, const double* Ap, int nmat, int N, long long ldp, double* A);
void pack_sym_batch(const LaCtx& la, const double* A, int nmat, int N, double* Ap, long long ldp);

}  // namespace rihf
