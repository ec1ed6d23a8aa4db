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

}  // namespace rihf
