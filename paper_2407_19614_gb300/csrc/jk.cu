// RI-J contraction passes over B (Eq. j_ri: d_P = sum B^P_{mu nu} D_{mu nu},
// J = sum_P d_P B^P) and small helpers.  Both passes stream B once from HBM with
// coalesced loads; the row pass gives each auxiliary index its own CTA, the
// column pass splits the auxiliary range and reduces the partial sums in a
// fixed order.
#include <algorithm>

#include "jk.cuh"

namespace rihf {

__global__ void __launch_bounds__(256) gemv_rows_kernel(const double* __restrict__ A, int M, long long K,
                                                        const double* __restrict__ x, double alpha, double* y) {
  __shared__ double red[8];
  for (int r = blockIdx.x; r < M; r += gridDim.x) {
    const double* row = A + (long long)r * K;
    double s = 0.0;
    for (long long j = threadIdx.x; j < K; j += 256) s = fma(row[j], x[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      y[r] = alpha * t;
    }
    __syncthreads();
  }
}

void gemv_rows(const LaCtx& la, const double* A, int M, long long K, const double* x, double alpha, double* y) {
  int blocks = std::min(M, 16 * la.sms);
  gemv_rows_kernel<<<blocks, 256, 0, la.stream>>>(A, M, K, x, alpha, y);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

__global__ void __launch_bounds__(256) gemv_cols_kernel(const double* __restrict__ A, int M, long long K,
                                                        const double* __restrict__ x, int rows_per,
                                                        double* __restrict__ part) {
  long long j = blockIdx.x * 256LL + threadIdx.x;
  int r0 = blockIdx.y * rows_per, r1 = min(M, r0 + rows_per);
  if (j >= K) return;
  double s = 0.0;
  for (int r = r0; r < r1; ++r) s = fma(x[r], A[(long long)r * K + j], s);
  part[(long long)blockIdx.y * K + j] = s;
}

__global__ void cols_reduce_kernel(const double* __restrict__ part, int nchunk, long long K, double alpha,
                                   double* y) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < K; j += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * K + j];
    y[j] = alpha * s;
  }
}

void gemv_cols(const LaCtx& la, const double* A, int M, long long K, const double* x, double alpha, double* y) {
  long long colblocks = (K + 255) / 256;
  int nchunk = (int)std::max<long long>(1, std::min<long long>(M, (8LL * la.sms + colblocks - 1) / colblocks));
  while (nchunk > 1 && (size_t)nchunk * K > la.work_elems) nchunk /= 2;
  int rows_per = ceil_div(M, nchunk);
  nchunk = ceil_div(M, rows_per);
  gemv_cols_kernel<<<dim3((unsigned)colblocks, nchunk), 256, 0, la.stream>>>(A, M, K, x, rows_per, la.work);
  RIHF_LAUNCH_CHECK();
  int blocks = (int)std::min<long long>((K + 255) / 256, 8LL * la.sms);
  cols_reduce_kernel<<<blocks, 256, 0, la.stream>>>(la.work, nchunk, K, alpha, y);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 2;
}

// One CTA per slice r; warp w takes rows mu = w, w + 8, ..., lanes the columns
// nu <= mu of the row (fixed order per thread and a fixed reduction tree).
__global__ void __launch_bounds__(256) gemv_rows_sym_kernel(const double* __restrict__ A, int M, int N,
                                                            const double* __restrict__ x, double alpha, double* y) {
  __shared__ double red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n2 = (long long)N * N;
  for (int r = blockIdx.x; r < M; r += gridDim.x) {
    const double* slice = A + (long long)r * n2;
    double s = 0.0, t = 0.0;   // strictly lower part, diagonal (one FP64 FMA per element)
    for (int mu = warp; mu < N; mu += 8) {
      const double* row = slice + (long long)mu * N;
      const double* xr = x + (long long)mu * N;
      for (int nu = lane; nu < mu; nu += 32) s = fma(row[nu], xr[nu], s);
      if (lane == (mu & 31)) t = fma(row[mu], xr[mu], t);
    }
    s = 2.0 * s + t;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      y[r] = alpha * t;
    }
    __syncthreads();
  }
}

void gemv_rows_sym(const LaCtx& la, const double* A, int M, int N, const double* x, double alpha, double* y) {
  int blocks = std::min(M, 16 * la.sms);
  gemv_rows_sym_kernel<<<blocks, 256, 0, la.stream>>>(A, M, N, x, alpha, y);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

// Thread per element j = mu N + nu of the flattened slice; the upper triangle
// (nu > mu) is neither read nor written until the reduction mirrors it.
__global__ void __launch_bounds__(256) gemv_cols_sym_kernel(const double* __restrict__ A, int M, int N,
                                                            const double* __restrict__ x, int rows_per,
                                                            double* __restrict__ part) {
  const long long n2 = (long long)N * N;
  const long long j = blockIdx.x * 256LL + threadIdx.x;
  if (j >= n2) return;
  const int mu = (int)(j / N), nu = (int)(j - (long long)mu * N);
  if (nu > mu) return;
  int r0 = blockIdx.y * rows_per, r1 = min(M, r0 + rows_per);
  double s = 0.0;
  for (int r = r0; r < r1; ++r) s = fma(x[r], A[(long long)r * n2 + j], s);
  part[(long long)blockIdx.y * n2 + j] = s;
}

__global__ void cols_reduce_sym_kernel(const double* __restrict__ part, int nchunk, int N, double alpha, double* y) {
  const long long n2 = (long long)N * N;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n2; j += (long long)gridDim.x * blockDim.x) {
    const int mu = (int)(j / N), nu = (int)(j - (long long)mu * N);
    if (nu > mu) continue;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * n2 + j];
    y[j] = alpha * s;
    y[(long long)nu * N + mu] = alpha * s;
  }
}

void gemv_cols_sym(const LaCtx& la, const double* A, int M, int N, const double* x, double alpha, double* y) {
  const long long n2 = (long long)N * N;
  long long colblocks = (n2 + 255) / 256;
  // about half the column blocks do work: twice the row chunks of the full pass
  int nchunk = (int)std::max<long long>(1, std::min<long long>(M, (16LL * la.sms + colblocks - 1) / colblocks));
  while (nchunk > 1 && (size_t)nchunk * n2 > la.work_elems) nchunk /= 2;
  int rows_per = ceil_div(M, nchunk);
  nchunk = ceil_div(M, rows_per);
  gemv_cols_sym_kernel<<<dim3((unsigned)colblocks, nchunk), 256, 0, la.stream>>>(A, M, N, x, rows_per, la.work);
  RIHF_LAUNCH_CHECK();
  int blocks = (int)std::min<long long>((n2 + 255) / 256, 8LL * la.sms);
  cols_reduce_sym_kernel<<<blocks, 256, 0, la.stream>>>(la.work, nchunk, N, alpha, y);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 2;
}

__global__ void __launch_bounds__(256) gemv_rows_f32_kernel(const float* __restrict__ A, int M, long long K,
                                                            const float* __restrict__ x, double alpha, double* y) {
  __shared__ double red[8];
  for (int r = blockIdx.x; r < M; r += gridDim.x) {
    const float4* row = reinterpret_cast<const float4*>(A + (long long)r * K);
    const float4* xv = reinterpret_cast<const float4*>(x);
    float s = 0.f;
    long long K4 = K / 4;
    for (long long j = threadIdx.x; j < K4; j += 256) {
      float4 a = row[j], b = xv[j];
      s = fmaf(a.x, b.x, s); s = fmaf(a.y, b.y, s); s = fmaf(a.z, b.z, s); s = fmaf(a.w, b.w, s);
    }
    for (long long j = 4 * K4 + threadIdx.x; j < K; j += 256) s = fmaf(A[(long long)r * K + j], x[j], s);
    double d = s;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      y[r] = alpha * t;
    }
    __syncthreads();
  }
}

void gemv_rows_f32(const LaCtx& la, const float* A, int M, long long K, const float* x, double alpha, double* y) {
  int blocks = std::min(M, 16 * la.sms);
  const bool aligned = (K % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                       ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
  if (!aligned) throw RihfError(-1, "gemv_rows_f32 needs 16-byte aligned rows");
  gemv_rows_f32_kernel<<<blocks, 256, 0, la.stream>>>(A, M, K, x, alpha, y);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

__global__ void __launch_bounds__(256) gemv_cols_f32_kernel(const float* __restrict__ A, int M, long long K,
                                                            const double* __restrict__ x, int rows_per,
                                                            double* __restrict__ part) {
  long long j = blockIdx.x * 256LL + threadIdx.x;
  int r0 = blockIdx.y * rows_per, r1 = min(M, r0 + rows_per);
  if (j >= K) return;
  float s = 0.f;
  for (int r = r0; r < r1; ++r) s = fmaf((float)x[r], A[(long long)r * K + j], s);
  part[(long long)blockIdx.y * K + j] = (double)s;
}

void gemv_cols_f32(const LaCtx& la, const float* A, int M, long long K, const double* x, double alpha, double* y) {
  long long colblocks = (K + 255) / 256;
  int nchunk = (int)std::max<long long>(1, std::min<long long>(M, (8LL * la.sms + colblocks - 1) / colblocks));
  while (nchunk > 1 && (size_t)nchunk * K > la.work_elems) nchunk /= 2;
  int rows_per = ceil_div(M, nchunk);
  nchunk = ceil_div(M, rows_per);
  gemv_cols_f32_kernel<<<dim3((unsigned)colblocks, nchunk), 256, 0, la.stream>>>(A, M, K, x, rows_per, la.work);
  RIHF_LAUNCH_CHECK();
  int blocks = (int)std::min<long long>((K + 255) / 256, 8LL * la.sms);
  cols_reduce_kernel<<<blocks, 256, 0, la.stream>>>(la.work, nchunk, K, alpha, y);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 2;
}

__global__ void outer_fill_kernel(const double* __restrict__ c, int naux, const double* __restrict__ D, long long n2,
                                  double* __restrict__ Y) {
  long long total = (long long)naux * n2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x)
    Y[idx] = c[idx / n2] * D[idx % n2];
}

void outer_fill(const LaCtx& la, const double* c, int naux, const double* D, long long n2, double* Y) {
  long long total = (long long)naux * n2;
  int blocks = (int)std::min<long long>((total + 255) / 256, 16LL * la.sms);
  outer_fill_kernel<<<blocks, 256, 0, la.stream>>>(c, naux, D, n2, Y);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

// ------------------------------------------------------------ packed storage
//
// One CTA per (matrix, row mu) at a time; its threads run along the row, so the
// packed row segment nu <= mu (contiguous) and the unpacked row are both
// accessed with coalesced loads and stores, and no index needs a square root.

__global__ void __launch_bounds__(256) pack_sym_batch_kernel(const double* __restrict__ A, int nmat, int N, double w,
                                                             double* __restrict__ Ap, long long ldp) {
  const long long rows = (long long)nmat * N, n2 = (long long)N * N;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const long long m = r / N;
    const int mu = (int)(r - m * N);
    const double* src = A + m * n2 + (long long)mu * N;
    double* dst = Ap + m * ldp + (long long)mu * (mu + 1) / 2;
    for (int nu = threadIdx.x; nu <= mu; nu += blockDim.x) dst[nu] = src[nu] * (nu == mu ? 1.0 : w);
  }
}

void pack_sym_batch(const LaCtx& la, const double* A, int nmat, int N, double* Ap, long long ldp) {
  const long long rows = (long long)nmat * N;
  pack_sym_batch_kernel<<<(int)std::max<long long>(1, std::min<long long>(rows, 32LL * la.sms)), 256, 0, la.stream>>>(
      A, nmat, N, 1.0, Ap, ldp);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

void pack_sym(const LaCtx& la, const double* A, int N, double w, double* Ap) {
  pack_sym_batch_kernel<<<std::max(1, std::min(N, 32 * la.sms)), 256, 0, la.stream>>>(A, 1, N, w, Ap, 0);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

// Row mu of A[m]: nu <= mu from the packed row (coalesced), nu > mu from
// column mu of the lower triangle (entry mu of the packed rows nu > mu).
__global__ void __launch_bounds__(256) unpack_sym_batch_kernel(const double* __restrict__ Ap, int nmat, int N,
                                                               long long ldp, double* __restrict__ A) {
  const long long rows = (long long)nmat * N, n2 = (long long)N * N;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const long long m = r / N;
    const int mu = (int)(r - m * N);
    const double* src = Ap + m * ldp;
    double* dst = A + m * n2 + (long long)mu * N;
    for (int nu = threadIdx.x; nu < N; nu += blockDim.x)
      dst[nu] = nu <= mu ? src[(long long)mu * (mu + 1) / 2 + nu] : src[(long long)nu * (nu + 1) / 2 + mu];
  }
}

void unpack_sym_batch(const LaCtx& la, const double* Ap, int nmat, int N, long long ldp, double* A) {
  const long long rows = (long long)nmat * N;
  unpack_sym_batch_kernel<<<(int)std::max<long long>(1, std::min<long long>(rows, 32LL * la.sms)), 256, 0,
                            la.stream>>>(Ap, nmat, N, ldp, A);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

void unpack_sym(const LaCtx& la, const double* Ap, int N, double* A) { unpack_sym_batch(la, Ap, 1, N, 0, A); }

}  // namespace rihf
