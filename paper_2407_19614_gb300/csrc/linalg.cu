// Dense linear algebra kernels of librihf.
#include <algorithm>
#include <cmath>

#include "../../include/rihf.h"
#include "linalg.cuh"
#include "tc_gemm.cuh"

#include <mutex>
#include <unordered_map>

namespace rihf {

void raise_smem_limit(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cur;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  RIHF_CUDA(cudaGetDevice(&dev));
  const void* key = (const void*)((const char*)kernel + dev);   // per device
  auto it = cur.find(key);
  if (it != cur.end() && it->second >= bytes) return;
  RIHF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  cur[key] = bytes;
}

}  // namespace rihf

namespace rihf {

static inline void count(const LaCtx& la, int n = 1) {
  if (la.launches) *la.launches += n;
}

// ------------------------------------------------------------ GEMM (FP64)

constexpr int GT = 32;   // output tile
constexpr int GK = 16;   // K step

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(GemmArgs g, int nsplit, int kper, int bper,
                                                    double* __restrict__ work) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int n0 = blockIdx.x * GT, m0 = blockIdx.y * GT;
  const int z = blockIdx.z;
  if (g.symcols > 0) {
    int j0 = n0, j1 = min(n0 + GT, g.N) - 1;
    bool spans = (j0 / g.symcols) != (j1 / g.symcols);
    if (!spans && (j0 % g.symcols) > (j0 / g.symcols)) return;
  }
  if (g.lower_only && n0 > m0) return;
  int b_lo, b_hi, k_lo, k_hi, slot_b, slot_s;
  if (g.reduce_batch) {
    slot_s = z;
    slot_b = 0;
    b_lo = z * bper;
    b_hi = min(g.batch, b_lo + bper);
    k_lo = 0;
    k_hi = g.K;
  } else {
    slot_b = z / nsplit;
    slot_s = z % nsplit;
    b_lo = slot_b;
    b_hi = slot_b + 1;
    k_lo = slot_s * kper;
    k_hi = min(g.K, k_lo + kper);
  }
  if (g.lowerA) k_hi = min(k_hi, m0 + GT);
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int b = b_lo; b < b_hi; ++b) {
    const double* A = g.A + (long long)b * g.sA;
    const double* B = g.B + (long long)b * g.sB;
    for (int k0 = k_lo; k0 < k_hi; k0 += GK) {
      for (int r = 0; r < 2; ++r) {
        int idx = tid + r * 256;
        int mm, kk;
        if (TA) { mm = idx % GT; kk = idx / GT; } else { kk = idx % GK; mm = idx / GK; }
        int m = m0 + mm, k = k0 + kk;
        double v = 0.0;
        if (m < g.M && k < k_hi) v = TA ? A[(long long)k * g.lda + m] : A[(long long)m * g.lda + k];
        As[kk][mm] = v;
        int nn, kb;
        if (TB) { kb = idx % GK; nn = idx / GK; } else { nn = idx % GT; kb = idx / GT; }
        int n = n0 + nn, kq = k0 + kb;
        double w = 0.0;
        if (n < g.N && kq < k_hi) w = TB ? B[(long long)n * g.ldb + kq] : B[(long long)kq * g.ldb + n];
        Bs[kb][nn] = w;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
        double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
      }
      __syncthreads();
    }
  }
  const bool direct = g.reduce_batch ? (gridDim.z == 1) : (nsplit == 1);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      int m = m0 + ty * 2 + i, n = n0 + tx * 2 + j;
      if (m >= g.M || n >= g.N) continue;
      if (direct) {
        double* C = g.C + (g.reduce_batch ? 0 : (long long)slot_b * g.sC);
        double* c = C + (long long)m * g.ldc + n;
        *c = g.beta == 0.0 ? g.alpha * acc[i][j] : g.alpha * acc[i][j] + g.beta * *c;
      } else {
        long long slot = (long long)slot_b * (g.reduce_batch ? gridDim.z : nsplit) + slot_s;
        work[slot * g.M * g.N + (long long)m * g.N + n] = acc[i][j];
      }
    }
}

__global__ void splitk_reduce_kernel(GemmArgs g, int nsplit, const double* __restrict__ work) {
  long long total = (long long)g.M * g.N * (g.reduce_batch ? 1 : g.batch);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long mn = idx % ((long long)g.M * g.N);
    int b = (int)(idx / ((long long)g.M * g.N));
    int m = (int)(mn / g.N), n = (int)(mn % g.N);
    if (g.symcols > 0) {
      // tiles skipped in the product were never written; mirror does the rest
      int j0 = (n / GT) * GT, j1 = min(j0 + GT, g.N) - 1;
      bool spans = (j0 / g.symcols) != (j1 / g.symcols);
      if (!spans && (j0 % g.symcols) > (j0 / g.symcols)) continue;
    }
    if (g.lower_only && (n / GT) > (m / GT)) continue;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += work[((long long)b * nsplit + q) * g.M * g.N + mn];
    double* c = g.C + (g.reduce_batch ? 0 : (long long)b * g.sC) + (long long)m * g.ldc + n;
    *c = g.beta == 0.0 ? g.alpha * s : g.alpha * s + g.beta * *c;
  }
}

// The tensor-core route of dgemm (see LaCtx::tcA): op(A) as rows M, K and
// op(B)^T as rows N, K, both sliced into 7 digits; C stored (beta 0) or
// accumulated (beta 1).  Returns false when the product does not qualify.
static bool dgemm_tc(const LaCtx& la, const GemmArgs& g) {
  if (!la.tcA || !la.tcB || g.batch != 1 || g.reduce_batch || g.lowerA || g.symcols != 0 ||
      !(g.beta == 0.0 || g.beta == 1.0) || g.K <= 0)
    return false;
  if ((double)g.M * g.N * g.K < la.tc_min_work) return false;
  if ((g.K + kOzChunk - 1) / kOzChunk > kOzMaxChunksPerBlock) return false;
  auto fits = [](const OzBuf* b, int rows, int K) {
    return oz_plane_elems(rows, K, kOzMaxDigits) <= b->cap &&
           (size_t)((rows + kOzTileM - 1) / kOzTileM * kOzTileM) <= b->ecap;
  };
  if (!fits(la.tcA, g.M, g.K) || !fits(la.tcB, g.N, g.K)) return false;
  // element (m, k) of op(A) and (n, k) of op(B)^T
  OzGemmArgs o;
  o.A = oz_slice(la, g.A, g.M, g.K, g.transA ? 1 : g.lda, g.transA ? g.lda : 1, 0, g.K, kOzMaxDigits, 0, *la.tcA);
  o.B = oz_slice(la, g.B, g.N, g.K, g.transB ? g.ldb : 1, g.transB ? 1 : g.ldb, 0, g.K, kOzMaxDigits, 0, *la.tcB);
  o.M = g.M; o.N = g.N; o.s = kOzMaxDigits; o.alpha = g.alpha; o.C = g.C; o.cs_m1 = g.ldc; o.cs_n = 1;
  o.accumulate = g.beta == 1.0;
  o.lower_only = g.lower_only;
  oz_gemm(la, o);
  return true;
}

void dgemm(const LaCtx& la, const GemmArgs& g) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  if (dgemm_tc(la, g)) return;
  int tm = ceil_div(g.M, GT), tn = ceil_div(g.N, GT);
  if (tm > 65535) {
    // row tiles run on grid.y (at most 65535): tall products (rows (P, mu) of
    // Naux N) go in row slabs
    if (g.batch != 1 || g.reduce_batch || g.lowerA || g.lower_only || g.symcols)
      throw RihfError(RIHF_ERR_INVALID_ARG, "dgemm: too many row tiles for this product shape");
    const int slab = 65535 * GT;
    for (int r0 = 0; r0 < g.M; r0 += slab) {
      GemmArgs h = g;
      h.M = std::min(slab, g.M - r0);
      h.A = g.A + (size_t)r0 * (g.transA ? 1 : g.lda);
      h.C = g.C + (size_t)r0 * g.ldc;
      dgemm(la, h);
    }
    return;
  }
  long long tiles = (long long)tm * tn * (g.reduce_batch ? 1 : g.batch);
  int nsplit = 1, kper = g.K, bper = g.batch;
  const long long target = 4LL * la.sms;
  if (g.reduce_batch) {
    nsplit = (int)std::min<long long>(g.batch, std::max<long long>(1, (target + tiles - 1) / tiles));
    while (nsplit > 1 && (size_t)nsplit * g.M * g.N > la.work_elems) nsplit /= 2;
    bper = ceil_div(g.batch, nsplit);
    nsplit = ceil_div(g.batch, bper);
  } else if (tiles < target && g.K > 2 * GK) {
    nsplit = (int)std::min<long long>((target + tiles - 1) / tiles, g.K / GK);
    while (nsplit > 1 && (size_t)nsplit * g.M * g.N * g.batch > la.work_elems) nsplit /= 2;
    kper = ceil_div(ceil_div(g.K, nsplit), GK) * GK;
    nsplit = ceil_div(g.K, kper);
  }
  if (g.lowerA && nsplit > 1 && !g.reduce_batch) {
    // the triangular cut is per row tile; keep it simple and exact
    nsplit = 1;
    kper = g.K;
  }
  dim3 grid(tn, tm, g.reduce_batch ? nsplit : g.batch * nsplit);
  if (g.transA && g.transB)
    dgemm_kernel<true, true><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, la.work);
  else if (g.transA)
    dgemm_kernel<true, false><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, la.work);
  else if (g.transB)
    dgemm_kernel<false, true><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, la.work);
  else
    dgemm_kernel<false, false><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, la.work);
  RIHF_LAUNCH_CHECK();
  count(la);
  if (nsplit > 1) {
    long long total = (long long)g.M * g.N * (g.reduce_batch ? 1 : g.batch);
    int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * la.sms);
    splitk_reduce_kernel<<<blocks, 256, 0, la.stream>>>(g, nsplit, la.work);
    RIHF_LAUNCH_CHECK();
    count(la);
  }
}

// ------------------------------------------------------------ GEMM (FP32)

constexpr int ST = 64;   // output tile
constexpr int SK = 16;   // K step

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(SGemmArgs g, int nsplit, int kper, int bper, float* work) {
  __shared__ float As[SK][ST + 4];
  __shared__ float Bs[SK][ST + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int n0 = blockIdx.x * ST, m0 = blockIdx.y * ST;
  const int z = blockIdx.z;
  int b_lo, b_hi, k_lo, k_hi, slot_b, slot_s;
  if (g.reduce_batch) {
    slot_s = z; slot_b = 0; b_lo = z * bper; b_hi = min(g.batch, b_lo + bper); k_lo = 0; k_hi = g.K;
  } else {
    slot_b = z / nsplit; slot_s = z % nsplit; b_lo = slot_b; b_hi = slot_b + 1;
    k_lo = slot_s * kper; k_hi = min(g.K, k_lo + kper);
  }
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int b = b_lo; b < b_hi; ++b) {
    const float* A = g.A + (long long)b * g.sA;
    const float* B = g.B + (long long)b * g.sB;
    for (int k0 = k_lo; k0 < k_hi; k0 += SK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int idx = tid + r * 256;   // 1024 = 64 x 16
        int mm, kk;
        if (TA) { mm = idx % ST; kk = idx / ST; } else { kk = idx % SK; mm = idx / SK; }
        int m = m0 + mm, k = k0 + kk;
        float v = 0.f;
        if (m < g.M && k < k_hi) v = TA ? A[(long long)k * g.lda + m] : A[(long long)m * g.lda + k];
        As[kk][mm] = v;
        int nn, kb;
        if (TB) { kb = idx % SK; nn = idx / SK; } else { nn = idx % ST; kb = idx / ST; }
        int n = n0 + nn, kq = k0 + kb;
        float w = 0.f;
        if (n < g.N && kq < k_hi) w = TB ? B[(long long)n * g.ldb + kq] : B[(long long)kq * g.ldb + n];
        Bs[kb][nn] = w;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < SK; ++kk) {
        float a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  const int nslots = g.reduce_batch ? (int)gridDim.z : nsplit;
  const bool direct = nslots == 1;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m >= g.M || n >= g.N) continue;
      if (direct && !g.Cd) {
        float* c = g.C + (g.reduce_batch ? 0 : (long long)slot_b * g.sC) + (long long)m * g.ldc + n;
        *c = (float)(g.beta == 0.0 ? g.alpha * acc[i][j] : g.alpha * acc[i][j] + g.beta * *c);
      } else {
        long long slot = (long long)slot_b * nslots + slot_s;
        work[slot * g.M * g.N + (long long)m * g.N + n] = acc[i][j];
      }
    }
}

__global__ void sgemm_reduce_kernel(SGemmArgs g, int nslots, const float* __restrict__ work) {
  long long total = (long long)g.M * g.N * (g.reduce_batch ? 1 : g.batch);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long mn = idx % ((long long)g.M * g.N);
    int b = (int)(idx / ((long long)g.M * g.N));
    int m = (int)(mn / g.N), n = (int)(mn % g.N);
    double s = 0.0;
    for (int q = 0; q < nslots; ++q) s += (double)work[((long long)b * nslots + q) * g.M * g.N + mn];
    long long off = (g.reduce_batch ? 0 : (long long)b * g.sC) + (long long)m * g.ldc + n;
    if (g.Cd) g.Cd[off] = g.beta == 0.0 ? g.alpha * s : g.alpha * s + g.beta * g.Cd[off];
    else g.C[off] = (float)(g.beta == 0.0 ? g.alpha * s : g.alpha * s + g.beta * g.C[off]);
  }
}

void sgemm(const LaCtx& la, const SGemmArgs& g) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  int tm = ceil_div(g.M, ST), tn = ceil_div(g.N, ST);
  long long tiles = (long long)tm * tn * (g.reduce_batch ? 1 : g.batch);
  int nsplit = 1, kper = g.K, bper = g.batch;
  const long long target = 4LL * la.sms;
  const size_t cap = la.work_elems * 2;   // the workspace holds twice as many floats
  if (g.reduce_batch) {
    nsplit = (int)std::min<long long>(g.batch, std::max<long long>(1, (target + tiles - 1) / tiles));
    while (nsplit > 1 && (size_t)nsplit * g.M * g.N > cap) nsplit /= 2;
    bper = ceil_div(g.batch, nsplit);
    nsplit = ceil_div(g.batch, bper);
  } else if (tiles < target && g.K > 4 * SK) {
    nsplit = (int)std::min<long long>((target + tiles - 1) / tiles, g.K / (2 * SK));
    while (nsplit > 1 && (size_t)nsplit * g.M * g.N * g.batch > cap) nsplit /= 2;
    kper = ceil_div(ceil_div(g.K, nsplit), SK) * SK;
    nsplit = ceil_div(g.K, kper);
  }
  float* work = reinterpret_cast<float*>(la.work);
  dim3 grid(tn, tm, g.reduce_batch ? nsplit : g.batch * nsplit);
  if (g.transA && g.transB) sgemm_kernel<true, true><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, work);
  else if (g.transA) sgemm_kernel<true, false><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, work);
  else if (g.transB) sgemm_kernel<false, true><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, work);
  else sgemm_kernel<false, false><<<grid, 256, 0, la.stream>>>(g, nsplit, kper, bper, work);
  RIHF_LAUNCH_CHECK();
  count(la);
  if (nsplit > 1 || g.Cd) {
    long long total = (long long)g.M * g.N * (g.reduce_batch ? 1 : g.batch);
    int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * la.sms);
    sgemm_reduce_kernel<<<blocks, 256, 0, la.stream>>>(g, nsplit, work);
    RIHF_LAUNCH_CHECK();
    count(la);
  }
}

__global__ void to_float_kernel(const double* __restrict__ in, long long n, float* __restrict__ out, double s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)(s * in[i]);
}
void to_float(const LaCtx& la, const double* in, long long n, float* out, double scale) {
  int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 16LL * la.sms));
  to_float_kernel<<<blocks, 256, 0, la.stream>>>(in, n, out, scale);
  RIHF_LAUNCH_CHECK();
  count(la);
}

// ------------------------------------------------------------ symmetrize

__global__ void symmetrize_lower_kernel(double* X, int n) {
  __shared__ double t[32][33];
  int bi = blockIdx.y, bj = blockIdx.x;   // destination tile (bi, bj) with bi <= bj (upper)
  if (bi > bj) return;
  double* S = X + (size_t)blockIdx.z * n * n;
  // source tile (bj, bi) in the lower triangle
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = bj * 32 + r, j = bi * 32 + threadIdx.x;
    t[r][threadIdx.x] = (i < n && j < n) ? S[(size_t)i * n + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = bi * 32 + r, j = bj * 32 + threadIdx.x;   // upper element (i, j), j > i
    if (i < n && j < n && j > i) S[(size_t)i * n + j] = t[threadIdx.x][r];
  }
}

void symmetrize_lower(const LaCtx& la, double* X, int n, int batch) {
  int nt = ceil_div(n, 32);
  symmetrize_lower_kernel<<<dim3(nt, nt, batch), dim3(32, 8), 0, la.stream>>>(X, n);
  RIHF_LAUNCH_CHECK();
  count(la);
}

// ------------------------------------------------------------ Cholesky

constexpr int CB = 32;

// One step of the right-looking blocked Cholesky (block CB = 32), in one launch
// of 128-thread blocks.  Every block factors the diagonal block L_kk itself
// (the same instructions on the same data, so every block gets the same bits):
// lane r holds row r, warp w the columns c = 4 t + w, and each pivot column is
// broadcast through shared memory, so the narrow FP64 pipes of all four SM
// sub-partitions share the rank-1 updates while one warp runs the pivot's
// reciprocal square root.  Block 0 stores L_kk in Ld (the diagonal block of A
// is still being read by the other blocks; chol_finish_kernel copies it in).
// Then the panel rows r >= k + b solve y L_kk^T = a_r by forward substitution,
// four lanes per row (eight rows per warp) splitting each dot product.
__global__ void __launch_bounds__(128) chol_step_kernel(double* A, int n, int k, int b, int* flag, double* Ld) {
  __shared__ double l[CB][CB + 1];
  __shared__ double piv[2][CB];
  __shared__ double rd[CB];
  __shared__ double ys[4][8][CB + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double a[CB / 4];
#pragma unroll
  for (int t = 0; t < CB / 4; ++t) {
    const int c = 4 * t + w;
    a[t] = (lane < b && c < b && c <= lane) ? A[(size_t)(k + lane) * n + k + c] : 0.0;
  }
#pragma unroll
  for (int j = 0; j < CB; ++j) {
    if (j < b) {
      if (w == (j & 3)) {
        double d = __shfl_sync(0xffffffffu, a[j >> 2], j);
        if (!(d > 0.0)) {
          if (lane == 0 && blockIdx.x == 0) atomicExch(flag, 1);
          d = 1.0;
          if (lane == j) a[j >> 2] = 1.0;
        }
        // rows above the pivot hold zeros and row j holds d itself, so one
        // multiply gives l_jj = d r and the column below scaled by r
        a[j >> 2] *= rsqrt(d);
        piv[j & 1][lane] = a[j >> 2];
      }
      __syncthreads();   // also orders the reuse of piv[j & 1] two steps on
      const double lj = piv[j & 1][lane];
#pragma unroll
      for (int t = 0; t < CB / 4; ++t) {
        const int c = 4 * t + w;
        if (c > j && lane >= c) a[t] = fma(-lj, piv[j & 1][c], a[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < CB / 4; ++t) {
    const int c = 4 * t + w;
    l[lane][c] = a[t];
    if (blockIdx.x == 0 && lane < b && c < b) Ld[(size_t)(k + lane) * CB + c] = a[t];
  }
  __syncthreads();
  if (threadIdx.x < CB) rd[threadIdx.x] = threadIdx.x < b ? 1.0 / l[threadIdx.x][threadIdx.x] : 0.0;
  __syncthreads();
  const int rs = lane >> 2, sub = lane & 3;
  double* y = ys[w][rs];
  for (int r0 = k + b + (blockIdx.x * 4 + w) * 8; r0 < n; r0 += gridDim.x * 32) {
    const int r = r0 + rs;
    const bool valid = r < n;
    for (int i = sub; i < b; i += 4) y[i] = valid ? A[(size_t)r * n + k + i] : 0.0;
    __syncwarp();
    for (int i = 0; i < b; ++i) {
      double part = sub == 0 ? y[i] : 0.0;
      for (int q = sub; q < i; q += 4) part = fma(-l[i][q], y[q], part);
      part += __shfl_xor_sync(0xffffffffu, part, 1);
      part += __shfl_xor_sync(0xffffffffu, part, 2);
      if (sub == 0) y[i] = part * rd[i];
      __syncwarp();
    }
    if (valid)
      for (int i = sub; i < b; i += 4) A[(size_t)r * n + k + i] = y[i];
    __syncwarp();
  }
}

// The diagonal blocks from Ld into A; the upper triangle zeroed.
__global__ void chol_finish_kernel(double* A, int n, const double* __restrict__ Ld) {
  long long total = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / n), j = (int)(idx % n);
    if (j > i) A[idx] = 0.0;
    else if (i / CB == j / CB) A[idx] = Ld[(size_t)i * CB + (j % CB)];
  }
}

void cholesky(const LaCtx& la, double* A, int n, double* scratch) {
  double* Ld = scratch;   // n x CB: the factored diagonal blocks
  for (int k = 0; k < n; k += CB) {
    int b = std::min(CB, n - k);
    int rest = n - k - b;
    // L_kk, and A[k+b:, k:k+b] <- A[k+b:, k:k+b] L_kk^{-T}
    chol_step_kernel<<<std::max(1, ceil_div(rest, 32)), 128, 0, la.stream>>>(A, n, k, b, la.flag, Ld);
    RIHF_LAUNCH_CHECK();
    count(la);
    if (rest <= 0) break;
    // trailing update: A[k+b:, k+b:] -= panel panel^T, lower tiles only (the
    // factorisation never reads the upper triangle; it is zeroed at the end)
    GemmArgs u;
    u.M = rest; u.N = rest; u.K = b;
    u.A = A + (size_t)(k + b) * n + k; u.lda = n;
    u.B = A + (size_t)(k + b) * n + k; u.ldb = n; u.transB = true;
    u.C = A + (size_t)(k + b) * n + k + b; u.ldc = n;
    u.alpha = -1.0; u.beta = 1.0;
    u.lower_only = true;
    dgemm(la, u);
  }
  chol_finish_kernel<<<std::max(1, std::min(ceil_div((long long)n * n, 256), 8 * la.sms)), 256, 0, la.stream>>>(
      A, n, Ld);
  RIHF_LAUNCH_CHECK();
  count(la);
}

__global__ void identity_kernel(double* X, int n) {
  long long total = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x)
    X[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

void identity(const LaCtx& la, double* X, int n) {
  identity_kernel<<<std::max(1, std::min(ceil_div((long long)n * n, 256), 8 * la.sms)), 256, 0, la.stream>>>(X, n);
  RIHF_LAUNCH_CHECK();
  count(la);
}

// Substitution inside one diagonal block: every thread owns one column j of the
// b x ncol slab X[k:k+b, :] and solves L_kk y = x (trans = 0) or L_kk^T y = x
// (trans = 1) in registers; L_kk is staged in shared memory.  Substitution (not
// a product with an explicit block inverse) keeps the accuracy of the classical
// algorithm when the auxiliary functions of one atom make L_kk ill-conditioned.
__global__ void __launch_bounds__(256) trsv_block_kernel(const double* __restrict__ L, int n, int k, int b,
                                                         double* __restrict__ X, long long ncol, int trans,
                                                         int symcols) {
  __shared__ double l[CB][CB + 1];
  __shared__ double rd[CB];
  for (int i = threadIdx.x; i < CB * CB; i += blockDim.x) {
    int r = i / CB, c = i % CB;
    l[r][c] = (r < b && c < b) ? L[(size_t)(k + r) * n + k + c] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CB; i += blockDim.x) rd[i] = i < b ? 1.0 / l[i][i] : 0.0;
  __syncthreads();
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < ncol; j += (long long)gridDim.x * blockDim.x) {
    if (symcols > 0 && (j % symcols) > (j / symcols)) continue;   // strict upper triangle: never used
    double y[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) y[i] = i < b ? X[(size_t)(k + i) * ncol + j] : 0.0;
    if (!trans) {
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        if (i >= b) break;
        double s = y[i];
#pragma unroll
        for (int q = 0; q < i; ++q) s -= l[i][q] * y[q];
        y[i] = s * rd[i];
      }
    } else {
#pragma unroll
      for (int i = CB - 1; i >= 0; --i) {
        if (i >= b) continue;
        double s = y[i];
#pragma unroll
        for (int q = i + 1; q < CB; ++q)
          if (q < b) s -= l[q][i] * y[q];
        y[i] = s * rd[i];
      }
    }
#pragma unroll
    for (int i = 0; i < CB; ++i)
      if (i < b) X[(size_t)(k + i) * ncol + j] = y[i];
  }
}

// Launch shape of trsv_block_kernel: every column is a chain of dependent FP64
// operations, so narrow blocks spread few columns over many SMs.
static void trsv_shape(const LaCtx& la, long long ncol, int& blocks, int& threads) {
  const long long per = (ncol + 2LL * la.sms - 1) / (2LL * la.sms);   // columns per block for two blocks per SM
  threads = (int)std::min<long long>(256, std::max<long long>(32, (per + 31) / 32 * 32));
  blocks = (int)std::max<long long>(1, std::min<long long>((ncol + threads - 1) / threads, 16LL * la.sms));
}

void trsm_lower(const LaCtx& la, const double* L, int n, double* X, long long ncol, bool trans, int symcols,
                double* tmp) {
  (void)tmp;
  const int nb = ceil_div(n, CB);
  int blocks, threads;
  trsv_shape(la, ncol, blocks, threads);
  for (int q = 0; q < nb; ++q) {
    const int kb = trans ? nb - 1 - q : q;
    const int k = kb * CB, b = std::min(CB, n - k);
    trsv_block_kernel<<<blocks, threads, 0, la.stream>>>(L, n, k, b, X, ncol, trans ? 1 : 0, symcols);
    RIHF_LAUNCH_CHECK();
    count(la);
    GemmArgs u;
    u.N = (int)ncol; u.K = b;
    u.B = X + (size_t)k * ncol; u.ldb = (int)ncol;
    u.alpha = -1.0; u.beta = 1.0;
    u.symcols = symcols;
    if (!trans) {
      // X[k+b:, :] -= L[k+b:, k:k+b] X_k
      u.M = n - k - b;
      u.A = L + (size_t)(k + b) * n + k; u.lda = n;
      u.C = X + (size_t)(k + b) * ncol; u.ldc = (int)ncol;
    } else {
      // X[0:k, :] -= L[k:k+b, 0:k]^T X_k
      u.M = k;
      u.A = L + (size_t)k * n; u.lda = n; u.transA = true;
      u.C = X; u.ldc = (int)ncol;
    }
    if (u.M > 0) dgemm(la, u);
  }
}

void trsm_lower_tc(const LaCtx& la, const double* L, int n, double* X, long long ncol, int symcols,
                   const TrsmTcScratch& sc) {
  constexpr int PB = kTrsmPanel;   // inner panel width (K of the inner digit-plane updates)
  int blocks, threads;
  trsv_shape(la, ncol, blocks, threads);
  // X[r0 + M rows] -= L[r0.., k..k+kk) X[k..k+kk) on the tensor cores
  auto tc_update = [&](int r0, int M, int k, int kk) {
    if (M <= 0) return;
    OzGemmArgs g;
    g.A = oz_slice(la, L + (size_t)r0 * n + k, M, kk, n, 1, 0, kk, kOzMaxDigits, 0, sc.L);
    g.B = oz_slice(la, X + (size_t)k * ncol, (int)ncol, kk, 1, ncol, 0, kk, kOzMaxDigits, 0, sc.X);
    g.M = M; g.N = (int)ncol; g.s = kOzMaxDigits; g.alpha = -1.0;
    g.C = X + (size_t)r0 * ncol; g.cs_m1 = ncol; g.cs_n = 1;
    g.accumulate = true; g.symcols = symcols;
    oz_gemm(la, g);
  };
  for (int ko = 0; ko < n; ko += kTrsmOuter) {
  const int ke = std::min(n, ko + kTrsmOuter);
  for (int k = ko; k < ke; k += PB) {
    const int pb = std::min(PB, ke - k);
    // the panel in FP64: 32-row substitution blocks and their in-panel updates
    for (int k2 = k; k2 < k + pb; k2 += CB) {
      const int b = std::min(CB, k + pb - k2);
      trsv_block_kernel<<<blocks, threads, 0, la.stream>>>(L, n, k2, b, X, ncol, 0, symcols);
      RIHF_LAUNCH_CHECK();
      count(la);
      const int m2 = k + pb - (k2 + b);
      if (m2 > 0) {
        GemmArgs u;
        u.M = m2; u.N = (int)ncol; u.K = b;
        u.A = L + (size_t)(k2 + b) * n + k2; u.lda = n;
        u.B = X + (size_t)k2 * ncol; u.ldb = (int)ncol;
        u.C = X + (size_t)(k2 + b) * ncol; u.ldc = (int)ncol;
        u.alpha = -1.0; u.beta = 1.0; u.symcols = symcols;
        dgemm(la, u);
      }
    }
    // rows of the outer panel below this panel
    tc_update(k + pb, ke - k - pb, k, pb);
  }
  // all rows below the outer panel: one rank-(ke - ko) update
  tc_update(ke, n - ke, ko, ke - ko);
  }
}

void trsm_lower_t_tc(const LaCtx& la, const double* L, int n, double* X, long long ncol, int symcols,
                     const TrsmTcScratch& sc) {
  constexpr int PB = kTrsmPanel;
  int blocks, threads;
  trsv_shape(la, ncol, blocks, threads);
  // X[r0 .. r0+M) -= L[k..k+kk, r0..r0+M)^T X[k..k+kk) on the tensor cores
  auto tc_update = [&](int r0, int M, int k, int kk) {
    if (M <= 0) return;
    OzGemmArgs g;
    g.A = oz_slice(la, L + (size_t)k * n + r0, M, kk, 1, n, 0, kk, kOzMaxDigits, 0, sc.L);
    g.B = oz_slice(la, X + (size_t)k * ncol, (int)ncol, kk, 1, ncol, 0, kk, kOzMaxDigits, 0, sc.X);
    g.M = M; g.N = (int)ncol; g.s = kOzMaxDigits; g.alpha = -1.0;
    g.C = X + (size_t)r0 * ncol; g.cs_m1 = ncol; g.cs_n = 1;
    g.accumulate = true; g.symcols = symcols;
    oz_gemm(la, g);
  };
  // outer panels [ko, ke) from the bottom; inner 64-row panels and 32-row
  // substitution blocks aligned to multiples of their size, also from the bottom
  for (int ko = (n - 1) / kTrsmOuter * kTrsmOuter; ko >= 0; ko -= kTrsmOuter) {
    const int ke = std::min(n, ko + kTrsmOuter);
    for (int k = ko + (ke - ko - 1) / PB * PB; k >= ko; k -= PB) {
      const int kend = std::min(ke, k + PB);
      for (int k2 = k + (kend - k - 1) / CB * CB; k2 >= k; k2 -= CB) {
        const int b = std::min(CB, kend - k2);
        trsv_block_kernel<<<blocks, threads, 0, la.stream>>>(L, n, k2, b, X, ncol, 1, symcols);
        RIHF_LAUNCH_CHECK();
        count(la);
        if (k2 > k) {   // rows [k, k2) of the panel: X -= L[k2:k2+b, k:k2]^T X_k2
          GemmArgs u;
          u.M = k2 - k; u.N = (int)ncol; u.K = b;
          u.A = L + (size_t)k2 * n + k; u.lda = n; u.transA = true;
          u.B = X + (size_t)k2 * ncol; u.ldb = (int)ncol;
          u.C = X + (size_t)k * ncol; u.ldc = (int)ncol;
          u.alpha = -1.0; u.beta = 1.0; u.symcols = symcols;
          dgemm(la, u);
        }
      }
      // rows of the outer panel above this panel
      tc_update(ko, k - ko, k, kend - k);
    }
    // all rows above the outer panel: one rank-(ke - ko) update
    tc_update(0, ko, ko, ke - ko);
  }
}

// ------------------------------------------------------------ eigensolver

constexpr int JT = 1024;   // Jacobi threads (one CTA)
constexpr int kJRows = 8;  // rows per lane of the register-resident one-sided Jacobi (n <= 256)

// Parallel cyclic Jacobi (round-robin pairing) in FP32, one CTA.  a: m x m
// working matrix (shared or global), v: n x m eigenvector matrix (global).
__device__ void jacobi_f32(float* a, float* v, int n, int m, int max_sweeps, float* cs, float* sn, float* tt,
                           int* pp, int* qq, float* red) {
  const int tid = threadIdx.x;
  const int half = m / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test: off-diagonal vs diagonal Frobenius mass
    float off = 0.f, dia = 0.f;
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = warp; i < m; i += JT / 32)
      for (int j = lane; j < m; j += 32) {
        float x = a[i * m + j];
        if (i == j) dia += x * x; else off += x * x;
      }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) { red[tid / 32] = off; red[32 + tid / 32] = dia; }
    __syncthreads();
    if (tid == 0) {
      float so = 0.f, sd = 0.f;
      for (int w = 0; w < JT / 32; ++w) { so += red[w]; sd += red[32 + w]; }
      red[64] = so;
      red[65] = sd;
    }
    __syncthreads();
    float so = red[64], sd = red[65];
    __syncthreads();
    // FP32 stops near its rounding floor; the FP64 refinement takes over
    if (so <= 1e-10f * sd || so == 0.f) break;
    for (int r = 0; r < m - 1; ++r) {
      // pairs: (m-1, r) and ((r+k) mod (m-1), (r-k) mod (m-1)), k = 1..half-1
      for (int k = tid; k < half; k += JT) {
        int p, q;
        if (k == 0) { p = r; q = m - 1; }
        else { p = (r + k) % (m - 1); q = (r - k + (m - 1)) % (m - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        float apq = a[p * m + q], app = a[p * m + p], aqq = a[q * m + q];
        float c = 1.f, s = 0.f, t = 0.f;
        if (fabsf(apq) > 1e-30f && fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq))) {
          float tau = (aqq - app) / (2.f * apq);
          t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = rsqrtf(1.f + t * t);
          s = t * c;
        }
        pp[k] = p; qq[k] = q; cs[k] = c; sn[k] = s; tt[k] = t;
      }
      __syncthreads();
      // two-sided update of all 2x2 blocks (k1, k2): warp per k1, lane per k2
      for (int k1 = warp; k1 < half; k1 += JT / 32) {
        const int p1 = pp[k1], q1 = qq[k1];
        const float c1 = cs[k1], s1 = sn[k1];
        for (int k2 = lane; k2 < half; k2 += 32) {
          const int p2 = pp[k2], q2 = qq[k2];
          if (k1 == k2) {
            float apq = a[p1 * m + q1];
            a[p1 * m + p1] -= tt[k1] * apq;
            a[q1 * m + q1] += tt[k1] * apq;
            a[p1 * m + q1] = 0.f;
            a[q1 * m + p1] = 0.f;
            continue;
          }
          const float c2 = cs[k2], s2 = sn[k2];
          float app = a[p1 * m + p2], apq = a[p1 * m + q2], aqp = a[q1 * m + p2], aqq = a[q1 * m + q2];
          // right rotation (columns p2, q2)
          float xp = c2 * app - s2 * apq, xq = s2 * app + c2 * apq;
          float yp = c2 * aqp - s2 * aqq, yq = s2 * aqp + c2 * aqq;
          // left rotation (rows p1, q1)
          a[p1 * m + p2] = c1 * xp - s1 * yp;
          a[p1 * m + q2] = c1 * xq - s1 * yq;
          a[q1 * m + p2] = s1 * xp + c1 * yp;
          a[q1 * m + q2] = s1 * xq + c1 * yq;
        }
      }
      // eigenvectors: V <- V J
      for (int i = warp; i < n; i += JT / 32)
        for (int k = lane; k < half; k += 32) {
          int p = pp[k], q = qq[k];
          float c = cs[k], s = sn[k];
          float vp = v[i * m + p], vq = v[i * m + q];
          v[i * m + p] = c * vp - s * vq;
          v[i * m + q] = s * vp + c * vq;
        }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(JT) jacobi_kernel(const double* __restrict__ A, int n, int m, float* gA,
                                                    float* V, float* W, int use_smem, int max_sweeps) {
  extern __shared__ float sm[];
  __shared__ float cs[1024], sn[1024], tt[1024];
  __shared__ int pp[1024], qq[1024];
  __shared__ float red[72];
  float* a = use_smem ? sm : gA;
  for (int idx = threadIdx.x; idx < m * m; idx += JT) {
    int i = idx / m, j = idx % m;
    a[idx] = (i < n && j < n) ? (float)A[(size_t)i * n + j] : 0.f;
  }
  for (int idx = threadIdx.x; idx < n * m; idx += JT) {
    int i = idx / m, j = idx % m;
    V[idx] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  jacobi_f32(a, V, n, m, max_sweeps, cs, sn, tt, pp, qq, red);
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += JT) W[i] = a[i * m + i];
}

constexpr int kJB = 64;   // column blocks of the block one-sided Jacobi (two per warp)

// U (column-major, n x n) = A + sigma I with the Gershgorin shift sigma =
// 1.05 max_i sum_j |A_ij|, which makes the matrix positive definite.
__device__ float jacobi_shifted_copy(const double* __restrict__ A, int n, float* U, float* red) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float g = 0.f;
  for (int i = warp; i < n; i += JT / 32) {
    float s = 0.f;
    for (int j = lane; j < n; j += 32) s += fabsf((float)A[(size_t)i * n + j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    g = fmaxf(g, s);
  }
  if (lane == 0) red[warp] = g;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < JT / 32; ++w) t = fmaxf(t, red[w]);
    red[0] = 1.05f * t + 1e-20f;
  }
  __syncthreads();
  const float sigma = red[0];
  for (int j = warp; j < n; j += JT / 32)
    for (int i = lane; i < n; i += 32) U[(size_t)j * n + i] = (float)A[(size_t)i * n + j] + (i == j ? sigma : 0.f);
  __syncthreads();
  return sigma;
}

// Eigenpairs of the orthogonalised columns: v_j = u_j / |u_j|, lambda_j =
// |u_j| - sigma; V row-major n x m.
__device__ void jacobi_eigenpairs(const float* U, int n, int m, float sigma, float* V, float* W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < n; j += JT / 32) {
    const float* u = U + (size_t)j * n;
    float s = 0.f;
    for (int i = lane; i < n; i += 32) s = fmaf(u[i], u[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    float nrm = sqrtf(s);
    float inv = nrm > 0.f ? 1.f / nrm : 0.f;
    for (int i = lane; i < n; i += 32) V[(size_t)i * m + j] = u[i] * inv;
    if (lane == 0) W[j] = nrm - sigma;
  }
}

// One-sided (Hestenes) Jacobi in FP32, one CTA: with B = A + sigma I positive
// definite (sigma from a Gershgorin bound), column rotations U <- U J drive the
// columns of U = B V to mutual orthogonality; then v_j = u_j / |u_j| and
// lambda_j = |u_j| - sigma.  Only U (n x n, column-major, shared memory when it
// fits) is stored; a warp owns one column pair per round (round-robin pairing),
// its dot products reduced with shuffles.  For n <= 256 a pair's columns stay
// in registers between the dot product and the rotation, and the squared
// column norms are carried along by the rotation identities
// |u_p'|^2 = |u_p|^2 - t (u_p . u_q), |u_q'|^2 = |u_q|^2 + t (u_p . u_q)
// (recomputed at every sweep), so a pair costs one reduction, not three.
__global__ void __launch_bounds__(JT) jacobi1s_kernel(const double* __restrict__ A, int n, int m, float* gU, float* V,
                                                      float* W, int use_smem, int max_sweeps, float tol) {
  extern __shared__ float sm[];
  __shared__ float red[32];
  __shared__ float nrm[32 * kJRows];
  __shared__ int notconv;
  float* U = use_smem ? sm : gU;   // column j at U[j*n .. j*n+n)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float sigma = jacobi_shifted_copy(A, n, U, red);
  const int half = m / 2;
  const bool in_regs = n <= 32 * kJRows;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) notconv = 0;
    if (in_regs) {
      for (int j = warp; j < n; j += JT / 32) {
        const float* u = U + (size_t)j * n;
        float s2 = 0.f;
        for (int i = lane; i < n; i += 32) s2 = fmaf(u[i], u[i], s2);
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) nrm[j] = s2;
      }
    }
    __syncthreads();
    for (int r = 0; r < m - 1 && in_regs; ++r) {
      for (int k = warp; k < half; k += JT / 32) {
        int p, q;
        if (k == 0) { p = r; q = m - 1; }
        else { p = (r + k) % (m - 1); q = (r - k + (m - 1)) % (m - 1); }
        if (p >= n || q >= n) continue;   // padding column
        float* up = U + (size_t)p * n;
        float* uq = U + (size_t)q * n;
        float x[kJRows], y[kJRows];
        float c = 0.f;
#pragma unroll
        for (int e = 0; e < kJRows; ++e) {
          const int i = lane + 32 * e;
          x[e] = i < n ? up[i] : 0.f;
          y[e] = i < n ? uq[i] : 0.f;
          c = fmaf(x[e], y[e], c);
        }
        const float a = nrm[p], b = nrm[q];
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (fabsf(c) <= tol * sqrtf(a * b)) continue;
        if (lane == 0) notconv = 1;
        float zeta = (b - a) / (2.f * c);
        float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        float cs = rsqrtf(1.f + t * t), sn = cs * t;
#pragma unroll
        for (int e = 0; e < kJRows; ++e) {
          const int i = lane + 32 * e;
          if (i < n) {
            up[i] = cs * x[e] - sn * y[e];
            uq[i] = sn * x[e] + cs * y[e];
          }
        }
        if (lane == 0) {
          nrm[p] = a - t * c;
          nrm[q] = b + t * c;
        }
      }
      __syncthreads();
    }
    for (int r = 0; r < m - 1 && !in_regs; ++r) {
      for (int k = warp; k < half; k += JT / 32) {
        int p, q;
        if (k == 0) { p = r; q = m - 1; }
        else { p = (r + k) % (m - 1); q = (r - k + (m - 1)) % (m - 1); }
        if (p >= n || q >= n) continue;   // padding column
        float* up = U + (size_t)p * n;
        float* uq = U + (size_t)q * n;
        float a = 0.f, b = 0.f, c = 0.f;
        for (int i = lane; i < n; i += 32) {
          float x = up[i], y = uq[i];
          a = fmaf(x, x, a);
          b = fmaf(y, y, b);
          c = fmaf(x, y, c);
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (fabsf(c) <= tol * sqrtf(a * b)) continue;
        if (lane == 0) notconv = 1;
        float zeta = (b - a) / (2.f * c);
        float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        float cs = rsqrtf(1.f + t * t), sn = cs * t;
        for (int i = lane; i < n; i += 32) {
          float x = up[i], y = uq[i];
          up[i] = cs * x - sn * y;
          uq[i] = sn * x + cs * y;
        }
      }
      __syncthreads();
    }
    if (!notconv) break;
    __syncthreads();
  }
  jacobi_eigenpairs(U, n, m, sigma, V, W);
}

// Block one-sided Jacobi (n <= 64 H): the columns form kJB = 64 blocks of H;
// warp w holds two blocks in registers (H columns x R rows per lane each), and
// a round rotates every pair across its two blocks (round 0 also the pairs
// inside each block) before the blocks move on through U in shared memory.
// The block pairs follow the round-robin order of the column kernel, so a
// sweep is kJB - 1 rounds instead of n - 1 and moves a third of the shared-
// memory traffic; column norms are carried as there.
template <int H>
__global__ void __launch_bounds__(JT) jacobi1s_block_kernel(const double* __restrict__ A, int n, int m, float* gU,
                                                            float* V, float* W, int use_smem, int max_sweeps,
                                                            float tol) {
  constexpr int R = 2 * H;   // rows per lane
  extern __shared__ float sm[];
  __shared__ float red[32];
  __shared__ float nrm[kJB * H];
  __shared__ int notconv;
  float* U = use_smem ? sm : gU;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float sigma = jacobi_shifted_copy(A, n, U, red);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) notconv = 0;
    for (int j = warp; j < kJB * H; j += JT / 32) {
      float s2 = 0.f;
      if (j < n) {
        const float* u = U + (size_t)j * n;
        for (int i = lane; i < n; i += 32) s2 = fmaf(u[i], u[i], s2);
      }
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) nrm[j] = s2;
    }
    __syncthreads();
    for (int r = 0; r < kJB - 1; ++r) {
      int bA, bB;
      if (warp == 0) {
        bA = kJB - 1;
        bB = r;
      } else {
        bA = (r + warp) % (kJB - 1);
        bB = (r - warp + (kJB - 1)) % (kJB - 1);
      }
      float x[2 * H][R];
      float cn[2 * H];
#pragma unroll
      for (int c = 0; c < 2 * H; ++c) {
        const int g = (c < H ? bA * H + c : bB * H + c - H);
        cn[c] = nrm[g];
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const int i = lane + 32 * e;
          x[c][e] = (g < n && i < n) ? U[(size_t)g * n + i] : 0.f;
        }
      }
      bool rotated = false;
      auto rot = [&](float (&xp)[R], float (&xq)[R], float& a, float& b) {
        float c = 0.f;
#pragma unroll
        for (int e = 0; e < R; ++e) c = fmaf(xp[e], xq[e], c);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (fabsf(c) <= tol * sqrtf(a * b)) return;   // converged pair, or a zero (padding) column
        rotated = true;
        const float zeta = (b - a) / (2.f * c);
        const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float cs = rsqrtf(1.f + t * t), sn = cs * t;
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const float u = xp[e], v = xq[e];
          xp[e] = cs * u - sn * v;
          xq[e] = sn * u + cs * v;
        }
        a -= t * c;
        b += t * c;
      };
      if (r == 0) {
#pragma unroll
        for (int p = 0; p < H; ++p)
#pragma unroll
          for (int q = p + 1; q < H; ++q) {
            rot(x[p], x[q], cn[p], cn[q]);
            rot(x[H + p], x[H + q], cn[H + p], cn[H + q]);
          }
      }
#pragma unroll
      for (int p = 0; p < H; ++p)
#pragma unroll
        for (int q = 0; q < H; ++q) rot(x[p], x[H + q], cn[p], cn[H + q]);
#pragma unroll
      for (int c = 0; c < 2 * H; ++c) {
        const int g = (c < H ? bA * H + c : bB * H + c - H);
        if (g < n) {
#pragma unroll
          for (int e = 0; e < R; ++e) {
            const int i = lane + 32 * e;
            if (i < n) U[(size_t)g * n + i] = x[c][e];
          }
          if (lane == 0) nrm[g] = cn[c];
        }
      }
      if (rotated && lane == 0) notconv = 1;
      __syncthreads();
    }
    if (!notconv) break;
    __syncthreads();
  }
  jacobi_eigenpairs(U, n, m, sigma, V, W);
}

// Sort eigenpairs ascending (rank sort) and expand to FP64: X[:, rank] = V[:, i].
__global__ void eig_sort_kernel(const float* __restrict__ V, const float* __restrict__ W, int n, int m, double* X,
                                double* Wd) {
  __shared__ int rank[4096];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float wi = W[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      float wj = W[j];
      if (wj < wi || (wj == wi && j < i)) ++r;
    }
    rank[i] = r;
  }
  __syncthreads();
  // every block ranks all n values, then moves its own rows
  for (int row = blockIdx.x; row < n; row += gridDim.x)
    for (int i = threadIdx.x; i < n; i += blockDim.x) X[(size_t)row * n + rank[i]] = (double)V[row * m + i];
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) Wd[rank[i]] = (double)W[i];
}

// Ogita-Aishima step pieces: lam_i = S_ii/(1-R_ii); E_ij as in their Algorithm 1.
__global__ void oa_lambda_kernel(const double* R, const double* S, int n, double* lam) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    lam[i] = S[(size_t)i * n + i] / (1.0 - R[(size_t)i * n + i]);
}

// Partial sums of ||S - diag(lam)||_F^2, ||R||_F^2 and ||A||_F^2, block b into
// part[3b .. 3b+2] (oa_e_kernel folds them in a fixed order).
constexpr int kOaParts = 64;
__global__ void oa_norms_kernel(const double* R, const double* S, const double* A, const double* lam, int n,
                                double* part) {
  __shared__ double r0[32], r1[32], r2[32];
  double a0 = 0, a1 = 0, a2 = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / n), j = (int)(idx % n);
    double s = S[idx] - (i == j ? lam[i] : 0.0);
    a0 += s * s;
    a1 += R[idx] * R[idx];
    a2 += A[idx] * A[idx];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if ((threadIdx.x & 31) == 0) { r0[threadIdx.x / 32] = a0; r1[threadIdx.x / 32] = a1; r2[threadIdx.x / 32] = a2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) { s0 += r0[w]; s1 += r1[w]; s2 += r2[w]; }
    part[3 * blockIdx.x] = s0; part[3 * blockIdx.x + 1] = s1; part[3 * blockIdx.x + 2] = s2;
  }
}

__global__ void oa_e_kernel(const double* R, const double* S, const double* lam, const double* part, int nparts,
                            int n, double* E) {
  __shared__ double sh_delta;
  if (threadIdx.x < 32) {   // fold the partial sums (fixed order: deterministic)
    double s0 = 0, s1 = 0, s2 = 0;
    for (int b = threadIdx.x; b < nparts; b += 32) {
      s0 += part[3 * b];
      s1 += part[3 * b + 1];
      s2 += part[3 * b + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (threadIdx.x == 0) sh_delta = 2.0 * (sqrt(s0) + sqrt(s2) * sqrt(s1));
  }
  __syncthreads();
  const double delta = sh_delta;
  // A pair is rotated when its gap exceeds the global cluster threshold (as in
  // the method), or when its own first-order correction is small, |E_ij| < 1/8.
  // The threshold bounds the spectral norms of the residuals by their
  // Frobenius norms, which for large n exceed them by up to sqrt(n): pairs far
  // apart relative to their own coupling would otherwise count as clustered and
  // never rotate (at n = 1856 the refinement then stalls near FP32 accuracy).
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / n), j = (int)(idx % n);
    double r = R[idx];
    const double num = S[idx] + lam[j] * r, dl = lam[j] - lam[i];
    double e;
    if (i != j && (fabs(dl) > delta || fabs(dl) > 8.0 * fabs(num))) e = num / dl;
    else e = 0.5 * r;
    E[idx] = e;
  }
}

__global__ void add_inplace_kernel(double* X, const double* Y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    X[i] += Y[i];
}

__global__ void i_minus_kernel(double* R, int n) {   // R <- I - R
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / n), j = (int)(idx % n);
    R[idx] = (i == j ? 1.0 : 0.0) - R[idx];
  }
}


static int elem_blocks(const LaCtx& la, long long n) {
  return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * la.sms));
}

// Ascending reorder of FP64 eigenpairs: Vout[:, rank(i)] = V[:, i], Wout[rank(i)] = lam[i].
__global__ void eig_sort64_kernel(const double* __restrict__ V, const double* __restrict__ lam, int n, double* Vout,
                                  double* Wout) {
  __shared__ int rank[4096];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double wi = lam[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      double wj = lam[j];
      if (wj < wi || (wj == wi && j < i)) ++r;
    }
    rank[i] = r;
  }
  __syncthreads();
  // every block ranks all n values, then moves its own rows
  for (int row = blockIdx.x; row < n; row += gridDim.x)
    for (int i = threadIdx.x; i < n; i += blockDim.x) Vout[(size_t)row * n + rank[i]] = V[(size_t)row * n + i];
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) Wout[rank[i]] = lam[i];
}

// ------------------------------------------------------------ block Jacobi (large n)
//
// Two-sided cyclic Jacobi for orders above kBlockJacobiMin, spread over many
// CTAs, in FP32 (fast, to ~1e-6 of the norm) and then in FP64 from the FP32
// vectors (a few quadratically convergent sweeps).  The FP64 stage is what
// resolves the small end of a spectrum spanning many orders of magnitude: an
// overlap matrix with eigenvalues down to 3e-9 (the canonical orthogonaliser
// must drop those below 1e-8), or the orthonormal-basis Fock matrix built from
// it, whose near-dependent directions lie at ~1e8 Eh while the occupied ones,
// a few Eh apart, are all that the SCF needs: FP32 rounding of such a matrix
// is larger than the occupied spectrum.
//
// The (padded) indices form nb = np / kBJW blocks; a sweep is nb - 1 rounds of
// the round-robin pairing of blocks (block 0 fixed, the others circulating); in
// a round every block pair -- one CTA -- diagonalises its 2 kBJW x 2 kBJW
// submatrix by one cyclic sweep of plane rotations and a Newton-Schulz step,
// giving Q; then all pairs' columns are rotated (A <- A Q, V <- V Q) and, after
// them, all rows (A <- Q^T A).  Pairs own disjoint rows and columns, so the
// three launches of a round are the only synchronisation.  Padding indices
// (n..np) have zero coupling and are never rotated.  After each sweep the
// squared off-diagonal norm over the real indices is folded in a fixed order
// and compared with tol^2 times the diagonal's; a device flag then turns the
// remaining launches into no-ops (no host synchronisation, so the sweeps can
// sit in a CUDA graph).
constexpr int kBJW = 16, kBJ2 = 2 * kBJW, kBJParts = 256;

__device__ inline int bj_index(int pair, int k, int round, int nb) {
  const int pos = k < kBJW ? pair : nb - 1 - pair;
  const int blk = pos == 0 ? 0 : 1 + (pos - 1 + round) % (nb - 1);
  return blk * kBJW + (k % kBJW);
}

__device__ inline float bj_sqrt(float x) { return sqrtf(x); }
__device__ inline double bj_sqrt(double x) { return sqrt(x); }

template <class T>
__global__ void bj_init_kernel(const double* __restrict__ A, int n, int np, T* __restrict__ At, T* __restrict__ Vt,
                               int* done) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)np * np;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / np), j = (int)(e % np);
    At[e] = (i < n && j < n) ? (T)A[(size_t)i * n + j] : (T)0;
    Vt[e] = i == j ? (T)1 : (T)0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *done = 0;
}

template <class T>
__global__ void __launch_bounds__(256) bj_solve_kernel(const T* __restrict__ A, int np, int round, int nb,
                                                       T* __restrict__ Qg, const int* done) {
  if (*done) return;
  __shared__ T S[kBJ2][kBJ2 + 1], Q[kBJ2][kBJ2 + 1];
  __shared__ T cs[kBJW], sn[kBJW];
  __shared__ int ra[kBJW], rb[kBJW], idx[kBJ2];
  const int pair = blockIdx.x, t = threadIdx.x;
  if (t < kBJ2) idx[t] = bj_index(pair, t, round, nb);
  __syncthreads();
  for (int e = t; e < kBJ2 * kBJ2; e += blockDim.x) {
    const int i = e / kBJ2, j = e % kBJ2;
    S[i][j] = A[(size_t)idx[i] * np + idx[j]];
    Q[i][j] = i == j ? (T)1 : (T)0;
  }
  __syncthreads();
  // one cyclic sweep over the 2w indices: 2w - 1 rounds of w disjoint rotations
  for (int r = 0; r < kBJ2 - 1; ++r) {
    if (t < kBJW) {
      int a = t == 0 ? 0 : 1 + (t - 1 + r) % (kBJ2 - 1);
      int b = 1 + (kBJ2 - 2 - t + r) % (kBJ2 - 1);   // position 2w - 1 - t
      if (a > b) { const int x = a; a = b; b = x; }
      const T app = S[a][a], aqq = S[b][b], apq = S[a][b];
      T c = 1, s = 0;
      if (apq != (T)0) {
        // symmetric Schur rotation: J = [c s; -s c] zeroes the (a, b) entry of J^T S J
        const T th = (aqq - app) / (2 * apq);
        const T tt = (th >= 0 ? (T)1 : (T)-1) / (fabs(th) + bj_sqrt(th * th + 1));
        c = 1 / bj_sqrt(tt * tt + 1);
        s = tt * c;
      }
      cs[t] = c; sn[t] = s; ra[t] = a; rb[t] = b;
    }
    __syncthreads();
    for (int e = t; e < kBJW * kBJ2; e += blockDim.x) {   // S <- S J, Q <- Q J (columns a, b)
      const int k = e / kBJ2, i = e % kBJ2, a = ra[k], b = rb[k];
      const T c = cs[k], s = sn[k];
      const T x = S[i][a], y = S[i][b];
      S[i][a] = c * x - s * y;
      S[i][b] = s * x + c * y;
      const T u = Q[i][a], v = Q[i][b];
      Q[i][a] = c * u - s * v;
      Q[i][b] = s * u + c * v;
    }
    __syncthreads();
    for (int e = t; e < kBJW * kBJ2; e += blockDim.x) {   // S <- J^T S (rows a, b)
      const int k = e / kBJ2, j = e % kBJ2, a = ra[k], b = rb[k];
      const T c = cs[k], s = sn[k];
      const T x = S[a][j], y = S[b][j];
      S[a][j] = c * x - s * y;
      S[b][j] = s * x + c * y;
    }
    __syncthreads();
  }
  // one Newton-Schulz step, Q <- Q (3 I - Q^T Q) / 2: the 496 rotations leave Q
  // orthogonal to a few hundred rounding units only, and V multiplies about a
  // thousand such blocks
  for (int e = t; e < kBJ2 * kBJ2; e += blockDim.x) {   // S <- (3 I - Q^T Q) / 2
    const int i = e / kBJ2, j = e % kBJ2;
    T g = 0;
    for (int k = 0; k < kBJ2; ++k) g += Q[k][i] * Q[k][j];
    S[i][j] = (T)0.5 * ((i == j ? (T)3 : (T)0) - g);
  }
  __syncthreads();
  T* q = Qg + (size_t)pair * kBJ2 * kBJ2;
  for (int e = t; e < kBJ2 * kBJ2; e += blockDim.x) {
    const int i = e / kBJ2, j = e % kBJ2;
    T v = 0;
    for (int k = 0; k < kBJ2; ++k) v += Q[i][k] * S[k][j];
    q[e] = v;
  }
}

// A[r][idx] <- A[r][idx] Q and V[r][idx] <- V[r][idx] Q for every row r: one
// warp per row, lane k holds entry idx[k] (two contiguous segments per row).
template <class T>
__global__ void __launch_bounds__(256) bj_cols_kernel(T* __restrict__ A, T* __restrict__ V, int np, int round, int nb,
                                                      const T* __restrict__ Qg, const int* done) {
  if (*done) return;
  __shared__ T Q[kBJ2][kBJ2 + 1];
  const int pair = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* q = Qg + (size_t)pair * kBJ2 * kBJ2;
  for (int e = threadIdx.x; e < kBJ2 * kBJ2; e += blockDim.x) Q[e / kBJ2][e % kBJ2] = q[e];
  __syncthreads();
  const int col = bj_index(pair, lane, round, nb);
  for (int r = blockIdx.y * 8 + warp; r < np; r += gridDim.y * 8) {
    T x = A[(size_t)r * np + col], y = 0;
    T u = V[(size_t)r * np + col], w = 0;
#pragma unroll
    for (int m = 0; m < kBJ2; ++m) {
      const T qm = Q[m][lane];
      y += __shfl_sync(0xffffffffu, x, m) * qm;
      w += __shfl_sync(0xffffffffu, u, m) * qm;
    }
    A[(size_t)r * np + col] = y;
    V[(size_t)r * np + col] = w;
  }
}

// A[idx][c] <- Q^T A[idx][c] for every column c: one thread per column holds
// the 2w results of its column (coalesced across the warp).
template <class T>
__global__ void __launch_bounds__(128) bj_rows_kernel(T* __restrict__ A, int np, int round, int nb,
                                                      const T* __restrict__ Qg, const int* done) {
  if (*done) return;
  __shared__ T Q[kBJ2][kBJ2 + 1];
  __shared__ int idx[kBJ2];
  const int pair = blockIdx.x;
  const T* q = Qg + (size_t)pair * kBJ2 * kBJ2;
  for (int e = threadIdx.x; e < kBJ2 * kBJ2; e += blockDim.x) Q[e / kBJ2][e % kBJ2] = q[e];
  if (threadIdx.x < kBJ2) idx[threadIdx.x] = bj_index(pair, threadIdx.x, round, nb);
  __syncthreads();
  for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < np; c += gridDim.y * blockDim.x) {
    T o[kBJ2];
#pragma unroll
    for (int l = 0; l < kBJ2; ++l) o[l] = 0;
#pragma unroll 1
    for (int m = 0; m < kBJ2; ++m) {   // kept rolled: unrolled, the 1024 FMAs spill the outputs
      const T zm = A[(size_t)idx[m] * np + c];
#pragma unroll
      for (int l = 0; l < kBJ2; ++l) o[l] += Q[m][l] * zm;
    }
#pragma unroll
    for (int l = 0; l < kBJ2; ++l) A[(size_t)idx[l] * np + c] = o[l];
  }
}

// Squared off-diagonal and diagonal norms over the real indices, per block.
template <class T>
__global__ void __launch_bounds__(256) bj_norm_kernel(const T* __restrict__ A, int n, int np, double* part,
                                                      const int* done) {
  if (*done) return;
  __shared__ double r0[8], r1[8];
  double off = 0.0, dg = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double v = A[(size_t)i * np + j];
    if (i == j) dg += v * v;
    else off += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    dg += __shfl_xor_sync(0xffffffffu, dg, o);
  }
  if ((threadIdx.x & 31) == 0) { r0[threadIdx.x >> 5] = off; r1[threadIdx.x >> 5] = dg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < 8; ++w) { a += r0[w]; b += r1[w]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void bj_check_kernel(const double* part, int nparts, double tol2, int* done) {
  if (*done) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nparts; ++k) { a += part[2 * k]; b += part[2 * k + 1]; }   // fixed order
  if (a <= tol2 * b) *done = 1;
}

// FP64 copies of the real block: Vd (n x n) and the diagonal lam (n).
template <class T>
__global__ void bj_extract_kernel(const T* __restrict__ A, const T* __restrict__ V, int n, int np,
                                  double* __restrict__ Vd, double* __restrict__ lam) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    Vd[e] = (double)V[(size_t)i * np + j];
    if (i == j) lam[i] = (double)A[(size_t)i * np + i];
  }
}

// Unsorted eigenpairs of the n x n FP64 matrix Ain: Vd (n x n, FP64) and lam.
template <class T>
static void block_jacobi(const LaCtx& la, const double* Ain, int n, double* Vd, double* lam, double* bjws,
                         int max_sweeps, double tol) {
  const int np = (n + kBJ2 - 1) / kBJ2 * kBJ2, nb = np / kBJW, npair = nb / 2;
  T* At = reinterpret_cast<T*>(bjws);
  T* Vt = At + (size_t)np * np;
  T* Qg = Vt + (size_t)np * np;
  double* part = bjws + 2 * (size_t)np * np + (size_t)npair * kBJ2 * kBJ2;
  int* done = reinterpret_cast<int*>(part + 2 * kBJParts);
  bj_init_kernel<T><<<elem_blocks(la, (long long)np * np), 256, 0, la.stream>>>(Ain, n, np, At, Vt, done);
  RIHF_LAUNCH_CHECK();
  count(la);
  const int rowblk = std::max(1, std::min(ceil_div(np, 8), 4 * la.sms / std::max(1, npair)));
  const int colblk = std::max(1, std::min(ceil_div(np, 128), 4 * la.sms / std::max(1, npair)));
  const int nparts = std::min(kBJParts, ceil_div(n * n, 256));
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < nb - 1; ++r) {
      bj_solve_kernel<T><<<npair, 256, 0, la.stream>>>(At, np, r, nb, Qg, done);
      bj_cols_kernel<T><<<dim3(npair, rowblk), 256, 0, la.stream>>>(At, Vt, np, r, nb, Qg, done);
      bj_rows_kernel<T><<<dim3(npair, colblk), 128, 0, la.stream>>>(At, np, r, nb, Qg, done);
      RIHF_LAUNCH_CHECK();
      count(la, 3);
    }
    bj_norm_kernel<T><<<nparts, 256, 0, la.stream>>>(At, n, np, part, done);
    bj_check_kernel<<<1, 1, 0, la.stream>>>(part, nparts, tol * tol, done);
    RIHF_LAUNCH_CHECK();
    count(la, 2);
  }
  bj_extract_kernel<T><<<elem_blocks(la, (long long)n * n), 256, 0, la.stream>>>(At, Vt, n, np, Vd, lam);
  RIHF_LAUNCH_CHECK();
  count(la);
}

// Both stages for order n > kBlockJacobiMin: sorted eigenpairs (V, W) of Ain.
// FP32 sweeps to tol32, one FP64 Newton-Schulz step on the vectors, then FP64
// sweeps on Vs^T Ain Vs (nearly diagonal) to 1e-13 and V = Vs V2.  Scratch:
// the refinement slots R, S, AX, E, XE of the eigh workspace.
static void block_jacobi_2stage(const LaCtx& la, const double* Ain, int n, double* V, double* W, double* bjws,
                                int max_sweeps, float tol32, double* R, double* S, double* AX, double* E,
                                double* XE, double* lam) {
  block_jacobi<float>(la, Ain, n, XE, lam, bjws, max_sweeps, tol32);
  // XE holds the FP32 vectors (orthogonal to ~1e-6): Newton-Schulz, then
  // E = Vs^T Ain Vs and the FP64 sweeps
  GemmArgs gr;
  gr.M = n; gr.N = n; gr.K = n; gr.A = XE; gr.lda = n; gr.transA = true; gr.B = XE; gr.ldb = n; gr.C = R; gr.ldc = n;
  gr.alpha = -0.5;
  dgemm(la, gr);
  identity(la, S, n);
  axpby(la, n * n, 1.0, R, 1.5, S, R);   // R = (3 I - Vs^T Vs) / 2
  GemmArgs gn;
  gn.M = n; gn.N = n; gn.K = n; gn.A = XE; gn.lda = n; gn.B = R; gn.ldb = n; gn.C = S; gn.ldc = n;
  dgemm(la, gn);                          // S = Vs (orthonormal to ~1e-12)
  GemmArgs ga;
  ga.M = n; ga.N = n; ga.K = n; ga.A = Ain; ga.lda = n; ga.B = S; ga.ldb = n; ga.C = AX; ga.ldc = n;
  dgemm(la, ga);
  GemmArgs gs;
  gs.M = n; gs.N = n; gs.K = n; gs.A = S; gs.lda = n; gs.transA = true; gs.B = AX; gs.ldb = n; gs.C = E; gs.ldc = n;
  dgemm(la, gs);
  block_jacobi<double>(la, E, n, R, lam, bjws, 6, 1e-13);
  GemmArgs gv;
  gv.M = n; gv.N = n; gv.K = n; gv.A = S; gv.lda = n; gv.B = R; gv.ldb = n; gv.C = XE; gv.ldc = n;
  dgemm(la, gv);
  eig_sort64_kernel<<<std::min(n, 32), 256, 0, la.stream>>>(XE, lam, n, V, W);
  RIHF_LAUNCH_CHECK();
  count(la);
}

void eigh(const LaCtx& la, const double* A, int n, double* W, double* V, double* ws, int refine,
          const double* Vguess, bool skip_jacobi, int max_sweeps, int ns_steps) {
  int m = n + (n & 1);
  if (skip_jacobi && Vguess && refine > 0) {
    // Late SCF iterations: the previous eigenvectors are already close, so the
    // FP64 refinement alone converges (quadratically) without a Jacobi pass.
    double* d = ws + ((size_t)m * m + (size_t)n * m + m + 1) / 2;
    double* Vs = d + 4 * (size_t)n * n;   // the XE slot of the workspace
    double* lam = d + 6 * (size_t)n * n;
    RIHF_CUDA(cudaMemcpyAsync(V, Vguess, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, la.stream));
    eigh(la, A, n, W, V, ws, -refine, nullptr, false, max_sweeps, ns_steps);
    eig_sort64_kernel<<<std::min(n, 32), 256, 0, la.stream>>>(V, lam, n, Vs, W);
    RIHF_LAUNCH_CHECK();
    count(la);
    RIHF_CUDA(cudaMemcpyAsync(V, Vs, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, la.stream));
    return;
  }
  const bool refine_only = refine < 0;   // V already holds the starting vectors
  if (refine_only) refine = -refine;
  float* fA = reinterpret_cast<float*>(ws);
  float* fV = fA + (size_t)m * m;
  float* fW = fV + (size_t)n * m;
  double* d = ws + ((size_t)m * m + (size_t)n * m + m + 1) / 2;
  double* R = d;
  double* S = R + (size_t)n * n;
  double* AX = S + (size_t)n * n;
  double* E = AX + (size_t)n * n;
  double* XE = E + (size_t)n * n;
  double* Ag = XE + (size_t)n * n;
  double* lam = Ag + (size_t)n * n;
  double* sums = lam + n;
  const double* Ain = A;
  if (!refine_only) {
  if (Vguess) {
    // warm start: diagonalise Vg^T A Vg and rotate back
    GemmArgs g1;
    g1.M = n; g1.N = n; g1.K = n; g1.A = A; g1.lda = n; g1.B = Vguess; g1.ldb = n; g1.C = AX; g1.ldc = n;
    dgemm(la, g1);
    GemmArgs g2;
    g2.M = n; g2.N = n; g2.K = n; g2.A = Vguess; g2.lda = n; g2.transA = true; g2.B = AX; g2.ldb = n;
    g2.C = Ag; g2.ldc = n;
    dgemm(la, g2);
    Ain = Ag;
  }
  size_t smem = (size_t)n * n * sizeof(float);
  int use_smem = smem <= 215 * 1024 ? 1 : 0;
  // a looser stop (n eps) leaves close clusters too coarse for the FP64
  // refinement to separate
  const float tol = 2e-6f;
  const int hb = (n + kJB - 1) / kJB;   // block width of the block kernel
  if (n > kBlockJacobiMin) {
    block_jacobi_2stage(la, Ain, n, V, W, ws + eig_workspace_base(n), max_sweeps, tol, R, S, AX, E, XE, lam);
  } else {
  if (hb <= 3) {
    const void* fn = hb == 1 ? (const void*)jacobi1s_block_kernel<1>
                   : hb == 2 ? (const void*)jacobi1s_block_kernel<2> : (const void*)jacobi1s_block_kernel<3>;
    if (use_smem) raise_smem_limit(fn, (int)smem);
    const int sz = use_smem ? (int)smem : 0;
    if (hb == 1)
      jacobi1s_block_kernel<1><<<1, JT, sz, la.stream>>>(Ain, n, m, fA, fV, fW, use_smem, max_sweeps, tol);
    else if (hb == 2)
      jacobi1s_block_kernel<2><<<1, JT, sz, la.stream>>>(Ain, n, m, fA, fV, fW, use_smem, max_sweeps, tol);
    else
      jacobi1s_block_kernel<3><<<1, JT, sz, la.stream>>>(Ain, n, m, fA, fV, fW, use_smem, max_sweeps, tol);
  } else {
    if (use_smem) raise_smem_limit((const void*)jacobi1s_kernel, (int)smem);
    jacobi1s_kernel<<<1, JT, use_smem ? smem : 0, la.stream>>>(Ain, n, m, fA, fV, fW, use_smem, max_sweeps, tol);
  }
  RIHF_LAUNCH_CHECK();
  count(la);
  eig_sort_kernel<<<std::min(n, 32), 256, 0, la.stream>>>(fV, fW, n, m, V, W);
  RIHF_LAUNCH_CHECK();
  count(la);
  }   // one-CTA Jacobi
  if (Vguess) {
    // V <- Vguess * V
    GemmArgs g;
    g.M = n; g.N = n; g.K = n; g.A = Vguess; g.lda = n; g.B = V; g.ldb = n; g.C = XE; g.ldc = n;
    dgemm(la, g);
    RIHF_CUDA(cudaMemcpyAsync(V, XE, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, la.stream));
  }
  }   // !refine_only
  for (int it = 0; it < refine; ++it) {
    GemmArgs gr;   // R = V^T V
    gr.M = n; gr.N = n; gr.K = n; gr.A = V; gr.lda = n; gr.transA = true; gr.B = V; gr.ldb = n; gr.C = R; gr.ldc = n;
    dgemm(la, gr);
    i_minus_kernel<<<elem_blocks(la, (long long)n * n), 256, 0, la.stream>>>(R, n);
    RIHF_LAUNCH_CHECK();
    GemmArgs ga;   // AX = A V
    ga.M = n; ga.N = n; ga.K = n; ga.A = A; ga.lda = n; ga.B = V; ga.ldb = n; ga.C = AX; ga.ldc = n;
    dgemm(la, ga);
    GemmArgs gs;   // S = V^T A V
    gs.M = n; gs.N = n; gs.K = n; gs.A = V; gs.lda = n; gs.transA = true; gs.B = AX; gs.ldb = n; gs.C = S; gs.ldc = n;
    dgemm(la, gs);
    oa_lambda_kernel<<<elem_blocks(la, n), 256, 0, la.stream>>>(R, S, n, lam);
    // partial norms in the XE slot (written only by the update GEMM below)
    const int nparts = (int)std::max<long long>(1, std::min<long long>(kOaParts, (long long)n * n / 1024));
    double* part = (long long)n * n >= 3LL * nparts ? XE : sums;   // sums: 8 doubles, enough for one part
    oa_norms_kernel<<<nparts, 256, 0, la.stream>>>(R, S, A, lam, n, part);
    oa_e_kernel<<<elem_blocks(la, (long long)n * n), 256, 0, la.stream>>>(R, S, lam, part, nparts, n, E);
    RIHF_LAUNCH_CHECK();
    GemmArgs ge;   // XE = V E ; V += XE
    ge.M = n; ge.N = n; ge.K = n; ge.A = V; ge.lda = n; ge.B = E; ge.ldb = n; ge.C = XE; ge.ldc = n;
    dgemm(la, ge);
    add_inplace_kernel<<<elem_blocks(la, (long long)n * n), 256, 0, la.stream>>>(V, XE, (long long)n * n);
    RIHF_LAUNCH_CHECK();
    count(la, 5);
  }
  if (refine > 0) {
    RIHF_CUDA(cudaMemcpyAsync(W, lam, sizeof(double) * n, cudaMemcpyDeviceToDevice, la.stream));
    // Newton-Schulz re-orthonormalisation V <- V (3I - V^T V)/2: columns inside
    // near-degenerate clusters are only orthonormalised to first order by the
    // refinement's r_ij/2 rule; two quadratic steps take V^T V to I.
    for (int it = 0; it < ns_steps; ++it) {
      GemmArgs gr;
      gr.M = n; gr.N = n; gr.K = n; gr.A = V; gr.lda = n; gr.transA = true; gr.B = V; gr.ldb = n; gr.C = R;
      gr.ldc = n; gr.alpha = -0.5;
      dgemm(la, gr);
      identity(la, E, n);
      axpby(la, n * n, 1.0, R, 1.5, E, R);
      GemmArgs gv;
      gv.M = n; gv.N = n; gv.K = n; gv.A = V; gv.lda = n; gv.B = R; gv.ldb = n; gv.C = XE; gv.ldc = n;
      dgemm(la, gv);
      RIHF_CUDA(cudaMemcpyAsync(V, XE, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, la.stream));
    }
  }
}

// ------------------------------------------------------------ elementwise

__global__ void axpby_kernel(long long n, double a, const double* x, double b, const double* y, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}
void axpby(const LaCtx& la, int n, double a, const double* x, double b, const double* y, double* out) {
  axpby_kernel<<<elem_blocks(la, n), 256, 0, la.stream>>>(n, a, x, b, y, out);
  RIHF_LAUNCH_CHECK();
  count(la);
}

__global__ void add3_kernel(long long n, const double* x, const double* y, const double* z, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = x[i] + y[i] + z[i];
}
void add3(const LaCtx& la, int n, const double* x, const double* y, const double* z, double* out) {
  add3_kernel<<<elem_blocks(la, n), 256, 0, la.stream>>>(n, x, y, z, out);
  RIHF_LAUNCH_CHECK();
  count(la);
}

// Deterministic single-block reductions (n up to a few million).
__global__ void dot_kernel(long long n, const double* x, const double* y, double* out) {
  __shared__ double r[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * y[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) r[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; ++w) t += r[w];
    *out = t;
  }
}
void dot(const LaCtx& la, int n, const double* x, const double* y, double* out) {
  dot_kernel<<<1, 1024, 0, la.stream>>>(n, x, y, out);
  RIHF_LAUNCH_CHECK();
  count(la);
}

__global__ void scale_copy_kernel(long long n, double a, const double* x, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i];
}
void scale_copy(const LaCtx& la, int n, double a, const double* x, double* out) {
  scale_copy_kernel<<<elem_blocks(la, n), 256, 0, la.stream>>>(n, a, x, out);
  RIHF_LAUNCH_CHECK();
  count(la);
}

__global__ void antisym_kernel(const double* A, double* C, int n) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / n), j = (int)(idx % n);
    C[idx] = A[idx] - A[(size_t)j * n + i];
  }
}
void antisym(const LaCtx& la, const double* A, double* C, int n) {
  antisym_kernel<<<elem_blocks(la, (long long)n * n), 256, 0, la.stream>>>(A, C, n);
  RIHF_LAUNCH_CHECK();
  count(la);
}

__global__ void copy_cols_kernel(const double* src, int nrows, int ld, int ncol, double s, double* dst) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)nrows * ncol;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx / ncol), j = (int)(idx % ncol);
    dst[idx] = s * src[(size_t)i * ld + j];
  }
}
void copy_cols(const LaCtx& la, const double* src, int nrows, int ld, int ncol, double s, double* dst) {
  copy_cols_kernel<<<elem_blocks(la, (long long)nrows * ncol), 256, 0, la.stream>>>(src, nrows, ld, ncol, s, dst);
  RIHF_LAUNCH_CHECK();
  count(la);
}

__global__ void transpose_kernel(const double* __restrict__ src, int rows, int cols, double* __restrict__ dst) {
  __shared__ double t[32][33];
  int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = r0 + r, j = c0 + threadIdx.x;
    t[r][threadIdx.x] = (i < rows && j < cols) ? src[(size_t)i * cols + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = c0 + r, j = r0 + threadIdx.x;   // dst row i (source column), dst column j (source row)
    if (i < cols && j < rows) dst[(size_t)i * rows + j] = t[threadIdx.x][r];
  }
}
void transpose(const LaCtx& la, const double* src, int rows, int cols, double* dst) {
  transpose_kernel<<<dim3(ceil_div(cols, 32), ceil_div(rows, 32)), dim3(32, 8), 0, la.stream>>>(src, rows, cols, dst);
  RIHF_LAUNCH_CHECK();
  count(la);
}

__global__ void scale_cols_kernel(const double* X, const double* v, int nrows, int ncol, double* out) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)nrows * ncol;
       idx += (long long)gridDim.x * blockDim.x)
    out[idx] = X[idx] * v[idx % ncol];
}
void scale_cols(const LaCtx& la, const double* X, const double* v, int nrows, int ncol, double* out) {
  scale_cols_kernel<<<elem_blocks(la, (long long)nrows * ncol), 256, 0, la.stream>>>(X, v, nrows, ncol, out);
  RIHF_LAUNCH_CHECK();
  count(la);
}

}  // namespace rihf
