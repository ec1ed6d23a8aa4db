// rihf_eigh_noalloc: the library's symmetric eigensolver for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc: an MD engine or plugin that owns a
// fixed, pre-reserved memory pool and forbids allocations once its time loop has
// started, or a host process whose device allocation is capped by its framework.
// For them this entry point takes device pointers for its input and outputs and
// uses, as workspace, a fixed array in this file's device memory instead of
// allocating one.  The array is a file-scope __device__ variable, so every GPU
// that loads the library holds it (about 7.9 MB) until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/rihf.h"
#include "common.cuh"
#include "linalg.cuh"

using namespace rihf;

namespace {

// Largest matrix order the fixed workspace supports.
constexpr int kNoAllocMaxN = 256;
// Eigen-decomposition workspace for n = kNoAllocMaxN and the split-K partial
// sums of its GEMMs (8 n^2 doubles), plus a small tail for the error flag.
constexpr size_t kEigWs = eig_workspace(kNoAllocMaxN);
constexpr size_t kWork = 8 * (size_t)kNoAllocMaxN * kNoAllocMaxN;
// every order the entry point accepts fits: the workspace grows with n
static_assert(eig_workspace(kNoAllocMaxN - 1) <= kEigWs && eig_workspace(kNoAllocMaxN) <= kEigWs,
              "fixed eigensolver workspace smaller than eig_workspace(kNoAllocMaxN)");
constexpr size_t kScratch = kEigWs + kWork + 64;
// the check after the solve keeps A V and V^T V in the eigensolver's workspace
static_assert(2 * (size_t)kNoAllocMaxN * kNoAllocMaxN <= kEigWs, "workspace for the residual check");

static __device__ __align__(256) double g_eigh_scratch[kScratch];

// One block: out[0] = max_ij |(A V)_ij - V_ij W_j|, out[1] = max_ij |(V^T V)_ij -
// delta_ij|, out[2] = max_j |W_j|.
__global__ void __launch_bounds__(256) eig_residual_kernel(const double* __restrict__ AV, const double* __restrict__ V,
                                                           const double* __restrict__ W,
                                                           const double* __restrict__ VtV, int n, double* out) {
  double r = 0.0, o = 0.0, w = 0.0;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - (idx / n) * n;
    r = fmax(r, fabs(AV[idx] - V[idx] * W[j]));
    o = fmax(o, fabs(VtV[idx] - (i == j ? 1.0 : 0.0)));
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) w = fmax(w, fabs(W[j]));
  __shared__ double sh[3][256];
  sh[0][threadIdx.x] = r;
  sh[1][threadIdx.x] = o;
  sh[2][threadIdx.x] = w;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = fmax(sh[q][threadIdx.x], sh[q][threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) out[q] = sh[q][0];
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};   // device address of g_eigh_scratch, per device
int g_sms[kMaxDevices] = {};

}  // namespace

extern "C" int rihf_eigh_noalloc(int n, const double* A, double* W, double* V, void* stream) {
  try {
    if (n <= 0 || !A || !W || !V) return RIHF_ERR_INVALID_ARG;
    if (n > kNoAllocMaxN) return RIHF_ERR_INVALID_ARG;   // beyond the fixed workspace
    int dev = 0;
    RIHF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return RIHF_ERR_INVALID_ARG;
    double* scratch = nullptr;
    int sms = 0;
    {
      // First call on a device: resolve the device address of the array with
      // that device current.  In host code g_eigh_scratch names a host-side
      // stand-in, never a device address.
      std::lock_guard<std::mutex> lock(g_mutex);
      if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_eigh_scratch);
        if (e != cudaSuccess || !p) return RIHF_ERR_CUDA;
        int s = 0;
        e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return RIHF_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
        g_sms[dev] = s;
      }
      scratch = g_scratch_ptr[dev];
      sms = g_sms[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* ws = scratch;
    double* work = scratch + kEigWs;
    int* flag = reinterpret_cast<int*>(scratch + kEigWs + kWork);
    // the array keeps the previous call's contents; the flag must start at zero
    // (every other workspace entry is written before it is read)
    RIHF_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    LaCtx la;
    la.stream = s;
    la.work = work;
    la.work_elems = kWork;
    la.sms = sms > 0 ? sms : 152;
    la.flag = flag;
    eigh(la, A, n, W, V, ws, 4, nullptr);
    // Outside stream capture: wait for the result and check it (a Jacobi
    // pass that stopped at its sweep limit, or a refinement that did not
    // converge, shows here).  The eigensolver's workspace is free again and
    // holds A V and V^T V; the three maxima go to the array's tail.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    RIHF_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return RIHF_OK;
    double* AV = ws;
    double* VtV = ws + (size_t)n * n;
    double* res = scratch + kEigWs + kWork + 8;
    GemmArgs g1;   // A V
    g1.M = n; g1.N = n; g1.K = n; g1.A = A; g1.lda = n; g1.B = V; g1.ldb = n; g1.C = AV; g1.ldc = n;
    dgemm(la, g1);
    GemmArgs g2;   // V^T V
    g2.M = n; g2.N = n; g2.K = n; g2.A = V; g2.lda = n; g2.transA = true; g2.B = V; g2.ldb = n; g2.C = VtV;
    g2.ldc = n;
    dgemm(la, g2);
    eig_residual_kernel<<<1, 256, 0, s>>>(AV, V, W, VtV, n, res);
    RIHF_LAUNCH_CHECK();
    double h[3] = {0.0, 0.0, 0.0};
    RIHF_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    // bounds with room above the refined decomposition (residual ~1e-13 of
    // max|W|, orthonormality ~1e-15) and far below an unconverged one
    if (!(h[0] <= 1e-9 * std::max(h[2], 1e-300) * n) || !(h[1] <= 1e-9 * n)) return RIHF_ERR_NOT_CONVERGED;
    return RIHF_OK;
  } catch (const CudaError&) {
    return RIHF_ERR_CUDA;
  } catch (...) {
    return RIHF_ERR_INVALID_ARG;
  }
}
