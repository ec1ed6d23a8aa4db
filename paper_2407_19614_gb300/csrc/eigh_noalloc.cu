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

static __device__ __align__(256) double g_eigh_scratch[kScratch];

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
    return RIHF_OK;
  } catch (const CudaError&) {
    return RIHF_ERR_CUDA;
  } catch (...) {
    return RIHF_ERR_INVALID_ARG;
  }
}
