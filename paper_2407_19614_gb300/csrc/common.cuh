// Shared device/host helpers of librihf (no method arithmetic here).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>

namespace rihf {

// Maximum angular momenta supported by the integral kernels.
constexpr int kMaxLPrim = 3;   // f on the primary basis
constexpr int kMaxLAux = 4;    // g on the auxiliary basis
constexpr int kMaxPrim = 16;   // primitives per contracted shell

struct CudaError : std::runtime_error {
  explicit CudaError(const std::string& s) : std::runtime_error(s) {}
};
struct RihfError : std::runtime_error {
  int code;
  RihfError(int c, const std::string& s) : std::runtime_error(s), code(c) {}
};

#define RIHF_CUDA(call)                                                                     \
  do {                                                                                      \
    cudaError_t _e = (call);                                                                \
    if (_e != cudaSuccess)                                                                  \
      throw ::rihf::CudaError(std::string(#call) + ": " + cudaGetErrorString(_e) + " at " + \
                              __FILE__ + ":" + std::to_string(__LINE__));                  \
  } while (0)

#define RIHF_LAUNCH_CHECK() RIHF_CUDA(cudaGetLastError())

// Raise (never lower) a kernel's dynamic shared-memory limit.  The attribute
// is process-wide, so contexts driven from several host threads must not set
// it back below a size another thread is about to launch with; serialised.
void raise_smem_limit(const void* kernel, int bytes);

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int nsph(int l) { return 2 * l + 1; }
// Number of Cartesian components of all shells 0..l-1 (offset of shell l in a
// concatenated list ordered by l).
__host__ __device__ constexpr int cart_offset(int l) { return l * (l + 1) * (l + 2) / 6; }
// Index of (lx, ly, lz) inside a Cartesian shell ordered lx = l..0, ly = l-lx..0.
__host__ __device__ inline int cart_index(int l, int lx, int ly) {
  int a = l - lx;
  return a * (a + 1) / 2 + (a - ly);
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace rihf
