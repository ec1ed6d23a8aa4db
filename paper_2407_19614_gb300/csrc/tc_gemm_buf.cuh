// Sizes and device storage of BF16 digit planes for the tensor-core GEMM of
// tc_gemm.cuh (kept apart so the dense linear algebra can hold such buffers).
#pragma once
#include <cstddef>
#include <cstdint>

namespace rihf {

constexpr int kOzChunk = 32;        // K elements per chunk (one smem stage)
constexpr int kOzTileM = 128;       // rows per operand tile (UMMA M)
constexpr int kOzMaxDigits = 7;
constexpr int kOzMaxTN = 64;        // columns per output tile (TMEM: 7 x 64 of 512)
constexpr int kOzMaxChunksPerBlock = 60;   // int64 headroom: chunks * 2^56 < 2^62

// Plane entries for `rows` x `K` with smax digits (rows padded to the tile).
inline size_t oz_plane_elems(int rows, int K, int smax) {
  size_t rp = (size_t)((rows + kOzTileM - 1) / kOzTileM) * kOzTileM;
  size_t kc = (size_t)((K + kOzChunk - 1) / kOzChunk);
  return rp * kc * kOzChunk * smax;
}

// Device storage for the digit planes and exponents of one operand, with its
// capacity (elements); oz_slice refuses a buffer that is too small.
struct OzBuf {
  uint16_t* planes = nullptr;
  size_t cap = 0;
  int* exps = nullptr;
  size_t ecap = 0;
};
// Buffer for up to `rows` x `K` with smax digits and at most nkb K blocks.
OzBuf oz_buf_alloc(int rows, int K, int smax, int nkb);
// Buffer with the given plane and exponent capacities (entries), for one
// buffer that serves operands of different shapes in turn.
OzBuf oz_buf_alloc_raw(size_t plane_elems, size_t exp_elems);
void oz_buf_free(OzBuf& b);

}  // namespace rihf
