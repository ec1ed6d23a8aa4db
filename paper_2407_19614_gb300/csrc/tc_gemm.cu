// BF16 digit-plane GEMM on the 5th-generation tensor cores (tcgen05 + TMEM),
// operands staged in shared memory by bulk asynchronous copies.  See
// tc_gemm.cuh for the number format.
#include <algorithm>

#include "../../include/rihf.h"
#include "tc_gemm.cuh"

namespace rihf {

namespace {

constexpr int kOzThreads = 256;                                  // slicing kernel
constexpr int kPlaneElems = kOzTileM * kOzChunk;                // 4096 BF16 = 8 KB
constexpr int kMaxChunksPerBlock = kOzMaxChunksPerBlock;
constexpr int kCoreK = kOzChunk / 8;                             // core matrices along K per chunk
constexpr unsigned long long kWaitNs = 2000000000ULL;     // bounded waits: 2 s

// ------------------------------------------------------------ PTX wrappers

__device__ inline uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Spin on an mbarrier phase with a wall-clock limit; false when it ran out.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ inline void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ inline void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A (smem) . B (smem)^T [+ D], BF16 inputs, FP32 accumulator.
__device__ inline void mma_bf16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ inline void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// 32 lanes x 8 consecutive 32-bit columns; thread i gets lane (base + i).
__device__ inline void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}

__device__ inline void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major core matrices of
// 8 rows x 16 bytes: 128 B between K-adjacent core matrices (leading byte
// offset), kCoreK * 128 B between 8-row groups (stride byte offset), version 1.
__device__ inline uint64_t smem_desc(uint32_t addr) {
  const uint64_t base = ((uint64_t)(128 >> 4) << 16) | ((uint64_t)((kCoreK * 128) >> 4) << 32) | (1ULL << 46);
  return base | (uint64_t)((addr & 0x3FFFF) >> 4);
}

// ------------------------------------------------------------ number format

// x as a signed fixed-point integer V = x * 2^{1077 - E} (|V| < 2^55 when E is
// the largest biased exponent of the block), rounded to nearest.
__device__ inline long long oz_fixed(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  if (e == 0 || E == 0) return 0;
  const long long mant = (long long)((bits & ((1ULL << 52) - 1)) | (1ULL << 52));
  const int sh = E - e - 2;
  long long V;
  if (sh < 0) V = mant << (-sh);
  else if (sh == 0) V = mant;
  else if (sh < 62) V = (mant + (1LL << (sh - 1))) >> sh;
  else V = 0;
  return (bits >> 63) ? -V : V;
}

// BF16 bit pattern of a small integer |d| <= 256 (exact).
__device__ inline uint32_t bf16_of_int(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

// S * 2^e2 as the nearest double (integer construction, no FP64 arithmetic).
__device__ inline double oz_to_double(long long S, int e2) {
  if (S == 0) return 0.0;
  const unsigned long long sign = S < 0 ? (1ULL << 63) : 0ULL;
  const unsigned long long a = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  const int lz = __clzll((long long)a);
  const unsigned long long n = a << lz;
  unsigned long long m = n >> 11;
  const unsigned long long rem = n & 0x7FF;
  if (rem > 0x400 || (rem == 0x400 && (m & 1))) ++m;
  int ex = 63 - lz + e2;
  if (m >> 53) {
    m >>= 1;
    ++ex;
  }
  const int be = ex + 1023;
  if (be <= 0) return 0.0;
  if (be >= 2047) return __longlong_as_double((long long)(sign | (0x7FFULL << 52)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (m & ((1ULL << 52) - 1))));
}

// ------------------------------------------------------------ slicing

// Both passes run one thread per (row, chunk, lane j): a kCoreK-lane group per
// row, lane j owning K elements 8j..8j+7 of the chunk (blockIdx.y = chunk).
// Element (r, k) of the operand is X[r*s_r + (k % KR)*s_k1 + (k / KR)*s_k2].
struct OzSrc {
  const double* X;
  int rows, K;
  long long s_r, s_k1, s_k2;
  int KR;
  int RR;             // > 0: rows split as (r % RR, r / RR) with strides s_r, s_r2
  long long s_r2;
  int PN;             // > 0: pair-packed symmetric PN x PN matrices, s_r2 apart:
                      // row r = (matrix r / PN, mu = r % PN), column k = nu
};

__device__ inline double oz_load(const OzSrc& S, int r, int k) {
  if (r >= S.rows || k >= S.K) return 0.0;
  if (S.PN > 0) {
    const int mu = r % S.PN;
    const long long a = mu > k ? mu : k, b = mu > k ? k : mu;
    return S.X[(long long)(r / S.PN) * S.s_r2 + a * (a + 1) / 2 + b];
  }
  const int q = k / S.KR, m = k - q * S.KR;
  const long long ro = S.RR > 0 ? (long long)(r % S.RR) * S.s_r + (long long)(r / S.RR) * S.s_r2 : (long long)r * S.s_r;
  return S.X[ro + (long long)m * S.s_k1 + (long long)q * S.s_k2];
}

// exps[r * nkb + kb] = largest biased exponent of row r over K block kb
// (exps zeroed before; atomicMax is order-independent).
__global__ void __launch_bounds__(kOzThreads) oz_emax_kernel(OzSrc S, int kb_chunks, int nkb, int* __restrict__ exps) {
  const int tid = threadIdx.x;
  const int r = blockIdx.x * (kOzThreads / kCoreK) + tid / kCoreK;
  const int j = tid % kCoreK;
  const int c = blockIdx.y;
  int emax = 0;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const double x = oz_load(S, r, c * kOzChunk + 8 * j + e);
    emax = max(emax, (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF));
  }
#pragma unroll
  for (int o = 1; o < kCoreK; o <<= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if (j == 0 && r < S.rows && emax > 0) atomicMax(exps + (size_t)r * nkb + c / kb_chunks, emax);
}

// The digits of chunk c of row r relative to its block exponent.
__global__ void __launch_bounds__(kOzThreads) oz_slice_kernel(OzSrc S, int kchunks, int smax, int kb_chunks, int nkb,
                                                              const int* __restrict__ exps,
                                                              uint16_t* __restrict__ planes) {
  const int tid = threadIdx.x;
  const int r = blockIdx.x * (kOzThreads / kCoreK) + tid / kCoreK;
  const int j = tid % kCoreK;
  const int c = blockIdx.y;
  const int emax = exps[(size_t)r * nkb + c / kb_chunks];
  long long V[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) V[e] = oz_fixed(oz_load(S, r, c * kOzChunk + 8 * j + e), emax);
  const int rt = r / kOzTileM, rr = r % kOzTileM;
  uint16_t* dst =
      planes + ((size_t)rt * kchunks + c) * smax * kPlaneElems + (rr / 8) * (kCoreK * 64) + j * 64 + (rr % 8) * 8;
  for (int t = 0; t < smax; ++t) {
    const int p = 48 - 8 * t;
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      int d0, d1;
      if (p > 0) {
        d0 = (int)((V[e] + (1LL << (p - 1))) >> p);
        d1 = (int)((V[e + 1] + (1LL << (p - 1))) >> p);
        V[e] -= (long long)d0 << p;
        V[e + 1] -= (long long)d1 << p;
      } else {
        d0 = (int)V[e];
        d1 = (int)V[e + 1];
        V[e] = V[e + 1] = 0;
      }
      w[e / 2] = bf16_of_int(d0) | (bf16_of_int(d1) << 16);
    }
    *reinterpret_cast<uint4*>(dst + (size_t)t * kPlaneElems) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ------------------------------------------------------------ GEMM
//
// Persistent, warp-specialised kernel (one CTA per SM: it holds all 512 TMEM
// columns).  Work items are (row tile, column tile, K block) triples taken from
// a global counter, so tiles that the symmetry options skip cost nothing and
// the SMs stay balanced.
//   warp 9 (one lane): takes items, streams their K chunks' digit planes into
//     a ring of shared-memory stages with bulk copies;
//   warp 8 (one lane): issues the MMAs of each chunk, diagonal by diagonal, and
//     commits stage releases and, every G chunks, a full accumulator group;
//   warps 0-7: drain the s TMEM accumulators of each group (a row and half the
//     columns per thread) into int64 fixed-point sums; each diagonal is
//     released (its own mbarrier) as soon as it is in registers, so the next
//     group's MMAs on it overlap the conversion of the rest.
// A group spans G = floor(1024 / s) / kOzChunk chunks: every diagonal sum then
// stays below s * 32G * 128^2 <= 2^24 and is exact in FP32.  Every wait is
// bounded; the first one that runs out raises a shared abort flag, all roles
// leave, the copies and MMAs still in flight are awaited (bounded) and
// la.flag[1] is set.

constexpr int kGemmThreads = 320;
constexpr int kDrainThreads = 256;
constexpr int kMaxStages = 4;
constexpr int kItemSlots = 2;
constexpr int kTmemCols = 512;
constexpr int kSmemMax = 227 * 1024;
constexpr int kSmemMin = 116 * 1024;   // more than half an SM's shared memory: one CTA per SM
constexpr int kBookBytes = 1024;

// One MMA of a K chunk, precomputed: TMEM column offset (bit 31: the MMA
// starts its accumulator when the chunk opens a group), A and B descriptor
// address offsets in 16-byte units, instruction descriptor.
constexpr int kMaxChunkMmas = 32;

struct OzBook {
  uint4 mmas[kMaxChunkMmas];
  uint64_t full[kMaxStages], empty[kMaxStages];
  uint64_t accfull, accempty[kOzMaxDigits];
  uint64_t item_full[kItemSlots], item_empty[kItemSlots];
  int item[kItemSlots];
  uint32_t tslot;
  int abort;
  int issued, consumed;
  int dwait[2];        // the drain poller's wait results, alternating slots
};
static_assert(sizeof(OzBook) <= kBookBytes, "bookkeeping block");

struct OzTiling {
  int M, N, TN, mtiles, ntiles, nsplit, nitems, nfast;
  int lower_only, symcols, kb_chunks, kchunks;
  int s, G, nst, stage_bytes;
};

__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Wait for a phase; false if the shared abort flag is up or the time ran out
// (which raises the flag).
__device__ inline bool oz_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > kWaitNs) {
      *abort = 1;
      return false;
    }
  }
}

__device__ inline void oz_decode(const OzTiling& T, int idx, int& mt, int& nt, int& split, int& c0, int& c1) {
  split = idx % T.nsplit;
  const int tile = idx / T.nsplit;
  if (T.nfast) {
    nt = tile % T.ntiles;
    mt = tile / T.ntiles;
  } else {
    mt = tile % T.mtiles;
    nt = tile / T.mtiles;
  }
  c0 = split * T.kb_chunks;
  c1 = min(c0 + T.kb_chunks, T.kchunks);
}

// Whether an item has work: a non-empty K range, a tile that meets the lower
// triangle (lower_only), a column tile with a needed column (symcols).
__device__ inline bool oz_valid(const OzTiling& T, int mt, int nt, int c0, int c1) {
  if (c0 >= c1) return false;
  if (T.lower_only && mt * kOzTileM + kOzTileM - 1 < nt * T.TN) return false;
  if (T.symcols > 0) {
    // columns n = a * symcols + b are needed when b <= a; a range inside one
    // a holds b from n0 % symcols up, a range across two holds b = 0
    const int n0 = nt * T.TN, n1 = min(n0 + T.TN, T.N) - 1;
    const int a0 = n0 / T.symcols;
    if (n1 / T.symcols == a0 && n0 % T.symcols > a0) return false;
  }
  return true;
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    oz_gemm_kernel(OzOperand A, OzOperand B, OzTiling T, double alpha, double* C, long long MR, long long cs_m1,
                   long long cs_m2, long long cs_n, int atomic, int* flag, int* sched) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  OzBook* bk = reinterpret_cast<OzBook*>(smem + (size_t)T.nst * T.stage_bytes);
  volatile int* abort = &bk->abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = T.s, TN = T.TN;
  const uint32_t a_bytes = (uint32_t)s * kPlaneElems * 2, b_plane = (uint32_t)TN * kOzChunk * 2;

  if (tid == 0) {
    for (int i = 0; i < T.nst; ++i) {
      mbar_init(&bk->full[i], 1);
      mbar_init(&bk->empty[i], 1);
    }
    mbar_init(&bk->accfull, 1);
    // one arrival per drain warp (its lane 0, after the warp's reads)
    for (int d = 0; d < kOzMaxDigits; ++d) mbar_init(&bk->accempty[d], kDrainThreads / 32);
    for (int k = 0; k < kItemSlots; ++k) {
      mbar_init(&bk->item_full[k], 1);
      mbar_init(&bk->item_empty[k], kDrainThreads / 32 + 1);
    }
    bk->abort = 0;
    bk->issued = bk->consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) tmem_alloc(&bk->tslot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = bk->tslot;

  if (warp == 9) {
    if (lane == 0) {   // ---------------- producer
      uint32_t i = 0;
      bool ok = true;
      for (int q = 0; ok; ++q) {
        int idx, mt = 0, nt = 0, split = 0, c0 = 0, c1 = 0;
        for (;;) {
          idx = atomicAdd(sched, 1);
          if (idx >= T.nitems) break;
          oz_decode(T, idx, mt, nt, split, c0, c1);
          if (oz_valid(T, mt, nt, c0, c1)) break;
        }
        const int slot = q % kItemSlots;
        if (q >= kItemSlots && !oz_wait(&bk->item_empty[slot], ((q / kItemSlots) - 1) & 1, abort)) break;
        bk->item[slot] = idx < T.nitems ? idx : -1;
        mbar_arrive(&bk->item_full[slot]);
        if (idx >= T.nitems) break;
        const int b_rt = (nt * TN) / kOzTileM, b_off = (nt * TN) % kOzTileM;
        for (int c = c0; c < c1; ++c, ++i) {
          const int st = (int)(i % (uint32_t)T.nst);
          if (i >= (uint32_t)T.nst && !oz_wait(&bk->empty[st], ((i / T.nst) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          uint8_t* As = smem + (size_t)st * T.stage_bytes;
          uint8_t* Bs = As + a_bytes;
          mbar_expect_tx(&bk->full[st], a_bytes + (uint32_t)s * b_plane);
          bulk_load(As, A.planes + ((size_t)mt * A.kchunks + c) * A.smax * kPlaneElems, a_bytes, &bk->full[st]);
          for (int u = 0; u < s; ++u)
            bulk_load(Bs + u * b_plane,
                      B.planes + (((size_t)b_rt * B.kchunks + c) * B.smax + u) * kPlaneElems +
                          (size_t)b_off * kOzChunk,
                      b_plane, &bk->full[st]);
        }
      }
      bk->issued = (int)i;
      // every CTA counts itself once it takes no more items; the last one
      // resets the counters for the next launch on this stream
      __threadfence();
      if (atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
        atomicExch(sched, 0);
        atomicExch(sched + 1, 0);
      }
    }
    __syncwarp();
  } else if (warp == 8) {
    if (lane == 0) {   // ---------------- MMA issuer
      // BF16 x BF16 -> FP32, M = 128; N is set per MMA
      const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzTileM >> 4) << 24);
      const int planes_per_mma = 256 / TN;
      // the MMAs of one chunk: per K step j, A plane t and group of B planes,
      // one MMA; the B planes u = 1..s+1-t lie one after another in shared
      // memory with the same 8-row-group stride, so up to 256 / TN of them form
      // one operand of N = count * TN rows, and the product (t, u) lands on the
      // columns of anti-diagonal t + u.  Built once: the issue loop then costs
      // a table load and two adds per MMA instead of the index arithmetic.
      int nm = 0;
      for (int j = 0; j < kOzChunk / 16; ++j)
        for (int t = 1; t <= s; ++t)
          for (int u0 = 1; u0 <= s + 1 - t; u0 += planes_per_mma) {
            const int np = min(planes_per_mma, s + 2 - t - u0);
            uint4 m;
            m.x = (uint32_t)((t + u0 - 2) * TN) | ((t == 1 && j == 0) ? 0x80000000u : 0u);
            m.y = (uint32_t)(((t - 1) * kPlaneElems * 2 + j * 256) >> 4);
            m.z = (uint32_t)(((u0 - 1) * b_plane + j * 256) >> 4);
            m.w = idesc0 | ((uint32_t)((np * TN) >> 3) << 17);
            if (nm < kMaxChunkMmas) bk->mmas[nm] = m;
            ++nm;
          }
      if (nm > kMaxChunkMmas) {   // cannot happen for s <= 7 and TN >= 16 (at most 28)
        *abort = 1;
        nm = 0;
      }
      uint32_t i = 0, grp = 0;
      int last_st = -1;
      uint32_t last_par = 0;
      bool ok = !*abort;
      for (int q = 0; ok; ++q) {
        const int slot = q % kItemSlots;
        if (!oz_wait(&bk->item_full[slot], (q / kItemSlots) & 1, abort)) break;
        const int idx = *(volatile int*)&bk->item[slot];
        mbar_arrive(&bk->item_empty[slot]);
        if (idx < 0) break;
        int mt, nt, split, c0, c1;
        oz_decode(T, idx, mt, nt, split, c0, c1);
        for (int c = c0; c < c1; ++c, ++i) {
          const int st = (int)(i % (uint32_t)T.nst);
          if (!oz_wait(&bk->full[st], (i / T.nst) & 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const bool first = (c - c0) % T.G == 0, last = (c - c0) % T.G == T.G - 1 || c == c1 - 1;
          if (first && grp > 0) {   // every diagonal of the last group read out
            for (int d = 0; d < s && ok; ++d)
              if (!oz_wait(&bk->accempty[d], (grp - 1) & 1, abort)) ok = false;
            if (!ok) {
              ++i;
              break;
            }
            tc_fence_after();
          }
          // descriptors of the stage's first planes; plane and K-step offsets go
          // into the 14-bit address field (shared addresses stay below 256 KB)
          const uint32_t a_s = smem_addr(smem + (size_t)st * T.stage_bytes);
          const uint64_t a_d0 = smem_desc(a_s), b_d0 = smem_desc(a_s + a_bytes);
#pragma unroll 4
          for (int e = 0; e < nm; ++e) {
            const uint4 m = bk->mmas[e];
            const uint32_t init = (m.x >> 31) & (first ? 1u : 0u);
            mma_bf16(taddr + (m.x & 0x7FFFFFFFu), a_d0 + m.y, b_d0 + m.z, m.w, init ^ 1u);
          }
          mma_commit(&bk->empty[st]);   // the stage is free once these MMAs are done
          last_st = st;
          last_par = (i / T.nst) & 1;
          if (last) {
            mma_commit(&bk->accfull);
            ++grp;
          }
        }
      }
      bk->consumed = (int)i;
      if (*abort && last_st >= 0) mbar_wait(&bk->empty[last_st], last_par);   // MMAs in flight
    }
    __syncwarp();
  } else {   // ---------------- drain: warps 0-7
    const int row = 32 * (warp & 3) + lane;
    const int ncol = TN / 2, col0 = (warp >> 2) * ncol;
    const uint32_t t_row = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
    // one thread polls, the other drain threads wait on a hardware named
    // barrier (spinning 256 threads would compete with the copy and MMA
    // threads for issue slots and for the barrier unit); the poller is lane 0
    // of warp 2, on a scheduler that neither the MMA warp (8) nor the copy
    // warp (9) uses
    int nwait = 0;
    auto drain_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
      const int k = nwait++ & 1;
      if (tid == 64) bk->dwait[k] = oz_wait(bar, parity, abort) ? 1 : 0;
      asm volatile("bar.sync 1, %0;" ::"r"(kDrainThreads) : "memory");
      return *(volatile int*)&bk->dwait[k] != 0;
    };
    uint32_t grp = 0;
    for (int q = 0;; ++q) {
      const int slot = q % kItemSlots;
      bool ok = drain_wait(&bk->item_full[slot], (q / kItemSlots) & 1);
      if (!ok) break;
      const int idx = *(volatile int*)&bk->item[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&bk->item_empty[slot]);
      if (idx < 0) break;
      int mt, nt, split, c0, c1;
      oz_decode(T, idx, mt, nt, split, c0, c1);
      long long acc[kOzMaxTN / 2];
#pragma unroll
      for (int k = 0; k < kOzMaxTN / 2; ++k) acc[k] = 0;
      for (int c = c0; c < c1 && ok; c += T.G) {
        ok = drain_wait(&bk->accfull, grp & 1);
        if (!ok) break;
        tc_fence_after();
        for (int g = 2; g <= s + 1; ++g) {
          const int sh = 37 - 8 * (g - 2);
          const uint32_t tg = t_row + (uint32_t)((g - 2) * TN + col0);
          uint32_t r[kOzMaxTN / 16][8];
#pragma unroll
          for (int q8 = 0; q8 < kOzMaxTN / 16; ++q8)
            if (8 * q8 < ncol) tmem_ld8(tg + 8 * q8, r[q8]);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bk->accempty[g - 2]);
#pragma unroll
          for (int q8 = 0; q8 < kOzMaxTN / 16; ++q8) {
            if (8 * q8 < ncol) {
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const long long v = (long long)__float2int_rn(__uint_as_float(r[q8][e]));
                acc[8 * q8 + e] += sh >= 0 ? (v << sh) : (v >> (-sh));
              }
            }
          }
        }
        ++grp;
      }
      if (!ok) break;
      const long long m = (long long)mt * kOzTileM + row;
      if (m < T.M) {
        // all of the thread's values first (the exponent loads overlap), then
        // the stores: 16-byte pairs when the row is contiguous and aligned
        const int ea = A.exps[(size_t)m * A.nkb + split] - 2095;
        const int n0 = nt * TN + col0;
        const int nv = min(ncol, T.N - n0);
        double v[kOzMaxTN / 2];
#pragma unroll
        for (int k = 0; k < kOzMaxTN / 2; ++k) {
          v[k] = 0.0;
          if (k < nv) {
            v[k] = oz_to_double(acc[k], ea + B.exps[(size_t)(n0 + k) * B.nkb + split]);
            if (alpha != 1.0) v[k] *= alpha;
          }
        }
        double* dst = C + (m % MR) * cs_m1 + (m / MR) * cs_m2 + (long long)n0 * cs_n;
        if (atomic == 1) {
#pragma unroll
          for (int k = 0; k < kOzMaxTN / 2; ++k)
            if (k < nv) atomicAdd(dst + (long long)k * cs_n, v[k]);
        } else if (cs_n == 1 && ((uintptr_t)dst & 15) == 0) {
          double2* d2 = reinterpret_cast<double2*>(dst);
          if (atomic == 2) {
#pragma unroll
            for (int k0 = 0; k0 < kOzMaxTN / 4; k0 += 4) {   // four pairs in flight at a time
              double2 old[4];
#pragma unroll
              for (int k = k0; k < k0 + 4; ++k)
                if (2 * k + 1 < nv) old[k - k0] = d2[k];
#pragma unroll
              for (int k = k0; k < k0 + 4; ++k) {
                if (2 * k + 1 < nv) d2[k] = make_double2(old[k - k0].x + v[2 * k], old[k - k0].y + v[2 * k + 1]);
                else if (2 * k < nv) dst[2 * k] += v[2 * k];
              }
            }
          } else {
#pragma unroll
            for (int k = 0; k < kOzMaxTN / 4; ++k) {
              if (2 * k + 1 < nv) d2[k] = make_double2(v[2 * k], v[2 * k + 1]);
              else if (2 * k < nv) dst[2 * k] = v[2 * k];
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < kOzMaxTN / 2; ++k) {
            if (k < nv) {
              double* d = dst + (long long)k * cs_n;
              if (atomic == 2) *d += v[k];
              else *d = v[k];
            }
          }
        }
      }
    }
  }

  __syncthreads();
  if (*abort) {
    if (warp == 9 && lane == 0) {
      // copies still in flight: chunks issued but never consumed
      for (int i = bk->consumed; i < bk->issued; ++i) mbar_wait(&bk->full[i % T.nst], (i / T.nst) & 1);
    }
    if (tid == 0) atomicOr(flag + 1, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    tmem_dealloc(taddr, kTmemCols);
  }
}

}  // namespace

OzBuf oz_buf_alloc(int rows, int K, int smax, int nkb) {
  return oz_buf_alloc_raw(oz_plane_elems(rows, K, smax),
                          (size_t)((rows + kOzTileM - 1) / kOzTileM) * kOzTileM * std::max(nkb, 1));
}

OzBuf oz_buf_alloc_raw(size_t plane_elems, size_t exp_elems) {
  OzBuf b;
  b.cap = plane_elems;
  b.ecap = exp_elems;
  void* p = nullptr;
  if (cudaMalloc(&p, sizeof(uint16_t) * b.cap) != cudaSuccess) throw RihfError(RIHF_ERR_OOM, "cudaMalloc failed");
  b.planes = static_cast<uint16_t*>(p);
  if (cudaMalloc(&p, sizeof(int) * b.ecap) != cudaSuccess) {
    cudaFree(b.planes);
    throw RihfError(RIHF_ERR_OOM, "cudaMalloc failed");
  }
  b.exps = static_cast<int*>(p);
  return b;
}

void oz_buf_free(OzBuf& b) {
  if (b.planes) cudaFree(b.planes);
  if (b.exps) cudaFree(b.exps);
  b = OzBuf();
}

OzOperand oz_slice(const LaCtx& la, const double* X, int rows, int K, long long s_r, long long s_k1,
                   long long s_k2, int KR, int smax, int kb_chunks, const OzBuf& buf, int RR, long long s_r2,
                   int packed_n) {
  if (rows <= 0 || K <= 0 || smax < 1 || smax > kOzMaxDigits || KR <= 0)
    throw RihfError(RIHF_ERR_INVALID_ARG, "oz_slice: bad arguments");
  uint16_t* planes = buf.planes;
  int* exps = buf.exps;
  OzOperand op;
  op.planes = planes;
  op.exps = exps;
  op.rows = rows;
  op.rows_pad = (rows + kOzTileM - 1) / kOzTileM * kOzTileM;
  op.kchunks = (K + kOzChunk - 1) / kOzChunk;
  op.smax = smax;
  op.kb_chunks = (kb_chunks <= 0 || kb_chunks > op.kchunks) ? op.kchunks : kb_chunks;
  op.nkb = (op.kchunks + op.kb_chunks - 1) / op.kb_chunks;
  if (oz_plane_elems(rows, K, smax) > buf.cap || (size_t)op.rows_pad * op.nkb > buf.ecap)
    throw RihfError(RIHF_ERR_INVALID_ARG, "oz_slice: digit-plane buffer too small");
  if (op.kchunks > 65535) throw RihfError(RIHF_ERR_INVALID_ARG, "oz_slice: K too long");
  if (packed_n > 0 && (K != packed_n || rows % packed_n != 0))
    throw RihfError(RIHF_ERR_INVALID_ARG, "oz_slice: packed rows must be whole matrices");
  OzSrc S{X, rows, K, s_r, s_k1, s_k2, KR, RR, s_r2, packed_n};
  dim3 grid(op.rows_pad / (kOzThreads / kCoreK), op.kchunks);
  RIHF_CUDA(cudaMemsetAsync(exps, 0, sizeof(int) * (size_t)op.rows_pad * op.nkb, la.stream));
  oz_emax_kernel<<<grid, kOzThreads, 0, la.stream>>>(S, op.kb_chunks, op.nkb, exps);
  RIHF_LAUNCH_CHECK();
  oz_slice_kernel<<<grid, kOzThreads, 0, la.stream>>>(S, op.kchunks, smax, op.kb_chunks, op.nkb, exps, planes);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 2;
  return op;
}

void oz_gemm(const LaCtx& la, const OzGemmArgs& g) {
  if (g.M <= 0 || g.N <= 0) return;
  const OzOperand &A = g.A, &B = g.B;
  if (g.s < 1 || g.s > kOzMaxDigits || g.s > A.smax || g.s > B.smax || A.kchunks != B.kchunks ||
      A.kb_chunks != B.kb_chunks || A.nkb != B.nkb || A.rows < g.M || B.rows < g.N)
    throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: operands do not match");
  if (A.kb_chunks > kMaxChunksPerBlock)
    throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: K block longer than the int64 accumulator allows");
  if (!g.atomic && A.nkb > 1) throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: K blocks need atomic output");
  if (g.atomic && g.accumulate) throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: atomic and accumulate");
  if (!la.sched) throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: no work counter");
  // column tile: the whole of N when it fits (multiple of 16), else kOzMaxTN
  // (a divisor of 128, so no tile straddles a 128-row plane)
  OzTiling T;
  T.M = g.M;
  T.N = g.N;
  if (g.tn < 0 || g.tn % 16 || g.tn > kOzMaxTN || (g.tn > 0 && g.N > g.tn && 128 % g.tn))
    throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: bad column tile");
  T.TN = g.tn > 0 ? g.tn : (g.N <= kOzMaxTN ? (g.N + 15) / 16 * 16 : kOzMaxTN);
  T.s = g.s;
  if (T.s * T.TN > kTmemCols) throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: accumulators exceed TMEM");
  T.mtiles = (g.M + kOzTileM - 1) / kOzTileM;
  T.ntiles = (g.N + T.TN - 1) / T.TN;
  T.nsplit = A.nkb;
  const long long nitems = (long long)T.mtiles * T.ntiles * T.nsplit;
  if (nitems >= (1LL << 30)) throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: too many tiles");
  T.nitems = (int)nitems;
  T.nfast = g.M > g.N ? 1 : 0;   // items next to each other share the larger operand's tile
  T.lower_only = g.lower_only ? 1 : 0;
  T.symcols = g.symcols;
  T.kb_chunks = A.kb_chunks;
  T.kchunks = A.kchunks;
  T.G = std::max(1, (1024 / T.s) / kOzChunk);
  T.stage_bytes = T.s * (kPlaneElems * 2 + T.TN * kOzChunk * 2);
  T.nst = std::min(kMaxStages, (kSmemMax - kBookBytes - 1024) / T.stage_bytes);
  if (T.nst < 1) throw RihfError(RIHF_ERR_INVALID_ARG, "oz_gemm: stage exceeds shared memory");
  const int smem = std::max(kSmemMin, T.nst * T.stage_bytes + kBookBytes + 1024);
  raise_smem_limit((const void*)oz_gemm_kernel, kSmemMax);
  const int grid = (int)std::min<long long>(nitems, la.sms > 0 ? la.sms : 152);
  oz_gemm_kernel<<<grid, kGemmThreads, smem, la.stream>>>(A, B, T, g.alpha, g.C, g.MR, g.cs_m1, g.cs_m2, g.cs_n,
                                                          g.atomic ? 1 : (g.accumulate ? 2 : 0), la.flag, la.sched);
  RIHF_LAUNCH_CHECK();
  if (la.launches) *la.launches += 1;
}

}  // namespace rihf
