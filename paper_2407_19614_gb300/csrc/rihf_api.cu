// librihf C ABI (include/rihf.h): context, setup, SCF (Alg. 1) and gradient
// (Alg. 2) orchestration on one GPU.  All heavy work runs in this library's
// kernels (integrals.cu, grad_integrals.cu, linalg.cu, jk.cu); the host only
// sequences launches and reads two scalars per SCF iteration for the
// convergence test.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <functional>
#include <thread>
#include <vector>

#include "../../include/rihf.h"
#include "common.cuh"
#include "integrals.cuh"
#include "jk.cuh"
#include "linalg.cuh"
#include "os_hgp.cuh"
#include "mlp.cuh"
#include "tc_gemm.cuh"

using namespace rihf;

static thread_local std::string g_last_error;

// ============================================================ host basis

namespace {

double dfact(int n) {   // (n)!! with (-1)!! = 1
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

using Poly = std::vector<double>;   // coefficients over Cartesian monomials of one degree

// Real solid harmonics S_lm (m = -l..l) as polynomials in x, y, z, built by the
// recursions (Helgaker, Joergensen, Olsen, Eqs. 6.4.70-6.4.73).
std::vector<std::vector<Poly>> solid_harmonics(int lmax) {
  std::vector<std::vector<Poly>> S(lmax + 1);
  auto mul = [](const Poly& p, int l, int dx, int dy, int dz) {   // multiply a degree-l poly by x^dx y^dy z^dz
    int L = l + dx + dy + dz;
    Poly out(ncart(L), 0.0);
    for (int k = 0; k < ncart(l); ++k) {
      if (p[k] == 0.0) continue;
      int a = 0;
      while ((a + 1) * (a + 2) / 2 <= k) ++a;
      int lx = l - a, ly = a - (k - a * (a + 1) / 2), lz = l - lx - ly;
      int nx = lx + dx, ny = ly + dy;
      out[cart_index(L, nx, ny)] += p[k];
      (void)lz;
    }
    return out;
  };
  auto axpy = [](Poly& y, double a, const Poly& x) {
    for (size_t i = 0; i < y.size(); ++i) y[i] += a * x[i];
  };
  S[0] = {Poly{1.0}};
  for (int l = 0; l < lmax; ++l) {
    int L = l + 1;
    std::vector<Poly> next(2 * L + 1, Poly(ncart(L), 0.0));
    const Poly& sll = S[l][2 * l];      // m = +l
    const Poly& slml = S[l][0];         // m = -l
    double f = std::sqrt((l == 0 ? 2.0 : 1.0) * (2 * l + 1) / (2.0 * l + 2));
    Poly top = mul(sll, l, 1, 0, 0);
    Poly bot = mul(sll, l, 0, 1, 0);
    if (l > 0) {
      axpy(top, -1.0, mul(slml, l, 0, 1, 0));
      axpy(bot, 1.0, mul(slml, l, 1, 0, 0));
    }
    for (auto& v : top) v *= f;
    for (auto& v : bot) v *= f;
    next[2 * L] = top;   // m = +L
    next[0] = bot;       // m = -L
    for (int m = -l; m <= l; ++m) {
      Poly v = mul(S[l][m + l], l, 0, 0, 1);
      for (auto& c : v) c *= (2 * l + 1);
      if (l >= 1 && std::abs(m) <= l - 1) {
        const Poly& lo = S[l - 1][m + l - 1];
        Poly r2 = mul(lo, l - 1, 2, 0, 0);
        axpy(r2, 1.0, mul(lo, l - 1, 0, 2, 0));
        axpy(r2, 1.0, mul(lo, l - 1, 0, 0, 2));
        axpy(v, -std::sqrt((double)(l + m) * (l - m)), r2);
      }
      double d = std::sqrt((double)(l + m + 1) * (l - m + 1));
      for (auto& c : v) c /= d;
      next[m + L] = v;
    }
    S[L] = next;
  }
  return S;
}

// Self-overlap of sum_a c_a x^a e^{-r^2} relative to that of x^l e^{-r^2}.
double relative_norm(const Poly& c, int l) {
  double s = 0.0;
  for (int a = 0; a < ncart(l); ++a)
    for (int b = 0; b < ncart(l); ++b) {
      if (c[a] == 0.0 || c[b] == 0.0) continue;
      int ia = 0;
      while ((ia + 1) * (ia + 2) / 2 <= a) ++ia;
      int ib = 0;
      while ((ib + 1) * (ib + 2) / 2 <= b) ++ib;
      int ax = l - ia, ay = ia - (a - ia * (ia + 1) / 2), az = l - ax - ay;
      int bx = l - ib, by = ib - (b - ib * (ib + 1) / 2), bz = l - bx - by;
      int n[3] = {ax + bx, ay + by, az + bz};
      if ((n[0] | n[1] | n[2]) & 1) continue;
      s += c[a] * c[b] * dfact(n[0] - 1) * dfact(n[1] - 1) * dfact(n[2] - 1);
    }
  return s / dfact(2 * l - 1);
}

// Transform table kTrL x 15 x 15 and output-function counts.
void build_transforms(bool pure, std::vector<double>& tr, std::vector<int>& nf) {
  tr.assign(kTrL * kTrStride * kTrStride, 0.0);
  nf.assign(kTrL, 0);
  auto S = solid_harmonics(kTrL - 1);
  for (int l = 0; l < kTrL; ++l) {
    double* T = tr.data() + l * kTrStride * kTrStride;
    if (pure) {
      nf[l] = 2 * l + 1;
      for (int m = 0; m < 2 * l + 1; ++m) {
        const Poly& p = S[l][m];
        double nrm = std::sqrt(relative_norm(p, l));
        for (int k = 0; k < ncart(l); ++k) T[m * kTrStride + k] = p[k] / nrm;
      }
    } else {
      nf[l] = ncart(l);
      for (int k = 0; k < ncart(l); ++k) {
        Poly e(ncart(l), 0.0);
        e[k] = 1.0;
        T[k * kTrStride + k] = 1.0 / std::sqrt(relative_norm(e, l));
      }
    }
  }
}

struct HostShells {
  int nshell = 0, nfunc = 0, lmax = 0;
  std::vector<int> l, atom, nprim, pstart, ao;
  std::vector<double> exps, coefs;
  std::vector<double> raw_coefs;   // the caller's coefficients (before normalisation)
};

// Primitive normalisation of x^l e^{-a r^2} times the caller's coefficient,
// then the contracted function is renormalised.
int build_host_shells(int n, const rihf_shell* sh, int natoms, int lmax_allowed, const std::vector<int>& nf,
                      HostShells& out) {
  out = HostShells();
  out.nshell = n;
  int ao = 0;
  for (int s = 0; s < n; ++s) {
    const rihf_shell& x = sh[s];
    if (x.l < 0 || x.l > lmax_allowed || x.nprim < 1 || x.nprim > kMaxPrim || x.atom < 0 || x.atom >= natoms ||
        !x.exps || !x.coefs)
      return RIHF_ERR_INVALID_ARG;
    out.l.push_back(x.l);
    out.atom.push_back(x.atom);
    out.nprim.push_back(x.nprim);
    out.pstart.push_back((int)out.exps.size());
    out.ao.push_back(ao);
    ao += nf[x.l];
    out.lmax = std::max(out.lmax, x.l);
    std::vector<double> c(x.nprim);
    for (int k = 0; k < x.nprim; ++k) {
      double a = x.exps[k];
      if (!(a > 0.0)) return RIHF_ERR_INVALID_ARG;
      c[k] = x.coefs[k] * std::sqrt(std::pow(4.0 * a, x.l) * std::pow(2.0 * a / M_PI, 1.5) / dfact(2 * x.l - 1));
    }
    double norm = 0.0;
    for (int i = 0; i < x.nprim; ++i)
      for (int j = 0; j < x.nprim; ++j) {
        double p = x.exps[i] + x.exps[j];
        norm += c[i] * c[j] * std::pow(M_PI / p, 1.5) * dfact(2 * x.l - 1) / std::pow(2.0 * p, x.l);
      }
    double f = 1.0 / std::sqrt(norm);
    for (int k = 0; k < x.nprim; ++k) {
      out.exps.push_back(x.exps[k]);
      out.coefs.push_back(c[k] * f);
      out.raw_coefs.push_back(x.coefs[k]);
    }
  }
  out.nfunc = ao;
  return RIHF_OK;
}

template <typename T>
T* dalloc(size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) throw RihfError(RIHF_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes");
  return (T*)p;
}

template <typename T>
void upload(T* d, const std::vector<T>& h, cudaStream_t s) {
  if (!h.empty()) RIHF_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

}  // namespace

// ============================================================ DIIS kernels

// Pulay system [B -1; -1 0] [c; lambda] = [0; -1], B scaled by its largest
// diagonal entry; Gaussian elimination with partial pivoting (one warp).
__global__ void diis_solve_kernel(const double* __restrict__ Bm, int ld, int m, double* coef) {
  __shared__ double a[17][18];
  int lane = threadIdx.x;
  int n = m + 1;
  double sc = 0.0;
  for (int i = 0; i < m; ++i) sc = fmax(sc, fabs(Bm[i * ld + i]));
  if (sc == 0.0) sc = 1.0;
  for (int i = lane; i < n * n; i += 32) {
    int r = i / n, c = i % n;
    double v;
    if (r < m && c < m) v = Bm[r * ld + c] / sc;
    else if (r == m && c == m) v = 0.0;
    else v = -1.0;
    a[r][c] = v;
  }
  for (int r = lane; r < n; r += 32) a[r][n] = (r == m) ? -1.0 : 0.0;
  __syncwarp();
  for (int k = 0; k < n; ++k) {
    if (lane == 0) {
      int piv = k;
      for (int r = k + 1; r < n; ++r)
        if (fabs(a[r][k]) > fabs(a[piv][k])) piv = r;
      if (piv != k)
        for (int c = 0; c <= n; ++c) {
          double t = a[k][c];
          a[k][c] = a[piv][c];
          a[piv][c] = t;
        }
    }
    __syncwarp();
    double pk = a[k][k];
    for (int r = lane; r < n; r += 32) {
      if (r == k || pk == 0.0) continue;
      double f = a[r][k] / pk;
      for (int c = k; c <= n; ++c) a[r][c] -= f * a[k][c];
    }
    __syncwarp();
  }
  for (int r = lane; r < m; r += 32) coef[r] = a[r][r] != 0.0 ? a[r][n] / a[r][r] : 0.0;
}

__global__ void diis_extrap_kernel(const double* __restrict__ ring, long long len, int m,
                                   const double* __restrict__ coef, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += coef[j] * ring[(long long)j * len + i];
    out[i] = s;
  }
}

// out[0] = max_ij |A_ij - sub * delta_ij| over all i, j (offdiag = 0), over
// i != j (offdiag = 1), or over the block i < offdiag - 1 <= j, i.e. between
// the first (offdiag - 1) indices and the rest (offdiag > 1); one block.
// ---------------------------------------------------------------- multi-block reductions
// Small reductions over n^2 elements spread over kRedBlocks blocks: every block
// leaves a partial in part[], the last block to finish (a ticket counter)
// folds the partials in block order -- deterministic -- and resets the ticket.
constexpr int kRedBlocks = 32;
constexpr int kRedDiis = 8;   // blocks per DIIS dot product
constexpr int kRedSlots = 128;

__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;   // valid in thread 0
}

__device__ inline double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
  return t;
}

// Thread 0 stores the block's result; true in the block that finishes last.
__device__ inline bool red_finish(double v, double* part, int slot, int* ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[slot] = v;
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)(gridDim.x * gridDim.y) - 1;
  }
  __syncthreads();
  return last;
}

// out[0] = 1/2 sum D (h + F) + Vnn (Vnn read from out[5], so graphs stay valid).
__global__ void energy_mb_kernel(const double* __restrict__ D, const double* __restrict__ h,
                                 const double* __restrict__ F, long long n2, double* part, int* ticket,
                                 double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x)
    s += D[i] * (h[i] + F[i]);
  const double b = block_sum(s, red);
  if (red_finish(b, part, blockIdx.x, ticket) && threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) t += __ldcg(part + k);
    out[0] = 0.5 * t + out[5];
    *ticket = 0;
  }
}

// out[0] = max |x_i|
__global__ void maxabs_mb_kernel(long long n, const double* __restrict__ x, double* part, int* ticket, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  const double b = block_max(m, red);
  if (red_finish(b, part, blockIdx.x, ticket) && threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) t = fmax(t, __ldcg(part + k));
    out[0] = t;
    *ticket = 0;
  }
}

// out[0] = max |A_ij - sub delta_ij| over all (i, j) (offdiag 0), i != j
// (offdiag 1), or i < offdiag - 1 <= j (offdiag > 1: an off-diagonal block).
__global__ void eig_check_mb_kernel(const double* __restrict__ A, int n, double sub, int offdiag, double* part,
                                    int* ticket, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (offdiag == 1 && i == j) continue;
    if (offdiag > 1 && !(i < offdiag - 1 && j >= offdiag - 1)) continue;
    m = fmax(m, fabs(A[idx] - (i == j ? sub : 0.0)));
  }
  const double b = block_max(m, red);
  if (red_finish(b, part, blockIdx.x, ticket) && threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) t = fmax(t, __ldcg(part + k));
    out[0] = t;
    *ticket = 0;
  }
}

// Row / column s of the DIIS matrix: Bm[s][j] = Bm[j][s] = <e_s, e_j> for j < m,
// each dot over kRedDiis blocks (blockIdx.x the slice, blockIdx.y = j).
__global__ void diis_dots_mb_kernel(const double* __restrict__ ring, long long len, int s, int m, double* Bm, int ld,
                                    double* part, int* ticket) {
  __shared__ double red[32];
  const int j = blockIdx.y;
  const double* a = ring + (long long)s * len;
  const double* b = ring + (long long)j * len;
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    v += a[i] * b[i];
  const double t = block_sum(v, red);
  if (red_finish(t, part, j * kRedDiis + blockIdx.x, ticket) && threadIdx.x == 0) {
    for (int jj = 0; jj < m; ++jj) {
      double d = 0.0;
      for (int k = 0; k < kRedDiis; ++k) d += __ldcg(part + jj * kRedDiis + k);
      Bm[s * ld + jj] = d;
      Bm[jj * ld + s] = d;
    }
    *ticket = 0;
  }
}

// ============================================================ tracing

struct TraceStat {
  long long launches = 0;
  double ms = 0.0, work = 0.0;
  int kind = 0;
};
struct TracePending {
  std::string name;
  double work;
  int kind;
  cudaEvent_t a, b;
};

struct Tracer {
  bool on = false;
  std::vector<std::pair<std::string, TraceStat>> stats;
  std::vector<TracePending> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (pool.empty()) {
      cudaEvent_t e;
      RIHF_CUDA(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  // Resolve recorded pairs (the stream must be idle).
  void flush() {
    for (auto& p : pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.a, p.b);
      TraceStat* st = nullptr;
      for (auto& kv : stats)
        if (kv.first == p.name) st = &kv.second;
      if (!st) {
        stats.push_back({p.name, TraceStat()});
        st = &stats.back().second;
      }
      st->launches += 1;
      st->ms += ms;
      st->work += p.work;
      st->kind = p.kind;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  ~Tracer() {
    for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// RAII scope: events around one instrumented launch (or fused launch group).
struct TraceScope {
  Tracer* t;
  cudaStream_t s;
  TracePending p;
  TraceScope(Tracer& tr, cudaStream_t st, const char* name, double work, int kind) : t(tr.on ? &tr : nullptr), s(st) {
    if (!t) return;
    p.name = name;
    p.work = work;
    p.kind = kind;
    p.a = t->get();
    p.b = t->get();
    cudaEventRecord(p.a, s);
  }
  ~TraceScope() {
    if (!t) return;
    cudaEventRecord(p.b, s);
    t->pending.push_back(p);
  }
};

// ============================================================ context

struct rihf_ctx {
  Tracer tracer;
  rihf_options opt;
  int natoms = 0, nelec = 0, nocc = 0, N = 0, NA = 0, nind = 0;
  int max_lp = 0, max_la = 0;
  std::vector<int> Z;
  std::vector<double> xyz;
  double vnn = 0.0;
  HostShells hp, ha;
  std::vector<double> tr_h;
  std::vector<int> nf_h;
  std::vector<ShellPair> pairs_h;
  int npairs = 0, npairs_total = 0;

  cudaStream_t stream = nullptr;
  long long launches = 0;
  int sms = 152;

  // device basis
  int *d_pl = nullptr, *d_patom = nullptr, *d_pnprim = nullptr, *d_pps = nullptr, *d_pao = nullptr;
  double *d_pxyz = nullptr, *d_pexp = nullptr, *d_pcoef = nullptr, *d_piexp = nullptr;
  int *d_al = nullptr, *d_aatom = nullptr, *d_anprim = nullptr, *d_aps = nullptr, *d_aao = nullptr;
  double *d_axyz_sh = nullptr, *d_aexp = nullptr, *d_acoef = nullptr, *d_aiexp = nullptr;
  int* d_pp_off = nullptr;        // primitive-pair table offsets per listed shell pair
  PairPrim* d_pp = nullptr;       // primitive-pair data (per geometry)
  double* d_tr = nullptr;
  int* d_nf = nullptr;
  int* d_Z = nullptr;
  double* d_xyz = nullptr;
  double* d_boys = nullptr;
  int* d_counter = nullptr;
  int* d_flag = nullptr;
  int* d_sched = nullptr;   // work counter of the tensor-core GEMM (zero between launches)
  double* d_red = nullptr;  // partials of the multi-block reductions
  int* d_ticket = nullptr;  // their ticket counter (zero between launches)
  ShellPair* d_pairs = nullptr;
  int2* d_tasks = nullptr;           // (pair, auxiliary shell) tasks, grouped by shared-memory class
  TaskGroup groups[kTaskGroups];
  double* d_schwarz = nullptr;
  bool schwarz_ok = false;
  bool schwarz_fresh = false;   // d_schwarz holds Q of the current geometry
  double schwarz_max_dropped = 0.0;

  // geometry-dependent matrices
  double *S = nullptr, *H = nullptr, *Tk = nullptr, *V = nullptr;
  double *A = nullptr, *L = nullptr, *Linv = nullptr;
  // The fitted tensor, pair-packed: Bp[P][tri(mu) + nu] (mu >= nu), Naux x
  // N(N+1)/2 FP64.  The 3-centre integrals are written here and the fit
  // B = L^{-1} T runs in place.  Consumers that need whole N x N slices (the
  // RI-K and gradient products) expand chunks of `pc` auxiliary functions:
  // into Bu (FP64) or straight into digit planes (mixed mode).  When every
  // slice fits at once the expansion is done once per geometry: Bu holds all
  // of B (bu_is_B, FP64 mode) or Bz all of B's 7-digit planes (planes_all).
  long long npp = 0;
  double *Bp = nullptr, *Yp = nullptr, *Bu = nullptr;
  double *Dp = nullptr, *Jp = nullptr;   // packed weighted density and packed J of the RI-J passes
  int pc = 0;
  bool bu_is_B = false, planes_all = false;
  double *Xo = nullptr;     // N x nind orthogonaliser
  double *Sw = nullptr, *Sv = nullptr;

  // SCF
  double *C = nullptr, *eps = nullptr, *Ct = nullptr, *D = nullptr, *J = nullptr, *K = nullptr, *F = nullptr;
  double *Fx = nullptr, *T1 = nullptr, *T2 = nullptr, *Err = nullptr, *Fp = nullptr, *Cp = nullptr, *Hb = nullptr;
  double *dvec = nullptr, *Fring = nullptr, *Ering = nullptr, *Bdiis = nullptr, *coef = nullptr;
  double* scal = nullptr;   // [0] energy, [1] max|err|
  double* Cprev = nullptr;  // previous eigenvectors in the orthonormal basis (warm start)
  bool have_cprev = false;

  // gradient
  double* na2tmp = nullptr;
  // mixed precision: FP32 copy of B and FP32 operands of the SCF-iteration builds
  // mixed precision: BF16 digit planes of B (per geometry), C~^T and H (per
  // build) for the tensor-core RI-K, with their block exponents
  OzBuf Bz, Cz, Hz;
  OzOperand Bop;
  TrsmTcScratch trsm_sc;          // tensor-core fit (mixed mode)
  // tensor-core gradient GEMMs (mixed mode): planes of C~ as a B operand
  // (rows N, K = nocc), of G' (rows Naux N, K = nocc) and of X~ (rows Naux, K = nocc^2)
  OzBuf Ctz, Gz, Xz;
  // mixed mode, N > 256: operand planes for the dense N^3 products routed to
  // the tensor cores by dgemm (DIIS error, orthogonalisation, eigenvector
  // refinement), see LaCtx::tcA
  OzBuf tcA, tcB;
  int tc_builds = 0, confirm_builds = 0, last_iters = 0, last_digits = 0;
  double flops_eri3 = 0.0, flops_grad3 = 0.0;   // algorithmic FP64 operations of the 3-centre kernels
  int k_nsplit = 0;             // K splits of the tensor-core K GEMM (0: not tuned yet)
  int k_tn = 0;                 // its column tile
  // per-iteration CUDA graphs (Fock build + DIIS error), one per variant:
  // [0] FP64 build, [d] tensor-core build with d digits
  struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    long long uses = 0;
  } graphs[kOzMaxDigits + 1];
  // diagonalisation: [refine-only, warm Jacobi, light warm Jacobi] x [F, extrapolated F]
  IterGraph diag_graphs[6];
  bool graphs_ok = true;

  // learned / extrapolated guess: the last three converged densities, the
  // overlap and nuclear positions of the last geometry, features of the
  // current step and the network
  int *d_ao_atom = nullptr, *d_ao_l = nullptr;
  double* hist_D[3] = {nullptr, nullptr, nullptr};   // D_t, D_{t-1}, D_{t-2}
  double* hist_S = nullptr;                          // S_t
  double* hist_xyz[2] = {nullptr, nullptr};          // R_t, R_{t-1}
  int nhist = 0;
  // the history holds Loewdin densities D_L = S^{1/2} D S^{1/2} of their own
  // geometries (from the first extrapolated or learned guess on): S^{1/2},
  // S^{-1/2} of the current geometry (built once per geometry), D_L scratch
  bool hist_lowdin = false;
  double *Shalf = nullptr, *Smhalf = nullptr, *DL = nullptr;
  long long geom_serial = 0, lowdin_serial = -1;
  double* Dpred = nullptr;
  float *mlX = nullptr, *mly = nullptr, *mlt = nullptr;
  double* mlDx = nullptr;
  double* ml_sums = nullptr;                          // feature scale sums (device, 3)
  double ml_sd = 0.0, ml_ss = 0.0, ml_sr = 0.0;       // feature scales, fixed at the first build
  static constexpr int kReplay = 8;                   // training examples kept for replay
  float *rep_X = nullptr, *rep_t = nullptr;
  int nrep = 0, rep_head = 0;
  MlpDev net;
  bool net_on = false, pending_example = false;
  int train_steps = 200, adam_iters = 4, trained_steps = 0, last_guess = 0;
  double ml_lr = 1e-3, ml_scale = 0.0, ml_last_ratio = 1e300;
  double ml_ratios[3] = {1e300, 1e300, 1e300};        // last three out-of-sample ratios
  double* trsm_tmp = nullptr;
  double *cvec = nullptr, *W = nullptr, *Bij = nullptr, *Xt = nullptr, *Zm = nullptr;
  double* G = nullptr;   // the gradient's G' = C~ X~ (shares Hb's memory: H is spent by then)
  double* grad_parts = nullptr;   // 5 x natoms x 3 on device (one, overlap, three, two, nuc)
  std::vector<double> grad_parts_h;

  double* work = nullptr;
  size_t work_elems = 0;
  double* eigws = nullptr;
  double* scratch = nullptr;

  // Occupations: empty = closed shell (2 per occupied orbital, C~ = sqrt(2) C_occ);
  // otherwise n_i per occupied column (C~ = C_occ diag(sqrt(n_i))), as for the
  // spherically averaged atoms of the SAD guess
  std::vector<double> occ;
  double* d_occw = nullptr;
  // SAD guess (guess 5): block-diagonal factor Fs (N x sad_m) of the
  // superposition of atomic densities, D_SAD = Fs Fs^T, built on first use
  double* d_sad = nullptr;
  int sad_m = 0;
  // SAD atoms (spherical basis): every Fock matrix is replaced by its spherical
  // average (per function: first function of its shell, l, m index)
  bool sph_avg = false;
  int *d_fao0 = nullptr, *d_fl = nullptr, *d_fm = nullptr;
  std::vector<int> fl_h;     // l of every basis function (host)
  std::vector<int> occ_l;    // l of each occupied orbital: occupation by configuration, not eigenvalue order
  bool sad_built = false, sad_ok = false;
  std::string sad_note;
  bool converged = false;
  bool have_orbitals = false;
  bool verbose = getenv("RIHF_VERBOSE") != nullptr;
  bool have_linv = false;
  double last_err = 1.0;   // max|e| of the latest SCF iteration
  double prev_err = 1.0;   // and of the one before
  bool force_cold = false; // next diagonalisation: full Jacobi from scratch (SCF stall recovery)
  double timings[5] = {0, 0, 0, 0, 0};
  cudaEvent_t ev[8];

  LaCtx la() const {
    LaCtx l;
    l.stream = stream;
    l.work = work;
    l.work_elems = work_elems;
    l.launches = const_cast<long long*>(&launches);
    l.sms = sms;
    l.flag = d_flag;
    l.sched = d_sched;
    if (tcA.planes) {
      l.tcA = &tcA;
      l.tcB = &tcB;
      l.tc_min_work = 256.0 * 256.0 * 256.0;
    }
    return l;
  }
  IntegralCtx ic() const {
    IntegralCtx c;
    c.boys = d_boys;
    c.counter = d_counter;
    c.stream = stream;
    c.launches = const_cast<long long*>(&launches);
    return c;
  }
  PairTable ptab() const {
    PairTable t;
    t.pp = d_pp;
    t.off = d_pp_off;
    return t;
  }
  DevShells prim() const {
    DevShells s;
    s.nshell = hp.nshell; s.nfunc = N; s.l = d_pl; s.atom = d_patom; s.xyz = d_pxyz; s.nprim = d_pnprim;
    s.pstart = d_pps; s.exps = d_pexp; s.iexps = d_piexp; s.coefs = d_pcoef; s.ao = d_pao; s.tr = d_tr; s.nf = d_nf;
    return s;
  }
  DevShells aux() const {
    DevShells s;
    s.nshell = ha.nshell; s.nfunc = NA; s.l = d_al; s.atom = d_aatom; s.xyz = d_axyz_sh; s.nprim = d_anprim;
    s.pstart = d_aps; s.exps = d_aexp; s.iexps = d_aiexp; s.coefs = d_acoef; s.ao = d_aao; s.tr = d_tr; s.nf = d_nf;
    return s;
  }
};

static const std::vector<double>& boys_host() {
  // built once, thread-safely (function-local static initialisation)
  static const std::vector<double> tab = [] {
    std::vector<double> t((size_t)kBoysN * kBoysM);
    boys_table_host(t.data());
    return t;
  }();
  return tab;
}

// Rebuild the class-grouped 3-centre task lists from the current pair list.
static void refresh_tasks(rihf_ctx* c) {
  upload(c->d_pp_off, pair_prim_offsets(c->pairs_h, c->hp.nprim), c->stream);
  std::vector<std::vector<int2>> tasks;
  std::vector<int> se, sg;
  // largest primitive exponent per primary shell, smallest per auxiliary shell
  std::vector<double> pmax(c->hp.nshell, 0.0), qmin(c->ha.nshell, 0.0);
  for (int i = 0; i < c->hp.nshell; ++i)
    for (int k = 0; k < c->hp.nprim[i]; ++k) pmax[i] = std::max(pmax[i], c->hp.exps[c->hp.pstart[i] + k]);
  for (int i = 0; i < c->ha.nshell; ++i) {
    qmin[i] = c->ha.exps[c->ha.pstart[i]];
    for (int k = 1; k < c->ha.nprim[i]; ++k) qmin[i] = std::min(qmin[i], c->ha.exps[c->ha.pstart[i] + k]);
  }
  build_task_groups(c->pairs_h, c->hp.l, c->hp.nprim, c->ha.l, c->ha.nprim, pmax, qmin, tasks, se, sg);
  task_flops(c->pairs_h, c->hp.l, c->hp.nprim, c->hp.atom, c->ha.l, c->ha.nprim, c->ha.atom, c->nf_h, pmax, qmin,
             &c->flops_eri3, &c->flops_grad3);
  size_t off = 0;
  for (int g = 0; g < kTaskGroups; ++g) {
    c->groups[g].tasks = c->d_tasks + off;
    c->groups[g].ntask = (long long)tasks[g].size();
    c->groups[g].smem_eri3 = se[g];
    c->groups[g].smem_grad = sg[g];
    c->groups[g].width = task_group_width(g);
    upload(c->d_tasks + off, tasks[g], c->stream);
    off += tasks[g].size();
  }
}

static void free_all(rihf_ctx* c) {
  void* ptrs[] = {c->d_pl, c->d_patom, c->d_pnprim, c->d_pps, c->d_pao, c->d_pxyz, c->d_pexp, c->d_pcoef,
                  c->d_al, c->d_aatom, c->d_anprim, c->d_aps, c->d_aao, c->d_axyz_sh, c->d_aexp, c->d_acoef,
                  c->d_piexp, c->d_aiexp, c->d_pp_off, c->d_pp,
                  c->d_ao_atom, c->d_ao_l, c->hist_D[0], c->hist_D[1], c->hist_D[2], c->hist_S, c->hist_xyz[0],
                  c->hist_xyz[1], c->Shalf, c->Smhalf, c->DL, c->Dpred, c->mlX, c->mly, c->mlt, c->mlDx, c->ml_sums, c->rep_X, c->rep_t, c->net.master, c->net.wbf, c->net.grad,
                  c->net.m, c->net.v, c->net.loss,
                  c->d_tr, c->d_nf, c->d_Z, c->d_xyz, c->d_boys, c->d_counter, c->d_flag, c->d_sched, c->d_red, c->d_ticket, c->d_pairs, c->d_tasks, c->d_schwarz,
                  c->S, c->H, c->Tk, c->V, c->A, c->L, c->Linv, c->Bp, c->Yp, c->Bu, c->Dp, c->Jp, c->Xo, c->Sw, c->Sv,
                  c->C, c->eps, c->Ct, c->D, c->J, c->K, c->F, c->Fx, c->T1, c->T2, c->Err, c->Fp, c->Cp, c->Hb,
                  c->dvec, c->Fring, c->Ering, c->Bdiis, c->coef, c->scal, c->Cprev,
                  c->na2tmp, c->trsm_tmp, c->cvec, c->W, c->Bij, c->Xt, c->Zm, c->grad_parts, c->work, c->eigws, c->scratch,
                  c->d_occw, c->d_sad, c->d_fao0, c->d_fl, c->d_fm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (OzBuf* b : {&c->Bz, &c->Cz, &c->Hz, &c->Ctz, &c->Gz, &c->Xz, &c->trsm_sc.L, &c->trsm_sc.X, &c->tcA, &c->tcB})
    oz_buf_free(*b);
}

// Geometry-dependent part of setup: shell centres, one-electron, metric,
// Cholesky, 3-centre integrals, fit, orthogonaliser.
static void compute_geometry_rest(rihf_ctx* c);

// Integrals and fit of the current geometry.  defer_eri3: stop once the
// primitive-pair table is built, leaving the 3-centre integrals to a batched
// launch over several contexts (launch_eri3_batch) and the rest of the setup
// to compute_geometry_rest.
static void compute_geometry(rihf_ctx* c, bool defer_eri3 = false) {
  cudaStream_t s = c->stream;
  const int N = c->N, NA = c->NA;
  ++c->geom_serial;
  LaCtx la = c->la();
  IntegralCtx ic = c->ic();
  // shell centres
  std::vector<double> pxyz(3 * c->hp.nshell), axyz(3 * c->ha.nshell);
  for (int i = 0; i < c->hp.nshell; ++i)
    for (int d = 0; d < 3; ++d) pxyz[3 * i + d] = c->xyz[3 * c->hp.atom[i] + d];
  for (int i = 0; i < c->ha.nshell; ++i)
    for (int d = 0; d < 3; ++d) axyz[3 * i + d] = c->xyz[3 * c->ha.atom[i] + d];
  upload(c->d_pxyz, pxyz, s);
  upload(c->d_axyz_sh, axyz, s);
  upload(c->d_xyz, c->xyz, s);
  c->vnn = 0.0;
  for (int a = 0; a < c->natoms; ++a)
    for (int b = 0; b < a; ++b) {
      double r2 = 0.0;
      for (int d = 0; d < 3; ++d) r2 += (c->xyz[3 * a + d] - c->xyz[3 * b + d]) * (c->xyz[3 * a + d] - c->xyz[3 * b + d]);
      c->vnn += c->Z[a] * c->Z[b] / std::sqrt(r2);
    }
  RIHF_CUDA(cudaMemcpyAsync(c->scal + 5, &c->vnn, sizeof(double), cudaMemcpyHostToDevice, s));
  RIHF_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
  cudaEventRecord(c->ev[0], s);
  DevShells P = c->prim(), X = c->aux();
  { TraceScope t(c->tracer, s, "one_electron_kernel (S,T,V)", 3.0 * N * N * 8, 1);
    launch_one_electron(ic, P, c->max_lp, c->natoms, c->d_Z, c->d_xyz, c->S, c->Tk, c->V); }
  axpby(la, N * N, 1.0, c->Tk, 1.0, c->V, c->H);
  // metric, Cholesky, L^{-1}
  { TraceScope t(c->tracer, s, "eri2_kernel (P|Q)", (double)NA * NA * 8, 1);
    launch_eri2(ic, X, c->max_la, c->A); }
  RIHF_CUDA(cudaMemcpyAsync(c->L, c->A, sizeof(double) * NA * NA, cudaMemcpyDeviceToDevice, s));
  { TraceScope t(c->tracer, s, "cholesky A=LL^T", (double)NA * NA * NA / 3.0, 0);
    cholesky(la, c->L, NA, c->scratch); }
  c->have_linv = false;
  // Schwarz screening (Sec. 3.1.1): keep shell pairs with max (mu nu|mu nu) > tau.
  // With tau <= 0 no pair can drop out (every Q_ab > 0): the pair list stays
  // complete, and the factors are computed only when rihf_get_matrix asks
  c->schwarz_fresh = false;
  if (c->schwarz_ok && c->opt.schwarz_tau > 0.0) {
    TraceScope t(c->tracer, s, "schwarz_kernel (ab|ab)", 0.0, 0);
    launch_schwarz(ic, P, c->max_lp, c->d_schwarz);
    c->schwarz_fresh = true;
    std::vector<double> q(c->npairs_total);
    RIHF_CUDA(cudaMemcpyAsync(q.data(), c->d_schwarz, sizeof(double) * q.size(), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    const std::vector<ShellPair> old = c->pairs_h;
    c->pairs_h.clear();
    c->schwarz_max_dropped = 0.0;
    for (int a = 0; a < c->hp.nshell; ++a)
      for (int b = 0; b <= a; ++b) {
        double qa = q[(size_t)a * (a + 1) / 2 + b];
        if (qa * qa > c->opt.schwarz_tau) c->pairs_h.push_back({a, b});
        else c->schwarz_max_dropped = std::max(c->schwarz_max_dropped, qa * qa);
      }
    const bool same = old.size() == c->pairs_h.size() &&
                      std::equal(old.begin(), old.end(), c->pairs_h.begin(),
                                 [](const ShellPair& x, const ShellPair& y) { return x.a == y.a && x.b == y.b; });
    if (!same) {
      c->npairs = (int)c->pairs_h.size();
      upload(c->d_pairs, c->pairs_h, s);
      refresh_tasks(c);
    }
  }
  // (mu nu|P) for shell pairs a >= b into the pair-packed Bp, then
  // B = L^{-1} T (Eq. biap with A^L = L^{-T}) in place by blocked forward
  // substitution over the Naux x N(N+1)/2 matrix; an explicit L^{-1} product
  // loses accuracy when cond(A) reaches 1e9 (diffuse auxiliary sets)
  RIHF_CUDA(cudaMemsetAsync(c->Bp, 0, sizeof(double) * (size_t)NA * c->npp, s));
  if (defer_eri3) {
    launch_pair_prims(ic, P, c->d_pairs, c->npairs, c->d_pp_off, c->d_pp);
    return;
  }
  { TraceScope t(c->tracer, s, "eri3_kernel (mu nu|P)", c->flops_eri3, 0);
    launch_pair_prims(ic, P, c->d_pairs, c->npairs, c->d_pp_off, c->d_pp);
    launch_eri3(ic, P, X, c->d_pairs, c->ptab(), c->groups, kTaskGroups, c->Bp); }
  compute_geometry_rest(c);
}

// The fit, the planes or expansion of B and the orthogonaliser, after the
// 3-centre integrals of this geometry are in Bp.
static void compute_geometry_rest(rihf_ctx* c) {
  cudaStream_t s = c->stream;
  const int N = c->N, NA = c->NA;
  LaCtx la = c->la();
  if (c->trsm_sc.X.planes) {
    // mixed mode: rank-64 updates on the tensor cores (7 digits), panels in FP64
    TraceScope t(c->tracer, s, "fit trsm B=L^-1 T (tcgen05 digit updates)", (double)NA * NA * c->npp, 0);
    trsm_lower_tc(la, c->L, NA, c->Bp, c->npp, 0, c->trsm_sc);
  } else {
    TraceScope t(c->tracer, s, "fit trsm B=L^-1 T", (double)NA * NA * c->npp, 0);
    trsm_lower(la, c->L, NA, c->Bp, c->npp, false, 0, c->trsm_tmp);
  }
  c->bu_is_B = false;
  if (c->planes_all) {   // digit planes of all of B for the tensor-core RI-K (rows (P, mu), K = nu)
    TraceScope t(c->tracer, s, "B digit planes (oz_slice)", (double)NA * c->npp * 8 + (double)NA * N * N * 2 * kOzMaxDigits, 1);
    c->Bop = oz_slice(la, c->Bp, NA * N, N, 0, 0, 0, 1, kOzMaxDigits, 0, c->Bz, 0, c->npp, N);
  } else if (!c->Bz.planes && c->pc == NA) {   // FP64 mode, all slices fit: expand B once
    TraceScope t(c->tracer, s, "B expanded to N x N slices", (double)NA * c->npp * 8 + (double)NA * N * N * 8, 1);
    unpack_sym_batch(la, c->Bp, NA, N, c->npp, c->Bu);
    c->bu_is_B = true;
  }
  int flag = 0;
  RIHF_CUDA(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  RIHF_CUDA(cudaStreamSynchronize(s));
  if (flag) throw RihfError(RIHF_ERR_NOT_POSITIVE_DEFINITE, "metric (P|Q) is not positive definite");
  // Orthogonaliser.  First try X = L_S^{-T} (S = L_S L_S^T); since
  // lambda_min(S) >= 1 / Tr(S^{-1}) = 1 / ||L_S^{-1}||_F^2, a bound above
  // lindep_tau proves that canonical orthogonalisation would drop nothing, and
  // then the SCF fixed point does not depend on the choice of orthogonaliser.
  int k0 = 0;
  bool chol_ok = false;
  {
    TraceScope t(c->tracer, s, "orthogonaliser (cholesky S)", (double)N * N * N / 3.0, 0);
    RIHF_CUDA(cudaMemcpyAsync(c->T2, c->S, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, s));
    cholesky(la, c->T2, N, c->scratch);
    identity(la, c->T1, N);
    trsm_lower(la, c->T2, N, c->T1, N, false, 0, c->trsm_tmp);
    dot(la, N * N, c->T1, c->T1, c->scal + 3);
    double tr = 0.0;
    RIHF_CUDA(cudaMemcpyAsync(&tr, c->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    chol_ok = !flag && std::isfinite(tr) && tr > 0.0 && 1.0 / tr > c->opt.lindep_tau;
    RIHF_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
  }
  std::vector<double> sw;
  if (!chol_ok) {
    TraceScope t(c->tracer, s, "eigh S", 0.0, 0);
    eigh(la, c->S, N, c->Sw, c->Sv, c->eigws, 4, nullptr);
    sw.resize(N);
    RIHF_CUDA(cudaMemcpyAsync(sw.data(), c->Sw, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    while (k0 < N && sw[k0] <= c->opt.lindep_tau) ++k0;
    if (k0 == N) throw RihfError(RIHF_ERR_NOT_POSITIVE_DEFINITE, "overlap matrix has no eigenvalue above lindep_tau");
  }
  int nind = N - k0;
  if (c->verbose || getenv("RIHF_VERBOSE"))
    fprintf(stderr, "rihf: orthogonaliser %s, %d of %d functions kept%s\n",
            chol_ok ? "L_S^-T (Cholesky bound proves nothing would be dropped)" : "canonical", nind, N,
            chol_ok ? "" : (" (smallest kept overlap eigenvalue " + std::to_string(sw.empty() ? 0.0 : sw[k0]) + ")").c_str());
  if (c->nind != 0 && nind != c->nind) {
    c->have_cprev = false;
    for (auto* arr : {c->graphs, c->diag_graphs}) {   // captured work assumes the old basis size
      const int cnt = arr == c->graphs ? kOzMaxDigits + 1 : 6;
      for (int i = 0; i < cnt; ++i)
        if (arr[i].exec) {
          cudaGraphExecDestroy(arr[i].exec);
          arr[i].exec = nullptr;
        }
    }
  }
  c->nind = nind;
  if (chol_ok) {
    transpose(la, c->T1, N, N, c->Xo);
  } else if (k0 == 0) {
    // Cholesky failed the bound but nothing is dropped: canonical with all vectors
    std::vector<double> invs(nind);
    for (int i = 0; i < nind; ++i) invs[i] = 1.0 / std::sqrt(sw[i]);
    RIHF_CUDA(cudaMemcpyAsync(c->dvec, invs.data(), sizeof(double) * nind, cudaMemcpyHostToDevice, s));
    scale_cols(la, c->Sv, c->dvec, N, nind, c->Xo);
    RIHF_CUDA(cudaStreamSynchronize(s));
  } else {
    std::vector<double> invs(nind);
    for (int i = 0; i < nind; ++i) invs[i] = 1.0 / std::sqrt(sw[k0 + i]);
    RIHF_CUDA(cudaMemcpyAsync(c->dvec, invs.data(), sizeof(double) * nind, cudaMemcpyHostToDevice, s));
    // canonical orthogonalisation: Xo[mu][k] = Sv[mu][k0 + k] / sqrt(s_{k0+k})
    copy_cols(la, c->Sv + k0, N, N, nind, 1.0, c->T1);
    scale_cols(la, c->T1, c->dvec, N, nind, c->Xo);
    RIHF_CUDA(cudaStreamSynchronize(s));
  }
  // Newton-Schulz S-orthonormalisation, X <- X (3I - X^T S X) / 2, so that
  // X^T S X = I holds to rounding whatever the eigensolver's residual.
  for (int it = 0; it < (chol_ok ? 1 : 3); ++it) {
    GemmArgs g1;   // T1 (N x n) = S X
    g1.M = N; g1.N = nind; g1.K = N; g1.A = c->S; g1.lda = N; g1.B = c->Xo; g1.ldb = nind; g1.C = c->T1;
    g1.ldc = nind;
    dgemm(la, g1);
    GemmArgs g2;   // T2 (n x n) = -1/2 X^T T1, then + 3/2 I
    g2.M = nind; g2.N = nind; g2.K = N; g2.A = c->Xo; g2.lda = nind; g2.transA = true; g2.B = c->T1;
    g2.ldb = nind; g2.C = c->T2; g2.ldc = nind; g2.alpha = -0.5;
    dgemm(la, g2);
    identity(la, c->Err, nind);
    axpby(la, nind * nind, 1.0, c->T2, 1.5, c->Err, c->T2);
    GemmArgs g3;   // Xo <- Xo T2  (via T1)
    g3.M = N; g3.N = nind; g3.K = nind; g3.A = c->Xo; g3.lda = nind; g3.B = c->T2; g3.ldb = nind; g3.C = c->T1;
    g3.ldc = nind;
    dgemm(la, g3);
    RIHF_CUDA(cudaMemcpyAsync(c->Xo, c->T1, sizeof(double) * N * nind, cudaMemcpyDeviceToDevice, s));
  }
  cudaEventRecord(c->ev[1], s);
  RIHF_CUDA(cudaStreamSynchronize(s));
  c->tracer.flush();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
  c->timings[0] = ms;
}

extern "C" {

void rihf_default_options(rihf_options* o) {
  if (!o) return;
  o->precision = RIHF_PRECISION_FP64;
  o->pure = 1;
  o->schwarz_tau = 0.0;   // keep every pair: the fit amplifies dropped integrals when cond(P|Q) is large
  o->lindep_tau = 1e-8;
  o->conv_e = 1e-10;
  o->conv_diis = 1e-9;
  o->max_iter = 100;
  o->diis_size = 8;
  o->mixed_digits = 0;
  o->device = 0;
  o->cuda_graphs = 1;
  o->confirm_fp64 = 0;
  o->aux_chunk = 0;
}

const char* rihf_strerror(int code) {
  switch (code) {
    case RIHF_OK: return "ok";
    case RIHF_ERR_INVALID_ARG: return "invalid argument";
    case RIHF_ERR_OOM: return "out of device memory";
    case RIHF_ERR_CUDA: return "CUDA error";
    case RIHF_ERR_NOT_CONVERGED: return "SCF not converged";
    case RIHF_ERR_TIMEOUT: return "device wait timed out";
    case RIHF_ERR_NOT_POSITIVE_DEFINITE: return "matrix not positive definite";
    case RIHF_ERR_STATE: return "invalid call order";
    default: return "unknown error";
  }
}

const char* rihf_last_error(void) { return g_last_error.c_str(); }

#define RIHF_API_BEGIN try {
#define RIHF_API_END                                  \
  }                                                   \
  catch (const RihfError& e) {                        \
    g_last_error = e.what();                          \
    return e.code;                                    \
  }                                                   \
  catch (const CudaError& e) {                        \
    g_last_error = e.what();                          \
    return RIHF_ERR_CUDA;                             \
  }                                                   \
  catch (const std::exception& e) {                   \
    g_last_error = e.what();                          \
    return RIHF_ERR_INVALID_ARG;                      \
  }

}  // extern "C"

// Context construction.  occ: occupation numbers of the nocc = occ->size()
// lowest orbitals (spherically averaged atoms of the SAD guess), or NULL for
// the closed shell with nelec / 2 doubly occupied orbitals.
static rihf_ctx* setup_impl(int natoms, const int* Z, const double* xyz, int nprim_shells, const rihf_shell* prim,
                            int naux_shells, const rihf_shell* aux, int nelec, const rihf_options* opt,
                            const std::vector<double>* occ) {
  rihf_ctx* c = new rihf_ctx();
  if (opt) c->opt = *opt; else rihf_default_options(&c->opt);
  if (c->opt.diis_size < 2) c->opt.diis_size = 2;
  if (c->opt.diis_size > 16) c->opt.diis_size = 16;
  try {
    RIHF_CUDA(cudaSetDevice(c->opt.device));
    RIHF_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->opt.device));
    RIHF_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    for (auto& e : c->ev) RIHF_CUDA(cudaEventCreate(&e));
    c->natoms = natoms;
    c->nelec = nelec;
    c->nocc = occ ? (int)occ->size() : nelec / 2;
    c->Z.assign(Z, Z + natoms);
    c->xyz.assign(xyz, xyz + 3 * natoms);
    build_transforms(c->opt.pure != 0, c->tr_h, c->nf_h);
    int rc = build_host_shells(nprim_shells, prim, natoms, kMaxLPrim, c->nf_h, c->hp);
    if (rc == RIHF_OK) rc = build_host_shells(naux_shells, aux, natoms, kMaxLAux, c->nf_h, c->ha);
    if (rc != RIHF_OK) throw RihfError(rc, "shell with unsupported l, nprim, atom index or exponent");
    c->N = c->hp.nfunc;
    c->NA = c->ha.nfunc;
    c->max_lp = c->hp.lmax;
    c->max_la = c->ha.lmax;
    if (c->nocc > c->N) throw RihfError(RIHF_ERR_INVALID_ARG, "more occupied orbitals than basis functions");
    const int N = c->N, NA = c->NA;
    cudaStream_t s = c->stream;
    // basis arrays
    c->d_pl = dalloc<int>(c->hp.nshell); upload(c->d_pl, c->hp.l, s);
    c->d_patom = dalloc<int>(c->hp.nshell); upload(c->d_patom, c->hp.atom, s);
    c->d_pnprim = dalloc<int>(c->hp.nshell); upload(c->d_pnprim, c->hp.nprim, s);
    c->d_pps = dalloc<int>(c->hp.nshell); upload(c->d_pps, c->hp.pstart, s);
    c->d_pao = dalloc<int>(c->hp.nshell); upload(c->d_pao, c->hp.ao, s);
    c->d_pexp = dalloc<double>(c->hp.exps.size()); upload(c->d_pexp, c->hp.exps, s);
    {
      std::vector<double> ie(c->hp.exps.size());
      for (size_t i = 0; i < ie.size(); ++i) ie[i] = 1.0 / c->hp.exps[i];
      c->d_piexp = dalloc<double>(ie.size()); upload(c->d_piexp, ie, s);
    }
    c->d_pcoef = dalloc<double>(c->hp.coefs.size()); upload(c->d_pcoef, c->hp.coefs, s);
    c->d_pxyz = dalloc<double>(3 * c->hp.nshell);
    c->d_al = dalloc<int>(c->ha.nshell); upload(c->d_al, c->ha.l, s);
    c->d_aatom = dalloc<int>(c->ha.nshell); upload(c->d_aatom, c->ha.atom, s);
    c->d_anprim = dalloc<int>(c->ha.nshell); upload(c->d_anprim, c->ha.nprim, s);
    c->d_aps = dalloc<int>(c->ha.nshell); upload(c->d_aps, c->ha.pstart, s);
    c->d_aao = dalloc<int>(c->ha.nshell); upload(c->d_aao, c->ha.ao, s);
    c->d_aexp = dalloc<double>(c->ha.exps.size()); upload(c->d_aexp, c->ha.exps, s);
    {
      std::vector<double> ie(c->ha.exps.size());
      for (size_t i = 0; i < ie.size(); ++i) ie[i] = 1.0 / c->ha.exps[i];
      c->d_aiexp = dalloc<double>(ie.size()); upload(c->d_aiexp, ie, s);
    }
    c->d_acoef = dalloc<double>(c->ha.coefs.size()); upload(c->d_acoef, c->ha.coefs, s);
    c->d_axyz_sh = dalloc<double>(3 * c->ha.nshell);
    c->d_tr = dalloc<double>(c->tr_h.size()); upload(c->d_tr, c->tr_h, s);
    c->d_nf = dalloc<int>(c->nf_h.size()); upload(c->d_nf, c->nf_h, s);
    c->d_Z = dalloc<int>(natoms); upload(c->d_Z, c->Z, s);
    c->d_xyz = dalloc<double>(3 * natoms);
    c->d_boys = dalloc<double>((size_t)kBoysN * kBoysM); upload(c->d_boys, boys_host(), s);
    c->d_counter = dalloc<int>(4);
    c->d_flag = dalloc<int>(4);
    c->d_sched = dalloc<int>(2);
    RIHF_CUDA(cudaMemset(c->d_sched, 0, 2 * sizeof(int)));
    c->d_red = dalloc<double>(kRedSlots);
    c->d_ticket = dalloc<int>(1);
    RIHF_CUDA(cudaMemset(c->d_ticket, 0, sizeof(int)));
    // shell pairs a >= b; compute_geometry screens them (Schwarz) when the
    // four-centre class fits in shared memory, otherwise all pairs are kept
    for (int a = 0; a < c->hp.nshell; ++a)
      for (int b = 0; b <= a; ++b) c->pairs_h.push_back({a, b});
    c->npairs = c->npairs_total = (int)c->pairs_h.size();
    c->d_pairs = dalloc<ShellPair>(c->pairs_h.size()); upload(c->d_pairs, c->pairs_h, s);
    c->d_schwarz = dalloc<double>(c->pairs_h.size());
    c->d_tasks = dalloc<int2>(c->pairs_h.size() * (size_t)c->ha.nshell);
    c->d_pp_off = dalloc<int>(c->pairs_h.size() + 1);
    c->d_pp = dalloc<PairPrim>(std::max(1, pair_prim_offsets(c->pairs_h, c->hp.nprim).back()));
    refresh_tasks(c);
    {
      int maxsm = 0;
      RIHF_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->opt.device));
      c->schwarz_ok = schwarz_smem_bytes(c->max_lp) <= maxsm;
    }
    // matrices
    size_t n2 = (size_t)N * N, na2 = (size_t)NA * NA, big = (size_t)NA * n2;
    c->S = dalloc<double>(n2); c->H = dalloc<double>(n2); c->Tk = dalloc<double>(n2); c->V = dalloc<double>(n2);
    c->A = dalloc<double>(na2); c->L = dalloc<double>(na2); c->Linv = dalloc<double>(na2);
    c->npp = (long long)N * (N + 1) / 2;
    c->Bp = dalloc<double>((size_t)NA * c->npp); c->Yp = dalloc<double>((size_t)NA * c->npp);
    c->Dp = dalloc<double>(c->npp); c->Jp = dalloc<double>(c->npp);
    (void)big;
    c->Xo = dalloc<double>(n2); c->Sw = dalloc<double>(N); c->Sv = dalloc<double>(n2);
    c->C = dalloc<double>(n2); c->eps = dalloc<double>(N); c->Ct = dalloc<double>((size_t)N * c->nocc);
    c->D = dalloc<double>(n2); c->J = dalloc<double>(n2); c->K = dalloc<double>(n2); c->F = dalloc<double>(n2);
    c->Fx = dalloc<double>(n2); c->T1 = dalloc<double>(n2); c->T2 = dalloc<double>(n2); c->Err = dalloc<double>(n2);
    c->Fp = dalloc<double>(n2); c->Cp = dalloc<double>(n2); c->Cprev = dalloc<double>(n2);
    c->Hb = dalloc<double>((size_t)NA * N * c->nocc);
    c->dvec = dalloc<double>(std::max(N, NA));
    c->Fring = dalloc<double>((size_t)c->opt.diis_size * n2);
    c->Ering = dalloc<double>((size_t)c->opt.diis_size * n2);
    c->Bdiis = dalloc<double>(16 * 16);
    c->coef = dalloc<double>(16);
    c->scal = dalloc<double>(8);
    c->cvec = dalloc<double>(NA); c->W = dalloc<double>(n2);
    c->Bij = dalloc<double>((size_t)NA * c->nocc * c->nocc);
    c->Xt = dalloc<double>((size_t)NA * (c->nocc * c->nocc + 1));   // [X~ | c] per row P
    c->Zm = dalloc<double>(na2);
    c->na2tmp = dalloc<double>(na2);
    c->G = c->Hb;   // G' of the gradient reuses H's memory (H is spent by then)
    const bool mixed = c->opt.precision == RIHF_PRECISION_MIXED;
    if (mixed) {
      const int nkb_max = (NA * c->nocc + kOzChunk - 1) / kOzChunk;
      const int no = c->nocc;
      c->Cz = oz_buf_alloc(no, N, kOzMaxDigits, 1);
      c->Hz = oz_buf_alloc(N, NA * no, kOzMaxDigits, nkb_max);
      c->trsm_sc.L = oz_buf_alloc(NA, kTrsmOuter, kOzMaxDigits, 1);
      c->trsm_sc.X = oz_buf_alloc((int)c->npp, kTrsmOuter, kOzMaxDigits, 1);
      c->Ctz = oz_buf_alloc(N, no, kOzMaxDigits, 1);
      const int xch = (no * no + kOzChunk - 1) / kOzChunk;
      c->Xz = oz_buf_alloc(NA, no * no, kOzMaxDigits, (xch + kOzMaxChunksPerBlock - 1) / kOzMaxChunksPerBlock);
      if (N > 256) {
        c->tcA = oz_buf_alloc(std::max(N, NA), N, kOzMaxDigits, 1);
        c->tcB = oz_buf_alloc(std::max(N, NA), N, kOzMaxDigits, 1);
      }
    }
    c->trsm_tmp = dalloc<double>(32 * std::max<size_t>({(size_t)c->npp, (size_t)NA, (size_t)c->nocc * c->nocc}) + 1024);
    {   // guess history and learned-guess buffers
      std::vector<int> aoat(N), aol(N);
      for (int i = 0; i < c->hp.nshell; ++i)
        for (int k = 0; k < c->nf_h[c->hp.l[i]]; ++k) {
          aoat[c->hp.ao[i] + k] = c->hp.atom[i];
          aol[c->hp.ao[i] + k] = c->hp.l[i];
        }
      c->d_ao_atom = dalloc<int>(N); upload(c->d_ao_atom, aoat, s);
      c->d_ao_l = dalloc<int>(N); upload(c->d_ao_l, aol, s);
      for (auto& h : c->hist_D) h = dalloc<double>(n2);
      c->hist_S = dalloc<double>(n2);
      for (auto& h : c->hist_xyz) h = dalloc<double>(3 * natoms);
      c->Dpred = dalloc<double>(n2);
      const size_t M = (size_t)N * (N + 1) / 2;
      c->mlX = dalloc<float>(M * kMlpF);
      c->mly = dalloc<float>(M);
      c->mlt = dalloc<float>(M);
      c->mlDx = dalloc<double>(M);
      c->ml_sums = dalloc<double>(3);
      c->rep_X = dalloc<float>(M * kMlpF * rihf_ctx::kReplay);
      c->rep_t = dalloc<float>(M * rihf_ctx::kReplay);
    }
    c->grad_parts = dalloc<double>(5 * 3 * natoms);
    c->work_elems = std::max<size_t>({(size_t)1 << 24, 8 * n2 * 4, (size_t)NA * 64});
    c->work = dalloc<double>(c->work_elems);
    c->eigws = dalloc<double>(eig_workspace(N));
    c->scratch = dalloc<double>(32 * 32 + (size_t)std::max(N, NA) * 32 + 64);
    {
      // Chunk buffers for the expanded N x N slices of B (and of Y): as many
      // auxiliary functions per chunk as the free device memory holds, less a
      // reserve, capped at Naux and at opt.aux_chunk.  FP64 slices in Bu; in
      // mixed mode also their digit planes (Bz) and the gradient's chunk
      // planes (Gz: rows (P, j) of H with K = N, or rows (P, mu) of G' with K = nocc).
      const int no = c->nocc;
      size_t fr = 0, tot = 0;
      RIHF_CUDA(cudaMemGetInfo(&fr, &tot));
      const size_t reserve = std::max<size_t>((size_t)2 << 30, tot / 32);
      auto gz_elems = [&](int np) {
        return std::max(oz_plane_elems(np * no, N, kOzMaxDigits), oz_plane_elems(np * N, no, kOzMaxDigits));
      };
      auto bytes = [&](int np) {
        size_t b = (size_t)np * n2 * sizeof(double);
        if (mixed)
          b += oz_plane_elems(np * N, N, kOzMaxDigits) * sizeof(uint16_t) + gz_elems(np) * sizeof(uint16_t) +
               2 * ((size_t)np * std::max(N, no) + 2 * kOzTileM) * sizeof(int);
        return b;
      };
      int pc = NA;
      if (c->opt.aux_chunk > 0) pc = std::min(pc, c->opt.aux_chunk);
      while (pc > 1 && bytes(pc) + reserve > fr) pc = std::max(1, pc * 7 / 8);
      if (bytes(pc) + reserve > fr) throw RihfError(RIHF_ERR_OOM, "no device memory left for one auxiliary chunk");
      c->pc = pc;
      c->Bu = dalloc<double>((size_t)pc * n2);
      if (mixed) {
        c->Bz = oz_buf_alloc(pc * N, N, kOzMaxDigits, 1);
        c->Gz = oz_buf_alloc_raw(gz_elems(pc),
                                 (size_t)((std::max(pc * no, pc * N) + kOzTileM - 1) / kOzTileM) * kOzTileM);
        c->planes_all = pc == NA;
      }
    }
    if (occ) {
      c->occ = *occ;
      std::vector<double> w(occ->size());
      for (size_t k = 0; k < w.size(); ++k) w[k] = std::sqrt((*occ)[k]);
      c->d_occw = dalloc<double>(w.size());
      upload(c->d_occw, w, s);
    }
    compute_geometry(c);
  } catch (...) {
    free_all(c);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    throw;
  }
  return c;
}

extern "C" {

int rihf_setup(int natoms, const int* Z, const double* xyz, int nprim_shells, const rihf_shell* prim,
               int naux_shells, const rihf_shell* aux, int nelec, const rihf_options* opt, rihf_ctx** out) {
  RIHF_API_BEGIN
  if (!out || natoms <= 0 || !Z || !xyz || nprim_shells <= 0 || !prim || naux_shells <= 0 || !aux || nelec <= 0 ||
      (nelec & 1)) {
    g_last_error = "invalid sizes or pointers (nelec must be positive and even)";
    return RIHF_ERR_INVALID_ARG;
  }
  *out = nullptr;
  *out = setup_impl(natoms, Z, xyz, nprim_shells, prim, naux_shells, aux, nelec, opt, nullptr);
  return RIHF_OK;
  RIHF_API_END
}

int rihf_update_geometry(rihf_ctx* c, const double* xyz) {
  RIHF_API_BEGIN
  if (!c || !xyz) return RIHF_ERR_INVALID_ARG;
  c->xyz.assign(xyz, xyz + 3 * c->natoms);
  c->converged = false;
  compute_geometry(c);
  return RIHF_OK;
  RIHF_API_END
}

// Orbitals from a Fock matrix: F' = Xo^T F Xo, eigh, C = Xo C'.
// Runs `body` (work on the context stream only, no host synchronisation) from
// the CUDA graph in g, capturing it on its second use (the first runs eagerly,
// so one-time set-up such as kernel attributes happens outside a capture);
// eagerly when graphs are off or a capture fails.  Trace events are not
// captured; the replay is traced as one entry named `name`.
extern "C++" {
template <class Body>
static void graph_or_eager(rihf_ctx* c, rihf_ctx::IterGraph& g, const char* name, Body&& body) {
  if (!c->opt.cuda_graphs || !c->graphs_ok || g.uses++ == 0) {
    TraceScope t(c->tracer, c->stream, name, 0.0, 0);
    body();
    return;
  }
  if (!g.exec) {
    const long long l0 = c->launches;
    const bool tr = c->tracer.on;
    c->tracer.on = false;
    RIHF_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(c->stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      c->launches = l0;
      c->graphs_ok = false;
      c->tracer.on = tr;
      TraceScope t(c->tracer, c->stream, name, 0.0, 0);
      body();
      return;
    }
    c->tracer.on = tr;
    RIHF_CUDA(cudaStreamEndCapture(c->stream, &graph));
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    g.launches = c->launches - l0;
    c->launches = l0;
    if (e != cudaSuccess) {
      cudaGetLastError();
      g.exec = nullptr;
      c->graphs_ok = false;
      TraceScope t(c->tracer, c->stream, name, 0.0, 0);
      body();
      return;
    }
  }
  TraceScope t(c->tracer, c->stream, name, 0.0, 0);
  RIHF_CUDA(cudaGraphLaunch(g.exec, c->stream));
  c->launches += g.launches;
}
}  // extern "C++"

static void occupy_by_l(rihf_ctx* c);

static void diagonalise(rihf_ctx* c, const double* Fin, bool warm) {
  LaCtx la = c->la();
  const int N = c->N, n = c->nind;
  // refinement from the previous eigenvectors once the SCF error is moderate;
  // the guard below falls back to a Jacobi pass unless the refined vectors
  // are orthonormal and diagonalise F'
  const bool use_prev = warm && c->have_cprev && !c->force_cold;
  c->force_cold = false;
  const bool skip = use_prev && c->last_err < 1e-2;
  auto form_fp = [&]() {
    GemmArgs g1;   // T1 (N x n) = F Xo
    g1.M = N; g1.N = n; g1.K = N; g1.A = Fin; g1.lda = N; g1.B = c->Xo; g1.ldb = n; g1.C = c->T1; g1.ldc = n;
    dgemm(la, g1);
    GemmArgs g2;   // Fp (n x n) = Xo^T T1
    g2.M = n; g2.N = n; g2.K = N; g2.A = c->Xo; g2.lda = n; g2.transA = true; g2.B = c->T1; g2.ldb = n;
    g2.C = c->Fp; g2.ldc = n;
    dgemm(la, g2);
    RIHF_CUDA(cudaMemsetAsync(c->eps, 0, sizeof(double) * N, c->stream));
  };
  if (!use_prev) {
    // cold start: a full Jacobi pass, not replayed
    form_fp();
    TraceScope t(c->tracer, c->stream, "eigh F' (jacobi+refine)", 0.0, 0);
    eigh(la, c->Fp, n, c->eps, c->Cp, c->eigws, 3, nullptr, false, 20);
  } else if (!skip) {
    // warm-started iterations (max|e| >= 1e-2): Jacobi sweeps from the
    // previous vectors, then FP64 refinement; these iterations need the
    // eigenvectors only to the accuracy of the SCF iterate, and the later
    // refine-only iterations start from them.  Below max|e| = 0.1 (the first
    // iterations after a nuclear step) two sweeps reach ~1e-5 and one
    // refinement and one re-orthonormalisation step suffice; larger errors
    // (a cold start) take three sweeps and three refinement steps.
    const bool light = c->last_err < 0.1;
    graph_or_eager(c, c->diag_graphs[(light ? 4 : 2) + (Fin == c->F ? 0 : 1)], "eigh F' (jacobi+refine)", [&]() {
      form_fp();
      if (light) eigh(la, c->Fp, n, c->eps, c->Cp, c->eigws, 1, c->Cprev, false, 2, 1);
      else eigh(la, c->Fp, n, c->eps, c->Cp, c->eigws, 3, c->Cprev, false, 3);
    });
  } else {
    graph_or_eager(c, c->diag_graphs[Fin == c->F ? 0 : 1], "eigh F' (refine only)", [&]() {
      form_fp();
      // two quadratically convergent steps from vectors accurate to ~max|e| < 1e-2,
      // then three Newton-Schulz re-orthonormalisations: refined vectors whose
      // V^T V is off by ~1e-2 reach ~1e-4 after two and ~1e-8 after three,
      // which the guard below needs (each miss costs a Jacobi redo)
      eigh(la, c->Fp, n, c->eps, c->Cp, c->eigws, 2, c->Cprev, true, 20, 3);
      // guard: orthonormality and the off-diagonal of Cp^T F' Cp
      GemmArgs go;   // T2 = Cp^T Cp
      go.M = n; go.N = n; go.K = n; go.A = c->Cp; go.lda = n; go.transA = true; go.B = c->Cp; go.ldb = n;
      go.C = c->T2; go.ldc = n;
      dgemm(la, go);
      eig_check_mb_kernel<<<kRedBlocks, 256, 0, c->stream>>>(c->T2, n, 1.0, 0, c->d_red, c->d_ticket, c->scal + 2);
      RIHF_LAUNCH_CHECK();
      GemmArgs gf;   // T1 = F' Cp, T2 = Cp^T T1
      gf.M = n; gf.N = n; gf.K = n; gf.A = c->Fp; gf.lda = n; gf.B = c->Cp; gf.ldb = n; gf.C = c->T1; gf.ldc = n;
      dgemm(la, gf);
      GemmArgs gt;
      gt.M = n; gt.N = n; gt.K = n; gt.A = c->Cp; gt.lda = n; gt.transA = true; gt.B = c->T1; gt.ldb = n;
      gt.C = c->T2; gt.ldc = n;
      dgemm(la, gt);
      // occupied-virtual block only: rotations inside the occupied or the
      // virtual space (near-degenerate pairs) leave the density unchanged
      eig_check_mb_kernel<<<kRedBlocks, 256, 0, c->stream>>>(c->T2, n, 0.0, c->nocc + 1, c->d_red, c->d_ticket,
                                                             c->scal + 3);
      RIHF_LAUNCH_CHECK();
      c->launches += 2;
    });
    double dev[2] = {0.0, 0.0};
    RIHF_CUDA(cudaMemcpyAsync(dev, c->scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    RIHF_CUDA(cudaStreamSynchronize(c->stream));
    // The occupied-virtual block of C^T F' C must end well below the SCF
    // error, or the density carries the eigensolver's error and the SCF stalls
    // at that level (a bound proportional to max|e| with a factor above one
    // accepted exactly that fixed point).  Two quadratically convergent steps
    // from vectors of the previous iterate normally leave it near rounding; a
    // refinement that rotated too little (the cluster threshold treats
    // separated pairs as clustered when the residual norms are large) fails
    // here and is redone by Jacobi sweeps.
    const double offd_tol = std::max(1e-11, 0.05 * c->last_err);
    if (!(dev[0] < 1e-8) || !(dev[1] < offd_tol)) {
      if (c->verbose || getenv("RIHF_VERBOSE"))
        fprintf(stderr, "rihf: refine-only eigh deviation %.3e, off-diagonal %.3e, redo\n", dev[0], dev[1]);
      // warm-started from near-converged vectors: three Jacobi sweeps reach
      // the FP32 floor, the four FP64 refinement steps the rest
      TraceScope t(c->tracer, c->stream, "eigh F' (jacobi redo)", 0.0, 0);
      eigh(la, c->Fp, n, c->eps, c->Cp, c->eigws, 4, c->Cprev, false, 3);
    }
  }
  RIHF_CUDA(cudaMemcpyAsync(c->Cprev, c->Cp, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->stream));
  c->have_cprev = true;
  // C (N x N): first n columns = Xo Cp, rest zero
  RIHF_CUDA(cudaMemsetAsync(c->C, 0, sizeof(double) * N * N, c->stream));
  GemmArgs g3;
  g3.M = N; g3.N = n; g3.K = n; g3.A = c->Xo; g3.lda = n; g3.B = c->Cp; g3.ldb = n; g3.C = c->C; g3.ldc = N;
  dgemm(la, g3);
  if (c->sph_avg && !c->occ_l.empty()) occupy_by_l(c);
}

// Spherical average of a matrix over real solid harmonics: zero between
// different l or m, and for equal l and m the mean over m of the shell pair's
// (m, m) entries (the rotation average, exact for the Fock operator of a
// spherically symmetric density).
__global__ void sph_avg_kernel(const double* __restrict__ F, int N, const int* __restrict__ ao0,
                               const int* __restrict__ fl, const int* __restrict__ fm, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N * N;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    double v = 0.0;
    if (fl[i] == fl[j] && fm[i] == fm[j]) {
      const int l = fl[i];
      for (int m = 0; m <= 2 * l; ++m) v += F[(size_t)(ao0[i] + m) * N + ao0[j] + m];
      v /= (2 * l + 1);
    }
    out[e] = v;
  }
}

// C~ = C_occ diag(sqrt(n_i)): sqrt(2) C_occ for the closed shell (D = C~ C~^T).
static void form_Ct(rihf_ctx* c) {
  LaCtx la = c->la();
  const int N = c->N, no = c->nocc;
  copy_cols(la, c->C, N, N, no, c->d_occw ? 1.0 : std::sqrt(2.0), c->Ct);
  if (c->d_occw) scale_cols(la, c->Ct, c->d_occw, N, no, c->Ct);
}

// RI-J (Eq. j_ri) over the pair-packed B: d_P = sum_{mu >= nu} w B^P D (w = 2
// off the diagonal), then J = sum_P d_P B^P; two streaming passes over B.
static void ri_j(rihf_ctx* c) {
  LaCtx la = c->la();
  const int N = c->N, NA = c->NA;
  pack_sym(la, c->D, N, 2.0, c->Dp);
  { TraceScope t(c->tracer, c->stream, "RI-J d=B.D (gemv over packed rows)", (double)NA * c->npp * 8, 1);
    gemv_rows(la, c->Bp, NA, c->npp, c->Dp, 1.0, c->dvec); }
  { TraceScope t(c->tracer, c->stream, "RI-J J=B^T d (gemv over packed columns)", (double)NA * c->npp * 8, 1);
    gemv_cols(la, c->Bp, NA, c->npp, c->dvec, 1.0, c->Jp);
    unpack_sym(la, c->Jp, N, c->J); }
}

// Hb[(P, mu)][i] = sum_nu B^P_{mu nu} C~_{nu i} (Eq. tp) for every P: in FP64
// (digits = 0) from the expanded slices (Bu, chunk by chunk unless it holds all
// of B), or on the tensor cores with `digits` digits against the planes Cop of
// C~^T (all of B's planes at once, or chunk planes cut from the packed rows).
static void form_H(rihf_ctx* c, int digits, const OzOperand* Cop, const char* name) {
  LaCtx la = c->la();
  const int N = c->N, NA = c->NA, no = c->nocc;
  const size_t n2 = (size_t)N * N;
  const double prod = digits > 0 ? oz_products(digits) : 1.0;
  const int npad = (no + 15) / 16 * 16, kpadN = (N + kOzChunk - 1) / kOzChunk * kOzChunk;
  TraceScope t(c->tracer, c->stream, name,
               digits > 0 ? 2.0 * (double)((NA * N + kOzTileM - 1) / kOzTileM * kOzTileM) * npad * kpadN * prod
                          : 2.0 * NA * n2 * no,
               digits > 0 ? 3 : 0);
  if (digits > 0 && c->planes_all) {
    OzGemmArgs g1;
    g1.A = c->Bop; g1.B = *Cop; g1.M = NA * N; g1.N = no; g1.s = digits; g1.C = c->Hb; g1.cs_m1 = no; g1.cs_n = 1;
    oz_gemm(la, g1);
    return;
  }
  if (digits == 0 && c->bu_is_B) {
    GemmArgs gh;
    gh.M = NA * N; gh.N = no; gh.K = N; gh.A = c->Bu; gh.lda = N; gh.B = c->Ct; gh.ldb = no; gh.C = c->Hb; gh.ldc = no;
    dgemm(la, gh);
    return;
  }
  for (int P0 = 0; P0 < NA; P0 += c->pc) {
    const int np = std::min(c->pc, NA - P0);
    double* Hc = c->Hb + (size_t)P0 * N * no;
    if (digits > 0) {
      OzGemmArgs g1;
      g1.A = oz_slice(la, c->Bp + (size_t)P0 * c->npp, np * N, N, 0, 0, 0, 1, digits, 0, c->Bz, 0, c->npp, N);
      g1.B = *Cop; g1.M = np * N; g1.N = no; g1.s = digits; g1.C = Hc; g1.cs_m1 = no; g1.cs_n = 1;
      oz_gemm(la, g1);
    } else {
      unpack_sym_batch(la, c->Bp + (size_t)P0 * c->npp, np, N, c->npp, c->Bu);
      GemmArgs gh;
      gh.M = np * N; gh.N = no; gh.K = N; gh.A = c->Bu; gh.lda = N; gh.B = c->Ct; gh.ldb = no; gh.C = Hc;
      gh.ldc = no;
      dgemm(la, gh);
    }
  }
}

// F = h + J + K for the current C; writes D, J, K, F, Ct and scal[0] = E.
static void fock_build(rihf_ctx* c) {
  LaCtx la = c->la();
  const int N = c->N, NA = c->NA, no = c->nocc;
  const size_t n2 = (size_t)N * N;
  // Ct = sqrt(2) C[:, :nocc]; D = Ct Ct^T
  form_Ct(c);
  GemmArgs gd;
  gd.M = N; gd.N = N; gd.K = no; gd.A = c->Ct; gd.lda = no; gd.B = c->Ct; gd.ldb = no; gd.transB = true;
  gd.C = c->D; gd.ldc = N;
  dgemm(la, gd);
  ri_j(c);
  // RI-K: Hb[P] = B^P Ct (N x nocc); K = -1/2 sum_P Hb[P] Hb[P]^T
  form_H(c, 0, nullptr, "RI-K H=B C~ (dgemm)");
  GemmArgs gk;
  gk.M = N; gk.N = N; gk.K = no; gk.A = c->Hb; gk.lda = no; gk.sA = (long long)N * no;
  gk.B = c->Hb; gk.ldb = no; gk.sB = (long long)N * no; gk.transB = true;
  gk.C = c->K; gk.ldc = N; gk.batch = NA; gk.reduce_batch = true; gk.alpha = -0.5;
  gk.lower_only = true;   // K is symmetric: lower tiles only, then mirror
  { TraceScope t(c->tracer, c->stream, "RI-K K=-1/2 sum H H^T (dgemm)", 2.0 * NA * n2 * no, 0);
    dgemm(la, gk);
    symmetrize_lower(la, c->K, N, 1); }
  add3(la, (int)n2, c->H, c->J, c->K, c->F);
  if (c->sph_avg) {
    sph_avg_kernel<<<std::max(1, std::min(ceil_div((long long)n2, 256), 8 * c->sms)), 256, 0, c->stream>>>(
        c->F, N, c->d_fao0, c->d_fl, c->d_fm, c->T1);
    RIHF_LAUNCH_CHECK();
    RIHF_CUDA(cudaMemcpyAsync(c->F, c->T1, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->stream));
    c->launches += 1;
  }
  energy_mb_kernel<<<kRedBlocks, 256, 0, c->stream>>>(c->D, c->H, c->F, (long long)n2, c->d_red, c->d_ticket,
                                                        c->scal);
  RIHF_LAUNCH_CHECK();
  c->launches += 1;
}

// Mixed-precision Fock build: D, RI-J (Eq. j_ri) and everything else in FP64;
// RI-K (Eqs. k_ri_2, tp) on the tensor cores from `digits` BF16 digit planes:
// H = B C~ with B's planes cut once per geometry, then K = -1/2 sum_P H^P H^P^T
// with H cut per K block (one block per split of the long (P, i) axis).
// Autotuner of the tensor-core K GEMM: the number of splits of the long (P, i)
// axis (one CTA per lower tile and split; at most 30 chunks per split) is timed
// for a few candidates around one wave of CTAs on the first build (H is
// already formed), and the fastest is kept for the context.
// Output tiles of the lower triangle of an N x N result with column tile TN.
static int k_lower_tiles(int N, int TN) {
  int n = 0;
  for (int mt = 0; mt * kOzTileM < N; ++mt)
    for (int nt = 0; nt * TN < N; ++nt)
      if (mt * kOzTileM + kOzTileM - 1 >= nt * TN) ++n;
  return n;
}

// Tile-shape autotuner of the tensor-core K GEMM (K = -1/2 H H^T, K dimension
// (P, i)): times each candidate column tile (the whole of N when N <= 64, else
// 32 and 64) with K split counts around one wave of items over the SMs, on
// this context's own H, and keeps the fastest (c->k_tn, c->k_nsplit).
static void tune_k_gemm(rihf_ctx* c, int digits, int kch) {
  LaCtx la = c->la();
  const int N = c->N, NA = c->NA, no = c->nocc;
  const int lo = (kch + kOzMaxChunksPerBlock - 1) / kOzMaxChunksPerBlock;
  std::vector<int> tns;
  if (N <= kOzMaxTN) tns.push_back((N + 15) / 16 * 16);
  else tns = {32, kOzMaxTN};
  cudaEvent_t e0, e1;
  RIHF_CUDA(cudaEventCreate(&e0));
  RIHF_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  for (int tn : tns) {
    const int wave = std::max(1, c->sms / std::max(1, k_lower_tiles(N, tn)));
    std::vector<int> cand;
    for (int k : {wave / 2, wave, 2 * wave, 4 * wave}) {
      const int v = std::min(std::max(k, lo), kch);
      if (std::find(cand.begin(), cand.end(), v) == cand.end()) cand.push_back(v);
    }
    for (int ns : cand) {
      const int kbc = (kch + ns - 1) / ns;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {   // the first pass warms up
        RIHF_CUDA(cudaEventRecord(e0, c->stream));
        OzOperand Hop = oz_slice(la, c->Hb, N, NA * no, no, 1, (long long)N * no, no, digits, kbc, c->Hz);
        RIHF_CUDA(cudaMemsetAsync(c->K, 0, sizeof(double) * N * N, c->stream));
        OzGemmArgs g2;
        g2.A = Hop; g2.B = Hop; g2.M = N; g2.N = N; g2.s = digits; g2.alpha = -0.5; g2.C = c->K; g2.cs_m1 = N;
        g2.cs_n = 1; g2.atomic = true; g2.lower_only = true; g2.tn = tn;
        oz_gemm(la, g2);
        RIHF_CUDA(cudaEventRecord(e1, c->stream));
        RIHF_CUDA(cudaEventSynchronize(e1));
        RIHF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      }
      if (ms < best_ms) {
        best_ms = ms;
        c->k_tn = tn;
        c->k_nsplit = ns;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (c->verbose || getenv("RIHF_VERBOSE"))
    fprintf(stderr, "rihf: K GEMM column tile %d, splits %d (%.3f ms)\n", c->k_tn, c->k_nsplit, best_ms);
}

static void fock_build_tc(rihf_ctx* c, int digits) {
  LaCtx la = c->la();
  const int N = c->N, NA = c->NA, no = c->nocc;
  const size_t n2 = (size_t)N * N;
  form_Ct(c);
  GemmArgs gd;
  gd.M = N; gd.N = N; gd.K = no; gd.A = c->Ct; gd.lda = no; gd.B = c->Ct; gd.ldb = no; gd.transB = true;
  gd.C = c->D; gd.ldc = N;
  dgemm(la, gd);
  ri_j(c);
  const double prod = oz_products(digits);
  OzOperand Cop = oz_slice(la, c->Ct, no, N, 1, no, 0, N, digits, 0, c->Cz);
  // H[(P, mu)][i] = sum_nu B[(P, mu)][nu] C~[nu][i]
  form_H(c, digits, &Cop, "RI-K H=B C~ (tcgen05 digits)");
  // K blocks of the (P, i) axis: enough splits to cover the SMs, at most
  // kOzMaxChunksPerBlock chunks each (int64 headroom of the accumulators)
  const int kch = (NA * no + kOzChunk - 1) / kOzChunk;
  if (c->k_nsplit <= 0) tune_k_gemm(c, digits, kch);
  const int TN = c->k_tn;
  const int lower_tiles = k_lower_tiles(N, TN);
  const int kbc = (kch + c->k_nsplit - 1) / c->k_nsplit;
  OzOperand Hop;
  { TraceScope t(c->tracer, c->stream, "RI-K H digit planes (oz_slice)", (double)NA * N * no * (8 + 2 * digits), 1);
    Hop = oz_slice(la, c->Hb, N, NA * no, no, 1, (long long)N * no, no, digits, kbc, c->Hz); }
  RIHF_CUDA(cudaMemsetAsync(c->K, 0, sizeof(double) * n2, c->stream));
  OzGemmArgs g2;   // K = -1/2 sum_(P, i) H[mu][(P, i)] H[nu][(P, i)], lower tiles
  g2.A = Hop; g2.B = Hop; g2.M = N; g2.N = N; g2.s = digits; g2.alpha = -0.5; g2.C = c->K; g2.cs_m1 = N;
  g2.cs_n = 1; g2.atomic = true; g2.lower_only = true; g2.tn = TN;
  { TraceScope t(c->tracer, c->stream, "RI-K K=-1/2 sum H H^T (tcgen05 digits)",
                 2.0 * lower_tiles * kOzTileM * TN * (double)kch * kOzChunk * prod, 3);
    oz_gemm(la, g2);
    symmetrize_lower(la, c->K, N, 1); }
  add3(la, (int)n2, c->H, c->J, c->K, c->F);
  energy_mb_kernel<<<kRedBlocks, 256, 0, c->stream>>>(c->D, c->H, c->F, (long long)n2, c->d_red, c->d_ticket,
                                                        c->scal);
  RIHF_LAUNCH_CHECK();
  c->launches += 1;
}

// DIIS error X^T (F D S - S D F) X into Err (nind x nind) and scal[1] = max|e|.
static void diis_error(rihf_ctx* c) {
  LaCtx la = c->la();
  const int N = c->N, n = c->nind;
  GemmArgs g1;   // T1 = F D
  g1.M = N; g1.N = N; g1.K = N; g1.A = c->F; g1.lda = N; g1.B = c->D; g1.ldb = N; g1.C = c->T1; g1.ldc = N;
  dgemm(la, g1);
  GemmArgs g2;   // T2 = T1 S
  g2.M = N; g2.N = N; g2.K = N; g2.A = c->T1; g2.lda = N; g2.B = c->S; g2.ldb = N; g2.C = c->T2; g2.ldc = N;
  dgemm(la, g2);
  antisym(la, c->T2, c->T1, N);   // T1 = FDS - SDF
  GemmArgs g3;   // T2 (N x n) = T1 Xo
  g3.M = N; g3.N = n; g3.K = N; g3.A = c->T1; g3.lda = N; g3.B = c->Xo; g3.ldb = n; g3.C = c->T2; g3.ldc = n;
  dgemm(la, g3);
  GemmArgs g4;   // Err = Xo^T T2
  g4.M = n; g4.N = n; g4.K = N; g4.A = c->Xo; g4.lda = n; g4.transA = true; g4.B = c->T2; g4.ldb = n;
  g4.C = c->Err; g4.ldc = n;
  dgemm(la, g4);
  maxabs_mb_kernel<<<kRedBlocks, 256, 0, c->stream>>>((long long)n * n, c->Err, c->d_red, c->d_ticket, c->scal + 1);
  RIHF_LAUNCH_CHECK();
  c->launches += 1;
}

// S^{1/2} and S^{-1/2} of the current geometry's overlap matrix, once per
// geometry.  With nothing below lindep_tau (the orthogonaliser kept all N
// functions) by the scaled coupled Newton-Schulz iteration
//   Y_0 = S / c, Z_0 = I,  T = (3I - Z Y) / 2,  Y <- Y T,  Z <- T Z
// (c = ||S||_F >= lambda_max), which converges to (S/c)^{1/2}, (S/c)^{-1/2}
// quadratically once the small eigenvalues have grown by ~1.5x per step:
// eigenvectors of nearly degenerate small eigenvalues of S, as an eigensolver
// returns them mixed inside their cluster, would leave errors of
// (sqrt(w_i) - sqrt(w_j)) times the mixing.  With dropped eigenvalues, from
// the eigenpairs: S^{1/2} over all, the pseudo-inverse S^{-1/2} over the kept.
static void lowdin_factors(rihf_ctx* c) {
  if (c->lowdin_serial == c->geom_serial) return;
  LaCtx la = c->la();
  cudaStream_t s = c->stream;
  const int N = c->N;
  const size_t n2 = (size_t)N * N;
  if (!c->Shalf) {
    c->Shalf = dalloc<double>(n2);
    c->Smhalf = dalloc<double>(n2);
    c->DL = dalloc<double>(n2);
  }
  TraceScope t(c->tracer, s, "Loewdin factors S^{+-1/2} of the guess", 0.0, 0);
  if (c->nind == N) {
    dot(la, N * N, c->S, c->S, c->scal + 4);
    double fro2 = 0.0;
    RIHF_CUDA(cudaMemcpyAsync(&fro2, c->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    const double cs = std::sqrt(fro2);
    if (!(cs > 0.0) || !std::isfinite(cs)) throw RihfError(RIHF_ERR_NOT_POSITIVE_DEFINITE, "overlap matrix norm");
    scale_copy(la, N * N, 1.0 / cs, c->S, c->Shalf);   // Y
    identity(la, c->Smhalf, N);                         // Z
    for (int it = 0; it < 80; ++it) {
      GemmArgs e;   // T1 = Z Y
      e.M = N; e.N = N; e.K = N; e.A = c->Smhalf; e.lda = N; e.B = c->Shalf; e.ldb = N; e.C = c->T1; e.ldc = N;
      dgemm(la, e);
      if (it >= 12 && it % 3 == 0) {
        eig_check_mb_kernel<<<kRedBlocks, 256, 0, s>>>(c->T1, N, 1.0, 0, c->d_red, c->d_ticket, c->scal + 4);
        RIHF_LAUNCH_CHECK();
        double r = 1.0;
        RIHF_CUDA(cudaMemcpyAsync(&r, c->scal + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
        RIHF_CUDA(cudaStreamSynchronize(s));
        if (r < 1e-12) break;     // Z Y = I: the factors stand
      }
      identity(la, c->T2, N);
      axpby(la, N * N, -0.5, c->T1, 1.5, c->T2, c->T2);        // T2 = (3I - Z Y) / 2
      GemmArgs y;   // T1 = Y T2
      y.M = N; y.N = N; y.K = N; y.A = c->Shalf; y.lda = N; y.B = c->T2; y.ldb = N; y.C = c->T1; y.ldc = N;
      dgemm(la, y);
      GemmArgs z;   // DL = T2 Z
      z.M = N; z.N = N; z.K = N; z.A = c->T2; z.lda = N; z.B = c->Smhalf; z.ldb = N; z.C = c->DL; z.ldc = N;
      dgemm(la, z);
      RIHF_CUDA(cudaMemcpyAsync(c->Shalf, c->T1, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
      RIHF_CUDA(cudaMemcpyAsync(c->Smhalf, c->DL, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
      c->launches += 6;
    }
    scale_copy(la, N * N, std::sqrt(cs), c->Shalf, c->Shalf);
    scale_copy(la, N * N, 1.0 / std::sqrt(cs), c->Smhalf, c->Smhalf);
    RIHF_CUDA(cudaStreamSynchronize(s));
  } else {
    eigh(la, c->S, N, c->Sw, c->Sv, c->eigws, 4, nullptr);
    std::vector<double> w(N);
    RIHF_CUDA(cudaMemcpyAsync(w.data(), c->Sw, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    int k0 = 0;
    while (k0 < N && w[k0] <= c->opt.lindep_tau) ++k0;
    if (k0 == N) throw RihfError(RIHF_ERR_NOT_POSITIVE_DEFINITE, "overlap matrix has no eigenvalue above lindep_tau");
    std::vector<double> r(N);
    for (int i = 0; i < N; ++i) r[i] = std::sqrt(std::max(w[i], 0.0));
    RIHF_CUDA(cudaMemcpyAsync(c->dvec, r.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    scale_cols(la, c->Sv, c->dvec, N, N, c->T1);                  // U diag(sqrt w)
    GemmArgs g1;   // S^{1/2} = T1 U^T
    g1.M = N; g1.N = N; g1.K = N; g1.A = c->T1; g1.lda = N; g1.B = c->Sv; g1.ldb = N; g1.transB = true;
    g1.C = c->Shalf; g1.ldc = N;
    dgemm(la, g1);
    RIHF_CUDA(cudaStreamSynchronize(s));
    const int nk = N - k0;
    for (int i = 0; i < nk; ++i) r[i] = 1.0 / std::sqrt(w[k0 + i]);
    RIHF_CUDA(cudaMemcpyAsync(c->dvec, r.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, s));
    copy_cols(la, c->Sv + k0, N, N, nk, 1.0, c->T2);              // kept eigenvectors
    scale_cols(la, c->T2, c->dvec, N, nk, c->T1);                 // U_k diag(1/sqrt w_k)
    GemmArgs g2;   // S^{-1/2} = T1 U_k^T
    g2.M = N; g2.N = N; g2.K = nk; g2.A = c->T1; g2.lda = nk; g2.B = c->T2; g2.ldb = nk; g2.transB = true;
    g2.C = c->Smhalf; g2.ldc = N;
    dgemm(la, g2);
    RIHF_CUDA(cudaStreamSynchronize(s));
    c->launches += 6;
  }
  c->lowdin_serial = c->geom_serial;
}

// out = X D X for symmetric X (in place allowed: out may be D).
static void congruence(rihf_ctx* c, const double* X, const double* D, double* out) {
  LaCtx la = c->la();
  const int N = c->N;
  GemmArgs g1;   // T1 = X D
  g1.M = N; g1.N = N; g1.K = N; g1.A = X; g1.lda = N; g1.B = D; g1.ldb = N; g1.C = c->T1; g1.ldc = N;
  dgemm(la, g1);
  GemmArgs g2;   // out = T1 X
  g2.M = N; g2.N = N; g2.K = N; g2.A = c->T1; g2.lda = N; g2.B = X; g2.ldb = N; g2.C = out; g2.ldc = N;
  dgemm(la, g2);
}

// After a converged SCF: one online training step of the network on this
// geometry's example (features built for the guess, target = converged D minus
// the extrapolation, scaled by the RMS of the first target), then push D, S and
// the nuclear positions into the history.
static void learn_and_push_history(rihf_ctx* c) {
  cudaStream_t s = c->stream;
  const int N = c->N;
  const size_t n2 = (size_t)N * N;
  const double* Dh = c->D;   // the density as the history holds it
  if (c->hist_lowdin) {
    lowdin_factors(c);
    congruence(c, c->Shalf, c->D, c->DL);
    Dh = c->DL;
  }
  if (c->pending_example) {
    const int M = N * (N + 1) / 2;
    if (c->ml_scale <= 0.0) {
      // RMS of the first target fixes the output scale
      mlp_target(s, N, Dh, c->mlDx, 1.0, c->mlt);
      std::vector<float> t(M);
      RIHF_CUDA(cudaMemcpyAsync(t.data(), c->mlt, sizeof(float) * M, cudaMemcpyDeviceToHost, s));
      RIHF_CUDA(cudaStreamSynchronize(s));
      double ss = 0.0;
      for (float v : t) ss += (double)v * v;
      c->ml_scale = std::max(std::sqrt(ss / M), 1e-12);
    }
    mlp_target(s, N, Dh, c->mlDx, c->ml_scale, c->mlt);
    // out-of-sample check on this (not yet seen) example, then replay
    // training on the last kReplay examples
    float first[2] = {0.f, 0.f};
    mlp_backward(s, c->net, c->mlX, c->mlt, M);
    RIHF_CUDA(cudaMemcpyAsync(first, c->net.loss, sizeof(first), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaMemcpyAsync(c->rep_X + (size_t)c->rep_head * M * kMlpF, c->mlX, sizeof(float) * M * kMlpF,
                              cudaMemcpyDeviceToDevice, s));
    RIHF_CUDA(cudaMemcpyAsync(c->rep_t + (size_t)c->rep_head * M, c->mlt, sizeof(float) * M,
                              cudaMemcpyDeviceToDevice, s));
    c->rep_head = (c->rep_head + 1) % rihf_ctx::kReplay;
    c->nrep = std::min(c->nrep + 1, rihf_ctx::kReplay);
    for (int k = 0; k < c->adam_iters; ++k) {
      mlp_backward(s, c->net, c->rep_X, c->rep_t, c->nrep * M);
      mlp_adam(s, c->net, (float)c->ml_lr);
    }
    c->launches += 2 + 2 * c->adam_iters;
    RIHF_CUDA(cudaStreamSynchronize(s));
    // loss of the network before this step's update, relative to the
    // extrapolation's (y = 0): an out-of-sample check of the prediction
    c->ml_last_ratio = first[1] > 0.f ? (double)first[0] / first[1] : 1e300;
    c->ml_ratios[c->trained_steps % 3] = c->ml_last_ratio;
    ++c->trained_steps;
    c->pending_example = false;
  }
  std::swap(c->hist_D[2], c->hist_D[1]);
  std::swap(c->hist_D[1], c->hist_D[0]);
  RIHF_CUDA(cudaMemcpyAsync(c->hist_D[0], Dh, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
  RIHF_CUDA(cudaMemcpyAsync(c->hist_S, c->S, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
  std::swap(c->hist_xyz[1], c->hist_xyz[0]);
  RIHF_CUDA(cudaMemcpyAsync(c->hist_xyz[0], c->d_xyz, sizeof(double) * 3 * c->natoms, cudaMemcpyDeviceToDevice, s));
  c->nhist = std::min(c->nhist + 1, 3);
}

// One SCF iteration's Fock build (variant 0: FP64, d: tensor-core RI-K with d
// digits) and DIIS error, replayed from a CUDA graph captured on first use
// (launch overhead matters for small molecules in batches).  The captured
// work reads and writes only the context's fixed buffers; the autotuner runs
// eagerly before the first capture of a tensor-core variant.
static void fock_and_error(rihf_ctx* c, int variant) {
  auto eager = [&]() {
    if (variant == 0) fock_build(c);
    else fock_build_tc(c, variant);
    diis_error(c);
  };
  if (!c->opt.cuda_graphs || !c->graphs_ok || (variant > 0 && c->k_nsplit <= 0)) {
    eager();
    return;
  }
  auto& g = c->graphs[variant];
  if (!g.exec) {
    const long long l0 = c->launches;
    const bool tr = c->tracer.on;   // no trace events inside the captured graph
    c->tracer.on = false;
    RIHF_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
      eager();
    } catch (...) {
      cudaStreamEndCapture(c->stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      c->launches = l0;
      c->graphs_ok = false;
      c->tracer.on = tr;
      eager();
      return;
    }
    c->tracer.on = tr;
    RIHF_CUDA(cudaStreamEndCapture(c->stream, &graph));
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    g.launches = c->launches - l0;
    c->launches = l0;
    if (e != cudaSuccess) {
      cudaGetLastError();
      g.exec = nullptr;
      c->graphs_ok = false;
      eager();
      return;
    }
  }
  {
    static const char* names[kOzMaxDigits + 1] = {
        "SCF iteration graph: FP64 Fock build + DIIS error", "SCF iteration graph: tensor-core RI-K, 1 digit",
        "SCF iteration graph: tensor-core RI-K, 2 digits", "SCF iteration graph: tensor-core RI-K, 3 digits",
        "SCF iteration graph: tensor-core RI-K, 4 digits", "SCF iteration graph: tensor-core RI-K, 5 digits",
        "SCF iteration graph: tensor-core RI-K, 6 digits", "SCF iteration graph: tensor-core RI-K, 7 digits"};
    TraceScope t(c->tracer, c->stream, names[variant], 0.0, 0);
    RIHF_CUDA(cudaGraphLaunch(g.exec, c->stream));
  }
  c->launches += g.launches;
}

// Superposition of atomic densities (the paper's cold-start guess, Sec. 2.2):
// occupation numbers of the spherically averaged ground-state atom (aufbau
// 1s 2s 2p, the open shell shared evenly over its orbitals), H to Ne.
static bool sad_occupations(int Z, std::vector<double>& occ, std::vector<int>& occ_l) {
  occ.clear();
  occ_l.clear();
  if (Z < 1 || Z > 10) return false;
  int left = Z;
  for (int k = 0; k < 2 && left > 0; ++k) {   // 1s, 2s
    occ.push_back(std::min(2, left));
    occ_l.push_back(0);
    left -= std::min(2, left);
  }
  if (left > 0)
    for (int k = 0; k < 3; ++k) {   // 2p, spherically averaged
      occ.push_back(left / 3.0);
      occ_l.push_back(1);
    }
  return true;
}

// SAD atoms: after a diagonalisation, the occupied columns follow the
// configuration (occ_l: the l of each occupied orbital, lowest orbital of that
// l first) rather than the eigenvalue order; the spherical average makes every
// eigenvector pure in l.  The small basis sets of the workloads put the O 2p
// level below 2s, where eigenvalue order would occupy a non-spherical set.
static void occupy_by_l(rihf_ctx* c) {
  const int N = c->N, n = c->nind;
  std::vector<double> C((size_t)N * N), e(N);
  RIHF_CUDA(cudaMemcpyAsync(C.data(), c->C, sizeof(double) * C.size(), cudaMemcpyDeviceToHost, c->stream));
  RIHF_CUDA(cudaMemcpyAsync(e.data(), c->eps, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
  RIHF_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<int> lcol(n), order(n), chosen;
  for (int j = 0; j < n; ++j) {
    int best = 0;
    for (int i = 1; i < N; ++i)
      if (std::fabs(C[(size_t)i * N + j]) > std::fabs(C[(size_t)best * N + j])) best = i;
    lcol[j] = c->fl_h[best];
    order[j] = j;   // columns are already in ascending eigenvalue order
  }
  for (int l : c->occ_l) {
    int pick = -1;
    for (int j : order)
      if (lcol[j] == l && std::find(chosen.begin(), chosen.end(), j) == chosen.end()) { pick = j; break; }
    if (pick < 0) return;   // configuration not representable: keep the eigenvalue order
    chosen.push_back(pick);
  }
  std::vector<int> idx = chosen;
  for (int j : order)
    if (std::find(chosen.begin(), chosen.end(), j) == chosen.end()) idx.push_back(j);
  std::vector<double> C2(C), e2(e);
  for (int q = 0; q < n; ++q) {
    e2[q] = e[idx[q]];
    for (int i = 0; i < N; ++i) C2[(size_t)i * N + q] = C[(size_t)i * N + idx[q]];
  }
  upload(c->C, C2, c->stream);
  upload(c->eps, e2, c->stream);
}

// Builds the SAD factor Fs (N x m): for every atom type (element and identical
// primary and auxiliary shells) one RI-HF SCF of the isolated, spherically
// averaged atom (fractional occupations, FP64, this library's kernels), its
// occupied orbitals scaled by sqrt(n_i) placed on each atom's basis-function
// block.  D_SAD = Fs Fs^T.  On any obstacle (elements beyond Ne, an atom's
// functions not contiguous) sad_ok stays false and the core guess is used.
static void build_sad(rihf_ctx* c) {
  c->sad_built = true;
  c->sad_ok = false;
  const int N = c->N;
  const HostShells &hp = c->hp, &ha = c->ha;
  std::vector<int> p0(c->natoms, -1), p1(c->natoms, -1), a0(c->natoms, -1), a1(c->natoms, -1);
  for (int i = 0; i < hp.nshell; ++i) {
    const int a = hp.atom[i];
    if (p0[a] < 0) p0[a] = i;
    else if (p1[a] != i) { c->sad_note = "primary shells of an atom are not contiguous"; return; }
    p1[a] = i + 1;
  }
  for (int i = 0; i < ha.nshell; ++i) {
    const int a = ha.atom[i];
    if (a0[a] < 0) a0[a] = i;
    else if (a1[a] != i) { c->sad_note = "auxiliary shells of an atom are not contiguous"; return; }
    a1[a] = i + 1;
  }
  auto sig = [&](int a) {   // element and shells of atom a, exactly
    std::string k = std::to_string(c->Z[a]) + "|";
    auto add = [&](const HostShells& h, int s0, int s1) {
      for (int i = s0; i < s1; ++i) {
        k += std::to_string(h.l[i]) + ":";
        for (int q = 0; q < h.nprim[i]; ++q) {
          char buf[64];
          snprintf(buf, sizeof(buf), "%.17g/%.17g,", h.exps[h.pstart[i] + q], h.raw_coefs[h.pstart[i] + q]);
          k += buf;
        }
        k += ";";
      }
      k += "|";
    };
    if (p0[a] >= 0) add(hp, p0[a], p1[a]);
    if (a0[a] >= 0) add(ha, a0[a], a1[a]);
    return k;
  };
  struct AtomType {
    int na = 0, m = 0;
    std::vector<double> F;   // na x m, row-major
  };
  std::vector<std::string> keys;
  std::vector<AtomType> types;
  std::vector<int> type_of(c->natoms);
  double zsum = 0.0;
  for (int a = 0; a < c->natoms; ++a) {
    zsum += c->Z[a];
    if (p0[a] < 0 || a0[a] < 0) { c->sad_note = "an atom without primary or auxiliary shells"; return; }
    const std::string k = sig(a);
    int t = (int)(std::find(keys.begin(), keys.end(), k) - keys.begin());
    if (t == (int)keys.size()) {
      std::vector<double> occ;
      std::vector<int> occ_l;
      if (!sad_occupations(c->Z[a], occ, occ_l)) { c->sad_note = "SAD occupations known for H to Ne only"; return; }
      std::vector<rihf_shell> ps, as;
      for (int i = p0[a]; i < p1[a]; ++i)
        ps.push_back({0, hp.l[i], hp.nprim[i], &hp.exps[hp.pstart[i]], &hp.raw_coefs[hp.pstart[i]]});
      for (int i = a0[a]; i < a1[a]; ++i)
        as.push_back({0, ha.l[i], ha.nprim[i], &ha.exps[ha.pstart[i]], &ha.raw_coefs[ha.pstart[i]]});
      rihf_options o = c->opt;
      o.precision = RIHF_PRECISION_FP64;
      o.cuda_graphs = 0;
      o.aux_chunk = 0;
      o.schwarz_tau = 0.0;
      o.max_iter = 200;
      o.conv_e = 1e-10;
      o.conv_diis = 1e-7;
      const int zc = c->Z[a];
      const double origin[3] = {0.0, 0.0, 0.0};
      rihf_ctx* sub = nullptr;
      try {
        sub = setup_impl(1, &zc, origin, (int)ps.size(), ps.data(), (int)as.size(), as.data(), zc, &o, &occ);
      } catch (const std::exception& ex) {
        c->sad_note = std::string("atomic context: ") + ex.what();
        cudaGetLastError();
        return;
      }
      if (o.pure) {   // spherical basis: average every Fock matrix of the atom
        std::vector<int> ao0(sub->N), fl(sub->N), fm(sub->N);
        for (int i = 0; i < sub->hp.nshell; ++i)
          for (int k = 0; k < sub->nf_h[sub->hp.l[i]]; ++k) {
            ao0[sub->hp.ao[i] + k] = sub->hp.ao[i];
            fl[sub->hp.ao[i] + k] = sub->hp.l[i];
            fm[sub->hp.ao[i] + k] = k;
          }
        sub->d_fao0 = dalloc<int>(sub->N); upload(sub->d_fao0, ao0, sub->stream);
        sub->d_fl = dalloc<int>(sub->N); upload(sub->d_fl, fl, sub->stream);
        sub->d_fm = dalloc<int>(sub->N); upload(sub->d_fm, fm, sub->stream);
        sub->sph_avg = true;
        sub->fl_h = fl;
        sub->occ_l = occ_l;
      }
      AtomType at;
      at.na = sub->N;
      at.m = sub->nocc;
      std::vector<double> C((size_t)sub->N * sub->N);
      double e = 0.0;
      int it = 0;
      const int rc = rihf_scf(sub, 0, nullptr, &e, nullptr, C.data(), nullptr, &it);
      rihf_destroy(sub);
      if (rc != RIHF_OK && rc != RIHF_ERR_NOT_CONVERGED) { c->sad_note = "atomic SCF failed"; return; }
      at.F.resize((size_t)at.na * at.m);
      for (int r = 0; r < at.na; ++r)
        for (int q = 0; q < at.m; ++q) at.F[(size_t)r * at.m + q] = C[(size_t)r * sub->N + q] * std::sqrt(occ[q]);
      if (c->verbose || getenv("RIHF_VERBOSE"))
        fprintf(stderr, "rihf: SAD atom Z=%d: %d functions, %d occupied, E = %.10f (%d iterations)\n", zc, at.na,
                at.m, e, it);
      keys.push_back(k);
      types.push_back(std::move(at));
    }
    type_of[a] = t;
  }
  // block-diagonal assembly; for an ion the factor is scaled to nelec electrons
  int m = 0;
  for (int a = 0; a < c->natoms; ++a) m += types[type_of[a]].m;
  const double scale = std::sqrt(c->nelec / zsum);
  std::vector<double> Fs((size_t)N * m, 0.0);
  int col = 0;
  for (int a = 0; a < c->natoms; ++a) {
    const AtomType& at = types[type_of[a]];
    const int r0 = hp.ao[p0[a]];
    if (r0 + at.na > N) { c->sad_note = "atom block outside the basis"; return; }
    for (int r = 0; r < at.na; ++r)
      for (int q = 0; q < at.m; ++q) Fs[(size_t)(r0 + r) * m + col + q] = scale * at.F[(size_t)r * at.m + q];
    col += at.m;
  }
  if (c->d_sad) cudaFree(c->d_sad);
  c->d_sad = dalloc<double>(Fs.size());
  upload(c->d_sad, Fs, c->stream);
  RIHF_CUDA(cudaStreamSynchronize(c->stream));
  c->sad_m = m;
  c->sad_ok = true;
}

// First Fock build of a SAD start: D = Fs Fs^T, RI-J from D and RI-K from the
// factor (Eq. k_ri_2 with C~ -> Fs: K = -1/2 sum_P (B^P Fs)(B^P Fs)^T, i.e. the
// density form Eq. k_ri_1 for D_SAD), nocc columns at a time since Fs has more
// columns than occupied orbitals; variant 0 in FP64, else on the tensor cores
// with that many digits.
static void fock_build_factor(rihf_ctx* c, int variant) {
  LaCtx la = c->la();
  const int N = c->N, NA = c->NA, no = c->nocc, m = c->sad_m;
  const size_t n2 = (size_t)N * N;
  cudaStream_t s = c->stream;
  GemmArgs gd;
  gd.M = N; gd.N = N; gd.K = m; gd.A = c->d_sad; gd.lda = m; gd.B = c->d_sad; gd.ldb = m; gd.transB = true;
  gd.C = c->D; gd.ldc = N;
  dgemm(la, gd);
  ri_j(c);
  for (int c0 = 0; c0 < m; c0 += no) {
    const int w = std::min(no, m - c0);
    const bool first = c0 == 0;
    RIHF_CUDA(cudaMemsetAsync(c->Ct, 0, sizeof(double) * N * no, s));
    RIHF_CUDA(cudaMemcpy2DAsync(c->Ct, no * sizeof(double), c->d_sad + c0, m * sizeof(double), w * sizeof(double), N,
                                cudaMemcpyDeviceToDevice, s));
    if (variant > 0) {
      OzOperand Cop = oz_slice(la, c->Ct, no, N, 1, no, 0, N, variant, 0, c->Cz);
      form_H(c, variant, &Cop, "SAD RI-K H=B Fs (tcgen05 digits)");
      const int kch = (NA * no + kOzChunk - 1) / kOzChunk;
      if (c->k_nsplit <= 0) tune_k_gemm(c, variant, kch);   // writes K
      if (first) RIHF_CUDA(cudaMemsetAsync(c->K, 0, sizeof(double) * n2, s));
      const int kbc = (kch + c->k_nsplit - 1) / c->k_nsplit;
      OzOperand Hop = oz_slice(la, c->Hb, N, NA * no, no, 1, (long long)N * no, no, variant, kbc, c->Hz);
      OzGemmArgs g2;
      g2.A = Hop; g2.B = Hop; g2.M = N; g2.N = N; g2.s = variant; g2.alpha = -0.5; g2.C = c->K; g2.cs_m1 = N;
      g2.cs_n = 1; g2.atomic = true; g2.lower_only = true; g2.tn = c->k_tn;
      oz_gemm(la, g2);
    } else {
      form_H(c, 0, nullptr, "SAD RI-K H=B Fs (dgemm)");
      GemmArgs gk;
      gk.M = N; gk.N = N; gk.K = no; gk.A = c->Hb; gk.lda = no; gk.sA = (long long)N * no;
      gk.B = c->Hb; gk.ldb = no; gk.sB = (long long)N * no; gk.transB = true;
      gk.C = c->K; gk.ldc = N; gk.batch = NA; gk.reduce_batch = true; gk.alpha = -0.5; gk.beta = first ? 0.0 : 1.0;
      gk.lower_only = true;
      dgemm(la, gk);
    }
  }
  symmetrize_lower(la, c->K, N, 1);
  add3(la, (int)n2, c->H, c->J, c->K, c->F);
  energy_mb_kernel<<<kRedBlocks, 256, 0, s>>>(c->D, c->H, c->F, (long long)n2, c->d_red, c->d_ticket, c->scal);
  RIHF_LAUNCH_CHECK();
  c->launches += 1;
}

int rihf_scf(rihf_ctx* c, int guess, const double* C_guess, double* energy, double* Dout, double* Cout,
             double* epsout, int* iters) {
  RIHF_API_BEGIN
  if (!c) return RIHF_ERR_INVALID_ARG;
  LaCtx la = c->la();
  const int N = c->N, n = c->nind;
  const size_t n2 = (size_t)N * N;
  cudaStream_t s = c->stream;
  c->timings[1] = c->timings[2] = 0.0;
  cudaEventRecord(c->ev[7], s);   // SCF start (diagonalisation time = total - builds)
  if (!c->Bz.planes && c->pc == c->NA && !c->bu_is_B) {
    // FP64 mode holds all of B expanded in Bu, which the captured Fock-build
    // graphs read; a gradient since the last geometry used Bu as scratch
    unpack_sym_batch(la, c->Bp, c->NA, N, c->npp, c->Bu);
    c->bu_is_B = true;
  }
  if ((guess == 3 || guess == 4) && !c->hist_lowdin) {
    // the history restarts in the Loewdin representation
    c->hist_lowdin = true;
    c->nhist = 0;
  }
  if (guess == 1) {
    if (!C_guess) return RIHF_ERR_INVALID_ARG;
    RIHF_CUDA(cudaMemcpyAsync(c->C, C_guess, sizeof(double) * n2, cudaMemcpyHostToDevice, s));
  } else if (guess >= 2 && guess <= 4 && c->have_orbitals) {
    // previous converged orbitals (the paper's AIMD guess, Sec. 3.3); after a
    // geometry change they are re-orthonormalised against the new overlap:
    // M = Co^T S Co = L_M L_M^T, Co <- Co L_M^{-T} (Cholesky / Gram-Schmidt,
    // stable however far the nuclei moved)
    const int no = c->nocc;
    if (c->have_cprev) {
      // previous eigenvectors expressed in the new orthonormal basis,
      // C' = Xo^T S C_AO (Xo^T S Xo = I), as the eigensolver's starting vectors
      GemmArgs m1;   // T1 (N x n) = S C[:, :n]
      m1.M = N; m1.N = n; m1.K = N; m1.A = c->S; m1.lda = N; m1.B = c->C; m1.ldb = N; m1.C = c->T1; m1.ldc = n;
      dgemm(la, m1);
      GemmArgs m2;   // T2 (n x n) = Xo^T T1
      m2.M = n; m2.N = n; m2.K = N; m2.A = c->Xo; m2.lda = n; m2.transA = true; m2.B = c->T1; m2.ldb = n;
      m2.C = c->T2; m2.ldc = n;
      dgemm(la, m2);
      // orthonormal again by Cholesky (Gram-Schmidt): M = V^T V = L L^T,
      // Cprev^T = L^{-1} V^T; large nuclear steps leave V far from orthonormal
      GemmArgs m3;   // Cprev = T2^T T2
      m3.M = n; m3.N = n; m3.K = n; m3.A = c->T2; m3.lda = n; m3.transA = true; m3.B = c->T2; m3.ldb = n;
      m3.C = c->Cprev; m3.ldc = n;
      dgemm(la, m3);
      RIHF_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
      cholesky(la, c->Cprev, n, c->scratch);
      transpose(la, c->T2, n, n, c->T1);                                // T1 = V^T
      trsm_lower(la, c->Cprev, n, c->T1, n, false, 0, c->trsm_tmp);     // L^{-1} V^T
      transpose(la, c->T1, n, n, c->Cprev);
    }
    copy_cols(la, c->C, N, N, no, 1.0, c->Ct);
    c->last_guess = 2;
    c->pending_example = false;
    if (guess >= 3 && c->nhist >= 3) {
      // density guess: three-point extrapolation D_x = 3 D_t - 3 D_{t-1} + D_{t-2}
      // of the Loewdin densities (guess 3) plus, for guess 4, the network's
      // correction once it beats the extrapolation on its last training
      // example, taken back to the AO basis with this geometry's S^{-1/2};
      // the previous occupied orbitals are carried into the predicted
      // occupied space by one projection Co <- D_pred S Co before the
      // Gram-Schmidt step below
      if (c->ml_sd <= 0.0) {
        // feature scales: RMS of the first observed changes (fixed from then on)
        mlp_scale_sums(s, N, c->hist_D[0], c->hist_D[1], c->S, c->hist_S, c->d_xyz, c->hist_xyz[0], c->d_ao_atom,
                       c->ml_sums);
        double sums[3];
        RIHF_CUDA(cudaMemcpyAsync(sums, c->ml_sums, sizeof(sums), cudaMemcpyDeviceToHost, s));
        RIHF_CUDA(cudaStreamSynchronize(s));
        const double Mh = (double)N * (N + 1) / 2;
        c->ml_sd = std::max(std::sqrt(sums[0] / Mh), 1e-12);
        c->ml_ss = std::max(std::sqrt(sums[1] / Mh), 1e-12);
        c->ml_sr = std::max(std::sqrt(sums[2] / Mh), 1e-12);
        c->launches += 1;
      }
      mlp_features(s, N, c->hist_D[0], c->hist_D[1], c->hist_D[2], c->S, c->hist_S, c->d_xyz, c->hist_xyz[0],
                   c->hist_xyz[1], c->d_ao_atom, c->d_ao_l, c->ml_sd, c->ml_ss, c->ml_sr, c->mlX, c->mlDx);
      const int M = N * (N + 1) / 2;
      // the network is used while the median of its last three out-of-sample
      // ratios (loss / loss of the bare extrapolation) is below 0.8
      double r3[3] = {c->ml_ratios[0], c->ml_ratios[1], c->ml_ratios[2]};
      std::sort(r3, r3 + 3);
      const bool use_net = guess == 4 && c->net_on && c->trained_steps >= 3 && r3[1] < 0.8;
      if (use_net) mlp_forward(s, c->net, c->mlX, M, c->mly);
      mlp_apply(s, N, c->mlDx, use_net ? c->mly : nullptr, c->ml_scale, c->Dpred);
      lowdin_factors(c);
      congruence(c, c->Smhalf, c->Dpred, c->Dpred);
      c->launches += use_net ? 5 : 4;
      c->last_guess = use_net ? 4 : 3;
      c->pending_example = guess == 4 && c->net_on && c->trained_steps < c->train_steps;
      GemmArgs p1;   // T1 (N x no) = S Co
      p1.M = N; p1.N = no; p1.K = N; p1.A = c->S; p1.lda = N; p1.B = c->Ct; p1.ldb = no; p1.C = c->T1; p1.ldc = no;
      dgemm(la, p1);
      GemmArgs p2;   // Co = D_pred T1
      p2.M = N; p2.N = no; p2.K = N; p2.A = c->Dpred; p2.lda = N; p2.B = c->T1; p2.ldb = no; p2.C = c->Ct;
      p2.ldc = no;
      dgemm(la, p2);
    }
    GemmArgs g1;   // T1 (N x no) = S Co
    g1.M = N; g1.N = no; g1.K = N; g1.A = c->S; g1.lda = N; g1.B = c->Ct; g1.ldb = no; g1.C = c->T1; g1.ldc = no;
    dgemm(la, g1);
    GemmArgs g2;   // T2 (no x no) = Co^T T1
    g2.M = no; g2.N = no; g2.K = N; g2.A = c->Ct; g2.lda = no; g2.transA = true; g2.B = c->T1; g2.ldb = no;
    g2.C = c->T2; g2.ldc = no;
    dgemm(la, g2);
    cholesky(la, c->T2, no, c->scratch);
    transpose(la, c->Ct, N, no, c->T1);                        // T1 = Co^T (no x N)
    trsm_lower(la, c->T2, no, c->T1, N, false, 0, c->trsm_tmp);   // L_M^{-1} Co^T
    transpose(la, c->T1, no, N, c->Ct);
    RIHF_CUDA(cudaMemcpy2DAsync(c->C, N * sizeof(double), c->Ct, no * sizeof(double), no * sizeof(double), N,
                                cudaMemcpyDeviceToDevice, s));
  } else if (guess == 5 && (c->sad_built ? c->sad_ok : (build_sad(c), c->sad_ok))) {
    // SAD: the first iteration's Fock matrix comes from D_SAD (below); the
    // first diagonalisation then starts cold
    c->have_cprev = false;
    c->last_guess = 5;
    c->pending_example = false;
  } else {
    if (guess == 5 && (c->verbose || getenv("RIHF_VERBOSE")))
      fprintf(stderr, "rihf: SAD guess unavailable (%s), core Hamiltonian instead\n", c->sad_note.c_str());
    diagonalise(c, c->H, false);
    c->last_guess = 0;
    c->pending_example = false;
  }
  const bool sad_first = c->last_guess == 5;
  const int size = c->opt.diis_size;
  double E = 0.0, Eold = 0.0, emax = 0.0;
  int it = 0;
  bool conv = false;
  float ms = 0.f;
  // Precision ladder (mixed mode): RI-K on the tensor cores with a digit count
  // that follows the SCF error (5 digits, about 39 bits, while max|e| > 1e-2;
  // 6 while > 1e-5; then 7, about 55 bits), or the fixed count of
  // opt.mixed_digits.  When the convergence test passes on a ladder build of
  // fewer digits, the next build is a confirmation build and convergence is
  // declared only on one (or on a 7-digit ladder build, which is the same
  // arithmetic): 7 digits (products with FP64-class accuracy, 55 bits per K block),
  // or FP64 with opt.confirm_fp64; either way the converged energy and density
  // do not carry the ladder's shorter digit counts.  Three ladder builds in a
  // row without a new lowest max|e| also move on to confirmation builds.
  const bool mixed = c->opt.precision == RIHF_PRECISION_MIXED && c->Bz.planes != nullptr;
  bool fp64_next = !mixed;
  double best_tc = 1e300, emax_prev = 1.0;
  int stall = 0;
  // SCF stall recovery: when max|e| has not fallen below 0.9 of its best value
  // for kStallIters iterations, the DIIS history restarts from the current
  // Fock matrix and the next diagonalisation is a full Jacobi pass, so that no
  // fixed point of the warm-started eigensolver or of a degenerate DIIS
  // subspace can hold the iteration
  constexpr int kStallIters = 6;
  double best_err = 1e300;
  int since_best = 0, dbase = 0;
  c->tc_builds = 0;
  c->confirm_builds = 0;
  RIHF_CUDA(cudaMemsetAsync(c->d_flag + 1, 0, sizeof(int), s));
  for (it = 1; it <= c->opt.max_iter; ++it) {
    cudaEventRecord(c->ev[2], s);
    const bool full = fp64_next;
    int variant = 0;
    if (!full) {
      int digits = c->opt.mixed_digits;
      if (digits <= 0) digits = emax_prev > 1e-2 ? 5 : emax_prev > 1e-5 ? 6 : 7;
      variant = std::min(digits, kOzMaxDigits);
      c->last_digits = variant;
      ++c->tc_builds;
    } else if (mixed && !c->opt.confirm_fp64) {
      variant = kOzMaxDigits;
      c->last_digits = variant;
      ++c->confirm_builds;
    }
    if (it == 1 && sad_first) {
      fock_build_factor(c, variant);
      diis_error(c);
    } else {
      fock_and_error(c, variant);
    }
    cudaEventRecord(c->ev[3], s);
    int slot = (it - 1 - dbase) % size;
    int m = std::min(it - dbase, size);
    RIHF_CUDA(cudaMemcpyAsync(c->Fring + slot * n2, c->F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
    RIHF_CUDA(cudaMemcpyAsync(c->Ering + (size_t)slot * n * n, c->Err, sizeof(double) * n * n,
                              cudaMemcpyDeviceToDevice, s));
    double sc[2];
    RIHF_CUDA(cudaMemcpyAsync(sc, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);   // both recorded before the sync
    c->timings[1] += ms;
    E = sc[0];
    emax = sc[1];
    c->prev_err = c->last_err;
    c->last_err = emax;
    if (c->verbose || getenv("RIHF_VERBOSE")) fprintf(stderr, "rihf_scf it %3d  E = %.12f  max|e| = %.3e  dE = %.3e\n", it, E, emax, E - Eold);
    if (!std::isfinite(E)) throw RihfError(RIHF_ERR_NOT_CONVERGED, "SCF energy is not finite");
    const bool crit = it > 1 && std::fabs(E - Eold) < c->opt.conv_e && emax < c->opt.conv_diis;
    emax_prev = emax;
    if (mixed && !full) {
      if (emax < best_tc) {
        best_tc = emax;
        stall = 0;
      } else {
        ++stall;
      }
      if (crit || stall >= 3) fp64_next = true;
    }
    // a ladder build that already used 7 digits is a confirmation build (the
    // same arithmetic): convergence on it is declared at once
    const bool seven = mixed && !full && variant == kOzMaxDigits && !c->opt.confirm_fp64;
    if (crit && (full || seven)) {
      if (seven) {
        --c->tc_builds;
        ++c->confirm_builds;
      }
      conv = true;
      break;
    }
    Eold = E;
    bool restart = false;
    if (emax < 0.9 * best_err) {
      best_err = emax;
      since_best = 0;
    } else if (++since_best >= kStallIters) {
      restart = true;
      since_best = 0;
      best_err = emax;
      dbase = it;              // the next iteration starts a new DIIS history
      c->force_cold = true;    // and this one diagonalises F from scratch
      if (c->verbose || getenv("RIHF_VERBOSE"))
        fprintf(stderr, "rihf_scf it %3d  stalled at max|e| = %.3e: DIIS restart, full diagonalisation\n", it, emax);
    }
    const double* Fuse = c->F;
    if (!restart) {
      TraceScope t(c->tracer, s, "DIIS (dots, solve, extrapolation)", 0.0, 0);
      diis_dots_mb_kernel<<<dim3(kRedDiis, m), 256, 0, s>>>(c->Ering, (long long)n * n, slot, m, c->Bdiis, 16, c->d_red,
                                                             c->d_ticket);
      RIHF_LAUNCH_CHECK();
      if (m >= 2) {
        diis_solve_kernel<<<1, 32, 0, s>>>(c->Bdiis, 16, m, c->coef);
        diis_extrap_kernel<<<std::max(1, std::min(ceil_div((long long)n2, 256), 8 * c->sms)), 256, 0, s>>>(
            c->Fring, (long long)n2, m, c->coef, c->Fx);
        RIHF_LAUNCH_CHECK();
        Fuse = c->Fx;
      }
    }
    if (!restart) c->launches += 3;
    // no host synchronisation here: the next Fock build queues behind the
    // diagonalisation on the stream
    diagonalise(c, Fuse, true);
  }
  if (it > c->opt.max_iter) it = c->opt.max_iter;
  // final orbitals diagonalise the last (unextrapolated) Fock matrix
  diagonalise(c, c->F, true);
  c->converged = conv;
  c->have_orbitals = true;
  int tc_flag = 0;
  RIHF_CUDA(cudaMemcpyAsync(&tc_flag, c->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  cudaEventRecord(c->ev[4], s);
  RIHF_CUDA(cudaStreamSynchronize(s));
  cudaEventElapsedTime(&ms, c->ev[7], c->ev[4]);
  c->timings[2] = std::max(0.0, (double)ms - c->timings[1]);
  c->tracer.flush();
  if (tc_flag) throw RihfError(RIHF_ERR_TIMEOUT, "tensor-core RI-K: a bounded device wait ran out");
  if (conv) learn_and_push_history(c);
  if (energy) *energy = E;
  if (iters) *iters = it;
  c->last_iters = it;
  if (Dout) RIHF_CUDA(cudaMemcpy(Dout, c->D, sizeof(double) * n2, cudaMemcpyDeviceToHost));
  if (Cout) RIHF_CUDA(cudaMemcpy(Cout, c->C, sizeof(double) * n2, cudaMemcpyDeviceToHost));
  if (epsout) RIHF_CUDA(cudaMemcpy(epsout, c->eps, sizeof(double) * N, cudaMemcpyDeviceToHost));
  if (!conv) {
    g_last_error = "SCF did not converge in max_iter iterations (max|e| = " + std::to_string(emax) + ")";
    return RIHF_ERR_NOT_CONVERGED;
  }
  return RIHF_OK;
  RIHF_API_END
}

// The gradient up to its per-atom parts on the device (Eq. rihf_gradient):
// fitted densities, Y, Z and the fused derivative contractions.  defer_eri3:
// the 3-centre contraction is left to a batched launch over several contexts
// (launch_grad_eri3_batch into grad_parts + 6 natoms).
static void gradient_launch(rihf_ctx* c, bool defer_eri3) {
  LaCtx la = c->la();
  IntegralCtx ic = c->ic();
  const int N = c->N, NA = c->NA, no = c->nocc, nat = c->natoms;
  const size_t n2 = (size_t)N * N;
  cudaStream_t s = c->stream;
  cudaEventRecord(c->ev[5], s);
  // Ct, D from the final orbitals; W = Ct diag(eps_occ) Ct^T
  form_Ct(c);
  GemmArgs gd;
  gd.M = N; gd.N = N; gd.K = no; gd.A = c->Ct; gd.lda = no; gd.B = c->Ct; gd.ldb = no; gd.transB = true;
  gd.C = c->D; gd.ldc = N;
  dgemm(la, gd);
  // W = 2 sum_i eps_i C_i C_i^T = 1/2 D F D at convergence (C~^T F C~ = 2 diag(eps_occ));
  // this form needs no individual eigenvectors inside near-degenerate clusters
  GemmArgs gf;
  gf.M = N; gf.N = N; gf.K = N; gf.A = c->F; gf.lda = N; gf.B = c->D; gf.ldb = N; gf.C = c->T2; gf.ldc = N;
  dgemm(la, gf);
  GemmArgs gw;
  gw.M = N; gw.N = N; gw.K = N; gw.A = c->D; gw.lda = N; gw.B = c->T2; gw.ldb = N; gw.C = c->W; gw.ldc = N;
  gw.alpha = 0.5;
  dgemm(la, gw);
  // d = B vec D; c = L^{-T} d (the paper's L^P) is solved below together with X~
  { TraceScope t(c->tracer, s, "grad d = B D (gemv over packed rows)", (double)NA * c->npp * 8, 1);
    pack_sym(la, c->D, N, 2.0, c->Dp);
    gemv_rows(la, c->Bp, NA, c->npp, c->Dp, 1.0, c->dvec); }
  const long long ldx = (long long)no * no + 1;   // row P of Xt: X~^P (nocc^2) then c_P
  // Hb[P] = B^P Ct ; Bij[P] = Ct^T Hb[P]
  const bool tc = c->Gz.planes != nullptr;   // mixed mode: 7-digit tensor-core GEMMs (FP64-class products)
  OzOperand Cop;   // C~^T planes: rows i, K = mu (tensor-core path)
  if (tc) {
    Cop = oz_slice(la, c->Ct, no, N, 1, no, 0, N, kOzMaxDigits, 0, c->Cz);
    form_H(c, kOzMaxDigits, &Cop, "grad H=B C~ (tcgen05 7 digits)");
  } else {
    form_H(c, 0, nullptr, "grad H=B C~ (dgemm)");
  }
  // Bij on the tensor cores when K = N fits one exponent block, chunk by chunk
  // of auxiliary functions in the G' plane buffer (rows (P, j) of H)
  const bool tc_bij = tc && (N + kOzChunk - 1) / kOzChunk <= kOzMaxChunksPerBlock &&
                      oz_plane_elems(c->pc * no, N, kOzMaxDigits) <= c->Gz.cap &&
                      (size_t)((c->pc * no + kOzTileM - 1) / kOzTileM * kOzTileM) <= c->Gz.ecap;
  if (tc_bij) {
    // rows (P, j) of H (element (P, mu, j) at Hb[P N nocc + mu nocc + j]), K = mu; Bij[P]
    // is symmetric in (i, j) and goes per P as [j][i] straight into [X~ | c]
    TraceScope t(c->tracer, s, "grad Bij = C~^T H (tcgen05 7 digits)", 0.0, 0);
    for (int P0 = 0; P0 < NA; P0 += c->pc) {
      const int np = std::min(c->pc, NA - P0);
      OzOperand Hop = oz_slice(la, c->Hb + (size_t)P0 * N * no, np * no, N, 1, no, 0, N, kOzMaxDigits, 0, c->Gz, no,
                               (long long)N * no);
      OzGemmArgs gb;
      gb.A = Hop; gb.B = Cop; gb.M = np * no; gb.N = no; gb.s = kOzMaxDigits; gb.C = c->Xt + (size_t)P0 * ldx;
      gb.MR = no; gb.cs_m1 = no; gb.cs_m2 = ldx; gb.cs_n = 1;
      oz_gemm(la, gb);
    }
  } else {
    TraceScope t(c->tracer, s, "grad Bij = C~^T H (batched dgemm)", 2.0 * NA * N * no * no, 0);
    GemmArgs gb;
    gb.M = no; gb.N = no; gb.K = N; gb.A = c->Ct; gb.lda = no; gb.transA = true;
    gb.B = c->Hb; gb.ldb = no; gb.sB = (long long)N * no; gb.C = c->Bij; gb.ldc = no; gb.sC = (long long)no * no;
    gb.batch = NA;
    dgemm(la, gb);
    RIHF_CUDA(cudaMemcpy2DAsync(c->Xt, ldx * sizeof(double), c->Bij, (size_t)no * no * sizeof(double),
                                (size_t)no * no * sizeof(double), NA, cudaMemcpyDeviceToDevice, s));
  }
  // [X~ | c] = L^{-T} [Bij | d]  (NA x (nocc^2 + 1)): the paper's X^P_ij = sum_Q A^L_PQ B^Q_ij
  // and L^P in one blocked solve (the solve is latency-bound, one extra column is free)
  { TraceScope t(c->tracer, s, "grad [X | c] = L^-T [Bij | d] (trsm; tcgen05 updates in mixed mode)",
                 (double)NA * NA * ldx, 0);
    RIHF_CUDA(cudaMemcpy2DAsync(c->Xt + (size_t)no * no, ldx * sizeof(double), c->dvec, sizeof(double),
                                sizeof(double), NA, cudaMemcpyDeviceToDevice, s));
    if (c->trsm_sc.X.planes && oz_plane_elems(ldx, kTrsmOuter, kOzMaxDigits) <= c->trsm_sc.X.cap)
      trsm_lower_t_tc(la, c->L, NA, c->Xt, ldx, 0, c->trsm_sc);   // mixed mode: tensor-core updates
    else
      trsm_lower(la, c->L, NA, c->Xt, ldx, true, 0, c->trsm_tmp);
    RIHF_CUDA(cudaMemcpy2DAsync(c->cvec, sizeof(double), c->Xt + (size_t)no * no, ldx * sizeof(double),
                                sizeof(double), NA, cudaMemcpyDeviceToDevice, s)); }
  // Z = c c^T - 1/2 Xt Xt^T (tensor cores: K = nocc^2 in exponent blocks of at
  // most kOzMaxChunksPerBlock chunks, summed atomically into a zeroed Zm)
  if (tc) {
    TraceScope t(c->tracer, s, "grad Z=-1/2 X X^T (tcgen05 7 digits)", 0.0, 0);
    const int kch = (no * no + kOzChunk - 1) / kOzChunk;
    const bool blocks = kch > kOzMaxChunksPerBlock;
    OzOperand Xop = oz_slice(la, c->Xt, NA, no * no, ldx, 1, 0, no * no, kOzMaxDigits,
                             blocks ? kOzMaxChunksPerBlock : 0, c->Xz);
    if (blocks) RIHF_CUDA(cudaMemsetAsync(c->Zm, 0, sizeof(double) * (size_t)NA * NA, s));
    OzGemmArgs gz;
    gz.A = Xop; gz.B = Xop; gz.M = NA; gz.N = NA; gz.s = kOzMaxDigits; gz.alpha = -0.5; gz.C = c->Zm;
    gz.cs_m1 = NA; gz.cs_n = 1; gz.lower_only = true; gz.atomic = blocks;
    oz_gemm(la, gz);
  } else {
    GemmArgs gz;
    gz.M = NA; gz.N = NA; gz.K = no * no; gz.A = c->Xt; gz.lda = (int)ldx; gz.B = c->Xt; gz.ldb = (int)ldx;
    gz.transB = true; gz.C = c->Zm; gz.ldc = NA; gz.alpha = -0.5;
    gz.lower_only = true;   // Z is symmetric
    dgemm(la, gz);
  }
  GemmArgs gc;
  gc.M = NA; gc.N = NA; gc.K = 1; gc.A = c->cvec; gc.lda = 1; gc.B = c->cvec; gc.ldb = NA; gc.C = c->Zm; gc.ldc = NA;
  gc.beta = 1.0;
  dgemm(la, gc);
  symmetrize_lower(la, c->Zm, NA, 1);
  // Y[P] = D c_P - 1/2 Ct Xt[P] Ct^T: G'[P] = Ct Xt[P] for all P, then per chunk of
  // auxiliary functions the N x N slices in Bu (D c_P plus the product), packed into Yp
  c->bu_is_B = false;
  if (tc) {
    // G'[P] = Ct Xt[P] (N x nocc, Xt[P] symmetric), then one GEMM over rows
    // (P, mu): Y[(P, mu)][nu] += -1/2 sum_i G'[(P, mu)][i] Ct[nu][i]
    OzOperand Top = oz_slice(la, c->Ct, N, no, no, 1, 0, no, kOzMaxDigits, 0, c->Ctz);   // rows mu, K = j
    const bool tc_g = (no + kOzChunk - 1) / kOzChunk <= kOzMaxChunksPerBlock &&
                      oz_plane_elems(NA * no, no, kOzMaxDigits) <= c->Hz.cap &&
                      (size_t)((NA * no + kOzTileM - 1) / kOzTileM * kOzTileM) <= c->Hz.ecap;
    if (tc_g) {
      // rows (P, i) of X~ (element (P, i, j) at Xt[P ldx + i nocc + j]), K = j, in the
      // idle RI-K H plane buffer; G'[P][mu][i] through the output's row split
      TraceScope t(c->tracer, s, "grad G' = C~ X (tcgen05 7 digits)", 0.0, 0);
      OzOperand Xr = oz_slice(la, c->Xt, NA * no, no, no, 1, 0, no, kOzMaxDigits, 0, c->Hz, no, ldx);
      OzGemmArgs gg;
      gg.A = Xr; gg.B = Top; gg.M = NA * no; gg.N = N; gg.s = kOzMaxDigits; gg.C = c->G;
      gg.MR = no; gg.cs_m1 = 1; gg.cs_m2 = (long long)N * no; gg.cs_n = no;
      oz_gemm(la, gg);
    } else {
      TraceScope t(c->tracer, s, "grad G' = C~ X (batched dgemm)", 2.0 * NA * N * no * no, 0);
      GemmArgs gg;
      gg.M = N; gg.N = no; gg.K = no; gg.A = c->Ct; gg.lda = no; gg.B = c->Xt; gg.ldb = no;
      gg.sB = ldx; gg.C = c->G; gg.ldc = no; gg.sC = (long long)N * no; gg.batch = NA;
      dgemm(la, gg);
    }
    TraceScope t(c->tracer, s, "grad Y=Dc-1/2 C~XC~^T (tcgen05 7 digits)", 0.0, 0);
    for (int P0 = 0; P0 < NA; P0 += c->pc) {
      const int np = std::min(c->pc, NA - P0);
      outer_fill(la, c->cvec + P0, np, c->D, (long long)n2, c->Bu);
      OzOperand Gop = oz_slice(la, c->G + (size_t)P0 * N * no, np * N, no, no, 1, 0, no, kOzMaxDigits, 0, c->Gz);
      OzGemmArgs gy;
      gy.A = Gop; gy.B = Top; gy.M = np * N; gy.N = N; gy.s = kOzMaxDigits; gy.alpha = -0.5; gy.C = c->Bu;
      gy.cs_m1 = N; gy.cs_n = 1; gy.accumulate = true;
      oz_gemm(la, gy);
      pack_sym_batch(la, c->Bu, np, N, c->Yp + (size_t)P0 * c->npp, c->npp);
    }
  } else {
    // G[P] = Xt[P] Ct^T (nocc x N)
    GemmArgs gg;
    gg.M = no; gg.N = N; gg.K = no; gg.A = c->Xt; gg.lda = no; gg.sA = ldx;
    gg.B = c->Ct; gg.ldb = no; gg.transB = true; gg.C = c->G; gg.ldc = N; gg.sC = (long long)no * N; gg.batch = NA;
    dgemm(la, gg);
    TraceScope t(c->tracer, s, "grad Y=Dc-1/2 C~XC~^T (dgemm)", 2.0 * NA * n2 * no, 0);
    for (int P0 = 0; P0 < NA; P0 += c->pc) {
      const int np = std::min(c->pc, NA - P0);
      outer_fill(la, c->cvec + P0, np, c->D, (long long)n2, c->Bu);
      GemmArgs gy;
      gy.M = N; gy.N = N; gy.K = no; gy.A = c->Ct; gy.lda = no; gy.B = c->G + (size_t)P0 * no * N; gy.ldb = N;
      gy.sB = (long long)no * N; gy.C = c->Bu; gy.ldc = N; gy.sC = (long long)n2; gy.batch = np; gy.alpha = -0.5;
      gy.beta = 1.0;
      dgemm(la, gy);
      pack_sym_batch(la, c->Bu, np, N, c->Yp + (size_t)P0 * c->npp, c->npp);
    }
  }
  // fused derivative-integral contractions
  RIHF_CUDA(cudaMemsetAsync(c->grad_parts, 0, sizeof(double) * 15 * nat, s));
  double* g_one = c->grad_parts;
  double* g_ovl = c->grad_parts + 3 * nat;
  double* g_three = c->grad_parts + 6 * nat;
  double* g_two = c->grad_parts + 9 * nat;
  { TraceScope t(c->tracer, s, "grad_one_electron_kernel", 0.0, 0);
    launch_grad_one_electron(ic, c->prim(), c->max_lp, nat, c->d_Z, c->d_xyz, c->D, c->W, g_one, g_ovl); }
  if (!defer_eri3) {
    TraceScope t(c->tracer, s, "grad_eri3_kernel (fused d(mu nu|P) . Y)", c->flops_grad3, 0);
    launch_grad_eri3(ic, c->prim(), c->aux(), c->d_pairs, c->ptab(), c->groups, kTaskGroups, c->Yp, g_three);
  }
  { TraceScope t(c->tracer, s, "grad_eri2_kernel (fused d(P|Q) . Z)", (double)NA * NA * 8, 1);
    launch_grad_eri2(ic, c->aux(), c->max_la, c->Zm, g_two); }
}

// Per-atom parts back to the host, nuclear repulsion, the sum.
static void gradient_finish(rihf_ctx* c, double* grad) {
  cudaStream_t s = c->stream;
  const int nat = c->natoms;
  c->grad_parts_h.assign(15 * nat, 0.0);
  RIHF_CUDA(cudaMemcpyAsync(c->grad_parts_h.data(), c->grad_parts, sizeof(double) * 12 * nat,
                            cudaMemcpyDeviceToHost, s));
  cudaEventRecord(c->ev[6], s);
  RIHF_CUDA(cudaStreamSynchronize(s));
  c->tracer.flush();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev[5], c->ev[6]);
  c->timings[3] = ms;
  // nuclear repulsion gradient (host, O(natoms^2))
  double* gnn = c->grad_parts_h.data() + 12 * nat;
  for (int a = 0; a < nat; ++a)
    for (int b = 0; b < nat; ++b) {
      if (a == b) continue;
      double r[3], r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        r[d] = c->xyz[3 * a + d] - c->xyz[3 * b + d];
        r2 += r[d] * r[d];
      }
      double f = c->Z[a] * c->Z[b] / (r2 * std::sqrt(r2));
      for (int d = 0; d < 3; ++d) gnn[3 * a + d] -= f * r[d];
    }
  for (int i = 0; i < 3 * nat; ++i) {
    double t = 0.0;
    for (int p = 0; p < 5; ++p) t += c->grad_parts_h[p * 3 * nat + i];
    grad[i] = t;
  }
}

int rihf_gradient(rihf_ctx* c, double* grad) {
  RIHF_API_BEGIN
  if (!c || !grad) return RIHF_ERR_INVALID_ARG;
  if (!c->converged) {
    g_last_error = "rihf_gradient needs a converged rihf_scf on this context";
    return RIHF_ERR_STATE;
  }
  gradient_launch(c, false);
  gradient_finish(c, grad);
  return RIHF_OK;
  RIHF_API_END
}

int rihf_query(rihf_ctx* c, int* N, int* Naux, int* nocc, int* natoms) {
  if (!c) return RIHF_ERR_INVALID_ARG;
  if (N) *N = c->N;
  if (Naux) *Naux = c->NA;
  if (nocc) *nocc = c->nocc;
  if (natoms) *natoms = c->natoms;
  return RIHF_OK;
}

int rihf_get_matrix(rihf_ctx* c, int which, double* out) {
  RIHF_API_BEGIN
  if (!c || !out) return RIHF_ERR_INVALID_ARG;
  const size_t n2 = (size_t)c->N * c->N, na2 = (size_t)c->NA * c->NA;
  RIHF_CUDA(cudaStreamSynchronize(c->stream));
  switch (which) {
    case RIHF_MAT_S: RIHF_CUDA(cudaMemcpy(out, c->S, n2 * 8, cudaMemcpyDeviceToHost)); break;
    case RIHF_MAT_H: RIHF_CUDA(cudaMemcpy(out, c->H, n2 * 8, cudaMemcpyDeviceToHost)); break;
    case RIHF_MAT_J: RIHF_CUDA(cudaMemcpy(out, c->J, n2 * 8, cudaMemcpyDeviceToHost)); break;
    case RIHF_MAT_K: RIHF_CUDA(cudaMemcpy(out, c->K, n2 * 8, cudaMemcpyDeviceToHost)); break;
    case RIHF_MAT_F: RIHF_CUDA(cudaMemcpy(out, c->F, n2 * 8, cudaMemcpyDeviceToHost)); break;
    case RIHF_MAT_D: RIHF_CUDA(cudaMemcpy(out, c->D, n2 * 8, cudaMemcpyDeviceToHost)); break;
    case RIHF_MAT_A: RIHF_CUDA(cudaMemcpy(out, c->A, na2 * 8, cudaMemcpyDeviceToHost)); break;
    case RIHF_MAT_LINV: {
      // L^{-1} is not formed on the hot path; solve L X = I on request
      if (!c->have_linv) {
        LaCtx la = c->la();
        identity(la, c->Linv, c->NA);
        trsm_lower(la, c->L, c->NA, c->Linv, c->NA, false, 0, c->trsm_tmp);
        RIHF_CUDA(cudaStreamSynchronize(c->stream));
        c->have_linv = true;
      }
      RIHF_CUDA(cudaMemcpy(out, c->Linv, na2 * 8, cudaMemcpyDeviceToHost));
      break;
    }
    case RIHF_MAT_B:
    case RIHF_MAT_T3: {
      // B: the packed device tensor; T3: the fit overwrote it, so the
      // integrals are evaluated again into a temporary packed buffer.  Both are
      // expanded to Naux x N x N on the host.
      const int N = c->N, NA = c->NA;
      std::vector<double> pk((size_t)NA * c->npp);
      if (which == RIHF_MAT_B) {
        RIHF_CUDA(cudaMemcpy(pk.data(), c->Bp, sizeof(double) * pk.size(), cudaMemcpyDeviceToHost));
      } else {
        double* tmp = dalloc<double>(pk.size());
        try {
          RIHF_CUDA(cudaMemsetAsync(tmp, 0, sizeof(double) * pk.size(), c->stream));
          launch_eri3(c->ic(), c->prim(), c->aux(), c->d_pairs, c->ptab(), c->groups, kTaskGroups, tmp);
          RIHF_CUDA(cudaMemcpyAsync(pk.data(), tmp, sizeof(double) * pk.size(), cudaMemcpyDeviceToHost, c->stream));
          RIHF_CUDA(cudaStreamSynchronize(c->stream));
        } catch (...) {
          cudaFree(tmp);
          throw;
        }
        cudaFree(tmp);
      }
      for (int P = 0; P < NA; ++P)
        for (int mu = 0; mu < N; ++mu)
          for (int nu = 0; nu < N; ++nu)
            out[(size_t)P * n2 + (size_t)mu * N + nu] = pk[(size_t)P * c->npp + tri_index(mu, nu)];
      break;
    }
    case RIHF_MAT_FEATURES: {
      const size_t nf = (size_t)c->N * (c->N + 1) / 2 * kMlpF;
      std::vector<float> f(nf);
      RIHF_CUDA(cudaMemcpy(f.data(), c->mlX, sizeof(float) * nf, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < nf; ++i) out[i] = f[i];
      break;
    }
    case RIHF_MAT_DSAD: {
      // the SAD guess density D_SAD = Fs Fs^T (after a guess-5 SCF built it)
      if (!c->sad_ok) return RIHF_ERR_STATE;
      const int N = c->N, m = c->sad_m;
      std::vector<double> F((size_t)N * m);
      RIHF_CUDA(cudaMemcpy(F.data(), c->d_sad, sizeof(double) * F.size(), cudaMemcpyDeviceToHost));
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
          double t = 0.0;
          for (int q = 0; q < m; ++q) t += F[(size_t)i * m + q] * F[(size_t)j * m + q];
          out[(size_t)i * N + j] = t;
        }
      break;
    }
    case RIHF_MAT_DPRED:
      RIHF_CUDA(cudaMemcpy(out, c->Dpred, n2 * 8, cudaMemcpyDeviceToHost));
      break;
    case RIHF_MAT_SCHWARZ:
      if (c->schwarz_ok) {
        if (!c->schwarz_fresh) {   // tau <= 0: not needed for the screening, computed on request
          launch_schwarz(c->ic(), c->prim(), c->max_lp, c->d_schwarz);
          RIHF_CUDA(cudaStreamSynchronize(c->stream));
          c->schwarz_fresh = true;
        }
        RIHF_CUDA(cudaMemcpy(out, c->d_schwarz, sizeof(double) * c->npairs_total, cudaMemcpyDeviceToHost));
      } else {
        std::memset(out, 0, sizeof(double) * c->npairs_total);
      }
      break;
    case RIHF_MAT_GRAD_PARTS:
      if (c->grad_parts_h.empty()) return RIHF_ERR_STATE;
      std::memcpy(out, c->grad_parts_h.data(), sizeof(double) * 15 * c->natoms);
      break;
    default: return RIHF_ERR_INVALID_ARG;
  }
  return RIHF_OK;
  RIHF_API_END
}

// Seeded initial weights: W1 ~ U(-1/sqrt(F), 1/sqrt(F)), w2 ~ U(-0.1/sqrt(H), 0.1/sqrt(H)), biases 0
// (splitmix64 stream, so the same seed gives the same network on any host).
static std::vector<float> mlp_init_params(int H, unsigned long long seed) {
  std::vector<float> p(mlp_nparams(H), 0.f);
  unsigned long long x = seed;
  auto next = [&]() {
    unsigned long long z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
  };
  const double a1 = 1.0 / std::sqrt((double)kMlpF), a2 = 0.1 / std::sqrt((double)H);
  for (int i = 0; i < H * kMlpF; ++i) p[i] = (float)((2.0 * next() - 1.0) * a1);
  for (int j = 0; j < H; ++j) p[H * kMlpF + H + j] = (float)((2.0 * next() - 1.0) * a2);
  return p;
}

static void mlp_alloc(MlpDev& net, int H) {
  const int np = mlp_nparams(H);
  net.H = H;
  net.master = dalloc<float>(np);
  net.wbf = dalloc<uint16_t>(np);
  net.grad = dalloc<float>(np);
  net.m = dalloc<float>(np);
  net.v = dalloc<float>(np);
  net.loss = dalloc<float>(2);
  net.adam_t = 0;
}

int rihf_learn_config(rihf_ctx* c, int hidden, int train_steps, int adam_iters, double lr, unsigned long long seed) {
  RIHF_API_BEGIN
  if (!c || hidden < 32 || hidden > kMlpMaxH || hidden % 32 || train_steps < 0 || adam_iters < 1 || !(lr > 0.0))
    return RIHF_ERR_INVALID_ARG;
  cudaStream_t s = c->stream;
  if (c->net.master) {
    void* ptrs[] = {c->net.master, c->net.wbf, c->net.grad, c->net.m, c->net.v, c->net.loss};
    RIHF_CUDA(cudaStreamSynchronize(s));
    for (void* p : ptrs) cudaFree(p);
    c->net = MlpDev();
  }
  mlp_alloc(c->net, hidden);
  const int np = mlp_nparams(hidden);
  std::vector<float> p = mlp_init_params(hidden, seed);
  RIHF_CUDA(cudaMemcpyAsync(c->net.master, p.data(), sizeof(float) * np, cudaMemcpyHostToDevice, s));
  RIHF_CUDA(cudaMemsetAsync(c->net.m, 0, sizeof(float) * np, s));
  RIHF_CUDA(cudaMemsetAsync(c->net.v, 0, sizeof(float) * np, s));
  mlp_round_weights(s, c->net);
  RIHF_CUDA(cudaStreamSynchronize(s));
  c->net_on = true;
  if (!c->hist_lowdin) {   // the history restarts in the Loewdin representation
    c->hist_lowdin = true;
    c->nhist = 0;
  }
  c->train_steps = train_steps;
  c->adam_iters = adam_iters;
  c->ml_lr = lr;
  c->trained_steps = 0;
  c->ml_scale = 0.0;
  c->ml_sd = c->ml_ss = c->ml_sr = 0.0;
  c->nrep = c->rep_head = 0;
  c->ml_last_ratio = 1e300;
  c->ml_ratios[0] = c->ml_ratios[1] = c->ml_ratios[2] = 1e300;
  return RIHF_OK;
  RIHF_API_END
}

int rihf_learn_stats(rihf_ctx* c, int* trained_steps, double* last_ratio, int* last_guess, double* scale) {
  if (!c) return RIHF_ERR_INVALID_ARG;
  if (trained_steps) *trained_steps = c->trained_steps;
  if (last_ratio) *last_ratio = c->ml_last_ratio;
  if (last_guess) *last_guess = c->last_guess;
  if (scale) *scale = c->ml_scale;
  return RIHF_OK;
}

int rihf_batch_step(int nmol, rihf_ctx* const* ctx, const double* const* xyz, int guess, double* energies,
                    double* grads, int* iters, int nthreads) {
  if (nmol < 0 || (nmol > 0 && !ctx)) return RIHF_ERR_INVALID_ARG;
  for (int i = 0; i < nmol; ++i)
    if (!ctx[i]) return RIHF_ERR_INVALID_ARG;
  for (int i = 0; i < nmol; ++i)
    for (int j = 0; j < i; ++j)
      if (ctx[i] == ctx[j]) return RIHF_ERR_INVALID_ARG;
  std::vector<size_t> goff(nmol + 1, 0);
  for (int i = 0; i < nmol; ++i) goff[i + 1] = goff[i] + 3 * (size_t)ctx[i]->natoms;
  std::vector<int> rc(nmol, RIHF_OK);
  std::vector<std::string> err(nmol);
  // The 3-centre integrals and the 3-centre derivative contraction, the
  // largest per-geometry launches, run as one launch per class group over all
  // molecules (launch_eri3_batch / launch_grad_eri3_batch: ragged task lists
  // behind an int64 offsets table) when every context lives on one device;
  // everything else runs per context on its own stream, host threads driving
  // the contexts between the batched launches.
  bool batched = nmol > 1;
  for (int i = 1; i < nmol && batched; ++i) batched = ctx[i]->opt.device == ctx[0]->opt.device;
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nw = std::max(1, std::min(nmol, nthreads > 0 ? nthreads : hw));
  auto parallel = [&](const std::function<void(int)>& f) {
    auto work = [&](int w) {
      for (int i = w; i < nmol; i += nw) {
        if (rc[i] != RIHF_OK) continue;
        if (cudaSetDevice(ctx[i]->opt.device) != cudaSuccess) {
          rc[i] = RIHF_ERR_CUDA;
          err[i] = "cudaSetDevice failed";
          continue;
        }
        try {
          f(i);
        } catch (const RihfError& e) {
          rc[i] = e.code;
          err[i] = e.what();
        } catch (const CudaError& e) {
          rc[i] = RIHF_ERR_CUDA;
          err[i] = e.what();
        } catch (const std::exception& e) {
          rc[i] = RIHF_ERR_INVALID_ARG;
          err[i] = e.what();
        }
      }
    };
    if (nw <= 1) {
      work(0);
    } else {
      std::vector<std::thread> pool;
      for (int w = 0; w < nw; ++w) pool.emplace_back(work, w);
      for (auto& t : pool) t.join();
    }
  };
  // batched launch over the contexts still in good standing, on a stream of
  // its own that waits for every context's stream and that every context's
  // stream then waits for
  cudaStream_t bs = nullptr;
  BatchTables tab;
  int* bcount = nullptr;
  std::vector<cudaEvent_t> evs;
  auto release = [&]() {
    if (tab.geoms) cudaFree(tab.geoms);
    if (tab.off) cudaFree(tab.off);
    if (bcount) cudaFree(bcount);
    for (auto e : evs) cudaEventDestroy(e);
    if (bs) cudaStreamDestroy(bs);
  };
  auto batched_launch = [&](bool grad) -> bool {
    std::vector<BatchGeom> batch;
    std::vector<int> members;
    for (int i = 0; i < nmol; ++i) {
      if (rc[i] != RIHF_OK) continue;
      rihf_ctx* c = ctx[i];
      BatchGeom b;
      b.g.prim = c->prim();
      b.g.aux = c->aux();
      b.g.pairs = c->d_pairs;
      b.g.ptab = c->ptab();
      b.g.out = grad ? c->grad_parts + 6 * c->natoms : c->Bp;
      b.g.Y = grad ? c->Yp : nullptr;
      b.groups = c->groups;
      batch.push_back(b);
      members.push_back(i);
    }
    if (batch.empty()) return true;
    try {
      for (int i : members) {
        RIHF_CUDA(cudaEventRecord(evs[i], ctx[i]->stream));
        RIHF_CUDA(cudaStreamWaitEvent(bs, evs[i], 0));
      }
      IntegralCtx ic = ctx[members[0]]->ic();
      ic.stream = bs;
      ic.counter = bcount;
      ic.launches = nullptr;
      if (grad) launch_grad_eri3_batch(ic, batch, kTaskGroups, tab);
      else launch_eri3_batch(ic, batch, kTaskGroups, tab);
      RIHF_CUDA(cudaEventRecord(evs[nmol], bs));
      for (int i : members) {
        RIHF_CUDA(cudaStreamWaitEvent(ctx[i]->stream, evs[nmol], 0));
        ctx[i]->launches += kTaskGroups;
      }
    } catch (const RihfError& e) {
      g_last_error = std::string("batched launch: ") + e.what();
      return false;
    } catch (const CudaError& e) {
      g_last_error = std::string("batched launch: ") + e.what();
      return false;
    }
    return true;
  };
  if (batched) {
    if (cudaSetDevice(ctx[0]->opt.device) != cudaSuccess) return RIHF_ERR_CUDA;
    bool ok = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess;
    tab.cap = nmol;
    ok = ok && cudaMalloc(&tab.geoms, sizeof(GeomTasks) * (size_t)kTaskGroups * nmol) == cudaSuccess;
    ok = ok && cudaMalloc(&tab.off, sizeof(long long) * (size_t)kTaskGroups * (nmol + 1)) == cudaSuccess;
    ok = ok && cudaMalloc(&bcount, sizeof(int)) == cudaSuccess;
    evs.resize(nmol + 1);
    for (auto& e : evs) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      release();
      g_last_error = "rihf_batch_step: could not create the batch stream and tables";
      return RIHF_ERR_OOM;
    }
  }
  std::vector<double> etmp(nmol, 0.0);
  std::vector<int> itmp(nmol, 0);
  // 1. geometry: one-electron, metric, Cholesky, pair tables (3-centre
  //    integrals deferred to the batched launch)
  parallel([&](int i) {
    rihf_ctx* c = ctx[i];
    if (xyz && xyz[i]) c->xyz.assign(xyz[i], xyz[i] + 3 * c->natoms);
    c->converged = false;
    compute_geometry(c, batched);
  });
  if (batched && !batched_launch(false)) {
    release();
    return RIHF_ERR_CUDA;
  }
  // 2. fit, SCF, gradient up to the 3-centre derivative contraction
  parallel([&](int i) {
    rihf_ctx* c = ctx[i];
    if (batched) compute_geometry_rest(c);
    int it = 0;
    double e = 0.0;
    const int r = rihf_scf(c, guess, nullptr, &e, nullptr, nullptr, nullptr, &it);
    etmp[i] = e;
    itmp[i] = it;
    if (r != RIHF_OK) throw RihfError(r, rihf_last_error());
    gradient_launch(c, batched);
  });
  if (batched && !batched_launch(true)) {
    release();
    return RIHF_ERR_CUDA;
  }
  // 3. the per-atom parts back and summed
  parallel([&](int i) {
    std::vector<double> gl;
    double* gp = grads ? grads + goff[i] : (gl.resize(3 * (size_t)ctx[i]->natoms), gl.data());
    gradient_finish(ctx[i], gp);
  });
  release();
  for (int i = 0; i < nmol; ++i) {
    if (energies) energies[i] = etmp[i];
    if (iters) iters[i] = itmp[i];
  }
  for (int i = 0; i < nmol; ++i)
    if (rc[i] != RIHF_OK) {
      g_last_error = "molecule " + std::to_string(i) + ": " + err[i];
      return rc[i];
    }
  return RIHF_OK;
}

int rihf_learn_params(rihf_ctx* c, float* out) {
  RIHF_API_BEGIN
  if (!c || !out || !c->net_on) return RIHF_ERR_INVALID_ARG;
  RIHF_CUDA(cudaStreamSynchronize(c->stream));
  RIHF_CUDA(cudaMemcpy(out, c->net.master, sizeof(float) * mlp_nparams(c->net.H), cudaMemcpyDeviceToHost));
  return RIHF_OK;
  RIHF_API_END
}

int rihf_mlp_eval(int hidden, int M, const float* params, const float* X, const float* t, float lr, int iters,
                  float* y, float* grad, float* params_out, float* loss2, float* losses, int device) {
  RIHF_API_BEGIN
  if (hidden < 32 || hidden > kMlpMaxH || hidden % 32 || M < 0 || !params || (M > 0 && !X) ||
      (t == nullptr && (grad || loss2 || params_out || losses)) || (params_out && (!(lr > 0.f) || iters < 1)) ||
      (losses && !params_out))
    return RIHF_ERR_INVALID_ARG;
  RIHF_CUDA(cudaSetDevice(device));
  cudaStream_t s;
  RIHF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  MlpDev net;
  float *dX = nullptr, *dt = nullptr, *dy = nullptr;
  auto release = [&]() {
    void* ptrs[] = {net.master, net.wbf, net.grad, net.m, net.v, net.loss, dX, dt, dy};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    cudaStreamDestroy(s);
  };
  try {
    const int np = mlp_nparams(hidden);
    mlp_alloc(net, hidden);
    const size_t Mx = std::max(M, 1);
    dX = dalloc<float>(Mx * kMlpF);
    dt = dalloc<float>(Mx);
    dy = dalloc<float>(Mx);
    RIHF_CUDA(cudaMemcpyAsync(net.master, params, sizeof(float) * np, cudaMemcpyHostToDevice, s));
    if (M > 0) RIHF_CUDA(cudaMemcpyAsync(dX, X, sizeof(float) * M * kMlpF, cudaMemcpyHostToDevice, s));
    if (t && M > 0) RIHF_CUDA(cudaMemcpyAsync(dt, t, sizeof(float) * M, cudaMemcpyHostToDevice, s));
    RIHF_CUDA(cudaMemsetAsync(net.m, 0, sizeof(float) * np, s));
    RIHF_CUDA(cudaMemsetAsync(net.v, 0, sizeof(float) * np, s));
    mlp_round_weights(s, net);
    if (y) {
      mlp_forward(s, net, dX, M, dy);
      if (M > 0) RIHF_CUDA(cudaMemcpyAsync(y, dy, sizeof(float) * M, cudaMemcpyDeviceToHost, s));
    }
    if (t) {
      mlp_backward(s, net, dX, dt, M);
      if (grad) RIHF_CUDA(cudaMemcpyAsync(grad, net.grad, sizeof(float) * np, cudaMemcpyDeviceToHost, s));
      if (loss2) RIHF_CUDA(cudaMemcpyAsync(loss2, net.loss, 2 * sizeof(float), cudaMemcpyDeviceToHost, s));
      if (params_out) {
        for (int k = 0; k < iters; ++k) {
          if (k > 0) mlp_backward(s, net, dX, dt, M);
          if (losses) RIHF_CUDA(cudaMemcpyAsync(losses + k, net.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
          mlp_adam(s, net, lr);
        }
        RIHF_CUDA(cudaMemcpyAsync(params_out, net.master, sizeof(float) * np, cudaMemcpyDeviceToHost, s));
      }
    }
    RIHF_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    release();
    throw;
  }
  release();
  return RIHF_OK;
  RIHF_API_END
}

int rihf_screening_stats(rihf_ctx* c, int* kept, int* total) {
  if (!c) return RIHF_ERR_INVALID_ARG;
  if (kept) *kept = c->npairs;
  if (total) *total = c->npairs_total;
  return RIHF_OK;
}

int rihf_timings(rihf_ctx* c, double* out5) {
  if (!c || !out5) return RIHF_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i) out5[i] = c->timings[i];
  out5[4] = (double)c->launches;
  return RIHF_OK;
}

void* rihf_stream(rihf_ctx* c) { return c ? (void*)c->stream : nullptr; }

int rihf_scf_stats(rihf_ctx* c, int* tc_builds, int* fp64_builds, int* confirm_builds) {
  if (!c) return RIHF_ERR_INVALID_ARG;
  if (tc_builds) *tc_builds = c->tc_builds;
  if (fp64_builds) *fp64_builds = c->last_iters - c->tc_builds - c->confirm_builds;
  if (confirm_builds) *confirm_builds = c->confirm_builds;
  return RIHF_OK;
}

int rihf_trace(rihf_ctx* c, int enable) {
  if (!c) return RIHF_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  c->tracer.flush();
  if (enable) c->tracer.stats.clear();
  c->tracer.on = enable != 0;
  return RIHF_OK;
}

int rihf_trace_stats(rihf_ctx* c, int max, char* names, double* launches, double* ms, double* work, int* kind) {
  if (!c || max < 0) return RIHF_ERR_INVALID_ARG;
  cudaStreamSynchronize(c->stream);
  c->tracer.flush();
  int n = 0;
  for (auto& kv : c->tracer.stats) {
    if (n >= max) break;
    if (names) {
      std::strncpy(names + 48 * n, kv.first.c_str(), 47);
      names[48 * n + 47] = 0;
    }
    if (launches) launches[n] = (double)kv.second.launches;
    if (ms) ms[n] = kv.second.ms;
    if (work) work[n] = kv.second.work;
    if (kind) kind[n] = kv.second.kind;
    ++n;
  }
  return (int)std::min<size_t>(c->tracer.stats.size(), (size_t)std::max(max, 0)) >= 0 ? n : n;
}

int rihf_eigh(int n, const double* A, double* W, double* V, int device) {
  RIHF_API_BEGIN
  if (n <= 0 || n > 4096 || !A || !W || !V) return RIHF_ERR_INVALID_ARG;
  RIHF_CUDA(cudaSetDevice(device));
  cudaStream_t s;
  RIHF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  size_t n2 = (size_t)n * n;
  double *dA = nullptr, *dW = nullptr, *dV = nullptr, *ws = nullptr, *work = nullptr;
  int* flag = nullptr;
  size_t work_elems = std::max<size_t>((size_t)1 << 22, 8 * n2);
  try {
    dA = dalloc<double>(n2); dW = dalloc<double>(n); dV = dalloc<double>(n2);
    ws = dalloc<double>(eig_workspace(n)); work = dalloc<double>(work_elems); flag = dalloc<int>(1);
    RIHF_CUDA(cudaMemcpyAsync(dA, A, n2 * 8, cudaMemcpyHostToDevice, s));
    LaCtx la;
    la.stream = s; la.work = work; la.work_elems = work_elems; la.sms = sms; la.flag = flag;
    // above order 1024 the block Jacobi's FP32 start carries the rounding of
    // more rounds: two more refinement steps
    eigh(la, dA, n, dW, dV, ws, n > 1024 ? 6 : 4, nullptr);
    RIHF_CUDA(cudaMemcpyAsync(W, dW, n * 8, cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaMemcpyAsync(V, dV, n2 * 8, cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    cudaFree(dA); cudaFree(dW); cudaFree(dV); cudaFree(ws); cudaFree(work); cudaFree(flag);
    cudaStreamDestroy(s);
    throw;
  }
  cudaFree(dA); cudaFree(dW); cudaFree(dV); cudaFree(ws); cudaFree(work); cudaFree(flag);
  cudaStreamDestroy(s);
  return RIHF_OK;
  RIHF_API_END
}

int rihf_tc_dgemm(int M, int N, int K, const double* A, const double* B, double* C, int digits, int kblock,
                  int device) {
  RIHF_API_BEGIN
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || digits < 1 || digits > kOzMaxDigits || kblock < 0)
    return RIHF_ERR_INVALID_ARG;
  RIHF_CUDA(cudaSetDevice(device));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t s;
  RIHF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  std::vector<void*> bufs;
  auto alloc = [&](size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) throw RihfError(RIHF_ERR_OOM, "cudaMalloc failed");
    bufs.push_back(p);
    return p;
  };
  auto release = [&]() {
    for (void* p : bufs) cudaFree(p);
    cudaStreamDestroy(s);
  };
  try {
    const int kchunks = (K + kOzChunk - 1) / kOzChunk;
    const int kbc = kblock > 0 ? std::min(kblock, kchunks) : kchunks;
    const int nkb = (kchunks + kbc - 1) / kbc;
    double* dA = (double*)alloc(sizeof(double) * M * K);
    double* dB = (double*)alloc(sizeof(double) * N * K);
    double* dC = (double*)alloc(sizeof(double) * M * N);
    int* flag = (int*)alloc(4 * sizeof(int));
    OzBuf za, zb;
    za.cap = oz_plane_elems(M, K, digits);
    za.ecap = (size_t)(M + kOzTileM - 1) / kOzTileM * kOzTileM * nkb;
    zb.cap = oz_plane_elems(N, K, digits);
    zb.ecap = (size_t)(N + kOzTileM - 1) / kOzTileM * kOzTileM * nkb;
    za.planes = (uint16_t*)alloc(sizeof(uint16_t) * za.cap);
    zb.planes = (uint16_t*)alloc(sizeof(uint16_t) * zb.cap);
    za.exps = (int*)alloc(sizeof(int) * za.ecap);
    zb.exps = (int*)alloc(sizeof(int) * zb.ecap);
    RIHF_CUDA(cudaMemcpyAsync(dA, A, sizeof(double) * M * K, cudaMemcpyHostToDevice, s));
    RIHF_CUDA(cudaMemcpyAsync(dB, B, sizeof(double) * N * K, cudaMemcpyHostToDevice, s));
    RIHF_CUDA(cudaMemsetAsync(dC, 0, sizeof(double) * M * N, s));
    RIHF_CUDA(cudaMemsetAsync(flag, 0, 4 * sizeof(int), s));
    LaCtx la;
    la.stream = s; la.flag = flag; la.sched = flag + 2;
    la.sms = sms;
    OzGemmArgs g;
    g.A = oz_slice(la, dA, M, K, K, 1, 0, K, digits, kbc, za);
    g.B = oz_slice(la, dB, N, K, K, 1, 0, K, digits, kbc, zb);
    g.M = M; g.N = N; g.s = digits; g.C = dC; g.cs_m1 = N; g.cs_n = 1; g.atomic = nkb > 1;
    oz_gemm(la, g);
    int hflag[4];
    RIHF_CUDA(cudaMemcpyAsync(C, dC, sizeof(double) * M * N, cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaMemcpyAsync(hflag, flag, sizeof(hflag), cudaMemcpyDeviceToHost, s));
    RIHF_CUDA(cudaStreamSynchronize(s));
    if (hflag[1]) throw RihfError(RIHF_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait ran out");
  } catch (...) {
    release();
    throw;
  }
  release();
  return RIHF_OK;
  RIHF_API_END
}

void rihf_destroy(rihf_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& g : c->diag_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  free_all(c);
  for (auto& e : c->ev) cudaEventDestroy(e);
  cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
