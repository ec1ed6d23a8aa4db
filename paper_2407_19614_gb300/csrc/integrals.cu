// Integral kernels of librihf: (mu nu|P), (P|Q), S, T, V and, in grad_integrals.cu,
// their derivative contractions.  One warp (one 32-thread block) per task; tasks
// are handed out through a device counter so that heavy and light shell classes
// balance across the 152 SMs.
#include <algorithm>
#include <array>
#include <map>
#include <cmath>
#include <vector>

#include "../../include/rihf.h"
#include "integrals.cuh"
#include "os_hgp.cuh"

namespace rihf {

// ------------------------------------------------------------ Boys table

// F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt by 128-point Gauss-Legendre quadrature
// in long double (nodes from Newton iteration on P_128).
void boys_table_host(double* out) {
  const int n = 128;
  std::vector<long double> x(n), w(n);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    long double z = cosl(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = z;
      for (int k = 2; k <= n; ++k) {
        long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      long double dp = n * (z * p1 - p0) / (z * z - 1.0L);
      long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-21L) {
        // recompute derivative at the converged node for the weight
        p0 = 1.0L;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
          long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0L);
        x[i] = z;
        w[i] = 2.0L / ((1.0L - z * z) * dp * dp);
        break;
      }
    }
  }
  for (int k = 0; k < kBoysN; ++k) {
    long double T = k * (long double)kBoysStep;
    for (int m = 0; m < kBoysM; ++m) {
      // map [-1,1] -> [0,1]: t = (x+1)/2, dt = dx/2
      long double s = 0.0L;
      for (int i = 0; i < n; ++i) {
        long double t = 0.5L * (x[i] + 1.0L);
        s += w[i] * powl(t, 2 * m) * expl(-T * t * t);
      }
      out[(size_t)k * kBoysM + m] = (double)(0.5L * s);
    }
  }
}

// ------------------------------------------------------------ helpers

template <int W = 32>
__device__ inline int warp_next_task(int* counter, int lane) {
  int t = 0;
  if (lane == 0) t = atomicAdd(counter, 1);
  return __shfl_sync(lane_group_mask<W>(), t, (threadIdx.x & 31) / W * W);
}

// out[sa][sb][sc] = sum tra[sa][ka] trb[sb][kb] trc[sc][kc] cart[ka][kb][kc]
// (three passes through shared memory).  Returns the result pointer.
template <int W = 32>
__device__ inline const double* warp_transform3(const double* cart, int la, int lb, int lc, const double* tra,
                                                const double* trb, const double* trc, int nfa, int nfb, int nfc,
                                                double* s1, double* s2, int lane) {
  const int na = ncart(la), nb = ncart(lb), nc = ncart(lc);
  // pass c: s1[ka][kb][sc]
  for (int idx = lane; idx < na * nb * nfc; idx += W) {
    int sc = idx % nfc, r = idx / nfc;
    const double* row = cart + r * nc;
    const double* t = trc + sc * kTrStride;
    double v = 0.0;
    for (int k = 0; k < nc; ++k) v += t[k] * row[k];
    s1[idx] = v;
  }
  __syncwarp(lane_group_mask<W>());
  // pass b: s2[ka][sb][sc]
  for (int idx = lane; idx < na * nfb * nfc; idx += W) {
    int sc = idx % nfc, r = idx / nfc;
    int sb = r % nfb, ka = r / nfb;
    const double* t = trb + sb * kTrStride;
    double v = 0.0;
    for (int k = 0; k < nb; ++k) v += t[k] * s1[(ka * nb + k) * nfc + sc];
    s2[idx] = v;
  }
  __syncwarp(lane_group_mask<W>());
  // pass a: s1[sa][sb][sc]
  for (int idx = lane; idx < nfa * nfb * nfc; idx += W) {
    int rest = idx % (nfb * nfc), sa = idx / (nfb * nfc);
    const double* t = tra + sa * kTrStride;
    double v = 0.0;
    for (int k = 0; k < na; ++k) v += t[k] * s2[k * nfb * nfc + rest];
    s1[idx] = v;
  }
  __syncwarp(lane_group_mask<W>());
  return s1;
}

// Shared-memory plan for one (la, lb | lc) class, in doubles.
// With `mirror` the transfer region also holds the mirrored recursion's levels
// (tasks whose triples may need it, see mirror_prim3).  With `alias` (the
// 3-centre task) the HRR and transform scratch lie over the F_m block and the
// VRR table, both dead once the primitive loop ends; the transfer levels and
// the accumulator, which the HRR reads, stay apart.
struct Eri3Plan {
  int fm, vrr, etr, acc, hrr, half, t1, t2, total;
  __device__ __host__ Eri3Plan(int la, int lb, int lc, int emin, int emax, int nacc, bool mirror = false,
                               bool alias = false) {
    int L = emax + lc;
    EtrShape sh{lc, emin, emax};
    int etr_n = lc > 0 ? sh.total() : 0;
    if (mirror) {
      const int m = EtrShape{emax, lc, lc}.total();
      if (m > etr_n) etr_n = m;
    }
    int accsz = acc_size(emin, emax, lc);
    half = hrr_scratch(la, lb, lc, emax) / 2;
    int big = ncart(la + 1) * ncart(lb + 1) * ncart(lc);
    if (big > half) half = big;
    fm = 0;
    vrr = fm + kFmRegion;
    if (alias) {
      hrr = 0;
      t1 = hrr + 2 * half;
      t2 = t1 + big;
      const int lo = vrr + vrr_size(L), hi = t2 + big + 8;   // 8 doubles of slack after the scratch
      etr = lo > hi ? lo : hi;
      acc = etr + etr_n;
      total = acc + nacc * accsz;
    } else {
      etr = vrr + vrr_size(L);
      acc = etr + etr_n;
      hrr = acc + nacc * accsz;
      t1 = hrr + 2 * half;
      t2 = t1 + big;
      total = t2 + big;
    }
  }
};

int smem_eri3_doubles(int la, int lb, int lc, bool mirror, bool alias) {
  Eri3Plan p(la, lb, lc, la, la + lb, 1, mirror, alias);
  return p.total;
}

// ------------------------------------------------------------ (mu nu|P)

// One task of the 3-centre integrals: the shell triple (pairs[tk.x] | tk.y)
// (tk.y < 0: ~tk.y, with the mirrored recursion for triples with p > q),
// written pair-packed into T.  smem: this task group's slice.
template <int W>
__device__ inline void eri3_task(const DevShells& prim, const DevShells& aux, const ShellPair* __restrict__ pairs,
                                 const PairTable& ptab, int2 tk, const double* __restrict__ boys,
                                 double* __restrict__ T, double* smem, int lane) {
  const int N = prim.nfunc;
  const size_t Npp = (size_t)N * (N + 1) / 2;
  // a negative auxiliary index marks a task whose triples with p > q take the
  // mirrored recursion (see mirror_prim3)
  const bool mir = tk.y < 0;
  int ip = tk.x, sc = mir ? ~tk.y : tk.y;
  int sa = pairs[ip].a, sb = pairs[ip].b;
  // compute with la >= lb (cheaper HRR); the stored block keeps mu in pairs[ip].a
  const bool swp = prim.l[sa] < prim.l[sb];
  if (swp) { int t = sa; sa = sb; sb = t; }
  int la = prim.l[sa], lb = prim.l[sb], lc = aux.l[sc];
  int emin = la, emax = la + lb, L = emax + lc;
  Eri3Plan pl(la, lb, lc, emin, emax, 1, mir, true);
  double* Fm = smem + pl.fm;
  double* vrr = smem + pl.vrr;
  double* etr = smem + pl.etr;
  double* acc = smem + pl.acc;
  const int nab = prim.nprim[sa] * prim.nprim[sb];
  // one primitive triple and a ket above s: the last electron-transfer level
  // ([e][ke][kc], e in [emin, emax]) is the accumulator itself, read in place
  const PairPrim* pr = ptab.pp + ptab.off[ip];
  // one primitive triple: a mirrored one writes its final values into acc
  // (no zeroing, no sums); a forward one with a ket above s leaves them in
  // place as the last transfer level
  const bool one = nab == 1 && aux.nprim[sc] == 1;
  const bool one_mir = one && mir && pr[0].p > aux.exps[aux.pstart[sc]];
  const bool single = one && !one_mir && lc > 0;
  int accsz = acc_size(emin, emax, lc);
  if (!single && !one_mir)
    for (int i = lane; i < accsz; i += W) acc[i] = 0.0;
  const double* A = prim.xyz + 3 * sa;
  const double* B = prim.xyz + 3 * sb;
  const double* C = aux.xyz + 3 * sc;
  const double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
  EtrShape sh{lc, emin, emax};
  const EtrShape shm{emax, lc, lc};
  for (int ab = 0; ab < nab; ++ab) {
    const PairPrim q = pr[ab];
    for (int pc = 0; pc < aux.nprim[sc]; ++pc) {
      const int ic = aux.pstart[sc] + pc;
      Prim3 t = make_prim3_pp(q, aux.exps[ic], aux.iexps[ic], aux.coefs[ic], C, AB);
      for (int m = lane; m <= L; m += W) Fm[m] = boys_eval(m, t.T, boys);
      __syncwarp(lane_group_mask<W>());
      if (mir && t.p > t.q) {
        const Prim3 tm = mirror_prim3(t);
        warp_vrr<W>(vrr, L, tm, Fm, lane);
        warp_etr<W>(vrr, L, etr, shm, tm, Fm, lane);
        if (one_mir) warp_acc_mirror<W, true>(vrr, L, etr, shm, emin, emax, lc, 1.0, acc, lane);
        else warp_acc_mirror<W>(vrr, L, etr, shm, emin, emax, lc, 1.0, acc, lane);
        continue;
      }
      warp_vrr<W>(vrr, L, t, Fm, lane);
      if (single) warp_etr<W>(vrr, L, etr, sh, t, Fm, lane);
      else warp_etr_accumulate<W>(vrr, L, etr, sh, t, 1.0, acc, Fm, lane);
    }
  }
  const double* cart = warp_hrr<W>(single ? etr + sh.level_off(lc) : acc, emin, la, lb, lc, AB, smem + pl.hrr,
                                   pl.half, lane);
  int nfa = prim.nf[la], nfb = prim.nf[lb], nfc = aux.nf[lc];
  const double* out = warp_transform3<W>(cart, la, lb, lc, prim.tr + la * kTrStride * kTrStride,
                                      prim.tr + lb * kTrStride * kTrStride, aux.tr + lc * kTrStride * kTrStride,
                                      nfa, nfb, nfc, smem + pl.t1, smem + pl.t2, lane);
  // pair-packed store: row = the function of pairs[ip].a (the larger shell
  // index, so the larger function index), column = that of pairs[ip].b;
  // inside a diagonal shell block only row >= column
  const int mu0 = prim.ao[sa], nu0 = prim.ao[sb], P0 = aux.ao[sc];
  const bool diag = pairs[ip].a == pairs[ip].b;
  const int n = nfa * nfb * nfc;
  for (int idx = lane; idx < n; idx += W) {
    int sbb = idx % nfb, r = idx / nfb;
    int saa = r % nfa, scc = r / nfa;
    const long long row = swp ? nu0 + sbb : mu0 + saa, col = swp ? mu0 + saa : nu0 + sbb;
    if (diag && row < col) continue;
    T[(size_t)(P0 + scc) * Npp + row * (row + 1) / 2 + col] = out[(saa * nfb + sbb) * nfc + scc];
  }
  __syncwarp(lane_group_mask<W>());
}

template <int W>
__global__ void __launch_bounds__(32, kEri3BlocksPerSM) eri3_kernel(DevShells prim, DevShells aux, const ShellPair* __restrict__ pairs,
                                                  PairTable ptab, const int2* __restrict__ tasks, long long ntask,
                                                  const double* __restrict__ boys, int* counter,
                                                  double* __restrict__ T, int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % W;
  double* smem = smem_all + (threadIdx.x / W) * slice;   // this task group's slice
  for (;;) {
    const long long task = warp_claim<W>(counter) + (threadIdx.x & 31) / W;
    if (task - (threadIdx.x & 31) / W >= ntask) break;   // the same for the whole warp
    if (task < ntask) eri3_task<W>(prim, aux, pairs, ptab, tasks[task], boys, T, smem, lane);
    __syncwarp();
  }
}

// The same over a batch of geometries: task t belongs to the geometry g with
// off[g] <= t < off[g + 1] (an int64 offsets table of the geometries' task
// counts in this class group), its own shells, pairs and output.
template <int W>
__global__ void __launch_bounds__(32, kEri3BlocksPerSM) eri3_batch_kernel(const GeomTasks* __restrict__ geoms,
                                                        const long long* __restrict__ off, int ngeom,
                                                        const double* __restrict__ boys, int* counter, int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % W;
  double* smem = smem_all + (threadIdx.x / W) * slice;
  const long long ntask = off[ngeom];
  for (;;) {
    const long long task = warp_claim<W>(counter) + (threadIdx.x & 31) / W;
    if (task - (threadIdx.x & 31) / W >= ntask) break;   // the same for the whole warp
    if (task < ntask) {
      int lo = 0, hi = ngeom;   // off[lo] <= task < off[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= task) lo = mid;
        else hi = mid;
      }
      const GeomTasks& G = geoms[lo];
      eri3_task<W>(G.prim, G.aux, G.pairs, G.ptab, G.tasks[task - off[lo]], boys, G.out, smem, lane);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ (P|Q)

// G = 8 runs the classes set in small_mask (bit 8 la + lc), G = 32 the others.
template <int G>
__global__ void __launch_bounds__(32) eri2_kernel(DevShells aux, const double* __restrict__ boys, int* counter,
                                                  double* __restrict__ A, unsigned long long small_mask,
                                                  int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % G;
  double* smem = smem_all + (threadIdx.x / G) * slice;   // this task group's slice
  const unsigned gm = lane_group_mask<G>();
  const int ns = aux.nshell;
  const long long ntask = (long long)ns * (ns + 1) / 2;
  const int NA = aux.nfunc;
  for (;;) {
    long long task = warp_next_task<G>(counter, lane);
    if (task >= ntask) break;
    // task -> (sa >= sc)
    int sa = (int)((sqrt(8.0 * (double)task + 1.0) - 1.0) * 0.5);
    while ((long long)sa * (sa + 1) / 2 > task) --sa;
    while ((long long)(sa + 1) * (sa + 2) / 2 <= task) ++sa;
    int sc = (int)(task - (long long)sa * (sa + 1) / 2);
    if ((int)((small_mask >> (8 * aux.l[sa] + aux.l[sc])) & 1ull) != (G == 8 ? 1 : 0)) continue;
    // the more diffuse shell is the bra: the transfer then multiplies by p/q <= 1
    // (with a compact bra and a diffuse ket of high l the factor p/q, raised
    // to l, amplifies the bra recursion's rounding); the small-class mask is
    // symmetric, and both triangles of A are written
    if (aux_max_exp(aux, sa) > aux_max_exp(aux, sc)) { int t = sa; sa = sc; sc = t; }
    int la = aux.l[sa], lc = aux.l[sc];
    int emin = la, emax = la, L = la + lc;
    Eri3Plan pl(la, 0, lc, emin, emax, 1);
    double* Fm = smem + pl.fm;
    double* vrr = smem + pl.vrr;
    double* etr = smem + pl.etr;
    double* acc = smem + pl.acc;
    int accsz = acc_size(emin, emax, lc);
    for (int i = lane; i < accsz; i += G) acc[i] = 0.0;
    const double* PA = aux.xyz + 3 * sa;
    const double* PC = aux.xyz + 3 * sc;
    EtrShape sh{lc, emin, emax};
    for (int pa = 0; pa < aux.nprim[sa]; ++pa)
      for (int pc = 0; pc < aux.nprim[sc]; ++pc) {
        double al = aux.exps[aux.pstart[sa] + pa], ga = aux.exps[aux.pstart[sc] + pc];
        double w = aux.coefs[aux.pstart[sa] + pa] * aux.coefs[aux.pstart[sc] + pc];
        Prim3 t = make_prim3(al, PA, 0.0, PA, ga, PC);
        for (int m = lane; m <= L; m += G) Fm[m] = boys_eval(m, t.T, boys);
        __syncwarp(gm);
        warp_vrr<G>(vrr, L, t, Fm, lane);
        warp_etr_accumulate<G>(vrr, L, etr, sh, t, w, acc, Fm, lane);
      }
    // acc holds [a][c] directly (lb = 0); transform with b = s (identity 1x1)
    int nfa = aux.nf[la], nfc = aux.nf[lc];
    const double* tra = aux.tr + la * kTrStride * kTrStride;
    const double* trc = aux.tr + lc * kTrStride * kTrStride;
    double* s1 = smem + pl.t1;
    double* s2 = smem + pl.t2;
    const int na = ncart(la), nc = ncart(lc);
    for (int idx = lane; idx < na * nfc; idx += G) {
      int scc = idx % nfc, ka = idx / nfc;
      double v = 0.0;
      for (int k = 0; k < nc; ++k) v += trc[scc * kTrStride + k] * acc[ka * nc + k];
      s1[idx] = v;
    }
    __syncwarp(gm);
    for (int idx = lane; idx < nfa * nfc; idx += G) {
      int scc = idx % nfc, saa = idx / nfc;
      double v = 0.0;
      for (int k = 0; k < na; ++k) v += tra[saa * kTrStride + k] * s1[k * nfc + scc];
      s2[idx] = v;
    }
    __syncwarp(gm);
    const int P0 = aux.ao[sa], Q0 = aux.ao[sc];
    for (int idx = lane; idx < nfa * nfc; idx += G) {
      int scc = idx % nfc, saa = idx / nfc;
      double v = s2[idx];
      A[(size_t)(P0 + saa) * NA + Q0 + scc] = v;
      A[(size_t)(Q0 + scc) * NA + P0 + saa] = v;
    }
    __syncwarp(gm);
  }
}

// ------------------------------------------------------------ S, T, V

// Obara-Saika 1D overlap table s[i][j] (i <= imax, j <= jmax) of
// x_A^i e^{-a x_A^2} x_B^j e^{-b x_B^2}, including sqrt(pi/p) exp(-mu X_AB^2).
__device__ inline void os_overlap_1d(double a, double b, double XA, double XB, int imax, int jmax, double* s,
                                     int ld) {
  double p = a + b, P = (a * XA + b * XB) / p, PA = P - XA, PB = P - XB, X = XA - XB;
  double inv2p = 0.5 / p;
  s[0] = sqrt(3.14159265358979323846 / p) * exp(-a * b / p * X * X);
  for (int i = 1; i <= imax; ++i) {
    double v = PA * s[(i - 1) * ld];
    if (i >= 2) v += (i - 1) * inv2p * s[(i - 2) * ld];
    s[i * ld] = v;
  }
  for (int j = 1; j <= jmax; ++j)
    for (int i = 0; i <= imax; ++i) {
      double v = PB * s[i * ld + j - 1];
      if (j >= 2) v += (j - 1) * inv2p * s[i * ld + j - 2];
      if (i >= 1) v += i * inv2p * s[(i - 1) * ld + j - 1];
      s[i * ld + j] = v;
    }
}

template <int G>
__global__ void __launch_bounds__(32) one_electron_kernel(DevShells prim, int natoms, const int* __restrict__ Z,
                                                          const double* __restrict__ axyz,
                                                          const double* __restrict__ boys, int* counter,
                                                          double* __restrict__ S, double* __restrict__ Tk,
                                                          double* __restrict__ V, int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % G;
  double* smem = smem_all + (threadIdx.x / G) * slice;   // this task group's slice
  const unsigned gm = lane_group_mask<G>();
  const int ns = prim.nshell;
  const long long ntask = (long long)ns * (ns + 1) / 2;
  const int N = prim.nfunc;
  for (;;) {
    long long task = warp_next_task<G>(counter, lane);
    if (task >= ntask) break;
    int sa = (int)((sqrt(8.0 * (double)task + 1.0) - 1.0) * 0.5);
    while ((long long)sa * (sa + 1) / 2 > task) --sa;
    while ((long long)(sa + 1) * (sa + 2) / 2 <= task) ++sa;
    int sb = (int)(task - (long long)sa * (sa + 1) / 2);
    int la = prim.l[sa], lb = prim.l[sb];
    int na = ncart(la), nb = ncart(lb);
    const double* A = prim.xyz + 3 * sa;
    const double* B = prim.xyz + 3 * sb;
    // smem: sacc[na*nb], tacc[na*nb], then V machinery
    double* sacc = smem;
    double* tacc = sacc + na * nb;
    double* s1d = tacc + na * nb;               // 3 x 8 x 8 per primitive pair
    int emin = la, emax = la + lb, L = emax;
    Eri3Plan pl(la, lb, 0, emin, emax, 1);
    double* base = s1d + 3 * 64;
    double* Fm = base + pl.fm;
    double* vrr = base + pl.vrr;
    double* acc = base + pl.acc;
    for (int i = lane; i < na * nb; i += G) {
      sacc[i] = 0.0;
      tacc[i] = 0.0;
    }
    for (int i = lane; i < acc_size(emin, emax, 0); i += G) acc[i] = 0.0;
    __syncwarp(gm);
    EtrShape sh{0, emin, emax};
    for (int pa = 0; pa < prim.nprim[sa]; ++pa)
      for (int pb = 0; pb < prim.nprim[sb]; ++pb) {
        double al = prim.exps[prim.pstart[sa] + pa], be = prim.exps[prim.pstart[sb] + pb];
        double w = prim.coefs[prim.pstart[sa] + pa] * prim.coefs[prim.pstart[sb] + pb];
        if (lane < 3) os_overlap_1d(al, be, A[lane], B[lane], la, lb + 2, s1d + lane * 64, 8);
        __syncwarp(gm);
        for (int idx = lane; idx < na * nb; idx += G) {
          int ka = idx / nb, kb = idx % nb;
          int ca[3], cb[3];
          cart_decode(la, ka, ca[0], ca[1], ca[2]);
          cart_decode(lb, kb, cb[0], cb[1], cb[2]);
          double sd[3], kd[3];
          for (int d = 0; d < 3; ++d) {
            const double* s = s1d + d * 64;
            int i = ca[d], j = cb[d];
            sd[d] = s[i * 8 + j];
            double k2 = 4.0 * be * be * s[i * 8 + j + 2] - 2.0 * be * (2 * j + 1) * s[i * 8 + j];
            if (j >= 2) k2 += j * (j - 1) * s[i * 8 + j - 2];
            kd[d] = k2;
          }
          sacc[idx] += w * sd[0] * sd[1] * sd[2];
          tacc[idx] += -0.5 * w * (kd[0] * sd[1] * sd[2] + sd[0] * kd[1] * sd[2] + sd[0] * sd[1] * kd[2]);
        }
        __syncwarp(gm);
        for (int C = 0; C < natoms; ++C) {
          Prim3 t = make_prim_point(al, A, be, B, axyz + 3 * C);
          for (int m = lane; m <= L; m += G) Fm[m] = boys_eval(m, t.T, boys);
          __syncwarp(gm);
          warp_vrr<G>(vrr, L, t, Fm, lane);
          warp_etr_accumulate<G>(vrr, L, nullptr, sh, t, -w * Z[C], acc, Fm, lane);
        }
      }
    double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
    const double* vcart = warp_hrr<G>(acc, emin, la, lb, 0, AB, base + pl.hrr, pl.half, lane);
    int nfa = prim.nf[la], nfb = prim.nf[lb];
    const double* tra = prim.tr + la * kTrStride * kTrStride;
    const double* trb = prim.tr + lb * kTrStride * kTrStride;
    double* o1 = base + pl.t1;
    double* o2 = base + pl.t2;
    const double* srcs[3] = {sacc, tacc, vcart};
    double* dsts[3] = {S, Tk, V};
    for (int q = 0; q < 3; ++q) {
      const double* src = srcs[q];
      for (int idx = lane; idx < na * nfb; idx += G) {
        int sbb = idx % nfb, ka = idx / nfb;
        double v = 0.0;
        for (int k = 0; k < nb; ++k) v += trb[sbb * kTrStride + k] * src[ka * nb + k];
        o1[idx] = v;
      }
      __syncwarp(gm);
      for (int idx = lane; idx < nfa * nfb; idx += G) {
        int sbb = idx % nfb, saa = idx / nfb;
        double v = 0.0;
        for (int k = 0; k < na; ++k) v += tra[saa * kTrStride + k] * o1[k * nfb + sbb];
        o2[idx] = v;
      }
      __syncwarp(gm);
      const int mu0 = prim.ao[sa], nu0 = prim.ao[sb];
      for (int idx = lane; idx < nfa * nfb; idx += G) {
        int sbb = idx % nfb, saa = idx / nfb;
        dsts[q][(size_t)(mu0 + saa) * N + nu0 + sbb] = o2[idx];
        dsts[q][(size_t)(nu0 + sbb) * N + mu0 + saa] = o2[idx];
      }
      __syncwarp(gm);
    }
  }
}

// ------------------------------------------------------------ Schwarz (ab|ab)

// Shared-memory size (doubles) of schwarz_kernel for one (la, lb) class, and the
// ping-pong half size used by both HRR stages.
__host__ __device__ inline int schwarz_smem(int la, int lb, int* half_out) {
  const int lc = la, ld = lb, lf = lc + ld, emin = la, emax = la + lb, L = emax + lf;
  const int nab = ncart(la) * ncart(lb);
  EtrShape sh{lf, emin, emax};
  int accsz = 0, brasz = 0, half = 0;
  for (int f = lc; f <= lf; ++f) {
    accsz += (cart_offset(emax + 1) - cart_offset(emin)) * ncart(f);
    brasz += nab * ncart(f);
    int h = hrr_scratch(la, lb, f, emax) / 2;
    if (h > half) half = h;
  }
  for (int d = 1; d <= ld; ++d) {
    int n = 0;
    for (int f = lc; f <= lf - d; ++f) n += nab * ncart(f) * ncart(d);
    if (n > half) half = n;
  }
  if (half_out) *half_out = half;
  return kFmRegion + vrr_size(L) + (lf > 0 ? sh.total() : 0) + accsz + brasz + 2 * half;
}

// Q_ab = sqrt(max_{mu in a, nu in b} (mu nu|mu nu)) over Cartesian components
// (Sec. 3.1.1: the Schwarz bound |(mu nu|lam sig)| <= Q_{mu nu} Q_{lam sig}).
// Four-centre recursion with the ket pair equal to the bra pair: bra VRR with
// W = (pP + qQ)/(p+q), electron transfer to f = lc..lc+ld with the
// -(beta AB + delta CD)/q term, bra HRR on every ket level f, then ket HRR.
// G = 8 runs the classes set in small_mask (bit 8 la + lb, la >= lb), G = 32
// the others.
template <int G>
__global__ void __launch_bounds__(32) schwarz_kernel(DevShells prim, const double* __restrict__ boys, int* counter,
                                                     double* __restrict__ Q, unsigned long long small_mask,
                                                     int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % G;
  double* smem = smem_all + (threadIdx.x / G) * slice;   // this task group's slice
  const unsigned gm = lane_group_mask<G>();
  const int ns = prim.nshell;
  const long long ntask = (long long)ns * (ns + 1) / 2;
  for (;;) {
    long long task = warp_next_task<G>(counter, lane);
    if (task >= ntask) break;
    int sa = (int)((sqrt(8.0 * (double)task + 1.0) - 1.0) * 0.5);
    while ((long long)sa * (sa + 1) / 2 > task) --sa;
    while ((long long)(sa + 1) * (sa + 2) / 2 <= task) ++sa;
    int sb = (int)(task - (long long)sa * (sa + 1) / 2);
    if (prim.l[sa] < prim.l[sb]) { int t = sa; sa = sb; sb = t; }
    const int la = prim.l[sa], lb = prim.l[sb];
    if ((int)((small_mask >> (8 * la + lb)) & 1ull) != (G == 8 ? 1 : 0)) continue;
    const int lc = la, ld = lb, lf = lc + ld;          // ket pair = bra pair
    const int emin = la, emax = la + lb, L = emax + lf;
    const int na = ncart(la), nb = ncart(lb);
    EtrShape sh{lf, emin, emax};
    // smem: Fm | vrr | etr | acc[f][e][kf] for f in [lc, lf] | bra-HRR out [f][ka][kb][kf] | scratch
    double* Fm = smem;
    double* vrr = Fm + kFmRegion;
    double* etr = vrr + vrr_size(L);
    double* acc = etr + (lf > 0 ? sh.total() : 0);
    int accsz = 0;
    for (int f = lc; f <= lf; ++f) accsz += (cart_offset(emax + 1) - cart_offset(emin)) * ncart(f);
    double* bra = acc + accsz;
    int brasz = 0;
    for (int f = lc; f <= lf; ++f) brasz += na * nb * ncart(f);
    double* scr = bra + brasz;
    int half = 0;
    schwarz_smem(la, lb, &half);
    for (int i = lane; i < accsz; i += G) acc[i] = 0.0;
    const double* A = prim.xyz + 3 * sa;
    const double* B = prim.xyz + 3 * sb;
    for (int pa = 0; pa < prim.nprim[sa]; ++pa)
      for (int pb = 0; pb < prim.nprim[sb]; ++pb)
        for (int pc = 0; pc < prim.nprim[sa]; ++pc)
          for (int pd = 0; pd < prim.nprim[sb]; ++pd) {
            double al = prim.exps[prim.pstart[sa] + pa], be = prim.exps[prim.pstart[sb] + pb];
            double ga = prim.exps[prim.pstart[sa] + pc], de = prim.exps[prim.pstart[sb] + pd];
            double w = prim.coefs[prim.pstart[sa] + pa] * prim.coefs[prim.pstart[sb] + pb] *
                       prim.coefs[prim.pstart[sa] + pc] * prim.coefs[prim.pstart[sb] + pd];
            Prim3 t;
            double p = al + be, q = ga + de, P[3], Qc[3], R2ab = 0.0, R2pq = 0.0;
            t.p = p; t.q = q; t.beta = be; t.rho = p * q / (p + q);
            for (int i = 0; i < 3; ++i) {
              P[i] = (al * A[i] + be * B[i]) / p;
              Qc[i] = (ga * A[i] + de * B[i]) / q;
              double AB = A[i] - B[i];
              R2ab += AB * AB;
              // fold -(beta AB + delta CD)/q into the ETR's beta AB / q (C = A, D = B)
              t.AB[i] = AB + (de / be) * AB;
            }
            for (int i = 0; i < 3; ++i) {
              double Wi = (p * P[i] + q * Qc[i]) / (p + q);
              t.PA[i] = P[i] - A[i];
              t.WP[i] = Wi - P[i];
              R2pq += (P[i] - Qc[i]) * (P[i] - Qc[i]);
            }
            t.T = t.rho * R2pq;
            t.pref = 34.98683665524972 / (p * q * sqrt(p + q)) * exp(-al * be / p * R2ab) * exp(-ga * de / q * R2ab);
            prim3_factors(t);
            for (int m = lane; m <= L; m += G) Fm[m] = boys_eval(m, t.T, boys);
            __syncwarp(gm);
            warp_vrr<G>(vrr, L, t, Fm, lane);
            warp_etr<G>(vrr, L, etr, sh, t, Fm, lane);
            // acc[f-block][e][ke][kf] += w * level f, e in [emin, emax]
            int off = 0;
            for (int f = lc; f <= lf; ++f) {
              int ncf = ncart(f);
              int n = (cart_offset(emax + 1) - cart_offset(emin)) * ncf;
              for (int idx = lane; idx < n; idx += G) {
                int r = idx / ncf, kf = idx - r * ncf;
                int e = emin;
                while (cart_offset(e + 1) - cart_offset(emin) <= r) ++e;
                int ke = r - (cart_offset(e) - cart_offset(emin));
                acc[off + idx] += w * etr_get(vrr, L, etr, sh, f, e, ke, kf);
              }
              off += n;
            }
            __syncwarp(gm);
          }
    // bra HRR for every ket level f
    double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
    {
      int aoff = 0, boff = 0;
      for (int f = lc; f <= lf; ++f) {
        int ncf = ncart(f);
        const double* out = warp_hrr<G>(acc + aoff, emin, la, lb, f, AB, scr, half, lane);
        for (int i = lane; i < na * nb * ncf; i += G) bra[boff + i] = out[i];
        __syncwarp(gm);
        aoff += (cart_offset(emax + 1) - cart_offset(emin)) * ncf;
        boff += na * nb * ncf;
      }
    }
    // ket HRR: (ab|c, d+1_i) = (ab|c+1_i, d) + CD_i (ab|c, d), CD = AB; rows f in
    // [lc, lf - d]; ping-pong in scr; diagonal (mu nu|mu nu) at the end
    double qmax = 0.0;
    {
      const int nab = na * nb;
      const double* prev = bra;           // level d' = 0: [f][ab][kf] packed by f blocks
      int prev_nd = 1;
      double* bufs[2] = {scr, scr + half};
      for (int d = 1; d <= ld; ++d) {
        double* cur = bufs[(d - 1) & 1];
        int nd = ncart(d);
        int fhi = lf - d;
        int n = 0;
        for (int f = lc; f <= fhi; ++f) n += nab * ncart(f) * nd;
        for (int idx = lane; idx < n; idx += G) {
          // decode idx -> (f, ab, kf, kd) with layout [f-block][ab][kf][kd]
          int rem = idx, f = lc;
          while (rem >= nab * ncart(f) * nd) { rem -= nab * ncart(f) * nd; ++f; }
          int ncf = ncart(f);
          int kd = rem % nd, r2 = rem / nd, kf = r2 % ncf, ab = r2 / ncf;
          int dx, dy, dz, fx, fy, fz;
          cart_decode(d, kd, dx, dy, dz);
          cart_decode(f, kf, fx, fy, fz);
          int i = dx > 0 ? 0 : (dy > 0 ? 1 : 2);
          int dl[3] = {dx, dy, dz};
          dl[i] -= 1;
          int kdl = cart_index(d - 1, dl[0], dl[1]);
          int fp[3] = {fx, fy, fz};
          fp[i] += 1;
          int kfp = cart_index(f + 1, fp[0], fp[1]);
          // offsets of level f and f+1 in prev: [f-block][ab][kf][kd_prev]
          int o_f = 0;
          for (int g = lc; g < f; ++g) o_f += nab * ncart(g) * prev_nd;
          int o_f1 = o_f + nab * ncf * prev_nd;
          double v = prev[o_f1 + (ab * ncart(f + 1) + kfp) * prev_nd + kdl] +
                     AB[i] * prev[o_f + (ab * ncf + kf) * prev_nd + kdl];
          cur[idx] = v;
        }
        __syncwarp(gm);
        prev = cur;
        prev_nd = nd;
      }
      // prev now holds level f = lc only: [ab][kc][kd] with (kc, kd) over (la, lb) = (ka, kb)
      for (int idx = lane; idx < nab; idx += G) {
        int ka = idx / nb, kb = idx % nb;
        double v = prev[(idx * ncart(lc) + ka) * prev_nd + kb];
        qmax = fmax(qmax, fabs(v));
      }
    }
    for (int o = G / 2; o > 0; o >>= 1) qmax = fmax(qmax, __shfl_xor_sync(gm, qmax, o));
    if (lane == 0) {
      int a0 = max(sa, sb), b0 = min(sa, sb);
      Q[(long long)a0 * (a0 + 1) / 2 + b0] = sqrt(qmax);
    }
    __syncwarp(gm);
  }
}

// ------------------------------------------------------------ launchers

// ordered: only classes with la >= lb occur
static int max_smem_eri3(int max_la, int max_lb, int max_lc, bool ordered = true) {
  int best = 0;
  for (int la = 0; la <= max_la; ++la)
    for (int lb = 0; lb <= (ordered ? std::min(la, max_lb) : max_lb); ++lb)
      for (int lc = 0; lc <= max_lc; ++lc) {
        int s = smem_eri3_doubles(la, lb, lc);
        if (s > best) best = s;
      }
  return best;
}

static int grid_for(int smem_bytes) {
  int dev = 0, sms = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int per_sm = smem_bytes > 0 ? maxsm / (smem_bytes + 1024) : 32;
  if (per_sm > 32) per_sm = 32;
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

static void set_smem(const void* fn, int bytes) {
  raise_smem_limit(fn, bytes);
}

void launch_eri3(const IntegralCtx& ic, const DevShells& prim, const DevShells& aux, const ShellPair* pairs,
                 const PairTable& pt, const TaskGroup* groups, int ngroups, double* T) {
  for (int g = 0; g < ngroups; ++g) {
    if (groups[g].ntask == 0) continue;
    const int W = groups[g].width, slice = groups[g].smem_eri3 / (int)sizeof(double);
    const int smem = (32 / W) * slice * (int)sizeof(double);
    RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
    auto run = [&](auto kernel) {
      set_smem((const void*)kernel, smem);
      kernel<<<grid_for(smem), 32, smem, ic.stream>>>(prim, aux, pairs, pt, groups[g].tasks, groups[g].ntask, ic.boys,
                                                      ic.counter, T, slice);
    };
    if (W == 8) run(eri3_kernel<8>);
    else if (W == 16) run(eri3_kernel<16>);
    else run(eri3_kernel<32>);
    RIHF_LAUNCH_CHECK();
    if (ic.launches) *ic.launches += 1;
  }
}

bool batch_tables(const IntegralCtx& ic, const std::vector<BatchGeom>& batch, int g, BatchTables& t, bool grad,
                  int& slice_bytes, long long& ntask) {
  const int n = (int)batch.size();
  std::vector<GeomTasks> geoms(n);
  std::vector<long long> off(n + 1, 0);
  slice_bytes = 0;
  for (int i = 0; i < n; ++i) {
    geoms[i] = batch[i].g;
    geoms[i].tasks = batch[i].groups[g].tasks;
    off[i + 1] = off[i] + batch[i].groups[g].ntask;
    if (batch[i].groups[g].ntask > 0)
      slice_bytes = std::max(slice_bytes, grad ? batch[i].groups[g].smem_grad : batch[i].groups[g].smem_eri3);
  }
  ntask = off[n];
  if (ntask == 0) return false;
  RIHF_CUDA(cudaMemcpyAsync(t.geoms + (size_t)g * t.cap, geoms.data(), sizeof(GeomTasks) * n,
                            cudaMemcpyHostToDevice, ic.stream));
  RIHF_CUDA(cudaMemcpyAsync(t.off + (size_t)g * (t.cap + 1), off.data(), sizeof(long long) * (n + 1),
                            cudaMemcpyHostToDevice, ic.stream));
  RIHF_CUDA(cudaStreamSynchronize(ic.stream));   // the host arrays are temporaries
  return true;
}

void launch_eri3_batch(const IntegralCtx& ic, const std::vector<BatchGeom>& batch, int ngroups, BatchTables& t) {
  const int n = (int)batch.size();
  if (n == 0) return;
  if (n > t.cap) throw RihfError(RIHF_ERR_INVALID_ARG, "launch_eri3_batch: batch tables too small");
  for (int g = 0; g < ngroups; ++g) {
    int slice_bytes = 0;
    long long ntask = 0;
    if (!batch_tables(ic, batch, g, t, false, slice_bytes, ntask)) continue;
    const int W = task_group_width(g), slice = slice_bytes / (int)sizeof(double);
    const int smem = (32 / W) * slice * (int)sizeof(double);
    RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
    auto run = [&](auto kernel) {
      set_smem((const void*)kernel, smem);
      kernel<<<grid_for(smem), 32, smem, ic.stream>>>(t.geoms + (size_t)g * t.cap, t.off + (size_t)g * (t.cap + 1),
                                                      n, ic.boys, ic.counter, slice);
    };
    if (W == 8) run(eri3_batch_kernel<8>);
    else if (W == 16) run(eri3_batch_kernel<16>);
    else run(eri3_batch_kernel<32>);
    RIHF_LAUNCH_CHECK();
    if (ic.launches) *ic.launches += 1;
  }
}

// ------------------------------------------------------------ pair table

// One thread per shell pair: p, 1/p, P, P - A and the Gaussian-product
// prefactor of every primitive pair, in the la >= lb order of the kernels.
__global__ void pair_prim_kernel(DevShells prim, const ShellPair* __restrict__ pairs, int npairs,
                                 const int* __restrict__ off, PairPrim* __restrict__ pp) {
  const int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= npairs) return;
  int sa = pairs[ip].a, sb = pairs[ip].b;
  if (prim.l[sa] < prim.l[sb]) { int t = sa; sa = sb; sb = t; }
  const double* A = prim.xyz + 3 * sa;
  const double* B = prim.xyz + 3 * sb;
  double R2 = 0.0;
  for (int i = 0; i < 3; ++i) R2 += (A[i] - B[i]) * (A[i] - B[i]);
  PairPrim* out = pp + off[ip];
  const int nb = prim.nprim[sb];
  for (int pa = 0; pa < prim.nprim[sa]; ++pa)
    for (int pb = 0; pb < nb; ++pb) {
      const double al = prim.exps[prim.pstart[sa] + pa], be = prim.exps[prim.pstart[sb] + pb];
      const double p = al + be, ip_ = 1.0 / p;
      PairPrim q;
      q.p = p;
      q.inv_p = ip_;
      q.alpha = al;
      q.beta = be;
      q.K = 34.98683665524972 * prim.coefs[prim.pstart[sa] + pa] * prim.coefs[prim.pstart[sb] + pb] *
            exp(-al * be * ip_ * R2) * ip_;
      for (int i = 0; i < 3; ++i) {
        q.P[i] = (al * A[i] + be * B[i]) * ip_;
        q.PA[i] = q.P[i] - A[i];
      }
      q.pad = 0.0;
      out[pa * nb + pb] = q;
    }
}

std::vector<int> pair_prim_offsets(const std::vector<ShellPair>& pairs, const std::vector<int>& nprim) {
  std::vector<int> off(pairs.size() + 1, 0);
  for (size_t i = 0; i < pairs.size(); ++i) off[i + 1] = off[i] + nprim[pairs[i].a] * nprim[pairs[i].b];
  return off;
}

void launch_pair_prims(const IntegralCtx& ic, const DevShells& prim, const ShellPair* pairs, int npairs,
                       const int* off, PairPrim* pp) {
  if (npairs <= 0) return;
  pair_prim_kernel<<<(npairs + 127) / 128, 128, 0, ic.stream>>>(prim, pairs, npairs, off, pp);
  RIHF_LAUNCH_CHECK();
  if (ic.launches) *ic.launches += 1;
}

// ------------------------------------------------------------ flop model

namespace {

double vrr_flops(int L) {
  double f = 3.0 * (L + 1);   // prefactor and the k/(2p), k/(2q) tables
  for (int e = 1; e <= L; ++e)
    for (int k = 0; k < ncart(e); ++k) {
      int lx, ly, lz;
      cart_decode(e, k, lx, ly, lz);
      int c[3] = {lx, ly, lz};
      const int i = lx > 0 ? 0 : (ly > 0 ? 1 : 2);
      c[i] -= 1;
      f += (L - e + 1) * (3.0 + (c[i] > 0 ? 4.0 : 0.0));
    }
  return f;
}

double etr_flops(const EtrShape& sh) {
  double f = 0.0;
  for (int c = 1; c <= sh.lc; ++c)
    for (int e = sh.elo(c); e <= sh.ehi(c); ++e)
      for (int ke = 0; ke < ncart(e); ++ke)
        for (int kc = 0; kc < ncart(c); ++kc) {
          int ex, ey, ez, cx, cy, cz;
          cart_decode(e, ke, ex, ey, ez);
          cart_decode(c, kc, cx, cy, cz);
          const int i = cx > 0 ? 0 : (cy > 0 ? 1 : 2);
          const int eo[3] = {ex, ey, ez};
          int cl[3] = {cx, cy, cz};
          cl[i] -= 1;
          f += 3.0 + (eo[i] > 0 ? 2.0 : 0.0) + (cl[i] > 0 ? 2.0 : 0.0);
        }
  return f;
}

double hrr_flops(int la, int lb, int lc) {
  double f = 0.0;
  for (int b = 1; b <= lb; ++b)
    f += 2.0 * (cart_offset(la + lb - b + 1) - cart_offset(la)) * ncart(b) * ncart(lc);
  return f;
}

}  // namespace

void task_flops(const std::vector<ShellPair>& pairs, const std::vector<int>& lprim, const std::vector<int>& nprim,
                const std::vector<int>& patom, const std::vector<int>& laux, const std::vector<int>& naux_prim,
                const std::vector<int>& aatom, const std::vector<int>& nf, const std::vector<double>& pmax,
                const std::vector<double>& qmin, double* eri3, double* grad3) {
  constexpr int nl = kMaxLPrim + 1, nc = kMaxLAux + 1;
  double e_prim[nl][nl][nc], e_task[nl][nl][nc], g_prim[nl][nl][nc], g_task[nl][nl][nc];
  double e_mir[nl][nl][nc], g_mir[nl][nl][nc];   // per-triple recursion work of the mirrored path
  double e_acc[nl][nl][nc], g_acc[nl][nl][nc];   // accumulation passes (skipped by single-triple tasks with lc > 0)
  for (int la = 0; la < nl; ++la)
    for (int lb = 0; lb <= la; ++lb)
      for (int lc = 0; lc < nc; ++lc) {
        const int na = ncart(la), nb = ncart(lb), ncc = ncart(lc);
        const int fa = nf[la], fb = nf[lb], fc = nf[lc];
        const double setup = 25.0;
        {
          const int L = la + lb + lc;
          e_prim[la][lb][lc] = setup + 14.0 * (L + 1) + vrr_flops(L) + etr_flops(EtrShape{lc, la, la + lb});
          e_mir[la][lb][lc] = setup + 14.0 * (L + 1) + vrr_flops(L) + etr_flops(EtrShape{la + lb, lc, lc});
          e_acc[la][lb][lc] = 2.0 * acc_size(la, la + lb, lc);
          e_task[la][lb][lc] = hrr_flops(la, lb, lc) +
                               2.0 * ((double)na * nb * fc * ncc + (double)na * fb * fc * nb + (double)fa * fb * fc * na);
        }
        {
          const int emin = la > 0 ? la - 1 : 0, emax = la + lb + 1, L = emax + lc;
          g_prim[la][lb][lc] = setup + 14.0 * (L + 1) + vrr_flops(L) + etr_flops(EtrShape{lc, emin, emax});
          g_mir[la][lb][lc] = setup + 14.0 * (L + 1) + vrr_flops(L) + etr_flops(EtrShape{emax, lc, lc});
          g_acc[la][lb][lc] = 6.0 * acc_size(emin, emax, lc);
          g_task[la][lb][lc] = 2.0 * ((double)fa * fb * ncc * fc + (double)fa * nb * ncc * fb + (double)na * nb * ncc * fa) +
                               hrr_flops(la + 1, lb, lc) + (la > 0 ? hrr_flops(la - 1, lb, lc) : 0.0) +
                               hrr_flops(la, lb + 1, lc) + (lb > 0 ? hrr_flops(la, lb - 1, lc) : 0.0) +
                               24.0 * na * nb * ncc;
        }
      }
  double fe = 0.0, fg = 0.0;
  for (const ShellPair& sp : pairs) {
    int a = sp.a, b = sp.b;
    if (lprim[a] < lprim[b]) std::swap(a, b);
    const int la = lprim[a], lb = lprim[b];
    const double npab = (double)nprim[a] * nprim[b];
    for (int c = 0; c < (int)laux.size(); ++c) {
      const int lc = laux[c];
      const double np3 = npab * naux_prim[c];
      // marked tasks run mirrored (counted so when their largest bra exponent
      // sum exceeds the auxiliary exponent) and always accumulate
      const bool mir = mirror_task(pmax[a] + pmax[b], qmin[c], lc);
      // one triple: the kernels read the last transfer level in place, or
      // (mirrored) store it once; either way no accumulation passes
      const bool single = np3 == 1.0 && lc > 0;
      fe += np3 * (mir ? e_mir : e_prim)[la][lb][lc] + e_task[la][lb][lc] + (single ? 0.0 : np3 * e_acc[la][lb][lc]);
      if (!(patom[a] == patom[b] && patom[b] == aatom[c]))
        fg += np3 * (mir ? g_mir : g_prim)[la][lb][lc] + g_task[la][lb][lc] +
              (single ? 6.0 : np3 * g_acc[la][lb][lc]);
    }
  }
  *eri3 = fe;
  *grad3 = fg;
}

// Class-grouped task lists: every (pair, auxiliary shell) task goes to the first
// group whose shared-memory bound covers both its integral and its derivative
// class, so light classes run with many resident warps per SM.  Inside a group
// the tasks are ordered by shape (mirror flag, la, lb, lc and the three shells'
// primitive counts), the heaviest shapes first and auxiliary shell by shell
// within a shape: the lane groups of a warp, which claim neighbouring tasks
// together, then run the same recursion with the same trip counts in lockstep
// instead of one after another, warps resident on one SM share their code, and
// the lightest tasks fill the end of the launch.
void build_task_groups(const std::vector<ShellPair>& pairs, const std::vector<int>& lprim,
                       const std::vector<int>& nprim, const std::vector<int>& laux,
                       const std::vector<int>& naux_prim, const std::vector<double>& pmax,
                       const std::vector<double>& qmin, std::vector<std::vector<int2>>& tasks,
                       std::vector<int>& smem_eri3, std::vector<int>& smem_grad) {
  // group 0: tiny classes as 8-lane groups (4 tasks per warp); group 1: small
  // classes as 16-lane groups (2 tasks per warp, about 15 warps per SM); then
  // about 17, 7, 3, 1-2 and 1 warps per SM (228 KB shared memory, 1 KB
  // reserved per block): the f and g classes of larger basis sets span 28 to
  // 205 KB, and one bound for all of them would hold every such task to the
  // residency of the largest
  const int limits[kTaskGroups] = {3584, 7168, 12 * 1024, 28 * 1024, 56 * 1024, 112 * 1024, 1 << 30};
  // pair shapes (la >= lb and the primitive counts in that order; equal l:
  // the larger count first) and auxiliary shapes (lc, primitive count)
  std::map<std::array<int, 4>, int> pmap;
  std::map<std::array<int, 2>, int> amap;
  std::vector<std::array<int, 4>> pkey;
  std::vector<std::array<int, 2>> akey;
  std::vector<int> pshape(pairs.size()), ashape(laux.size());
  for (size_t p = 0; p < pairs.size(); ++p) {
    int a = pairs[p].a, b = pairs[p].b;
    if (lprim[a] < lprim[b] || (lprim[a] == lprim[b] && nprim[a] < nprim[b])) std::swap(a, b);
    const std::array<int, 4> k{lprim[a], lprim[b], nprim[a], nprim[b]};
    auto it = pmap.find(k);
    if (it == pmap.end()) {
      it = pmap.emplace(k, (int)pkey.size()).first;
      pkey.push_back(k);
    }
    pshape[p] = it->second;
  }
  for (size_t c = 0; c < laux.size(); ++c) {
    const std::array<int, 2> k{laux[c], naux_prim[c]};
    auto it = amap.find(k);
    if (it == amap.end()) {
      it = amap.emplace(k, (int)akey.size()).first;
      akey.push_back(k);
    }
    ashape[c] = it->second;
  }
  const int nps = (int)pkey.size(), nas = (int)akey.size();
  const int nbucket = 2 * nps * nas;   // (mirror, pair shape, auxiliary shape)
  auto mirror_of = [&](int p, int c) {
    return mirror_task(pmax[pairs[p].a] + pmax[pairs[p].b], qmin[c], laux[c]) ? 1 : 0;
  };
  // pass 1: bucket sizes
  std::vector<long long> count(nbucket, 0);
  for (int c = 0; c < (int)laux.size(); ++c)
    for (int p = 0; p < (int)pairs.size(); ++p) ++count[((size_t)mirror_of(p, c) * nps + pshape[p]) * nas + ashape[c]];
  // per bucket its shared-memory plans (the derivative task's compact plan
  // when it has one primitive triple) and the first group that holds both;
  // per group, its buckets heaviest first (primitive triples x derivative
  // working set), and each bucket's start in the group's list
  tasks.assign(kTaskGroups, {});
  smem_eri3.assign(kTaskGroups, 0);
  smem_grad.assign(kTaskGroups, 0);
  std::vector<std::vector<std::pair<double, int>>> order(kTaskGroups);
  for (int bkt = 0; bkt < nbucket; ++bkt) {
    if (count[bkt] == 0) continue;
    const int mi = bkt / (nps * nas), ps = bkt / nas % nps, as = bkt % nas;
    const int la = pkey[ps][0], lb = pkey[ps][1], lc = akey[as][0];
    const int np3 = pkey[ps][2] * pkey[ps][3] * akey[as][1];
    const int se = smem_eri3_doubles(la, lb, lc, mi == 1, true) * (int)sizeof(double);
    const int sg = smem_grad_doubles(la, lb, lc, mi == 1, np3 == 1) * (int)sizeof(double);
    int g = 0;
    while (g + 1 < kTaskGroups && std::max(se, sg) > limits[g]) ++g;
    order[g].emplace_back(-(double)np3 * sg, bkt);
    smem_eri3[g] = std::max(smem_eri3[g], se);
    smem_grad[g] = std::max(smem_grad[g], sg);
  }
  std::vector<long long> start(nbucket, 0);
  std::vector<int> group_of(nbucket, 0);
  for (int g = 0; g < kTaskGroups; ++g) {
    std::sort(order[g].begin(), order[g].end());
    long long n = 0;
    for (const auto& e : order[g]) {
      start[e.second] = n;
      group_of[e.second] = g;
      n += count[e.second];
    }
    if (n > kMaxGroupTasks) throw RihfError(RIHF_ERR_INVALID_ARG, "build_task_groups: too many 3-centre tasks");
    tasks[g].resize((size_t)n);
  }
  // pass 2: fill, auxiliary shell by shell (then pair) within each bucket
  for (int c = 0; c < (int)laux.size(); ++c)
    for (int p = 0; p < (int)pairs.size(); ++p) {
      const int mi = mirror_of(p, c);
      const size_t bkt = ((size_t)mi * nps + pshape[p]) * nas + ashape[c];
      tasks[group_of[bkt]][(size_t)start[bkt]++] = make_int2(p, mi ? ~c : c);
    }
}

unsigned long long eri2_small_classes(int max_la, int* slice_doubles) {
  // the 3.5 KB working-set limit of the 8-lane 3-centre group, applied to
  // both the (P|Q) integrals and their derivatives, in both orders (the
  // kernels may exchange bra and ket), so the mask is symmetric
  unsigned long long mask = 0;
  int slice = 0;
  for (int la = 0; la <= max_la; ++la)
    for (int lc = 0; lc <= max_la; ++lc) {
      const int e = std::max(smem_eri3_doubles(la, 0, lc), smem_eri3_doubles(lc, 0, la));
      const int g = std::max(smem_grad_doubles(la, 0, lc), smem_grad_doubles(lc, 0, la));
      if (std::max(e, g) * (int)sizeof(double) > 3584) continue;
      mask |= 1ull << (8 * la + lc);
      slice = std::max(slice, std::max(e, g));
    }
  if (slice_doubles) *slice_doubles = slice;
  return mask;
}

void launch_eri2(const IntegralCtx& ic, const DevShells& aux, int max_la, double* A) {
  // small classes as 8-lane groups (four tasks per warp), then the rest with
  // whole warps; each launch claims every task and skips the other's classes
  int small_slice = 0;
  const unsigned long long mask = eri2_small_classes(max_la, &small_slice);
  if (mask) {
    const int smem = 4 * small_slice * (int)sizeof(double);
    set_smem((const void*)eri2_kernel<8>, smem);
    RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
    eri2_kernel<8><<<grid_for(smem), 32, smem, ic.stream>>>(aux, ic.boys, ic.counter, A, mask, small_slice);
    RIHF_LAUNCH_CHECK();
    if (ic.launches) *ic.launches += 1;
  }
  const int smem = max_smem_eri3(max_la, 0, max_la) * (int)sizeof(double);
  set_smem((const void*)eri2_kernel<32>, smem);
  RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
  eri2_kernel<32><<<grid_for(smem), 32, smem, ic.stream>>>(aux, ic.boys, ic.counter, A, mask, 0);
  RIHF_LAUNCH_CHECK();
  if (ic.launches) *ic.launches += 1;
}

int schwarz_smem_bytes(int max_lp) {
  int best = 0;
  for (int la = 0; la <= max_lp; ++la)
    for (int lb = 0; lb <= la; ++lb) best = std::max(best, schwarz_smem(la, lb, nullptr));
  return best * (int)sizeof(double);
}

void launch_schwarz(const IntegralCtx& ic, const DevShells& prim, int max_lp, double* Q) {
  // small classes (working set within 3.5 KB) as 8-lane groups, four tasks
  // per warp, then the rest with whole warps; each launch claims every task
  // and skips the other's classes
  unsigned long long mask = 0;
  int small_slice = 0;
  for (int la = 0; la <= max_lp; ++la)
    for (int lb = 0; lb <= la; ++lb) {
      const int d = schwarz_smem(la, lb, nullptr);
      if (d * (int)sizeof(double) > 3584) continue;
      mask |= 1ull << (8 * la + lb);
      small_slice = std::max(small_slice, d);
    }
  if (mask) {
    const int smem = 4 * small_slice * (int)sizeof(double);
    set_smem((const void*)schwarz_kernel<8>, smem);
    RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
    schwarz_kernel<8><<<grid_for(smem), 32, smem, ic.stream>>>(prim, ic.boys, ic.counter, Q, mask, small_slice);
    RIHF_LAUNCH_CHECK();
    if (ic.launches) *ic.launches += 1;
  }
  const int smem = schwarz_smem_bytes(max_lp);
  set_smem((const void*)schwarz_kernel<32>, smem);
  RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
  schwarz_kernel<32><<<grid_for(smem), 32, smem, ic.stream>>>(prim, ic.boys, ic.counter, Q, mask, 0);
  RIHF_LAUNCH_CHECK();
  if (ic.launches) *ic.launches += 1;
}

void launch_one_electron(const IntegralCtx& ic, const DevShells& prim, int max_lp, int natoms, const int* Z,
                         const double* axyz, double* S, double* Tk, double* V) {
  // every class of this kernel is small (la, lb <= 2 for the primary sets
  // here): 8-lane task groups, four tasks per warp, each with its own slice
  const int nc = ncart(max_lp);
  const int slice = 2 * nc * nc + 3 * 64 + max_smem_eri3(max_lp, max_lp, 0, false);
  const int smem = 4 * slice * (int)sizeof(double);
  set_smem((const void*)one_electron_kernel<8>, smem);
  RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
  one_electron_kernel<8><<<grid_for(smem), 32, smem, ic.stream>>>(prim, natoms, Z, axyz, ic.boys, ic.counter, S,
                                                                  Tk, V, slice);
  RIHF_LAUNCH_CHECK();
  if (ic.launches) *ic.launches += 1;
}

}  // namespace rihf
