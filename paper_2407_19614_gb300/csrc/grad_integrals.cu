// Fused derivative-integral contractions for the RI-HF gradient (Eq. rihf_gradient,
// Alg. 2): the derivative integrals (mu nu|P)^xi, (P|Q)^xi, S^xi, T^xi, V^xi are
// evaluated warp-cooperatively in shared memory and contracted immediately with
// Y, Z, D or W; only the per-atom 3-vectors leave the SM.
//
// Derivatives use d/dA_x [x_A^i e^{-a r_A^2}] = 2a x_A^{i+1}(..) - i x_A^{i-1}(..):
// the exponent-weighted accumulators accA (2 alpha), accB (2 beta) and the plain
// acc0 feed four horizontal recurrences, (la+1, lb), (la-1, lb), (la, lb+1),
// (la, lb-1).  The auxiliary (or nuclear) centre follows from translational
// invariance, d/dC = -(d/dA + d/dB).
#include <cmath>

#include "../../include/rihf.h"
#include "integrals.cuh"
#include "os_hgp.cuh"

namespace rihf {

template <int W = 32>
__device__ inline int warp_next(int* counter, int lane) {
  int t = 0;
  if (lane == 0) t = atomicAdd(counter, 1);
  return __shfl_sync(lane_group_mask<W>(), t, (threadIdx.x & 31) / W * W);
}

template <int W = 32>
__device__ inline double warp_sum(double v) {
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(lane_group_mask<W>(), v, o);
  return v;
}

// 8-byte asynchronous global -> shared copies (cp.async), waited for by the
// issuing thread; a group barrier then makes them visible to its other lanes.
__device__ inline void cp_async8(double* smem_dst, const double* gsrc) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gsrc) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared-memory plan of the derivative kernels.
struct DerivPlan {
  int emin, emax, L;
  int fm, vrr, etr, acc0, accA, accB, ycart, t1, t2, hrr, half, total;
  // mirror: the transfer region also holds the mirrored recursion's levels.
  // one (3-centre tasks of one primitive triple): acc0 alone -- such tasks
  // never touch accA and accB, which alias acc0 here -- and the HRR scratch
  // (with the Y back-transform's t1, t2) over the VRR table and the F_m block,
  // both dead once the primitive loop ends
  __device__ __host__ DerivPlan(int la, int lb, int lc, bool mirror = false, bool one = false) {
    emin = la > 0 ? la - 1 : 0;
    emax = la + lb + 1;
    L = emax + lc;
    EtrShape sh{lc, emin, emax};
    int accsz = acc_size(emin, emax, lc);
    int nabc = ncart(la) * ncart(lb) * ncart(lc);
    int etr_n = lc > 0 ? sh.total() : 0;
    if (mirror) {
      const int m = EtrShape{emax, lc, lc}.total();
      if (m > etr_n) etr_n = m;
    }
    half = nabc;   // the Y back-transform scratch (t1, t2) reuses the HRR region
    int cand[4] = {hrr_scratch(la + 1, lb, lc, emax), la > 0 ? hrr_scratch(la - 1, lb, lc, emax) : 0,
                   hrr_scratch(la, lb + 1, lc, emax), lb > 0 ? hrr_scratch(la, lb - 1, lc, emax) : 0};
    for (int i = 0; i < 4; ++i)
      if (cand[i] / 2 > half) half = cand[i] / 2;
    // the single-triple path's one recurrence over a in [emin, ...]: level b
    // holds (a, b) for a in [emin, la + 1 + lb - b] (b <= lb) and a = la (b = lb + 1)
    for (int b = 1; b <= lb + 1; ++b) {
      const int lo = b == lb + 1 ? la : emin, hi = b == lb + 1 ? la : la + 1 + lb - b;
      const int sz = (cart_offset(hi + 1) - cart_offset(lo)) * ncart(b) * ncart(lc);
      if (sz > half) half = sz;
    }
    fm = 0;
    vrr = kFmRegion;
    if (one) {
      hrr = 0;
      const int lo = kFmRegion + vrr_size(L), hi = 2 * half + 8;   // 8: the slack that followed the HRR region
      etr = lo > hi ? lo : hi;
      acc0 = accA = accB = etr + etr_n;
      ycart = acc0 + accsz;
      total = ycart + nabc;
    } else {
      etr = vrr + vrr_size(L);
      acc0 = etr + etr_n;
      accA = acc0 + accsz;
      accB = accA + accsz;
      ycart = accB + accsz;
      hrr = ycart + nabc;
      total = hrr + 2 * half;
    }
    t1 = hrr;
    t2 = hrr + half;
  }
};

// Strided source of warp_back_transform: element (k, a, b) at p[k sP + a sM + b sN].
struct StridedSrc {
  const double* p;
  long long sP, sM, sN;
  __device__ double operator()(int k, int a, int b) const { return p[k * sP + a * sM + b * sN]; }
};

// Ycart[ka][kb][kc] = sum tra[sa][ka] trb[sb][kb] trc[sc][kc] Y(sa, sb, sc), with
// Y(sa, sb, sc) = src(sc, sa, sb) (an accessor: strided or pair-packed).
template <int W = 32, class Src>
__device__ inline void warp_back_transform(const Src& src, int la, int lb, int lc, const double* tra,
                                           const double* trb, const double* trc, int nfa, int nfb, int nfc,
                                           double* t1, double* t2, double* out, int lane) {
  const int na = ncart(la), nb = ncart(lb), nc = ncart(lc);
  // t1[sa][sb][kc] = sum_sc trc[sc][kc] Y
  for (int idx = lane; idx < nfa * nfb * nc; idx += W) {
    int kc = idx % nc, r = idx / nc;
    int sb = r % nfb, sa = r / nfb;
    double v = 0.0;
    for (int sc = 0; sc < nfc; ++sc) v += trc[sc * kTrStride + kc] * src(sc, sa, sb);
    t1[idx] = v;
  }
  __syncwarp(lane_group_mask<W>());
  // t2[sa][kb][kc]
  for (int idx = lane; idx < nfa * nb * nc; idx += W) {
    int kc = idx % nc, r = idx / nc;
    int kb = r % nb, sa = r / nb;
    double v = 0.0;
    for (int sb = 0; sb < nfb; ++sb) v += trb[sb * kTrStride + kb] * t1[(sa * nfb + sb) * nc + kc];
    t2[idx] = v;
  }
  __syncwarp(lane_group_mask<W>());
  // out[ka][kb][kc]
  for (int idx = lane; idx < na * nb * nc; idx += W) {
    int rest = idx % (nb * nc), ka = idx / (nb * nc);
    double v = 0.0;
    for (int sa = 0; sa < nfa; ++sa) v += tra[sa * kTrStride + ka] * t2[sa * nb * nc + rest];
    out[idx] = v;
  }
  __syncwarp(lane_group_mask<W>());
}

// g[0..2] += sum_{ka,kb,kc} Y[ka][kb][kc] * (d/dA_x), g[3..5] += ... (d/dB_x) from
// the four shifted HRR products of one shell triple.  Returns per-lane partials.
// The (la+1) and (lb+1) terms come from accA and accB times sA and sB; the
// contracted triples that use it pass their three weighted sums and 1, 1
// (single primitive triples take warp_deriv_contract_single).
template <int W = 32>
__device__ inline void warp_deriv_contract(const DerivPlan& pl, double* smem, const double* acc0, const double* accA,
                                           const double* accB, double sA, double sB, int la, int lb, int lc,
                                           const double* AB, int lane, double g[6]) {
  const int na = ncart(la), nb = ncart(lb), nc = ncart(lc);
  const double* Y = smem + pl.ycart;
  double* scr = smem + pl.hrr;
  for (int i = 0; i < 6; ++i) g[i] = 0.0;
  // (la+1, lb) from accA
  {
    const double* I = warp_hrr<W>(accA, pl.emin, la + 1, lb, lc, AB, scr, pl.half, lane);
    int nap = ncart(la + 1);
    for (int idx = lane; idx < na * nb * nc; idx += W) {
      int kc = idx % nc, r = idx / nc, kb = r % nb, ka = r / nb;
      int ax, ay, az;
      cart_decode(la, ka, ax, ay, az);
      double y = Y[idx];
      int kx = cart_index(la + 1, ax + 1, ay), ky = cart_index(la + 1, ax, ay + 1), kz = cart_index(la + 1, ax, ay);
      g[0] += y * I[(kx * nb + kb) * nc + kc];
      g[1] += y * I[(ky * nb + kb) * nc + kc];
      g[2] += y * I[(kz * nb + kb) * nc + kc];
      (void)nap;
    }
    for (int i = 0; i < 3; ++i) g[i] *= sA;
    __syncwarp(lane_group_mask<W>());
  }
  if (la > 0) {
    const double* I = warp_hrr<W>(acc0, pl.emin, la - 1, lb, lc, AB, scr, pl.half, lane);
    for (int idx = lane; idx < na * nb * nc; idx += W) {
      int kc = idx % nc, r = idx / nc, kb = r % nb, ka = r / nb;
      int ax, ay, az;
      cart_decode(la, ka, ax, ay, az);
      double y = Y[idx];
      if (ax > 0) g[0] -= ax * y * I[(cart_index(la - 1, ax - 1, ay) * nb + kb) * nc + kc];
      if (ay > 0) g[1] -= ay * y * I[(cart_index(la - 1, ax, ay - 1) * nb + kb) * nc + kc];
      if (az > 0) g[2] -= az * y * I[(cart_index(la - 1, ax, ay) * nb + kb) * nc + kc];
    }
    __syncwarp(lane_group_mask<W>());
  }
  {
    const double* I = warp_hrr<W>(accB, pl.emin, la, lb + 1, lc, AB, scr, pl.half, lane);
    int nbp = ncart(lb + 1);
    for (int idx = lane; idx < na * nb * nc; idx += W) {
      int kc = idx % nc, r = idx / nc, kb = r % nb, ka = r / nb;
      int bx, by, bz;
      cart_decode(lb, kb, bx, by, bz);
      double y = Y[idx];
      g[3] += y * I[(ka * nbp + cart_index(lb + 1, bx + 1, by)) * nc + kc];
      g[4] += y * I[(ka * nbp + cart_index(lb + 1, bx, by + 1)) * nc + kc];
      g[5] += y * I[(ka * nbp + cart_index(lb + 1, bx, by)) * nc + kc];
    }
    for (int i = 3; i < 6; ++i) g[i] *= sB;
    __syncwarp(lane_group_mask<W>());
  }
  if (lb > 0) {
    const double* I = warp_hrr<W>(acc0, pl.emin, la, lb - 1, lc, AB, scr, pl.half, lane);
    int nbm = ncart(lb - 1);
    for (int idx = lane; idx < na * nb * nc; idx += W) {
      int kc = idx % nc, r = idx / nc, kb = r % nb, ka = r / nb;
      int bx, by, bz;
      cart_decode(lb, kb, bx, by, bz);
      double y = Y[idx];
      if (bx > 0) g[3] -= bx * y * I[(ka * nbm + cart_index(lb - 1, bx - 1, by)) * nc + kc];
      if (by > 0) g[4] -= by * y * I[(ka * nbm + cart_index(lb - 1, bx, by - 1)) * nc + kc];
      if (bz > 0) g[5] -= bz * y * I[(ka * nbm + cart_index(lb - 1, bx, by)) * nc + kc];
    }
    __syncwarp(lane_group_mask<W>());
  }
}

// The same contraction for a single primitive triple (one array lvl for
// all four shifted products, sA = 2 alpha, sB = 2 beta): one horizontal
// recurrence over a in [emin, la + 1 + lb - b] at level b yields (la +- 1, lb)
// at level lb, (la, lb - 1) at level lb - 1 and (la, lb + 1) at level lb + 1,
// each contracted with Y as soon as it is built, instead of four recurrences
// from the transfer level.
template <int W = 32>
__device__ inline void warp_deriv_contract_single(const DerivPlan& pl, double* smem, const double* lvl, double sA,
                                                  double sB, int la, int lb, int lc, const double* AB, int lane,
                                                  double g[6]) {
  const int na = ncart(la), nb = ncart(lb), nc = ncart(lc);
  const double* Y = smem + pl.ycart;
  double* bufs[2] = {smem + pl.hrr, smem + pl.hrr + pl.half};
  const int alo = pl.emin;
  double gp[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, gm[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  // (la +- 1, lb) from the level holding b = lb (rows a in [alo, ...], nbb columns of b)
  auto a_terms = [&](const double* I, int nbb) {
    for (int idx = lane; idx < na * nb * nc; idx += W) {
      int kc = idx % nc, r = idx / nc, kb = r % nb, ka = r / nb;
      int ax, ay, az;
      cart_decode(la, ka, ax, ay, az);
      const double y = Y[idx];
      const int rp = cart_offset(la + 1) - cart_offset(alo);
      gp[0] += y * I[((rp + cart_index(la + 1, ax + 1, ay)) * nbb + kb) * nc + kc];
      gp[1] += y * I[((rp + cart_index(la + 1, ax, ay + 1)) * nbb + kb) * nc + kc];
      gp[2] += y * I[((rp + cart_index(la + 1, ax, ay)) * nbb + kb) * nc + kc];
      if (la > 0) {
        const int rm = cart_offset(la - 1) - cart_offset(alo);
        if (ax > 0) gm[0] += ax * y * I[((rm + cart_index(la - 1, ax - 1, ay)) * nbb + kb) * nc + kc];
        if (ay > 0) gm[1] += ay * y * I[((rm + cart_index(la - 1, ax, ay - 1)) * nbb + kb) * nc + kc];
        if (az > 0) gm[2] += az * y * I[((rm + cart_index(la - 1, ax, ay)) * nbb + kb) * nc + kc];
      }
    }
  };
  // (la, lb - 1) from the level holding b = lb - 1 (rows a in [lo, ...], nbm columns)
  auto bminus_terms = [&](const double* I, int lo, int nbm) {
    const int r0 = cart_offset(la) - cart_offset(lo);
    for (int idx = lane; idx < na * nb * nc; idx += W) {
      int kc = idx % nc, r = idx / nc, kb = r % nb, ka = r / nb;
      int bx, by, bz;
      cart_decode(lb, kb, bx, by, bz);
      const double y = Y[idx];
      const double* row = I + (size_t)(r0 + ka) * nbm * nc;
      if (bx > 0) gm[3] += bx * y * row[cart_index(lb - 1, bx - 1, by) * nc + kc];
      if (by > 0) gm[4] += by * y * row[cart_index(lb - 1, bx, by - 1) * nc + kc];
      if (bz > 0) gm[5] += bz * y * row[cart_index(lb - 1, bx, by) * nc + kc];
    }
  };
  // level 0 is the transfer level itself
  if (lb == 0) a_terms(lvl, 1);
  if (lb == 1) bminus_terms(lvl, alo, 1);
  const double* prev = lvl;
  int prev_lo = alo, prev_nb = 1;
  for (int b = 1; b <= lb + 1; ++b) {
    double* cur = bufs[(b - 1) & 1];
    const int lo = b == lb + 1 ? la : alo, hi = b == lb + 1 ? la : la + 1 + lb - b;
    const int ncb = ncart(b);
    const int n = (cart_offset(hi + 1) - cart_offset(lo)) * ncb * nc;
    for (int idx = lane; idx < n; idx += W) {
      const int kc = idx % nc, rest = idx / nc;
      const int kb = rest % ncb, r = rest / ncb;
      int a = lo;
      while (cart_offset(a + 1) - cart_offset(lo) <= r) ++a;
      const int ka = r - (cart_offset(a) - cart_offset(lo));
      int bx, by, bz, ax, ay, az;
      cart_decode(b, kb, bx, by, bz);
      cart_decode(a, ka, ax, ay, az);
      const int i = bx > 0 ? 0 : (by > 0 ? 1 : 2);
      int bl[3] = {bx, by, bz};
      bl[i] -= 1;
      const int kbl = cart_index(b - 1, bl[0], bl[1]);
      int ap[3] = {ax, ay, az};
      ap[i] += 1;
      const int rp = cart_offset(a + 1) - cart_offset(prev_lo) + cart_index(a + 1, ap[0], ap[1]);
      const int r0 = cart_offset(a) - cart_offset(prev_lo) + ka;
      cur[idx] = prev[(rp * prev_nb + kbl) * nc + kc] + AB[i] * prev[(r0 * prev_nb + kbl) * nc + kc];
    }
    __syncwarp(lane_group_mask<W>());
    if (b == lb - 1) {
      bminus_terms(cur, lo, ncb);
    } else if (b == lb) {
      a_terms(cur, ncb);
    } else if (b == lb + 1) {   // (la, lb + 1): the level holds a = la only
      for (int idx = lane; idx < na * nb * nc; idx += W) {
        int kc = idx % nc, r = idx / nc, kb = r % nb, ka = r / nb;
        int bx, by, bz;
        cart_decode(lb, kb, bx, by, bz);
        const double y = Y[idx];
        const double* row = cur + (size_t)ka * ncb * nc;
        gp[3] += y * row[cart_index(lb + 1, bx + 1, by) * nc + kc];
        gp[4] += y * row[cart_index(lb + 1, bx, by + 1) * nc + kc];
        gp[5] += y * row[cart_index(lb + 1, bx, by) * nc + kc];
      }
    }
    __syncwarp(lane_group_mask<W>());
    prev = cur;
    prev_lo = lo;
    prev_nb = ncb;
  }
  for (int x = 0; x < 3; ++x) {
    g[x] = sA * gp[x] - gm[x];
    g[3 + x] = sB * gp[3 + x] - gm[3 + x];
  }
}

// ------------------------------------------------------------ 3-centre

// One task of the fused 3-centre derivative contraction: the shell triple
// (pairs[tk.x] | tk.y) (tk.y < 0: ~tk.y, mirrored for p > q), its derivative
// integrals contracted with the pair-packed Y; the per-atom sums are added
// into grad.  smem: this task group's slice.
template <int W>
__device__ inline void grad_eri3_task(const DevShells& prim, const DevShells& aux, const ShellPair* __restrict__ pairs,
                                      const PairTable& ptab, int2 tk, const double* __restrict__ boys,
                                      const double* __restrict__ Y, double* grad, double* smem, int lane) {
  const int N = prim.nfunc;
  const long long Npp = (long long)N * (N + 1) / 2;
  const bool mir = tk.y < 0;   // marked task: triples with p > q run mirrored (mirror_prim3)
  int ip = tk.x, sc = mir ? ~tk.y : tk.y;
  int sa = pairs[ip].a, sb = pairs[ip].b;
  if (prim.l[sa] < prim.l[sb]) { int t = sa; sa = sb; sb = t; }   // Y is symmetric in mu, nu
  int ata = prim.atom[sa], atb = prim.atom[sb], atc = aux.atom[sc];
  if (ata == atb && atb == atc) return;   // one-centre: derivative sums to zero
  int la = prim.l[sa], lb = prim.l[sb], lc = aux.l[sc];
  const int nab = prim.nprim[sa] * prim.nprim[sb];
  // one primitive triple: the derivative weights 2 alpha and 2 beta scale the
  // contractions instead of weighted sums; a forward triple with a ket above
  // s leaves its final values in place as the last transfer level, a
  // mirrored one stores them once into acc0 (the compact plan: no accA, accB)
  const bool one = nab == 1 && aux.nprim[sc] == 1;
  DerivPlan pl(la, lb, lc, mir, one);
  double* Fm = smem + pl.fm;
  double* vrr = smem + pl.vrr;
  double* etr = smem + pl.etr;
  int accsz = acc_size(pl.emin, pl.emax, lc);
  // the task's block of Y (auxiliary function k, then the functions a of sa
  // and b of sb; Y pair-packed per auxiliary function, symmetric) copied
  // asynchronously into the slice's Y region, which the primitive loop leaves
  // alone: the scattered loads overlap the recursion instead of stalling the
  // back-transform (the block, spherical, never exceeds the Cartesian region)
  const int nfa = prim.nf[la], nfb = prim.nf[lb], nfc = aux.nf[lc];
  double* ystage = smem + pl.ycart;
  {
    const double* Yc = Y + (long long)aux.ao[sc] * Npp;
    const long long mu0 = prim.ao[sa], nu0 = prim.ao[sb];
    for (int idx = lane; idx < nfa * nfb * nfc; idx += W) {
      const int b = idx % nfb, r = idx / nfb, a = r % nfa, k = r / nfa;
      const long long row = mu0 + a, col = nu0 + b;
      cp_async8(ystage + idx, Yc + k * Npp + (row >= col ? row * (row + 1) / 2 + col : col * (col + 1) / 2 + row));
    }
    cp_async_commit();
  }
  const PairPrim* pr = ptab.pp + ptab.off[ip];
  const bool one_mir = one && mir && pr[0].p > aux.exps[aux.pstart[sc]];
  const bool single = one && !one_mir && lc > 0;
  // one primitive triple with an s auxiliary function: its values go to acc0
  // alone (there is no transfer level to read in place), contracted like the
  // other single triples with 2 alpha and 2 beta
  const bool one_s = one && !one_mir && lc == 0;
  if (!single && !one_mir)
    for (int i = lane; i < (one_s ? 1 : 3) * accsz; i += W) smem[pl.acc0 + i] = 0.0;
  const double* A = prim.xyz + 3 * sa;
  const double* B = prim.xyz + 3 * sb;
  const double* C = aux.xyz + 3 * sc;
  EtrShape sh{lc, pl.emin, pl.emax};
  const EtrShape shm{pl.emax, lc, lc};
  const double ABv[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
  for (int ab = 0; ab < nab; ++ab) {
    const PairPrim q = pr[ab];
    for (int pc = 0; pc < aux.nprim[sc]; ++pc) {
      const int ic = aux.pstart[sc] + pc;
      Prim3 t = make_prim3_pp(q, aux.exps[ic], aux.iexps[ic], aux.coefs[ic], C, ABv);
      for (int m = lane; m <= pl.L; m += W) Fm[m] = boys_eval(m, t.T, boys);
      __syncwarp(lane_group_mask<W>());
      if (mir && t.p > t.q) {
        const Prim3 tm = mirror_prim3(t);
        warp_vrr<W>(vrr, pl.L, tm, Fm, lane);
        warp_etr<W>(vrr, pl.L, etr, shm, tm, Fm, lane);
        if (one_mir) {
          warp_acc_mirror<W, true>(vrr, pl.L, etr, shm, pl.emin, pl.emax, lc, 1.0, smem + pl.acc0, lane);
        } else {
          warp_acc_mirror<W>(vrr, pl.L, etr, shm, pl.emin, pl.emax, lc, 1.0, smem + pl.acc0, lane);
          warp_acc_mirror<W>(vrr, pl.L, etr, shm, pl.emin, pl.emax, lc, 2.0 * q.alpha, smem + pl.accA, lane);
          warp_acc_mirror<W>(vrr, pl.L, etr, shm, pl.emin, pl.emax, lc, 2.0 * q.beta, smem + pl.accB, lane);
        }
        continue;
      }
      warp_vrr<W>(vrr, pl.L, t, Fm, lane);
      warp_etr<W>(vrr, pl.L, etr, sh, t, Fm, lane);
      if (!single) {
        warp_acc_level<W>(vrr, pl.L, etr, sh, 1.0, smem + pl.acc0, lane);
        if (!one_s) {
          warp_acc_level<W>(vrr, pl.L, etr, sh, 2.0 * q.alpha, smem + pl.accA, lane);
          warp_acc_level<W>(vrr, pl.L, etr, sh, 2.0 * q.beta, smem + pl.accB, lane);
        }
      }
    }
  }
  // staged Y block -> Cartesian (its last pass overwrites the staged block)
  cp_async_wait_all();
  __syncwarp(lane_group_mask<W>());
  const StridedSrc ysrc{ystage, (long long)nfa * nfb, nfb, 1};
  warp_back_transform<W>(ysrc, la, lb, lc, prim.tr + la * kTrStride * kTrStride,
                      prim.tr + lb * kTrStride * kTrStride, aux.tr + lc * kTrStride * kTrStride, nfa, nfb, nfc,
                      smem + pl.t1, smem + pl.t2, smem + pl.ycart, lane);
  double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
  double g[6];
  if (single || one_mir || one_s) {
    const double* lvl = single ? etr + sh.level_off(lc) : smem + pl.acc0;
    warp_deriv_contract_single<W>(pl, smem, lvl, 2.0 * pr[0].alpha, 2.0 * pr[0].beta, la, lb, lc, AB, lane, g);
  } else {
    warp_deriv_contract<W>(pl, smem, smem + pl.acc0, smem + pl.accA, smem + pl.accB, 1.0, 1.0, la, lb, lc, AB,
                           lane, g);
  }
  double wgt = (sa == sb) ? 1.0 : 2.0;
  for (int i = 0; i < 6; ++i) g[i] = warp_sum<W>(g[i]) * wgt;
  if (lane == 0) {
    for (int x = 0; x < 3; ++x) {
      atomicAdd(grad + 3 * ata + x, g[x]);
      atomicAdd(grad + 3 * atb + x, g[3 + x]);
      atomicAdd(grad + 3 * atc + x, -(g[x] + g[3 + x]));
    }
  }
  __syncwarp(lane_group_mask<W>());
}

template <int W>
__global__ void __launch_bounds__(32, kGradBlocksPerSM) grad_eri3_kernel(DevShells prim, DevShells aux,
                                                       const ShellPair* __restrict__ pairs, PairTable ptab,
                                                       const int2* __restrict__ tasks, long long ntask,
                                                       const double* __restrict__ boys, int* counter,
                                                       const double* __restrict__ Y, double* grad, int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % W;
  double* smem = smem_all + (threadIdx.x / W) * slice;   // this task group's slice
  for (;;) {
    const long long task = warp_claim<W>(counter) + (threadIdx.x & 31) / W;
    if (task - (threadIdx.x & 31) / W >= ntask) break;   // the same for the whole warp
    if (task < ntask) grad_eri3_task<W>(prim, aux, pairs, ptab, tasks[task], boys, Y, grad, smem, lane);
    __syncwarp();
  }
}

// The same over a batch of geometries (task t of geometry g with off[g] <= t <
// off[g + 1]): each geometry's Y in, its per-atom gradient (out) added to.
template <int W>
__global__ void __launch_bounds__(32, kGradBlocksPerSM) grad_eri3_batch_kernel(const GeomTasks* __restrict__ geoms,
                                                             const long long* __restrict__ off, int ngeom,
                                                             const double* __restrict__ boys, int* counter,
                                                             int slice) {
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
      grad_eri3_task<W>(G.prim, G.aux, G.pairs, G.ptab, G.tasks[task - off[lo]], boys, G.Y, G.out, smem, lane);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ 2-centre

// G = 8 runs the classes set in small_mask (bit 8 la + lc), G = 32 the others.
template <int G>
__global__ void __launch_bounds__(32) grad_eri2_kernel(DevShells aux, const double* __restrict__ boys, int* counter,
                                                       const double* __restrict__ Z, double* grad,
                                                       unsigned long long small_mask, int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % G;
  double* smem = smem_all + (threadIdx.x / G) * slice;   // this task group's slice
  const unsigned gm = lane_group_mask<G>();
  __shared__ double one_tr[kTrStride];   // the unit transform of the s "b" function
  if (threadIdx.x < kTrStride) one_tr[threadIdx.x] = threadIdx.x == 0 ? 1.0 : 0.0;
  __syncwarp();
  const int ns = aux.nshell;
  const long long ntask = (long long)ns * (ns + 1) / 2;
  const int NA = aux.nfunc;
  for (;;) {
    long long task = warp_next<G>(counter, lane);
    if (task >= ntask) break;
    int sa = (int)((sqrt(8.0 * (double)task + 1.0) - 1.0) * 0.5);
    while ((long long)sa * (sa + 1) / 2 > task) --sa;
    while ((long long)(sa + 1) * (sa + 2) / 2 <= task) ++sa;
    int sc = (int)(task - (long long)sa * (sa + 1) / 2);
    if (aux.atom[sa] == aux.atom[sc]) continue;
    if ((int)((small_mask >> (8 * aux.l[sa] + aux.l[sc])) & 1ull) != (G == 8 ? 1 : 0)) continue;
    // the more diffuse shell is the bra, so the transfer's p/q factor is at
    // most one (the small-class mask is symmetric, so the launch still holds
    // the task; Z is symmetric, so the swapped block is read the same way)
    if (aux_max_exp(aux, sa) > aux_max_exp(aux, sc)) { int t = sa; sa = sc; sc = t; }
    int ata = aux.atom[sa], atc = aux.atom[sc];
    int la = aux.l[sa], lc = aux.l[sc];
    DerivPlan pl(la, 0, lc);
    double* Fm = smem + pl.fm;
    double* vrr = smem + pl.vrr;
    double* etr = smem + pl.etr;
    int accsz = acc_size(pl.emin, pl.emax, lc);
    for (int i = lane; i < 3 * accsz; i += G) smem[pl.acc0 + i] = 0.0;
    const double* PA = aux.xyz + 3 * sa;
    const double* PC = aux.xyz + 3 * sc;
    EtrShape sh{lc, pl.emin, pl.emax};
    for (int pa = 0; pa < aux.nprim[sa]; ++pa)
      for (int pc = 0; pc < aux.nprim[sc]; ++pc) {
        double al = aux.exps[aux.pstart[sa] + pa], ga = aux.exps[aux.pstart[sc] + pc];
        double w = aux.coefs[aux.pstart[sa] + pa] * aux.coefs[aux.pstart[sc] + pc];
        Prim3 t = make_prim3(al, PA, 0.0, PA, ga, PC);
        for (int m = lane; m <= pl.L; m += G) Fm[m] = boys_eval(m, t.T, boys);
        __syncwarp(gm);
        warp_vrr<G>(vrr, pl.L, t, Fm, lane);
        warp_etr<G>(vrr, pl.L, etr, sh, t, Fm, lane);
        warp_acc_level<G>(vrr, pl.L, etr, sh, w, smem + pl.acc0, lane);
        warp_acc_level<G>(vrr, pl.L, etr, sh, 2.0 * al * w, smem + pl.accA, lane);
      }
    // Z block (P in sa, Q in sc) -> Cartesian with a unit s "b" function
    int nfa = aux.nf[la], nfc = aux.nf[lc];
    const double* zsrc = Z + (long long)aux.ao[sa] * NA + aux.ao[sc];
    // layout Y(sa, sb=0, sc) = Z[P0 + sa][Q0 + sc]
    auto src = [&](int k, int a, int b) -> double { return zsrc[(long long)a * NA + k + 0 * b]; };
    warp_back_transform<G>(src, la, 0, lc, aux.tr + la * kTrStride * kTrStride, one_tr,
                        aux.tr + lc * kTrStride * kTrStride, nfa, 1, nfc, smem + pl.t1, smem + pl.t2,
                        smem + pl.ycart, lane);
    double AB[3] = {0.0, 0.0, 0.0};
    double g[6];
    // only the A-side derivative is needed (lb = 0, beta = 0): zero accB so the
    // (la, lb+1) term vanishes
    for (int i = lane; i < accsz; i += G) smem[pl.accB + i] = 0.0;
    __syncwarp(gm);
    warp_deriv_contract<G>(pl, smem, smem + pl.acc0, smem + pl.accA, smem + pl.accB, 1.0, 1.0, la, 0, lc, AB, lane, g);
    // E term -1/2 sum_PQ Z_PQ (P|Q)^xi over ordered pairs: off-diagonal shell
    // pairs appear twice.
    double wgt = (sa == sc) ? -0.5 : -1.0;
    for (int i = 0; i < 3; ++i) g[i] = warp_sum<G>(g[i]) * wgt;
    if (lane == 0) {
      for (int x = 0; x < 3; ++x) {
        atomicAdd(grad + 3 * ata + x, g[x]);
        atomicAdd(grad + 3 * atc + x, -g[x]);
      }
    }
    __syncwarp(gm);
  }
}

// ------------------------------------------------------------ one-electron

__device__ inline void os_overlap_1d_g(double a, double b, double XA, double XB, int imax, int jmax, double* s,
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

// 1D overlap and kinetic factors for exponents (i, j) from the table s (ld 8).
__device__ inline double k1d(const double* s, int i, int j, double b) {
  if (i < 0) return 0.0;
  double v = 4.0 * b * b * s[i * 8 + j + 2] - 2.0 * b * (2 * j + 1) * s[i * 8 + j];
  if (j >= 2) v += j * (j - 1) * s[i * 8 + j - 2];
  return v;
}
__device__ inline double s1(const double* s, int i, int j) { return (i < 0 || j < 0) ? 0.0 : s[i * 8 + j]; }

// Task = primary shell pair (a >= b) x (1 + natoms): slot 0 handles overlap and
// kinetic, slot 1 + C the attraction of nucleus C.
template <int G>
__global__ void __launch_bounds__(32) grad_one_electron_kernel(DevShells prim, int natoms, const int* __restrict__ Z,
                                                               const double* __restrict__ axyz,
                                                               const double* __restrict__ boys, int* counter,
                                                               const double* __restrict__ D,
                                                               const double* __restrict__ W, double* grad_one,
                                                               double* grad_ovl, int slice) {
  extern __shared__ double smem_all[];
  const int lane = threadIdx.x % G;
  double* smem = smem_all + (threadIdx.x / G) * slice;   // this task group's slice
  __shared__ double one_tr[kTrStride];   // the unit transform of the s "c" function
  if (threadIdx.x < kTrStride) one_tr[threadIdx.x] = threadIdx.x == 0 ? 1.0 : 0.0;
  __syncwarp();
  const int ns = prim.nshell;
  const long long npair = (long long)ns * (ns + 1) / 2;
  const long long ntask = npair * (1 + natoms);
  const int N = prim.nfunc;
  for (;;) {
    long long task = warp_next<G>(counter, lane);
    if (task >= ntask) break;
    long long pidx = task % npair;
    int slot = (int)(task / npair);
    int sa = (int)((sqrt(8.0 * (double)pidx + 1.0) - 1.0) * 0.5);
    while ((long long)sa * (sa + 1) / 2 > pidx) --sa;
    while ((long long)(sa + 1) * (sa + 2) / 2 <= pidx) ++sa;
    int sb = (int)(pidx - (long long)sa * (sa + 1) / 2);
    int la = prim.l[sa], lb = prim.l[sb];
    int ata = prim.atom[sa], atb = prim.atom[sb];
    const double* A = prim.xyz + 3 * sa;
    const double* B = prim.xyz + 3 * sb;
    int nfa = prim.nf[la], nfb = prim.nf[lb];
    const double* tra = prim.tr + la * kTrStride * kTrStride;
    const double* trb = prim.tr + lb * kTrStride * kTrStride;
    double wgt = (sa == sb) ? 1.0 : 2.0;
    DerivPlan pl(la, lb, 0);
    const int na = ncart(la), nb = ncart(lb);
    if (slot == 0) {
      if (ata == atb) continue;   // overlap and kinetic depend on A - B only
      // Dcart (for T) into ycart, Wcart into t1-region copy
      double* Dc = smem + pl.ycart;
      double* Wc = smem + pl.total;   // past the plan (the HRR region holds t1/t2)
      double* s1d = Wc + 128;         // 3 x 64
      warp_back_transform<G>(StridedSrc{D + (long long)prim.ao[sa] * N + prim.ao[sb], 0, N, 1}, la, lb, 0, tra, trb, one_tr, nfa,
                          nfb, 1, smem + pl.t1, smem + pl.t2, Dc, lane);
      warp_back_transform<G>(StridedSrc{W + (long long)prim.ao[sa] * N + prim.ao[sb], 0, N, 1}, la, lb, 0, tra, trb, one_tr, nfa,
                          nfb, 1, smem + pl.t1, smem + pl.t2, Wc, lane);
      double gT[3] = {0, 0, 0}, gS[3] = {0, 0, 0};
      for (int pa = 0; pa < prim.nprim[sa]; ++pa)
        for (int pb = 0; pb < prim.nprim[sb]; ++pb) {
          double al = prim.exps[prim.pstart[sa] + pa], be = prim.exps[prim.pstart[sb] + pb];
          double w = prim.coefs[prim.pstart[sa] + pa] * prim.coefs[prim.pstart[sb] + pb];
          if (lane < 3) os_overlap_1d_g(al, be, A[lane], B[lane], la + 1, lb + 2, s1d + lane * 64, 8);
          __syncwarp(lane_group_mask<G>());
          for (int idx = lane; idx < na * nb; idx += G) {
            int ka = idx / nb, kb = idx % nb;
            int c[3], d[3];
            cart_decode(la, ka, c[0], c[1], c[2]);
            cart_decode(lb, kb, d[0], d[1], d[2]);
            const double* sx[3] = {s1d, s1d + 64, s1d + 128};
            double S0[3], K0[3];
            for (int q = 0; q < 3; ++q) {
              S0[q] = s1(sx[q], c[q], d[q]);
              K0[q] = k1d(sx[q], c[q], d[q], be);
            }
            for (int x = 0; x < 3; ++x) {
              // d/dA_x of the 1D factors along x
              double dS = 2.0 * al * s1(sx[x], c[x] + 1, d[x]) - (c[x] > 0 ? c[x] * s1(sx[x], c[x] - 1, d[x]) : 0.0);
              double dK = 2.0 * al * k1d(sx[x], c[x] + 1, d[x], be) -
                          (c[x] > 0 ? c[x] * k1d(sx[x], c[x] - 1, d[x], be) : 0.0);
              int y = (x + 1) % 3, z = (x + 2) % 3;
              double dSfull = dS * S0[y] * S0[z];
              double dTfull = -0.5 * (dK * S0[y] * S0[z] + dS * K0[y] * S0[z] + dS * S0[y] * K0[z]);
              gS[x] += w * Wc[idx] * dSfull;
              gT[x] += w * Dc[idx] * dTfull;
            }
          }
          __syncwarp(lane_group_mask<G>());
        }
      for (int x = 0; x < 3; ++x) {
        double t = warp_sum<G>(gT[x]) * wgt, s = warp_sum<G>(gS[x]) * wgt;
        if (lane == 0) {
          atomicAdd(grad_one + 3 * ata + x, t);
          atomicAdd(grad_one + 3 * atb + x, -t);
          atomicAdd(grad_ovl + 3 * ata + x, -s);
          atomicAdd(grad_ovl + 3 * atb + x, s);
        }
      }
      __syncwarp(lane_group_mask<G>());
      continue;
    }
    // nuclear attraction of nucleus C = slot - 1
    int Cn = slot - 1;
    const double* Cx = axyz + 3 * Cn;
    if (ata == atb && atb == Cn) continue;
    double* Fm = smem + pl.fm;
    double* vrr = smem + pl.vrr;
    int accsz = acc_size(pl.emin, pl.emax, 0);
    for (int i = lane; i < 3 * accsz; i += G) smem[pl.acc0 + i] = 0.0;
    EtrShape sh{0, pl.emin, pl.emax};
    for (int pa = 0; pa < prim.nprim[sa]; ++pa)
      for (int pb = 0; pb < prim.nprim[sb]; ++pb) {
        double al = prim.exps[prim.pstart[sa] + pa], be = prim.exps[prim.pstart[sb] + pb];
        double w = -Z[Cn] * prim.coefs[prim.pstart[sa] + pa] * prim.coefs[prim.pstart[sb] + pb];
        Prim3 t = make_prim_point(al, A, be, B, Cx);
        for (int m = lane; m <= pl.L; m += G) Fm[m] = boys_eval(m, t.T, boys);
        __syncwarp(lane_group_mask<G>());
        warp_vrr<G>(vrr, pl.L, t, Fm, lane);
        warp_acc_level<G>(vrr, pl.L, nullptr, sh, w, smem + pl.acc0, lane);
        warp_acc_level<G>(vrr, pl.L, nullptr, sh, 2.0 * al * w, smem + pl.accA, lane);
        warp_acc_level<G>(vrr, pl.L, nullptr, sh, 2.0 * be * w, smem + pl.accB, lane);
      }
    warp_back_transform<G>(StridedSrc{D + (long long)prim.ao[sa] * N + prim.ao[sb], 0, N, 1}, la, lb, 0, tra, trb, one_tr, nfa, nfb,
                        1, smem + pl.t1, smem + pl.t2, smem + pl.ycart, lane);
    double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
    double g[6];
    warp_deriv_contract<G>(pl, smem, smem + pl.acc0, smem + pl.accA, smem + pl.accB, 1.0, 1.0, la, lb, 0, AB, lane, g);
    for (int i = 0; i < 6; ++i) g[i] = warp_sum<G>(g[i]) * wgt;
    if (lane == 0) {
      for (int x = 0; x < 3; ++x) {
        atomicAdd(grad_one + 3 * ata + x, g[x]);
        atomicAdd(grad_one + 3 * atb + x, g[3 + x]);
        atomicAdd(grad_one + 3 * Cn + x, -(g[x] + g[3 + x]));
      }
    }
    __syncwarp(lane_group_mask<G>());
  }
}

// ------------------------------------------------------------ launchers

static int grid_for_smem(int smem_bytes) {
  int dev = 0, sms = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  int per_sm = maxsm / (smem_bytes + 1024);
  if (per_sm > 32) per_sm = 32;
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

static int deriv_smem(int max_la, int max_lb, int max_lc) {
  int best = 0;
  for (int la = 0; la <= max_la; ++la)
    for (int lb = 0; lb <= max_lb; ++lb)
      for (int lc = 0; lc <= max_lc; ++lc) {
        DerivPlan p(la, lb, lc);
        if (p.total > best) best = p.total;
      }
  return (best + 8) * (int)sizeof(double);
}

int smem_grad_doubles(int la, int lb, int lc, bool mirror, bool one) {
  DerivPlan p(la, lb, lc, mirror, one);
  return p.total + 8;
}

void launch_grad_eri3(const IntegralCtx& ic, const DevShells& prim, const DevShells& aux, const ShellPair* pairs,
                      const PairTable& pt, const TaskGroup* groups, int ngroups, const double* Y, double* grad) {
  for (int g = 0; g < ngroups; ++g) {
    if (groups[g].ntask == 0) continue;
    const int W = groups[g].width, slice = groups[g].smem_grad / (int)sizeof(double);
    const int smem = (32 / W) * slice * (int)sizeof(double);
    RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
    auto run = [&](auto kernel) {
      raise_smem_limit((const void*)kernel, smem);
      kernel<<<grid_for_smem(smem), 32, smem, ic.stream>>>(prim, aux, pairs, pt, groups[g].tasks, groups[g].ntask,
                                                           ic.boys, ic.counter, Y, grad, slice);
    };
    if (W == 8) run(grad_eri3_kernel<8>);
    else if (W == 16) run(grad_eri3_kernel<16>);
    else run(grad_eri3_kernel<32>);
    RIHF_LAUNCH_CHECK();
    if (ic.launches) *ic.launches += 1;
  }
}

void launch_grad_eri3_batch(const IntegralCtx& ic, const std::vector<BatchGeom>& batch, int ngroups,
                            BatchTables& t) {
  const int n = (int)batch.size();
  if (n == 0) return;
  if (n > t.cap) throw RihfError(RIHF_ERR_INVALID_ARG, "launch_grad_eri3_batch: batch tables too small");
  for (int g = 0; g < ngroups; ++g) {
    int slice_bytes = 0;
    long long ntask = 0;
    if (!batch_tables(ic, batch, g, t, true, slice_bytes, ntask)) continue;
    GeomTasks* dg = t.geoms + (size_t)g * t.cap;
    long long* doff = t.off + (size_t)g * (t.cap + 1);
    const int W = task_group_width(g), slice = slice_bytes / (int)sizeof(double);
    const int smem = (32 / W) * slice * (int)sizeof(double);
    RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
    auto run = [&](auto kernel) {
      raise_smem_limit((const void*)kernel, smem);
      kernel<<<grid_for_smem(smem), 32, smem, ic.stream>>>(dg, doff, n, ic.boys, ic.counter, slice);
    };
    if (W == 8) run(grad_eri3_batch_kernel<8>);
    else if (W == 16) run(grad_eri3_batch_kernel<16>);
    else run(grad_eri3_batch_kernel<32>);
    RIHF_LAUNCH_CHECK();
    if (ic.launches) *ic.launches += 1;
  }
}

void launch_grad_eri2(const IntegralCtx& ic, const DevShells& aux, int max_la, const double* Z, double* grad) {
  // small classes as 8-lane groups (four tasks per warp), then the rest with
  // whole warps; each launch claims every task and skips the other's classes
  int small_slice = 0;
  const unsigned long long mask = eri2_small_classes(max_la, &small_slice);
  if (mask) {
    const int smem = 4 * small_slice * (int)sizeof(double);
    raise_smem_limit((const void*)grad_eri2_kernel<8>, smem);
    RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
    grad_eri2_kernel<8><<<grid_for_smem(smem), 32, smem, ic.stream>>>(aux, ic.boys, ic.counter, Z, grad, mask,
                                                                      small_slice);
    RIHF_LAUNCH_CHECK();
    if (ic.launches) *ic.launches += 1;
  }
  const int smem = deriv_smem(max_la, 0, max_la);
  raise_smem_limit((const void*)grad_eri2_kernel<32>, smem);
  RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
  grad_eri2_kernel<32><<<grid_for_smem(smem), 32, smem, ic.stream>>>(aux, ic.boys, ic.counter, Z, grad, mask, 0);
  RIHF_LAUNCH_CHECK();
  if (ic.launches) *ic.launches += 1;
}

void launch_grad_one_electron(const IntegralCtx& ic, const DevShells& prim, int max_lp, int natoms, const int* Z,
                              const double* axyz, const double* D, const double* W, double* grad_one,
                              double* grad_ovl) {
  // every class of this kernel is small (la, lb <= 2 for the primary sets
  // here): 8-lane task groups, four tasks per warp, each with its own slice
  const int bytes = deriv_smem(max_lp, max_lp, 0) + (128 + 3 * 64) * (int)sizeof(double);
  const int slice = (bytes + (int)sizeof(double) - 1) / (int)sizeof(double);
  const int smem = 4 * slice * (int)sizeof(double);
  raise_smem_limit((const void*)grad_one_electron_kernel<8>, smem);
  RIHF_CUDA(cudaMemsetAsync(ic.counter, 0, sizeof(int), ic.stream));
  grad_one_electron_kernel<8><<<grid_for_smem(smem), 32, smem, ic.stream>>>(prim, natoms, Z, axyz, ic.boys,
                                                                            ic.counter, D, W, grad_one, grad_ovl,
                                                                            slice);
  RIHF_LAUNCH_CHECK();
  if (ic.launches) *ic.launches += 1;
}

}  // namespace rihf
