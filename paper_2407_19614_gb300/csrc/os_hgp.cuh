// Warp-cooperative Obara-Saika / Head-Gordon-Pople Gaussian integral machinery.
//
// One warp evaluates one primitive (or contracted) shell triple (ab|c): the 32
// lanes split each recursion level's Cartesian components, and every
// intermediate lives in the warp's slice of shared memory.  The chain is
//   Boys F_m(T) (tabulated Taylor grid, FP64)
//   -> bra vertical recurrence  [e0|00]^(m), e = 0..L          (Obara-Saika)
//   -> electron transfer       [e0|c0], c = 1..lc              (Head-Gordon-Pople)
//   -> bra horizontal recurrence (a b|c)                       (Head-Gordon-Pople)
//   -> Cartesian -> real solid harmonic (or normalised Cartesian) transform.
// The three-centre integrals (mu nu|P) of Sec. 2.1, the metric (P|Q) (b = s with
// zero exponent) and, with a point-charge ket, nuclear attraction all use it.
#pragma once
#include "common.cuh"

namespace rihf {

// Boys table: F_m(T_k) on T_k = k * kBoysStep, k = 0..kBoysN-1, m = 0..kBoysM-1.
constexpr int kBoysM = 24;
constexpr int kBoysN = 801;
constexpr double kBoysStep = 0.05;
constexpr double kBoysTmax = 40.0;
constexpr int kBoysTaylor = 7;

// Per-primitive scalar region at the head of every warp's shared-memory slice:
// Boys values F_m (24), then the recursion factors k / (2p) and k / (2q) for
// k = 0..23.  On GB300 every FP64 warp instruction occupies the SM's narrow
// FP64 pipe whatever its active-lane count, so these factors are read from
// shared memory instead of being rebuilt (int -> double, multiply) per element.
constexpr int kFmRegion = 72;
constexpr int kH2p = 24, kH2q = 48;

// Cartesian (or solid harmonic) transform per l: rows = output functions,
// cols = Cartesian components; kTrStride x kTrStride per l.
constexpr int kTrStride = 15;
constexpr int kTrL = 5;
__constant__ double c_tr_prim[kTrL * kTrStride * kTrStride];
__constant__ double c_tr_aux[kTrL * kTrStride * kTrStride];
__constant__ int c_nfunc_prim[kTrL];
__constant__ int c_nfunc_aux[kTrL];

// F_m(T) for one m, from the table by a Taylor step from the nearest grid point,
// or from the large-T closed form with upward recursion.
__device__ inline double boys_eval(int m, double T, const double* __restrict__ tab) {
  if (T < kBoysTmax) {
    int k = __double2int_rn(T * (1.0 / kBoysStep));
    double d = T - k * kBoysStep;
    const double* row = tab + (size_t)k * kBoysM + m;
    // sum_j F_{m+j}(T_k) (-d)^j / j!   (d/dT F_m = -F_{m+1})
    // 1/j as constants: an FP64 division costs a dozen FP64-pipe instructions
    const double inv_j[kBoysTaylor] = {0.0, 1.0, 0.5, 1.0 / 3.0, 0.25, 0.2, 1.0 / 6.0};
    double s = row[kBoysTaylor - 1];
#pragma unroll
    for (int j = kBoysTaylor - 1; j >= 1; --j) s = fma(-d * inv_j[j], s, row[j - 1]);
    return s;
  }
  double f = 0.5 * sqrt(3.14159265358979323846 / T);
  double e = exp(-T);
  double inv2t = 0.5 / T;
  for (int n = 0; n < m; ++n) f = ((2 * n + 1) * f - e) * inv2t;
  return f;
}

// Largest primitive exponent of shell sh of a device shell list.
template <class Shells>
__device__ inline double aux_max_exp(const Shells& b, int sh) {
  double e = b.exps[b.pstart[sh]];
  for (int k = 1; k < b.nprim[sh]; ++k) e = fmax(e, b.exps[b.pstart[sh] + k]);
  return e;
}

// Decode component k of a Cartesian shell of angular momentum l.
__host__ __device__ inline void cart_decode(int l, int k, int& lx, int& ly, int& lz) {
  int a = 0;
  while ((a + 1) * (a + 2) / 2 <= k) ++a;
  lx = l - a;
  ly = a - (k - a * (a + 1) / 2);
  lz = l - lx - ly;
}

// Per primitive-triple geometry, identical on every lane.
struct Prim3 {
  double p, q, rho;       // bra exponent sum, ket exponent, reduced exponent
  double PA[3], WP[3];    // P - A, W - P
  double AB[3];           // A - B
  double beta;            // exponent of the bra's second function
  double pref;            // prefactor of [00|00]^(m)
  double T;               // Boys argument
  double inv2p, rp;       // 1/(2p), rho/p                  (vertical recurrence)
  double inv2q, poq;      // 1/(2q), p/q                    (electron transfer)
  double bqAB[3];         // beta AB_i / q                  (electron transfer)
  double WQ[3];           // W - C                          (mirrored recursion)
};

// Shell-pair primitive data (a, b) with la >= lb, built once per geometry.
struct PairPrim {
  double p, inv_p, alpha, beta;
  double K;               // 2 pi^{5/2} c_a c_b exp(-alpha beta/p |AB|^2) / p
  double P[3], PA[3];
  double pad;
};

// Three-centre triple from the pair table and one auxiliary primitive
// (exponent ga, 1/ga, contraction coefficient cc at C): one rsqrt, no division.
__device__ inline Prim3 make_prim3_pp(const PairPrim& q, double ga, double iga, double cc, const double* C,
                                      const double* AB) {
  Prim3 t;
  t.p = q.p;
  t.q = ga;
  t.beta = q.beta;
  const double CP0 = C[0] - q.P[0], CP1 = C[1] - q.P[1], CP2 = C[2] - q.P[2];
  const double R2 = fma(CP0, CP0, fma(CP1, CP1, CP2 * CP2));
  const double r = rsqrt(q.p + ga);      // (p + gamma)^{-1/2}
  const double gi = ga * (r * r);        // gamma / (p + gamma)
  const double pi = q.p * (r * r);       // p / (p + gamma)
  t.rho = q.p * gi;
  t.rp = gi;
  t.WP[0] = gi * CP0;
  t.WP[1] = gi * CP1;
  t.WP[2] = gi * CP2;
  t.WQ[0] = -pi * CP0;
  t.WQ[1] = -pi * CP1;
  t.WQ[2] = -pi * CP2;
  t.T = t.rho * R2;
  t.pref = q.K * (cc * iga) * r;
  t.inv2p = 0.5 * q.inv_p;
  t.inv2q = 0.5 * iga;
  t.poq = q.p * iga;
  const double bq = q.beta * iga;
  for (int i = 0; i < 3; ++i) {
    t.PA[i] = q.PA[i];
    t.AB[i] = AB[i];
    t.bqAB[i] = bq * AB[i];
  }
  return t;
}

// The derived recursion factors of a triple whose p, q, rho, beta, AB are set.
__device__ inline void prim3_factors(Prim3& t) {
  t.inv2p = 0.5 / t.p;
  t.rp = t.rho / t.p;
  t.inv2q = 0.5 / t.q;
  t.poq = t.p / t.q;
  for (int i = 0; i < 3; ++i) t.bqAB[i] = t.beta / t.q * t.AB[i];
}

// Normal three-centre triple (ab|c): A(alpha), B(beta), C(gamma).
__device__ inline Prim3 make_prim3(double al, const double* A, double be, const double* B, double ga,
                                   const double* C) {
  Prim3 t;
  double p = al + be;
  t.p = p;
  t.q = ga;
  t.beta = be;
  double P[3], R2ab = 0.0, R2pq = 0.0;
  for (int i = 0; i < 3; ++i) {
    P[i] = (al * A[i] + be * B[i]) / p;
    t.AB[i] = A[i] - B[i];
    R2ab += t.AB[i] * t.AB[i];
  }
  double pq = p + ga;
  t.rho = p * ga / pq;
  for (int i = 0; i < 3; ++i) {
    double W = (p * P[i] + ga * C[i]) / pq;
    t.PA[i] = P[i] - A[i];
    t.WP[i] = W - P[i];
    t.WQ[i] = W - C[i];
    R2pq += (P[i] - C[i]) * (P[i] - C[i]);
  }
  t.T = t.rho * R2pq;
  const double two_pi_52 = 34.98683665524972;   // 2 pi^{5/2}
  t.pref = two_pi_52 / (p * ga * sqrt(pq)) * exp(-al * be / p * R2ab);
  prim3_factors(t);
  return t;
}

// Point-charge ket at C (nuclear attraction <a|1/|r-C||b>): the q -> infinity
// limit of the three-centre recurrence with a unit-charge s function at C.
__device__ inline Prim3 make_prim_point(double al, const double* A, double be, const double* B, const double* C) {
  Prim3 t;
  double p = al + be;
  t.p = p;
  t.q = 1.0;
  t.beta = be;
  t.rho = p;
  double P[3], R2ab = 0.0, R2pc = 0.0;
  for (int i = 0; i < 3; ++i) {
    P[i] = (al * A[i] + be * B[i]) / p;
    t.AB[i] = A[i] - B[i];
    R2ab += t.AB[i] * t.AB[i];
    t.PA[i] = P[i] - A[i];
    t.WP[i] = C[i] - P[i];
    R2pc += (P[i] - C[i]) * (P[i] - C[i]);
  }
  t.T = p * R2pc;
  t.pref = 6.283185307179586 / p * exp(-al * be / p * R2ab);
  t.inv2p = 0.5 / p;
  t.rp = 1.0;
  t.inv2q = 0.0;
  t.poq = 0.0;
  t.bqAB[0] = t.bqAB[1] = t.bqAB[2] = 0.0;
  t.WQ[0] = t.WQ[1] = t.WQ[2] = 0.0;
  return t;
}

// Mirrored recursion.  The transfer above moves the ket's angular momentum over
// from the bra with the factor -p/q per unit; when the bra's exponent sum is
// much larger than the ket's (a compact primary pair against a diffuse
// auxiliary d, f or g function) that factor, raised to l_c, amplifies the
// rounding of the bra recursion far beyond FP64 precision.  The same integrals
// follow, with every factor bounded by one, from the Obara-Saika recursion on
// the ket centre,
//   [0|f+1_i]^(m) = WQ_i [0|f]^(m+1) + f_i/(2q) ([0|f-1_i]^(m) - rho/q [0|f-1_i]^(m+1))
// (Q = C: a single auxiliary function), and the transfer in the other
// direction (the same relation with bra and ket exchanged),
//   [e+1_i|f] = e_i/(2p)[e-1_i|f] + f_i/(2p)[e|f-1_i] - q/p [e|f+1_i] - beta AB_i/p [e|f].
// Both reuse warp_vrr and warp_etr with the roles of the triple exchanged:
// mirror_prim3 gives the exchanged factors, EtrShape{emax, lc, lc} the levels
// (bra angular momentum 1..emax, each over the ket range its successors need).
__device__ inline Prim3 mirror_prim3(const Prim3& t) {
  Prim3 m = t;
  const double ip = 2.0 * t.inv2p, iq = 2.0 * t.inv2q;   // 1/p, 1/q
  m.p = t.q;
  m.q = t.p;
  m.rp = t.rho * iq;       // rho/q
  m.inv2p = t.inv2q;       // k/(2q): the ket recursion
  m.inv2q = t.inv2p;       // k/(2p): the transfer to the bra
  m.poq = t.q * ip;        // q/p
  for (int i = 0; i < 3; ++i) {
    m.PA[i] = 0.0;         // Q - C
    m.WP[i] = t.WQ[i];
    m.bqAB[i] = t.beta * t.AB[i] * ip;
  }
  return m;
}

// Lanes of one task group: W consecutive lanes of a warp (W = 32: the whole
// warp).  Small shell classes run W = 8 groups, four tasks per warp, so the
// narrow FP64 pipe is not spent on idle lanes.
template <int W>
__device__ inline unsigned lane_group_mask() {
  return W == 32 ? 0xffffffffu : (((1u << W) - 1u) << ((threadIdx.x & 31) / W * W));
}

// One atomic per warp claims 32 / W consecutive tasks, task first + k for the
// k-th lane group, so the groups of a warp start together on neighbouring
// tasks.  Every lane of the warp calls it, converged.
template <int W>
__device__ inline long long warp_claim(int* counter) {
  int t = 0;
  if ((threadIdx.x & 31) == 0) t = atomicAdd(counter, 32 / W);
  return __shfl_sync(0xffffffffu, t, 0);
}

// ---------------------------------------------------------------- layouts

// VRR table [e][m][k], e = 0..L, m = 0..L-e.
__device__ __host__ inline int vrr_size(int L) {
  int s = 0;
  for (int e = 0; e <= L; ++e) s += ncart(e) * (L - e + 1);
  return s;
}
__device__ inline int vrr_level_off(int L, int e) {
  int s = 0;
  for (int x = 0; x < e; ++x) s += ncart(x) * (L - x + 1);
  return s;
}

// ETR levels c = 1..lc: e in [elo(c), ehi(c)], stored [e][ke][kc].
struct EtrShape {
  int lc, emin, emax;   // final e range at level lc
  __device__ __host__ int elo(int c) const { int v = emin - (lc - c); return v < 0 ? 0 : v; }
  __device__ __host__ int ehi(int c) const { return emax + (lc - c); }
  __device__ __host__ int level_size(int c) const {
    return (cart_offset(ehi(c) + 1) - cart_offset(elo(c))) * ncart(c);
  }
  __device__ __host__ int level_off(int c) const {
    int s = 0;
    for (int x = 1; x < c; ++x) s += level_size(x);
    return s;
  }
  __device__ __host__ int total() const { return level_off(lc + 1); }
};

// Accumulator of the final level: [e in emin..emax][ke][kc].
__device__ __host__ inline int acc_size(int emin, int emax, int lc) {
  return (cart_offset(emax + 1) - cart_offset(emin)) * ncart(lc);
}

// HRR: from [e][ke][kc], e in [emin, emax], produce (a b|c) for (la, lb),
// la + lb <= emax, la >= emin.  Scratch: two levels of at most
// (cart_offset(emax+1)-cart_offset(la)) * ncart(lb) * ncart(lc).
__device__ __host__ inline int hrr_scratch(int la, int lb, int lc, int emax) {
  int lvl = 0;
  for (int b = 0; b <= lb; ++b) {
    int s = (cart_offset(la + lb - b + 1) - cart_offset(la)) * ncart(b) * ncart(lc);
    if (s > lvl) lvl = s;
  }
  (void)emax;
  return 2 * lvl;
}

// ---------------------------------------------------------------- VRR

// [e0|00]^(m) for e = 0..L, m = 0..L-e into vrr; Fm (smem, L+1) must hold the
// Boys values.  Obara-Saika:
//   [e+1_i]^(m) = PA_i [e]^(m) + WP_i [e]^(m+1) + e_i/(2p) ([e-1_i]^(m) - rho/p [e-1_i]^(m+1))
// Fm points at the warp's kFmRegion block: F_m in [0, L], and this routine
// writes the k/(2p), k/(2q) factors at kH2p, kH2q for the electron transfer.
template <int W = 32>
__device__ inline void warp_vrr(double* vrr, int L, const Prim3& t, double* Fm, int lane) {
  for (int m = lane; m <= L; m += W) {
    const double k = (double)m;
    vrr[m] = t.pref * Fm[m];
    Fm[kH2p + m] = k * t.inv2p;
    Fm[kH2q + m] = k * t.inv2q;
  }
  __syncwarp(lane_group_mask<W>());
  const double* h2p = Fm + kH2p;
  const double rp = t.rp;
  int off_m2 = 0, off_m1 = 0, off = L + 1;   // offsets of levels e-2, e-1, e
  for (int e = 1; e <= L; ++e) {
    int nc = ncart(e), nc1 = ncart(e - 1), nc2 = e >= 2 ? ncart(e - 2) : 0;
    int n = nc * (L - e + 1);
    for (int idx = lane; idx < n; idx += W) {
      int m = idx / nc, k = idx - m * nc;
      int lx, ly, lz;
      cart_decode(e, k, lx, ly, lz);
      int i = lx > 0 ? 0 : (ly > 0 ? 1 : 2);
      int c1[3] = {lx, ly, lz};
      c1[i] -= 1;
      int k1 = cart_index(e - 1, c1[0], c1[1]);
      double v = t.PA[i] * vrr[off_m1 + m * nc1 + k1] + t.WP[i] * vrr[off_m1 + (m + 1) * nc1 + k1];
      int ei = c1[i];
      if (ei > 0) {
        c1[i] -= 1;
        int k2 = cart_index(e - 2, c1[0], c1[1]);
        v = fma(h2p[ei], fma(-rp, vrr[off_m2 + (m + 1) * nc2 + k2], vrr[off_m2 + m * nc2 + k2]), v);
      }
      vrr[off + m * nc + k] = v;
    }
    off_m2 = off_m1;
    off_m1 = off;
    off += n;
    __syncwarp(lane_group_mask<W>());
  }
}

// ---------------------------------------------------------------- ETR

// Electron transfer (HGP) for a three-centre ket with one function at C:
//   [e|c'+1_i] = e_i/(2q)[e-1_i|c'] + c'_i/(2q)[e|c'-1_i] - p/q [e+1_i|c'] - beta AB_i/q [e|c']
// The final level c = lc (e in [emin, emax]) is added, times w, into acc.
// Level 0 is the m = 0 slice of the VRR table.
__device__ inline double etr_get(const double* vrr, int L, const double* etr, const EtrShape& sh, int c, int e,
                                 int ke, int kc) {
  if (c == 0) return vrr[vrr_level_off(L, e) + ke];
  int lo = sh.elo(c);
  return etr[sh.level_off(c) + (cart_offset(e) - cart_offset(lo) + ke) * ncart(c) + kc];
}

// acc[e][ke][kc] += w * level lc (level 0 is the VRR m = 0 slice).
template <int W = 32>
__device__ inline void warp_acc_level(const double* vrr, int L, const double* etr, const EtrShape& sh, double w,
                                      double* acc, int lane) {
  const int lc = sh.lc;
  int n = acc_size(sh.emin, sh.emax, lc);
  int ncc = ncart(lc);
  for (int idx = lane; idx < n; idx += W) {
    int r = idx / ncc, kc = idx - r * ncc;
    int e = sh.emin;
    while (cart_offset(e + 1) - cart_offset(sh.emin) <= r) ++e;
    int ke = r - (cart_offset(e) - cart_offset(sh.emin));
    acc[idx] += w * etr_get(vrr, L, etr, sh, lc, e, ke, kc);
  }
  __syncwarp(lane_group_mask<W>());
}

// Fm: the warp's scalar region after warp_vrr (reads the k/(2q) factors).
template <int W = 32>
__device__ inline void warp_etr(const double* vrr, int L, double* etr, const EtrShape& sh, const Prim3& t,
                                const double* Fm, int lane) {
  const int lc = sh.lc;
  const double poq = t.poq;
  const double* h2q = Fm + kH2q;
  auto get = [&](int c, int e, int ke, int kc) -> double { return etr_get(vrr, L, etr, sh, c, e, ke, kc); };
  for (int c = 1; c <= lc; ++c) {
    int lo = sh.elo(c), hi = sh.ehi(c);
    int ncc = ncart(c);
    int nrows = cart_offset(hi + 1) - cart_offset(lo);
    int n = nrows * ncc;
    double* lvl = etr + sh.level_off(c);
    for (int idx = lane; idx < n; idx += W) {
      int r = idx / ncc, kc = idx - r * ncc;
      int e = lo;
      while (cart_offset(e + 1) - cart_offset(lo) <= r) ++e;
      int ke = r - (cart_offset(e) - cart_offset(lo));
      int ex, ey, ez, cx, cy, cz;
      cart_decode(e, ke, ex, ey, ez);
      cart_decode(c, kc, cx, cy, cz);
      int i = cx > 0 ? 0 : (cy > 0 ? 1 : 2);
      int cl[3] = {cx, cy, cz};
      cl[i] -= 1;
      int kcl = cart_index(c - 1, cl[0], cl[1]);
      int eo[3] = {ex, ey, ez};
      // - p/q [e+1_i|c'] - beta AB_i / q [e|c']
      eo[i] += 1;
      double v = -poq * get(c - 1, e + 1, cart_index(e + 1, eo[0], eo[1]), kcl);
      v = fma(-t.bqAB[i], get(c - 1, e, ke, kcl), v);
      eo[i] -= 1;
      if (eo[i] > 0) {   // e_i/(2q) [e-1_i|c']
        int ei = eo[i];
        eo[i] -= 1;
        v = fma(h2q[ei], get(c - 1, e - 1, cart_index(e - 1, eo[0], eo[1]), kcl), v);
        eo[i] += 1;
      }
      if (cl[i] > 0) {   // c'_i/(2q) [e|c'-1_i]
        int ci = cl[i];
        cl[i] -= 1;
        v = fma(h2q[ci], get(c - 2, e, ke, cart_index(c - 2, cl[0], cl[1])), v);
      }
      lvl[idx] = v;
    }
    __syncwarp(lane_group_mask<W>());
  }
}

// acc[e][ke][kc] += w * [e|lc] for e in [emin, emax] from the mirrored tables of
// shape EtrShape{emax, lc, lc} (level e holds [e|f] for f around lc; level 0 is
// the m = 0 slice of the ket recursion).  Same accumulator layout as
// warp_acc_level, so everything after the transfer is shared.
// With Store the values are written (acc = w * value): a task of one primitive
// triple needs no accumulation.
template <int W = 32, bool Store = false>
__device__ inline void warp_acc_mirror(const double* vrr, int L, const double* etr, const EtrShape& shm, int emin,
                                       int emax, int lc, double w, double* acc, int lane) {
  const int ncc = ncart(lc);
  const int n = acc_size(emin, emax, lc);
  for (int idx = lane; idx < n; idx += W) {
    int r = idx / ncc, kc = idx - r * ncc;
    int e = emin;
    while (cart_offset(e + 1) - cart_offset(emin) <= r) ++e;
    int ke = r - (cart_offset(e) - cart_offset(emin));
    const double v = etr_get(vrr, L, etr, shm, e, lc, kc, ke);
    if (Store) acc[idx] = v;
    else acc[idx] += w * v;
  }
  (void)emax;
  __syncwarp(lane_group_mask<W>());
}

template <int W = 32>
__device__ inline void warp_etr_accumulate(const double* vrr, int L, double* etr, const EtrShape& sh,
                                           const Prim3& t, double w, double* acc, const double* Fm, int lane) {
  warp_etr<W>(vrr, L, etr, sh, t, Fm, lane);
  warp_acc_level<W>(vrr, L, etr, sh, w, acc, lane);
}

// ---------------------------------------------------------------- HRR

// (a, b+1_i| = (a+1_i, b| + AB_i (a, b|.  Input acc [e][ke][kc] for e in
// [emin, emax]; output out[ka][kb][kc] for (la, lb).  Returns pointer to the
// result (inside scratch or acc itself when lb == 0).
template <int W = 32>
__device__ inline const double* warp_hrr(const double* acc, int emin, int la, int lb, int lc, const double* AB,
                                         double* scratch, int half, int lane) {
  const int ncc = ncart(lc);
  if (lb == 0) return acc + (cart_offset(la) - cart_offset(emin)) * ncc;
  // level 0 is read straight from acc: rows e in [la, la+lb]
  const double* prev = acc + (cart_offset(la) - cart_offset(emin)) * ncc;
  int prev_nb = 1;   // ncart(b-1)
  double* bufs[2] = {scratch, scratch + half};
  double* cur = nullptr;
  for (int b = 1; b <= lb; ++b) {
    cur = bufs[(b - 1) & 1];
    int ahi = la + lb - b;
    int nrows = cart_offset(ahi + 1) - cart_offset(la);
    int nb = ncart(b);
    int n = nrows * nb * ncc;
    for (int idx = lane; idx < n; idx += W) {
      int kc = idx % ncc;
      int rest = idx / ncc;
      int kb = rest % nb;
      int r = rest / nb;
      int a = la;
      while (cart_offset(a + 1) - cart_offset(la) <= r) ++a;
      int ka = r - (cart_offset(a) - cart_offset(la));
      int bx, by, bz, ax, ay, az;
      cart_decode(b, kb, bx, by, bz);
      cart_decode(a, ka, ax, ay, az);
      int i = bx > 0 ? 0 : (by > 0 ? 1 : 2);
      int bl[3] = {bx, by, bz};
      bl[i] -= 1;
      int kbl = cart_index(b - 1, bl[0], bl[1]);
      int ap[3] = {ax, ay, az};
      ap[i] += 1;
      int kap = cart_index(a + 1, ap[0], ap[1]);
      // rows of prev level: a' in [la, la+lb-b+1]
      int rp = cart_offset(a + 1) - cart_offset(la) + kap;
      int r0 = cart_offset(a) - cart_offset(la) + ka;
      double v = prev[(rp * prev_nb + kbl) * ncc + kc] + AB[i] * prev[(r0 * prev_nb + kbl) * ncc + kc];
      cur[idx] = v;
    }
    __syncwarp(lane_group_mask<W>());
    prev = cur;
    prev_nb = nb;
  }
  return cur;
}

}  // namespace rihf
