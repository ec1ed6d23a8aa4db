/*
 * oracle/md_integrals.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow FP64 (long double where cheap) Gaussian integrals by the
 * McMurchie-Davidson Hermite scheme.  Only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark load this file; the product library never
 * does, and this file shares no code with it.
 *
 * Quantities (chemists' notation, Sec. 2.1 of the paper):
 *   S_ab, T_ab = -1/2 <a|lap|b>, V_ab(C) = <a|1/|r-C||b>,
 *   (P|Q), (ab|P), (ab|cd)  -- Eqs. for the 2-, 3- and 4-centre ERIs,
 * and first derivatives of S, T, V, (P|Q), (ab|P) with respect to one atomic
 * coordinate (Eq. hf_gradient / rihf_gradient need S^xi, h^xi, A^xi, (mu nu|P)^xi).
 *
 * Basis functions are contracted Cartesian monomials
 *     phi(r) = sum_k d_k (x-Ax)^i (y-Ay)^j (z-Az)^k exp(-a_k |r-A|^2)
 * with the d_k supplied by the caller (the caller owns normalisation).
 * Derivatives use d/dAx [x_A^i e^{-a x_A^2}] = 2a x_A^{i+1} e - i x_A^{i-1} e.
 *
 * Hermite coefficients E^{ij}_t and Hermite Coulomb integrals R_{tuv} follow the
 * textbook recurrences (Helgaker, Joergensen, Olsen, Molecular Electronic-
 * Structure Theory, ch. 9).  The Boys function is summed as its power series in
 * long double for T < 40 and from erf plus upward recursion above.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LE 9                 /* max 1D index in E tables                      */
#define LT (2 * LE + 1)      /* max Hermite index t                           */
#define LRMAX 20             /* max total Hermite order in R tables           */

/* ------------------------------------------------------------------ Boys */

static long double boys_series(int n, long double T) {
  long double term = 1.0L / (2 * n + 1), sum = term;
  for (int k = 1; k < 2000; ++k) {
    term *= 2.0L * T / (2 * n + 2 * k + 1);
    sum += term;
    if (term < 1e-24L * sum) break;
  }
  return expl(-T) * sum;
}

/* F_0..F_nmax at T: series for the top order then downward recursion for T < 40,
   erf and upward recursion for T >= 40 (both directions are stable there). */
static void boys_all(int nmax, long double T, long double* F) {
  if (T < 40.0L) {
    F[nmax] = boys_series(nmax, T);
    long double e = expl(-T);
    for (int n = nmax - 1; n >= 0; --n) F[n] = (2.0L * T * F[n + 1] + e) / (2 * n + 1);
  } else {
    long double e = expl(-T), st = sqrtl(T);
    F[0] = 0.5L * sqrtl(3.14159265358979323846264338327950288L / T) * erfl(st);
    for (int n = 0; n < nmax; ++n) F[n + 1] = ((2 * n + 1) * F[n] - e) / (2.0L * T);
  }
}

double oracle_boys(int n, double T) {
  long double F[64];
  if (n < 0 || n > 60) return NAN;
  boys_all(n, (long double)T, F);
  return (double)F[n];
}

/* ------------------------------------------------------- Hermite tables */

typedef struct {
  double p, P[3];
  double E[3][LE + 1][LE + 1][LT + 1];   /* E[dim][i][j][t] */
  int imax, jmax;
} hpair;

/* E^{ij}_t for the product of x_A^i e^{-a x_A^2} and x_B^j e^{-b x_B^2}. */
static void hpair_init(hpair* h, double a, const double* A, double b, const double* B, int imax, int jmax) {
  double p = a + b;
  h->p = p; h->imax = imax; h->jmax = jmax;
  memset(h->E, 0, sizeof(h->E));
  for (int d = 0; d < 3; ++d) {
    double Pd = (a * A[d] + b * B[d]) / p;
    h->P[d] = Pd;
    double XAB = A[d] - B[d], XPA = Pd - A[d], XPB = Pd - B[d];
    double (*E)[LE + 1][LT + 1] = h->E[d];
    E[0][0][0] = exp(-(a * b / p) * XAB * XAB);
    for (int i = 0; i <= imax; ++i) {
      if (i > 0) {
        for (int t = 0; t <= i; ++t) {
          double v = XPA * E[i - 1][0][t];
          if (t > 0) v += E[i - 1][0][t - 1] / (2 * p);
          if (t + 1 <= i - 1) v += (t + 1) * E[i - 1][0][t + 1];
          E[i][0][t] = v;
        }
      }
      for (int j = 1; j <= jmax; ++j) {
        for (int t = 0; t <= i + j; ++t) {
          double v = XPB * E[i][j - 1][t];
          if (t > 0) v += E[i][j - 1][t - 1] / (2 * p);
          if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
          E[i][j][t] = v;
        }
      }
    }
  }
}

/* R_{tuv}(alpha, PC) for t+u+v <= L, n = 0, stored R[(t*D+u)*D+v], D = L+1.
   scratch must hold (L+1)^4 doubles. */
static void hermite_R(int L, double alpha, const double* PC, double* scratch, double* R) {
  int D = L + 1;
#define RI(n, t, u, v) ((((n) * D + (t)) * D + (u)) * D + (v))
  long double F[LRMAX + 2];
  double T = alpha * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
  boys_all(L, (long double)T, F);
  double f = 1.0;
  for (int n = 0; n <= L; ++n) {
    scratch[RI(n, 0, 0, 0)] = f * (double)F[n];
    f *= -2.0 * alpha;
  }
  for (int s = 1; s <= L; ++s)
    for (int n = 0; n + s <= L; ++n)
      for (int t = 0; t <= s; ++t)
        for (int u = 0; u + t <= s; ++u) {
          int v = s - t - u;
          double val;
          if (t > 0) {
            val = PC[0] * scratch[RI(n + 1, t - 1, u, v)];
            if (t > 1) val += (t - 1) * scratch[RI(n + 1, t - 2, u, v)];
          } else if (u > 0) {
            val = PC[1] * scratch[RI(n + 1, t, u - 1, v)];
            if (u > 1) val += (u - 1) * scratch[RI(n + 1, t, u - 2, v)];
          } else {
            val = PC[2] * scratch[RI(n + 1, t, u, v - 1)];
            if (v > 1) val += (v - 1) * scratch[RI(n + 1, t, u, v - 2)];
          }
          scratch[RI(n, t, u, v)] = val;
        }
  for (int t = 0; t <= L; ++t)
    for (int u = 0; u + t <= L; ++u)
      for (int v = 0; v + u + t <= L; ++v) R[(t * D + u) * D + v] = scratch[RI(0, t, u, v)];
#undef RI
}

/* ------------------------------------------------------- basis helpers */

typedef struct {
  int nshell;
  const int* l;          /* angular momentum per shell                      */
  const int* atom;       /* atom index per shell                            */
  const double* xyz;     /* shell centre, 3 per shell                       */
  const int* nprim;      /* primitives per shell                            */
  const int* pstart;     /* first primitive of each shell                   */
  const double* exps;    /* primitive exponents                             */
  const double* coefs;   /* primitive coefficients (caller-normalised)      */
  int* off;              /* Cartesian offset per shell (filled here)        */
  int ncart;
} basis_t;

static int ncart_of(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian components in the order lx = l..0, ly = l-lx..0, lz = l-lx-ly. */
static void cart_comp(int l, int idx, int* c) {
  int n = 0;
  for (int lx = l; lx >= 0; --lx)
    for (int ly = l - lx; ly >= 0; --ly) {
      if (n == idx) { c[0] = lx; c[1] = ly; c[2] = l - lx - ly; return; }
      ++n;
    }
}

static void basis_setup(basis_t* b) {
  int o = 0;
  for (int s = 0; s < b->nshell; ++s) { b->off[s] = o; o += ncart_of(b->l[s]); }
  b->ncart = o;
}

#define MAKE_BASIS(name, ns, l_, at_, xyz_, np_, ps_, ex_, cf_)                                  \
  basis_t name = {ns, l_, at_, xyz_, np_, ps_, ex_, cf_, (int*)malloc(sizeof(int) * ((ns) + 1)), 0}; \
  basis_setup(&name)

/* --------------------------------------------------- one-electron pieces */

/* 1D overlap of x_A^i e^{-a..} x_B^j e^{-b..} without the (pi/p)^(1/2) factor. */
static double s1d(const hpair* h, int d, int i, int j) {
  if (i < 0 || j < 0) return 0.0;
  return h->E[d][i][j][0];
}

/* 1D second-derivative matrix element <i| d^2/dx^2 |j> / sqrt(pi/p). */
static double k1d(const hpair* h, int d, int i, int j, double b) {
  double v = 4.0 * b * b * s1d(h, d, i, j + 2) - 2.0 * b * (2 * j + 1) * s1d(h, d, i, j);
  if (j >= 2) v += j * (j - 1) * s1d(h, d, i, j - 2);
  return v;
}

static double prim_overlap(const hpair* h, const int* ci, const int* cj) {
  if (ci[0] < 0 || ci[1] < 0 || ci[2] < 0 || cj[0] < 0 || cj[1] < 0 || cj[2] < 0) return 0.0;
  double f = pow(M_PI / h->p, 1.5);
  return f * s1d(h, 0, ci[0], cj[0]) * s1d(h, 1, ci[1], cj[1]) * s1d(h, 2, ci[2], cj[2]);
}

static double prim_kinetic(const hpair* h, const int* ci, const int* cj, double b) {
  if (ci[0] < 0 || ci[1] < 0 || ci[2] < 0 || cj[0] < 0 || cj[1] < 0 || cj[2] < 0) return 0.0;
  double f = pow(M_PI / h->p, 1.5);
  double sx = s1d(h, 0, ci[0], cj[0]), sy = s1d(h, 1, ci[1], cj[1]), sz = s1d(h, 2, ci[2], cj[2]);
  double kx = k1d(h, 0, ci[0], cj[0], b), ky = k1d(h, 1, ci[1], cj[1], b), kz = k1d(h, 2, ci[2], cj[2], b);
  return -0.5 * f * (kx * sy * sz + sx * ky * sz + sx * sy * kz);
}

/* <i|1/|r-C||j> = 2 pi / p sum_tuv E_t E_u E_v R_{t+ex,u+ey,v+ez}(p, P-C); (ex,ey,ez)
   shifts the Hermite index, which gives -d/dC of the operator (d/dC_x R_tuv = -R_{t+1,u,v}). */
static double prim_nuclear(const hpair* h, const int* ci, const int* cj, const double* R, int D, const int* sh) {
  if (ci[0] < 0 || ci[1] < 0 || ci[2] < 0 || cj[0] < 0 || cj[1] < 0 || cj[2] < 0) return 0.0;
  double s = 0.0;
  for (int t = 0; t <= ci[0] + cj[0]; ++t) {
    double et = h->E[0][ci[0]][cj[0]][t];
    if (et == 0.0) continue;
    for (int u = 0; u <= ci[1] + cj[1]; ++u) {
      double eu = h->E[1][ci[1]][cj[1]][u];
      if (eu == 0.0) continue;
      for (int v = 0; v <= ci[2] + cj[2]; ++v)
        s += et * eu * h->E[2][ci[2]][cj[2]][v] * R[((t + sh[0]) * D + (u + sh[1])) * D + (v + sh[2])];
    }
  }
  return 2.0 * M_PI / h->p * s;
}

/* ------------------------------------------------------- two-electron */

/* (ij|kl) over primitives from Hermite tables of the bra pair h1 and ket pair h2:
   2 pi^{5/2}/(p q sqrt(p+q)) sum E^{ij}_{tuv} (-1)^{tau+nu+phi} E^{kl}_{tau nu phi} R_{t+tau,...}. */
static double prim_eri(const hpair* h1, const int* ci, const int* cj, const hpair* h2, const int* ck,
                       const int* cl, const double* R, int D) {
  for (int d = 0; d < 3; ++d)
    if (ci[d] < 0 || cj[d] < 0 || ck[d] < 0 || cl[d] < 0) return 0.0;
  double s = 0.0;
  for (int t = 0; t <= ci[0] + cj[0]; ++t) {
    double e1t = h1->E[0][ci[0]][cj[0]][t];
    if (e1t == 0.0) continue;
    for (int u = 0; u <= ci[1] + cj[1]; ++u) {
      double e1u = h1->E[1][ci[1]][cj[1]][u];
      if (e1u == 0.0) continue;
      for (int v = 0; v <= ci[2] + cj[2]; ++v) {
        double e1 = e1t * e1u * h1->E[2][ci[2]][cj[2]][v];
        if (e1 == 0.0) continue;
        for (int tau = 0; tau <= ck[0] + cl[0]; ++tau) {
          double e2t = h2->E[0][ck[0]][cl[0]][tau];
          if (e2t == 0.0) continue;
          for (int nu = 0; nu <= ck[1] + cl[1]; ++nu) {
            double e2u = h2->E[1][ck[1]][cl[1]][nu];
            if (e2u == 0.0) continue;
            for (int phi = 0; phi <= ck[2] + cl[2]; ++phi) {
              double e2 = e2t * e2u * h2->E[2][ck[2]][cl[2]][phi];
              double sg = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
              s += e1 * sg * e2 * R[((t + tau) * D + (u + nu)) * D + (v + phi)];
            }
          }
        }
      }
    }
  }
  double p = h1->p, q = h2->p;
  return 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * s;
}

/* ------------------------------------------------ derivative bookkeeping */

/* Value of a primitive integral after differentiating the function with
   Cartesian exponents c (exponent a) along dim: 2a I(c+1) - c_d I(c-1).
   'eval' closes over the other functions. */
typedef double (*eval_fn)(const int* c, void* ctx);

static double deriv_combo(const int* c, int dim, double a, eval_fn f, void* ctx) {
  int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
  cp[dim] += 1;
  cm[dim] -= 1;
  double v = 2.0 * a * f(cp, ctx);
  if (c[dim] > 0) v -= c[dim] * f(cm, ctx);
  return v;
}

/* ------------------------------------------------ public: one-electron */

typedef struct {
  const hpair* h; const int* other; int which; double b; int kind;
  const double* R; int D; const int* sh;
} ctx1;

static double ev1(const int* c, void* vp) {
  ctx1* x = (ctx1*)vp;
  const int* ci = x->which == 0 ? c : x->other;
  const int* cj = x->which == 0 ? x->other : c;
  if (x->kind == 0) return prim_overlap(x->h, ci, cj);
  if (x->kind == 1) return prim_kinetic(x->h, ci, cj, x->b);
  return prim_nuclear(x->h, ci, cj, x->R, x->D, x->sh);
}

/*
 * kind: 0 overlap, 1 kinetic, 2 nuclear attraction sum_C -Z_C <a|1/r_C|b>.
 * datom/ddim: -1 for the integrals themselves, else the derivative with respect
 * to coordinate ddim of atom datom (basis-centre terms, and for kind 2 also the
 * operator term of nucleus datom).  out is ncart x ncart, row-major.
 */
void oracle_one_electron(int kind, int nshell, const int* l, const int* atom, const double* xyz, const int* nprim,
                         const int* pstart, const double* exps, const double* coefs, int natoms, const int* Z,
                         const double* axyz, int datom, int ddim, double* out) {
  MAKE_BASIS(B, nshell, l, atom, xyz, nprim, pstart, exps, coefs);
  int n = B.ncart;
  memset(out, 0, sizeof(double) * n * n);
#pragma omp parallel
  {
    int Lmax = 2 * LE;
    int D = Lmax + 1;
    double* scratch = (double*)malloc(sizeof(double) * D * D * D * D);
    double* R = (double*)malloc(sizeof(double) * D * D * D);
    hpair* h = (hpair*)malloc(sizeof(hpair));
#pragma omp for schedule(dynamic)
    for (int sa = 0; sa < nshell; ++sa)
      for (int sb = 0; sb < nshell; ++sb) {
        int da = (datom >= 0 && atom[sa] == datom), db = (datom >= 0 && atom[sb] == datom);
        if (datom >= 0 && kind != 2 && !da && !db) continue;
        int la = l[sa], lb = l[sb];
        for (int pa = 0; pa < nprim[sa]; ++pa)
          for (int pb = 0; pb < nprim[sb]; ++pb) {
            double a = exps[pstart[sa] + pa], b = exps[pstart[sb] + pb];
            double cc = coefs[pstart[sa] + pa] * coefs[pstart[sb] + pb];
            hpair_init(h, a, xyz + 3 * sa, b, xyz + 3 * sb, la + 1, lb + 3);
            int Lh = la + lb + 2;
            int DL = Lh + 1;
            if (kind < 2) {
              for (int ia = 0; ia < ncart_of(la); ++ia)
                for (int ib = 0; ib < ncart_of(lb); ++ib) {
                  int ca[3], cb[3];
                  cart_comp(la, ia, ca);
                  cart_comp(lb, ib, cb);
                  double v = 0.0;
                  ctx1 xa = {h, cb, 0, b, kind, 0, 0, 0}, xb = {h, ca, 1, b, kind, 0, 0, 0};
                  if (datom < 0) v = ev1(ca, &xa);
                  else {
                    if (da) v += deriv_combo(ca, ddim, a, ev1, &xa);
                    if (db) v += deriv_combo(cb, ddim, b, ev1, &xb);
                  }
                  out[(B.off[sa] + ia) * n + B.off[sb] + ib] += cc * v;
                }
              continue;
            }
            for (int C = 0; C < natoms; ++C) {
              int oc = (datom == C);
              if (datom >= 0 && !da && !db && !oc) continue;
              double PC[3] = {h->P[0] - axyz[3 * C], h->P[1] - axyz[3 * C + 1], h->P[2] - axyz[3 * C + 2]};
              hermite_R(Lh, h->p, PC, scratch, R);
              for (int ia = 0; ia < ncart_of(la); ++ia)
                for (int ib = 0; ib < ncart_of(lb); ++ib) {
                  int ca[3], cb[3];
                  cart_comp(la, ia, ca);
                  cart_comp(lb, ib, cb);
                  int zero[3] = {0, 0, 0}, shd[3] = {0, 0, 0};
                  ctx1 xa = {h, cb, 0, b, 2, R, DL, zero}, xb = {h, ca, 1, b, 2, R, DL, zero};
                  double w = 0.0;
                  if (datom < 0) w = ev1(ca, &xa);
                  else {
                    if (da) w += deriv_combo(ca, ddim, a, ev1, &xa);
                    if (db) w += deriv_combo(cb, ddim, b, ev1, &xb);
                    if (oc) {
                      /* d/dC_x of R_{tuv}(P-C) = -R_{t+1,u,v} */
                      shd[ddim] = 1;
                      ctx1 xo = {h, cb, 0, b, 2, R, DL, shd};
                      w -= ev1(ca, &xo);
                    }
                  }
                  out[(B.off[sa] + ia) * n + B.off[sb] + ib] += cc * (-Z[C] * w);
                }
            }
          }
      }
    free(scratch); free(R); free(h);
  }
  free(B.off);
}

/* ------------------------------------------------- public: (P|Q), (ab|P) */

typedef struct {
  const hpair* h1; const hpair* h2; const int *ci, *cj, *ck, *cl; int which; const double* R; int D;
} ctx2;

static double ev2(const int* c, void* vp) {
  ctx2* x = (ctx2*)vp;
  const int* a = x->which == 0 ? c : x->ci;
  const int* b = x->which == 1 ? c : x->cj;
  const int* k = x->which == 2 ? c : x->ck;
  return prim_eri(x->h1, a, b, x->h2, k, x->cl, x->R, x->D);
}

/*
 * 3-centre integrals (ab|P): out[(mu*nprim_cart + nu)*naux_cart + P].
 * With datom >= 0, the derivative of (ab|P) with respect to coordinate ddim of
 * atom datom (every centre on that atom differentiated, including the
 * auxiliary one).
 */
void oracle_eri3(int ns, const int* l, const int* atom, const double* xyz, const int* nprim, const int* pstart,
                 const double* exps, const double* coefs, int nsa, const int* la_, const int* atoma,
                 const double* xyza, const int* nprima, const int* pstarta, const double* expsa,
                 const double* coefsa, int datom, int ddim, double* out) {
  MAKE_BASIS(B, ns, l, atom, xyz, nprim, pstart, exps, coefs);
  MAKE_BASIS(X, nsa, la_, atoma, xyza, nprima, pstarta, expsa, coefsa);
  int n = B.ncart, nx = X.ncart;
  memset(out, 0, sizeof(double) * (size_t)n * n * nx);
#pragma omp parallel
  {
    int D = LRMAX + 1;
    double* scratch = (double*)malloc(sizeof(double) * D * D * D * D);
    double* R = (double*)malloc(sizeof(double) * D * D * D);
    hpair* h1 = (hpair*)malloc(sizeof(hpair));
    hpair* h2 = (hpair*)malloc(sizeof(hpair));
#pragma omp for schedule(dynamic)
    for (int sab = 0; sab < ns * ns; ++sab) {
      int sa = sab / ns, sb = sab % ns;
      if (sb > sa) continue;
      for (int sc = 0; sc < nsa; ++sc) {
        int da = datom >= 0 && atom[sa] == datom, db = datom >= 0 && atom[sb] == datom,
            dc = datom >= 0 && atoma[sc] == datom;
        if (datom >= 0 && !da && !db && !dc) continue;
        int l1 = l[sa], l2 = l[sb], l3 = la_[sc];
        int ext = datom >= 0 ? 1 : 0;
        int L = l1 + l2 + l3 + ext, DL = L + 1;
        for (int pa = 0; pa < nprim[sa]; ++pa)
          for (int pb = 0; pb < nprim[sb]; ++pb)
            for (int pc = 0; pc < nprima[sc]; ++pc) {
              double a = exps[pstart[sa] + pa], b = exps[pstart[sb] + pb], c = expsa[pstarta[sc] + pc];
              double cc = coefs[pstart[sa] + pa] * coefs[pstart[sb] + pb] * coefsa[pstarta[sc] + pc];
              hpair_init(h1, a, xyz + 3 * sa, b, xyz + 3 * sb, l1 + ext, l2 + ext);
              hpair_init(h2, c, xyza + 3 * sc, 0.0, xyza + 3 * sc, l3 + ext, 0);
              double PQ[3] = {h1->P[0] - h2->P[0], h1->P[1] - h2->P[1], h1->P[2] - h2->P[2]};
              double alpha = h1->p * h2->p / (h1->p + h2->p);
              hermite_R(L, alpha, PQ, scratch, R);
              for (int ia = 0; ia < ncart_of(l1); ++ia)
                for (int ib = 0; ib < ncart_of(l2); ++ib)
                  for (int ic = 0; ic < ncart_of(l3); ++ic) {
                    int ca[3], cb[3], ck[3], z0[3] = {0, 0, 0};
                    cart_comp(l1, ia, ca);
                    cart_comp(l2, ib, cb);
                    cart_comp(l3, ic, ck);
                    double v = 0.0;
                    if (datom < 0) {
                      v = prim_eri(h1, ca, cb, h2, ck, z0, R, DL);
                    } else {
                      ctx2 x0 = {h1, h2, ca, cb, ck, z0, 0, R, DL};
                      ctx2 x1 = x0, x2 = x0;
                      x1.which = 1;
                      x2.which = 2;
                      if (da) v += deriv_combo(ca, ddim, a, ev2, &x0);
                      if (db) v += deriv_combo(cb, ddim, b, ev2, &x1);
                      if (dc) v += deriv_combo(ck, ddim, c, ev2, &x2);
                    }
                    v *= cc;
                    int mu = B.off[sa] + ia, nu = B.off[sb] + ib, P = X.off[sc] + ic;
                    out[((size_t)mu * n + nu) * nx + P] += v;
                    if (sa != sb) out[((size_t)nu * n + mu) * nx + P] += v;
                  }
            }
      }
    }
    free(scratch); free(R); free(h1); free(h2);
  }
  free(B.off); free(X.off);
}

/* 2-centre metric (P|Q) (or its derivative w.r.t. coordinate ddim of atom datom). */
void oracle_eri2(int nsa, const int* la_, const int* atoma, const double* xyza, const int* nprima,
                 const int* pstarta, const double* expsa, const double* coefsa, int datom, int ddim, double* out) {
  MAKE_BASIS(X, nsa, la_, atoma, xyza, nprima, pstarta, expsa, coefsa);
  int nx = X.ncart;
  memset(out, 0, sizeof(double) * nx * nx);
#pragma omp parallel
  {
    int D = LRMAX + 1;
    double* scratch = (double*)malloc(sizeof(double) * D * D * D * D);
    double* R = (double*)malloc(sizeof(double) * D * D * D);
    hpair* h1 = (hpair*)malloc(sizeof(hpair));
    hpair* h2 = (hpair*)malloc(sizeof(hpair));
#pragma omp for schedule(dynamic)
    for (int sa = 0; sa < nsa; ++sa)
      for (int sb = 0; sb < nsa; ++sb) {
        int da = datom >= 0 && atoma[sa] == datom, db = datom >= 0 && atoma[sb] == datom;
        if (datom >= 0 && !da && !db) continue;
        int l1 = la_[sa], l2 = la_[sb], ext = datom >= 0 ? 1 : 0;
        int L = l1 + l2 + ext, DL = L + 1;
        for (int pa = 0; pa < nprima[sa]; ++pa)
          for (int pb = 0; pb < nprima[sb]; ++pb) {
            double a = expsa[pstarta[sa] + pa], b = expsa[pstarta[sb] + pb];
            double cc = coefsa[pstarta[sa] + pa] * coefsa[pstarta[sb] + pb];
            hpair_init(h1, a, xyza + 3 * sa, 0.0, xyza + 3 * sa, l1 + ext, 0);
            hpair_init(h2, b, xyza + 3 * sb, 0.0, xyza + 3 * sb, l2 + ext, 0);
            double PQ[3] = {h1->P[0] - h2->P[0], h1->P[1] - h2->P[1], h1->P[2] - h2->P[2]};
            double alpha = h1->p * h2->p / (h1->p + h2->p);
            hermite_R(L, alpha, PQ, scratch, R);
            for (int ia = 0; ia < ncart_of(l1); ++ia)
              for (int ib = 0; ib < ncart_of(l2); ++ib) {
                int ca[3], cb[3], z0[3] = {0, 0, 0};
                cart_comp(l1, ia, ca);
                cart_comp(l2, ib, cb);
                double v = 0.0;
                if (datom < 0) v = prim_eri(h1, ca, z0, h2, cb, z0, R, DL);
                else {
                  ctx2 x0 = {h1, h2, ca, z0, cb, z0, 0, R, DL};
                  ctx2 x2 = x0;
                  x2.which = 2;
                  if (da) v += deriv_combo(ca, ddim, a, ev2, &x0);
                  if (db) v += deriv_combo(cb, ddim, b, ev2, &x2);
                }
                out[(X.off[sa] + ia) * nx + X.off[sb] + ib] += cc * v;
              }
          }
      }
    free(scratch); free(R); free(h1); free(h2);
  }
  free(X.off);
}

/* Four-centre (ab|cd), out[((a*n+b)*n+c)*n+d]; tiny bases only (brute-force HF). */
void oracle_eri4(int ns, const int* l, const int* atom, const double* xyz, const int* nprim, const int* pstart,
                 const double* exps, const double* coefs, double* out) {
  MAKE_BASIS(B, ns, l, atom, xyz, nprim, pstart, exps, coefs);
  size_t n = B.ncart;
  memset(out, 0, sizeof(double) * n * n * n * n);
#pragma omp parallel
  {
    int D = LRMAX + 1;
    double* scratch = (double*)malloc(sizeof(double) * D * D * D * D);
    double* R = (double*)malloc(sizeof(double) * D * D * D);
    hpair* h1 = (hpair*)malloc(sizeof(hpair));
    hpair* h2 = (hpair*)malloc(sizeof(hpair));
#pragma omp for schedule(dynamic)
    for (int sab = 0; sab < ns * ns; ++sab) {
      int sa = sab / ns, sb = sab % ns;
      for (int sc = 0; sc < ns; ++sc)
        for (int sd = 0; sd < ns; ++sd) {
          int l1 = l[sa], l2 = l[sb], l3 = l[sc], l4 = l[sd];
          int L = l1 + l2 + l3 + l4, DL = L + 1;
          for (int pa = 0; pa < nprim[sa]; ++pa)
            for (int pb = 0; pb < nprim[sb]; ++pb)
              for (int pc = 0; pc < nprim[sc]; ++pc)
                for (int pd = 0; pd < nprim[sd]; ++pd) {
                  double a = exps[pstart[sa] + pa], b = exps[pstart[sb] + pb];
                  double c = exps[pstart[sc] + pc], d = exps[pstart[sd] + pd];
                  double cc = coefs[pstart[sa] + pa] * coefs[pstart[sb] + pb] * coefs[pstart[sc] + pc] *
                              coefs[pstart[sd] + pd];
                  hpair_init(h1, a, xyz + 3 * sa, b, xyz + 3 * sb, l1, l2);
                  hpair_init(h2, c, xyz + 3 * sc, d, xyz + 3 * sd, l3, l4);
                  double PQ[3] = {h1->P[0] - h2->P[0], h1->P[1] - h2->P[1], h1->P[2] - h2->P[2]};
                  double alpha = h1->p * h2->p / (h1->p + h2->p);
                  hermite_R(L, alpha, PQ, scratch, R);
                  for (int ia = 0; ia < ncart_of(l1); ++ia)
                    for (int ib = 0; ib < ncart_of(l2); ++ib)
                      for (int ic = 0; ic < ncart_of(l3); ++ic)
                        for (int id = 0; id < ncart_of(l4); ++id) {
                          int ca[3], cb[3], ck[3], cl[3];
                          cart_comp(l1, ia, ca);
                          cart_comp(l2, ib, cb);
                          cart_comp(l3, ic, ck);
                          cart_comp(l4, id, cl);
                          double v = cc * prim_eri(h1, ca, cb, h2, ck, cl, R, DL);
                          size_t i = B.off[sa] + ia, j = B.off[sb] + ib, k = B.off[sc] + ic, m = B.off[sd] + id;
                          out[((i * n + j) * n + k) * n + m] += v;
                        }
                }
        }
    }
    free(scratch); free(R); free(h1); free(h2);
  }
  free(B.off);
}
