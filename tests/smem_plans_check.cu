// Host-side checks of the 3-centre kernels' shared-memory plans and task lists
// (no device calls).  Built against the kernel sources themselves, so the plans
// checked are the ones the kernels use:
//  * every region live during the primitive loop (F_m, VRR table, transfer
//    levels, accumulators, the Y block staged by asynchronous copies) and
//    every region live after it (transfer level or
//    accumulator read by the HRR, back-transformed Y, HRR and transform
//    scratch) are pairwise disjoint and inside the plan, for every class
//    (la <= 3, lb <= la, lc <= 4), with and without the mirrored recursion,
//    and for derivative tasks of one primitive triple and of several;
//  * the task lists of a synthetic shell set (mixed l and primitive counts)
//    hold every (pair, auxiliary shell) task once, with the right mirror mark,
//    in a group whose slices cover the task's plans, each shape contiguous and
//    the shapes heaviest first.
// Prints "OK" and exits 0, or names the first violations and exits 1.
#include "integrals.cu"
#include "grad_integrals.cu"

#include <cstdio>
#include <random>
#include <set>

namespace rihf {
void raise_smem_limit(const void*, int) {}   // launch helper, not exercised here
}

using namespace rihf;

namespace {

struct Region {
  int lo, hi;
  const char* name;
};

int g_fail = 0;

void disjoint(const std::vector<Region>& v, int total, const char* what, int la, int lb, int lc, int mi, int one) {
  for (const Region& r : v)
    if (r.lo < 0 || r.hi > total || r.lo > r.hi) {
      if (g_fail++ < 20)
        printf("%s: %s outside the plan, (%d %d|%d) mirror %d one %d: [%d, %d) of %d\n", what, r.name, la, lb, lc, mi,
               one, r.lo, r.hi, total);
    }
  for (size_t i = 0; i < v.size(); ++i)
    for (size_t j = i + 1; j < v.size(); ++j) {
      const Region &a = v[i], &b = v[j];
      if (a.hi > a.lo && b.hi > b.lo && a.lo < b.hi && b.lo < a.hi && g_fail++ < 20)
        printf("%s: %s overlaps %s, (%d %d|%d) mirror %d one %d\n", what, a.name, b.name, la, lb, lc, mi, one);
    }
}

void check_plans() {
  for (int mi = 0; mi < 2; ++mi)
    for (int la = 0; la <= kMaxLPrim; ++la)
      for (int lb = 0; lb <= la; ++lb)
        for (int lc = 0; lc <= kMaxLAux; ++lc) {
          const int nabc = ncart(la) * ncart(lb) * ncart(lc);
          for (int one = 0; one < 2; ++one) {
            const DerivPlan p(la, lb, lc, mi == 1, one == 1);
            const int accsz = acc_size(p.emin, p.emax, lc);
            int etr_n = lc > 0 ? EtrShape{lc, p.emin, p.emax}.total() : 0;
            if (mi) etr_n = std::max(etr_n, EtrShape{p.emax, lc, lc}.total());
            std::vector<Region> loop = {{p.fm, p.fm + p.L + 1, "F_m"},
                                        {p.vrr, p.vrr + vrr_size(p.L), "VRR"},
                                        {p.etr, p.etr + etr_n, "transfer levels"},
                                        {p.acc0, p.acc0 + accsz, "acc0"},
                                        {p.ycart, p.ycart + nabc, "Y block (staged during the loop)"}};
            std::vector<Region> post = {{p.etr, p.etr + etr_n, "transfer levels"},
                                        {p.acc0, p.acc0 + accsz, "acc0"},
                                        {p.ycart, p.ycart + nabc, "Y (Cartesian)"},
                                        {p.hrr, p.hrr + 2 * p.half, "HRR scratch"}};
            if (!one) {
              for (auto* v : {&loop, &post}) {
                v->push_back({p.accA, p.accA + accsz, "accA"});
                v->push_back({p.accB, p.accB + accsz, "accB"});
              }
            }
            disjoint(loop, p.total, "derivative plan, primitive loop", la, lb, lc, mi, one);
            disjoint(post, p.total, "derivative plan, contraction", la, lb, lc, mi, one);
            if (p.t1 < p.hrr || p.t2 + p.half > p.hrr + 2 * p.half) {
              if (g_fail++ < 20) printf("derivative plan: back-transform scratch outside the HRR region\n");
            }
            if (smem_grad_doubles(la, lb, lc, mi == 1, one == 1) < p.total && g_fail++ < 20)
              printf("smem_grad_doubles below the plan, (%d %d|%d)\n", la, lb, lc);
          }
          const Eri3Plan e(la, lb, lc, la, la + lb, 1, mi == 1, true);
          const int L = la + lb + lc, big = ncart(la + 1) * ncart(lb + 1) * ncart(lc);
          int etr_n = lc > 0 ? EtrShape{lc, la, la + lb}.total() : 0;
          if (mi) etr_n = std::max(etr_n, EtrShape{la + lb, lc, lc}.total());
          const int accsz = acc_size(la, la + lb, lc);
          disjoint({{e.fm, e.fm + L + 1, "F_m"},
                    {e.vrr, e.vrr + vrr_size(L), "VRR"},
                    {e.etr, e.etr + etr_n, "transfer levels"},
                    {e.acc, e.acc + accsz, "accumulator"}},
                   e.total, "integral plan, primitive loop", la, lb, lc, mi, 0);
          disjoint({{e.etr, e.etr + etr_n, "transfer levels"},
                    {e.acc, e.acc + accsz, "accumulator"},
                    {e.hrr, e.hrr + 2 * e.half, "HRR scratch"},
                    {e.t1, e.t1 + big, "transform t1"},
                    {e.t2, e.t2 + big, "transform t2"}},
                   e.total, "integral plan, HRR and transforms", la, lb, lc, mi, 0);
          if (smem_eri3_doubles(la, lb, lc, mi == 1, true) < e.total && g_fail++ < 20)
            printf("smem_eri3_doubles below the plan, (%d %d|%d)\n", la, lb, lc);
        }
}

void check_task_lists() {
  std::mt19937 rng(7);
  const int nprim_shells = 40, naux_shells = 60;
  std::vector<int> lprim(nprim_shells), nprim(nprim_shells), laux(naux_shells), naux_prim(naux_shells);
  std::vector<double> pmax(nprim_shells), qmin(naux_shells);
  for (int i = 0; i < nprim_shells; ++i) {
    lprim[i] = rng() % (kMaxLPrim + 1);
    nprim[i] = i % 3 == 0 ? 1 + rng() % 4 : 1;   // contracted and single-primitive shells
    pmax[i] = 0.1 * std::pow(3.0, (double)(rng() % 8));
  }
  for (int c = 0; c < naux_shells; ++c) {
    laux[c] = rng() % (kMaxLAux + 1);
    naux_prim[c] = c % 5 == 0 ? 2 : 1;
    qmin[c] = 0.15 * std::pow(2.5, (double)(rng() % 10));
  }
  std::vector<ShellPair> pairs;
  for (int a = 0; a < nprim_shells; ++a)
    for (int b = 0; b <= a; ++b)
      if ((a + 2 * b) % 3 != 1) pairs.push_back({a, b});   // a screened pair list
  std::vector<std::vector<int2>> tasks;
  std::vector<int> se, sg;
  build_task_groups(pairs, lprim, nprim, laux, naux_prim, pmax, qmin, tasks, se, sg);
  if ((int)tasks.size() != kTaskGroups) {
    printf("task lists: %zu groups\n", tasks.size());
    ++g_fail;
    return;
  }
  std::set<std::pair<int, int>> seen;
  size_t n = 0;
  for (int g = 0; g < kTaskGroups; ++g) {
    std::set<std::array<int, 7>> done;   // shapes already closed in this group
    std::array<int, 7> cur{-1, -1, -1, -1, -1, -1, -1};
    double last_cost = 1e300;   // shapes come heaviest first (primitive triples x derivative plan)
    for (const int2& t : tasks[g]) {
      ++n;
      const int p = t.x, c = t.y < 0 ? ~t.y : t.y, mi = t.y < 0 ? 1 : 0;
      if (p < 0 || p >= (int)pairs.size() || c < 0 || c >= naux_shells) {
        if (g_fail++ < 20) printf("task lists: task (%d, %d) out of range\n", t.x, t.y);
        continue;
      }
      if (!seen.insert({p, c}).second && g_fail++ < 20) printf("task lists: task (%d, %d) twice\n", p, c);
      int a = pairs[p].a, b = pairs[p].b;
      if (lprim[a] < lprim[b]) std::swap(a, b);
      const int la = lprim[a], lb = lprim[b], lc = laux[c];
      if (mi != (mirror_task(pmax[pairs[p].a] + pmax[pairs[p].b], qmin[c], lc) ? 1 : 0) && g_fail++ < 20)
        printf("task lists: wrong mirror mark on (%d, %d)\n", p, c);
      const bool one = nprim[a] * nprim[b] * naux_prim[c] == 1;
      const int need_e = smem_eri3_doubles(la, lb, lc, mi == 1, true) * (int)sizeof(double);
      const int need_g = smem_grad_doubles(la, lb, lc, mi == 1, one) * (int)sizeof(double);
      if ((need_e > se[g] || need_g > sg[g]) && g_fail++ < 20)
        printf("task lists: group %d slices %d/%d below task (%d %d|%d) needs %d/%d\n", g, se[g], sg[g], la, lb, lc,
               need_e, need_g);
      // the shape key of the list builder: the pair ordered by l, then (equal
      // l) by primitive count
      int sa = pairs[p].a, sb = pairs[p].b;
      if (lprim[sa] < lprim[sb] || (lprim[sa] == lprim[sb] && nprim[sa] < nprim[sb])) std::swap(sa, sb);
      const std::array<int, 7> shape{mi, la, lb, lc, nprim[sa], nprim[sb], naux_prim[c]};
      if (shape != cur) {
        if (cur[0] >= 0) done.insert(cur);
        if (done.count(shape) && g_fail++ < 20) printf("task lists: shape split in group %d\n", g);
        cur = shape;
        const double cost = (double)nprim[a] * nprim[b] * naux_prim[c] * need_g;
        if (cost > last_cost && g_fail++ < 20) printf("task lists: a lighter shape before a heavier one in group %d\n", g);
        last_cost = cost;
      }
    }
  }
  if (n != pairs.size() * (size_t)naux_shells && g_fail++ < 20)
    printf("task lists: %zu tasks for %zu pairs x %d auxiliary shells\n", n, pairs.size(), naux_shells);
}

}  // namespace

int main() {
  check_plans();
  check_task_lists();
  if (g_fail) {
    printf("%d violations\n", g_fail);
    return 1;
  }
  printf("OK\n");
  return 0;
}
