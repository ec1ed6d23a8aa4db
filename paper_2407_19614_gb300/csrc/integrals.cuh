// Host-visible declarations of the integral kernels (integrals.cu).
#pragma once
#include <vector>

#include "common.cuh"

namespace rihf {

// Device view of a shell list (all arrays device-resident).
struct DevShells {
  int nshell = 0;
  int nfunc = 0;                 // AO count
  const int* l = nullptr;
  const int* atom = nullptr;
  const double* xyz = nullptr;   // 3 per shell
  const int* nprim = nullptr;
  const int* pstart = nullptr;
  const double* exps = nullptr;
  const double* iexps = nullptr; // 1 / exps
  const double* coefs = nullptr; // primitive coefficients times x^l normalisation
  const int* ao = nullptr;       // first AO of each shell
  const double* tr = nullptr;    // per-l transform, kTrL x 15 x 15 (rows: output functions)
  const int* nf = nullptr;       // per-l number of output functions
};

// Shell pair (a >= b) list entries.
struct ShellPair {
  int a, b;
};

struct PairPrim;   // os_hgp.cuh
// Primitive-pair data of the listed shell pairs: entries off[i] ..
// off[i] + nprim(a) nprim(b) - 1 of pp for pair i, ordered (pa, pb) with the
// pair's shells swapped to la >= lb (the order the kernels evaluate in).
struct PairTable {
  const PairPrim* pp = nullptr;
  const int* off = nullptr;
};
// Offsets for a pair list (host), and the per-geometry build of the table.
std::vector<int> pair_prim_offsets(const std::vector<ShellPair>& pairs, const std::vector<int>& nprim);


struct IntegralCtx {
  const double* boys = nullptr;  // Boys table on device
  int* counter = nullptr;        // device work counter (one int per launch kind)
  cudaStream_t stream = 0;
  long long* launches = nullptr; // host-side launch counter
};

// Build the primitive-pair table for `npairs` pairs (device), into pp (sized
// by the last offset from pair_prim_offsets plus the last pair's count).
void launch_pair_prims(const IntegralCtx& ic, const DevShells& prim, const ShellPair* pairs, int npairs,
                       const int* off, PairPrim* pp);

// Shared memory (doubles) one warp needs for a (la >= lb | lc) class of the
// integral and of the derivative kernel.
// alias: the 3-centre integral task's plan (scratch over the dead VRR table);
// one: the derivative task's plan for one primitive triple
int smem_eri3_doubles(int la, int lb, int lc, bool mirror = false, bool alias = false);
int smem_grad_doubles(int la, int lb, int lc, bool mirror = false, bool one = false);

// Whether a (pair, auxiliary shell) task may take the mirrored recursion
// (mirror_prim3): the forward transfer multiplies by p/q and by beta AB/q once
// per unit of l_c, so with p > q and l_c >= 2 it loses digits to rounding --
// measured against the oracle for an f/g auxiliary set, up to 1e-10 of the
// largest integral already at p/q between 2 and 8.  A task is marked when its
// largest bra exponent sum exceeds its smallest ket exponent; its triples with
// p > q then run mirrored, where every factor is at most one (or |AB|).
inline bool mirror_task(double pmax, double qmin, int lc) { return lc >= 2 && pmax > qmin; }
// (P|Q) classes (bit 8 la + lc, la, lc <= max_la) run by 8-lane task groups,
// and the shared-memory slice (doubles) one such group needs.
unsigned long long eri2_small_classes(int max_la, int* slice_doubles);

// (pair index, auxiliary shell) tasks of one shared-memory class group.
constexpr int kTaskGroups = 7;
// Resident one-warp blocks per SM the 3-centre kernels are compiled for.  The
// integral kernel at 20 (at most 96 registers a thread): its light class
// groups, whose shared-memory slices allow more, were held to 13 warps per SM
// by 150 registers alone.  The derivative kernel at 16 (126 registers, no
// spills): at 20 its spills cost what the extra warps gain.
constexpr int kEri3BlocksPerSM = 20;
constexpr int kGradBlocksPerSM = 16;
struct TaskGroup {
  const int2* tasks = nullptr;
  long long ntask = 0;
  int smem_eri3 = 0, smem_grad = 0;   // bytes per task
  int width = 32;                     // lanes per task (8: four tasks per warp, 16: two)
};
// Lanes per task of class group g (group 0 holds the tiny classes).
inline int task_group_width(int g) { return g == 0 ? 8 : g == 1 ? 16 : 32; }
// Largest task count of one class group: the kernels claim tasks through an
// int counter, which runs past the count by 32 / W per resident warp.
constexpr long long kMaxGroupTasks = (1LL << 31) - (1LL << 24);
// nprim / naux_prim: primitives per primary / auxiliary shell; pmax: largest
// primitive exponent per primary shell; qmin: smallest per auxiliary shell (for
// mirror_task).  A marked task stores ~c as its auxiliary index.  Each group's
// tasks come ordered by shape, heaviest first.
void build_task_groups(const std::vector<ShellPair>& pairs, const std::vector<int>& lprim,
                       const std::vector<int>& nprim, const std::vector<int>& laux,
                       const std::vector<int>& naux_prim, const std::vector<double>& pmax,
                       const std::vector<double>& qmin, std::vector<std::vector<int2>>& tasks,
                       std::vector<int>& smem_eri3, std::vector<int>& smem_grad);

// Algorithmic FP64 operation counts (an FMA counts two) of the 3-centre
// integral and derivative kernels over all (pair, auxiliary shell) tasks, from
// the loop structure of their recursions: per primitive triple the setup, Boys
// Taylor steps, vertical recurrence, electron transfer and accumulation(s); per
// task the horizontal recurrence(s), the spherical transforms and, for the
// gradient, the back-transform of Y and the contraction.  One-centre triples
// are skipped by the derivative kernel and not counted.
void task_flops(const std::vector<ShellPair>& pairs, const std::vector<int>& lprim, const std::vector<int>& nprim,
                const std::vector<int>& patom, const std::vector<int>& laux, const std::vector<int>& naux_prim,
                const std::vector<int>& aatom, const std::vector<int>& nf, const std::vector<double>& pmax,
                const std::vector<double>& qmin, double* eri3, double* grad3);

// Three-centre integrals T[P][mu][nu] = (mu nu|P) for the listed shell pairs
// (mu in a, nu in b, a >= b; both triangles inside diagonal shell blocks).
void launch_eri3(const IntegralCtx& ic, const DevShells& prim, const DevShells& aux, const ShellPair* pairs,
                 const PairTable& pt, const TaskGroup* groups, int ngroups, double* T);

// One geometry of a batched 3-centre launch (A14): its shells, pair list,
// primitive-pair table and tasks of the launch's class group; out = its
// pair-packed T (integrals) or its per-atom gradient (derivative
// contraction, with Y its pair-packed fitted density).
struct GeomTasks {
  DevShells prim, aux;
  const ShellPair* pairs = nullptr;
  PairTable ptab;
  const int2* tasks = nullptr;
  double* out = nullptr;
  const double* Y = nullptr;
};
// A batch of geometries for the batched launches: per geometry its
// descriptor (tasks unset), class groups and task counts.
struct BatchGeom {
  GeomTasks g;
  const TaskGroup* groups = nullptr;
};
// Device tables of a batched launch: ngeom descriptors and ngeom + 1 offsets
// per class group (kTaskGroups x ngeom, kTaskGroups x (ngeom + 1)).
struct BatchTables {
  GeomTasks* geoms = nullptr;
  long long* off = nullptr;
  int cap = 0;
};
// One launch per class group over every geometry's tasks of that group:
// task t of the launch belongs to geometry g with off[g] <= t < off[g + 1]
// (an int64 offsets table), so ragged geometries share the SMs with no
// per-geometry launch.  Shared memory per task: the largest of the
// geometries' slices of the group.  Uploads the tables (host -> device on
// ic.stream, then waits for them: the host arrays are temporaries).
void launch_eri3_batch(const IntegralCtx& ic, const std::vector<BatchGeom>& batch, int ngroups, BatchTables& t);
// Host side shared by the two: for class group g, the descriptors (with that
// group's task pointers) and the offsets table uploaded into t; the largest
// shared-memory slice of the group (grad: the derivative kernel's) and the
// task count.  False when the group has no task.
bool batch_tables(const IntegralCtx& ic, const std::vector<BatchGeom>& batch, int g, BatchTables& t, bool grad,
                  int& slice_bytes, long long& ntask);
void launch_grad_eri3_batch(const IntegralCtx& ic, const std::vector<BatchGeom>& batch, int ngroups,
                            BatchTables& t);

// Metric A[P][Q] = (P|Q) (full symmetric matrix).
void launch_eri2(const IntegralCtx& ic, const DevShells& aux, int max_la, double* A);

// One-electron S, T (kinetic) and V (nuclear attraction, sum_C -Z_C <a|1/r_C|b>).
void launch_one_electron(const IntegralCtx& ic, const DevShells& prim, int max_lp, int natoms, const int* Z,
                         const double* axyz, double* S, double* Tk, double* V);

// Schwarz factors Q_ab = sqrt(max |(ab|ab)|) over all shell pairs a >= b,
// pair index a*(a+1)/2 + b.
void launch_schwarz(const IntegralCtx& ic, const DevShells& prim, int max_lp, double* Q);
// Shared memory (bytes) launch_schwarz needs for primary l <= max_lp.
int schwarz_smem_bytes(int max_lp);

// Gradient contractions (derivative integrals evaluated on the fly):
//   grad[atom][x] += sum_{mu nu P} Y[P][mu][nu] d(mu nu|P)/dR          (3-centre)
//   grad[atom][x] += -1/2 sum_PQ Z[P][Q] d(P|Q)/dR                      (2-centre)
//   grad[atom][x] += sum D d(T+V)/dR - sum W dS/dR                      (one-electron)
void launch_grad_eri3(const IntegralCtx& ic, const DevShells& prim, const DevShells& aux, const ShellPair* pairs,
                      const PairTable& pt, const TaskGroup* groups, int ngroups, const double* Y, double* grad);
void launch_grad_eri2(const IntegralCtx& ic, const DevShells& aux, int max_la, const double* Z, double* grad);
void launch_grad_one_electron(const IntegralCtx& ic, const DevShells& prim, int max_lp, int natoms, const int* Z,
                              const double* axyz, const double* D, const double* W, double* grad_one,
                              double* grad_ovl);

// Boys table F_m(T_k) generated on the host (long double Gauss-Legendre
// quadrature of the defining integral), kBoysN x kBoysM doubles.
void boys_table_host(double* out);

}  // namespace rihf
