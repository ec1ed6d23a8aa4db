/*
 * rihf.h -- C ABI of librihf.so: RI-HF energies and analytic nuclear gradients on
 * one NVIDIA GB300 (sm_103a), following Stocks, Palethorpe and Barca,
 * "Multi-GPU RI-HF Energies and Analytic Gradients -- Towards High Throughput
 * Ab Initio Molecular Dynamics" (the paper).
 *
 * Conventions for every entry point
 *   - Units: bohr, hartree, hartree/bohr.  Arrays are row-major doubles unless
 *     stated otherwise.
 *   - Host pointers are read during the call and never retained; output buffers
 *     are caller-owned host memory of the documented size.
 *   - The context owns all of its device memory (allocated in rihf_setup, freed
 *     in rihf_destroy) and is not thread-safe.
 *   - Return value: RIHF_OK (0) or a negative error code; rihf_strerror() gives
 *     a message and rihf_last_error() the detail of the last failure.
 *   - Basis functions: each shell is contracted over primitive Gaussians whose
 *     coefficients refer to normalised primitives; the library normalises the
 *     primitives and the contracted functions.  pure = 1 uses real solid
 *     harmonics ordered m = -l..l, each normalised to one; pure = 0 uses
 *     Cartesian functions ordered lx = l..0, ly = l-lx..0, each normalised to one.
 *   - AO order: shells in the order given, functions within a shell as above.
 *     Auxiliary functions likewise.
 *   - Molecular orbital coefficients C are N x N with C[mu * N + k] the
 *     coefficient of AO mu in orbital k, orbitals in ascending energy.
 *   - Limits: primary l <= 3, auxiliary l <= 4, contraction length <= 16.
 */
#ifndef RIHF_H
#define RIHF_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RIHF_OK = 0,
  RIHF_ERR_INVALID_ARG = -1,
  RIHF_ERR_OOM = -2,
  RIHF_ERR_CUDA = -3,
  RIHF_ERR_NOT_CONVERGED = -4,
  RIHF_ERR_TIMEOUT = -5,
  RIHF_ERR_NOT_POSITIVE_DEFINITE = -6,
  RIHF_ERR_STATE = -7
};

enum { RIHF_PRECISION_FP64 = 0, RIHF_PRECISION_MIXED = 1 };

typedef struct rihf_ctx rihf_ctx;

/* One contracted shell on atom `atom` with angular momentum l and nprim
   primitives (exps[k], coefs[k]).  Pointers are read during rihf_setup only. */
typedef struct {
  int atom;
  int l;
  int nprim;
  const double* exps;
  const double* coefs;
} rihf_shell;

typedef struct {
  int precision;        /* RIHF_PRECISION_FP64 or RIHF_PRECISION_MIXED                     */
  int pure;             /* 1: spherical functions, 0: Cartesian                             */
  double schwarz_tau;   /* drop primary shell pairs with max (ab|ab) <= tau (paper: 1e-10) */
  double lindep_tau;    /* drop overlap eigenvalues below this (canonical orthogonalisation) */
  double conv_e;        /* converged when |E_k - E_{k-1}| < conv_e ...                    */
  double conv_diis;     /* ... and max |X^T (FDS - SDF) X| < conv_diis                    */
  int max_iter;         /* SCF iteration cap (RIHF_ERR_NOT_CONVERGED when reached)         */
  int diis_size;        /* Pulay DIIS subspace size, 2..16                                 */
  int mixed_digits;     /* mixed precision: BF16 digits of the tensor-core RI-K (1..7);   */
                        /* 0 = ladder 5 -> 6 -> 7 digits as max|e| falls                 */
  int device;           /* CUDA device ordinal                                             */
  int cuda_graphs;      /* 1: each SCF iteration's Fock build and DIIS error are captured  */
                        /* once per precision variant and replayed as a CUDA graph        */
  int confirm_fp64;     /* mixed precision: 1 = convergence is confirmed on an FP64 Fock  */
                        /* build; 0 = on a 7-digit build (55-bit products per K block)   */
  int aux_chunk;        /* auxiliary functions per chunk when the pair-packed fitted      */
                        /* tensor is expanded for RI-K and the gradient; 0 = as many as   */
                        /* the free device memory holds (all of them for small systems)  */
} rihf_options;

/* Fills *opt with the defaults: FP64, spherical, schwarz_tau 0 (no pair
   dropped; with ill-conditioned auxiliary metrics even pairs below 1e-14 move
   the energy by ~1e-6 Eh, see the screening tests), lindep_tau
   1e-8, conv_e 1e-10, conv_diis 1e-9, max_iter 100, diis_size 8,
   mixed_digits 0, device 0, cuda_graphs 1, confirm_fp64 0, aux_chunk 0.
   Mixed precision (RIHF_PRECISION_MIXED): RI-K in the SCF iterations runs on
   the tensor cores from BF16 digit planes (see rihf_tc_dgemm) with 5, 6, then
   7 digits as the SCF error falls; the fit B = L^{-1} T and the gradient's
   products H, Z and Y use 7 digits (FP64-class: 55 bits of every row's
   largest element per K block); RI-J, D, DIIS, the diagonalisation, the
   Cholesky factors and the integrals stay FP64.  When the convergence test
   passes on a ladder build, the next build is a confirmation build (7 digits,
   or FP64 with confirm_fp64 = 1) and convergence is declared only on one. */
void rihf_default_options(rihf_options* opt);

/*
 * Builds a context for one molecule: copies the geometry and basis sets to the
 * device and evaluates the geometry-dependent quantities of Alg. 1 (before its
 * SCF loop): one-electron h = T + V and S, the metric A_PQ = (P|Q) (Sec. 2.2),
 * its Cholesky factor A = L L^T and L^{-1} (the paper's A^L, read as L^{-T}),
 * the Schwarz-screened 3-centre integrals (mu nu|P) (Sec. 3.1.1) and the fitted
 * B^P_{mu nu} = sum_Q (L^{-1})_{PQ} (mu nu|Q) (Eq. biap), stored unpacked as
 * Naux x N x N.
 *   natoms, Z[natoms], xyz[natoms*3]: nuclei (bohr).
 *   prim[nprim_shells], aux[naux_shells]: shells (atom indices into Z).
 *   nelec: electron count (even; closed shell).
 *   opt: options or NULL for the defaults.
 * Errors: INVALID_ARG (sizes, l limits, odd nelec), OOM, CUDA,
 * NOT_POSITIVE_DEFINITE (metric or overlap).
 */
int rihf_setup(int natoms, const int* Z, const double* xyz, int nprim_shells, const rihf_shell* prim,
               int naux_shells, const rihf_shell* aux, int nelec, const rihf_options* opt, rihf_ctx** out);

/* Moves the nuclei to xyz[natoms*3] (same atoms and basis) and recomputes every
   geometry-dependent quantity listed for rihf_setup.  Converged orbitals of the
   previous geometry are kept as the default guess of the next rihf_scf. */
int rihf_update_geometry(rihf_ctx* ctx, const double* xyz);

/*
 * Closed-shell RI-HF SCF (Roothaan FC = SC eps, Sec. 2.2 and Alg. 1): each
 * iteration forms D = 2 C_occ C_occ^T, RI-J (Eq. j_ri) and RI-K (Eqs. k_ri_2,
 * tp), F = h + J + K (Eq. fock_split), E = 1/2 Tr D(h+F) + V_nn, the DIIS
 * error X^T(FDS - SDF)X, Pulay extrapolation and diagonalisation.
 *   guess: 0 core Hamiltonian, 1 C_guess (N*N, columns 0..nocc-1 used),
 *          2 the context's previous converged orbitals (the paper's AIMD
 *            guess, Sec. 3.3; falls back to 0),
 *          3 density extrapolation D_x = 3 D_t - 3 D_{t-1} + D_{t-2} over the
 *            last three converged SCFs of this context, in the Loewdin
 *            representation D_L = S^{1/2} D S^{1/2} of each geometry (falls
 *            back to 2),
 *          4 learned: D_x plus the correction of the network configured by
 *            rihf_learn_config, once it beats D_x on its last training
 *            example (else D_x; falls back to 2).  With guesses 3 and 4 the
 *            predicted Loewdin density returns to the AO basis with this
 *            geometry's S^{-1/2} (pseudo-inverse over the overlap
 *            eigenvalues above lindep_tau), and the previous occupied
 *            orbitals are projected onto it (C <- D_pred S C, then
 *            S-orthonormalised).  The first guess-3 or -4 call (or
 *            rihf_learn_config) restarts the history in that representation.
 *          5 superposition of atomic densities (SAD, the paper's cold start,
 *            Sec. 2.2): one RI-HF SCF per atom type of the isolated,
 *            spherically averaged atom (fractional occupations, H to Ne; the
 *            same basis sets), D_SAD block-diagonal over the atoms; the first
 *            iteration builds J from D_SAD and K from its factor (the density
 *            form, Eq. k_ri_1).  Falls back to 0 when unavailable (other
 *            elements, an atom's shells not contiguous).
 *          Every converged SCF pushes its D (as D_L once guesses 3/4 are in
 *          use), S and nuclear positions into the three-deep history; a
 *          guess-4 SCF first trains the network on its own example
 *          (rihf_learn_config).
 *   energy (1), D (N*N), C (N*N), eps (N), iters (1): outputs; any may be NULL.
 * Returns NOT_CONVERGED (outputs filled from the last iterate) after max_iter.
 */
int rihf_scf(rihf_ctx* ctx, int guess, const double* C_guess, double* energy, double* D, double* C, double* eps,
             int* iters);

/*
 * Analytic RI-HF gradient (Eq. rihf_gradient, Alg. 2) at the last converged
 * rihf_scf of this context:
 *   dE/dR = sum D h^xi - sum W S^xi + sum_P Y^P (mu nu|P)^xi - 1/2 sum Z_PQ (P|Q)^xi + V_nn^xi
 * with h^xi including the nuclear-attraction operator derivative.  The
 * derivative integrals are evaluated and contracted on the fly, never stored.
 *   grad: natoms*3 output, dE/dR (forces are its negative).
 * Errors: STATE if no converged SCF is available.
 */
int rihf_gradient(rihf_ctx* ctx, double* grad);

/*
 * One AIMD step for a batch of independent molecules (contexts of any sizes):
 * for each i, rihf_update_geometry(ctx[i], xyz[i]) when xyz and xyz[i] are
 * non-NULL, rihf_scf(ctx[i], guess) and rihf_gradient(ctx[i]).  The molecules
 * run concurrently, each on its context's stream, driven by nthreads host
 * threads (0: one per hardware thread, at most nmol), so kernels of small
 * molecules overlap on the GPU.  Outputs (each may be NULL): energies[nmol],
 * grads = the molecules' natoms_i x 3 gradients concatenated in order,
 * iters[nmol].  Contexts must be distinct.  Returns the first error of the
 * batch (rihf_last_error names the molecule) or RIHF_OK.
 */
int rihf_batch_step(int nmol, rihf_ctx* const* ctx, const double* const* xyz, int guess, double* energies,
                    double* grads, int* iters, int nthreads);

/* Sizes of the context: primary functions N, auxiliary functions Naux,
   occupied orbitals nocc, atoms natoms.  Any pointer may be NULL. */
int rihf_query(rihf_ctx* ctx, int* N, int* Naux, int* nocc, int* natoms);

/* Intermediates for element-wise checks, copied to host buffer out (doubles):
     RIHF_MAT_S, RIHF_MAT_H, RIHF_MAT_J, RIHF_MAT_K, RIHF_MAT_F, RIHF_MAT_D: N x N
     RIHF_MAT_A, RIHF_MAT_LINV: Naux x Naux
     RIHF_MAT_T3: (mu nu|P) as Naux x N x N;  RIHF_MAT_B: B^P as Naux x N x N
     RIHF_MAT_GRAD_PARTS: 5 x natoms x 3 (one-electron, overlap, 3-centre,
                          2-centre, nuclear-repulsion terms of Eq. rihf_gradient)
     RIHF_MAT_SCHWARZ: Q_ab = sqrt(max (mu nu|mu nu)) over the Cartesian
                          components of shells a >= b, packed a(a+1)/2 + b
                          (nshell(nshell+1)/2 values, of the current
                          geometry; zeros when the four-centre class does not
                          fit the kernel's shared memory).  With schwarz_tau
                          <= 0 no pair is screened and Q is computed only for
                          this request
     RIHF_MAT_DSAD: N x N, the SAD guess density (after a guess-5 SCF built
                          it; RIHF_ERR_STATE before, or when SAD was unavailable)
     RIHF_MAT_DPRED: N x N, the predicted AO density of the last guess-3 or
                          guess-4 SCF (extrapolation plus network correction,
                          taken back from the Loewdin representation)
     RIHF_MAT_FEATURES: N(N+1)/2 x 12, the network's features of that guess
                          (stored in FP32, returned as doubles)
   J, K, F, D refer to the last Fock build. */
enum {
  RIHF_MAT_S = 0, RIHF_MAT_H = 1, RIHF_MAT_A = 2, RIHF_MAT_LINV = 3, RIHF_MAT_T3 = 4, RIHF_MAT_B = 5,
  RIHF_MAT_J = 6, RIHF_MAT_K = 7, RIHF_MAT_F = 8, RIHF_MAT_D = 9, RIHF_MAT_GRAD_PARTS = 10,
  RIHF_MAT_SCHWARZ = 11, RIHF_MAT_DPRED = 12, RIHF_MAT_FEATURES = 13, RIHF_MAT_DSAD = 14
};
int rihf_get_matrix(rihf_ctx* ctx, int which, double* out);

/* Number of significant primary shell pairs kept by the Schwarz screen and
   the total number of shell pairs (a >= b). */
int rihf_screening_stats(rihf_ctx* ctx, int* kept, int* total);

/* Per-phase device time of the last rihf_scf / rihf_gradient in milliseconds,
   measured with CUDA events: [0] integrals+fit, [1] SCF Fock builds,
   [2] SCF diagonalisation/DIIS, [3] gradient; and the number of kernels the
   library launched since the context was created ([4], as a double). */
int rihf_timings(rihf_ctx* ctx, double* out5);

/* Fock builds of the last rihf_scf: tensor-core RI-K builds of the precision
   ladder, FP64 builds, and confirmation builds (7-digit tensor-core builds
   after the ladder's convergence test passed; with confirm_fp64 = 1 these are
   the FP64 builds instead and the count is 0).  Any pointer may be NULL. */
int rihf_scf_stats(rihf_ctx* ctx, int* tc_builds, int* fp64_builds, int* confirm_builds);

/* The CUDA stream (cudaStream_t, returned as void*) on which the context
   launches all of its work; callers may record CUDA events on it. */
void* rihf_stream(rihf_ctx* ctx);

/* Per-kernel tracing.  rihf_trace(ctx, 1) clears the statistics and starts
   timing every instrumented launch with CUDA events on the context stream
   (adds two event records per launch); rihf_trace(ctx, 0) stops.
   rihf_trace_stats fills, for up to `max` traced kernels: names (48 chars
   each, NUL-terminated), launches, total device milliseconds and the
   algorithmic work of those launches (flops or bytes; kind: 0 = FP64 flops,
   1 = HBM bytes, 2 = FP32 flops, 3 = BF16 tensor-core flops issued).  Returns
   the number of kernels. */
int rihf_trace(rihf_ctx* ctx, int enable);
int rihf_trace_stats(rihf_ctx* ctx, int max, char* names, double* launches, double* ms, double* work, int* kind);

/* The library's symmetric eigensolver (the diagonalisation step of Alg. 1) on
   one n x n host matrix A (row-major, symmetric): eigenvalues W (n, ascending)
   and eigenvectors V (n x n, column k = eigenvector k).  FP32 parallel Jacobi
   (one CTA up to n = 256, a two-sided block Jacobi over many CTAs above)
   followed by FP64 Ogita-Aishima refinement, on device `device`; n <= 4096.
   Allocates and frees its own device workspace.  Errors: INVALID_ARG, OOM, CUDA. */
int rihf_eigh(int n, const double* A, double* W, double* V, int device);

/* Allocation-free variant of rihf_eigh (the paper has no counterpart: this is a
   service for callers that cannot allocate device memory, such as an MD engine
   that owns a fixed memory pool and forbids cudaMalloc inside its time loop).
   A, W, V are DEVICE pointers: A n x n symmetric (row-major, read only),
   W (n) ascending eigenvalues, V (n x n, column k = eigenvector k); stream is a
   cudaStream_t (NULL = the default stream); its work is queued on it.
   n must not exceed 256: the workspace is one fixed device array in the
   library (about 7.9 MB, held on every GPU that loads the library until exit);
   larger n return RIHF_ERR_INVALID_ARG.  No memory is allocated or freed.
   The first call on each device resolves the array's device address (make it
   before any stream capture).  All calls share the array: calls whose work
   overlaps on the GPU (different streams or host threads) race and must be
   serialised by the caller.  Outside stream capture the call waits for its
   result and checks it: RIHF_ERR_NOT_CONVERGED when max|A V - V diag(W)|
   exceeds 1e-9 n max|W| or max|V^T V - I| exceeds 1e-9 n (a Jacobi pass that
   stopped at its sweep limit, a refinement that did not converge).  Inside a
   stream capture it stays asynchronous and reports argument and launch errors
   only.  Errors: INVALID_ARG, NOT_CONVERGED, CUDA. */
int rihf_eigh_noalloc(int n, const double* A, double* W, double* V, void* stream);

/* C = A B^T on the tensor cores with FP64-class accuracy (the engine of the
   mixed-precision RI-K builds, Eqs. k_ri_2 and tp).  A is M x K, B is N x K,
   C is M x N, all row-major FP64 HOST buffers owned by the caller (inputs
   copied in, C overwritten).  Every row of A and B is split, per K block of
   32 * kblock columns (kblock = 0: all of K in one block), into `digits`
   balanced 8-bit BF16 digits relative to the row's largest exponent in that
   block; the digit pairs (t, u) with t + u <= digits + 1 run as tcgen05 BF16
   MMAs with exact FP32 accumulation in tensor memory, folded into int64 sums
   and converted to FP64 once per output element.  digits = 7 keeps 55 bits of
   max|A row| * max|B row| per K block.  digits in 1..7, K blocks of at most
   60 chunks of 32 (int64 headroom): kblock <= 60, and kblock = 0 needs K <= 1920.  Uses the current device `device`; allocates its own buffers.
   Errors: INVALID_ARG, OOM, CUDA, TIMEOUT (a bounded device wait ran out). */
int rihf_tc_dgemm(int M, int N, int K, const double* A, const double* B, double* C, int digits, int kblock,
                  int device);

/* Learned SCF guess (guess 4 of rihf_scf): an elementwise-shared two-layer MLP
   x (12 features) -> tanh(W1 x + b1) (hidden units) -> y = w2 . h + b2 over the
   lower-triangle density elements mu >= nu, predicting
   (D_{t+1} - D_x) / scale, all densities Loewdin densities (rihf_scf guess 3).
   Features: D_t, D_{t-1}, D_{t-2}, D_x, S_{t+1}, S_t,
   |R_A - R_B| / 10 bohr at t+1, t, t-1 (A, B the atoms of mu, nu), same-atom
   flag, (l_mu + l_nu) / 4, |l_mu - l_nu| / 4.  Weights are used in BF16 (FP32
   master copies), products accumulated in FP32, loss (1/M) sum (y - t)^2,
   Adam (0.9, 0.999, 1e-8).  scale = RMS of the first target.
   rihf_learn_config (re)initialises the network from `seed` (W1 ~
   U(+-1/sqrt(12)), w2 ~ U(+-0.1/sqrt(hidden)), biases 0): hidden in 32..512
   (multiple of 32); the first `train_steps` guess-4 SCFs with enough history
   each run `adam_iters` Adam steps at learning rate lr on their example after
   converging.  Errors: INVALID_ARG, OOM, CUDA. */
int rihf_learn_config(rihf_ctx* ctx, int hidden, int train_steps, int adam_iters, double lr,
                      unsigned long long seed);
/* trained_steps; last_ratio = sum (y - t)^2 / sum t^2 of the last training
   example before its update (below 1: the network beat D_x on an unseen
   example; guess 4 uses the network only below 0.9); last_guess = the guess
   kind the last rihf_scf actually used (0, 1, 2, 3, 4 or 5; guess 4 runs the
   network once it has trained on three examples and the median of its last
   three out-of-sample ratios is below 0.8); scale.  Any pointer may be NULL. */
int rihf_learn_stats(rihf_ctx* ctx, int* trained_steps, double* last_ratio, int* last_guess, double* scale);
/* The network's FP32 master parameters (layout of rihf_mlp_eval) into out;
   INVALID_ARG before rihf_learn_config. */
int rihf_learn_params(rihf_ctx* ctx, float* out);
/* The network's kernels on host buffers (no context): params (mlp_nparams =
   12 hidden + 2 hidden + 1 floats, layout W1[hidden][12], b1, w2, b2) are
   rounded to BF16 as in training; X is M x 12 row-major.  y (M, or NULL) gets
   the forward pass; with targets t (M): grad (params layout) = dL/dparams,
   loss2 = {sum (y - t)^2, sum t^2}; with lr > 0, iters >= 1 and params_out:
   `iters` full-batch Adam steps from zero moments, params_out = the master
   parameters after them and losses[k] (optional) = sum (y - t)^2 before step
   k.  Errors: INVALID_ARG, OOM, CUDA. */
int rihf_mlp_eval(int hidden, int M, const float* params, const float* X, const float* t, float lr, int iters,
                  float* y, float* grad, float* params_out, float* loss2, float* losses, int device);

const char* rihf_strerror(int code);
const char* rihf_last_error(void);
void rihf_destroy(rihf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RIHF_H */
