// Learned SCF guess (mlp.cu): an elementwise-shared two-layer MLP over the
// lower-triangle density elements D_{mu nu} (mu >= nu) of an AIMD trajectory,
//   z = W1 x + b1,  h = tanh(z),  y = w2 . h + b2,
// predicting the correction to the three-point extrapolation
//   D_x = 3 D_t - 3 D_{t-1} + D_{t-2}.
// Weights are used in BF16 (rounded from FP32 master copies), all products are
// accumulated in FP32; training minimises the mean squared error with Adam.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace rihf {

constexpr int kMlpF = 12;         // features per element
constexpr int kMlpMaxH = 512;     // hidden width limit (one thread per unit)

// Parameter layout (FP32 master and BF16 working copies use the same order):
//   W1 [H][F], b1 [H], w2 [H], b2 [1]
inline int mlp_nparams(int H) { return H * kMlpF + 2 * H + 1; }

struct MlpDev {
  int H = 0;
  float* master = nullptr;        // FP32 parameters
  uint16_t* wbf = nullptr;        // BF16 parameters used by the kernels
  float* grad = nullptr;          // FP32 gradient accumulator
  float* m = nullptr;             // Adam moments
  float* v = nullptr;
  float* loss = nullptr;          // [0] sum (y - t)^2, [1] sum t^2
  long long adam_t = 0;
};

// BF16 working copy from the FP32 master (round to nearest even).
void mlp_round_weights(cudaStream_t s, const MlpDev& net);

// y[e] = MLP(X[e]) for e < M (X row-major M x kMlpF, FP32).
void mlp_forward(cudaStream_t s, const MlpDev& net, const float* X, int M, float* y);

// Gradient of L = (1/M) sum_e (y_e - t_e)^2 into net.grad (zeroed first) and
// loss[0] = sum (y - t)^2, loss[1] = sum t^2.
void mlp_backward(cudaStream_t s, const MlpDev& net, const float* X, const float* t, int M);

// One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) of the master weights from
// net.grad, then the BF16 copy.
void mlp_adam(cudaStream_t s, MlpDev& net, float lr);

// Features of element e = mu (mu + 1) / 2 + nu of the lower triangle, the
// history D_t, D_{t-1}, D_{t-2}, S_{t+1}, S_t and the atom-pair distances
// r = |R_A - R_B| (A, B the atoms of mu and nu) at t+1, t, t-1 re-expressed as
// well-scaled differences:
//   D_t, (D_t - D_{t-1}) / sd, (D_{t-1} - D_{t-2}) / sd, (D_t - 2 D_{t-1} + D_{t-2}) / sd,
//   S_{t+1}, (S_{t+1} - S_t) / ss, r_{t+1} / 10, (r_{t+1} - r_t) / sr, (r_t - r_{t-1}) / sr,
//   same-atom flag, (l_mu + l_nu) / 4, |l_mu - l_nu| / 4,
// and D_x = 3 D_t - 3 D_{t-1} + D_{t-2} into Dx[e].  xyz* are natoms x 3 (bohr).
void mlp_features(cudaStream_t s, int N, const double* D0, const double* D1, const double* D2, const double* S1,
                  const double* S0, const double* xyz1, const double* xyz0, const double* xyzm, const int* ao_atom,
                  const int* ao_l, double sd, double ss, double sr, float* X, double* Dx);

// Sums over the lower triangle of (D0 - D1)^2, (S1 - S0)^2 and (r_{t+1} - r_t)^2
// into out[0..2] (the feature scales are their RMS at the first build).
void mlp_scale_sums(cudaStream_t s, int N, const double* D0, const double* D1, const double* S1, const double* S0,
                    const double* xyz1, const double* xyz0, const int* ao_atom, double* out);

// Dpred (N x N, symmetric) = Dx + scale * y on the lower triangle, mirrored.
void mlp_apply(cudaStream_t s, int N, const double* Dx, const float* y, double scale, double* Dpred);

// Training target t[e] = (Dconv[mu nu] - Dx[e]) / scale.
void mlp_target(cudaStream_t s, int N, const double* Dconv, const double* Dx, double scale, float* t);

}  // namespace rihf
