// Learned SCF guess kernels: features, forward, fused forward + backward, Adam.
// One thread per hidden unit; a block walks tiles of kTE elements whose
// features sit in shared memory, so every weight is read once per block.
#include <algorithm>
#include <cmath>

#include "mlp.cuh"

namespace rihf {

namespace {

constexpr int kTE = 32;   // elements per tile

__device__ inline float bf16_to_f32(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ inline uint16_t f32_to_bf16(float f) {
  // round to nearest even (finite inputs)
  uint32_t u = __float_as_uint(f);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

__device__ inline void decode_lower(long long e, int& mu, int& nu) {
  int m = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
  while ((long long)m * (m + 1) / 2 > e) --m;
  while ((long long)(m + 1) * (m + 2) / 2 <= e) ++m;
  mu = m;
  nu = (int)(e - (long long)m * (m + 1) / 2);
}

struct UnitWeights {
  float w1[kMlpF];
  float b1, w2, b2;
};

__device__ inline UnitWeights load_unit(const uint16_t* __restrict__ w, int H, int j) {
  UnitWeights u;
#pragma unroll
  for (int f = 0; f < kMlpF; ++f) u.w1[f] = bf16_to_f32(w[j * kMlpF + f]);
  u.b1 = bf16_to_f32(w[H * kMlpF + j]);
  u.w2 = bf16_to_f32(w[H * kMlpF + H + j]);
  u.b2 = bf16_to_f32(w[H * kMlpF + 2 * H]);
  return u;
}

// One tile: xs [kTE][kMlpF] <- X, hs [kTE][H] <- tanh(W1 x + b1),
// ys [kTE] <- w2 . h + b2 (w2s [H] holds the BF16-rounded w2 in FP32).
__device__ inline void tile_forward(const UnitWeights& u, int H, const float* __restrict__ X, int M, int e0,
                                    float* xs, float* hs, const float* w2s, float* ys) {
  const int j = threadIdx.x, nt = blockDim.x;
  for (int i = j; i < kTE * kMlpF; i += nt) {
    const int e = e0 + i / kMlpF;
    xs[i] = e < M ? X[(size_t)e0 * kMlpF + i] : 0.f;
  }
  __syncthreads();
  for (int e = 0; e < kTE; ++e) {
    float z = u.b1;
#pragma unroll
    for (int f = 0; f < kMlpF; ++f) z = fmaf(u.w1[f], xs[e * kMlpF + f], z);
    hs[e * H + j] = tanhf(z);
  }
  __syncthreads();
  const int warp = j >> 5, lane = j & 31, nw = nt >> 5;
  for (int e = warp; e < kTE; e += nw) {
    float s = 0.f;
    for (int k = lane; k < H; k += 32) s = fmaf(w2s[k], hs[e * H + k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ys[e] = s + u.b2;
  }
  __syncthreads();
}

__global__ void mlp_round_kernel(const float* __restrict__ master, uint16_t* __restrict__ wbf, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    wbf[i] = f32_to_bf16(master[i]);
}

__global__ void mlp_fwd_kernel(const uint16_t* __restrict__ w, int H, const float* __restrict__ X, int M,
                               float* __restrict__ y) {
  extern __shared__ float sm[];
  float* xs = sm;
  float* hs = xs + kTE * kMlpF;
  float* w2s = hs + kTE * H;
  float* ys = w2s + H;
  const int j = threadIdx.x;
  const UnitWeights u = load_unit(w, H, j);
  w2s[j] = u.w2;
  for (int e0 = blockIdx.x * kTE; e0 < M; e0 += gridDim.x * kTE) {
    tile_forward(u, H, X, M, e0, xs, hs, w2s, ys);
    for (int e = j; e < kTE; e += blockDim.x)
      if (e0 + e < M) y[e0 + e] = ys[e];
    __syncthreads();
  }
}

// Fused forward + backward of L = (1/M) sum (y - t)^2: per unit j the block
// accumulates dW1[j][:], db1[j], dw2[j] over its tiles in registers and adds
// them to grad once; db2 and the loss sums go through warp reductions.
__global__ void mlp_bwd_kernel(const uint16_t* __restrict__ w, int H, const float* __restrict__ X,
                               const float* __restrict__ t, int M, float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* xs = sm;
  float* hs = xs + kTE * kMlpF;
  float* w2s = hs + kTE * H;
  float* ys = w2s + H;
  float* gs = ys + kTE;
  const int j = threadIdx.x;
  const UnitWeights u = load_unit(w, H, j);
  w2s[j] = u.w2;
  float dW1[kMlpF];
#pragma unroll
  for (int f = 0; f < kMlpF; ++f) dW1[f] = 0.f;
  float db1 = 0.f, dw2 = 0.f, db2 = 0.f, l0 = 0.f, l1 = 0.f;
  const float inv_m2 = 2.f / (float)M;
  for (int e0 = blockIdx.x * kTE; e0 < M; e0 += gridDim.x * kTE) {
    tile_forward(u, H, X, M, e0, xs, hs, w2s, ys);
    for (int e = j; e < kTE; e += blockDim.x) {
      const bool ok = e0 + e < M;
      const float r = ok ? ys[e] - t[e0 + e] : 0.f;
      gs[e] = r * inv_m2;
      if (ok) {
        l0 += r * r;
        l1 += t[e0 + e] * t[e0 + e];
        db2 += r * inv_m2;
      }
    }
    __syncthreads();
    for (int e = 0; e < kTE; ++e) {
      const float g = gs[e], h = hs[e * H + j];
      const float dz = g * u.w2 * (1.f - h * h);
      dw2 = fmaf(g, h, dw2);
      db1 += dz;
#pragma unroll
      for (int f = 0; f < kMlpF; ++f) dW1[f] = fmaf(dz, xs[e * kMlpF + f], dW1[f]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int f = 0; f < kMlpF; ++f) atomicAdd(grad + j * kMlpF + f, dW1[f]);
  atomicAdd(grad + H * kMlpF + j, db1);
  atomicAdd(grad + H * kMlpF + H + j, dw2);
  // db2 and loss partials live on threads j < kTE
  for (int o = 16; o > 0; o >>= 1) {
    db2 += __shfl_xor_sync(0xffffffffu, db2, o);
    l0 += __shfl_xor_sync(0xffffffffu, l0, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  if (j == 0) {
    atomicAdd(grad + H * kMlpF + 2 * H, db2);
    atomicAdd(loss, l0);
    atomicAdd(loss + 1, l1);
  }
}

__global__ void mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int n, float lr, float bc1, float bc2,
                                uint16_t* __restrict__ wbf) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    wbf[i] = f32_to_bf16(pi);
  }
}

__global__ void mlp_features_kernel(int N, const double* __restrict__ D0, const double* __restrict__ D1,
                                    const double* __restrict__ D2, const double* __restrict__ S1,
                                    const double* __restrict__ S0, const double* __restrict__ xyz1,
                                    const double* __restrict__ xyz0, const double* __restrict__ xyzm,
                                    const int* __restrict__ ao_atom, const int* __restrict__ ao_l, double isd,
                                    double iss, double isr, float* __restrict__ X, double* __restrict__ Dx) {
  const long long M = (long long)N * (N + 1) / 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M;
       e += (long long)gridDim.x * blockDim.x) {
    int mu, nu;
    decode_lower(e, mu, nu);
    const size_t ij = (size_t)mu * N + nu;
    const double d0 = D0[ij], d1 = D1[ij], d2 = D2[ij];
    const double dx = 3.0 * d0 - 3.0 * d1 + d2;
    Dx[e] = dx;
    const int A = ao_atom[mu], B = ao_atom[nu];
    auto dist = [&](const double* R) {
      const double x = R[3 * A] - R[3 * B], y = R[3 * A + 1] - R[3 * B + 1], z = R[3 * A + 2] - R[3 * B + 2];
      return sqrt(x * x + y * y + z * z);
    };
    const double r1 = dist(xyz1), r0 = dist(xyz0), rm = dist(xyzm);
    float* xe = X + e * kMlpF;
    xe[0] = (float)d0;
    xe[1] = (float)((d0 - d1) * isd);
    xe[2] = (float)((d1 - d2) * isd);
    xe[3] = (float)((d0 - 2.0 * d1 + d2) * isd);
    xe[4] = (float)S1[ij];
    xe[5] = (float)((S1[ij] - S0[ij]) * iss);
    xe[6] = (float)(0.1 * r1);
    xe[7] = (float)((r1 - r0) * isr);
    xe[8] = (float)((r0 - rm) * isr);
    xe[9] = A == B ? 1.f : 0.f;
    xe[10] = 0.25f * (float)(ao_l[mu] + ao_l[nu]);
    xe[11] = 0.25f * (float)abs(ao_l[mu] - ao_l[nu]);
  }
}

__global__ void mlp_scale_kernel(int N, const double* __restrict__ D0, const double* __restrict__ D1,
                                 const double* __restrict__ S1, const double* __restrict__ S0,
                                 const double* __restrict__ xyz1, const double* __restrict__ xyz0,
                                 const int* __restrict__ ao_atom, double* __restrict__ out) {
  const long long M = (long long)N * (N + 1) / 2;
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M;
       e += (long long)gridDim.x * blockDim.x) {
    int mu, nu;
    decode_lower(e, mu, nu);
    const size_t ij = (size_t)mu * N + nu;
    const double dd = D0[ij] - D1[ij], ds = S1[ij] - S0[ij];
    const int A = ao_atom[mu], B = ao_atom[nu];
    double r1 = 0.0, r0 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double x1 = xyz1[3 * A + k] - xyz1[3 * B + k], x0 = xyz0[3 * A + k] - xyz0[3 * B + k];
      r1 += x1 * x1;
      r0 += x0 * x0;
    }
    const double dr = sqrt(r1) - sqrt(r0);
    a += dd * dd;
    b += ds * ds;
    c += dr * dr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, a);
    atomicAdd(out + 1, b);
    atomicAdd(out + 2, c);
  }
}

__global__ void mlp_apply_kernel(int N, const double* __restrict__ Dx, const float* __restrict__ y, double scale,
                                 double* __restrict__ Dp) {
  const long long M = (long long)N * (N + 1) / 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M;
       e += (long long)gridDim.x * blockDim.x) {
    int mu, nu;
    decode_lower(e, mu, nu);
    const double v = Dx[e] + (y ? scale * (double)y[e] : 0.0);
    Dp[(size_t)mu * N + nu] = v;
    Dp[(size_t)nu * N + mu] = v;
  }
}

__global__ void mlp_target_kernel(int N, const double* __restrict__ Dc, const double* __restrict__ Dx, double inv_scale,
                                  float* __restrict__ t) {
  const long long M = (long long)N * (N + 1) / 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M;
       e += (long long)gridDim.x * blockDim.x) {
    int mu, nu;
    decode_lower(e, mu, nu);
    t[e] = (float)((Dc[(size_t)mu * N + nu] - Dx[e]) * inv_scale);
  }
}

int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)std::min<long long>(std::max<long long>(b, 1), 4096);
}

size_t tile_smem(int H) { return sizeof(float) * (kTE * kMlpF + kTE * H + H + 2 * kTE); }

void check_h(int H) {
  if (H < 32 || H > kMlpMaxH || H % 32) throw RihfError(-1, "MLP hidden width must be a multiple of 32 in 32..512");
}

}  // namespace

void mlp_round_weights(cudaStream_t s, const MlpDev& net) {
  const int n = mlp_nparams(net.H);
  mlp_round_kernel<<<blocks_for(n, 256), 256, 0, s>>>(net.master, net.wbf, n);
  RIHF_LAUNCH_CHECK();
}

void mlp_forward(cudaStream_t s, const MlpDev& net, const float* X, int M, float* y) {
  check_h(net.H);
  if (M <= 0) return;
  const size_t smem = tile_smem(net.H);
  if (smem > 48 * 1024) raise_smem_limit((const void*)mlp_fwd_kernel, (int)smem);
  const int tiles = (M + kTE - 1) / kTE;
  mlp_fwd_kernel<<<std::min(tiles, 1024), net.H, smem, s>>>(net.wbf, net.H, X, M, y);
  RIHF_LAUNCH_CHECK();
}

void mlp_backward(cudaStream_t s, const MlpDev& net, const float* X, const float* t, int M) {
  check_h(net.H);
  RIHF_CUDA(cudaMemsetAsync(net.grad, 0, sizeof(float) * mlp_nparams(net.H), s));
  RIHF_CUDA(cudaMemsetAsync(net.loss, 0, 2 * sizeof(float), s));
  if (M <= 0) return;
  const size_t smem = tile_smem(net.H);
  if (smem > 48 * 1024) raise_smem_limit((const void*)mlp_bwd_kernel, (int)smem);
  const int tiles = (M + kTE - 1) / kTE;
  mlp_bwd_kernel<<<std::min(tiles, 304), net.H, smem, s>>>(net.wbf, net.H, X, t, M, net.grad, net.loss);
  RIHF_LAUNCH_CHECK();
}

void mlp_adam(cudaStream_t s, MlpDev& net, float lr) {
  const int n = mlp_nparams(net.H);
  ++net.adam_t;
  const float bc1 = 1.f - powf(0.9f, (float)net.adam_t), bc2 = 1.f - powf(0.999f, (float)net.adam_t);
  mlp_adam_kernel<<<blocks_for(n, 256), 256, 0, s>>>(net.master, net.grad, net.m, net.v, n, lr, bc1, bc2, net.wbf);
  RIHF_LAUNCH_CHECK();
}

void mlp_features(cudaStream_t s, int N, const double* D0, const double* D1, const double* D2, const double* S1,
                  const double* S0, const double* xyz1, const double* xyz0, const double* xyzm, const int* ao_atom,
                  const int* ao_l, double sd, double ss, double sr, float* X, double* Dx) {
  const long long M = (long long)N * (N + 1) / 2;
  mlp_features_kernel<<<blocks_for(M, 256), 256, 0, s>>>(N, D0, D1, D2, S1, S0, xyz1, xyz0, xyzm, ao_atom, ao_l,
                                                         1.0 / sd, 1.0 / ss, 1.0 / sr, X, Dx);
  RIHF_LAUNCH_CHECK();
}

void mlp_scale_sums(cudaStream_t s, int N, const double* D0, const double* D1, const double* S1, const double* S0,
                    const double* xyz1, const double* xyz0, const int* ao_atom, double* out) {
  const long long M = (long long)N * (N + 1) / 2;
  RIHF_CUDA(cudaMemsetAsync(out, 0, 3 * sizeof(double), s));
  mlp_scale_kernel<<<std::min(blocks_for(M, 256), 304), 256, 0, s>>>(N, D0, D1, S1, S0, xyz1, xyz0, ao_atom, out);
  RIHF_LAUNCH_CHECK();
}

void mlp_apply(cudaStream_t s, int N, const double* Dx, const float* y, double scale, double* Dpred) {
  const long long M = (long long)N * (N + 1) / 2;
  mlp_apply_kernel<<<blocks_for(M, 256), 256, 0, s>>>(N, Dx, y, scale, Dpred);
  RIHF_LAUNCH_CHECK();
}

void mlp_target(cudaStream_t s, int N, const double* Dconv, const double* Dx, double scale, float* t) {
  const long long M = (long long)N * (N + 1) / 2;
  mlp_target_kernel<<<blocks_for(M, 256), 256, 0, s>>>(N, Dconv, Dx, 1.0 / scale, t);
  RIHF_LAUNCH_CHECK();
}

}  // namespace rihf
