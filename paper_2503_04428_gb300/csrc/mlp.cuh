// mlp.cuh -- training of the star-pressure guess network on the GPU.
//
// Network: x (6) -> SiLU(W1 x + b1) (64) -> SiLU(W2 h1 + b2) (64) -> w3.h2 + b3,
// FP32 weights, loss = mean (y - t)^2 with t = ln(p_star / p_ref),
// p_ref = sqrt(P_L P_R).  Only faces that pass mlp_gate (the only faces where
// the network is used) are trained on.
// One CTA handles 64 samples: the three layers and their reverse-mode
// derivatives are small dense products done in shared memory; each CTA
// writes its partial gradient, and a second kernel sums the partials in a
// fixed order (deterministic), then Adam (Kingma & Ba 2015) updates the
// weights.
#pragma once
#include "common.cuh"

namespace hydro {

constexpr int MLP_SB = 64;  // samples per CTA

struct MlpSmem {
  float w[MLP_NPARAM];
  float x[MLP_SB][MLP_IN];
  float z1[MLP_SB][MLP_H];   // later G1
  float h1[MLP_SB][MLP_H];
  float z2[MLP_SB][MLP_H];
  float h2[MLP_SB][MLP_H];   // later G2
  float gy[MLP_SB];
  float loss[MLP_SB];
};

__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// Features, targets and the "network is used here" flag (Toro's rule picks
// the two-shock estimate) from face states (double) -- once per training set.
__global__ void mlp_features_kernel(const double* faces6, const double* log_pstar, long long n,
                                    Gas<double> gas, float* X, float* Y, unsigned char* use) {
  const double gamma = gas.g;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* f = faces6 + 6 * i;
  const double rref = sqrt(f[0] * f[3]);
  const double pref = sqrt(f[2] * f[5]);
  const double icref = 1.0 / sqrt(gamma * pref / rref);
  X[6 * i + 0] = (float)log(f[0] / rref);
  X[6 * i + 1] = (float)log(f[3] / rref);
  X[6 * i + 2] = (float)log(f[2] / pref);
  X[6 * i + 3] = (float)log(f[5] / pref);
  X[6 * i + 4] = (float)(f[1] * icref);
  X[6 * i + 5] = (float)(f[4] * icref);
  if (Y) Y[i] = (float)(log_pstar[i] - log(pref));
  if (use) {
    const double cL = sqrt(gamma * f[2] / f[0]), cR = sqrt(gamma * f[5] / f[3]);
    int kind;
    toro_guess<double>(f[0], f[1], f[2], cL, f[3], f[4], f[5], cR, gas, kind);
    use[i] = mlp_gate<double>(kind, f[2], f[5]);
  }
}

// Forward + backward of 64 samples per CTA.  Samples are X[idx[first + s]]
// (idx may be null: identity); `count` samples in total, gradient scaled by
// inv_n.  Writes partial[blockIdx.x][p] and loss_partial[blockIdx.x].
__global__ void __launch_bounds__(256)
    mlp_grad_kernel(const float* __restrict__ W, const float* __restrict__ X,
                    const float* __restrict__ Y, const int* __restrict__ idx, long long first,
                    long long count, float inv_n, float* partial, double* loss_partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int p = tid; p < MLP_NPARAM; p += 256) s.w[p] = W[p];
  const long long s0 = (long long)blockIdx.x * MLP_SB;
  for (int q = tid; q < MLP_SB * MLP_IN; q += 256) {
    const int sm = q / MLP_IN, i = q % MLP_IN;
    const long long g = s0 + sm;
    float v = 0.f;
    if (g < count) {
      const long long row = idx ? idx[first + g] : first + g;
      v = X[row * MLP_IN + i];
    }
    s.x[sm][i] = v;
  }
  __syncthreads();
  // layer 1
  for (int q = tid; q < MLP_SB * MLP_H; q += 256) {
    const int sm = q / MLP_H, o = q % MLP_H;
    float a = s.w[MB1 + o];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) a = fmaf(s.w[MW1 + o * MLP_IN + i], s.x[sm][i], a);
    s.z1[sm][o] = a;
    s.h1[sm][o] = silu_f(a);
  }
  __syncthreads();
  // layer 2
  for (int q = tid; q < MLP_SB * MLP_H; q += 256) {
    const int sm = q / MLP_H, o = q % MLP_H;
    float a = s.w[MB2 + o];
#pragma unroll 16
    for (int i = 0; i < MLP_H; ++i) a = fmaf(s.w[MW2 + o * MLP_H + i], s.h1[sm][i], a);
    s.z2[sm][o] = a;
    s.h2[sm][o] = silu_f(a);
  }
  __syncthreads();
  // output, loss and dL/dy
  if (tid < MLP_SB) {
    const long long g = s0 + tid;
    float y = s.w[MB3];
    for (int i = 0; i < MLP_H; ++i) y = fmaf(s.w[MW3 + i], s.h2[tid][i], y);
    float r = 0.f;
    if (g < count) {
      const long long row = idx ? idx[first + g] : first + g;
      r = y - Y[row];
    }
    s.loss[tid] = r * r;
    s.gy[tid] = 2.0f * r * inv_n;
  }
  __syncthreads();
  float* P = partial + (long long)blockIdx.x * MLP_NPARAM;
  // output layer gradients
  if (tid < MLP_H) {
    float a = 0.f;
    for (int sm = 0; sm < MLP_SB; ++sm) a = fmaf(s.gy[sm], s.h2[sm][tid], a);
    P[MW3 + tid] = a;
  }
  if (tid == MLP_H) {
    float a = 0.f;
    double l = 0.0;
    for (int sm = 0; sm < MLP_SB; ++sm) {
      a += s.gy[sm];
      l += s.loss[sm];
    }
    P[MB3] = a;
    loss_partial[blockIdx.x] = l;
  }
  __syncthreads();
  // G2 = dL/dz2 (into h2)
  for (int q = tid; q < MLP_SB * MLP_H; q += 256) {
    const int sm = q / MLP_H, o = q % MLP_H;
    s.h2[sm][o] = s.gy[sm] * s.w[MW3 + o] * dsilu_f(s.z2[sm][o]);
  }
  __syncthreads();
  // dW2 = G2^T h1, db2 = sum G2
  for (int q = tid; q < MLP_H * MLP_H; q += 256) {
    const int o = q / MLP_H, i = q % MLP_H;
    float a = 0.f;
    for (int sm = 0; sm < MLP_SB; ++sm) a = fmaf(s.h2[sm][o], s.h1[sm][i], a);
    P[MW2 + q] = a;
  }
  if (tid < MLP_H) {
    float a = 0.f;
    for (int sm = 0; sm < MLP_SB; ++sm) a += s.h2[sm][tid];
    P[MB2 + tid] = a;
  }
  // G1 = (G2 W2) * silu'(z1)  (into z2, no longer needed)
  for (int q = tid; q < MLP_SB * MLP_H; q += 256) {
    const int sm = q / MLP_H, i = q % MLP_H;
    float a = 0.f;
#pragma unroll 16
    for (int o = 0; o < MLP_H; ++o) a = fmaf(s.h2[sm][o], s.w[MW2 + o * MLP_H + i], a);
    s.z2[sm][i] = a * dsilu_f(s.z1[sm][i]);
  }
  __syncthreads();
  // dW1 = G1^T x, db1 = sum G1
  for (int q = tid; q < MLP_H * MLP_IN; q += 256) {
    const int o = q / MLP_IN, i = q % MLP_IN;
    float a = 0.f;
    for (int sm = 0; sm < MLP_SB; ++sm) a = fmaf(s.z2[sm][o], s.x[sm][i], a);
    P[MW1 + q] = a;
  }
  if (tid < MLP_H) {
    float a = 0.f;
    for (int sm = 0; sm < MLP_SB; ++sm) a += s.z2[sm][tid];
    P[MB1 + tid] = a;
  }
}

// Sum the per-CTA partial gradients in a fixed order (FP64).
__global__ void mlp_reduce_kernel(const float* partial, int nblocks, double* grad,
                                  const double* loss_partial, double* loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAM) {
    double a = 0.0;
    for (int b = 0; b < nblocks; ++b) a += (double)partial[(long long)b * MLP_NPARAM + p];
    grad[p] = a;
  }
  if (p == 0 && loss_out) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += loss_partial[b];
    *loss_out += l;
  }
}

// Fixed-order sum of the partial gradients followed by the Adam update of
// that parameter (one thread per parameter); the loss partials go to loss_acc.
__global__ void mlp_reduce_adam_kernel(const float* partial, int nblocks, const double* loss_partial,
                                       double* loss_acc, float* W, float* m, float* v, int step,
                                       double lr, double b1, double b2, double eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += loss_partial[b];
    *loss_acc += l;
  }
  if (p >= MLP_NPARAM) return;
  double g = 0.0;
  for (int b = 0; b < nblocks; ++b) g += (double)partial[(long long)b * MLP_NPARAM + p];
  const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
  const double mm = b1 * m[p] + (1.0 - b1) * g;
  const double vv = b2 * v[p] + (1.0 - b2) * g * g;
  m[p] = (float)mm;
  v[p] = (float)vv;
  W[p] = (float)(W[p] - lr * (mm / c1) / (sqrt(vv / c2) + eps));
}

// Adam with bias-corrected moments; arithmetic in FP64, storage in FP32.
__global__ void adam_kernel(float* W, float* m, float* v, const double* grad, int step, double lr,
                            double b1, double b2, double eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
  const double g = grad[p];
  const double mm = b1 * m[p] + (1.0 - b1) * g;
  const double vv = b2 * v[p] + (1.0 - b2) * g * g;
  m[p] = (float)mm;
  v[p] = (float)vv;
  W[p] = (float)(W[p] - lr * (mm / c1) / (sqrt(vv / c2) + eps));
}

}  // namespace hydro
