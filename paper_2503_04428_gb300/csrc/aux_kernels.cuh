// aux_kernels.cuh -- small kernels around the fused sweep.
//
//   validate_kernel  a2 + a9 on a candidate state: rho > 0, P > 0, finite,
//                    and the CFL signal speed max_cells sum_d (|u_d|+c)/h_d
//                    (ideal gas, Eq. 5, or gas + radiation, Eq. 6-7).
//   totals kernels   a10: sum_cells U dV per variable; per-thread compensated
//                    (Kahan) partials in the state precision, FP64 block
//                    trees in a fixed order, so the result is deterministic.
//   monopole         a7 for Eq. 4: shell masses m_i = sum_jk rho dV (FP64),
//                    then M_i = Mc + (4 pi/Omega)(sum_{i'<i} m_i' + m_i/2)
//                    and g_i = -G M_i / r_i^2, in a fixed order.
#pragma once
#include "common.cuh"

namespace hydro {

template <typename T, int DIM, typename G>
__global__ void __launch_bounds__(256)
    validate_kernel(const T* __restrict__ U, long long ncell, int n0, int n1, int nv, G gas,
                    int spherical, const T* __restrict__ w0, const T* __restrict__ w1,
                    const T* __restrict__ w2, const T* __restrict__ ir, const T* __restrict__ is,
                    int* status, unsigned long long* smax_bits, int maxis, T wg) {
  double smax = 0.0;
  int err = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % n0);
    const int j = (int)((c / n0) % n1);
    const int k = (int)(c / ((long long)n0 * n1));
    T u[2 + DIM];
    bool finite = true;
#pragma unroll
    for (int v = 0; v < 2 + DIM; ++v) {
      u[v] = U[(long long)v * ncell + c];
      finite = finite && isfinite(u[v]);
    }
    for (int v = 2 + DIM; v < nv; ++v) finite = finite && isfinite(U[(long long)v * ncell + c]);
    if (!finite) { err = err ? err : ST_NONFINITE; continue; }
    const T rho = u[0];
    T ke = T(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) ke += u[1 + d] * u[1 + d];
    T p, c2;
    if constexpr (G::RAD) {
      gas.from_e(rho, u[1 + DIM] - T(0.5) * ke / rho, p, c2);
    } else {
      p = gas.gm1 * (u[1 + DIM] - T(0.5) * ke / rho);
      c2 = gas.g * p / rho;
    }
    if (!(rho > T(0)) || !(p > T(0))) { err = err ? err : ST_NEG; continue; }
    const T cs = dsqrt(c2);
    // (on a moving axis the speed relative to the faces)
    T sp = (fabs(u[1] / rho - (maxis == 0 ? wg : T(0))) + cs) * w0[i + 2];
    if (DIM >= 2) {
      const T ih = spherical ? w1[j + 2] * ir[i + 2] : w1[j + 2];
      sp += (fabs(u[2] / rho - (maxis == 1 ? wg : T(0))) + cs) * ih;
    }
    if (DIM == 3) {
      const T ih = spherical ? w2[k + 2] * ir[i + 2] * is[j + 2] : w2[k + 2];
      sp += (fabs(u[3] / rho - (maxis == 2 ? wg : T(0))) + cs) * ih;
    }
    smax = fmax(smax, (double)sp);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    const int e2 = __shfl_xor_sync(0xffffffffu, err, o);
    err = err ? err : e2;
  }
  if ((threadIdx.x & 31) == 0) {
    if (smax > 0.0) atomicMax(smax_bits, dbits(smax));
    if (err) atomicCAS(status, 0, err);
  }
}

// Pass 1 of the totals: block b of variable v = blockIdx.y writes its partial.
template <typename T>
__global__ void __launch_bounds__(256)
    totals_partial_kernel(const T* __restrict__ U, long long ncell, int n0, int n1,
                          const double* __restrict__ da, const double* __restrict__ db,
                          const double* __restrict__ dc, double* partial) {
  const int v = blockIdx.y;
  T sum = T(0), comp = T(0);  // Kahan-compensated running sum
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % n0);
    const int j = (int)((c / n0) % n1);
    const int k = (int)(c / ((long long)n0 * n1));
    const T dV = (T)(da[i] * db[j] * dc[k]);
    const T y = U[(long long)v * ncell + c] * dV - comp;
    const T t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  double s = (double)sum - (double)comp;
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long long)v * gridDim.x + blockIdx.x] = red[0];
}

// Pass 2: one thread per variable sums the block partials in order.
__global__ void totals_final_kernel(const double* partial, int nblocks, int nv, double* out) {
  const int v = threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(long long)v * nblocks + b];
  out[v] = s;
}

// Monopole pass 1: partial shell sums sum_{j,k in chunk} rho b_j c_k, for
// 32 radial cells per block and one axis-2 chunk per blockIdx.y.
template <typename T>
__global__ void __launch_bounds__(256)
    shell_partial_kernel(const Ctrl* ctrl, const T* A, const T* B, long long ncell, int n0, int n1,
                         int n2, int kchunk, const double* __restrict__ db,
                         const double* __restrict__ dc, double* partial) {
  if (((volatile const Ctrl*)ctrl)->status != 0) return;
  const T* U = ((volatile const Ctrl*)ctrl)->cur ? B : A;
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int k0 = blockIdx.y * kchunk, k1 = min(k0 + kchunk, n2);
  double s = 0.0;
  if (i < n0) {
    for (int k = k0; k < k1; ++k)
      for (int j = threadIdx.y; j < n1; j += 8)
        s += (double)U[((long long)k * n1 + j) * n0 + i] * (db[j] * dc[k]);
  }
  __shared__ double red[8][33];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && i < n0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
    partial[(long long)blockIdx.y * n0 + i] = t;
  }
}

// Monopole pass 2 (one block of MONO_THREADS): shell masses, their prefix
// sums by a block-wide Hillis-Steele scan (fixed order, so deterministic) and
// the enclosed-mass acceleration of every radial cell.
constexpr int MONO_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(MONO_THREADS)
    monopole_kernel(const Ctrl* ctrl, const double* partial, int nchunks, int n0,
                    const double* __restrict__ da, const double* __restrict__ rc, double G,
                    double Mc, double four_pi_over_omega, double inner, double* shell, T* gmono) {
  if (((volatile const Ctrl*)ctrl)->status != 0) return;
  __shared__ double sh[MONO_THREADS];
  const int tid = threadIdx.x;
  // mass of all shells of the previous chunks, starting from the shells
  // inside this subdomain (0 unless the grid is one slab of an r-split)
  double carry = inner;
  for (int base = 0; base < n0; base += MONO_THREADS) {
    const int i = base + tid;
    double m = 0.0;
    if (i < n0) {
      double s = 0.0;
      for (int q = 0; q < nchunks; ++q) s += partial[(long long)q * n0 + i];
      m = s * da[i];
    }
    sh[tid] = m;
    __syncthreads();
    for (int off = 1; off < MONO_THREADS; off <<= 1) {
      const double v = tid >= off ? sh[tid - off] : 0.0;
      __syncthreads();
      sh[tid] += v;
      __syncthreads();
    }
    const double below = carry + (tid > 0 ? sh[tid - 1] : 0.0);
    if (i < n0) {
      const double M = Mc + four_pi_over_omega * (below + 0.5 * m);
      gmono[i] = (T)(-G * M / (rc[i] * rc[i]));
      shell[i] = M;
    }
    carry += sh[MONO_THREADS - 1];
    __syncthreads();
  }
}

// Shell masses m_i = (sum of the chunk partials) * a_i, summed as in
// monopole_kernel, for the caller of a domain-decomposed run.
__global__ void shell_mass_kernel(const double* partial, int nchunks, int n0, const double* __restrict__ da,
                                  double* m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  double s = 0.0;
  for (int q = 0; q < nchunks; ++q) s += partial[(long long)q * n0 + i];
  m[i] = s * da[i];
}

// The 2 boundary layers of a state at side `side` of axis `axis`, as
// [v][layer][cross section] (layer l = the cell at distance l from the side;
// the cross section runs over the two other axes, the lower one fastest):
// the halo that the neighbouring subdomain reads.
template <typename T>
__global__ void pack_boundary_kernel(const Ctrl* ctrl, const T* A, const T* B, long long ncell, int n0, int n1,
                                     int n2, int nv, int axis, int side, T* out) {
  const T* U = ((volatile const Ctrl*)ctrl)->cur ? B : A;
  const int na = axis == 0 ? n0 : axis == 1 ? n1 : n2;
  const long long nx = axis == 0 ? (long long)n1 * n2 : axis == 1 ? (long long)n0 * n2 : (long long)n0 * n1;
  const long long total = (long long)nv * 2 * nx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long q = t % nx;
    const int l = (int)((t / nx) % 2);
    const int v = (int)(t / (2 * nx));
    const int g = side == 0 ? min(l, na - 1) : max(na - 1 - l, 0);
    long long c;
    if (axis == 0) c = q * n0 + g;                                          // q = k n1 + j
    else if (axis == 1) c = ((q / n0) * n1 + g) * n0 + q % n0;            // q = k n0 + i
    else c = (long long)g * n1 * n0 + q;                                   // q = j n0 + i
    out[t] = U[(long long)v * ncell + c];
  }
}

}  // namespace hydro
