// common.cuh -- argument blocks shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <map>
#include <set>
#include <utility>

#include "physics.cuh"

namespace hydro {

// BC_EXCHANGED: a side whose ghosts are a neighbouring subdomain's cells,
// supplied by the caller (domain decomposition, Sect. 3.3.1).
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_EXCHANGED = 3 };
enum { GRAV_NONE = 0, GRAV_UNIFORM = 1, GRAV_POINT = 2, GRAV_MONO = 3 };
enum { HEAT_NONE = 0, HEAT_CONST = 1, HEAT_NI56 = 2 };

// Device-resident control block of one handle.  Every step kernel reads it at
// start; the last CTA of a launch (ticket counter `done`) commits the step:
// it flips `cur`, advances t and step, and moves the next-state signal speed
// into smax_cur.  A failing launch never commits, so the input buffer of the
// failing step stays the current state.
struct Ctrl {
  double smax_cur;                  // max_cells sum_d (|u_d|+c)/h_d of the current state
  unsigned long long smax_next;     // same for the state being written (bits of a double >= 0)
  double t;                         // simulation time of the current state
  double last_dt;
  long long step;                   // committed steps
  long long err_step;               // step index of the first failure (-1 none)
  int status;                       // 0 or a hydro_status code
  int cur;                          // index of the buffer holding the current state
  unsigned int done;                // CTA tickets of the running launch
  unsigned int pad;
  unsigned long long iters;         // Newton iterations (exact solver)
  unsigned long long fallbacks;     // first-order face-state fallbacks
  unsigned long long mlp;           // faces whose guess came from the MLP
};

// Per-axis geometry, precomputed on the host in FP64 and stored as T.
// "ext" arrays are indexed by cell index + 2 for cells -2..n+1 (ghosts use
// the mirrored or wrapped interior widths); the others by interior cell
// (n entries) or interior face (n+1 entries).
template <typename T>
struct Geom {
  const T* inv_dxc[3];  // ext: 1/(x_i - x_{i-1})
  const T* hw[3];       // ext: half coordinate width
  const T* inv_w[3];    // ext: 1/coordinate width
  const T* inv_r;       // ext axis 0: 1/r_i (spherical)
  const T* inv_s;       // ext axis 1: 1/s_j, s_j = (sin th_- + sin th_+)/2 (spherical)
  const T* Af;          // axis-0 faces: r_f^2 (spherical) or 1
  const T* inva;        // axis 0: 1/a_i, a = (r+^3 - r-^3)/3 or dx
  const T* ga;          // axis 0: a2_i/a_i, a2 = (r+^2 - r-^2)/2 or dx
  const T* qr;          // axis 0: (r+ - r-)/((r+ + r-) a_i)
  const T* gr;          // axis 0: (Af_{i+1} - Af_i)/a_i
  const T* gpt;         // axis 0: point-mass acceleration -G Mc/r_i^2
  const T* Bf;          // axis-1 faces: sin th_f (spherical) or 1
  const T* invb;        // axis 1: 1/b_j, b = cos th_- - cos th_+ or dy
  const T* zc;          // axis 1: b3_j/b_j, b3 = dth or dy
  const T* gt;          // axis 1: (Bf_{j+1} - Bf_j)/b_j
  const T* qt;          // axis 1: (s+ - s-)/((s+ + s-) b_j)
  const T* invc;        // axis 2: 1/c_k, c = dphi or dz
};

template <typename T>
struct SweepArgs {
  const T* A;             // state buffer 0
  T* B;                   // state buffer 1 (in/out chosen by ctrl->cur)
  T* Aw;                  // writable alias of A
  int n[3];
  long long ncell;
  int bc[3][2];
  int ns;                 // passive scalars in use (<= the kernel's NSX)
  int limiter;
  int spherical;
  int gravity;
  T g0[3];
  const T* gmono;         // monopole acceleration per radial cell (device)
  int heating;
  int ni_index;
  T heat_q;               // CONST: volumetric rate
  double ni_lambda, ni_a, ni_qco, ni_tni, ni_tco;  // Eq. 8 constants (CGS)
  Gas<T> gas;
  GasRad<T> grad;         // gas + radiation constants (kernels instantiated for Eq. 6-7)
  T eps_dual;             // dual-energy criterion epsilon (Sect. 2.5); 0 = off
  double dt_host;         // > 0: use this dt; otherwise CFL on the device
  double cfl;
  double t_end;           // > 0: clip dt so t does not pass t_end
  int zchunk;             // planes per CTA along axis 2 (3D)
  Ctrl* ctrl;
  Geom<T> geo;
  // domain decomposition: the axis whose sides may be BC_EXCHANGED (-1 none)
  // and their ghost layers [v][layer][cross section] (layer l = the ghost at
  // distance l+1 from the side; the cross section runs over the two other
  // axes, the lower one fastest)
  int xaxis;
  const T* halo[2];
  // moving grid (Sect. 3.1.1): the faces of axis maxis (-1 none) move with
  // velocity wg; vr (spherical radial motion, else null) = a_old/a_new per
  // radial cell, the volume ratio that spreads a cell's content over its
  // new volume
  int maxis;
  T wg;
  const T* vr;
  const T* ir_new;  // moving radial grid: 1/r of every radial cell after the step (its CFL widths)
  // conserved totals of the new state, accumulated in the step (a10): per
  // CTA and variable, sum over the CTA's cells of U dV in FP64, stored
  // [v][cta] (cta = blockIdx.x + gridDim.x (blockIdx.y + gridDim.y
  // blockIdx.z)); null: not accumulated
  double* tot_part;
  const double* dvol[3];  // dV of cell (i, j, k) = dvol[0][i] dvol[1][j] dvol[2][k] (FP64)
  const float2* dvz32;    // dvol[2][k] as an FP32 pair (hi, lo) with hi + lo = dvol[2][k] to ~2^-48
};

template <typename T, int DIM>
cudaError_t sweep_dispatch(const SweepArgs<T>& a, int nsx, int rs, cudaStream_t s, int* tx, int* ty,
                           int* nt);
// The same with the dual-energy correction (Sect. 2.5).
template <typename T, int DIM>
cudaError_t sweep_dispatch_dual(const SweepArgs<T>& a, int nsx, int rs, cudaStream_t s, int* tx, int* ty,
                                int* nt);
// A slab of a decomposed grid or a moving grid (ideal gas, no dual energy).
template <typename T, int DIM>
cudaError_t sweep_dispatch_xm(const SweepArgs<T>& a, int nsx, int rs, cudaStream_t s, int* tx, int* ty,
                              int* nt);
// The gas + radiation EoS (HLL and HLLC only), with or without dual energy.
template <typename T, int DIM>
cudaError_t sweep_dispatch_rad(const SweepArgs<T>& a, int nsx, int rs, int dual, cudaStream_t s, int* tx,
                               int* ty, int* nt);

// Raise the dynamic shared-memory limit of kernel `fn` to at least `bytes`
// on the current device.  The attribute is a property of the kernel on one
// device, so it is set per (device, kernel) pair when a launch needs more
// than was set before, under a lock (host threads may make their first calls
// at the same time).
inline cudaError_t smem_attr_once(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({dev, fn});
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[{dev, fn}] = bytes;
  return e;
}

// Bits of a non-negative double, for an ordered atomicMax.
__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}

}  // namespace hydro
