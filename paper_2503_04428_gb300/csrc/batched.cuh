// batched.cuh -- thousands of independent 1D tubes advanced in one persistent launch.
//
// Each tube b is a uniform grid of n_b cells on [0,1] with transmissive ends
// and its own CFL time step dt_b = cfl / max_i (|u|+c) n_b (reading R4 in
// 1D).  The tubes are cut into work items of at most CH cells; a persistent
// grid of CTAs pulls items from an atomic counter.  Per item the CTA stages
// the cells plus two ghosts per side in shared memory and runs the same
// MUSCL-Hancock steps as the grid sweep (Sect. 3.2, Eq. 17-19) with the exact
// Riemann solver (App. C.1):
//   F1  predicted face states, Toro's guess; faces where Toro's rule picks
//       the two-shock estimate are queued for the MLP (and optionally
//       harvested as training data);
//   F2  the queued faces are evaluated by the 6-64-64-1 MLP, one per thread,
//       so that the network runs on full warps; it predicts
//       ln(p_star/p_ref), p_ref = sqrt(P_L P_R);
//   F3  Newton from the guess to 1e-10 (FP64) and one polishing step, sample
//       at x/t = 0, Godunov flux;
//   U   conservative update and the tube's next signal speed.
// The last CTA to finish commits the step (per-tube speeds, times, buffer).
#pragma once
#include "common.cuh"

namespace hydro {

struct BatchCtrl {
  Ctrl c;
  unsigned int next_item;  // work-queue head of the running launch
  unsigned int pad2;
};

template <typename T>
struct BatchArgs {
  const T* A;
  T* B;
  T* Aw;
  long long total;
  const long long* off;        // ntubes + 1 cell offsets
  const int* item_tube;
  const int* item_start;
  int nitems;
  int ntubes;
  const double* smax_cur;      // per tube: max (|u|+c)/h of the current state
  unsigned long long* smax_next;
  double* t_tube;
  double cfl;
  Gas<T> gas;
  int limiter;
  const float* mlp_w;          // 4673 weights (device) or null
  int mlp_on;
  double* harvest;             // capacity x 6 doubles or null
  unsigned long long* harvest_n;
  long long harvest_cap;
  unsigned long long harvest_thresh;
  unsigned long long harvest_seed;
  BatchCtrl* ctrl;
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // SplitMix64 finaliser (Steele, Lea & Flood 2014)
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T, int CH>
struct BatchSmem {
  T W[3][CH + 4];
  T D[3][CH + 2];
  T WLR[6][CH + 1];
  T pg[CH + 1];
  T F[3][CH + 1];
  int queue[CH + 1];
  int qn;
  int item;
  double red[CH / 32];
  float w[MLP_NPARAM];
};

template <typename T, int CH>
__global__ void __launch_bounds__(CH)
    batched_kernel(const BatchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem<T, CH>& sm = *reinterpret_cast<BatchSmem<T, CH>*>(smem_raw);
  const volatile Ctrl* vc = &a.ctrl->c;
  if (vc->status != 0) return;
  const int cur = vc->cur;
  const long long step = vc->step;
  const T* Uin = cur ? a.B : a.A;
  T* Uout = cur ? a.Aw : a.B;
  const int tid = threadIdx.x;
  const Gas<T>& gas = a.gas;
  if (a.mlp_on)
    for (int p = tid; p < MLP_NPARAM; p += CH) sm.w[p] = a.mlp_w[p];
  unsigned long long n_iters = 0, n_mlp = 0, n_fb = 0;
  int err = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      sm.item = (int)atomicAdd(&a.ctrl->next_item, 1u);
      sm.qn = 0;
    }
    __syncthreads();
    const int it = sm.item;
    if (it >= a.nitems) break;
    const int b = a.item_tube[it];
    const int s0 = a.item_start[it];
    const long long base = a.off[b];
    const int nb = (int)(a.off[b + 1] - base);
    const int L = min(CH, nb - s0);
    const T fn = (T)nb;          // 1/h
    const T hw = T(0.5) / fn;    // half width
    const double dtd = a.cfl / a.smax_cur[b];
    const T dt = (T)dtd;
    const T dtdx = dt * fn;

    // a1 + a2: stage cells s0-2 .. s0+L+1 (transmissive ends) as primitives
    for (int q = tid; q < L + 4; q += CH) {
      const int c = min(max(s0 - 2 + q, 0), nb - 1);
      T u[3], w[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) u[v] = __ldg(Uin + v * a.total + base + c);
      to_prim<T, 1, 0>(u, w, gas);
#pragma unroll
      for (int v = 0; v < 3; ++v) sm.W[v][q] = w[v];
    }
    __syncthreads();

    // a3 + a4: predictor increment of cells s0-1 .. s0+L
    for (int q = tid; q < L + 2; q += CH) {
      T wl[3], wh[3], fl[3], fh[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const T wc = sm.W[v][q + 1];
        const T sig = limit<T>(a.limiter, (wc - sm.W[v][q]) * fn, (sm.W[v][q + 2] - wc) * fn);
        wl[v] = wc - hw * sig;
        wh[v] = wc + hw * sig;
      }
      phys_flux<T, 1, 0, 0>(wl, fl, gas);
      phys_flux<T, 1, 0, 0>(wh, fh, gas);
#pragma unroll
      for (int v = 0; v < 3; ++v) sm.D[v][q] = T(0.5) * dtdx * (fl[v] - fh[v]);
    }
    __syncthreads();

    // F1: predicted face states and the guess of faces s0 .. s0+L
    for (int f = tid; f <= L; f += CH) {
      // faces shared with the next chunk are solved twice; count them once
      const bool owned = f < L || s0 + L == nb;
      T Wf[2][3];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        // side 0: high face of cell (f-1) [stage index f+1]; side 1: low face of cell f
        const int q = f + 1 + side;
        T w[3], u[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const T wc = sm.W[v][q];
          const T sig = limit<T>(a.limiter, (wc - sm.W[v][q - 1]) * fn, (sm.W[v][q + 1] - wc) * fn);
          w[v] = side == 0 ? wc + hw * sig : wc - hw * sig;
        }
        to_cons<T, 1, 0>(w, u, gas);
#pragma unroll
        for (int v = 0; v < 3; ++v) u[v] += sm.D[v][q - 1];
        to_prim<T, 1, 0>(u, Wf[side], gas);
        if (!(Wf[side][0] > T(0)) || !(Wf[side][2] > T(0))) {
#pragma unroll
          for (int v = 0; v < 3; ++v) Wf[side][v] = sm.W[v][q];
          if (owned) ++n_fb;
        }
      }
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        sm.WLR[v][f] = Wf[0][v];
        sm.WLR[3 + v][f] = Wf[1][v];
      }
      const T cL = dsqrt(gas.g * Wf[0][2] / Wf[0][0]), cR = dsqrt(gas.g * Wf[1][2] / Wf[1][0]);
      int kind;
      sm.pg[f] = toro_guess<T>(Wf[0][0], Wf[0][1], Wf[0][2], cL, Wf[1][0], Wf[1][1], Wf[1][2], cR, gas, kind);
      if (kind == 2) {
        if (a.mlp_on) sm.queue[atomicAdd(&sm.qn, 1)] = f;
        if (a.harvest) {
          const unsigned long long id = (unsigned long long)(base + b + s0 + f);
          const unsigned long long hsh = mix64(a.harvest_seed + 0x9E3779B97F4A7C15ull * (id + 1) +
                                               ((unsigned long long)step << 40));
          if (hsh < a.harvest_thresh) {
            const unsigned long long slot = atomicAdd(a.harvest_n, 1ull);
            if ((long long)slot < a.harvest_cap) {
#pragma unroll
              for (int v = 0; v < 3; ++v) {
                a.harvest[slot * 6 + v] = (double)Wf[0][v];
                a.harvest[slot * 6 + 3 + v] = (double)Wf[1][v];
              }
            }
          }
        }
      }
    }
    __syncthreads();

    // F2: MLP guess of the queued faces, one face per thread
    if (a.mlp_on) {
      const int qn = sm.qn;
      for (int q = tid; q < qn; q += CH) {
        const int f = sm.queue[q];
        float x[6], pref;
        mlp_features((float)gas.g, (float)sm.WLR[0][f], (float)sm.WLR[1][f], (float)sm.WLR[2][f],
                     (float)sm.WLR[3][f], (float)sm.WLR[4][f], (float)sm.WLR[5][f], x, pref);
        const float y = mlp_forward(sm.w, x);
        sm.pg[f] = (T)((double)pref * exp((double)y));
        if (f < L || s0 + L == nb) ++n_mlp;
      }
      __syncthreads();
    }

    // F3: Newton, sampling and the Godunov flux
    for (int f = tid; f <= L; f += CH) {
      T WL[3], WR[3], F[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        WL[v] = sm.WLR[v][f];
        WR[v] = sm.WLR[3 + v][f];
      }
      int its = 0, kind = 0;
      const int st = riemann_exact<T, 1, 0, 0>(WL, WR, F, gas, sm.pg[f], its, kind);
      if (f < L || s0 + L == nb) n_iters += its;
      if (st != ST_OK && err == 0) err = st;
#pragma unroll
      for (int v = 0; v < 3; ++v) sm.F[v][f] = F[v];
    }
    __syncthreads();

    // U: update cells s0 .. s0+L-1 and their signal speed
    double smax = 0.0;
    for (int q = tid; q < L; q += CH) {
      const long long c = base + s0 + q;
      T u[3], w[3];
      bool finite = true;
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        u[v] = Uin[v * a.total + c] + dtdx * (sm.F[v][q] - sm.F[v][q + 1]);
        finite = finite && isfinite(u[v]);
      }
      to_prim<T, 1, 0>(u, w, gas);
      if (!finite) err = err ? err : ST_NONFINITE;
      else if (!(w[0] > T(0)) || !(w[2] > T(0))) err = err ? err : ST_NEG;
      const T sp = (fabs(w[1]) + dsqrt(gas.g * w[2] / w[0])) * fn;
      smax = fmax(smax, (double)sp);
#pragma unroll
      for (int v = 0; v < 3; ++v) Uout[v * a.total + c] = u[v];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    if ((tid & 31) == 0) sm.red[tid >> 5] = smax;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < CH / 32; ++w) smax = fmax(smax, sm.red[w]);
      atomicMax(&a.smax_next[b], dbits(smax));
    }
  }

  // block totals of the counters and the error, then the last-CTA commit
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_iters += __shfl_xor_sync(0xffffffffu, n_iters, o);
    n_mlp += __shfl_xor_sync(0xffffffffu, n_mlp, o);
    n_fb += __shfl_xor_sync(0xffffffffu, n_fb, o);
    const int e2 = __shfl_xor_sync(0xffffffffu, err, o);
    err = err ? err : e2;
  }
  if ((tid & 31) == 0) {
    if (n_iters) atomicAdd(&a.ctrl->c.iters, n_iters);
    if (n_mlp) atomicAdd(&a.ctrl->c.mlp, n_mlp);
    if (n_fb) atomicAdd(&a.ctrl->c.fallbacks, n_fb);
    if (err && atomicCAS(&a.ctrl->c.status, 0, err) == 0) a.ctrl->c.err_step = step;
  }
  __syncthreads();
  __shared__ int last;
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(&a.ctrl->c.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  volatile BatchCtrl* vb = a.ctrl;
  const bool ok = vb->c.status == 0;
  if (ok) {
    double* smc = const_cast<double*>(a.smax_cur);
    for (int b = tid; b < a.ntubes; b += CH) {
      a.t_tube[b] += a.cfl / smc[b];
      const unsigned long long nbits = atomicExch(&a.smax_next[b], 0ull);
      smc[b] = __longlong_as_double((long long)nbits);
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (ok) {
      vb->c.step = step + 1;
      vb->c.cur = cur ^ 1;
    }
    vb->c.done = 0;
    vb->next_item = 0;
    __threadfence();
  }
}

// Signal speed of the current state per tube (after set_state).
template <typename T>
__global__ void batch_speed_kernel(const T* U, long long total, const long long* off, int ntubes,
                                   Gas<T> gas, unsigned long long* smax_bits, int* status) {
  const int b = blockIdx.x;
  if (b >= ntubes) return;
  const long long base = off[b];
  const int nb = (int)(off[b + 1] - base);
  double smax = 0.0;
  int err = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    T u[3], w[3];
    bool finite = true;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      u[v] = U[v * total + base + i];
      finite = finite && isfinite(u[v]);
    }
    if (!finite) { err = ST_NONFINITE; continue; }
    to_prim<T, 1, 0>(u, w, gas);
    if (!(w[0] > T(0)) || !(w[2] > T(0))) { err = err ? err : ST_NEG; continue; }
    smax = fmax(smax, (double)((fabs(w[1]) + dsqrt(gas.g * w[2] / w[0])) * (T)nb));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    const int e2 = __shfl_xor_sync(0xffffffffu, err, o);
    err = err ? err : e2;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&smax_bits[b], dbits(smax));
    if (err) atomicCAS(status, 0, err);
  }
}

// Exact star states of independent faces (one thread per face).
template <typename T>
__global__ void exact_list_kernel(const double* WL, const double* WR, long long n, Gas<T> gas,
                                  const float* mlp_w, double* pstar, double* ustar, int* iters) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T rL = (T)WL[3 * i], uL = (T)WL[3 * i + 1], pL = (T)WL[3 * i + 2];
  const T rR = (T)WR[3 * i], uR = (T)WR[3 * i + 1], pR = (T)WR[3 * i + 2];
  T guess = T(0);
  if (mlp_w) {
    const T cL = dsqrt(gas.g * pL / rL), cR = dsqrt(gas.g * pR / rR);
    int kind;
    toro_guess<T>(rL, uL, pL, cL, rR, uR, pR, cR, gas, kind);
    if (kind == 2) {
      float x[6], pref;
      mlp_features((float)gas.g, (float)rL, (float)uL, (float)pL, (float)rR, (float)uR, (float)pR, x, pref);
      guess = (T)((double)pref * exp((double)mlp_forward(mlp_w, x)));
    }
  }
  T ps = T(0), us = T(0);
  int its = 0, kind = 0;
  const int st = exact_star<T>(rL, uL, pL, rR, uR, pR, gas, guess, ps, us, its, kind);
  pstar[i] = st == ST_OK ? (double)ps : -1.0;
  ustar[i] = (double)us;
  iters[i] = st == ST_OK ? its : -st;
}

}  // namespace hydro
