// sweep.cuh -- fused MUSCL-Hancock time step for 1D/2D/3D grids.
//
// One kernel launch is one full time step (HERACLES++ Sect. 3.2):
//   a1 ghost cells, synthesised at load time from the boundary kinds;
//   a2 primitive recovery (Eq. 5) of every staged cell;
//   a3/a4 limited slopes (Eq. 17) and the unsplit Hancock predictor (Eq. 18),
//         whose increment dU is kept in shared memory;
//   a5 one Riemann solve per face (HLL, HLLC or exact);
//   a6 conservative update with dS/dV and the spherical sources (Eq. 13-16);
//   a7/a8 gravity (Eq. 2-4) and heating (Sect. 2.4) from the t^n state;
//   a9 the signal speed of the new state (max over cells) for the next CFL
//      time step, committed by the last CTA through the control block.
//
// Tiling: a CTA owns TX x TY cells of the (axis0, axis1) plane and, in 3D,
// marches along axis 2 over `zchunk` planes with rolling shared-memory
// windows: 5 planes of primitives (halo 2), 3 planes of predictor increments
// (halo 1) and the fluxes of the current plane's x/y faces plus two z-face
// planes.  Each value is read from HBM once per CTA (halo re-reads hit L2)
// and written once.
#pragma once
#include "common.cuh"

namespace hydro {

// Tile shape per (precision, dimension, scalar slots); NT (threads per CTA)
// is chosen so that the heavy phases (predictor over the tile plus halo,
// faces) take few, nearly full rounds of the CTA's threads.
template <typename T, int DIM, int NSX>
struct TileCfg;
// float
template <> struct TileCfg<float, 1, 0> { static constexpr int TX = 256, TY = 1; };
template <> struct TileCfg<float, 1, 1> { static constexpr int TX = 256, TY = 1; };
template <> struct TileCfg<float, 1, 3> { static constexpr int TX = 256, TY = 1; };
template <> struct TileCfg<float, 2, 0> { static constexpr int TX = 32, TY = 16; };
template <> struct TileCfg<float, 2, 1> { static constexpr int TX = 32, TY = 16; };
template <> struct TileCfg<float, 2, 3> { static constexpr int TX = 32, TY = 8; };
template <> struct TileCfg<float, 3, 0> { static constexpr int TX = 32, TY = 16, NT = 640; };
template <> struct TileCfg<float, 3, 1> { static constexpr int TX = 32, TY = 8, NT = 384; };
template <> struct TileCfg<float, 3, 3> { static constexpr int TX = 16, TY = 16, NT = 416; };
// double
template <> struct TileCfg<double, 1, 0> { static constexpr int TX = 256, TY = 1; };
template <> struct TileCfg<double, 1, 1> { static constexpr int TX = 256, TY = 1; };
template <> struct TileCfg<double, 1, 3> { static constexpr int TX = 256, TY = 1; };
template <> struct TileCfg<double, 2, 0> { static constexpr int TX = 32, TY = 8; };
template <> struct TileCfg<double, 2, 1> { static constexpr int TX = 32, TY = 8; };
template <> struct TileCfg<double, 2, 3> { static constexpr int TX = 32, TY = 8; };
template <> struct TileCfg<double, 3, 0> { static constexpr int TX = 16, TY = 16, NT = 416; };
template <> struct TileCfg<double, 3, 1> { static constexpr int TX = 16, TY = 16, NT = 416; };
template <> struct TileCfg<double, 3, 3> { static constexpr int TX = 16, TY = 8, NT = 224; };

template <typename C, typename = void>
struct TileThreads { static constexpr int value = C::TX * C::TY; };
template <typename C>
struct TileThreads<C, decltype((void)C::NT)> { static constexpr int value = C::NT; };

template <typename T, int DIM, int NSX>
struct SweepShape {
  static constexpr int NV = 2 + DIM + NSX;
  static constexpr int TX = TileCfg<T, DIM, NSX>::TX;
  static constexpr int TY = TileCfg<T, DIM, NSX>::TY;
  static constexpr int HY = DIM >= 2 ? 2 : 0;            // primitive halo along axis 1
  static constexpr int EX = TX + 4, EY = TY + 2 * HY;    // primitive plane extents
  static constexpr int QY = DIM >= 2 ? 1 : 0;            // predictor halo along axis 1
  static constexpr int PX = TX + 2, PY = TY + 2 * QY;    // predictor plane extents
  static constexpr int WP = DIM == 3 ? 5 : 1;            // primitive planes in flight
  static constexpr int DP = DIM == 3 ? 3 : 1;            // predictor planes in flight
  static constexpr int NT = TileThreads<TileCfg<T, DIM, NSX>>::value;  // threads per CTA
  static constexpr int WPL = EX * EY, DPL = PX * PY;
  static constexpr int NFX = (TX + 1) * TY;
  static constexpr int NFY = DIM >= 2 ? TX * (TY + 1) : 0;
  static constexpr int NFZ = DIM == 3 ? TX * TY : 0;
  static constexpr size_t smem_elems =
      (size_t)WP * NV * WPL + (size_t)DP * NV * DPL + (size_t)NV * NFX + (size_t)NV * NFY +
      (size_t)2 * NV * NFZ;
  static constexpr size_t smem_bytes = smem_elems * sizeof(T);
};

// Ghost mapping of one axis (periodic wrap, transmissive copy of the edge
// cell, reflective mirror with the normal momentum negated).  g in [-2, n+1].
__device__ __forceinline__ int map_axis(int g, int n, int lo, int hi, bool& flip) {
  flip = false;
  if (g < 0) {
    if (lo == BC_PERIODIC) return g + n;
    if (lo == BC_TRANSMISSIVE) return 0;
    flip = true;
    return -1 - g;
  }
  if (g >= n) {
    if (hi == BC_PERIODIC) return g - n;
    if (hi == BC_TRANSMISSIVE) return n - 1;
    flip = true;
    return 2 * n - 1 - g;
  }
  return g;
}

template <typename T, int DIM, int NSX, int RS>
struct Sweep {
  using S = SweepShape<T, DIM, NSX>;
  static constexpr int NV = S::NV, TX = S::TX, TY = S::TY, EX = S::EX, EY = S::EY, PX = S::PX,
                       PY = S::PY, HY = S::HY, QY = S::QY, NT = S::NT;

  const SweepArgs<T>& a;
  T* Ws;
  T* Ds;
  T* Fx;
  T* Fy;
  T* Fz;
  int x0, y0;
  T dt, half_dt;
  const T* Uin;
  T* Uout;
  unsigned long long n_fallback = 0, n_iters = 0;
  int err = 0;
  double smax = 0.0;
  T hfac = T(0);

  __device__ Sweep(const SweepArgs<T>& args, T* smem) : a(args) {
    Ws = smem;
    Ds = Ws + S::WP * NV * S::WPL;
    Fx = Ds + S::DP * NV * S::DPL;
    Fy = Fx + NV * S::NFX;
    Fz = Fy + NV * S::NFY;
  }

  __device__ __forceinline__ T& W(int slot, int v, int ey, int ex) {
    return Ws[((slot * NV + v) * EY + ey) * EX + ex];
  }
  __device__ __forceinline__ T& Dq(int slot, int v, int py, int px) {
    return Ds[((slot * NV + v) * PY + py) * PX + px];
  }
  static __device__ __forceinline__ int wslot(int gz) { return DIM == 3 ? (gz + 10) % 5 : 0; }
  static __device__ __forceinline__ int dslot(int gz) { return DIM == 3 ? (gz + 6) % 3 : 0; }

  // a1 + a2: stage plane gz (axis-2 index, may be a ghost) as primitives.
  __device__ void load_plane(int gz) {
    const int n0 = a.n[0], n1 = a.n[1];
    bool fz = false;
    const int sz = DIM == 3 ? map_axis(gz, a.n[2], a.bc[2][0], a.bc[2][1], fz) : 0;
    const int slot = wslot(gz);
    const int nvact = 2 + DIM + a.ns;
    for (int idx = threadIdx.x; idx < S::WPL; idx += NT) {
      const int ex = idx % EX, ey = idx / EX;
      const int gi = min(x0 - 2 + ex, n0 + 1);
      bool fx, fy = false;
      const int si = map_axis(gi, n0, a.bc[0][0], a.bc[0][1], fx);
      int sj = 0;
      if (DIM >= 2) sj = map_axis(min(y0 - HY + ey, n1 + 1), n1, a.bc[1][0], a.bc[1][1], fy);
      const long long c = ((long long)sz * n1 + sj) * n0 + si;
      T u[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = v < nvact ? __ldg(Uin + (long long)v * a.ncell + c) : T(0);
      if (fx) u[1] = -u[1];
      if (DIM >= 2 && fy) u[2] = -u[2];
      if (DIM == 3 && fz) u[3] = -u[3];
      to_prim<T, DIM, NSX>(u, w, a.gas);
#pragma unroll
      for (int v = 0; v < NV; ++v) W(slot, v, ey, ex) = w[v];
    }
  }

  // 1/h_d of a cell (physical width: h_r = dr, h_th = r dth, h_ph = r s dph).
  __device__ __forceinline__ T inv_h(int d, int gi, int gj, int gk) const {
    if (d == 0) return a.geo.inv_w[0][gi + 2];
    if (d == 1) {
      const T w = a.geo.inv_w[1][gj + 2];
      return a.spherical ? w * a.geo.inv_r[gi + 2] : w;
    }
    const T w = a.geo.inv_w[2][gk + 2];
    return a.spherical ? w * a.geo.inv_r[gi + 2] * a.geo.inv_s[gj + 2] : w;
  }

  // Limited low/high face states along DIR of the cell with centre Wc and
  // neighbours Wm/Wp; g = the cell's index along DIR.
  template <int DIR>
  __device__ __forceinline__ void faces_of(const T* Wm, const T* Wc, const T* Wp, int g, T* Wlo,
                                           T* Whi) const {
    const T idm = a.geo.inv_dxc[DIR][g + 2], idp = a.geo.inv_dxc[DIR][g + 3];
    const T h = a.geo.hw[DIR][g + 2];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T sig = limit<T>(a.limiter, (Wc[v] - Wm[v]) * idm, (Wp[v] - Wc[v]) * idp);
      Wlo[v] = Wc[v] - h * sig;
      Whi[v] = Wc[v] + h * sig;
    }
  }

  // Neighbour fetch of the primitive plane data.
  template <int DIR>
  __device__ __forceinline__ void neighbours(int slot, int ey, int ex, int gz, T* Wm, T* Wc,
                                             T* Wp) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Wc[v] = W(slot, v, ey, ex);
      if (DIR == 0) {
        Wm[v] = W(slot, v, ey, ex - 1);
        Wp[v] = W(slot, v, ey, ex + 1);
      } else if (DIR == 1) {
        Wm[v] = W(slot, v, ey - 1, ex);
        Wp[v] = W(slot, v, ey + 1, ex);
      } else {
        Wm[v] = W(wslot(gz - 1), v, ey, ex);
        Wp[v] = W(wslot(gz + 1), v, ey, ex);
      }
    }
  }

  // a3 + a4: predictor increment dU = dt/2 sum_d (F_d(W_lo) - F_d(W_hi))/h_d
  // for plane gz over the tile plus a one-cell halo.
  __device__ void predictor_plane(int gz) {
    const int n0 = a.n[0], n1 = a.n[1];
    const int slot = wslot(gz), ds = dslot(gz);
    for (int idx = threadIdx.x; idx < S::DPL; idx += NT) {
      const int px = idx % PX, py = idx / PX;
      const int gi = x0 - 1 + px;
      const int gj = DIM >= 2 ? y0 - 1 + py : 0;
      if (gi > n0 || (DIM >= 2 && gj > n1)) continue;
      const int ex = px + 1, ey = py + (DIM >= 2 ? 1 : 0);
      T acc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = T(0);
      {
        T Wm[NV], Wc[NV], Wp[NV], Wl[NV], Wh[NV], Fl[NV], Fh[NV];
        neighbours<0>(slot, ey, ex, gz, Wm, Wc, Wp);
        faces_of<0>(Wm, Wc, Wp, gi, Wl, Wh);
        phys_flux<T, DIM, NSX, 0>(Wl, Fl, a.gas);
        phys_flux<T, DIM, NSX, 0>(Wh, Fh, a.gas);
        const T ih = inv_h(0, gi, gj, gz);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += (Fl[v] - Fh[v]) * ih;
      }
      if constexpr (DIM >= 2) {
        T Wm[NV], Wc[NV], Wp[NV], Wl[NV], Wh[NV], Fl[NV], Fh[NV];
        neighbours<1>(slot, ey, ex, gz, Wm, Wc, Wp);
        faces_of<1>(Wm, Wc, Wp, gj, Wl, Wh);
        phys_flux<T, DIM, NSX, 1>(Wl, Fl, a.gas);
        phys_flux<T, DIM, NSX, 1>(Wh, Fh, a.gas);
        const T ih = inv_h(1, gi, gj, gz);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += (Fl[v] - Fh[v]) * ih;
      }
      if constexpr (DIM == 3) {
        T Wm[NV], Wc[NV], Wp[NV], Wl[NV], Wh[NV], Fl[NV], Fh[NV];
        neighbours<2>(slot, ey, ex, gz, Wm, Wc, Wp);
        faces_of<2>(Wm, Wc, Wp, gz, Wl, Wh);
        phys_flux<T, DIM, NSX, 2>(Wl, Fl, a.gas);
        phys_flux<T, DIM, NSX, 2>(Wh, Fh, a.gas);
        const T ih = inv_h(2, gi, gj, gz);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += (Fl[v] - Fh[v]) * ih;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) Dq(ds, v, py, px) = half_dt * acc[v];
    }
  }

  // Predicted face state (primitive) on side HI (1) or LO (0) of a cell.
  // A non-physical prediction falls back to the cell average.
  template <int DIR, int HI>
  __device__ __forceinline__ void face_state(int slot, int ey, int ex, int gz, int ds, int py,
                                             int px, int g, T* Wf) {
    T Wm[NV], Wc[NV], Wp[NV], Wl[NV], Wh[NV], U[NV];
    neighbours<DIR>(slot, ey, ex, gz, Wm, Wc, Wp);
    faces_of<DIR>(Wm, Wc, Wp, g, Wl, Wh);
    to_cons<T, DIM, NSX>(HI ? Wh : Wl, U, a.gas);
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] += Dq(ds, v, py, px);
    to_prim<T, DIM, NSX>(U, Wf, a.gas);
    if (!(Wf[0] > T(0)) || !(Wf[1 + DIM] > T(0))) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Wf[v] = Wc[v];
      ++n_fallback;
    }
  }

  template <int DIR>
  __device__ __forceinline__ void riemann(const T* WL, const T* WR, T* F) {
    if constexpr (RS == RS_HLL) {
      riemann_hll<T, DIM, NSX, DIR>(WL, WR, F, a.gas);
    } else if constexpr (RS == RS_HLLC) {
      riemann_hllc<T, DIM, NSX, DIR>(WL, WR, F, a.gas);
    } else {
      int it = 0, kind = 0;
      const int st = riemann_exact<T, DIM, NSX, DIR>(WL, WR, F, a.gas, T(0), it, kind);
      n_iters += it;
      if (st != ST_OK && err == 0) err = st;
    }
  }

  // The face between axis-2 planes zl and zl+1 (3D only), into Fz[(zl+1)&1].
  __device__ void zfaces(int zl) {
    const int n0 = a.n[0], n1 = a.n[1];
    T* Fzo = Fz + ((zl + 1) & 1) * NV * S::NFZ;
    for (int idx = threadIdx.x; idx < S::NFZ; idx += NT) {
      const int fi = idx % TX, fj = idx / TX;
      if (x0 + fi >= n0 || y0 + fj >= n1) continue;
      T WL[NV], WR[NV], F[NV];
      face_state<2, 1>(wslot(zl), fj + HY, fi + 2, zl, dslot(zl), fj + QY, fi + 1, zl, WL);
      face_state<2, 0>(wslot(zl + 1), fj + HY, fi + 2, zl + 1, dslot(zl + 1), fj + QY, fi + 1, zl + 1, WR);
      riemann<2>(WL, WR, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fzo[v * S::NFZ + idx] = F[v];
    }
  }

  // a5 for the x and y faces of plane gz and, in 3D, its top z face, in one
  // loop over all of them.
  __device__ void faces_plane(int gz) {
    const int n0 = a.n[0], n1 = a.n[1];
    const int slot = wslot(gz), ds = dslot(gz);
    T* Fzo = Fz + ((gz + 1) & 1) * NV * S::NFZ;
    for (int idx = threadIdx.x; idx < S::NFX + S::NFY + S::NFZ; idx += NT) {
      T WL[NV], WR[NV], F[NV];
      if (DIM == 3 && idx >= S::NFX + S::NFY) {
        const int k = idx - S::NFX - S::NFY;
        const int fi = k % TX, fj = k / TX;
        if (x0 + fi >= n0 || y0 + fj >= n1) continue;
        face_state<2, 1>(slot, fj + HY, fi + 2, gz, ds, fj + QY, fi + 1, gz, WL);
        face_state<2, 0>(wslot(gz + 1), fj + HY, fi + 2, gz + 1, dslot(gz + 1), fj + QY, fi + 1, gz + 1, WR);
        riemann<2>(WL, WR, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) Fzo[v * S::NFZ + k] = F[v];
      } else if (idx < S::NFX) {
        const int fi = idx % (TX + 1), fj = idx / (TX + 1);
        if (x0 + fi > n0 || (DIM >= 2 && y0 + fj >= n1)) continue;
        const int gi = x0 + fi, gj = y0 + fj;
        face_state<0, 1>(slot, fj + HY, fi + 1, gz, ds, fj + QY, fi, gi - 1, WL);
        face_state<0, 0>(slot, fj + HY, fi + 2, gz, ds, fj + QY, fi + 1, gi, WR);
        (void)gj;
        riemann<0>(WL, WR, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) Fx[v * S::NFX + idx] = F[v];
      } else if constexpr (DIM >= 2) {
        const int k = idx - S::NFX;
        const int fi = k % TX, fj = k / TX;
        if (x0 + fi >= n0 || y0 + fj > n1) continue;
        const int gj = y0 + fj;
        face_state<1, 1>(slot, fj - 1 + HY, fi + 2, gz, ds, fj - 1 + QY, fi + 1, gj - 1, WL);
        face_state<1, 0>(slot, fj + HY, fi + 2, gz, ds, fj + QY, fi + 1, gj, WR);
        riemann<1>(WL, WR, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) Fy[v * S::NFY + k] = F[v];
      }
    }
  }

  // a6-a9: update plane gz.
  __device__ void update_plane(int gz) {
    const int n0 = a.n[0], n1 = a.n[1];
    const int nvact = 2 + DIM + a.ns;
    const T* Fzb = Fz + (gz & 1) * NV * S::NFZ;
    const T* Fzt = Fz + ((gz + 1) & 1) * NV * S::NFZ;
    for (int idx = threadIdx.x; idx < TX * TY; idx += NT) {
      const int i = idx % TX, j = idx / TX;
      const int gi = x0 + i, gj = y0 + j;
      if (gi >= n0 || gj >= n1) continue;
      const long long c = ((long long)gz * n1 + gj) * n0 + gi;
      T Uo[NV], Un[NV], acc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uo[v] = v < nvact ? Uin[(long long)v * a.ncell + c] : T(0);
      const int fx = j * (TX + 1) + i;
      const T Afl = a.geo.Af[gi], Afh = a.geo.Af[gi + 1], ia = a.geo.inva[gi];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = (Fx[v * S::NFX + fx] * Afl - Fx[v * S::NFX + fx + 1] * Afh) * ia;
      T cy = T(0), Bfl = T(1), Bfh = T(1);
      if constexpr (DIM >= 2) {
        Bfl = a.geo.Bf[gj];
        Bfh = a.geo.Bf[gj + 1];
        cy = a.geo.ga[gi] * a.geo.invb[gj];
        const int fy = j * TX + i;
#pragma unroll
        for (int v = 0; v < NV; ++v)
          acc[v] += (Fy[v * S::NFY + fy] * Bfl - Fy[v * S::NFY + fy + TX] * Bfh) * cy;
      }
      if constexpr (DIM == 3) {
        const T cz = a.geo.ga[gi] * a.geo.zc[gj] * a.geo.invc[gz];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += (Fzb[v * S::NFZ + idx] - Fzt[v * S::NFZ + idx]) * cz;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) Un[v] = Uo[v] + dt * acc[v];

      if (a.spherical) {
        // Geometric momentum sources, Eq. 13-16 (face-flux forms).  An absent
        // axis uses the pressure of the half-step cell state U + dU (or of U
        // if that state is not physical).
        T P = T(0);
        if constexpr (DIM < 3) {
          T Uh[NV], Wh[NV], Wo[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) Uh[v] = Uo[v] + Dq(dslot(gz), v, j + QY, i + 1);
          to_prim<T, DIM, NSX>(Uh, Wh, a.gas);
          to_prim<T, DIM, NSX>(Uo, Wo, a.gas);
          P = (Wh[0] > T(0) && Wh[1 + DIM] > T(0)) ? Wh[1 + DIM] : Wo[1 + DIM];
        }
        T Tth = P, Tph = P;
        if constexpr (DIM >= 2) Tth = T(0.5) * (Fy[2 * S::NFY + j * TX + i] + Fy[2 * S::NFY + j * TX + i + TX]);
        if constexpr (DIM == 3) Tph = T(0.5) * (Fzb[3 * S::NFZ + idx] + Fzt[3 * S::NFZ + idx]);
        Un[1] += dt * T(0.5) * (Tth + Tph) * a.geo.gr[gi];
        if constexpr (DIM >= 2) {
          const T frl = Fx[2 * S::NFX + fx], frh = Fx[2 * S::NFX + fx + 1];
          Un[2] += dt * (-a.geo.qr[gi] * (frh * Afh + frl * Afl) + Tph * a.geo.ga[gi] * a.geo.gt[gj]);
        }
        if constexpr (DIM == 3) {
          const T frl = Fx[3 * S::NFX + fx], frh = Fx[3 * S::NFX + fx + 1];
          const T ftl = Fy[3 * S::NFY + j * TX + i], fth = Fy[3 * S::NFY + j * TX + i + TX];
          Un[3] += dt * (-a.geo.qr[gi] * (frh * Afh + frl * Afl) -
                         a.geo.ga[gi] * a.geo.qt[gj] * (fth * Bfh + ftl * Bfl));
        }
      }
      if (a.gravity != GRAV_NONE) {
        T g[3] = {T(0), T(0), T(0)};
        if (a.gravity == GRAV_UNIFORM) {
#pragma unroll
          for (int d = 0; d < DIM; ++d) g[d] = a.g0[d];
        } else if (a.gravity == GRAV_POINT) {
          g[0] = a.geo.gpt[gi];
        } else {
          g[0] = a.gmono[gi];
        }
        T work = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          Un[1 + d] += dt * Uo[0] * g[d];
          work += Uo[1 + d] * g[d];
        }
        Un[1 + DIM] += dt * work;
      }
      if (a.heating == HEAT_CONST) {
        Un[1 + DIM] += dt * a.heat_q;
      } else if (a.heating == HEAT_NI56) {
        T rf = T(0);
#pragma unroll
        for (int s = 0; s < NSX; ++s)
          if (s == a.ni_index) rf = Uo[2 + DIM + s];
        Un[1 + DIM] += dt * hfac * rf;
      }

      // validity and the signal speed of the new state
      T Wn[NV];
      to_prim<T, DIM, NSX>(Un, Wn, a.gas);
      bool finite = true;
#pragma unroll
      for (int v = 0; v < NV; ++v) finite = finite && isfinite(Un[v]);
      if (!finite) err = err ? err : ST_NONFINITE;
      else if (!(Wn[0] > T(0)) || !(Wn[1 + DIM] > T(0))) err = err ? err : ST_NEG;
      const T cs = dsqrt(a.gas.g * Wn[1 + DIM] / Wn[0]);
      T sp = T(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) sp += (fabs(Wn[1 + d]) + cs) * inv_h(d, gi, gj, gz);
      smax = fmax(smax, (double)sp);
#pragma unroll
      for (int v = 0; v < NV; ++v)
        if (v < nvact) Uout[(long long)v * a.ncell + c] = Un[v];
    }
  }
};

// Block-wide reductions into the control block, then the last-CTA commit.
template <int NT>
__device__ void finish_step(Ctrl* ctrl, double smax, int err, unsigned long long fb,
                            unsigned long long it, unsigned long long mlp, long long step,
                            double dt) {
  __shared__ double red_s[NT / 32];
  __shared__ int red_e[NT / 32];
  __shared__ unsigned long long red_f[NT / 32], red_i[NT / 32], red_m[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    const int e2 = __shfl_xor_sync(0xffffffffu, err, o);
    err = err ? err : e2;
    fb += __shfl_xor_sync(0xffffffffu, fb, o);
    it += __shfl_xor_sync(0xffffffffu, it, o);
    mlp += __shfl_xor_sync(0xffffffffu, mlp, o);
  }
  if (lane == 0) {
    red_s[wid] = smax;
    red_e[wid] = err;
    red_f[wid] = fb;
    red_i[wid] = it;
    red_m[wid] = mlp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) {
      smax = fmax(smax, red_s[w]);
      err = err ? err : red_e[w];
      fb += red_f[w];
      it += red_i[w];
      mlp += red_m[w];
    }
    if (smax > 0.0) atomicMax(&ctrl->smax_next, dbits(smax));
    if (fb) atomicAdd(&ctrl->fallbacks, fb);
    if (it) atomicAdd(&ctrl->iters, it);
    if (mlp) atomicAdd(&ctrl->mlp, mlp);
    if (err) {
      if (atomicCAS(&ctrl->status, 0, err) == 0) ctrl->err_step = step;
    }
    __threadfence();
    const unsigned int total = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int ticket = atomicAdd(&ctrl->done, 1u);
    if (ticket == total - 1) {
      __threadfence();
      volatile Ctrl* vc = ctrl;
      if (vc->status == 0) {
        const unsigned long long nb = atomicExch(&ctrl->smax_next, 0ull);
        vc->smax_cur = __longlong_as_double((long long)nb);
        vc->t = vc->t + dt;
        vc->last_dt = dt;
        vc->step = step + 1;
        vc->cur = vc->cur ^ 1;
      }
      vc->done = 0;
      __threadfence();
    }
  }
}

// Common step prologue: read the control block, decide dt.  Returns false
// when the launch must do nothing (earlier failure, or t_end reached).
__device__ __forceinline__ bool step_begin(const Ctrl* ctrl, double dt_host, double cfl,
                                           double t_end, double& dt, double& t, long long& step,
                                           int& cur) {
  const volatile Ctrl* vc = ctrl;
  if (vc->status != 0) return false;
  t = vc->t;
  step = vc->step;
  cur = vc->cur;
  if (dt_host > 0.0) {
    dt = dt_host;
  } else {
    dt = cfl / vc->smax_cur;
    if (t_end > 0.0) dt = fmin(dt, t_end - t);
  }
  return dt > 0.0;
}

template <typename T, int DIM, int NSX, int RS>
__global__ void __launch_bounds__(SweepShape<T, DIM, NSX>::NT, 1)
    sweep_kernel(const SweepArgs<T> args) {
  using S = SweepShape<T, DIM, NSX>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double dtd, t;
  long long step;
  int cur;
  if (!step_begin(args.ctrl, args.dt_host, args.cfl, args.t_end, dtd, t, step, cur)) return;

  Sweep<T, DIM, NSX, RS> sw(args, reinterpret_cast<T*>(smem_raw));
  sw.x0 = blockIdx.x * S::TX;
  sw.y0 = blockIdx.y * S::TY;
  sw.dt = (T)dtd;
  sw.half_dt = T(0.5) * sw.dt;
  sw.Uin = cur ? args.B : args.A;
  sw.Uout = cur ? args.Aw : args.B;
  if (args.heating == HEAT_NI56) {
    sw.hfac = (T)(args.ni_lambda * (args.ni_a * exp(-t / args.ni_tni) + args.ni_qco * exp(-t / args.ni_tco)));
  }

  if constexpr (DIM == 3) {
    const int z0 = blockIdx.z * args.zchunk;
    const int z1 = min(z0 + args.zchunk, args.n[2]);
    for (int q = z0 - 2; q <= z0 + 1; ++q) sw.load_plane(q);
    __syncthreads();
    sw.predictor_plane(z0 - 1);
    sw.predictor_plane(z0);
    __syncthreads();
    sw.zfaces(z0 - 1);
    for (int z = z0; z < z1; ++z) {
      sw.load_plane(z + 2);
      __syncthreads();
      sw.predictor_plane(z + 1);
      __syncthreads();
      sw.faces_plane(z);
      __syncthreads();
      sw.update_plane(z);
    }
  } else {
    sw.load_plane(0);
    __syncthreads();
    sw.predictor_plane(0);
    __syncthreads();
    sw.faces_plane(0);
    __syncthreads();
    sw.update_plane(0);
  }
  __syncthreads();
  finish_step<S::NT>(args.ctrl, sw.smax, sw.err, sw.n_fallback, sw.n_iters, 0ull, step, dtd);
}

template <typename T, int DIM, int NSX, int RS>
cudaError_t launch_sweep(const SweepArgs<T>& a, cudaStream_t s) {
  using S = SweepShape<T, DIM, NSX>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<T, DIM, NSX, RS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::smem_bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((a.n[0] + S::TX - 1) / S::TX, DIM >= 2 ? (a.n[1] + S::TY - 1) / S::TY : 1,
            DIM == 3 ? (a.n[2] + a.zchunk - 1) / a.zchunk : 1);
  sweep_kernel<T, DIM, NSX, RS><<<grid, S::NT, S::smem_bytes, s>>>(a);
  return cudaGetLastError();
}

// Launch one instantiation and report its tile shape and threads per CTA.
template <typename T, int DIM, int NSX, int RS>
cudaError_t launch_sweep_shape(const SweepArgs<T>& a, cudaStream_t s, int* tx, int* ty, int* nt) {
  using S = SweepShape<T, DIM, NSX>;
  *tx = S::TX;
  *ty = S::TY;
  *nt = S::NT;
  return launch_sweep<T, DIM, NSX, RS>(a, s);
}

// Instantiate the dispatcher of one (precision, dimension) pair.
#define HYDRO_SWEEP_DISPATCH(T, DIM)                                                          \
  template <>                                                                                 \
  cudaError_t sweep_dispatch<T, DIM>(const SweepArgs<T>& a, int nsx, int rs, cudaStream_t s,  \
                                     int* tx, int* ty, int* nt) {                             \
    switch (nsx * 4 + rs) {                                                                   \
      case 0: return launch_sweep_shape<T, DIM, 0, RS_HLL>(a, s, tx, ty, nt);                 \
      case 1: return launch_sweep_shape<T, DIM, 0, RS_HLLC>(a, s, tx, ty, nt);                \
      case 2: return launch_sweep_shape<T, DIM, 0, RS_EXACT>(a, s, tx, ty, nt);               \
      case 4: return launch_sweep_shape<T, DIM, 1, RS_HLL>(a, s, tx, ty, nt);                 \
      case 5: return launch_sweep_shape<T, DIM, 1, RS_HLLC>(a, s, tx, ty, nt);                \
      case 6: return launch_sweep_shape<T, DIM, 1, RS_EXACT>(a, s, tx, ty, nt);               \
      case 12: return launch_sweep_shape<T, DIM, 3, RS_HLL>(a, s, tx, ty, nt);                \
      case 13: return launch_sweep_shape<T, DIM, 3, RS_HLLC>(a, s, tx, ty, nt);               \
      case 14: return launch_sweep_shape<T, DIM, 3, RS_EXACT>(a, s, tx, ty, nt);              \
      default: return cudaErrorInvalidValue;                                                  \
    }                                                                                         \
  }

}  // namespace hydro
