// sweep.cuh -- fused MUSCL-Hancock time step for 1D/2D/3D grids.
//
// One kernel launch is one full time step (HERACLES++ Sect. 3.2):
//   a1 ghost cells, synthesised at load time from the boundary kinds;
//   a2 primitive recovery (Eq. 5) of every staged cell;
//   a3/a4 limited slopes (Eq. 17) and the unsplit Hancock predictor (Eq. 18);
//         every predicted face state is formed once, by the cell it belongs
//         to, and parked in a shared-memory slot of its face;
//   a5 one Riemann solve per face (HLL, HLLC or exact), whose flux is written
//      over the face's left state;
//   a6 conservative update with dS/dV and the spherical sources (Eq. 13-16);
//   a7/a8 gravity (Eq. 2-4) and heating (Sect. 2.4) from the t^n state;
//   a9 the signal speed of the new state (max over cells) for the next CFL
//      time step, committed by the last CTA through the control block.
//
// Tiling: a CTA owns TX x TY cells of the (axis0, axis1) plane and, in 3D,
// marches along axis 2 over `zchunk` planes.  Shared memory holds a ring of
// three primitive planes (halo 2 on axes 0/1), the left/right states of the
// current plane's x and y faces, and the z-face states (lower side: two
// planes, upper side: one).  Thread t < TX*TY owns tile cell t for the whole
// march and keeps the partial update of its cell in the plane below in
// registers until that plane's upper z flux is known.  Each state value is
// read from HBM once per CTA (halo re-reads hit L2) and written once.
#pragma once
#include "common.cuh"

namespace hydro {

// Tile shape per (precision, dimension, scalar slots) and the CTAs per SM
// the register budget is sized for (MB; the exact solver, whose Newton
// iteration needs more registers, always gets one CTA's budget).  The CTA has one thread per
// predictor cell (the tile plus a one-cell halo without corners), rounded up
// to whole warps.
template <typename T, int DIM, int NSX>
struct TileCfg;
// float
template <> struct TileCfg<float, 1, 0> { static constexpr int TX = 254, TY = 1, MB = 1; };
template <> struct TileCfg<float, 1, 1> { static constexpr int TX = 254, TY = 1, MB = 1; };
template <> struct TileCfg<float, 1, 3> { static constexpr int TX = 254, TY = 1, MB = 1; };
template <> struct TileCfg<float, 2, 0> { static constexpr int TX = 32, TY = 16, MB = 1; };
template <> struct TileCfg<float, 2, 1> { static constexpr int TX = 32, TY = 16, MB = 1; };
template <> struct TileCfg<float, 2, 3> { static constexpr int TX = 32, TY = 8, MB = 1; };
template <> struct TileCfg<float, 3, 0> { static constexpr int TX = 16, TY = 16, MB = 3; };
template <> struct TileCfg<float, 3, 1> { static constexpr int TX = 16, TY = 16, MB = 2; };
template <> struct TileCfg<float, 3, 3> { static constexpr int TX = 16, TY = 16, MB = 2; };
// double
template <> struct TileCfg<double, 1, 0> { static constexpr int TX = 254, TY = 1, MB = 1; };
template <> struct TileCfg<double, 1, 1> { static constexpr int TX = 254, TY = 1, MB = 1; };
template <> struct TileCfg<double, 1, 3> { static constexpr int TX = 254, TY = 1, MB = 1; };
template <> struct TileCfg<double, 2, 0> { static constexpr int TX = 32, TY = 8, MB = 1; };
template <> struct TileCfg<double, 2, 1> { static constexpr int TX = 32, TY = 8, MB = 1; };
template <> struct TileCfg<double, 2, 3> { static constexpr int TX = 32, TY = 8, MB = 1; };
template <> struct TileCfg<double, 3, 0> { static constexpr int TX = 16, TY = 16, MB = 1; };
template <> struct TileCfg<double, 3, 1> { static constexpr int TX = 16, TY = 16, MB = 1; };
template <> struct TileCfg<double, 3, 3> { static constexpr int TX = 16, TY = 8, MB = 1; };

// The smallest power of two >= n (n >= 1).
__host__ __device__ constexpr int pow2_ceil(int n) { return n <= 1 ? 1 : 2 * pow2_ceil((n + 1) / 2); }

template <typename T, int DIM, int NSX>
struct SweepShape {
  static constexpr int NV = 2 + DIM + NSX;
  static constexpr int TX = TileCfg<T, DIM, NSX>::TX;
  static constexpr int TY = TileCfg<T, DIM, NSX>::TY;
  static constexpr int HY = DIM >= 2 ? 2 : 0;              // primitive halo along axis 1
  static constexpr int EX = TX + 4, EY = TY + 2 * HY;      // primitive plane extents
  static constexpr int QY = DIM >= 2 ? 1 : 0;              // predictor halo along axis 1
  static constexpr int WP = DIM == 3 ? 3 : 1;              // primitive planes in flight
  static constexpr int NI = TX * TY;                        // tile cells, one owner thread each
  static constexpr int NH = 2 * TY + (DIM >= 2 ? 2 * TX : 0);  // halo predictor cells
  static constexpr int NP = NI + NH;                        // predictor cells
  static constexpr int NT = (NP + 31) / 32 * 32;            // threads per CTA
  static constexpr int MB = TileCfg<T, DIM, NSX>::MB;       // resident CTAs per SM (register budget)
  static constexpr int WPL = EX * EY;
  static constexpr int NFX = (TX + 1) * TY;
  static constexpr int NFY = DIM >= 2 ? TX * (TY + 1) : 0;
  static constexpr int NFZ = DIM == 3 ? TX * TY : 0;
  static constexpr size_t smem_elems = (size_t)WP * NV * WPL + (size_t)2 * NV * NFX +
                                       (size_t)2 * NV * NFY + (size_t)3 * NV * NFZ;
  static constexpr size_t dual_elems = (size_t)2 * (NFX + NFY + NFZ);  // dual-energy face terms
  // radiation EoS: face-state temperatures and those of the primitive planes
  static constexpr size_t rad_elems = (size_t)2 * NFX + 2 * NFY + 3 * NFZ + (size_t)WP * WPL;
  // the x and y geometry factors of the CTA's cells, staged once per CTA
  // (GX_N arrays over the TX + 2 predictor columns, GY_N over the TY + 2 rows)
  enum { GX_IDM, GX_IDP, GX_HW, GX_IW, GX_IR, GX_AF, GX_INVA, GX_GA, GX_QR, GX_GR, GX_G, GX_N };
  enum { GY_IDM, GY_IDP, GY_HW, GY_IW, GY_IS, GY_BF, GY_INVB, GY_ZC, GY_GT, GY_QT, GY_N };
  static constexpr size_t geo_elems = (size_t)GX_N * (TX + 2) + (DIM >= 2 ? (size_t)GY_N * (TY + 2) : 0);
  __host__ __device__ static constexpr size_t smem_bytes_for(int mode) {
    return (smem_elems + ((mode & 2) ? dual_elems : 0) + ((mode & 1) ? rad_elems : 0) + geo_elems) * sizeof(T);
  }
  // conserved totals accumulated in the step: one FP64 sum per owner and
  // variable, after the rest (16-byte aligned)
  __host__ __device__ static constexpr size_t tot_offset(int mode) { return (smem_bytes_for(mode) + 15) / 16 * 16; }
  static constexpr size_t tot_bytes = (size_t)NI * NV * sizeof(double);
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

// The same with exchanged sides (domain decomposition): a ghost of an
// exchanged side sets `layer` to its distance - 1 from the side and returns
// 0; layer stays -1 otherwise.
__device__ __forceinline__ int map_axis(int g, int n, int lo, int hi, bool& flip, int& layer) {
  flip = false;
  if ((g < 0 && lo == BC_EXCHANGED) || (g >= n && hi == BC_EXCHANGED)) {
    layer = g < 0 ? -1 - g : g - n;
    return 0;
  }
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

// Which face states a predictor pass writes.
enum { PRED_ALL = 0, PRED_ZHI = 1, PRED_ZLO = 2 };

// MODE bit 0: gas + radiation EoS (Eq. 6-7); bit 1: dual-energy correction
// (Sect. 2.5); bit 2: a slab of a decomposed grid or a moving grid (exchanged
// ghosts, moving faces; ideal gas only).  Each combination is its own
// instantiation, so the plain step carries none of the optional work.
template <typename T, int DIM, int NSX, int RS, int MODE>
struct Sweep {
  static constexpr int EOS = MODE & 1;
  static constexpr bool DUAL = (MODE & 2) != 0;
  static constexpr bool XM = (MODE & 4) != 0;
  // in-step totals as compensated FP32 column sums (FP32, 3D) instead of FP64 sums per cell
  static constexpr bool COLSUM = sizeof(T) == 4 && DIM == 3;
  using S = SweepShape<T, DIM, NSX>;
  static constexpr int NV = S::NV, TX = S::TX, TY = S::TY, EX = S::EX, EY = S::EY, HY = S::HY,
                       QY = S::QY, NT = S::NT, NI = S::NI, NP = S::NP, NFX = S::NFX,
                       NFY = S::NFY, NFZ = S::NFZ;

  const SweepArgs<T>& a;
  T* Ws;  // primitive planes [slot][v][ey][ex]
  T* XL;  // x faces [v][row*(TX+1)+f]: left state, then the flux
  T* XR;  // x faces: right state
  T* YL;  // y faces [v][fy*TX+col]: left (lower) state, then the flux
  T* YR;
  T* ZL;  // [2][v][j*TX+i]: state below the z face above plane (slot = plane & 1)
  T* ZR;  // [v][j*TX+i]: state above the z face below the current plane, then the flux
  T* XQ;  // dual energy (Sect. 2.5): [2][face] u_f e_f and u_f of the x faces
  T* YQ;  //   ... of the y faces
  T* ZQ;  //   ... of the z face below the current plane
  // radiation EoS: temperatures of the parked face states (same indices as
  // XL/XR, YL/YR, ZL (two planes), ZR)
  T* XTL;
  T* XTR;
  T* YTL;
  T* YTR;
  T* ZTL;
  T* ZTR;
  T* WT;  // [slot][ey][ex] temperatures of the primitive planes
  T* GXs;  // [GX_*][px] geometry of predictor column px (cell x0 - 1 + px)
  T* GYs;  // [GY_*][py] geometry of predictor row py (cell y0 - 1 + py)
  double* tsum;  // [v][owner] sums of U dV of the owner's new cells (FP32 3D: float2 column sums
                 // until the end of the CTA, see close_cell), or null (totals off)
  int x0, y0, z1, n2;
  T dt, half_dt;
  const T* Uin;
  T* Uout;
  unsigned long long n_fallback = 0, n_iters = 0;
  int t_iters = 0;  // radiation EoS: temperature Newton iterations of this thread (reported as n_iters)
  int err = 0;
  T smax = T(0);  // max of the new states' signal speeds (FP32: the FP64 max of
                  // the same values, converted once at the end: the conversion is exact)
  T hfac = T(0);
  // owner registers: partial update of the owned cell, its predictor
  // increment (1D/2D) and the spherical partial sums of Eq. 13-16
  T acc[NV];
  T dUo[NV];
  T fzb3 = T(0), tth = T(0), x2 = T(0), s3 = T(0);
  T aq1 = T(0), aq2 = T(0);  // dual energy: divergences of u e and of u (times dt^-1)

  __device__ Sweep(const SweepArgs<T>& args, T* smem) : a(args) {
    Ws = smem;
    tsum = args.tot_part ? reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(smem) + S::tot_offset(MODE))
                         : nullptr;
    XL = Ws + S::WP * NV * S::WPL;
    XR = XL + NV * NFX;
    YL = XR + NV * NFX;
    YR = YL + NV * NFY;
    ZL = YR + NV * NFY;
    ZR = ZL + 2 * NV * NFZ;
    // the dual-energy and temperature arrays exist only in the instantiations
    // that use them
    XQ = ZR + NV * NFZ;
    YQ = XQ + 2 * NFX;
    ZQ = YQ + 2 * NFY;
    XTL = DUAL ? ZQ + 2 * NFZ : XQ;
    XTR = XTL + NFX;
    YTL = XTR + NFX;
    YTR = YTL + NFY;
    ZTL = YTR + NFY;
    ZTR = ZTL + 2 * NFZ;
    WT = ZTR + NFZ;
    GXs = Ws + S::smem_elems + (DUAL ? S::dual_elems : 0) + (EOS == 1 ? S::rad_elems : 0);
    GYs = GXs + S::GX_N * (TX + 2);
  }

  __device__ __forceinline__ T gx(int k, int px) const { return GXs[k * (TX + 2) + px]; }
  __device__ __forceinline__ T gy(int k, int py) const { return GYs[k * (TY + 2) + py]; }

  // Stage the x and y geometry factors of the CTA's cells (constant over
  // the march; read after the first barrier).  Indices are clamped to the
  // arrays' ranges: entries of columns or rows beyond the domain are never
  // used.
  __device__ void stage_geometry() {
    const int n0 = a.n[0], n1 = a.n[1];
    for (int p = threadIdx.x; p < TX + 2; p += NT) {
      const int gi = x0 - 1 + p;              // >= -1
      const int ge = min(gi, n0 + 1) + 2;     // extended (ghost) index
      const int gp = min(gi, n0) + 3;         // the face above, extended
      const int gc = min(max(gi, 0), n0 - 1);  // interior cell
      const int gf = min(max(gi, 0), n0);      // interior face
      T* g = GXs + p;
      constexpr int st = TX + 2;
      g[S::GX_IDM * st] = a.geo.inv_dxc[0][ge];
      g[S::GX_IDP * st] = a.geo.inv_dxc[0][gp];
      g[S::GX_HW * st] = a.geo.hw[0][ge];
      g[S::GX_IW * st] = a.geo.inv_w[0][ge];
      g[S::GX_IR * st] = a.spherical ? a.geo.inv_r[ge] : T(1);
      g[S::GX_AF * st] = a.geo.Af[gf];
      g[S::GX_INVA * st] = a.geo.inva[gc];
      g[S::GX_GA * st] = a.geo.ga[gc];
      g[S::GX_QR * st] = a.geo.qr[gc];
      g[S::GX_GR * st] = a.geo.gr[gc];
      g[S::GX_G * st] = a.gravity == GRAV_POINT ? a.geo.gpt[gc] : a.gravity == GRAV_MONO ? a.gmono[gc] : T(0);
    }
    if constexpr (DIM >= 2) {
      for (int p = threadIdx.x; p < TY + 2; p += NT) {
        const int gj = y0 - 1 + p;
        const int ge = min(gj, n1 + 1) + 2;
        const int gp = min(gj, n1) + 3;
        const int gc = min(max(gj, 0), n1 - 1);
        const int gf = min(max(gj, 0), n1);
        T* g = GYs + p;
        constexpr int st = TY + 2;
        g[S::GY_IDM * st] = a.geo.inv_dxc[1][ge];
        g[S::GY_IDP * st] = a.geo.inv_dxc[1][gp];
        g[S::GY_HW * st] = a.geo.hw[1][ge];
        g[S::GY_IW * st] = a.geo.inv_w[1][ge];
        g[S::GY_IS * st] = a.spherical ? a.geo.inv_s[ge] : T(1);
        g[S::GY_BF * st] = a.geo.Bf[gf];
        g[S::GY_INVB * st] = a.geo.invb[gc];
        g[S::GY_ZC * st] = a.geo.zc[gc];
        g[S::GY_GT * st] = a.geo.gt[gc];
        g[S::GY_QT * st] = a.geo.qt[gc];
      }
    }
  }

  // Dual energy (Sect. 2.5, reading R15): the advected internal energy
  // u_f e_f = F_rho (e/rho)_upwind and the face velocity u_f = F_rho/rho_upwind,
  // upwind by the sign of the mass flux.
  __device__ __forceinline__ void dual_terms(const T* WL, const T* WR, const T* F, T* q, int st,
                                             int idx) const {
    const T* Wu = F[0] >= T(0) ? WL : WR;
    const T eu = eint_of(gas(), Wu[0], Wu[1 + DIM]);
    q[idx] = F[0] * eu / Wu[0];
    q[st + idx] = F[0] / Wu[0];
  }

  // the EoS of this instantiation: ideal gas (Eq. 5) or gas + radiation (Eq. 6-7)
  __device__ __forceinline__ const auto& gas() const {
    if constexpr (EOS == 1) return a.grad;
    else return a.gas;
  }

  __device__ __forceinline__ T& W(int slot, int v, int ey, int ex) {
    return Ws[((slot * NV + v) * EY + ey) * EX + ex];
  }
  static __device__ __forceinline__ int wslot(int gz) { return DIM == 3 ? (gz + 6) % 3 : 0; }

  // a1 + a2: stage plane gz (axis-2 index, may be a ghost) as primitives.
  __device__ void load_plane(int gz) {
    const int n0 = a.n[0], n1 = a.n[1];
    bool fz = false;
    int lz = -1;
    int sz = 0;
    if constexpr (DIM == 3) {
      if constexpr (XM) sz = map_axis(gz, a.n[2], a.bc[2][0], a.bc[2][1], fz, lz);
      else sz = map_axis(gz, a.n[2], a.bc[2][0], a.bc[2][1], fz);
    }
    const int slot = wslot(gz);
    const int nvact = 2 + DIM + a.ns;
    // a staged region inside the domain on every axis: no ghost mapping
    const bool inner = !XM && x0 >= 2 && x0 + TX + 2 <= n0 &&
                       (DIM < 2 || (y0 >= HY && y0 + TY + HY <= n1)) && (DIM < 3 || (gz >= 0 && gz < a.n[2]));
    if (inner) {
      const long long zoff = (long long)gz * n1 * n0;
      for (int idx = threadIdx.x; idx < S::WPL; idx += NT) {
        const int ex = idx % EX, ey = idx / EX;
        const long long c = zoff + (long long)(y0 - HY + ey) * n0 + (x0 - 2 + ex);
        T u[NV], w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = v < nvact ? __ldg(Uin + (long long)v * a.ncell + c) : T(0);
        if constexpr (EOS == 1) {
          T c2, t;
          int k = 0;
          to_prim_ct<T, DIM, NSX>(u, w, c2, t, a.grad, T(0), &k);
          t_iters += k;
          WT[(slot * EY + ey) * EX + ex] = t;
        } else {
          to_prim<T, DIM, NSX>(u, w, gas());
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) W(slot, v, ey, ex) = w[v];
      }
      return;
    }
    for (int idx = threadIdx.x; idx < S::WPL; idx += NT) {
      const int ex = idx % EX, ey = idx / EX;
      const int gi = min(x0 - 2 + ex, n0 + 1);
      bool fx, fy = false;
      int lx = -1, ly = -1;
      int si, sj = 0, gj = 0;
      if constexpr (XM) si = map_axis(gi, n0, a.bc[0][0], a.bc[0][1], fx, lx);
      else si = map_axis(gi, n0, a.bc[0][0], a.bc[0][1], fx);
      if (DIM >= 2) {
        gj = min(y0 - HY + ey, n1 + 1);
        if constexpr (XM) sj = map_axis(gj, n1, a.bc[1][0], a.bc[1][1], fy, ly);
        else sj = map_axis(gj, n1, a.bc[1][0], a.bc[1][1], fy);
      }
      T u[NV], w[NV];
      const int layer = XM ? max(lx, max(ly, lz)) : -1;  // >= 0: a ghost of an exchanged side
      if (layer < 0) {
        const long long c = ((long long)sz * n1 + sj) * n0 + si;
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = v < nvact ? __ldg(Uin + (long long)v * a.ncell + c) : T(0);
      } else {
        // the neighbour subdomain's cell, from the halo of that side; the
        // other axes are mapped (and flipped) as for any ghost
        const int side = (lx >= 0 ? gi : ly >= 0 ? gj : gz) < 0 ? 0 : 1;
        const long long nx = a.xaxis == 0 ? (long long)n1 * a.n[2] : a.xaxis == 1 ? (long long)n0 * a.n[2]
                                                                                 : (long long)n0 * n1;
        const long long q = a.xaxis == 0 ? (long long)sz * n1 + sj : a.xaxis == 1 ? (long long)sz * n0 + si
                                                                                 : (long long)sj * n0 + si;
        const T* hp = a.halo[side] + (long long)layer * nx + q;
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = v < nvact ? hp[(long long)v * 2 * nx] : T(0);
      }
      if (fx) u[1] = -u[1];
      if (DIM >= 2 && fy) u[2] = -u[2];
      if (DIM == 3 && fz) u[3] = -u[3];
      if constexpr (EOS == 1) {
        T c2, t;
        int k = 0;  // (a local counter: a register after inlining)
        to_prim_ct<T, DIM, NSX>(u, w, c2, t, a.grad, T(0), &k);
        t_iters += k;
        WT[(slot * EY + ey) * EX + ex] = t;
      } else {
        to_prim<T, DIM, NSX>(u, w, gas());
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) W(slot, v, ey, ex) = w[v];
    }
  }

  // 1/h_d of the cell in predictor column px, row py, plane gk (physical
  // width: h_r = dr, h_th = r dth, h_ph = r s dph).
  __device__ __forceinline__ T inv_h(int d, int px, int py, int gk) const {
    if (d == 0) return gx(S::GX_IW, px);
    if (d == 1) {
      const T w = gy(S::GY_IW, py);
      return a.spherical ? w * gx(S::GX_IR, px) : w;
    }
    const T w = a.geo.inv_w[2][gk + 2];
    if constexpr (DIM >= 2) return a.spherical ? w * gx(S::GX_IR, px) * gy(S::GY_IS, py) : w;
    else return w;
  }

  // Limited low/high face states along DIR of the cell with centre Wc and
  // neighbours Wm/Wp; l = the cell's predictor column (DIR 0), row (DIR 1)
  // or plane index (DIR 2).
  template <int DIR>
  __device__ __forceinline__ void faces_of(const T* Wm, const T* Wc, const T* Wp, int l, T* Wlo,
                                           T* Whi) const {
    T idm, idp, h;
    if constexpr (DIR == 0) {
      idm = gx(S::GX_IDM, l);
      idp = gx(S::GX_IDP, l);
      h = gx(S::GX_HW, l);
    } else if constexpr (DIR == 1) {
      idm = gy(S::GY_IDM, l);
      idp = gy(S::GY_IDP, l);
      h = gy(S::GY_HW, l);
    } else {
      idm = a.geo.inv_dxc[DIR][l + 2];
      idp = a.geo.inv_dxc[DIR][l + 3];
      h = a.geo.hw[DIR][l + 2];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T sig = limit<T>(a.limiter, (Wc[v] - Wm[v]) * idm, (Wp[v] - Wc[v]) * idp);
      Wlo[v] = Wc[v] - h * sig;
      Whi[v] = Wc[v] + h * sig;
    }
  }

  // Predictor cell of item t: (px, py) in the (TX+2) x (TY+2QY) region around
  // the tile.  Items 0..NI-1 are the tile cells in owner order, then the
  // axis-0 halo columns, then the axis-1 halo rows (corners are never needed).
  static __device__ __forceinline__ void item_cell(int t, int& px, int& py) {
    if (t < NI) {
      px = 1 + t % TX;
      py = QY + t / TX;
      return;
    }
    int h = t - NI;
    if (h < 2 * TY) {
      px = h < TY ? 0 : TX + 1;
      py = QY + (h < TY ? h : h - TY);
      return;
    }
    h -= 2 * TY;
    px = 1 + (h < TX ? h : h - TX);
    py = h < TX ? 0 : TY + 1;
  }

  // Turn the limited state parked at p (stride `st`) into the predicted face
  // state: W -> U, + dU, U -> W; a non-physical result falls back to Wc.
  // The radiation EoS parks the conserved state (the flux evaluation already
  // solved for its energy) and records the temperature of the result at tp.
  __device__ __forceinline__ void finish_state(T* p, int st, const T* Wc, const T* dU, bool owned,
                                               T* tp = nullptr) {
    T w[NV], u[NV];
    if constexpr (EOS == 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = p[v * st] + dU[v];
      const T rho = u[0], ir = T(1) / rho;
      T ke = T(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        w[1 + d] = u[1 + d] * ir;
        ke += u[1 + d] * w[1 + d];
      }
      w[0] = rho;
      T c2, t;
      int k = 0;
      a.grad.from_e_t(rho, u[1 + DIM] - T(0.5) * ke, w[1 + DIM], c2, t, *tp, &k);
#pragma unroll
      for (int s = 0; s < NSX; ++s) w[2 + DIM + s] = u[2 + DIM + s] * ir;
      if (!(w[0] > T(0)) || !(w[1 + DIM] > T(0))) {
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = Wc[v];
        t = a.grad.temp_p(Wc[0], Wc[1 + DIM], *tp, &k);
        if (owned) ++n_fallback;
      }
      *tp = t;
      t_iters += k;
    } else {
      // the slot holds the limited state's conserved form (limited_fluxes)
#pragma unroll
      for (int v = 0; v < NV; ++v) u[v] = p[v * st] + dU[v];
      to_prim<T, DIM, NSX>(u, w, gas());
      if (!(w[0] > T(0)) || !(w[1 + DIM] > T(0))) {
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = Wc[v];
        if (owned) ++n_fallback;
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) p[v * st] = w[v];
  }

  // Physical fluxes of the two limited states of one direction and what is
  // parked in their face slots: their conserved states (for the radiation
  // EoS from the same temperature solve).
  // (radiation EoS: tc = the cell's temperature, the Newton start; tl/th
  // receive the limited states' temperatures)
  template <int DIR>
  __device__ __forceinline__ void limited_fluxes(const T* Wl, const T* Wh, T* Fl, T* Fh, T* Pl, T* Ph,
                                                 T tc = T(0), T* tl = nullptr, T* th = nullptr) {
    if constexpr (EOS == 1) {
      T c2;
      int k = 0;
      *tl = a.grad.temp_p(Wl[0], Wl[1 + DIM], tc, &k);
      *th = a.grad.temp_p(Wh[0], Wh[1 + DIM], tc, &k);
      t_iters += k;
      T el, eh;
      a.grad.from_t(Wl[0], *tl, el, c2);
      a.grad.from_t(Wh[0], *th, eh, c2);
      flux_cons_e<T, DIM, NSX, DIR>(Wl, el, Fl, Pl);
      flux_cons_e<T, DIM, NSX, DIR>(Wh, eh, Fh, Ph);
    } else {
      // the fluxes and the conserved states together (the same operations
      // as phys_flux and to_cons, each done once)
      flux_cons_e<T, DIM, NSX, DIR>(Wl, Wl[1 + DIM] * a.gas.igm1, Fl, Pl);
      flux_cons_e<T, DIM, NSX, DIR>(Wh, Wh[1 + DIM] * a.gas.igm1, Fh, Ph);
    }
  }

  // Moving grid (reading R16): along the moving axis the predictor uses the
  // fluxes through faces that move with the grid, F - w U (ideal gas).
  // (ul, uh: the limited states' conserved forms, as parked by limited_fluxes)
  __device__ __forceinline__ void moving_fluxes(const T* ul, const T* uh, T* Fl, T* Fh) const {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Fl[v] -= a.wg * ul[v];
      Fh[v] -= a.wg * uh[v];
    }
  }

  // a3 + a4 for plane gz: the predictor increment dU = dt/2 sum_d
  // (F_d(W_lo) - F_d(W_hi))/h_d of every needed cell, and its predicted face
  // states.  PRED_ALL: tile plus halo, every face state of the plane;
  // PRED_ZHI / PRED_ZLO: tile cells only, the upper / lower z state.
  template <int PM>
  __device__ void predictor(int gz) {
    const int t = threadIdx.x;
    if (t >= (PM == PRED_ALL ? NP : NI)) return;
    const int n0 = a.n[0], n1 = a.n[1];
    int px, py;
    item_cell(t, px, py);
    const int gi = x0 - 1 + px;
    const int gj = DIM >= 2 ? y0 - 1 + py : 0;
    if (gi > n0 || (DIM >= 2 && gj > n1)) return;
    const int slot = wslot(gz);
    const int ex = px + 1, ey = py + (HY - QY);
    const bool trow = DIM < 2 || (py >= 1 && py <= TY);  // a tile row
    const bool tcol = px >= 1 && px <= TX;               // a tile column
    const bool rreal = DIM < 2 || gj < n1;               // a domain row
    const bool creal = gi < n0;                          // a domain column
    const int row = py - QY, col = px - 1;
    // face-state slots written by this cell
    const bool xlo = PM == PRED_ALL && px >= 1 && trow && rreal;
    const bool xhi = PM == PRED_ALL && px <= TX && trow && rreal && creal;
    const bool ylo = DIM >= 2 && PM == PRED_ALL && py >= 1 && tcol && creal;
    const bool yhi = DIM >= 2 && PM == PRED_ALL && py <= TY && tcol && creal && rreal;
    const bool zin = DIM == 3 && tcol && trow && creal && rreal;
    const bool zlo = zin && PM != PRED_ZHI;
    const bool zhi = zin && PM != PRED_ZLO;
    const int ixlo = row * (TX + 1) + px - 1, ixhi = ixlo + 1;
    const int iylo = (py - 1) * TX + col, iyhi = iylo + TX;
    const int iz = row * TX + col;
    T* zhp = ZL + (gz & 1) * NV * NFZ;

    T Wc[NV], dU[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Wc[v] = W(slot, v, ey, ex);
      dU[v] = T(0);
    }
    const T tcell = EOS == 1 ? WT[(slot * EY + ey) * EX + ex] : T(0);
    {
      T Wm[NV], Wp[NV], Wl[NV], Wh[NV], Fl[NV], Fh[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Wm[v] = W(slot, v, ey, ex - 1);
        Wp[v] = W(slot, v, ey, ex + 1);
      }
      faces_of<0>(Wm, Wc, Wp, px, Wl, Wh);
      T Pl[NV], Ph[NV], tl = T(0), th = T(0);
      limited_fluxes<0>(Wl, Wh, Fl, Fh, Pl, Ph, tcell, &tl, &th);
      if constexpr (XM) {
        if (a.maxis == 0) moving_fluxes(Pl, Ph, Fl, Fh);
      }
      if constexpr (EOS == 1) {
        if (xlo) XTR[ixlo] = tl;
        if (xhi) XTL[ixhi] = th;
      }
      const T ih = inv_h(0, px, py, gz);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        dU[v] += (Fl[v] - Fh[v]) * ih;
        if (xlo) XR[v * NFX + ixlo] = Pl[v];
        if (xhi) XL[v * NFX + ixhi] = Ph[v];
      }
    }
    if constexpr (DIM >= 2) {
      T Wm[NV], Wp[NV], Wl[NV], Wh[NV], Fl[NV], Fh[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Wm[v] = W(slot, v, ey - 1, ex);
        Wp[v] = W(slot, v, ey + 1, ex);
      }
      faces_of<1>(Wm, Wc, Wp, py, Wl, Wh);
      T Pl[NV], Ph[NV], tl = T(0), th = T(0);
      limited_fluxes<1>(Wl, Wh, Fl, Fh, Pl, Ph, tcell, &tl, &th);
      if constexpr (XM) {
        if (a.maxis == 1) moving_fluxes(Pl, Ph, Fl, Fh);
      }
      if constexpr (EOS == 1) {
        if (ylo) YTR[iylo] = tl;
        if (yhi) YTL[iyhi] = th;
      }
      const T ih = inv_h(1, px, py, gz);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        dU[v] += (Fl[v] - Fh[v]) * ih;
        if (ylo) YR[v * NFY + iylo] = Pl[v];
        if (yhi) YL[v * NFY + iyhi] = Ph[v];
      }
    }
    if constexpr (DIM == 3) {
      T Wm[NV], Wp[NV], Wl[NV], Wh[NV], Fl[NV], Fh[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Wm[v] = W(wslot(gz - 1), v, ey, ex);
        Wp[v] = W(wslot(gz + 1), v, ey, ex);
      }
      faces_of<2>(Wm, Wc, Wp, gz, Wl, Wh);
      T Pl[NV], Ph[NV], tl = T(0), th = T(0);
      limited_fluxes<2>(Wl, Wh, Fl, Fh, Pl, Ph, tcell, &tl, &th);
      if constexpr (XM) {
        if (a.maxis == 2) moving_fluxes(Pl, Ph, Fl, Fh);
      }
      if constexpr (EOS == 1) {
        if (zlo) ZTR[iz] = tl;
        if (zhi) ZTL[(gz & 1) * NFZ + iz] = th;
      }
      const T ih = inv_h(2, px, py, gz);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        dU[v] += (Fl[v] - Fh[v]) * ih;
        if (zlo) ZR[v * NFZ + iz] = Pl[v];
        if (zhi) zhp[v * NFZ + iz] = Ph[v];
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[v] = half_dt * dU[v];
    if constexpr (DIM < 3) {
      if (t < NI) {
#pragma unroll
        for (int v = 0; v < NV; ++v) dUo[v] = dU[v];
      }
    }
    // A face is counted (fallbacks, Newton iterations) by the one CTA that
    // owns it: its tile's faces except the upper edge, unless that is the
    // domain's last face.
    T* ztl = ZTL + (gz & 1) * NFZ;
    if (xlo) finish_state(XR + ixlo, NFX, Wc, dU, px - 1 < TX || gi == n0, XTR + ixlo);
    if (xhi) finish_state(XL + ixhi, NFX, Wc, dU, px < TX || gi + 1 == n0, XTL + ixhi);
    if constexpr (DIM >= 2) {
      if (ylo) finish_state(YR + iylo, NFY, Wc, dU, py - 1 < TY || gj == n1, YTR + iylo);
      if (yhi) finish_state(YL + iyhi, NFY, Wc, dU, py < TY || gj + 1 == n1, YTL + iyhi);
    }
    if constexpr (DIM == 3) {
      if (zlo) finish_state(ZR + iz, NFZ, Wc, dU, gz < z1 || gz == n2, ZTR + iz);
      if (zhi) finish_state(zhp + iz, NFZ, Wc, dU, gz + 1 < z1 || gz + 1 == n2, ztl + iz);
    }
  }

  // Riemann flux of a face along DIR.  On the moving axis (reading R16) the
  // flux through the moving face, F - w U on the face path x/t = w, is the
  // fixed-face flux of the same two states seen from the frame that moves
  // with the face (normal velocities minus w; every solver here is Galilean
  // invariant), taken back to the lab frame: mass flux unchanged, normal
  // momentum flux + w F_rho, energy flux + w F_m + w^2/2 F_rho.
  // (One call site of the solver: on a fixed axis w = 0 and the shift is
  // exact, so the fixed grid computes what it computed without this.)
  template <int DIR>
  __device__ __forceinline__ void riemann(const T* WL, const T* WR, T* F, bool owned, T TL = T(0),
                                          T TR = T(0)) {
    if constexpr (!XM) {
      riemann_fixed<DIR>(WL, WR, F, owned, TL, TR);
      return;
    }
    const bool mv = a.maxis == DIR;
    const T w = mv ? a.wg : T(0);
    T wl[NV], wr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wl[v] = WL[v];
      wr[v] = WR[v];
    }
    wl[1 + DIR] -= w;
    wr[1 + DIR] -= w;
    riemann_fixed<DIR>(wl, wr, F, owned, TL, TR);
    if (mv) {
      F[1 + DIM] += w * F[1 + DIR] + T(0.5) * w * w * F[0];
      F[1 + DIR] += w * F[0];
    }
  }

  template <int DIR>
  __device__ __forceinline__ void riemann_fixed(const T* WL, const T* WR, T* F, bool owned, T TL = T(0),
                                                T TR = T(0)) {
    if constexpr (EOS == 1 && RS == RS_HLL) {
      riemann_hll_rad<T, DIM, NSX, DIR>(WL, WR, F, a.grad, TL, TR);
    } else if constexpr (EOS == 1 && RS == RS_HLLC) {
      riemann_hllc_rad<T, DIM, NSX, DIR>(WL, WR, F, a.grad, TL, TR);
    } else if constexpr (RS == RS_HLL) {
      riemann_hll<T, DIM, NSX, DIR>(WL, WR, F, gas());
    } else if constexpr (RS == RS_HLLC) {
      riemann_hllc<T, DIM, NSX, DIR>(WL, WR, F, gas());
    } else {
      int it = 0, kind = 0;
      const int st = riemann_exact<T, DIM, NSX, DIR>(WL, WR, F, a.gas, T(0), it, kind);
      if (owned) n_iters += it;
      if (st != ST_OK && err == 0) err = st;
    }
  }

  // a5: one Riemann solve per face, the flux written over the left state.
  // XY: the x and y faces of the current plane; Z: the z face below plane gz.
  template <bool XY, bool Z>
  __device__ void faces(int gz) {
    const int n0 = a.n[0], n1 = a.n[1];
    constexpr int NXY = XY ? NFX + NFY : 0;
    constexpr int NALL = NXY + (Z ? NFZ : 0);
    const T* zlp = ZL + ((gz - 1) & 1) * NV * NFZ;
    constexpr bool dual = DUAL;
    for (int idx = threadIdx.x; idx < NALL; idx += NT) {
      T WL[NV], WR[NV], F[NV];
      if (XY && idx < NFX) {
        const int f = idx % (TX + 1), row = idx / (TX + 1);
        if (x0 + f > n0 || (DIM >= 2 && y0 + row >= n1)) continue;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          WL[v] = XL[v * NFX + idx];
          WR[v] = XR[v * NFX + idx];
        }
        riemann<0>(WL, WR, F, f < TX || x0 + f == n0, EOS ? XTL[idx] : T(0), EOS ? XTR[idx] : T(0));
        if constexpr (dual) dual_terms(WL, WR, F, XQ, NFX, idx);
#pragma unroll
        for (int v = 0; v < NV; ++v) XL[v * NFX + idx] = F[v];
      } else if (XY && DIM >= 2 && idx < NXY) {
        const int k = idx - NFX;
        const int col = k % TX, fy = k / TX;
        if (x0 + col >= n0 || y0 + fy > n1) continue;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          WL[v] = YL[v * NFY + k];
          WR[v] = YR[v * NFY + k];
        }
        riemann<(DIM >= 2 ? 1 : 0)>(WL, WR, F, fy < TY || y0 + fy == n1, EOS ? YTL[k] : T(0),
                                    EOS ? YTR[k] : T(0));
        if constexpr (dual) dual_terms(WL, WR, F, YQ, NFY, k);
#pragma unroll
        for (int v = 0; v < NV; ++v) YL[v * NFY + k] = F[v];
      } else if (DIM == 3 && Z) {
        const int k = idx - NXY;
        const int i = k % TX, j = k / TX;
        if (x0 + i >= n0 || y0 + j >= n1) continue;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          WL[v] = zlp[v * NFZ + k];
          WR[v] = ZR[v * NFZ + k];
        }
        riemann<(DIM == 3 ? 2 : 0)>(WL, WR, F, gz < z1 || gz == n2,
                                    EOS ? ZTL[((gz - 1) & 1) * NFZ + k] : T(0), EOS ? ZTR[k] : T(0));
        if constexpr (dual) dual_terms(WL, WR, F, ZQ, NFZ, k);
#pragma unroll
        for (int v = 0; v < NV; ++v) ZR[v * NFZ + k] = F[v];
      }
    }
  }

  // a6 flux differences of the owned cell (i, j) from the x and y faces of
  // the current plane, plus (3D) the lower z face of plane gz; also the
  // spherical partial sums that use these fluxes.
  __device__ __forceinline__ void open_cell(int gz, int i, int j, int gi, int gj) {
    const int fx = j * (TX + 1) + i;
    const T Afl = gx(S::GX_AF, i + 1), Afh = gx(S::GX_AF, i + 2), ia = gx(S::GX_INVA, i + 1);
    constexpr bool dual = DUAL;
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = (XL[v * NFX + fx] * Afl - XL[v * NFX + fx + 1] * Afh) * ia;
    if constexpr (dual) {
      aq1 = (XQ[fx] * Afl - XQ[fx + 1] * Afh) * ia;
      aq2 = (XQ[NFX + fx] * Afl - XQ[NFX + fx + 1] * Afh) * ia;
    }
    if constexpr (DIM >= 2) {
      const T Bfl = gy(S::GY_BF, j + 1), Bfh = gy(S::GY_BF, j + 2);
      const T cy = gx(S::GX_GA, i + 1) * gy(S::GY_INVB, j + 1);
      const int fy = j * TX + i;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += (YL[v * NFY + fy] * Bfl - YL[v * NFY + fy + TX] * Bfh) * cy;
      if constexpr (dual) {
        aq1 += (YQ[fy] * Bfl - YQ[fy + TX] * Bfh) * cy;
        aq2 += (YQ[NFY + fy] * Bfl - YQ[NFY + fy + TX] * Bfh) * cy;
      }
      if (a.spherical) {
        tth = T(0.5) * (YL[2 * NFY + fy] + YL[2 * NFY + fy + TX]);
        x2 = XL[2 * NFX + fx + 1] * Afh + XL[2 * NFX + fx] * Afl;
        if constexpr (DIM == 3) {
          const T frl = XL[3 * NFX + fx], frh = XL[3 * NFX + fx + 1];
          const T ftl = YL[3 * NFY + fy], fth = YL[3 * NFY + fy + TX];
          s3 = -gx(S::GX_QR, i + 1) * (frh * Afh + frl * Afl) -
               gx(S::GX_GA, i + 1) * gy(S::GY_QT, j + 1) * (fth * Bfh + ftl * Bfl);
        }
      }
    }
    if constexpr (DIM == 3) {
      const int iz = j * TX + i;
      const T cz = gx(S::GX_GA, i + 1) * gy(S::GY_ZC, j + 1) * a.geo.invc[gz];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += ZR[v * NFZ + iz] * cz;
      fzb3 = ZR[3 * NFZ + iz];
      if constexpr (dual) {
        aq1 += ZQ[iz] * cz;
        aq2 += ZQ[NFZ + iz] * cz;
      }
    }
  }

  // a6-a9: the new state of the owned cell (i, j) of plane gz from acc, the
  // sources, the validity checks and the signal speed.  fzt3 = the axis-2
  // momentum flux of the upper z face (3D).
  __device__ void close_cell(int gz, int i, int j, int gi, int gj, T fzt3) {
    const int n0 = a.n[0], n1 = a.n[1];
    const int nvact = 2 + DIM + a.ns;
    const long long c = ((long long)gz * n1 + gj) * n0 + gi;
    T Uo[NV], Un[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Uo[v] = v < nvact ? Uin[(long long)v * a.ncell + c] : T(0);
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
        for (int v = 0; v < NV; ++v) Uh[v] = Uo[v] + dUo[v];
        to_prim<T, DIM, NSX>(Uh, Wh, gas());
        to_prim<T, DIM, NSX>(Uo, Wo, gas());
        P = (Wh[0] > T(0) && Wh[1 + DIM] > T(0)) ? Wh[1 + DIM] : Wo[1 + DIM];
      }
      T Tth = P, Tph = P;
      if constexpr (DIM >= 2) Tth = tth;
      if constexpr (DIM == 3) Tph = T(0.5) * (fzb3 + fzt3);
      Un[1] += dt * T(0.5) * (Tth + Tph) * gx(S::GX_GR, i + 1);
      if constexpr (DIM >= 2)
        Un[2] += dt * (-gx(S::GX_QR, i + 1) * x2 + Tph * gx(S::GX_GA, i + 1) * gy(S::GY_GT, j + 1));
      if constexpr (DIM == 3) Un[3] += dt * s3;
    }
    if (a.gravity != GRAV_NONE) {
      T g[3] = {T(0), T(0), T(0)};
      if (a.gravity == GRAV_UNIFORM) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) g[d] = a.g0[d];
      } else {
        g[0] = gx(S::GX_G, i + 1);  // point mass or monopole
      }
      T work = T(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        Un[1 + d] += dt * Uo[0] * g[d];
        work += Uo[1 + d] * g[d];
      }
      Un[1 + DIM] += dt * work;
    }
    T dheat = T(0);
    if (a.heating == HEAT_CONST) {
      dheat = dt * a.heat_q;
      Un[1 + DIM] += dheat;
    } else if (a.heating == HEAT_NI56) {
      T rf = T(0);
#pragma unroll
      for (int s = 0; s < NSX; ++s)
        if (s == a.ni_index) rf = Uo[2 + DIM + s];
      dheat = dt * hfac * rf;
      Un[1 + DIM] += dheat;
    }

    // Dual energy (Sect. 2.5): where e is small against the kinetic energy
    // of the t^n state, blend the internal-energy change of the total-energy
    // update with that of de/dt + div(u e) + P div(u) = 0 (plus heating).
    if constexpr (DUAL) {
      T ke0 = T(0), ke1 = T(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        ke0 += T(0.5) * Uo[1 + d] * Uo[1 + d] / Uo[0];
        ke1 += T(0.5) * Un[1 + d] * Un[1 + d] / Un[0];
      }
      const T e0 = Uo[1 + DIM] - ke0;
      const T crit = a.eps_dual * ke0;
      const T alpha = e0 >= crit ? T(1) : (e0 > T(0.1) * crit ? (e0 / crit) * (e0 / crit) : T(0));
      if (alpha < T(1)) {
        T Wo[NV];
        to_prim<T, DIM, NSX>(Uo, Wo, gas());
        const T d1 = (Un[1 + DIM] - ke1) - e0;
        const T d2 = dt * (aq1 + Wo[1 + DIM] * aq2) + dheat;
        Un[1 + DIM] = e0 + alpha * d1 + (T(1) - alpha) * d2 + ke1;
      }
    }

    // moving radial grid: the old cell's content spread over the new volume
    if (XM && a.vr) {
      const T q = a.vr[gi];
#pragma unroll
      for (int v = 0; v < NV; ++v) Un[v] *= q;
    }

    // the new cell's share of the conserved totals, in the owner's sum
    if (tsum) {
      const int o = j * TX + i;
      if constexpr (COLSUM) {
        // FP32 3D: per owner and variable a compensated FP32 sum (hi, lo) of
        // U dz along the owner's column, dz = dvol[2][gz] given as the FP32
        // pair hi + lo.  Each product is split exactly by an FMA, the sum
        // kept as an unevaluated pair (TwoSum, then renormalised), so each
        // term costs ~2^-48 of the sum; the column's sum is multiplied by
        // dvol[0] dvol[1] in FP64 at the end of the CTA.  (The _rn
        // intrinsics keep the compiler from fusing these operations.)
        const float2 z = a.dvz32[gz];
        float2* ts = reinterpret_cast<float2*>(tsum);
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v < nvact) {
            const float x = Un[v];
            const float p = __fmul_rn(x, z.x);
            const float e = fmaf(x, z.y, fmaf(x, z.x, -p));
            float2 sv = ts[v * NI + o];
            const float t = __fadd_rn(sv.x, p);
            const float bb = __fsub_rn(t, sv.x);
            const float r = __fadd_rn(__fsub_rn(sv.x, __fsub_rn(t, bb)), __fsub_rn(p, bb));
            const float lo = __fadd_rn(sv.y, __fadd_rn(r, e));
            sv.x = __fadd_rn(t, lo);
            sv.y = __fsub_rn(lo, __fsub_rn(sv.x, t));
            ts[v * NI + o] = sv;
          }
      } else {
        // FP64 sums of U dV
        double dV = a.dvol[0][gi];
        if constexpr (DIM >= 2) dV *= a.dvol[1][gj];
        if constexpr (DIM == 3) dV *= a.dvol[2][gz];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v < nvact) tsum[v * NI + o] += (double)Un[v] * dV;
      }
    }

    // validity and the signal speed of the new state
    T Wn[NV], c2n;
    if constexpr (EOS == 1) {
      T tn;
      int k = 0;
      to_prim_ct<T, DIM, NSX>(Un, Wn, c2n, tn, a.grad, WT[(wslot(gz) * EY + j + HY) * EX + i + 2], &k);
      t_iters += k;
    } else {
      to_prim<T, DIM, NSX>(Un, Wn, a.gas);
      c2n = qdiv(a.gas.g * Wn[1 + DIM], Wn[0]);
    }
    bool finite = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) finite = finite && isfinite(Un[v]);
    if (!finite) err = err ? err : ST_NONFINITE;
    else if (!(Wn[0] > T(0)) || !(Wn[1 + DIM] > T(0))) err = err ? err : ST_NEG;
    const T cs = dsqrt(c2n);
    T sp = T(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      T ih = inv_h(d, i + 1, j + 1, gz);
      T ud = Wn[1 + d];
      if constexpr (XM) {
        // a moving radial grid: the new state lives in the moved cell, whose
        // angular widths scale with its new radius; on the moving axis the
        // speed counts relative to the faces
        if (d >= 1 && a.ir_new) ih *= a.ir_new[gi] / a.geo.inv_r[gi + 2];
        if (d == a.maxis) ud -= a.wg;
      }
      sp += (fabs(ud) + cs) * ih;
    }
    smax = fmax(smax, sp);
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (v < nvact) Uout[(long long)v * a.ncell + c] = Un[v];
  }

  // The owner's work after the face solves of plane gz: in 3D, close the
  // cell of plane gz-1 with the flux of the z face between them and open
  // the cell of plane gz; in 1D/2D both in one go.
  __device__ void owner_step(int gz, bool close_prev, bool open_cur) {
    const int t = threadIdx.x;
    if (t >= NI) return;
    const int i = t % TX, j = t / TX;
    const int gi = x0 + i, gj = y0 + j;
    if (gi >= a.n[0] || (DIM >= 2 && gj >= a.n[1])) return;
    if constexpr (DIM == 3) {
      if (close_prev) {
        const T cz = gx(S::GX_GA, i + 1) * gy(S::GY_ZC, j + 1) * a.geo.invc[gz - 1];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] -= ZR[v * NFZ + t] * cz;
        if constexpr (DUAL) {
          aq1 -= ZQ[t] * cz;
          aq2 -= ZQ[NFZ + t] * cz;
        }
        close_cell(gz - 1, i, j, gi, gj, ZR[3 * NFZ + t]);
      }
      if (open_cur) open_cell(gz, i, j, gi, gj);
    } else {
      open_cell(0, i, j, gi, gj);
      close_cell(0, i, j, gi, gj, T(0));
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

template <typename T, int DIM, int NSX, int RS, int MODE>
__global__ void __launch_bounds__(SweepShape<T, DIM, NSX>::NT,
                                  (RS == RS_EXACT || (MODE & 1)) ? 1 : SweepShape<T, DIM, NSX>::MB)
    sweep_kernel(const SweepArgs<T> args) {
  using S = SweepShape<T, DIM, NSX>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double dtd, t;
  long long step;
  int cur;
  if (!step_begin(args.ctrl, args.dt_host, args.cfl, args.t_end, dtd, t, step, cur)) return;

  Sweep<T, DIM, NSX, RS, MODE> sw(args, reinterpret_cast<T*>(smem_raw));
  if (sw.tsum)
    for (int q = threadIdx.x; q < S::NI * S::NV; q += S::NT) sw.tsum[q] = 0.0;  // (read after later barriers)
  sw.x0 = blockIdx.x * S::TX;
  sw.y0 = blockIdx.y * S::TY;
  sw.stage_geometry();  // (read after the first barrier below)
  sw.n2 = DIM == 3 ? args.n[2] : 1;
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
    sw.z1 = z1;
    for (int q = z0 - 2; q <= z0; ++q) sw.load_plane(q);
    __syncthreads();
    sw.template predictor<PRED_ZHI>(z0 - 1);
    __syncthreads();
    // Plane k: its face states, then its x/y faces and the z face below it;
    // the owners close plane k-1 and open plane k.  k = z1 only supplies the
    // z face above the chunk's last plane.
    for (int k = z0; k <= z1; ++k) {
      sw.load_plane(k + 1);
      __syncthreads();
      if (k < z1) sw.template predictor<PRED_ALL>(k);
      else sw.template predictor<PRED_ZLO>(k);
      __syncthreads();
      if (k < z1) sw.template faces<true, true>(k);
      else sw.template faces<false, true>(k);
      __syncthreads();
      sw.owner_step(k, k > z0, k < z1);
    }
  } else {
    sw.z1 = 1;
    sw.load_plane(0);
    __syncthreads();
    sw.template predictor<PRED_ALL>(0);
    __syncthreads();
    sw.template faces<true, false>(0);
    __syncthreads();
    sw.owner_step(0, false, true);
  }
  __syncthreads();
  if (sw.tsum) {
    if constexpr (decltype(sw)::COLSUM) {
      // each owner's compensated column sums, times its column's dvol[0]
      // dvol[1], in FP64 and in place
      for (int q = threadIdx.x; q < S::NI * S::NV; q += S::NT) {
        const int o = q % S::NI;
        const int gi = sw.x0 + o % S::TX, gj = sw.y0 + o / S::TX;
        const float2 c = reinterpret_cast<const float2*>(sw.tsum)[q];
        const double w = (gi < args.n[0] && gj < args.n[1]) ? args.dvol[0][gi] * args.dvol[1][gj] : 0.0;
        sw.tsum[q] = ((double)c.x + (double)c.y) * w;
      }
      __syncthreads();
    }
    // the CTA's totals: the owners' sums by a tree in a fixed order, per
    // variable, so the result does not depend on scheduling
    constexpr int P2 = pow2_ceil(S::NI);
    for (int w = P2 / 2; w > 0; w >>= 1) {
      for (int q = threadIdx.x; q < S::NV * w; q += S::NT) {
        const int v = q / w, o = q - v * w;
        if (o + w < S::NI) sw.tsum[v * S::NI + o] += sw.tsum[v * S::NI + o + w];
      }
      __syncthreads();
    }
    const long long ncta = (long long)gridDim.x * gridDim.y * gridDim.z;
    const long long cta = blockIdx.x + gridDim.x * ((long long)blockIdx.y + (long long)gridDim.y * blockIdx.z);
    if (threadIdx.x < S::NV) args.tot_part[threadIdx.x * ncta + cta] = sw.tsum[threadIdx.x * S::NI];
  }
  finish_step<S::NT>(args.ctrl, (double)sw.smax, sw.err, sw.n_fallback,
                     (MODE & 1) ? (unsigned long long)sw.t_iters : sw.n_iters, 0ull, step, dtd);
}

template <typename T, int DIM, int NSX, int RS, int MODE>
cudaError_t launch_sweep(const SweepArgs<T>& a, cudaStream_t s) {
  using S = SweepShape<T, DIM, NSX>;
  const size_t smem = a.tot_part ? S::tot_offset(MODE) + S::tot_bytes : S::smem_bytes_for(MODE);
  cudaError_t e = smem_attr_once((const void*)sweep_kernel<T, DIM, NSX, RS, MODE>, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.n[0] + S::TX - 1) / S::TX, DIM >= 2 ? (a.n[1] + S::TY - 1) / S::TY : 1,
            DIM == 3 ? (a.n[2] + a.zchunk - 1) / a.zchunk : 1);
  sweep_kernel<T, DIM, NSX, RS, MODE><<<grid, S::NT, smem, s>>>(a);
  return cudaGetLastError();
}

// Launch one instantiation and report its tile shape and threads per CTA.
template <typename T, int DIM, int NSX, int RS, int MODE = 0>
cudaError_t launch_sweep_shape(const SweepArgs<T>& a, cudaStream_t s, int* tx, int* ty, int* nt) {
  using S = SweepShape<T, DIM, NSX>;
  *tx = S::TX;
  *ty = S::TY;
  *nt = S::NT;
  return launch_sweep<T, DIM, NSX, RS, MODE>(a, s);
}

// Instantiate the dispatcher of one (precision, dimension) pair and MODE
// (ideal gas: 0, ideal gas + dual energy: 2).
#define HYDRO_SWEEP_DISPATCH_MODE(NAME, T, DIM, MODE)                                         \
  template <>                                                                                 \
  cudaError_t NAME<T, DIM>(const SweepArgs<T>& a, int nsx, int rs, cudaStream_t s, int* tx,   \
                           int* ty, int* nt) {                                                \
    switch (nsx * 4 + rs) {                                                                   \
      case 0: return launch_sweep_shape<T, DIM, 0, RS_HLL, MODE>(a, s, tx, ty, nt);           \
      case 1: return launch_sweep_shape<T, DIM, 0, RS_HLLC, MODE>(a, s, tx, ty, nt);          \
      case 2: return launch_sweep_shape<T, DIM, 0, RS_EXACT, MODE>(a, s, tx, ty, nt);         \
      case 4: return launch_sweep_shape<T, DIM, 1, RS_HLL, MODE>(a, s, tx, ty, nt);           \
      case 5: return launch_sweep_shape<T, DIM, 1, RS_HLLC, MODE>(a, s, tx, ty, nt);          \
      case 6: return launch_sweep_shape<T, DIM, 1, RS_EXACT, MODE>(a, s, tx, ty, nt);         \
      case 12: return launch_sweep_shape<T, DIM, 3, RS_HLL, MODE>(a, s, tx, ty, nt);          \
      case 13: return launch_sweep_shape<T, DIM, 3, RS_HLLC, MODE>(a, s, tx, ty, nt);         \
      case 14: return launch_sweep_shape<T, DIM, 3, RS_EXACT, MODE>(a, s, tx, ty, nt);        \
      default: return cudaErrorInvalidValue;                                                  \
    }                                                                                         \
  }
#define HYDRO_SWEEP_DISPATCH(T, DIM) HYDRO_SWEEP_DISPATCH_MODE(sweep_dispatch, T, DIM, 0)
#define HYDRO_SWEEP_DISPATCH_DUAL(T, DIM) HYDRO_SWEEP_DISPATCH_MODE(sweep_dispatch_dual, T, DIM, 2)
#define HYDRO_SWEEP_DISPATCH_XM(T, DIM) HYDRO_SWEEP_DISPATCH_MODE(sweep_dispatch_xm, T, DIM, 4)

// The gas + radiation dispatcher (HLL, HLLC) of one (precision, dimension)
// pair, without (MODE 1) and with (MODE 3) the dual-energy correction.
#define HYDRO_SWEEP_DISPATCH_RAD(T, DIM)                                                      \
  template <>                                                                                 \
  cudaError_t sweep_dispatch_rad<T, DIM>(const SweepArgs<T>& a, int nsx, int rs, int dual,    \
                                         cudaStream_t s, int* tx, int* ty, int* nt) {         \
    switch ((nsx * 4 + rs) * 2 + (dual ? 1 : 0)) {                                            \
      case 0: return launch_sweep_shape<T, DIM, 0, RS_HLL, 1>(a, s, tx, ty, nt);              \
      case 1: return launch_sweep_shape<T, DIM, 0, RS_HLL, 3>(a, s, tx, ty, nt);              \
      case 2: return launch_sweep_shape<T, DIM, 0, RS_HLLC, 1>(a, s, tx, ty, nt);             \
      case 3: return launch_sweep_shape<T, DIM, 0, RS_HLLC, 3>(a, s, tx, ty, nt);             \
      case 8: return launch_sweep_shape<T, DIM, 1, RS_HLL, 1>(a, s, tx, ty, nt);              \
      case 9: return launch_sweep_shape<T, DIM, 1, RS_HLL, 3>(a, s, tx, ty, nt);              \
      case 10: return launch_sweep_shape<T, DIM, 1, RS_HLLC, 1>(a, s, tx, ty, nt);            \
      case 11: return launch_sweep_shape<T, DIM, 1, RS_HLLC, 3>(a, s, tx, ty, nt);            \
      case 24: return launch_sweep_shape<T, DIM, 3, RS_HLL, 1>(a, s, tx, ty, nt);             \
      case 25: return launch_sweep_shape<T, DIM, 3, RS_HLL, 3>(a, s, tx, ty, nt);             \
      case 26: return launch_sweep_shape<T, DIM, 3, RS_HLLC, 1>(a, s, tx, ty, nt);            \
      case 27: return launch_sweep_shape<T, DIM, 3, RS_HLLC, 3>(a, s, tx, ty, nt);            \
      default: return cudaErrorInvalidValue;                                                  \
    }                                                                                         \
  }

}  // namespace hydro
