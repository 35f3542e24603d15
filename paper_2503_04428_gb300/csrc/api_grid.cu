// api_grid.cu -- C ABI of the grid solver (include/hydro.h): handle lifetime,
// geometry set-up, state transfer and validation, the step loop (one fused
// sweep launch per step, optionally preceded by the monopole kernels), CUDA
// graph capture of the device-dt step, the z-chunk autotuner and totals.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>
#include <algorithm>

#include "aux_kernels.cuh"
#include "common.cuh"
#include "runtime.h"

namespace hydro {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? HYDRO_ERR_OOM : HYDRO_ERR_CUDA;
}

int DeviceArena::alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  ptrs.push_back(*p);
  return HYDRO_OK;
}

void DeviceArena::release() {
  for (void* p : ptrs) cudaFree(p);
  ptrs.clear();
}

static int arg_error(const std::string& m) {
  set_error(m);
  return HYDRO_ERR_ARG;
}

static const double PI = 3.14159265358979323846;

// Extended-cell geometry of one axis (cells -2..n+1).  A ghost cell copies
// its source cell (periodic wrap, transmissive edge cell, reflective mirror):
// its width, and (through `src`) the radius / polar sine that enter its
// physical widths; ghost centres lie outside the boundary.
struct AxisExt {
  std::vector<double> lo, w;
  std::vector<int> src;  // interior source cell of each extended cell
};

static int src_cell(int g, int n, int bclo, int bchi) {
  if (g < 0) return bclo == BC_PERIODIC ? g + n : (bclo == BC_TRANSMISSIVE ? 0 : -1 - g);
  if (g >= n) return bchi == BC_PERIODIC ? g - n : (bchi == BC_TRANSMISSIVE ? n - 1 : 2 * n - 1 - g);
  return g;
}

static AxisExt axis_ext(const std::vector<double>& xf, int bclo, int bchi) {
  const int n = (int)xf.size() - 1;
  AxisExt a;
  a.lo.assign(n + 4, 0.0);
  a.w.assign(n + 4, 0.0);
  a.src.assign(n + 4, 0);
  for (int g = -2; g < n + 2; ++g) a.src[g + 2] = src_cell(g, n, bclo, bchi);
  auto width = [&](int g) {
    const int s = src_cell(g, n, bclo, bchi);
    return xf[s + 1] - xf[s];
  };
  for (int g = 0; g < n; ++g) {
    a.lo[g + 2] = xf[g];
    a.w[g + 2] = xf[g + 1] - xf[g];
  }
  a.w[1] = width(-1);
  a.lo[1] = xf[0] - a.w[1];
  a.w[0] = width(-2);
  a.lo[0] = a.lo[1] - a.w[0];
  a.w[n + 2] = width(n);
  a.lo[n + 2] = xf[n];
  a.w[n + 3] = width(n + 1);
  a.lo[n + 3] = a.lo[n + 2] + a.w[n + 2];
  return a;
}

// Upload a geometry array in the state precision; an array that exists
// already (a rebuild of the same grid) is overwritten in place.
template <typename T>
static int upload(hydro_ctx* h, const std::vector<double>& v, void** out) {
  std::vector<T> tmp(v.begin(), v.end());
  if (!*out) {
    int st = h->arena.alloc(out, tmp.size() * sizeof(T));
    if (st) return st;
  }
  HCK(cudaMemcpy(*out, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HYDRO_OK;
}

static int upload_d(hydro_ctx* h, const std::vector<double>& v, double** out) {
  if (!*out) {
    int st = h->arena.alloc((void**)out, v.size() * sizeof(double));
    if (st) return st;
  }
  HCK(cudaMemcpy(*out, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
  return HYDRO_OK;
}

// Index of each geometry array inside hydro_ctx::geo.
enum {
  G_IDXC0 = 0, G_IDXC1, G_IDXC2, G_HW0, G_HW1, G_HW2, G_IW0, G_IW1, G_IW2, G_IR, G_IS,
  G_AF, G_INVA, G_GA, G_QR, G_GR, G_GPT, G_BF, G_INVB, G_ZC, G_GT, G_QT, G_INVC, G_COUNT
};
static_assert(G_COUNT <= (int)(sizeof(((hydro_ctx*)nullptr)->geo) / sizeof(void*)),
              "hydro_ctx::geo too small");

template <typename T>
static int build_geometry(hydro_ctx* h) {
  const bool sph = h->coords == HYDRO_SPHERICAL;
  std::vector<double> xf[3];
  for (int d = 0; d < 3; ++d) {
    if (d < h->dim) xf[d] = h->faces[d];
    else if (!sph) xf[d] = {0.0, 1.0};
    else if (d == 1) xf[d] = {0.0, PI};
    else xf[d] = {0.0, 2.0 * PI};
  }
  std::vector<void*> g(h->geo, h->geo + G_COUNT);  // existing arrays are reused
  AxisExt ax[3];
  // per extended cell, the two faces whose mid-point is the radius or whose
  // sines give the mean polar sine of its physical widths
  std::vector<double> gf_lo[3], gf_hi[3];
  for (int d = 0; d < 3; ++d) {
    ax[d] = axis_ext(xf[d], d < h->dim ? h->bc[d][0] : BC_PERIODIC, d < h->dim ? h->bc[d][1] : BC_PERIODIC);
    const int me = (int)ax[d].w.size();
    gf_lo[d].assign(me, 0.0);
    gf_hi[d].assign(me, 0.0);
    for (int k = 0; k < me; ++k) {
      const int q = ax[d].src[k];
      gf_lo[d][k] = xf[d][q];
      gf_hi[d][k] = xf[d][q + 1];
    }
    if (d == h->xaxis) {
      // exchanged sides: the ghosts are the neighbour's cells, with their
      // own faces (the same operations as for an interior cell)
      const int n = (int)xf[d].size() - 1;
      if (h->xch[0]) {
        ax[d].lo[1] = h->xg[0][0];
        ax[d].w[1] = xf[d][0] - h->xg[0][0];
        ax[d].lo[0] = h->xg[0][1];
        ax[d].w[0] = h->xg[0][0] - h->xg[0][1];
        gf_lo[d][1] = h->xg[0][0], gf_hi[d][1] = xf[d][0];
        gf_lo[d][0] = h->xg[0][1], gf_hi[d][0] = h->xg[0][0];
      }
      if (h->xch[1]) {
        ax[d].lo[n + 2] = xf[d][n];
        ax[d].w[n + 2] = h->xg[1][0] - xf[d][n];
        ax[d].lo[n + 3] = h->xg[1][0];
        ax[d].w[n + 3] = h->xg[1][1] - h->xg[1][0];
        gf_lo[d][n + 2] = xf[d][n], gf_hi[d][n + 2] = h->xg[1][0];
        gf_lo[d][n + 3] = h->xg[1][0], gf_hi[d][n + 3] = h->xg[1][1];
      }
    }
    const int m = (int)ax[d].w.size();
    std::vector<double> idxc(m, 0.0), hw(m), iw(m);
    for (int k = 0; k < m; ++k) {
      hw[k] = 0.5 * ax[d].w[k];
      iw[k] = 1.0 / ax[d].w[k];
      if (k > 0) {
        const double cm = ax[d].lo[k - 1] + 0.5 * ax[d].w[k - 1];
        const double c0 = ax[d].lo[k] + 0.5 * ax[d].w[k];
        idxc[k] = 1.0 / (c0 - cm);
      }
    }
    int st;
    if ((st = upload<T>(h, idxc, &g[G_IDXC0 + d]))) return st;
    if ((st = upload<T>(h, hw, &g[G_HW0 + d]))) return st;
    if ((st = upload<T>(h, iw, &g[G_IW0 + d]))) return st;
  }
  // spherical width factors (ext)
  {
    const int m0 = (int)ax[0].w.size(), m1 = (int)ax[1].w.size();
    std::vector<double> ir(m0, 1.0), is(m1, 1.0);
    if (sph) {
      // radius and mean polar sine of the source cell (an exchanged ghost's own)
      for (int k = 0; k < m0; ++k) ir[k] = 1.0 / (0.5 * (gf_lo[0][k] + gf_hi[0][k]));
      for (int k = 0; k < m1; ++k) is[k] = 1.0 / (0.5 * (std::sin(gf_lo[1][k]) + std::sin(gf_hi[1][k])));
    }
    int st;
    if ((st = upload<T>(h, ir, &g[G_IR]))) return st;
    if ((st = upload<T>(h, is, &g[G_IS]))) return st;
  }
  // axis 0 interior factors
  const int n0 = (int)xf[0].size() - 1, n1 = (int)xf[1].size() - 1, n2 = (int)xf[2].size() - 1;
  std::vector<double> Af(n0 + 1), a(n0), inva(n0), ga(n0), qr(n0), gr(n0), gpt(n0, 0.0), rc(n0);
  for (int f = 0; f <= n0; ++f) Af[f] = sph ? xf[0][f] * xf[0][f] : 1.0;
  for (int i = 0; i < n0; ++i) {
    const double rm = xf[0][i], rp = xf[0][i + 1];
    if (sph) {
      a[i] = (rp * rp * rp - rm * rm * rm) / 3.0;
      ga[i] = 0.5 * (rp * rp - rm * rm) / a[i];
      qr[i] = (rp - rm) / ((rp + rm) * a[i]);
      gr[i] = (Af[i + 1] - Af[i]) / a[i];
    } else {
      a[i] = rp - rm;
      ga[i] = (rp - rm) / a[i];
      qr[i] = 0.0;
      gr[i] = 0.0;
    }
    inva[i] = 1.0 / a[i];
    rc[i] = 0.5 * (rm + rp);
    if (h->gravity == GRAV_POINT || h->gravity == GRAV_MONO) gpt[i] = -h->G * h->Mc / (rc[i] * rc[i]);
  }
  std::vector<double> Bf(n1 + 1), b(n1), invb(n1), zc(n1), gt(n1), qt(n1);
  for (int f = 0; f <= n1; ++f) Bf[f] = sph ? std::sin(xf[1][f]) : 1.0;
  for (int j = 0; j < n1; ++j) {
    const double tm = xf[1][j], tp = xf[1][j + 1];
    if (sph) {
      b[j] = std::cos(tm) - std::cos(tp);
      zc[j] = (tp - tm) / b[j];
      gt[j] = (Bf[j + 1] - Bf[j]) / b[j];
      const double sm = std::sin(tm), sp = std::sin(tp);
      qt[j] = (sp - sm) / ((sp + sm) * b[j]);
    } else {
      b[j] = tp - tm;
      zc[j] = (tp - tm) / b[j];
      gt[j] = 0.0;
      qt[j] = 0.0;
    }
    invb[j] = 1.0 / b[j];
  }
  std::vector<double> c(n2), invc(n2);
  for (int k = 0; k < n2; ++k) {
    c[k] = xf[2][k + 1] - xf[2][k];
    invc[k] = 1.0 / c[k];
  }
  int st;
  if ((st = upload<T>(h, Af, &g[G_AF]))) return st;
  if ((st = upload<T>(h, inva, &g[G_INVA]))) return st;
  if ((st = upload<T>(h, ga, &g[G_GA]))) return st;
  if ((st = upload<T>(h, qr, &g[G_QR]))) return st;
  if ((st = upload<T>(h, gr, &g[G_GR]))) return st;
  if ((st = upload<T>(h, gpt, &g[G_GPT]))) return st;
  if ((st = upload<T>(h, Bf, &g[G_BF]))) return st;
  if ((st = upload<T>(h, invb, &g[G_INVB]))) return st;
  if ((st = upload<T>(h, zc, &g[G_ZC]))) return st;
  if ((st = upload<T>(h, gt, &g[G_GT]))) return st;
  if ((st = upload<T>(h, qt, &g[G_QT]))) return st;
  if ((st = upload<T>(h, invc, &g[G_INVC]))) return st;
  if ((st = upload_d(h, a, &h->dvol[0]))) return st;
  if ((st = upload_d(h, b, &h->dvol[1]))) return st;
  if ((st = upload_d(h, c, &h->dvol[2]))) return st;
  {
    // the axis-2 factors split into FP32 pairs for the FP32 form's
    // compensated in-step totals
    std::vector<float> hl(2 * c.size());
    for (size_t k = 0; k < c.size(); ++k) {
      hl[2 * k] = (float)c[k];
      hl[2 * k + 1] = (float)(c[k] - (double)hl[2 * k]);
    }
    if (!h->dvz32 && (st = h->arena.alloc((void**)&h->dvz32, hl.size() * sizeof(float)))) return st;
    HCK(cudaMemcpy(h->dvz32, hl.data(), hl.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  if ((st = upload_d(h, rc, &h->rc_d))) return st;
  double bsum = 0.0, csum = 0.0;
  for (double v : b) bsum += v;
  for (double v : c) csum += v;
  h->omega = bsum * csum;
  for (int q = 0; q < G_COUNT; ++q) h->geo[q] = g[q];
  return HYDRO_OK;
}

// Moving radial grid (reading R16), for a step of size dt: the axis-0
// factors of the update with the face areas averaged over the step (a radial
// face sweeps r^2 from r to r + D, D = w dt, mean r^2 + r D + D^2/3; the
// theta and phi faces' (r+^2 - r-^2)/2 at mid-step) over the old volume
// factor a, and the volume ratio a/a' of every radial cell.  The faces
// themselves move after the step.
template <typename T>
static int moving_geometry(hydro_ctx* h, double dt) {
  const std::vector<double>& xf = h->faces[0];
  const int n0 = (int)xf.size() - 1;
  const double D = h->wgrid * dt;
  std::vector<double> Af(n0 + 1), ga(n0), qr(n0), gr(n0), vr(n0), irn(n0);
  for (int f = 0; f <= n0; ++f) Af[f] = xf[f] * xf[f] + xf[f] * D + D * D / 3.0;
  for (int i = 0; i < n0; ++i) {
    const double rm = xf[i], rp = xf[i + 1];
    const double a = (rp * rp * rp - rm * rm * rm) / 3.0;
    const double rm2 = rm + D, rp2 = rp + D;
    const double an = (rp2 * rp2 * rp2 - rm2 * rm2 * rm2) / 3.0;
    ga[i] = 0.5 * (rp - rm) * (rp + rm + D) / a;
    qr[i] = (rp - rm) / ((rp + rm + D) * a);
    gr[i] = (Af[i + 1] - Af[i]) / a;
    vr[i] = a / an;
    irn[i] = 1.0 / (0.5 * (rm2 + rp2));
  }
  int st;
  if ((st = upload<T>(h, Af, &h->geo[G_AF]))) return st;
  if ((st = upload<T>(h, ga, &h->geo[G_GA]))) return st;
  if ((st = upload<T>(h, qr, &h->geo[G_QR]))) return st;
  if ((st = upload<T>(h, gr, &h->geo[G_GR]))) return st;
  if ((st = upload<T>(h, irn, &h->irn_d))) return st;
  return upload<T>(h, vr, &h->vr_d);
}

template <typename T>
static Geom<T> geom_of(const hydro_ctx* h) {
  Geom<T> g;
  for (int d = 0; d < 3; ++d) {
    g.inv_dxc[d] = (const T*)h->geo[G_IDXC0 + d];
    g.hw[d] = (const T*)h->geo[G_HW0 + d];
    g.inv_w[d] = (const T*)h->geo[G_IW0 + d];
  }
  g.inv_r = (const T*)h->geo[G_IR];
  g.inv_s = (const T*)h->geo[G_IS];
  g.Af = (const T*)h->geo[G_AF];
  g.inva = (const T*)h->geo[G_INVA];
  g.ga = (const T*)h->geo[G_GA];
  g.qr = (const T*)h->geo[G_QR];
  g.gr = (const T*)h->geo[G_GR];
  g.gpt = (const T*)h->geo[G_GPT];
  g.Bf = (const T*)h->geo[G_BF];
  g.invb = (const T*)h->geo[G_INVB];
  g.zc = (const T*)h->geo[G_ZC];
  g.gt = (const T*)h->geo[G_GT];
  g.qt = (const T*)h->geo[G_QT];
  g.invc = (const T*)h->geo[G_INVC];
  return g;
}

template <typename T>
Gas<T> make_gas(double gm) {
  Gas<T> g;
  g.g = (T)gm;
  g.gm1 = (T)(gm - 1.0);
  g.igm1 = (T)(1.0 / (gm - 1.0));
  g.z = (T)((gm - 1.0) / (2.0 * gm));
  g.iz = (T)(2.0 * gm / (gm - 1.0));
  g.zp = (T)((gm + 1.0) / (2.0 * gm));
  g.A2 = (T)(2.0 / (gm + 1.0));
  g.Bq = (T)((gm - 1.0) / (gm + 1.0));
  g.two_gm1 = (T)(2.0 / (gm - 1.0));
  g.ig = (T)(1.0 / gm);
  g.pow_c = (T)(2.0 * gm / (gm - 1.0));
  return g;
}
template Gas<float> make_gas<float>(double);
template Gas<double> make_gas<double>(double);

template <typename T>
GasRad<T> make_gas_rad(double gm, double R, double a) {
  GasRad<T> g;
  static_cast<Gas<T>&>(g) = make_gas<T>(gm);
  g.R = (T)R;
  g.Rg = (T)(R / (gm - 1.0));
  g.a = (T)a;
  g.a3 = (T)(a / 3.0);
  g.c_g = (T)(gm / (gm - 1.0));
  g.c_1 = (T)(1.0 / (gm - 1.0));
  return g;
}
template GasRad<float> make_gas_rad<float>(double, double, double);
template GasRad<double> make_gas_rad<double>(double, double, double);

// Ni-56 decay heating constants of Eq. 8-9 (CGS).
static const double M_U = 1.66053906660e-24, MEV = 1.602176634e-6, DAY = 86400.0;

template <typename T>
static SweepArgs<T> sweep_args(hydro_ctx* h, double dt_host, double cfl, double t_end,
                               Ctrl* ctrl) {
  SweepArgs<T> a;
  a.A = (const T*)h->buf[0];
  a.Aw = (T*)h->buf[0];
  a.B = (T*)h->buf[1];
  for (int d = 0; d < 3; ++d) {
    a.n[d] = h->n[d];
    a.bc[d][0] = h->bc[d][0];
    a.bc[d][1] = h->bc[d][1];
    a.g0[d] = (T)h->g0[d];
  }
  a.ncell = h->ncell;
  a.ns = h->ns;
  a.limiter = h->limiter;
  a.spherical = h->coords == HYDRO_SPHERICAL;
  a.gravity = h->gravity;
  a.gmono = (const T*)h->gmono;
  a.heating = h->heating;
  a.ni_index = (int)h->heat_prm[0];
  a.heat_q = (T)h->heat_prm[0];
  const double qni = 1.75 * MEV, qco = 3.73 * MEV, tni = 8.8 * DAY, tco = 111.3 * DAY;
  a.ni_lambda = 1.0 / (56.0 * M_U * (tco - tni));
  a.ni_a = qni * (tco / tni - 1.0) - qco;
  a.ni_qco = qco;
  a.ni_tni = tni;
  a.ni_tco = tco;
  a.gas = make_gas<T>(h->gamma);
  a.grad = make_gas_rad<T>(h->gamma, h->R_gas, h->a_rad);
  a.eps_dual = (T)h->eps_dual;
  a.dt_host = dt_host;
  a.cfl = cfl;
  a.t_end = t_end;
  a.zchunk = h->zchunk;
  a.ctrl = ctrl;
  a.geo = geom_of<T>(h);
  a.xaxis = h->xaxis;
  a.halo[0] = (const T*)h->halo_d[0];
  a.halo[1] = (const T*)h->halo_d[1];
  a.maxis = h->maxis;
  a.wg = (T)h->wgrid;
  const bool mv_sph = h->maxis >= 0 && h->wgrid != 0.0 && h->coords == HYDRO_SPHERICAL;
  a.vr = mv_sph ? (const T*)h->vr_d : nullptr;
  a.ir_new = mv_sph && h->dim >= 2 ? (const T*)h->irn_d : nullptr;
  a.tot_part = h->step_tot ? h->step_tot_part : nullptr;
  for (int d = 0; d < 3; ++d) a.dvol[d] = h->dvol[d];
  a.dvz32 = reinterpret_cast<const float2*>(h->dvz32);
  return a;
}

template <typename T>
static int launch_step_t(hydro_ctx* h, double dt_host, double cfl, double t_end, Ctrl* ctrl) {
  if (h->gravity == GRAV_MONO) {
    dim3 gb((h->n[0] + 31) / 32, h->shell_nchunks), tb(32, 8);
    shell_partial_kernel<T><<<gb, tb, 0, h->stream>>>(ctrl, (const T*)h->buf[0], (const T*)h->buf[1],
                                                      h->ncell, h->n[0], h->n[1], h->n[2],
                                                      h->shell_kchunk, h->dvol[1], h->dvol[2],
                                                      h->shell_partial);
    HCK(cudaGetLastError());
    monopole_kernel<T><<<1, MONO_THREADS, 0, h->stream>>>(ctrl, h->shell_partial, h->shell_nchunks, h->n[0],
                                                 h->dvol[0], h->rc_d, h->G, h->Mc,
                                                 4.0 * PI / h->omega, h->inner_mass, h->shell,
                                                 (T*)h->gmono);
    HCK(cudaGetLastError());
  }
  SweepArgs<T> a = sweep_args<T>(h, dt_host, cfl, t_end, ctrl);
  cudaError_t e;
  int* tx = &h->tile_x;
  int* ty = &h->tile_y;
  int* nt = &h->threads;
  const int dual = h->eps_dual > 0.0;
  if (h->eos_rad) {
    switch (h->dim) {
      case 1: e = sweep_dispatch_rad<T, 1>(a, h->nsx, h->riemann, dual, h->stream, tx, ty, nt); break;
      case 2: e = sweep_dispatch_rad<T, 2>(a, h->nsx, h->riemann, dual, h->stream, tx, ty, nt); break;
      default: e = sweep_dispatch_rad<T, 3>(a, h->nsx, h->riemann, dual, h->stream, tx, ty, nt); break;
    }
  } else if (h->xaxis >= 0 || h->maxis >= 0) {
    switch (h->dim) {
      case 1: e = sweep_dispatch_xm<T, 1>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
      case 2: e = sweep_dispatch_xm<T, 2>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
      default: e = sweep_dispatch_xm<T, 3>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
    }
  } else if (dual) {
    switch (h->dim) {
      case 1: e = sweep_dispatch_dual<T, 1>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
      case 2: e = sweep_dispatch_dual<T, 2>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
      default: e = sweep_dispatch_dual<T, 3>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
    }
  } else {
    switch (h->dim) {
      case 1: e = sweep_dispatch<T, 1>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
      case 2: e = sweep_dispatch<T, 2>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
      default: e = sweep_dispatch<T, 3>(a, h->nsx, h->riemann, h->stream, tx, ty, nt); break;
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
  return HYDRO_OK;
}

static int launch_step(hydro_ctx* h, double dt_host, double cfl, double t_end, Ctrl* ctrl) {
  return h->precision == 64 ? launch_step_t<double>(h, dt_host, cfl, t_end, ctrl)
                            : launch_step_t<float>(h, dt_host, cfl, t_end, ctrl);
}

static int read_ctrl(hydro_ctx* h) {
  HCK(cudaMemcpyAsync(h->ctrl_host, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

static int write_ctrl(hydro_ctx* h) {
  HCK(cudaMemcpyAsync(h->ctrl, h->ctrl_host, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

// After a launch sequence: read the status; on failure clear it (the state
// is already the last good one) and report.
static int check_status(hydro_ctx* h, const char* what) {
  int st = read_ctrl(h);
  if (st) return st;
  const int code = h->ctrl_host->status;
  if (code == 0) return HYDRO_OK;
  std::ostringstream m;
  m << what << ": device status " << code << " at step " << h->ctrl_host->err_step
    << (code == HYDRO_ERR_NEGATIVE_STATE ? " (negative density or pressure)"
        : code == HYDRO_ERR_NONFINITE    ? " (non-finite state)"
        : code == HYDRO_ERR_NEWTON       ? " (Newton did not converge)"
        : code == HYDRO_ERR_VACUUM       ? " (vacuum generated)"
                                         : "");
  h->ctrl_host->status = 0;
  h->ctrl_host->done = 0;
  h->ctrl_host->err_step = -1;
  h->ctrl_host->smax_next = 0;
  if ((st = write_ctrl(h))) return st;
  set_error(m.str());
  return code;
}

// Cache of tuned launch parameters, one "key value us" line per entry, in the
// file named by HYDRO_TUNE_CACHE (no caching when unset).
int tune_cache_get(const std::string& key, int* value, double* us) {
  const char* path = std::getenv("HYDRO_TUNE_CACHE");
  if (!path) return 0;
  std::ifstream f(path);
  std::string k;
  int v;
  double u;
  while (f >> k >> v >> u)
    if (k == key) {
      *value = v;
      *us = u;
      return 1;
    }
  return 0;
}

void tune_cache_put(const std::string& key, int value, double us) {
  const char* path = std::getenv("HYDRO_TUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << value << " " << us << "\n";
}

std::string device_key() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, dev);
  std::string name = p.name;
  for (auto& ch : name)
    if (ch == ' ') ch = '_';
  return name + "_sm" + std::to_string(p.major) + std::to_string(p.minor);
}

// Autotuner of the 3D z-chunk: each candidate runs on a scratch control
// block (so the committed state is untouched; outputs land in the
// non-current buffer) and is timed with CUDA events.
static int autotune_grid(hydro_ctx* h, double cfl) {
  if (h->tuned) return HYDRO_OK;
  h->tuned = true;
  if (h->dim < 3) return HYDRO_OK;
  std::ostringstream key;
  key << "grid_d" << h->dim << "_p" << h->precision << "_r" << h->riemann << "_ns" << h->ns
      << (h->eos_rad ? "_rad" : "") << (h->eps_dual > 0.0 ? "_dual" : "") << "_n"
      << h->n[0] << "x" << h->n[1] << "x" << h->n[2] << "_" << device_key();
  int cached;
  double us;
  if (tune_cache_get(key.str(), &cached, &us)) {
    h->zchunk = cached;
    h->tuned_us = us;
    return HYDRO_OK;
  }
  int st = read_ctrl(h);
  if (st) return st;
  Ctrl* scratch = nullptr;
  HCK(cudaMalloc(&scratch, sizeof(Ctrl)));
  Ctrl base = *h->ctrl_host;
  base.status = 0;
  base.done = 0;
  base.smax_next = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // Powers of two, then (once the first launch has set the tile shape)
  // chunk lengths that make the CTA count just fill whole waves of the SMs.
  std::vector<int> cands = {4, 8, 16, 32, 64};
  double best = 1e300;
  int best_z = h->zchunk;
  double dt = base.smax_cur > 0.0 ? cfl / base.smax_cur : 1e-12;
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  bool waves_added = false;
  for (size_t ci = 0; ci < cands.size(); ++ci) {
    if (!waves_added && h->tile_x > 0 && h->tile_y > 0 && nsm > 0) {
      waves_added = true;
      const long long plane = (long long)((h->n[0] + h->tile_x - 1) / h->tile_x) *
                              ((h->n[1] + h->tile_y - 1) / h->tile_y);
      for (int w = 1; w <= 16; ++w) {
        const long long nch = (long long)w * nsm / plane;
        if (nch < 1) continue;
        const int z = (int)((h->n[2] + nch - 1) / nch);
        if (z >= 2 && z <= h->n[2] && std::find(cands.begin(), cands.end(), z) == cands.end())
          cands.push_back(z);
      }
    }
    const int zc = cands[ci];
    if (zc > h->n[2]) continue;
    h->zchunk = zc;
    const int reps = 3;
    float ms = 0.f;
    for (int r = 0; r < reps + 1; ++r) {
      cudaMemcpyAsync(scratch, &base, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream);
      if (r == 1) cudaEventRecord(e0, h->stream);
      if ((st = launch_step(h, dt, cfl, 0.0, scratch))) break;
    }
    if (st) break;
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    const double t = 1000.0 * ms / reps;
    if (t < best) {
      best = t;
      best_z = zc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(scratch);
  if (st) return st;
  h->zchunk = best_z;
  h->tuned_us = best;
  tune_cache_put(key.str(), best_z, best);
  return HYDRO_OK;
}

template <typename T>
static int validate_into(hydro_ctx* h, int slot, int* status_out, double* smax_out) {
  int* d_status = nullptr;
  unsigned long long* d_smax = nullptr;
  HCK(cudaMalloc(&d_status, sizeof(int) + sizeof(unsigned long long) + 8));
  d_smax = (unsigned long long*)(d_status + 2);
  HCK(cudaMemsetAsync(d_status, 0, sizeof(int) + sizeof(unsigned long long) + 8, h->stream));
  const int blocks = (int)std::max<long long>(1, std::min<long long>((h->ncell + 255) / 256, (long long)h->num_sms * 8));
  const Gas<T> gas = make_gas<T>(h->gamma);
  const GasRad<T> grad = make_gas_rad<T>(h->gamma, h->R_gas, h->a_rad);
  const T* U = (const T*)h->buf[slot];
  const T* w0 = (const T*)h->geo[G_IW0];
  const T* w1 = (const T*)h->geo[G_IW1];
  const T* w2 = (const T*)h->geo[G_IW2];
  const T* ir = (const T*)h->geo[G_IR];
  const T* is = (const T*)h->geo[G_IS];
  const int sph = h->coords == HYDRO_SPHERICAL;
  const long long nc = h->ncell;
  const int n0 = h->n[0], n1 = h->n[1], nv = h->nv;
  if (h->eos_rad) {
    switch (h->dim) {
      case 1: validate_kernel<T, 1><<<blocks, 256, 0, h->stream>>>(U, nc, n0, n1, nv, grad, sph, w0, w1, w2, ir, is, d_status, d_smax, h->maxis, (T)h->wgrid); break;
      case 2: validate_kernel<T, 2><<<blocks, 256, 0, h->stream>>>(U, nc, n0, n1, nv, grad, sph, w0, w1, w2, ir, is, d_status, d_smax, h->maxis, (T)h->wgrid); break;
      default: validate_kernel<T, 3><<<blocks, 256, 0, h->stream>>>(U, nc, n0, n1, nv, grad, sph, w0, w1, w2, ir, is, d_status, d_smax, h->maxis, (T)h->wgrid); break;
    }
  } else {
    switch (h->dim) {
      case 1: validate_kernel<T, 1><<<blocks, 256, 0, h->stream>>>(U, nc, n0, n1, nv, gas, sph, w0, w1, w2, ir, is, d_status, d_smax, h->maxis, (T)h->wgrid); break;
      case 2: validate_kernel<T, 2><<<blocks, 256, 0, h->stream>>>(U, nc, n0, n1, nv, gas, sph, w0, w1, w2, ir, is, d_status, d_smax, h->maxis, (T)h->wgrid); break;
      default: validate_kernel<T, 3><<<blocks, 256, 0, h->stream>>>(U, nc, n0, n1, nv, gas, sph, w0, w1, w2, ir, is, d_status, d_smax, h->maxis, (T)h->wgrid); break;
    }
  }
  HCK(cudaGetLastError());
  int hs[4];
  HCK(cudaMemcpyAsync(hs, d_status, 16, cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  cudaFree(d_status);
  *status_out = hs[0];
  unsigned long long bits;
  std::memcpy(&bits, &hs[2], 8);
  double s;
  std::memcpy(&s, &bits, 8);
  *smax_out = s;
  return HYDRO_OK;
}

}  // namespace hydro

using namespace hydro;

int hydro_common_init(hydro_ctx* h, int precision, void* stream) {
  if (precision != 32 && precision != 64) return arg_error("precision must be 32 or 64");
  h->precision = precision;
  h->esize = precision == 64 ? 8 : 4;
  HCK(cudaGetDevice(&h->device));
  HCK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    HCK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->owns_stream = true;
  }
  HCK(cudaMalloc(&h->ctrl, sizeof(Ctrl)));
  HCK(cudaMallocHost(&h->ctrl_host, sizeof(Ctrl)));
  std::memset(h->ctrl_host, 0, sizeof(Ctrl));
  h->ctrl_host->err_step = -1;
  return write_ctrl(h);
}

extern "C" {

const char* hydro_last_error(void) { return g_last_error.c_str(); }

int hydro_create(const hydro_grid* grid, int coords, const hydro_eos* eos, int riemann, int limiter,
                 int precision, void* stream, hydro_t* out) {
  if (!grid || !eos || !out) return arg_error("hydro_create: null argument");
  *out = nullptr;
  if (grid->dim < 1 || grid->dim > 3) return arg_error("hydro_create: dim must be 1, 2 or 3");
  if (coords != HYDRO_CARTESIAN && coords != HYDRO_SPHERICAL) return arg_error("hydro_create: bad coords");
  if (riemann < HYDRO_HLL || riemann > HYDRO_EXACT) return arg_error("hydro_create: bad riemann");
  if (limiter < HYDRO_FIRST_ORDER || limiter > HYDRO_VANALBADA) return arg_error("hydro_create: bad limiter");
  if (!(eos->gamma > 1.0)) return arg_error("hydro_create: gamma must exceed 1");
  if (eos->n_scalars < 0 || eos->n_scalars > HYDRO_MAX_SCALARS)
    return arg_error("hydro_create: n_scalars must be 0..3");
  if (riemann == HYDRO_EXACT && eos->n_scalars < 0) return arg_error("hydro_create: bad scalars");
  for (int d = 0; d < grid->dim; ++d) {
    if (grid->n[d] < 2) return arg_error("hydro_create: every active axis needs n >= 2");
    if (!grid->faces[d]) return arg_error("hydro_create: missing face coordinates");
    for (int s = 0; s < 2; ++s)
      if (grid->bc[d][s] < 0 || grid->bc[d][s] > 2) return arg_error("hydro_create: bad boundary kind");
    if ((grid->bc[d][0] == HYDRO_PERIODIC) != (grid->bc[d][1] == HYDRO_PERIODIC))
      return arg_error("hydro_create: periodic boundaries must be periodic on both sides");
    for (int f = 0; f < grid->n[d]; ++f)
      if (!(grid->faces[d][f + 1] > grid->faces[d][f]))
        return arg_error("hydro_create: face coordinates must increase");
  }
  if (coords == HYDRO_SPHERICAL) {
    if (!(grid->faces[0][0] >= 0.0)) return arg_error("hydro_create: spherical radius must be >= 0");
    if (grid->dim >= 2 && (grid->faces[1][0] < 0.0 || grid->faces[1][grid->n[1]] > PI))
      return arg_error("hydro_create: theta must lie in [0, pi]");
  }
  hydro_ctx* h = new hydro_ctx();
  int st = hydro_common_init(h, precision, stream);
  if (st) { hydro_destroy(h); return st; }
  h->dim = grid->dim;
  h->coords = coords;
  h->riemann = riemann;
  h->limiter = limiter;
  h->ns = eos->n_scalars;
  h->nsx = h->ns == 0 ? 0 : (h->ns == 1 ? 1 : 3);
  h->nv = 2 + h->dim + h->ns;
  h->gamma = eos->gamma;
  for (int d = 0; d < 3; ++d) {
    h->n[d] = d < h->dim ? grid->n[d] : 1;
    h->bc[d][0] = d < h->dim ? grid->bc[d][0] : 0;
    h->bc[d][1] = d < h->dim ? grid->bc[d][1] : 0;
    if (d < h->dim) h->faces[d].assign(grid->faces[d], grid->faces[d] + grid->n[d] + 1);
  }
  h->ncell = (long long)h->n[0] * h->n[1] * h->n[2];
  h->zchunk = std::min(32, h->n[2]);
  h->faces_per_step = (long long)(h->n[0] + 1) * h->n[1] * h->n[2];
  if (h->dim >= 2) h->faces_per_step += (long long)h->n[0] * (h->n[1] + 1) * h->n[2];
  if (h->dim == 3) h->faces_per_step += (long long)h->n[0] * h->n[1] * (h->n[2] + 1);
  const size_t bytes = (size_t)h->nv * h->ncell * h->esize;
  for (int b = 0; b < 2; ++b) {
    if ((st = h->arena.alloc(&h->buf[b], bytes))) { hydro_destroy(h); return st; }
    cudaMemsetAsync(h->buf[b], 0, bytes, h->stream);
  }
  st = h->precision == 64 ? build_geometry<double>(h) : build_geometry<float>(h);
  if (st) { hydro_destroy(h); return st; }
  h->tot_blocks = std::max(1, std::min(4 * h->num_sms, (int)((h->ncell + 255) / 256)));
  if ((st = h->arena.alloc((void**)&h->tot_partial, sizeof(double) * h->tot_blocks * h->nv)) ||
      (st = h->arena.alloc((void**)&h->tot_out, sizeof(double) * h->nv))) {
    hydro_destroy(h);
    return st;
  }
  *out = h;
  return HYDRO_OK;
}

int hydro_set_dual_energy(hydro_t h, double eps) {
  if (!h || h->batched) return arg_error("hydro_set_dual_energy: grid handle required");
  if (!(eps >= 0.0) || !std::isfinite(eps)) return arg_error("hydro_set_dual_energy: need eps >= 0");
  if (eps > 0.0 && (h->maxis >= 0 || h->xaxis >= 0)) {
    set_error("hydro_set_dual_energy: not built with the moving grid or the slabs");
    return HYDRO_ERR_UNSUPPORTED;
  }
  if ((eps > 0.0) != (h->eps_dual > 0.0)) h->tuned = false;  // another kernel: tune again
  h->eps_dual = eps;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return HYDRO_OK;
}

int hydro_set_eos_radiation(hydro_t h, double R_gas, double a_rad) {
  if (!h || h->batched) return arg_error("hydro_set_eos_radiation: grid handle required");
  if (!(R_gas > 0.0) || !(a_rad >= 0.0) || !std::isfinite(R_gas) || !std::isfinite(a_rad))
    return arg_error("hydro_set_eos_radiation: need R_gas > 0 and a_rad >= 0");
  if (h->riemann == HYDRO_EXACT) {
    set_error("hydro_set_eos_radiation: the exact Riemann solver assumes the ideal gas; use HLL or HLLC");
    return HYDRO_ERR_UNSUPPORTED;
  }
  if (h->maxis >= 0 || h->xaxis >= 0) {
    set_error("hydro_set_eos_radiation: the moving grid and the slabs are built for the ideal gas");
    return HYDRO_ERR_UNSUPPORTED;
  }
  h->eos_rad = 1;
  h->R_gas = R_gas;
  h->a_rad = a_rad;
  h->tuned = false;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return HYDRO_OK;
}

int hydro_set_sources(hydro_t h, int gravity, const double g0[3], double G, double Mc, int heating,
                      const double* heat_params) {
  if (!h || h->batched) return arg_error("hydro_set_sources: grid handle required");
  if (gravity < HYDRO_GRAV_NONE || gravity > HYDRO_GRAV_POINT_MONOPOLE) return arg_error("bad gravity kind");
  if (gravity >= HYDRO_GRAV_POINT && h->coords != HYDRO_SPHERICAL)
    return arg_error("point-mass and monopole gravity need spherical coordinates");
  if (heating < HYDRO_HEAT_NONE || heating > HYDRO_HEAT_NI56) return arg_error("bad heating kind");
  if (heating == HYDRO_HEAT_NI56 &&
      (!heat_params || heat_params[0] < 0 || heat_params[0] >= h->ns))
    return arg_error("Ni-56 heating needs heat_params[0] = index of an existing scalar");
  if (heating == HYDRO_HEAT_CONST && !heat_params) return arg_error("constant heating needs heat_params[0]");
  h->gravity = gravity;
  h->heating = heating;
  for (int d = 0; d < 3; ++d) h->g0[d] = g0 ? g0[d] : 0.0;
  h->G = G;
  h->Mc = Mc;
  for (int i = 0; i < 4; ++i) h->heat_prm[i] = heat_params ? heat_params[i] : 0.0;
  // point-mass acceleration per radial cell
  if (gravity == HYDRO_GRAV_POINT || gravity == HYDRO_GRAV_POINT_MONOPOLE) {
    std::vector<double> gpt(h->n[0]);
    for (int i = 0; i < h->n[0]; ++i) {
      const double rc = 0.5 * (h->faces[0][i] + h->faces[0][i + 1]);
      gpt[i] = -G * Mc / (rc * rc);
    }
    if (h->precision == 64) {
      std::vector<double> v(gpt);
      HCK(cudaMemcpy(h->geo[G_GPT], v.data(), v.size() * 8, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> v(gpt.begin(), gpt.end());
      HCK(cudaMemcpy(h->geo[G_GPT], v.data(), v.size() * 4, cudaMemcpyHostToDevice));
    }
  }
  if (gravity == HYDRO_GRAV_POINT_MONOPOLE && !h->gmono) {
    int st;
    h->shell_kchunk = std::max(1, h->n[2] / 16);
    h->shell_nchunks = (h->n[2] + h->shell_kchunk - 1) / h->shell_kchunk;
    if ((st = h->arena.alloc(&h->gmono, h->esize * h->n[0])) ||
        (st = h->arena.alloc((void**)&h->shell, sizeof(double) * h->n[0])) ||
        (st = h->arena.alloc((void**)&h->shell_partial, sizeof(double) * h->n[0] * h->shell_nchunks)))
      return st;
  }
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return HYDRO_OK;
}

int hydro_set_exchange(hydro_t h, int axis, int side, const double ghost_faces[2]) {
  if (!h || h->batched) return arg_error("hydro_set_exchange: grid handle required");
  if (axis < 0 || axis >= h->dim || side < 0 || side > 1 || !ghost_faces)
    return arg_error("hydro_set_exchange: bad axis, side or face coordinates");
  if (h->xaxis >= 0 && h->xaxis != axis)
    return arg_error("hydro_set_exchange: only the sides of one axis can be exchanged (slabs)");
  if (h->maxis >= 0) return arg_error("hydro_set_exchange: not with a moving grid");
  if (h->eos_rad || h->eps_dual > 0.0) {
    set_error("hydro_set_exchange: slabs are built for the ideal gas without the dual-energy correction");
    return HYDRO_ERR_UNSUPPORTED;
  }
  const double f0 = ghost_faces[0], f1 = ghost_faces[1];
  const std::vector<double>& xf = h->faces[axis];
  const bool ok = side == 0 ? (f1 < f0 && f0 < xf.front()) : (xf.back() < f0 && f0 < f1);
  if (!ok || !std::isfinite(f0) || !std::isfinite(f1))
    return arg_error("hydro_set_exchange: the two faces beyond the side must continue the axis monotonically");
  const long long nx = axis == 0 ? (long long)h->n[1] * h->n[2]
                     : axis == 1 ? (long long)h->n[0] * h->n[2] : (long long)h->n[0] * h->n[1];
  const size_t bytes = (size_t)h->nv * 2 * nx * h->esize;
  int st;
  if (!h->halo_d[side]) {
    if ((st = h->arena.alloc(&h->halo_d[side], bytes))) return st;
    HCK(cudaMemsetAsync(h->halo_d[side], 0, bytes, h->stream));
  }
  if (!h->pack_d && (st = h->arena.alloc(&h->pack_d, bytes))) return st;
  h->xaxis = axis;
  h->xch[side] = true;
  h->xg[side][0] = f0;
  h->xg[side][1] = f1;
  h->bc[axis][side] = BC_EXCHANGED;
  st = h->precision == 64 ? build_geometry<double>(h) : build_geometry<float>(h);
  if (st) return st;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

static long long halo_bytes(const hydro_ctx* h, int axis) {
  const long long nx = axis == 0 ? (long long)h->n[1] * h->n[2]
                     : axis == 1 ? (long long)h->n[0] * h->n[2] : (long long)h->n[0] * h->n[1];
  return (long long)h->nv * 2 * nx * (long long)h->esize;
}

int hydro_set_halo(hydro_t h, int axis, int side, const void* halo, int where) {
  if (!h || h->batched || !halo) return arg_error("hydro_set_halo: grid handle and halo required");
  if (axis != h->xaxis || side < 0 || side > 1 || !h->xch[side])
    return arg_error("hydro_set_halo: that side is not exchanged (hydro_set_exchange first)");
  HCK(cudaMemcpyAsync(h->halo_d[side], halo, (size_t)halo_bytes(h, axis),
                      where == HYDRO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  if (where != HYDRO_DEVICE) HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

int hydro_get_boundary(hydro_t h, int axis, int side, void* out, int where) {
  if (!h || h->batched || !out) return arg_error("hydro_get_boundary: grid handle and output required");
  if (axis < 0 || axis >= h->dim || side < 0 || side > 1) return arg_error("hydro_get_boundary: bad axis or side");
  int st;
  if (!h->pack_d && (st = h->arena.alloc(&h->pack_d, (size_t)halo_bytes(h, axis)))) return st;
  if (h->xaxis >= 0 && axis != h->xaxis) return arg_error("hydro_get_boundary: not the exchanged axis");
  void* dst = where == HYDRO_DEVICE ? out : h->pack_d;
  const long long n = halo_bytes(h, axis) / (long long)h->esize;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4LL * h->num_sms);
  if (h->precision == 64)
    pack_boundary_kernel<double><<<blocks, 256, 0, h->stream>>>(h->ctrl, (const double*)h->buf[0],
                                                                (const double*)h->buf[1], h->ncell, h->n[0],
                                                                h->n[1], h->n[2], h->nv, axis, side,
                                                                (double*)dst);
  else
    pack_boundary_kernel<float><<<blocks, 256, 0, h->stream>>>(h->ctrl, (const float*)h->buf[0],
                                                               (const float*)h->buf[1], h->ncell, h->n[0],
                                                               h->n[1], h->n[2], h->nv, axis, side, (float*)dst);
  HCK(cudaGetLastError());
  if (where != HYDRO_DEVICE)
    HCK(cudaMemcpyAsync(out, h->pack_d, (size_t)halo_bytes(h, axis), cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

int hydro_shell_masses(hydro_t h, double* m_out) {
  if (!h || h->batched || !m_out) return arg_error("hydro_shell_masses: grid handle and output required");
  if (h->gravity != HYDRO_GRAV_POINT_MONOPOLE)
    return arg_error("hydro_shell_masses: the handle has no monopole gravity");
  dim3 gb((h->n[0] + 31) / 32, h->shell_nchunks), tb(32, 8);
  if (h->precision == 64)
    shell_partial_kernel<double><<<gb, tb, 0, h->stream>>>(h->ctrl, (const double*)h->buf[0],
                                                           (const double*)h->buf[1], h->ncell, h->n[0], h->n[1],
                                                           h->n[2], h->shell_kchunk, h->dvol[1], h->dvol[2],
                                                           h->shell_partial);
  else
    shell_partial_kernel<float><<<gb, tb, 0, h->stream>>>(h->ctrl, (const float*)h->buf[0],
                                                          (const float*)h->buf[1], h->ncell, h->n[0], h->n[1],
                                                          h->n[2], h->shell_kchunk, h->dvol[1], h->dvol[2],
                                                          h->shell_partial);
  HCK(cudaGetLastError());
  shell_mass_kernel<<<(h->n[0] + 127) / 128, 128, 0, h->stream>>>(h->shell_partial, h->shell_nchunks, h->n[0],
                                                                  h->dvol[0], h->shell);
  HCK(cudaGetLastError());
  HCK(cudaMemcpyAsync(m_out, h->shell, sizeof(double) * h->n[0], cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

int hydro_set_inner_mass(hydro_t h, double mass) {
  if (!h || h->batched) return arg_error("hydro_set_inner_mass: grid handle required");
  if (!std::isfinite(mass) || mass < 0.0) return arg_error("hydro_set_inner_mass: need a finite mass >= 0");
  h->inner_mass = mass;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return HYDRO_OK;
}

int hydro_set_state(hydro_t h, const void* U, int where) {
  if (!h || !U) return arg_error("hydro_set_state: null argument");
  if (h->batched) return hydro_batch_set_state_impl(h, U, where);
  int st = read_ctrl(h);
  if (st) return st;
  const int slot = h->ctrl_host->cur ^ 1;
  const size_t bytes = (size_t)h->nv * h->ncell * h->esize;
  HCK(cudaMemcpyAsync(h->buf[slot], U, bytes, where == HYDRO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      h->stream));
  int status;
  double smax;
  st = h->precision == 64 ? validate_into<double>(h, slot, &status, &smax)
                          : validate_into<float>(h, slot, &status, &smax);
  if (st) return st;
  if (status) {
    set_error(status == HYDRO_ERR_NONFINITE ? "hydro_set_state: non-finite value in the state"
                                            : "hydro_set_state: density or pressure not positive");
    return status;
  }
  h->ctrl_host->cur = slot;
  h->ctrl_host->smax_cur = smax;
  h->ctrl_host->smax_next = 0;
  h->ctrl_host->status = 0;
  h->ctrl_host->done = 0;
  h->ctrl_host->err_step = -1;
  h->step_tot_ok = false;  // the step totals describe an earlier state
  return write_ctrl(h);
}

int hydro_get_state(hydro_t h, void* U_out, int where) {
  if (!h || !U_out) return arg_error("hydro_get_state: null argument");
  if (h->batched) return hydro_batch_get_state_impl(h, U_out, where);
  int st = read_ctrl(h);
  if (st) return st;
  const size_t bytes = (size_t)h->nv * h->ncell * h->esize;
  HCK(cudaMemcpyAsync(U_out, h->buf[h->ctrl_host->cur], bytes,
                      where == HYDRO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

int hydro_set_time(hydro_t h, double t) {
  if (!h) return arg_error("hydro_set_time: null handle");
  int st = read_ctrl(h);
  if (st) return st;
  h->ctrl_host->t = t;
  return write_ctrl(h);
}

int hydro_cfl_dt(hydro_t h, double cfl, double* dt_out) {
  if (!h || !dt_out || !(cfl > 0)) return arg_error("hydro_cfl_dt: bad argument");
  if (h->batched) return arg_error("hydro_cfl_dt: batched handles use per-tube time steps");
  int st = read_ctrl(h);
  if (st) return st;
  if (!(h->ctrl_host->smax_cur > 0.0)) return arg_error("hydro_cfl_dt: no signal speed (state not set?)");
  *dt_out = cfl / h->ctrl_host->smax_cur;
  return HYDRO_OK;
}

// After a step on a moving grid: the faces of the moving axis shift by w dt
// and the geometry is rebuilt for them.
static int move_faces(hydro_ctx* h, double dt) {
  for (double& f : h->faces[h->maxis]) f += h->wgrid * dt;
  return h->precision == 64 ? build_geometry<double>(h) : build_geometry<float>(h);
}

int hydro_step(hydro_t h, double dt) {
  if (!h || h->batched) return arg_error("hydro_step: grid handle required");
  if (!(dt > 0.0) || !std::isfinite(dt)) return arg_error("hydro_step: dt must be positive and finite");
  int st;
  const bool moving = h->maxis >= 0 && h->wgrid != 0.0;
  if (moving && h->coords == HYDRO_SPHERICAL) {
    st = h->precision == 64 ? moving_geometry<double>(h, dt) : moving_geometry<float>(h, dt);
    if (st) return st;
  }
  st = launch_step(h, dt, 0.0, 0.0, h->ctrl);
  if (st) return st;
  st = check_status(h, "hydro_step");
  h->step_tot_ok = h->step_tot && st == HYDRO_OK;
  if (moving) {
    // a failed step leaves the state and the faces as they were
    const int mv = st == HYDRO_OK ? move_faces(h, dt)
                   : (h->precision == 64 ? build_geometry<double>(h) : build_geometry<float>(h));
    if (mv) return mv;
  }
  return st;
}

int hydro_set_moving_grid(hydro_t h, int axis, double w) {
  if (!h || h->batched) return arg_error("hydro_set_moving_grid: grid handle required");
  if (axis < 0 || axis >= h->dim || !std::isfinite(w)) return arg_error("hydro_set_moving_grid: bad axis or velocity");
  if (h->coords == HYDRO_SPHERICAL && axis != 0)
    return arg_error("hydro_set_moving_grid: a spherical grid moves along r only");
  for (int s = 0; s < 2; ++s) {
    const int b = h->bc[axis][s];
    if (b == BC_REFLECTIVE || b == BC_EXCHANGED || (b == BC_PERIODIC && h->coords == HYDRO_SPHERICAL))
      return arg_error("hydro_set_moving_grid: the moving axis needs transmissive (or, Cartesian, periodic) ends");
  }
  if (h->eos_rad || h->eps_dual > 0.0) {
    set_error("hydro_set_moving_grid: built for the ideal gas without the dual-energy correction");
    return HYDRO_ERR_UNSUPPORTED;
  }
  if (h->step_tot) {
    set_error("hydro_set_moving_grid: turn the step totals off first (the cell volumes change in the step)");
    return HYDRO_ERR_UNSUPPORTED;
  }
  h->maxis = axis;
  h->wgrid = w;

  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return HYDRO_OK;
}

int hydro_get_faces(hydro_t h, int axis, double* out) {
  if (!h || h->batched || !out || axis < 0 || axis >= h->dim) return arg_error("hydro_get_faces: bad argument");
  std::copy(h->faces[axis].begin(), h->faces[axis].end(), out);
  return HYDRO_OK;
}

int hydro_run(hydro_t h, int nsteps, double cfl, double t_end, double* t_out) {
  if (!h || h->batched) return arg_error("hydro_run: grid handle required");
  if (nsteps < 0 || !(cfl > 0.0)) return arg_error("hydro_run: bad nsteps or cfl");
  if (h->xaxis >= 0) {
    set_error("hydro_run: a grid with exchanged sides needs its halos (and the global dt) before every step: "
              "use hydro_step");
    return HYDRO_ERR_UNSUPPORTED;
  }
  if (h->maxis >= 0 && h->wgrid != 0.0) {
    // a moving grid's geometry follows each step's dt: steps driven from the host
    int st;
    for (int s = 0; s < nsteps; ++s) {
      if ((st = read_ctrl(h))) return st;
      const double t0 = h->ctrl_host->t;
      if (t_end > 0.0 && t0 >= t_end) break;
      double dt = cfl / h->ctrl_host->smax_cur;
      if (t_end > 0.0 && t0 + dt > t_end) dt = t_end - t0;
      if ((st = hydro_step(h, dt))) return st;
    }
    if ((st = read_ctrl(h))) return st;
    if (t_out) *t_out = h->ctrl_host->t;
    return HYDRO_OK;
  }
  int st;
  if ((st = autotune_grid(h, cfl))) return st;
  if (!h->graph || h->graph_cfl != cfl || h->graph_tend != t_end) {
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    // make sure kernel attributes are set outside of capture
    cudaGraph_t g;
    HCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed));
    st = launch_step(h, 0.0, cfl, t_end, h->ctrl);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    h->graph_cfl = cfl;
    h->graph_tend = t_end;
  }
  const long long step0 = h->ctrl_host->step;
  for (int s = 0; s < nsteps; ++s) HCK(cudaGraphLaunch(h->graph, h->stream));
  st = check_status(h, "hydro_run");
  if (st != HYDRO_OK) h->step_tot_ok = false;
  else if (h->ctrl_host->step > step0) h->step_tot_ok = h->step_tot;
  if (t_out) *t_out = h->ctrl_host->t;
  return st;
}

int hydro_set_step_totals(hydro_t h, int on) {
  if (!h || h->batched) return arg_error("hydro_set_step_totals: grid handle required");
  if (on && h->maxis >= 0) {
    set_error("hydro_set_step_totals: not on a moving grid (its cell volumes change in the step)");
    return HYDRO_ERR_UNSUPPORTED;
  }
  if (on && !h->step_tot_part) {
    // partials for the most CTAs any launch shape gives (tiles of at least
    // 16 x 8 cells, z chunks of at least one plane)
    const long long ctas = (long long)((h->n[0] + 15) / 16) * ((h->n[1] + 7) / 8) * h->n[2];
    int st = h->arena.alloc((void**)&h->step_tot_part, sizeof(double) * h->nv * ctas);
    if (st) return st;
  }
  h->step_tot = on != 0;
  h->step_tot_ok = false;
  if (h->graph) {  // the captured step's arguments change
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return HYDRO_OK;
}

int hydro_step_totals(hydro_t h, double* out_nv) {
  if (!h || h->batched || !out_nv) return arg_error("hydro_step_totals: bad argument");
  if (!h->step_tot || !h->step_tot_ok)
    return arg_error("hydro_step_totals: no step with totals since they were turned on or the state was set");
  const long long ctas = (long long)((h->n[0] + h->tile_x - 1) / h->tile_x) *
                         (h->dim >= 2 ? (h->n[1] + h->tile_y - 1) / h->tile_y : 1) *
                         (h->dim == 3 ? (h->n[2] + h->zchunk - 1) / h->zchunk : 1);
  totals_final_kernel<<<1, 32, 0, h->stream>>>(h->step_tot_part, (int)ctas, h->nv, h->tot_out);
  HCK(cudaGetLastError());
  HCK(cudaMemcpyAsync(out_nv, h->tot_out, sizeof(double) * h->nv, cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

int hydro_totals(hydro_t h, double* out_nv) {
  if (!h || !out_nv) return arg_error("hydro_totals: null argument");
  if (h->batched) return arg_error("hydro_totals: grid handle required");
  int st = read_ctrl(h);
  if (st) return st;
  dim3 grid(h->tot_blocks, h->nv);
  if (h->precision == 64)
    totals_partial_kernel<double><<<grid, 256, 0, h->stream>>>((const double*)h->buf[h->ctrl_host->cur], h->ncell,
                                                               h->n[0], h->n[1], h->dvol[0], h->dvol[1],
                                                               h->dvol[2], h->tot_partial);
  else
    totals_partial_kernel<float><<<grid, 256, 0, h->stream>>>((const float*)h->buf[h->ctrl_host->cur], h->ncell,
                                                              h->n[0], h->n[1], h->dvol[0], h->dvol[1],
                                                              h->dvol[2], h->tot_partial);
  HCK(cudaGetLastError());
  totals_final_kernel<<<1, 32, 0, h->stream>>>(h->tot_partial, h->tot_blocks, h->nv, h->tot_out);
  HCK(cudaGetLastError());
  HCK(cudaMemcpyAsync(out_nv, h->tot_out, sizeof(double) * h->nv, cudaMemcpyDeviceToHost, h->stream));
  HCK(cudaStreamSynchronize(h->stream));
  return HYDRO_OK;
}

int hydro_stats(hydro_t h, hydro_stats_t* out) {
  if (!h || !out) return arg_error("hydro_stats: null argument");
  if (h->batched) return hydro_batch_stats_impl(h, out);
  int st = read_ctrl(h);
  if (st) return st;
  std::memset(out, 0, sizeof(*out));
  out->steps = h->ctrl_host->step;
  out->faces = h->ctrl_host->step * h->faces_per_step;
  out->newton_iters = (long long)h->ctrl_host->iters;
  out->fallbacks = (long long)h->ctrl_host->fallbacks;
  out->mlp_faces = (long long)h->ctrl_host->mlp;
  out->t = h->ctrl_host->t;
  out->last_dt = h->ctrl_host->last_dt;
  out->tile_x = h->tile_x;
  out->tile_y = h->tile_y;
  out->zchunk = h->zchunk;
  out->threads = h->threads;
  out->tuned_us_per_step = h->tuned_us;
  return HYDRO_OK;
}

void hydro_destroy(hydro_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->bs) hydro_batch_free_impl(h);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->arena.release();
  if (h->ctrl) cudaFree(h->ctrl);
  if (h->ctrl_host) cudaFreeHost(h->ctrl_host);
  if (h->owns_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
