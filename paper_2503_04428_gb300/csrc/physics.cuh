// physics.cuh -- per-cell and per-face device arithmetic of the Godunov update.
//
// Ideal-gas EoS (HERACLES++ Sect. 2.3 Eq. 5), physical fluxes of the Euler
// system (Sect. 2.1 Eq. 1), slope limiters (Sect. 3.2 Eq. 17), HLL/HLLC
// Riemann solvers (Sect. 3.2, Toro 2009 ch. 10), the exact Riemann solver
// (App. C.1, Toro 2009 ch. 4) and the MLP star-pressure guess.
//
// Vectors are register arrays of compile-time length NV = 2 + D + NSX:
// (rho, u_1..u_D, P, f_1..f_NSX) for primitives and (rho, m_1..m_D, E,
// rho f_1..rho f_NSX) for conserved variables.  Scalars beyond the run's
// actual count are carried as zeros and never stored.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace hydro {

enum { LIM_FIRST = 0, LIM_MINMOD = 1, LIM_VANLEER = 2, LIM_VANALBADA = 3 };
enum { RS_HLL = 0, RS_HLLC = 1, RS_EXACT = 2 };
enum { ST_OK = 0, ST_NEG = -3, ST_NONFINITE = -4, ST_NEWTON = -5, ST_VACUUM = -8 };

// Gas constants precomputed on the host (double) and passed by value.
// Gas<T> is the ideal gas of Eq. 5.
template <typename T>
struct Gas {
  static constexpr bool RAD = false;
  T g;        // gamma
  T gm1;      // gamma - 1
  T igm1;     // 1/(gamma - 1)
  T z;        // (gamma - 1)/(2 gamma)
  T iz;       // 1/z
  T zp;       // (gamma + 1)/(2 gamma)
  T A2;       // 2/(gamma + 1)
  T Bq;       // (gamma - 1)/(gamma + 1)
  T two_gm1;  // 2/(gamma - 1)
  T ig;       // 1/gamma
  T pow_c;    // 2 gamma/(gamma - 1)
};

// Square roots.  The FP32 bulk takes x rsqrt(x) (about 3 ulp; x > 0 on every
// path that uses it): the correctly rounded sqrtf sequence cost 2-3 % of the
// FP32 step's instructions.
template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return x * rsqrtf(x); }
// Powers (x > 0) as exp2(y log2 x): a few ulp (FP64: relative 1e-15 at the
// exponents of the exact solver), against the accurate pow/powf, whose
// extended-precision logarithm is several times longer and dominated the
// instruction stream of the exact solver.
template <typename T> __device__ __forceinline__ T dpow(T x, T y);
template <> __device__ __forceinline__ double dpow<double>(double x, double y) { return exp2(y * log2(x)); }
template <> __device__ __forceinline__ float dpow<float>(float x, float y) { return exp2f(y * log2f(x)); }

// Quotient of the state conversions, wave speeds and the exact solver
// (pressure functions, guess, Newton step, sampling): correctly rounded in
// FP64, the fast 2-ulp division in FP32 (the FP32 bulk's rounding error is
// ~1e-7 per operation either way, and Newton corrects its own iterates; the
// IEEE sequence is several times longer).
template <typename T> __device__ __forceinline__ T qdiv(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

template <typename T> __device__ __forceinline__ T temp_tol();
template <> __device__ __forceinline__ double temp_tol<double>() { return 1e-13; }
template <> __device__ __forceinline__ float temp_tol<float>() { return 1e-6f; }

// Ideal gas in equilibrium with radiation, Eq. 6-7: e = rho R T/(gamma-1) +
// a T^4, P = rho R T + a T^4/3 with R = k_b/(mu m_u), and the sound speed of
// Eq. 7.  The temperature comes from a Newton iteration (Sect. 2.3).
template <typename T>
struct GasRad : Gas<T> {
  static constexpr bool RAD = true;
  T R;    // specific gas constant k_b/(mu m_u)
  T Rg;   // R/(gamma - 1)
  T a;    // radiation constant
  T a3;   // a/3
  T c_g;  // gamma/(gamma - 1), numerator constant of Eq. 7
  T c_1;  // 1/(gamma - 1), denominator constant of Eq. 7

  // The temperature where c1 t + c4 t^4 = y (c1 > 0, c4 >= 0).  The left side
  // is increasing and convex in t > 0, so Newton from the upper bound
  // min(y/c1, (y/c4)^(1/4)) descends monotonically to the root; from any
  // other positive start t0 (a nearby temperature the caller knows) the first
  // step lands above the root and the descent follows.  It stops when the
  // relative step is below temp_tol and takes one more step; in FP32 the step
  // below temp_tol (1e-6) is the last (quadratic convergence leaves that
  // iterate ~1e-12 from the root, below FP32 resolution).  y <= 0 gives
  // y/c1 <= 0, which the positivity checks reject.
  // (its, if given, accumulates the Newton iterations taken.)
  __device__ __forceinline__ T temperature(T c1, T c4, T y, T t0 = T(0), int* its = nullptr) const {
    T t = qdiv(y, c1);
    if (!(y > T(0))) return t;
    if (t0 > T(0)) t = t0;
    else if (c4 > T(0)) t = fmin(t, dsqrt(dsqrt(qdiv(y, c4))));
    bool conv = false;
    int it = 0;
    for (; it < 60; ++it) {
      const T t3 = t * t * t;
      const T tn = t - qdiv(c1 * t + c4 * t3 * t - y, c1 + T(4) * c4 * t3);
      const T ch = qdiv(fabs(tn - t), tn);
      t = tn;
      if (conv) break;
      if (ch < temp_tol<T>()) {
        if constexpr (sizeof(T) == 4) break;  // FP32: this step was the last
        conv = true;
      }
    }
    if (its) *its += it < 60 ? it + 1 : 60;
    return t;
  }
  // Eq. 7 from the gas and radiation pressures
  __device__ __forceinline__ T sound2(T rho, T pg, T pr) const {
    const T al = qdiv(pr, pg);
    return qdiv(c_g + T(20) * al + T(16) * al * al, c_1 + T(12) * al) * qdiv(pg, rho);
  }
  // P and c^2 from (rho, e)
  __device__ __forceinline__ void from_e(T rho, T e, T& p, T& c2) const {
    const T t = temperature(rho * Rg, a, e);
    const T pg = rho * R * t, pr = a3 * t * t * t * t;
    p = pg + pr;
    c2 = sound2(rho, pg, pr);
  }
  // P, c^2 and the temperature from (rho, e) (t0: a start, see temperature)
  __device__ __forceinline__ void from_e_t(T rho, T e, T& p, T& c2, T& t, T t0 = T(0), int* its = nullptr) const {
    t = temperature(rho * Rg, a, e, t0, its);
    const T pg = rho * R * t, pr = a3 * t * t * t * t;
    p = pg + pr;
    c2 = sound2(rho, pg, pr);
  }
  // the temperature of (rho, P) (t0: a start, see temperature)
  __device__ __forceinline__ T temp_p(T rho, T p, T t0 = T(0), int* its = nullptr) const {
    return temperature(rho * R, a3, p, t0, its);
  }
  // e and c^2 of a state whose temperature is known
  __device__ __forceinline__ void from_t(T rho, T t, T& e, T& c2) const {
    const T pg = rho * R * t, pr = a3 * t * t * t * t;
    e = pg * c_1 + T(3) * pr;
    c2 = sound2(rho, pg, pr);
  }
  // e and c^2 from (rho, P)
  __device__ __forceinline__ void from_p(T rho, T p, T& e, T& c2) const {
    const T t = temperature(rho * R, a3, p);
    const T pg = rho * R * t, pr = a3 * t * t * t * t;
    e = pg * c_1 + T(3) * pr;
    c2 = sound2(rho, pg, pr);
  }
};

template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <typename T> __device__ __forceinline__ T dlog(T x);
template <> __device__ __forceinline__ double dlog<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float dlog<float>(float x) { return logf(x); }

// ---------------------------------------------------------------------------
// EoS conversions (Eq. 5 with E = e + rho|u|^2/2)
// ---------------------------------------------------------------------------
template <typename T, int D, int NSX, typename G>
__device__ __forceinline__ void to_prim(const T* U, T* W, const G& gas) {
  const T rho = U[0];
  const T ir = qdiv(T(1), rho);
  T ke = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    W[1 + d] = U[1 + d] * ir;
    ke += U[1 + d] * W[1 + d];
  }
  W[0] = rho;
  if constexpr (G::RAD) {
    T c2;
    gas.from_e(rho, U[1 + D] - T(0.5) * ke, W[1 + D], c2);
  } else {
    W[1 + D] = gas.gm1 * (U[1 + D] - T(0.5) * ke);
  }
#pragma unroll
  for (int s = 0; s < NSX; ++s) W[2 + D + s] = U[2 + D + s] * ir;
}

// to_prim for the gas + radiation EoS that also returns c^2 (Eq. 7) and the
// temperature of the same solve (t0: a Newton start, see GasRad::temperature).
template <typename T, int D, int NSX, typename G>
__device__ __forceinline__ void to_prim_ct(const T* U, T* W, T& c2, T& t, const G& gas, T t0 = T(0),
                                           int* its = nullptr) {
  const T rho = U[0];
  const T ir = qdiv(T(1), rho);
  T ke = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    W[1 + d] = U[1 + d] * ir;
    ke += U[1 + d] * W[1 + d];
  }
  W[0] = rho;
  gas.from_e_t(rho, U[1 + D] - T(0.5) * ke, W[1 + D], c2, t, t0, its);
#pragma unroll
  for (int s = 0; s < NSX; ++s) W[2 + D + s] = U[2 + D + s] * ir;
}

template <typename T, int D, int NSX, typename G>
__device__ __forceinline__ void to_prim_c2(const T* U, T* W, T& c2, const G& gas) {
  const T rho = U[0];
  const T ir = qdiv(T(1), rho);
  T ke = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    W[1 + d] = U[1 + d] * ir;
    ke += U[1 + d] * W[1 + d];
  }
  W[0] = rho;
  gas.from_e(rho, U[1 + D] - T(0.5) * ke, W[1 + D], c2);
#pragma unroll
  for (int s = 0; s < NSX; ++s) W[2 + D + s] = U[2 + D + s] * ir;
}

// Internal energy per volume of the primitive state (rho, p) (Eq. 5 or 6).
template <typename T, typename G>
__device__ __forceinline__ T eint_of(const G& gas, T rho, T p) {
  if constexpr (G::RAD) {
    T e, c2;
    gas.from_p(rho, p, e, c2);
    return e;
  } else {
    return p * gas.igm1;
  }
}

// Square of the sound speed at (rho, p): gamma p/rho (Eq. 5) or Eq. 7.
template <typename T, typename G>
__device__ __forceinline__ T sound2_of(const G& gas, T rho, T p) {
  if constexpr (G::RAD) {
    T e, c2;
    gas.from_p(rho, p, e, c2);
    return c2;
  } else {
    return qdiv(gas.g * p, rho);
  }
}

template <typename T, int D, int NSX, typename G>
__device__ __forceinline__ void to_cons(const T* W, T* U, const G& gas) {
  const T rho = W[0];
  T v2 = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    U[1 + d] = rho * W[1 + d];
    v2 += W[1 + d] * W[1 + d];
  }
  U[0] = rho;
  if constexpr (G::RAD) U[1 + D] = eint_of(gas, rho, W[1 + D]) + T(0.5) * rho * v2;
  else U[1 + D] = W[1 + D] * gas.igm1 + T(0.5) * rho * v2;
#pragma unroll
  for (int s = 0; s < NSX; ++s) U[2 + D + s] = rho * W[2 + D + s];
}

// Physical flux through a face normal to axis DIR, from primitives.
template <typename T, int D, int NSX, int DIR, typename G>
__device__ __forceinline__ void phys_flux(const T* W, T* F, const G& gas) {
  const T rho = W[0], un = W[1 + DIR], p = W[1 + D];
  T v2 = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) v2 += W[1 + d] * W[1 + d];
  T E;
  if constexpr (G::RAD) E = eint_of(gas, rho, p) + T(0.5) * rho * v2;
  else E = p * gas.igm1 + T(0.5) * rho * v2;
  const T mn = rho * un;
  F[0] = mn;
#pragma unroll
  for (int d = 0; d < D; ++d) F[1 + d] = mn * W[1 + d];
  F[1 + DIR] += p;
  F[1 + D] = un * (E + p);
#pragma unroll
  for (int s = 0; s < NSX; ++s) F[2 + D + s] = mn * W[2 + D + s];
}

// ---------------------------------------------------------------------------
// Slope limiters of Eq. 17 (minmod, van Leer, van Albada; 0 = first order),
// applied to the one-sided differences dm, dp; zero when they differ in sign.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T limit(int kind, T dm, T dp) {
  const T pr = dm * dp;
  if (kind == LIM_FIRST || !(pr > T(0))) return T(0);
  if (kind == LIM_MINMOD) return dm > T(0) ? fmin(dm, dp) : fmax(dm, dp);
  if (kind == LIM_VANLEER) return qdiv(T(2) * pr, dm + dp);
  return qdiv(pr * (dm + dp), dm * dm + dp * dp);
}

// ---------------------------------------------------------------------------
// HLL with Davis wave-speed bounds.
// ---------------------------------------------------------------------------
// Flux through a face normal to DIR and the conserved state of a primitive
// state whose internal energy per volume e is already known.
template <typename T, int D, int NSX, int DIR>
__device__ __forceinline__ void flux_cons_e(const T* W, T e, T* F, T* U) {
  const T rho = W[0], un = W[1 + DIR], p = W[1 + D];
  T v2 = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) v2 += W[1 + d] * W[1 + d];
  const T E = e + T(0.5) * rho * v2;
  const T mn = rho * un;
  F[0] = mn;
  U[0] = rho;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    F[1 + d] = mn * W[1 + d];
    U[1 + d] = rho * W[1 + d];
  }
  F[1 + DIR] += p;
  F[1 + D] = un * (E + p);
  U[1 + D] = E;
#pragma unroll
  for (int s = 0; s < NSX; ++s) {
    F[2 + D + s] = mn * W[2 + D + s];
    U[2 + D + s] = rho * W[2 + D + s];
  }
}

// HLL for the gas + radiation EoS: one temperature solve per side gives e
// and the Eq. 7 sound speed.
// (TL, TR > 0: the face states' temperatures, known to the caller; no solve)
template <typename T, int D, int NSX, int DIR, typename G>
__device__ __forceinline__ void riemann_hll_rad(const T* WL, const T* WR, T* F, const G& gas, T TL = T(0),
                                                T TR = T(0)) {
  constexpr int NV = 2 + D + NSX;
  T eL, c2L, eR, c2R;
  if (TL > T(0)) gas.from_t(WL[0], TL, eL, c2L);
  else gas.from_p(WL[0], WL[1 + D], eL, c2L);
  if (TR > T(0)) gas.from_t(WR[0], TR, eR, c2R);
  else gas.from_p(WR[0], WR[1 + D], eR, c2R);
  const T cL = dsqrt(c2L), cR = dsqrt(c2R);
  const T SL = fmin(WL[1 + DIR] - cL, WR[1 + DIR] - cR);
  const T SR = fmax(WL[1 + DIR] + cL, WR[1 + DIR] + cR);
  T FL[NV], FR[NV], UL[NV], UR[NV];
  flux_cons_e<T, D, NSX, DIR>(WL, eL, FL, UL);
  flux_cons_e<T, D, NSX, DIR>(WR, eR, FR, UR);
  if (SL >= T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = FL[v];
    return;
  }
  if (SR <= T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = FR[v];
    return;
  }
  const T inv = qdiv(T(1), SR - SL);
  const T sLR = SL * SR;
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = (SR * FL[v] - SL * FR[v] + sLR * (UR[v] - UL[v])) * inv;
}

// HLLC for the gas + radiation EoS (the star states need only E, p, rho, u).
template <typename T, int D, int NSX, int DIR, typename G>
__device__ __forceinline__ void riemann_hllc_rad(const T* WL, const T* WR, T* F, const G& gas, T TL = T(0),
                                                 T TR = T(0)) {
  constexpr int NV = 2 + D + NSX;
  const T rL = WL[0], rR = WR[0], uL = WL[1 + DIR], uR = WR[1 + DIR];
  const T pL = WL[1 + D], pR = WR[1 + D];
  T eL, c2L, eR, c2R;
  if (TL > T(0)) gas.from_t(rL, TL, eL, c2L);
  else gas.from_p(rL, pL, eL, c2L);
  if (TR > T(0)) gas.from_t(rR, TR, eR, c2R);
  else gas.from_p(rR, pR, eR, c2R);
  const T cL = dsqrt(c2L), cR = dsqrt(c2R);
  const T SL = fmin(uL - cL, uR - cR);
  const T SR = fmax(uL + cL, uR + cR);
  T Fk[NV], Uk[NV];
  if (SL >= T(0)) {
    flux_cons_e<T, D, NSX, DIR>(WL, eL, F, Uk);
    return;
  }
  if (SR <= T(0)) {
    flux_cons_e<T, D, NSX, DIR>(WR, eR, F, Uk);
    return;
  }
  const T aL = rL * (SL - uL), aR = rR * (SR - uR);
  const T Ss = qdiv(pR - pL + uL * aL - uR * aR, aL - aR);
  const bool left = Ss >= T(0);
  T W[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) W[v] = left ? WL[v] : WR[v];
  const T S = left ? SL : SR;
  const T a = left ? aL : aR;
  const T rho = W[0], un = W[1 + DIR], p = W[1 + D];
  flux_cons_e<T, D, NSX, DIR>(W, left ? eL : eR, Fk, Uk);
  const T fac = qdiv(a, S - Ss);
  T Us[NV];
  Us[0] = fac;
#pragma unroll
  for (int d = 0; d < D; ++d) Us[1 + d] = fac * W[1 + d];
  Us[1 + DIR] = fac * Ss;
  Us[1 + D] = fac * (qdiv(Uk[1 + D], rho) + (Ss - un) * (Ss + qdiv(p, a)));
#pragma unroll
  for (int s = 0; s < NSX; ++s) Us[2 + D + s] = fac * W[2 + D + s];
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = Fk[v] + S * (Us[v] - Uk[v]);
}

template <typename T, int D, int NSX, int DIR, typename G>
__device__ __forceinline__ void riemann_hll(const T* WL, const T* WR, T* F, const G& gas) {
  if constexpr (G::RAD) {
    riemann_hll_rad<T, D, NSX, DIR>(WL, WR, F, gas);
    return;
  }
  constexpr int NV = 2 + D + NSX;
  const T cL = dsqrt(qdiv(gas.g * WL[1 + D], WL[0]));
  const T cR = dsqrt(qdiv(gas.g * WR[1 + D], WR[0]));
  const T SL = fmin(WL[1 + DIR] - cL, WR[1 + DIR] - cR);
  const T SR = fmax(WL[1 + DIR] + cL, WR[1 + DIR] + cR);
  T FL[NV], FR[NV];
  if (SL >= T(0)) {
    phys_flux<T, D, NSX, DIR>(WL, F, gas);
    return;
  }
  if (SR <= T(0)) {
    phys_flux<T, D, NSX, DIR>(WR, F, gas);
    return;
  }
  T UL[NV], UR[NV];
  phys_flux<T, D, NSX, DIR>(WL, FL, gas);
  phys_flux<T, D, NSX, DIR>(WR, FR, gas);
  to_cons<T, D, NSX>(WL, UL, gas);
  to_cons<T, D, NSX>(WR, UR, gas);
  const T inv = qdiv(T(1), SR - SL);
  const T sLR = SL * SR;
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = (SR * FL[v] - SL * FR[v] + sLR * (UR[v] - UL[v])) * inv;
}

// ---------------------------------------------------------------------------
// HLLC: the contact is restored; star states keep their side's tangential
// velocities and scalars.  Branches: SL>=0 -> F_L; S*>=0 -> F*_L; SR>0 -> F*_R;
// otherwise F_R.
// ---------------------------------------------------------------------------
template <typename T, int D, int NSX, int DIR, typename G>
__device__ __forceinline__ void riemann_hllc(const T* WL, const T* WR, T* F, const G& gas) {
  if constexpr (G::RAD) {
    riemann_hllc_rad<T, D, NSX, DIR>(WL, WR, F, gas);
    return;
  }
  constexpr int NV = 2 + D + NSX;
  const T rL = WL[0], rR = WR[0], uL = WL[1 + DIR], uR = WR[1 + DIR];
  const T pL = WL[1 + D], pR = WR[1 + D];
  const T cL = dsqrt(qdiv(gas.g * pL, rL)), cR = dsqrt(qdiv(gas.g * pR, rR));
  const T SL = fmin(uL - cL, uR - cR);
  const T SR = fmax(uL + cL, uR + cR);
  if (SL >= T(0)) {
    phys_flux<T, D, NSX, DIR>(WL, F, gas);
    return;
  }
  if (SR <= T(0)) {
    phys_flux<T, D, NSX, DIR>(WR, F, gas);
    return;
  }
  const T aL = rL * (SL - uL), aR = rR * (SR - uR);
  const T Ss = qdiv(pR - pL + uL * aL - uR * aR, aL - aR);
  // pick the side of the contact
  const bool left = Ss >= T(0);
  T W[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) W[v] = left ? WL[v] : WR[v];
  const T S = left ? SL : SR;
  const T a = left ? aL : aR;  // rho_K (S_K - u_K)
  const T rho = W[0], un = W[1 + DIR], p = W[1 + D];
  T Fk[NV], Uk[NV];
  phys_flux<T, D, NSX, DIR>(W, Fk, gas);
  to_cons<T, D, NSX>(W, Uk, gas);
  const T fac = qdiv(a, S - Ss);
  T Us[NV];
  Us[0] = fac;
#pragma unroll
  for (int d = 0; d < D; ++d) Us[1 + d] = fac * W[1 + d];
  Us[1 + DIR] = fac * Ss;
  Us[1 + D] = fac * (qdiv(Uk[1 + D], rho) + (Ss - un) * (Ss + qdiv(p, a)));
#pragma unroll
  for (int s = 0; s < NSX; ++s) Us[2 + D + s] = fac * W[2 + D + s];
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = Fk[v] + S * (Us[v] - Uk[v]);
}

// ---------------------------------------------------------------------------
// Exact Riemann solver (Toro 2009 ch. 4).
// ---------------------------------------------------------------------------
// One side's pressure function f_K(p) and its derivative: shock branch
// (p > p_K) with A = 2/((g+1) rho_K), B = (g-1)/(g+1) p_K; rarefaction
// branch (p <= p_K) from the isentrope.
template <typename T>
__device__ __forceinline__ void press_fn(T p, T rK, T pK, T cK, const Gas<T>& gas, T& f, T& df) {
  if (p > pK) {
    const T A = qdiv(gas.A2, rK), B = gas.Bq * pK;
    const T q = dsqrt(qdiv(A, B + p));
    f = (p - pK) * q;
    df = q * (T(1) - T(0.5) * qdiv(p - pK, B + p));
  } else {
    const T pr = qdiv(p, pK);
    const T pz = dpow(pr, gas.z);  // (p/pK)^((g-1)/(2g))
    f = gas.two_gm1 * cK * (pz - T(1));
    // (p/pK)^(-(g+1)/(2g)) = (p/pK)^z / (p/pK)
    df = qdiv(pz, pr * rK * cK);
  }
}

// Toro's adaptive guess (Sect. 9.5.1 of Toro 2009): PVRS when the data are
// close (pmax/pmin <= 2 and PVRS within [pmin,pmax]); TRRS below pmin; TSRS
// otherwise.  kind: 0 PVRS, 1 TRRS, 2 TSRS.
template <typename T>
__device__ __forceinline__ T toro_guess(T rL, T uL, T pL, T cL, T rR, T uR, T pR, T cR,
                                        const Gas<T>& gas, int& kind) {
  T ppv = T(0.5) * (pL + pR) - T(0.125) * (uR - uL) * (rL + rR) * (cL + cR);
  ppv = fmax(ppv, T(0));
  const T pmin = fmin(pL, pR), pmax = fmax(pL, pR);
  if (qdiv(pmax, pmin) <= T(2) && ppv >= pmin && ppv <= pmax) {
    kind = 0;
    return ppv;
  }
  if (ppv < pmin) {
    kind = 1;
    const T num = cL + cR - T(0.5) * gas.gm1 * (uR - uL);
    const T den = qdiv(cL, dpow(pL, gas.z)) + qdiv(cR, dpow(pR, gas.z));
    return dpow(qdiv(num, den), gas.iz);
  }
  kind = 2;
  const T gL = dsqrt(qdiv(qdiv(gas.A2, rL), ppv + gas.Bq * pL));
  const T gR = dsqrt(qdiv(qdiv(gas.A2, rR), ppv + gas.Bq * pR));
  return qdiv(gL * pL + gR * pR - (uR - uL), gL + gR);
}

// Newton on f_L(p) + f_R(p) + (u_R - u_L) = 0 from p0: stop when the
// relative change 2|dp|/(p_k + p_{k-1}) < tol, then take one more step.
// Negative iterates are clamped to 1e-14 of the mean pressure.  In FP32 the
// step whose change is below tol (1e-6) is the last: Newton converges
// quadratically, so the iterate it gives is ~1e-12 from the root, far below
// FP32 resolution, and a further step would only move it within its own
// rounding.  The FP32 iteration also stops when the residual is within 8 ulp
// of the sum of the magnitudes of its terms (then with one more step): the
// rounding of f_L + f_R + du then decides the step, and no later iterate is
// better determined (near vacuum, where the two rarefaction terms nearly
// cancel du, the 1e-6 change is never reached).
template <typename T>
__device__ __forceinline__ int newton_star(T p, T rL, T uL, T pL, T cL, T rR, T uR, T pR, T cR,
                                           const Gas<T>& gas, T tol, T& ps, T& us, int& iters) {
  const T du = uR - uL;
  const T pfloor = T(1e-14) * T(0.5) * (pL + pR);
  if (!(p > pfloor)) p = pfloor;
  // One evaluation site for the pressure functions (the iterates and the
  // final p): the solver's code stays short.
  bool conv = false, fin = false;
  int it = 0;
  T fL, dfL, fR, dfR;
  for (;;) {
    press_fn(p, rL, pL, cL, gas, fL, dfL);
    press_fn(p, rR, pR, cR, gas, fR, dfR);
    if (fin || it >= 100) break;  // f at the final p (or the iteration limit)
    const T res = fL + fR + du;
    T pn = p - qdiv(res, dfL + dfR);
    if (pn < T(0)) pn = pfloor;
    ++it;
    const T ch = qdiv(T(2) * fabs(pn - p), pn + p);
    p = pn;
    if (conv) {
      fin = true;  // the extra step after convergence is done
      continue;
    }
    if (ch < tol) {
      conv = true;
      if constexpr (sizeof(T) == 4) fin = true;  // FP32: this step was the last
    }
    if constexpr (sizeof(T) == 4) {
      if (fabs(res) <= T(8 * 1.1920929e-7) * (fabs(fL) + fabs(fR) + fabs(du))) conv = true;
    }
  }
  iters = it;
  if (!conv) return ST_NEWTON;
  ps = p;
  us = T(0.5) * (uL + uR) + T(0.5) * (fR - fL);
  return ST_OK;
}

// A primitive 1D state returned by value (a local whose address an
// out-of-line function takes lives in local memory).
template <typename T>
struct Prim3 {
  T rho, u, p;
};

// The state inside a rarefaction fan at x/t = S (Toro ch. 4.5): sign = +1
// for the left fan (c = 2/(g+1) (cK + (g-1)/2 (uK - S)), u = c + S), -1 for
// the right one (c = 2/(g+1) (cK - (g-1)/2 (uK - S)), u = S - c); rho and P
// from the isentrope through (rK, pK).  Out of line: x/t = S lies inside a
// fan only near sonic points, and the hot solver code stays shorter.
template <typename T>
static __device__ __noinline__ Prim3<T> fan_state(T S, T sign, T rK, T uK, T pK, T cK, Gas<T> gas) {
  const T c = gas.A2 * (cK + sign * T(0.5) * gas.gm1 * (uK - S));
  Prim3<T> w;
  w.u = S + sign * c;
  w.rho = rK * dpow(qdiv(c, cK), gas.two_gm1);
  w.p = pK * dpow(qdiv(c, cK), gas.pow_c);
  return w;
}

// Sample the exact solution at x/t = S given the star state (Toro ch. 4.5);
// returns the (rho, u, P) there and whether it lies left of the contact
// (ties left).
template <typename T>
__device__ __forceinline__ bool sample_xi(T S, T rL, T uL, T pL, T cL, T rR, T uR, T pR, T cR, T ps,
                                          T us, const Gas<T>& gas, T& rho, T& u, T& p) {
  if (S <= us) {
    if (ps > pL) {
      const T SL = uL - cL * dsqrt(gas.zp * qdiv(ps, pL) + gas.z);
      if (S <= SL) { rho = rL; u = uL; p = pL; }
      else {
        const T q = qdiv(ps, pL);
        rho = qdiv(rL * (q + gas.Bq), gas.Bq * q + T(1));
        u = us; p = ps;
      }
    } else {
      const T SHL = uL - cL;
      const T cs = cL * dpow(qdiv(ps, pL), gas.z);
      const T STL = us - cs;
      if (S <= SHL) { rho = rL; u = uL; p = pL; }
      else if (S >= STL) {
        rho = rL * dpow(qdiv(ps, pL), gas.ig);
        u = us; p = ps;
      } else {
        {
          const Prim3<T> f = fan_state<T>(S, T(1), rL, uL, pL, cL, gas);
          rho = f.rho;
          u = f.u;
          p = f.p;
        }  // inside the left fan
      }
    }
    return true;
  }
  if (ps > pR) {
    const T SR = uR + cR * dsqrt(gas.zp * qdiv(ps, pR) + gas.z);
    if (S >= SR) { rho = rR; u = uR; p = pR; }
    else {
      const T q = qdiv(ps, pR);
      rho = qdiv(rR * (q + gas.Bq), gas.Bq * q + T(1));
      u = us; p = ps;
    }
  } else {
    const T SHR = uR + cR;
    const T cs = cR * dpow(qdiv(ps, pR), gas.z);
    const T STR = us + cs;
    if (S >= SHR) { rho = rR; u = uR; p = pR; }
    else if (S <= STR) {
      rho = rR * dpow(qdiv(ps, pR), gas.ig);
      u = us; p = ps;
    } else {
      {
          const Prim3<T> f = fan_state<T>(S, T(-1), rR, uR, pR, cR, gas);
          rho = f.rho;
          u = f.u;
          p = f.p;
        }  // inside the right fan
    }
  }
  return false;
}

// The same at x/t = 0, the value the Godunov flux needs.
template <typename T>
__device__ __forceinline__ bool sample0(T rL, T uL, T pL, T cL, T rR, T uR, T pR, T cR, T ps, T us,
                                        const Gas<T>& gas, T& rho, T& u, T& p) {
  return sample_xi<T>(T(0), rL, uL, pL, cL, rR, uR, pR, cR, ps, us, gas, rho, u, p);
}

// Newton tolerance per precision: 1e-10 in FP64; in FP32 the relative
// change cannot go below a few ulp, so 1e-6 is used there.
template <typename T> __device__ __forceinline__ T newton_tol();
template <> __device__ __forceinline__ double newton_tol<double>() { return 1e-10; }
template <> __device__ __forceinline__ float newton_tol<float>() { return 1e-6f; }

// Gas<double> from Gas<float> for the FP64 hard-face fallback.
__device__ __forceinline__ Gas<double> gas_double(const Gas<float>& g) {
  Gas<double> d;
  const double gg = (double)g.g;
  d.g = gg; d.gm1 = gg - 1.0; d.igm1 = 1.0 / (gg - 1.0); d.z = (gg - 1.0) / (2.0 * gg);
  d.iz = 1.0 / d.z; d.zp = (gg + 1.0) / (2.0 * gg); d.A2 = 2.0 / (gg + 1.0);
  d.Bq = (gg - 1.0) / (gg + 1.0); d.two_gm1 = 2.0 / (gg - 1.0); d.ig = 1.0 / gg;
  d.pow_c = 2.0 * gg / (gg - 1.0);
  return d;
}

// Star state of one face.  guess_in > 0 replaces Toro's guess (MLP).  In FP32
// a face near vacuum (margin below 20 %) or with a pressure ratio above 1e6
// is solved in FP64, where the FP32 pressure function loses digits.
// The FP64 Newton solve of an FP32 face near vacuum or with a pressure ratio
// above 1e6 (reading R12).  Kept out of line: it is rare, and its FP64 code
// would crowd the instruction cache of the FP32 kernels.
struct Star32 {
  float ps, us;
  int iters, st;
};
static __device__ __noinline__ Star32 newton_star_fp64(float p0, float rL, float uL, float pL, float rR, float uR,
                                                float pR, Gas<float> gas) {
  const Gas<double> g2 = gas_double(gas);
  double ps2 = 0.0, us2 = 0.0;
  const double cL2 = sqrt(g2.g * (double)pL / (double)rL), cR2 = sqrt(g2.g * (double)pR / (double)rR);
  Star32 r;
  r.iters = 0;
  r.st = newton_star<double>((double)p0, rL, uL, pL, cL2, rR, uR, pR, cR2, g2, 1e-10, ps2, us2, r.iters);
  r.ps = (float)ps2;
  r.us = (float)us2;
  return r;
}

// An FP32 face that is solved in FP64 (reading R12): pressure ratio above
// 1e6, or a velocity jump within 20 % of the vacuum limit vac =
// 2(cL+cR)/(g-1), where the FP32 residual loses more than ~5 of its bits to
// the cancellation of the two rarefaction terms against du.
template <typename T>
__device__ __forceinline__ bool hard_face(T pL, T pR, T du, T vac) {
  return qdiv(fmax(pL, pR), fmin(pL, pR)) > T(1e6) || vac - du < T(0.2) * vac;
}

// Star state from a given initial guess p0 and the sound speeds cL, cR of
// the two states (vacuum check, FP32 hard-face fallback, Newton).
template <typename T>
__device__ __forceinline__ int exact_star_from(T rL, T uL, T pL, T cL, T rR, T uR, T pR, T cR,
                                               const Gas<T>& gas, T p0, T& ps, T& us, int& iters) {
  const T vac = gas.two_gm1 * (cL + cR);
  if (vac <= uR - uL) return ST_VACUUM;
  if constexpr (sizeof(T) == 4) {
    if (hard_face<T>(pL, pR, uR - uL, vac)) {
      const Star32 r = newton_star_fp64(p0, rL, uL, pL, rR, uR, pR, gas);
      ps = r.ps;
      us = r.us;
      iters = r.iters;
      return r.st;
    }
  }
  return newton_star<T>(p0, rL, uL, pL, cL, rR, uR, pR, cR, gas, newton_tol<T>(), ps, us, iters);
}

template <typename T>
__device__ __forceinline__ int exact_star(T rL, T uL, T pL, T rR, T uR, T pR, const Gas<T>& gas,
                                          T guess_in, T& ps, T& us, int& iters, int& kind) {
  const T cL = dsqrt(qdiv(gas.g * pL, rL)), cR = dsqrt(qdiv(gas.g * pR, rR));
  if (gas.two_gm1 * (cL + cR) <= uR - uL) return ST_VACUUM;
  T p0 = toro_guess(rL, uL, pL, cL, rR, uR, pR, cR, gas, kind);
  if (guess_in > T(0)) p0 = guess_in;
  return exact_star_from<T>(rL, uL, pL, cL, rR, uR, pR, cR, gas, p0, ps, us, iters);
}

// Godunov flux from the exact solution at x/t = 0; tangential velocities and
// scalars come from the side of the contact.
template <typename T, int D, int NSX, int DIR>
__device__ __forceinline__ int riemann_exact(const T* WL, const T* WR, T* F, const Gas<T>& gas,
                                             T guess_in, int& iters, int& kind) {
  constexpr int NV = 2 + D + NSX;
  // Identical states: the solution is that state (no wave), and the general
  // path returns exactly its flux (PVRS gives p = P, Newton stops at once,
  // the sample is the state) -- take it directly.
  bool same = true;
#pragma unroll
  for (int v = 0; v < NV; ++v) same = same && WL[v] == WR[v];
  if (same) {
    iters = 0;
    kind = 0;
    phys_flux<T, D, NSX, DIR>(WL, F, gas);
    return ST_OK;
  }
  T ps, us;
  const T rL = WL[0], uL = WL[1 + DIR], pL = WL[1 + D];
  const T rR = WR[0], uR = WR[1 + DIR], pR = WR[1 + D];
  const int st = exact_star<T>(rL, uL, pL, rR, uR, pR, gas, guess_in, ps, us, iters, kind);
  if (st != ST_OK) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = T(0);
    return st;
  }
  const T cL = dsqrt(qdiv(gas.g * pL, rL)), cR = dsqrt(qdiv(gas.g * pR, rR));
  T rho, u, p;
  const bool left = sample0<T>(rL, uL, pL, cL, rR, uR, pR, cR, ps, us, gas, rho, u, p);
  T W[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) W[v] = left ? WL[v] : WR[v];
  W[0] = rho;
  W[1 + DIR] = u;
  W[1 + D] = p;
  phys_flux<T, D, NSX, DIR>(W, F, gas);
  return ST_OK;
}

// The Godunov flux of two different states (1D, no scalars) from a given
// initial guess p0 and their sound speeds: the batched path has both in
// hand from choosing the guess, so neither is computed twice.
template <typename T>
__device__ __forceinline__ int riemann_exact_from(const T* WL, const T* WR, T cL, T cR, T p0, T* F,
                                                  const Gas<T>& gas, int& iters) {
  T ps, us;
  const int st = exact_star_from<T>(WL[0], WL[1], WL[2], cL, WR[0], WR[1], WR[2], cR, gas, p0, ps, us, iters);
  if (st != ST_OK) {
#pragma unroll
    for (int v = 0; v < 3; ++v) F[v] = T(0);
    return st;
  }
  T W[3];
  const bool left = sample0<T>(WL[0], WL[1], WL[2], cL, WR[0], WR[1], WR[2], cR, ps, us, gas, W[0], W[1], W[2]);
  (void)left;
  phys_flux<T, 1, 0, 0>(W, F, gas);
  return ST_OK;
}

// ---------------------------------------------------------------------------
// MLP guess network: 6 -> 64 -> 64 -> 1 with SiLU, FP32 weights.
// ---------------------------------------------------------------------------
// Faces where the network replaces Toro's guess: his rule picks the two-shock
// estimate (kind 2) and the pressure jump exceeds a factor 4 -- where that
// estimate is poor; the two-rarefaction estimate is exact for two
// rarefactions and PVRS serves nearby states.
constexpr double MLP_GATE_RATIO = 4.0;
template <typename T>
__device__ __forceinline__ bool mlp_gate(int kind, T pL, T pR) {
  return kind == 2 && fmax(pL, pR) > T(MLP_GATE_RATIO) * fmin(pL, pR);
}

constexpr int MLP_IN = 6, MLP_H = 64;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
constexpr int MW1 = 0, MB1 = MW1 + MLP_H * MLP_IN, MW2 = MB1 + MLP_H, MB2 = MW2 + MLP_H * MLP_H,
              MW3 = MB2 + MLP_H, MB3 = MW3 + MLP_H;

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }

// Features of a face: log densities and pressures normalised by their
// geometric means, velocities by the reference sound speed; p_ref returned.
__device__ __forceinline__ void mlp_features(float g, float rL, float uL, float pL, float rR,
                                             float uR, float pR, float* x, float& pref) {
  const float rref = sqrtf(rL * rR);
  pref = sqrtf(pL * pR);
  const float icref = rsqrtf(g * pref / rref);
  x[0] = logf(rL / rref);
  x[1] = logf(rR / rref);
  x[2] = logf(pL / pref);
  x[3] = logf(pR / pref);
  x[4] = uL * icref;
  x[5] = uR * icref;
}

// Forward pass with the weights in shared (or global) memory; all lanes of a
// warp read the same weight at the same time (broadcast).
__device__ __forceinline__ float mlp_forward(const float* __restrict__ w, const float* x) {
  float h1[MLP_H];
#pragma unroll
  for (int o = 0; o < MLP_H; ++o) {
    float a = w[MB1 + o];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) a = fmaf(w[MW1 + o * MLP_IN + i], x[i], a);
    h1[o] = silu_f(a);
  }
  float y = w[MB3];
#pragma unroll 4
  for (int o = 0; o < MLP_H; ++o) {
    float a = w[MB2 + o];
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) a = fmaf(w[MW2 + o * MLP_H + i], h1[i], a);
    y = fmaf(w[MW3 + o], silu_f(a), y);
  }
  return y;
}

}  // namespace hydro
