/*
 * hydro_oracle.cpp -- plain FP64 CPU oracle of the HERACLES++ cell update.
 *
 * TEST INFRASTRUCTURE.  This is the slow reference the GPU library is checked
 * against; it is written for reading, not for speed.  Each step of the time
 * update is a separate pass over explicit arrays (ghost fill, primitives,
 * reconstruction + predictor, Riemann fluxes, update), in the order of
 * Sect. 3.2 of the paper, and every helper cites the passage it follows.
 * It shares no code with the CUDA library.
 *
 * Readings of passages the paper leaves silent or ambiguous (stated once here
 * and applied on both sides):
 *   R1  gravity sources are +rho g and +rho u.g with g the acceleration (the
 *       printed signs of Eq. 1b-c contradict Eq. 2-3 and the g_z<0 setups).
 *   R2  the multi-D Hancock predictor sums the flux differences of all
 *       directions (the unsplit form Eq. 18 refers to for 3D).
 *   R3  Davis wave-speed estimates for HLL/HLLC.
 *   R4  CFL time step dt = C / max_cells sum_d (|u_d| + c)/h_d.
 *   R5  spherical sources: Eq. 14 as printed for the rho u_phi u_r and
 *       rho u_phi u_theta terms; cot(theta)(rho u_phi^2 + P)/r and the radial
 *       ((rho u_theta^2+P)+(rho u_phi^2+P))/r written with face fluxes times
 *       (dS_+ - dS_-)/dV so that a static uniform state is exactly balanced
 *       (the printed Eq. 16 carries an extra cos/(2 sin) factor, read as a typo).
 *       For an axis the grid does not have, the face-flux mean is replaced by
 *       rho u^2 + P (absent velocity zero) of the cell's half-step state
 *       U_i + dU_i from the Hancock predictor -- what the face fluxes give for a
 *       state without structure along that axis -- or of U_i^n if that
 *       half-step state is not physical.
 *   R6  ghost cells: per-axis mapping (periodic wrap, transmissive copy of the
 *       edge cell, reflective mirror with the normal momentum negated).  A ghost
 *       copies its source cell's geometry too: its width, and the radius and
 *       mean polar sine that enter its physical widths h_d; ghost centres lie
 *       outside the boundary at the distances those widths give.  (With
 *       mirrored geometry a reflective wall stays exactly symmetric, so no
 *       mass or angular momentum crosses it.)
 *   R7  a predicted face state with rho<=0 or p<=0 falls back to the cell
 *       average (first order on that face).
 *   R8  gravity and heating are evaluated from the state at t^n.
 *   R9  monopole mass M_i = Mc + (4 pi/Omega)(sum_{i'<i} m_i' + m_i/2).
 *   R10 exact solver: Newton from a guess until 2|dp|/(p_k+p_{k-1}) < 1e-10,
 *       then one more Newton step; sampled at x/t = 0, ties go to the left.
 *   R13 gas + radiation EoS (Eq. 6): the gas part is rho R T with R = k_b/(mu
 *       m_u) (Eq. 6 prints k_b/mu without the atomic mass unit).
 *   R14 its temperature: Newton on the monotone, convex e(T) or P(T) from the
 *       upper bound min(gas-only, radiation-only temperature), until the
 *       relative step is below 1e-13, then one more step.
 *   R15 dual energy (Sect. 2.5): div(u e) and P div(u) use the face fluxes
 *       u_f e_f = F_rho (e/rho)_upwind and u_f = F_rho/rho_upwind (upwind by
 *       the sign of F_rho) with the dS/dV of the update; P is the cell's t^n
 *       pressure; alpha comes from the t^n state; heating enters delta2;
 *       where alpha = 1 the total energy is left as the update gives it;
 *       otherwise E = e_new + rho|u|^2/2 of the new state.
 */
#include "hydro_oracle.h"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double PI = 3.14159265358979323846;
const int NG = 2;  // ghost layers per side

/* ------------------------------------------------------------------ */
/* Ideal-gas EoS, Sect. 2.3 Eq. 5:  P = (gamma-1) e,  c = sqrt(gamma P/rho)   */
/* Gas + radiation EoS, Sect. 2.3 Eq. 6-7 (kind 1):                           */
/*   e = rho R T/(gamma-1) + a T^4,  P = rho R T + a T^4/3,                    */
/*   c^2 = (gamma/(gamma-1) + 20 alpha + 16 alpha^2)/(1/(gamma-1) + 12 alpha)  */
/*         * P_g/rho,  alpha = P_r/P_g,                                        */
/* with R = k_b/(mu m_u) the specific gas constant (reading R13: Eq. 6 prints  */
/* k_b/mu; the atomic mass unit belongs with mu) and a the radiation constant. */
/* Primitive vector W = (rho, u_1..u_D, P, f_1..f_S); conserved U = (rho,     */
/* rho u_1..rho u_D, E, rho f_1..rho f_S), E = e + rho|u|^2/2 (Sect. 2.1).      */
/* ------------------------------------------------------------------ */
struct Eos {
  double gamma;
  int D;  // number of velocity components (= dim)
  int S;  // passive scalars
  int kind = 0;              // 0 ideal gas, 1 gas + radiation
  double R = 0.0, a = 0.0;   // gas + radiation constants
  int nv() const { return 2 + D + S; }
};

/* Temperature where c1 T + c4 T^4 = y (c1 > 0, c4 >= 0, y > 0): the left side
 * is increasing and convex in T > 0, so Newton started from the upper bound
 * min(y/c1, (y/c4)^(1/4)) decreases monotonically to the root (the paper's
 * "Newton-Raphson approach", Sect. 2.3).  Reading R14: stop once the relative
 * step is below 1e-13, then take one more step.  y <= 0 returns y/c1 <= 0,
 * which the callers' positivity checks reject. */
double rad_temperature(double c1, double c4, double y) {
  double T = y / c1;
  if (!(y > 0.0)) return T;
  if (c4 > 0.0) T = std::fmin(T, std::pow(y / c4, 0.25));
  bool conv = false;
  for (int it = 0; it < 200; ++it) {
    double f = c1 * T + c4 * T * T * T * T - y;
    double df = c1 + 4.0 * c4 * T * T * T;
    double Tn = T - f / df;
    double ch = std::fabs(Tn - T) / Tn;
    T = Tn;
    if (conv) break;
    if (ch < 1e-13) conv = true;
  }
  return T;
}

/* Pressure from the internal energy per volume (Eq. 5 or Eq. 6). */
double eos_pressure(const Eos& eos, double rho, double e) {
  if (eos.kind == 0) return (eos.gamma - 1.0) * e;
  double T = rad_temperature(rho * eos.R / (eos.gamma - 1.0), eos.a, e);
  return rho * eos.R * T + eos.a * T * T * T * T / 3.0;
}

/* Internal energy per volume from the pressure. */
double eos_eint(const Eos& eos, double rho, double p) {
  if (eos.kind == 0) return p / (eos.gamma - 1.0);
  double T = rad_temperature(rho * eos.R, eos.a / 3.0, p);
  return rho * eos.R * T / (eos.gamma - 1.0) + eos.a * T * T * T * T;
}

double sound_speed(const Eos& eos, double rho, double p) {
  if (eos.kind == 0) return std::sqrt(eos.gamma * p / rho);
  double T = rad_temperature(rho * eos.R, eos.a / 3.0, p);
  double pg = rho * eos.R * T, pr = eos.a * T * T * T * T / 3.0;
  double al = pr / pg, g = eos.gamma;
  return std::sqrt((g / (g - 1.0) + 20.0 * al + 16.0 * al * al) / (1.0 / (g - 1.0) + 12.0 * al) * pg / rho);
}

void cons_to_prim(const Eos& eos, const double* U, double* W) {
  double rho = U[0];
  double ke = 0.0;
  W[0] = rho;
  for (int d = 0; d < eos.D; ++d) {
    W[1 + d] = U[1 + d] / rho;
    ke += 0.5 * U[1 + d] * W[1 + d];
  }
  if (eos.kind == 0) W[1 + eos.D] = (eos.gamma - 1.0) * (U[1 + eos.D] - ke);
  else W[1 + eos.D] = eos_pressure(eos, rho, U[1 + eos.D] - ke);
  for (int s = 0; s < eos.S; ++s) W[2 + eos.D + s] = U[2 + eos.D + s] / rho;
}

void prim_to_cons(const Eos& eos, const double* W, double* U) {
  double rho = W[0];
  double ke = 0.0;
  U[0] = rho;
  for (int d = 0; d < eos.D; ++d) {
    U[1 + d] = rho * W[1 + d];
    ke += 0.5 * rho * W[1 + d] * W[1 + d];
  }
  if (eos.kind == 0) U[1 + eos.D] = W[1 + eos.D] / (eos.gamma - 1.0) + ke;
  else U[1 + eos.D] = eos_eint(eos, rho, W[1 + eos.D]) + ke;
  for (int s = 0; s < eos.S; ++s) U[2 + eos.D + s] = rho * W[2 + eos.D + s];
}

/* Physical flux of Eq. 1 through a face normal to axis d (from the primitives). */
void phys_flux(const Eos& eos, const double* W, int d, double* F) {
  double rho = W[0], un = W[1 + d], p = W[1 + eos.D];
  double ke = 0.0;
  for (int e = 0; e < eos.D; ++e) ke += 0.5 * rho * W[1 + e] * W[1 + e];
  double E = (eos.kind == 0 ? p / (eos.gamma - 1.0) : eos_eint(eos, rho, p)) + ke;
  F[0] = rho * un;
  for (int e = 0; e < eos.D; ++e) F[1 + e] = rho * un * W[1 + e];
  F[1 + d] += p;
  F[1 + eos.D] = un * (E + p);
  for (int s = 0; s < eos.S; ++s) F[2 + eos.D + s] = rho * un * W[2 + eos.D + s];
}

bool state_ok(const Eos& eos, const double* U) {
  double W[16];
  cons_to_prim(eos, U, W);
  return W[0] > 0.0 && W[1 + eos.D] > 0.0;
}

bool all_finite(const double* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

/* ------------------------------------------------------------------ */
/* Slope limiters named in Sect. 3.2 (Eq. 17): minmod, van Leer, van Albada. */
/* The paper prints no formulas; these are the standard slope forms of the   */
/* two one-sided differences dm, dp, all zero when dm*dp <= 0.                */
/* ------------------------------------------------------------------ */
double limiter(int kind, double dm, double dp) {
  if (kind == ORC_FIRST_ORDER) return 0.0;
  if (dm * dp <= 0.0) return 0.0;
  if (kind == ORC_MINMOD) return dm > 0.0 ? std::fmin(dm, dp) : std::fmax(dm, dp);
  if (kind == ORC_VANLEER) return 2.0 * dm * dp / (dm + dp);
  /* van Albada */
  return dm * dp * (dm + dp) / (dm * dm + dp * dp);
}

/* ------------------------------------------------------------------ */
/* Riemann solvers.  Input: left/right primitive states on a face normal to  */
/* axis d.  Output: the numerical flux.                                      */
/* ------------------------------------------------------------------ */

/* HLL (Harten-Lax-van Leer; Toro 2009 ch.10), Davis wave speeds (reading R3). */
void flux_hll(const Eos& eos, const double* WL, const double* WR, int d, double* F) {
  int nv = eos.nv();
  double cL = sound_speed(eos, WL[0], WL[1 + eos.D]);
  double cR = sound_speed(eos, WR[0], WR[1 + eos.D]);
  double uL = WL[1 + d], uR = WR[1 + d];
  double SL = std::fmin(uL - cL, uR - cR);
  double SR = std::fmax(uL + cL, uR + cR);
  double FL[16], FR[16], UL[16], UR[16];
  phys_flux(eos, WL, d, FL);
  phys_flux(eos, WR, d, FR);
  if (SL >= 0.0) {
    for (int v = 0; v < nv; ++v) F[v] = FL[v];
    return;
  }
  if (SR <= 0.0) {
    for (int v = 0; v < nv; ++v) F[v] = FR[v];
    return;
  }
  prim_to_cons(eos, WL, UL);
  prim_to_cons(eos, WR, UR);
  for (int v = 0; v < nv; ++v)
    F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
}

/* HLLC (Toro 2009 ch.10): restores the contact; star states carry the
 * tangential velocities and the passive scalars of their side. */
void hllc_star(const Eos& eos, const double* W, const double* U, int d, double S, double Sstar,
               double* Us) {
  int D = eos.D;
  double rho = W[0], un = W[1 + d], p = W[1 + D];
  double fac = rho * (S - un) / (S - Sstar);
  Us[0] = fac;
  for (int e = 0; e < D; ++e) Us[1 + e] = fac * W[1 + e];
  Us[1 + d] = fac * Sstar;
  Us[1 + D] = fac * (U[1 + D] / rho + (Sstar - un) * (Sstar + p / (rho * (S - un))));
  for (int s = 0; s < eos.S; ++s) Us[2 + D + s] = fac * W[2 + D + s];
}

void flux_hllc(const Eos& eos, const double* WL, const double* WR, int d, double* F) {
  int nv = eos.nv(), D = eos.D;
  double rL = WL[0], rR = WR[0], uL = WL[1 + d], uR = WR[1 + d];
  double pL = WL[1 + D], pR = WR[1 + D];
  double cL = sound_speed(eos, rL, pL), cR = sound_speed(eos, rR, pR);
  double SL = std::fmin(uL - cL, uR - cR);
  double SR = std::fmax(uL + cL, uR + cR);
  double Sstar = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /
                 (rL * (SL - uL) - rR * (SR - uR));
  double FL[16], FR[16], UL[16], UR[16], Us[16];
  if (SL >= 0.0) {
    phys_flux(eos, WL, d, F);
  } else if (Sstar >= 0.0) {
    phys_flux(eos, WL, d, FL);
    prim_to_cons(eos, WL, UL);
    hllc_star(eos, WL, UL, d, SL, Sstar, Us);
    for (int v = 0; v < nv; ++v) F[v] = FL[v] + SL * (Us[v] - UL[v]);
  } else if (SR > 0.0) {
    phys_flux(eos, WR, d, FR);
    prim_to_cons(eos, WR, UR);
    hllc_star(eos, WR, UR, d, SR, Sstar, Us);
    for (int v = 0; v < nv; ++v) F[v] = FR[v] + SR * (Us[v] - UR[v]);
  } else {
    phys_flux(eos, WR, d, F);
  }
}

/* Exact Riemann solver for the ideal gas (Toro 2009 ch.4), used in the paper
 * as the "analytical" Sod solution (App. C.1).  Pressure function of one side:
 *   shock (p > pK):       (p - pK) sqrt(A_K / (p + B_K)),  A=2/((g+1) rho), B=(g-1)pK/(g+1)
 *   rarefaction (p<=pK):  2 cK/(g-1) ((p/pK)^((g-1)/(2g)) - 1)                               */
void pressure_fn(double g, double p, double rK, double pK, double cK, double* f, double* df) {
  if (p > pK) {
    double A = 2.0 / ((g + 1.0) * rK), B = (g - 1.0) / (g + 1.0) * pK;
    double q = std::sqrt(A / (B + p));
    *f = (p - pK) * q;
    *df = q * (1.0 - 0.5 * (p - pK) / (B + p));
  } else {
    double pr = p / pK;
    *f = 2.0 * cK / (g - 1.0) * (std::pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
    *df = 1.0 / (rK * cK) * std::pow(pr, -(g + 1.0) / (2.0 * g));
  }
}

/* Toro's adaptive initial guess (Toro 2009 Sect. 9.5.1): primitive-variable
 * (PVRS) when the data are close, two-rarefaction (TRRS) when the PVRS
 * pressure falls below both, two-shock (TSRS) otherwise.  kind: 0/1/2. */
double toro_guess(double g, double rL, double uL, double pL, double rR, double uR, double pR,
                  int* kind) {
  double cL = std::sqrt(g * pL / rL), cR = std::sqrt(g * pR / rR);
  double ppv = 0.5 * (pL + pR) - 0.125 * (uR - uL) * (rL + rR) * (cL + cR);
  if (ppv < 0.0) ppv = 0.0;
  double pmin = std::fmin(pL, pR), pmax = std::fmax(pL, pR);
  if (pmax / pmin <= 2.0 && ppv >= pmin && ppv <= pmax) {
    *kind = 0;
    return ppv;
  }
  if (ppv < pmin) {
    double z = (g - 1.0) / (2.0 * g);
    double num = cL + cR - 0.5 * (g - 1.0) * (uR - uL);
    double den = cL / std::pow(pL, z) + cR / std::pow(pR, z);
    *kind = 1;
    return std::pow(num / den, 1.0 / z);
  }
  double AL = 2.0 / ((g + 1.0) * rL), BL = (g - 1.0) / (g + 1.0) * pL;
  double AR = 2.0 / ((g + 1.0) * rR), BR = (g - 1.0) / (g + 1.0) * pR;
  double gL = std::sqrt(AL / (ppv + BL)), gR = std::sqrt(AR / (ppv + BR));
  *kind = 2;
  return (gL * pL + gR * pR - (uR - uL)) / (gL + gR);
}

/* MLP p* guess: 6 -> 64 -> 64 -> 1 with SiLU, FP32 weights evaluated in FP64.
 * Layout of the flat weight vector (4673 values): W1[64][6], b1[64],
 * W2[64][64], b2[64], w3[64], b3.  Output y = ln(p_star/p_ref) with p_ref
 * the geometric mean of the two pressures.  It replaces Toro's guess only
 * where Toro's rule picks the two-shock (TSRS) estimate and the pressure
 * jump exceeds a factor 4 (reading R11): PVRS serves nearby states, the
 * two-rarefaction estimate is exact when both waves are rarefactions, and
 * the two-shock estimate is good for mild jumps. */
const int MLP_IN = 6, MLP_H = 64;
const int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
const int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
          OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H;

double silu(double z) { return z / (1.0 + std::exp(-z)); }
double dsilu(double z) {
  double s = 1.0 / (1.0 + std::exp(-z));
  return s * (1.0 + z * (1.0 - s));
}

/* Features: states normalised by the geometric-mean density and pressure of
 * the two sides, velocities by the reference sound speed. */
void mlp_features(double g, const double* WL, const double* WR, double* x, double* pref) {
  double rref = std::sqrt(WL[0] * WR[0]);
  double p_ref = std::sqrt(WL[2] * WR[2]);
  double cref = std::sqrt(g * p_ref / rref);
  x[0] = std::log(WL[0] / rref);
  x[1] = std::log(WR[0] / rref);
  x[2] = std::log(WL[2] / p_ref);
  x[3] = std::log(WR[2] / p_ref);
  x[4] = WL[1] / cref;
  x[5] = WR[1] / cref;
  *pref = p_ref;
}

double mlp_eval(const float* w, const double* x, double* z1, double* h1, double* z2, double* h2) {
  for (int o = 0; o < MLP_H; ++o) {
    double a = w[OFF_B1 + o];
    for (int i = 0; i < MLP_IN; ++i) a += (double)w[OFF_W1 + o * MLP_IN + i] * x[i];
    z1[o] = a;
    h1[o] = silu(a);
  }
  for (int o = 0; o < MLP_H; ++o) {
    double a = w[OFF_B2 + o];
    for (int i = 0; i < MLP_H; ++i) a += (double)w[OFF_W2 + o * MLP_H + i] * h1[i];
    z2[o] = a;
    h2[o] = silu(a);
  }
  double y = w[OFF_B3];
  for (int i = 0; i < MLP_H; ++i) y += (double)w[OFF_W3 + i] * h2[i];
  return y;
}

struct ExactResult {
  double pstar, ustar;
  int iters;
  bool used_mlp;
  int status;
};

/* Star-region pressure and velocity by Newton iteration on
 * f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0 (reading R10). */
ExactResult exact_star(double g, const double* WL, const double* WR, int guess,
                       const float* mlpw) {
  ExactResult r = {0.0, 0.0, 0, false, ORC_OK};
  double rL = WL[0], uL = WL[1], pL = WL[2], rR = WR[0], uR = WR[1], pR = WR[2];
  double cL = std::sqrt(g * pL / rL), cR = std::sqrt(g * pR / rR);
  double du = uR - uL;
  if (2.0 * (cL + cR) / (g - 1.0) <= du) {  // vacuum is generated
    r.status = ORC_ERR_VACUUM;
    return r;
  }
  int kind = 0;
  double p = toro_guess(g, rL, uL, pL, rR, uR, pR, &kind);
  const bool gate = kind == 2 && std::fmax(pL, pR) > 4.0 * std::fmin(pL, pR);
  if (guess == ORC_GUESS_MLP && gate && mlpw != nullptr) {
    double x[6], pref, z1[64], h1[64], z2[64], h2[64];
    mlp_features(g, WL, WR, x, &pref);
    p = pref * std::exp(mlp_eval(mlpw, x, z1, h1, z2, h2));
    r.used_mlp = true;
  }
  double pfloor = 1e-14 * 0.5 * (pL + pR);
  if (!(p > pfloor)) p = pfloor;
  int it = 0;
  bool converged = false;
  while (it < 100) {
    double fL, dfL, fR, dfR;
    pressure_fn(g, p, rL, pL, cL, &fL, &dfL);
    pressure_fn(g, p, rR, pR, cR, &fR, &dfR);
    double pn = p - (fL + fR + du) / (dfL + dfR);
    if (pn < 0.0) pn = pfloor;
    ++it;
    double change = 2.0 * std::fabs(pn - p) / (pn + p);
    p = pn;
    if (converged) break;           // this was the extra polishing step
    if (change < 1e-10) converged = true;
  }
  if (!converged) {
    r.status = ORC_ERR_NEWTON;
    return r;
  }
  double fL, dfL, fR, dfR;
  pressure_fn(g, p, rL, pL, cL, &fL, &dfL);
  pressure_fn(g, p, rR, pR, cR, &fR, &dfR);
  r.pstar = p;
  r.ustar = 0.5 * (uL + uR) + 0.5 * (fR - fL);
  r.iters = it;
  return r;
}

/* Sample the exact solution at similarity coordinate xi = x/t (Toro ch.4).
 * Output (rho, u, p) and side = -1 (left of contact) / +1 (right). */
void exact_sample(double g, const double* WL, const double* WR, double ps, double us, double xi,
                  double* out, int* side) {
  double rL = WL[0], uL = WL[1], pL = WL[2], rR = WR[0], uR = WR[1], pR = WR[2];
  double cL = std::sqrt(g * pL / rL), cR = std::sqrt(g * pR / rR);
  double gm = (g - 1.0) / (g + 1.0);
  if (xi <= us) {  // left of the contact
    *side = -1;
    if (ps > pL) {  // left shock
      double SL = uL - cL * std::sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g));
      if (xi <= SL) {
        out[0] = rL; out[1] = uL; out[2] = pL;
      } else {
        out[0] = rL * (ps / pL + gm) / (gm * ps / pL + 1.0);
        out[1] = us; out[2] = ps;
      }
    } else {  // left rarefaction
      double SHL = uL - cL;
      double cs = cL * std::pow(ps / pL, (g - 1.0) / (2.0 * g));
      double STL = us - cs;
      if (xi <= SHL) {
        out[0] = rL; out[1] = uL; out[2] = pL;
      } else if (xi >= STL) {
        out[0] = rL * std::pow(ps / pL, 1.0 / g);
        out[1] = us; out[2] = ps;
      } else {
        double c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - xi));
        out[1] = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + xi);
        out[0] = rL * std::pow(c / cL, 2.0 / (g - 1.0));
        out[2] = pL * std::pow(c / cL, 2.0 * g / (g - 1.0));
      }
    }
  } else {  // right of the contact
    *side = 1;
    if (ps > pR) {  // right shock
      double SR = uR + cR * std::sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g));
      if (xi >= SR) {
        out[0] = rR; out[1] = uR; out[2] = pR;
      } else {
        out[0] = rR * (ps / pR + gm) / (gm * ps / pR + 1.0);
        out[1] = us; out[2] = ps;
      }
    } else {  // right rarefaction
      double SHR = uR + cR;
      double cs = cR * std::pow(ps / pR, (g - 1.0) / (2.0 * g));
      double STR = us + cs;
      if (xi >= SHR) {
        out[0] = rR; out[1] = uR; out[2] = pR;
      } else if (xi <= STR) {
        out[0] = rR * std::pow(ps / pR, 1.0 / g);
        out[1] = us; out[2] = ps;
      } else {
        double c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - xi));
        out[1] = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + xi);
        out[0] = rR * std::pow(c / cR, 2.0 / (g - 1.0));
        out[2] = pR * std::pow(c / cR, 2.0 * g / (g - 1.0));
      }
    }
  }
}

struct ExactStats {
  long long iters = 0, mlp = 0;
};

/* Godunov flux from the exact solution sampled at x/t = 0; tangential
 * velocities and scalars are taken from the side of the contact. */
int flux_exact(const Eos& eos, const double* WL, const double* WR, int d, int guess,
               const float* mlpw, double* F, ExactStats* st) {
  int D = eos.D;
  double wl[3] = {WL[0], WL[1 + d], WL[1 + D]};
  double wr[3] = {WR[0], WR[1 + d], WR[1 + D]};
  ExactResult er = exact_star(eos.gamma, wl, wr, guess, mlpw);
  if (er.status != ORC_OK) return er.status;
  st->iters += er.iters;
  if (er.used_mlp) st->mlp += 1;
  double s[3];
  int side;
  exact_sample(eos.gamma, wl, wr, er.pstar, er.ustar, 0.0, s, &side);
  const double* Wt = side < 0 ? WL : WR;
  double W[16];
  for (int v = 0; v < eos.nv(); ++v) W[v] = Wt[v];
  W[0] = s[0];
  W[1 + d] = s[1];
  W[1 + D] = s[2];
  phys_flux(eos, W, d, F);
  return ORC_OK;
}

/* Flux through a face that moves with velocity w along its normal d (the
 * moving grid of Sect. 3.1.1, reading R16): G = F(W) - w U(W) of the
 * Riemann solution sampled on the face's path x/t = w.  HLL and HLLC take
 * the state of the wave region that contains w (ties as at w = 0); the
 * exact solver samples its solution at x/t = w. */
int flux_moving(const Eos& eos, int riemann, const double* WL, const double* WR, int d, double w, int guess,
                const float* mlpw, double* G, ExactStats* st) {
  const int nv = eos.nv(), D = eos.D;
  double Wx[16], Ux[16], Fx[16];
  if (riemann == ORC_EXACT) {
    double wl[3] = {WL[0], WL[1 + d], WL[1 + D]};
    double wr[3] = {WR[0], WR[1 + d], WR[1 + D]};
    ExactResult er = exact_star(eos.gamma, wl, wr, guess, mlpw);
    if (er.status != ORC_OK) return er.status;
    st->iters += er.iters;
    if (er.used_mlp) st->mlp += 1;
    double smp[3];
    int side;
    exact_sample(eos.gamma, wl, wr, er.pstar, er.ustar, w, smp, &side);
    const double* Wt = side < 0 ? WL : WR;
    for (int v = 0; v < nv; ++v) Wx[v] = Wt[v];
    Wx[0] = smp[0];
    Wx[1 + d] = smp[1];
    Wx[1 + D] = smp[2];
    phys_flux(eos, Wx, d, Fx);
    prim_to_cons(eos, Wx, Ux);
    for (int v = 0; v < nv; ++v) G[v] = Fx[v] - w * Ux[v];
    return ORC_OK;
  }
  double rL = WL[0], rR = WR[0], uL = WL[1 + d], uR = WR[1 + d];
  double pL = WL[1 + D], pR = WR[1 + D];
  double cL = sound_speed(eos, rL, pL), cR = sound_speed(eos, rR, pR);
  double SL = std::fmin(uL - cL, uR - cR);
  double SR = std::fmax(uL + cL, uR + cR);
  double FL[16], FR[16], UL[16], UR[16];
  phys_flux(eos, WL, d, FL);
  phys_flux(eos, WR, d, FR);
  prim_to_cons(eos, WL, UL);
  prim_to_cons(eos, WR, UR);
  if (SL >= w) {
    for (int v = 0; v < nv; ++v) G[v] = FL[v] - w * UL[v];
    return ORC_OK;
  }
  if (riemann == ORC_HLL) {
    if (SR <= w) {
      for (int v = 0; v < nv; ++v) G[v] = FR[v] - w * UR[v];
      return ORC_OK;
    }
    for (int v = 0; v < nv; ++v) {
      double Fh = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
      double Uh = (SR * UR[v] - SL * UL[v] - (FR[v] - FL[v])) / (SR - SL);
      G[v] = Fh - w * Uh;
    }
    return ORC_OK;
  }
  double Sstar = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
  double Us[16];
  if (Sstar >= w) {
    hllc_star(eos, WL, UL, d, SL, Sstar, Us);
    for (int v = 0; v < nv; ++v) G[v] = FL[v] + SL * (Us[v] - UL[v]) - w * Us[v];
  } else if (SR > w) {
    hllc_star(eos, WR, UR, d, SR, Sstar, Us);
    for (int v = 0; v < nv; ++v) G[v] = FR[v] + SR * (Us[v] - UR[v]) - w * Us[v];
  } else {
    for (int v = 0; v < nv; ++v) G[v] = FR[v] - w * UR[v];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Heating / cooling source, Sect. 2.4.  NI56: Eq. 8-9 in CGS units.        */
/* ------------------------------------------------------------------ */
const double M_U = 1.66053906660e-24;     // atomic mass unit [g] (CODATA 2018)
const double MEV = 1.602176634e-6;        // 1 MeV [erg] (exact SI definition)
const double DAY = 86400.0;               // [s]
const double Q_NI = 1.75 * MEV, Q_CO = 3.73 * MEV;
const double TAU_NI = 8.8 * DAY, TAU_CO = 111.3 * DAY;

double heating_rate(int kind, const double* prm, double t, double rho_f_ni) {
  if (kind == ORC_HEAT_CONST) return prm[0];
  if (kind == ORC_HEAT_NI56) {
    double lambda = 1.0 / (56.0 * M_U * (TAU_CO - TAU_NI));
    return lambda * ((Q_NI * (TAU_CO / TAU_NI - 1.0) - Q_CO) * std::exp(-t / TAU_NI) +
                     Q_CO * std::exp(-t / TAU_CO)) * rho_f_ni;
  }
  return 0.0;
}

/* ------------------------------------------------------------------ */
/* The grid solver.                                                     */
/* ------------------------------------------------------------------ */
struct Solver {
  int dim, n[3], coords, riemann, lim, bc[3][2];
  Eos eos;
  int gravity = ORC_GRAV_NONE, heating = ORC_HEAT_NONE, guess = ORC_GUESS_TORO;
  double eps_dual = 0.0;        // dual-energy criterion epsilon (Sect. 2.5); 0 = off
  double g0[3] = {0, 0, 0}, G = 0.0, Mc = 0.0, heat_prm[4] = {0, 0, 0, 0};
  std::vector<float> mlpw;
  double t = 0.0;
  std::vector<double> xf[3];    // interior face coordinates per axis (n+1)
  std::vector<double> xfe[3];   // face coordinates including ghosts (n+2NG+1)
  std::vector<double> U;        // interior state [v][k][j][i]
  long long st_faces = 0, st_iters = 0, st_fallback = 0, st_mlp = 0;
  /* Domain decomposition (Sect. 3.3.1: one subdomain per process, ghost
   * layers exchanged with the neighbouring subdomains).  The sides of one
   * axis, xaxis, may be exchanged: their ghosts are the neighbour's cells,
   * given by the caller as halo[side] = [v][layer][cross section] (layer l =
   * the ghost at distance l+1 from the boundary; the cross section runs over
   * the two other axes, the lower axis fastest), and their geometry is that
   * of those cells, from xg[side] = the NG face coordinates beyond the side,
   * nearest first. */
  int xaxis = -1;
  bool xch[2] = {false, false};
  double xg[2][NG] = {{0.0, 0.0}, {0.0, 0.0}};
  std::vector<double> halo[2];
  /* Monopole of a subdomain split along r: the mass of all shells inside it
   * (reading R9's running sum where this subdomain's shells begin). */
  double inner_mass = 0.0;
  /* Moving grid (Sect. 3.1.1, reading R16): the faces of axis maxis move
   * with velocity wgrid; every step shifts them by wgrid dt. */
  int maxis = -1;
  double wgrid = 0.0;

  bool exch_ghost(int d, int g) const {
    return d == xaxis && ((g < 0 && xch[0]) || (g >= n[d] && xch[1]));
  }
  /* Cells of the cross section of axis a: the two other axes. */
  long cross(int a) const { return a == 0 ? (long)n[1] * n[2] : a == 1 ? (long)n[0] * n[2] : (long)n[0] * n[1]; }
  long cross_idx(int a, int i, int j, int k) const {
    return a == 0 ? (long)k * n[1] + j : a == 1 ? (long)k * n[0] + i : (long)j * n[0] + i;
  }

  int m(int d) const { return d < dim ? n[d] + 2 * NG : 1; }
  int off(int d) const { return d < dim ? NG : 0; }
  long ncell() const { return (long)n[0] * n[1] * n[2]; }
  long next() const { return (long)m(0) * m(1) * m(2); }
  long eidx(int i, int j, int k) const { return ((long)k * m(1) + j) * m(0) + i; }
  long iidx(int i, int j, int k) const { return ((long)k * n[1] + j) * n[0] + i; }

  /* Interior cell whose state (and geometry) a cell of axis-d index g copies
   * (reading R6); g itself for interior cells. */
  int src(int d, int g) const {
    if (d >= dim) return 0;
    int nn = n[d];
    if (g < 0) {
      if (bc[d][0] == ORC_PERIODIC) return g + nn;
      if (bc[d][0] == ORC_TRANSMISSIVE) return 0;
      return -1 - g;
    }
    if (g >= nn) {
      if (bc[d][1] == ORC_PERIODIC) return g - nn;
      if (bc[d][1] == ORC_TRANSMISSIVE) return nn - 1;
      return 2 * nn - 1 - g;
    }
    return g;
  }

  /* Ghost geometry (reading R6): a ghost has its source cell's width; face
   * positions accumulate outward from the boundary. */
  void build_ext_faces() {
    for (int d = 0; d < 3; ++d) {
      xfe[d].clear();
      if (d >= dim) {
        xfe[d] = {xf[d][0], xf[d][1]};
        continue;
      }
      int nn = n[d];
      auto width = [&](int g) {  // width of the ghost's source cell
        int sidx = src(d, g);
        return xf[d][sidx + 1] - xf[d][sidx];
      };
      xfe[d].assign(nn + 2 * NG + 1, 0.0);
      for (int f = 0; f <= nn; ++f) xfe[d][f + NG] = xf[d][f];
      for (int gcell = -1; gcell >= -NG; --gcell) xfe[d][gcell + NG] = xfe[d][gcell + NG + 1] - width(gcell);
      for (int gcell = nn; gcell < nn + NG; ++gcell)
        xfe[d][gcell + NG + 1] = xfe[d][gcell + NG] + width(gcell);
      /* exchanged sides: the neighbour's own faces */
      if (d == xaxis) {
        for (int l = 0; l < NG; ++l) {
          if (xch[0]) xfe[d][NG - 1 - l] = xg[0][l];
          if (xch[1]) xfe[d][nn + NG + 1 + l] = xg[1][l];
        }
      }
    }
  }
  double xlo(int d, int ie) const { return xfe[d][ie]; }
  double xhi(int d, int ie) const { return xfe[d][ie + 1]; }
  double xc(int d, int ie) const { return 0.5 * (xfe[d][ie] + xfe[d][ie + 1]); }

  /* Angular extents of the axes that are absent in lower-dimensional spherical
   * runs: the full sphere. */
  double th_lo(int je) const { return dim >= 2 ? xlo(1, je) : 0.0; }
  double th_hi(int je) const { return dim >= 2 ? xhi(1, je) : PI; }
  double ph_lo(int ke) const { return dim >= 3 ? xlo(2, ke) : 0.0; }
  double ph_hi(int ke) const { return dim >= 3 ? xhi(2, ke) : 2.0 * PI; }

  /* Cell volume and face areas, Sect. 3.1.1 ("computed based on the chosen
   * geometry"): Cartesian products of widths; spherical exact integrals. */
  double dV(int ie, int je, int ke) const {
    if (coords == ORC_CARTESIAN) {
      double v = 1.0;
      for (int d = 0; d < dim; ++d) v *= xhi(d, d == 0 ? ie : d == 1 ? je : ke) - xlo(d, d == 0 ? ie : d == 1 ? je : ke);
      return v;
    }
    double rm = xlo(0, ie), rp = xhi(0, ie);
    return (rp * rp * rp - rm * rm * rm) / 3.0 * (std::cos(th_lo(je)) - std::cos(th_hi(je))) *
           (ph_hi(ke) - ph_lo(ke));
  }
  /* Area of the face on the low (side=0) or high (side=1) side of cell e along d. */
  double dS(int d, int side, int ie, int je, int ke) const {
    if (coords == ORC_CARTESIAN) {
      double a = 1.0;
      int idx[3] = {ie, je, ke};
      for (int e = 0; e < dim; ++e)
        if (e != d) a *= xhi(e, idx[e]) - xlo(e, idx[e]);
      return a;
    }
    double rm = xlo(0, ie), rp = xhi(0, ie);
    if (d == 0) {
      double r = side ? rp : rm;
      return r * r * (std::cos(th_lo(je)) - std::cos(th_hi(je))) * (ph_hi(ke) - ph_lo(ke));
    }
    if (d == 1) {
      double th = side ? th_hi(je) : th_lo(je);
      return 0.5 * (rp * rp - rm * rm) * std::sin(th) * (ph_hi(ke) - ph_lo(ke));
    }
    return 0.5 * (rp * rp - rm * rm) * (th_hi(je) - th_lo(je));
  }
  /* Area of a face averaged over a step in which the faces of the moving
   * axis shift by Dl (reading R16): a radial face sweeps r^2 from r to r+Dl,
   * whose mean is r^2 + r Dl + Dl^2/3 (so that the swept volumes add up to
   * the change of the cell volumes); the theta and phi faces' (r+^2 - r-^2)/2
   * varies linearly, so its mean is the mid-step value.  Cartesian areas do
   * not change with a shift. */
  double dS_avg(int d, int side, int ie, int je, int ke, double Dl) const {
    if (coords == ORC_CARTESIAN) return dS(d, side, ie, je, ke);
    double rm = xlo(0, ie), rp = xhi(0, ie);
    if (d == 0) {
      double r = side ? rp : rm;
      return (r * r + r * Dl + Dl * Dl / 3.0) * (std::cos(th_lo(je)) - std::cos(th_hi(je))) *
             (ph_hi(ke) - ph_lo(ke));
    }
    double a2 = 0.5 * (rp - rm) * (rp + rm + Dl);
    if (d == 1) {
      double th = side ? th_hi(je) : th_lo(je);
      return a2 * std::sin(th) * (ph_hi(ke) - ph_lo(ke));
    }
    return a2 * (th_hi(je) - th_lo(je));
  }
  /* Physical width of cell e along d (used by the predictor and the CFL):
   * h_r = dr, h_theta = r_i dtheta, h_phi = r_i sin(theta)_j dphi with
   * r_i the mid radius and sin(theta)_j the mean of the face sines. */
  double h(int d, int ie, int je, int ke) const {
    /* geometry of the source cells (reading R6), interior extended indices;
     * an exchanged ghost is a real cell of the neighbour with its own */
    auto gidx = [&](int d2, int e) { return exch_ghost(d2, e - off(d2)) ? e : src(d2, e - off(d2)) + off(d2); };
    int i = gidx(0, ie), j = gidx(1, je);
    int idx[3] = {i, j, gidx(2, ke)};
    double w = xhi(d, idx[d]) - xlo(d, idx[d]);
    if (coords == ORC_CARTESIAN || d == 0) return w;
    double r = xc(0, i);
    if (d == 1) return r * w;
    double s = 0.5 * (std::sin(th_lo(j)) + std::sin(th_hi(j)));
    return r * s * w;
  }

  /* Step a1: ghost fill by per-axis index mapping (reading R6). */
  void fill_ext(std::vector<double>& Ue) const {
    int nv = eos.nv();
    long ne = next();
    Ue.assign((size_t)nv * ne, 0.0);
    for (int ke = 0; ke < m(2); ++ke)
      for (int je = 0; je < m(1); ++je)
        for (int ie = 0; ie < m(0); ++ie) {
          int src[3] = {ie - off(0), je - off(1), ke - off(2)};
          bool flip[3] = {false, false, false};
          int layer = -1, side = 0;  // an exchanged ghost: its halo layer and side
          for (int d = 0; d < dim; ++d) {
            int g = src[d], nn = n[d];
            if (exch_ghost(d, g)) {
              side = g < 0 ? 0 : 1;
              layer = g < 0 ? -1 - g : g - nn;
              src[d] = 0;
              continue;
            }
            if (g < 0) {
              if (bc[d][0] == ORC_PERIODIC) g += nn;
              else if (bc[d][0] == ORC_TRANSMISSIVE) g = 0;
              else { g = -1 - g; flip[d] = true; }
            } else if (g >= nn) {
              if (bc[d][1] == ORC_PERIODIC) g -= nn;
              else if (bc[d][1] == ORC_TRANSMISSIVE) g = nn - 1;
              else { g = 2 * nn - 1 - g; flip[d] = true; }
            }
            src[d] = g;
          }
          long e = eidx(ie, je, ke);
          if (layer >= 0) {
            const long nx = cross(xaxis);
            const long q = cross_idx(xaxis, src[0], src[1], src[2]);
            for (int v = 0; v < nv; ++v)
              Ue[(size_t)v * ne + e] = halo[side][((size_t)v * NG + layer) * nx + q];
          } else {
            long s = iidx(src[0], src[1], src[2]);
            for (int v = 0; v < nv; ++v) Ue[(size_t)v * ne + e] = U[(size_t)v * ncell() + s];
          }
          for (int d = 0; d < dim; ++d)
            if (flip[d]) Ue[(size_t)(1 + d) * ne + e] = -Ue[(size_t)(1 + d) * ne + e];
        }
  }

  /* Enclosed mass per radial cell (reading R9), FP64, fixed order. */
  /* Shell masses m_i = sum_jk rho dV (FP64, fixed order). */
  void shell_masses(std::vector<double>& shell) const {
    int nr = n[0];
    shell.assign(nr, 0.0);
    for (int i = 0; i < nr; ++i)
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          shell[i] += U[iidx(i, j, k)] * dV(i + off(0), j + off(1), k + off(2));
  }
  void monopole_mass(std::vector<double>& M) const {
    int nr = n[0];
    std::vector<double> shell;
    shell_masses(shell);
    double omega = (std::cos(th_lo(off(1))) - std::cos(th_hi(off(1) + n[1] - 1))) *
                   (ph_hi(off(2) + n[2] - 1) - ph_lo(off(2)));
    M.assign(nr, 0.0);
    double below = inner_mass;
    for (int i = 0; i < nr; ++i) {
      M[i] = Mc + 4.0 * PI / omega * (below + 0.5 * shell[i]);
      below += shell[i];
    }
  }

  int step(double dt);
  int cfl(double C, double* dt) const;
};

int Solver::cfl(double C, double* dtout) const {
  /* Reading R4: dt = C / max sum_d (|u_d| + c)/h_d over interior cells. */
  int nv = eos.nv();
  double W[16], Uc[16];
  double smax = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        for (int v = 0; v < nv; ++v) Uc[v] = U[(size_t)v * ncell() + iidx(i, j, k)];
        cons_to_prim(eos, Uc, W);
        if (!(W[0] > 0.0) || !(W[1 + dim] > 0.0)) return ORC_ERR_NEGATIVE_STATE;
        double c = sound_speed(eos, W[0], W[1 + dim]);
        double s = 0.0;
        /* on a moving axis the signal speed is taken relative to the faces */
        for (int d = 0; d < dim; ++d)
          s += (std::fabs(W[1 + d] - (d == maxis ? wgrid : 0.0)) + c) / h(d, i + off(0), j + off(1), k + off(2));
        if (s > smax) smax = s;
      }
  *dtout = C / smax;
  return ORC_OK;
}

int Solver::step(double dt) {
  const int nv = eos.nv();
  const long ne = next();
  const long nc = ncell();
  if (!all_finite(U.data(), U.size())) return ORC_ERR_NONFINITE;

  /* a1: ghost fill */
  std::vector<double> Ue;
  fill_ext(Ue);

  /* a2: primitives everywhere (Eq. 5) */
  std::vector<double> We((size_t)nv * ne);
  for (long e = 0; e < ne; ++e) {
    double u[16], w[16];
    for (int v = 0; v < nv; ++v) u[v] = Ue[(size_t)v * ne + e];
    cons_to_prim(eos, u, w);
    if (!(w[0] > 0.0) || !(w[1 + dim] > 0.0)) return ORC_ERR_NEGATIVE_STATE;
    for (int v = 0; v < nv; ++v) We[(size_t)v * ne + e] = w[v];
  }

  /* a3+a4: limited slopes, face states (Eq. 17) and the Hancock predictor
   * (Eq. 18, unsplit sum over directions, reading R2) for every extended cell
   * whose neighbours along all axes exist.  Uf[d][side] holds the predicted
   * conserved face states, side 0 = low face, 1 = high face. */
  std::vector<double> Uf[3][2];
  std::vector<double> dUc((size_t)nv * ne, 0.0);  // predictor increment per cell
  for (int d = 0; d < dim; ++d)
    for (int s = 0; s < 2; ++s) Uf[d][s].assign((size_t)nv * ne, 0.0);
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = d < dim ? 1 : 0;
    hi[d] = d < dim ? m(d) - 1 : 1;
  }
  for (int ke = lo[2]; ke < hi[2]; ++ke)
    for (int je = lo[1]; je < hi[1]; ++je)
      for (int ie = lo[0]; ie < hi[0]; ++ie) {
        long e = eidx(ie, je, ke);
        int idx[3] = {ie, je, ke};
        double Wc[16], Wfs[3][2][16], Ufs[3][2][16];
        for (int v = 0; v < nv; ++v) Wc[v] = We[(size_t)v * ne + e];
        for (int d = 0; d < dim; ++d) {
          long stride = d == 0 ? 1 : d == 1 ? m(0) : (long)m(0) * m(1);
          double xm = xc(d, idx[d] - 1), x0 = xc(d, idx[d]), xp = xc(d, idx[d] + 1);
          double wdt = xhi(d, idx[d]) - xlo(d, idx[d]);
          for (int v = 0; v < nv; ++v) {
            double wm = We[(size_t)v * ne + e - stride], wp = We[(size_t)v * ne + e + stride];
            double dm = (Wc[v] - wm) / (x0 - xm);
            double dp = (wp - Wc[v]) / (xp - x0);
            double sig = limiter(lim, dm, dp);
            Wfs[d][0][v] = Wc[v] - 0.5 * wdt * sig;
            Wfs[d][1][v] = Wc[v] + 0.5 * wdt * sig;
          }
          prim_to_cons(eos, Wfs[d][0], Ufs[d][0]);
          prim_to_cons(eos, Wfs[d][1], Ufs[d][1]);
        }
        double dU[16];
        for (int v = 0; v < nv; ++v) dU[v] = 0.0;
        for (int d = 0; d < dim; ++d) {
          double Fm[16], Fp[16];
          phys_flux(eos, Wfs[d][0], d, Fm);
          phys_flux(eos, Wfs[d][1], d, Fp);
          /* a moving axis: the fluxes through faces that move with the grid,
           * F - w U (reading R16) */
          if (d == maxis && wgrid != 0.0)
            for (int v = 0; v < nv; ++v) {
              Fm[v] -= wgrid * Ufs[d][0][v];
              Fp[v] -= wgrid * Ufs[d][1][v];
            }
          double hd = h(d, ie, je, ke);
          for (int v = 0; v < nv; ++v) dU[v] += 0.5 * dt * (Fm[v] - Fp[v]) / hd;
        }
        for (int v = 0; v < nv; ++v) dUc[(size_t)v * ne + e] = dU[v];
        for (int d = 0; d < dim; ++d) {
          double Um[16], Up[16];
          for (int v = 0; v < nv; ++v) {
            Um[v] = Ufs[d][0][v] + dU[v];
            Up[v] = Ufs[d][1][v] + dU[v];
          }
          /* reading R7: a non-physical predicted face state is replaced by the
           * cell average (first order in space and time on that face) */
          if (!state_ok(eos, Um)) {
            for (int v = 0; v < nv; ++v) Um[v] = Ue[(size_t)v * ne + e];
            ++st_fallback;
          }
          if (!state_ok(eos, Up)) {
            for (int v = 0; v < nv; ++v) Up[v] = Ue[(size_t)v * ne + e];
            ++st_fallback;
          }
          for (int v = 0; v < nv; ++v) {
            Uf[d][0][(size_t)v * ne + e] = Um[v];
            Uf[d][1][(size_t)v * ne + e] = Up[v];
          }
        }
      }

  /* a5: Riemann fluxes on every face of the interior cells.  Fx[d] is indexed
   * by the extended index of the cell on the LOW side of the face's high
   * neighbour, i.e. face (ie+1/2) is stored at ie. */
  std::vector<double> Fl[3];
  /* dual energy (Sect. 2.5, reading R15): per face the advected internal
   * energy u_f e_f = F_rho (e/rho)_upwind and the face velocity
   * u_f = F_rho / rho_upwind, upwind by the sign of the mass flux */
  std::vector<double> Q1[3], Q2[3];
  ExactStats est;
  for (int d = 0; d < dim; ++d) {
    Fl[d].assign((size_t)nv * ne, 0.0);
    Q1[d].assign((size_t)ne, 0.0);
    Q2[d].assign((size_t)ne, 0.0);
    long stride = d == 0 ? 1 : d == 1 ? m(0) : (long)m(0) * m(1);
    /* for axis d the face index runs 0..n[d]; the other axes over interior cells */
    int fl[3] = {0, 0, 0}, fh[3] = {n[0], n[1], n[2]};
    fh[d] = n[d] + 1;
    for (int k = fl[2]; k < fh[2]; ++k)
      for (int j = fl[1]; j < fh[1]; ++j)
        for (int i = fl[0]; i < fh[0]; ++i) {
          // high-side cell of face f along d has interior index f, low side f-1
          int ie = i + off(0), je = j + off(1), ke = k + off(2);
          long eR = eidx(ie, je, ke);
          long eL = eR - stride;
          double UL[16], UR[16], WL[16], WR[16], F[16];
          for (int v = 0; v < nv; ++v) {
            UL[v] = Uf[d][1][(size_t)v * ne + eL];
            UR[v] = Uf[d][0][(size_t)v * ne + eR];
          }
          cons_to_prim(eos, UL, WL);
          cons_to_prim(eos, UR, WR);
          if (d == maxis && wgrid != 0.0) {
            int s = flux_moving(eos, riemann, WL, WR, d, wgrid, guess, mlpw.empty() ? nullptr : mlpw.data(), F,
                                &est);
            if (s != ORC_OK) return s;
          } else if (riemann == ORC_HLL) flux_hll(eos, WL, WR, d, F);
          else if (riemann == ORC_HLLC) flux_hllc(eos, WL, WR, d, F);
          else {
            int s = flux_exact(eos, WL, WR, d, guess, mlpw.empty() ? nullptr : mlpw.data(), F, &est);
            if (s != ORC_OK) return s;
          }
          ++st_faces;
          for (int v = 0; v < nv; ++v) Fl[d][(size_t)v * ne + eL] = F[v];
          if (eps_dual > 0.0) {
            const double* Wu = F[0] >= 0.0 ? WL : WR;
            const double eu = eos_eint(eos, Wu[0], Wu[1 + dim]);
            Q1[d][(size_t)eL] = F[0] * eu / Wu[0];
            Q2[d][(size_t)eL] = F[0] / Wu[0];
          }
        }
  }
  st_iters += est.iters;
  st_mlp += est.mlp;

  std::vector<double> Mshell;
  if (gravity == ORC_GRAV_POINT_MONOPOLE) monopole_mass(Mshell);

  /* a6-a8: conservative update (Eq. 19 with dS/dV), geometric sources
   * (Eq. 13-16, reading R5), gravity (Eq. 2-4, R1, R8), heating (Sect. 2.4). */
  std::vector<double> Un(U.size());
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int ie = i + off(0), je = j + off(1), ke = k + off(2);
        long e = eidx(ie, je, ke);
        double vol = dV(ie, je, ke);
        /* moving grid (reading R16): face areas averaged over the step, the
         * volume after it, and the radii sum of the Eq. 14 weight at mid-step */
        const bool moving = maxis >= 0 && wgrid != 0.0;
        const double Dl = moving ? wgrid * dt : 0.0;
        double vol_new = vol;
        if (moving && coords == ORC_SPHERICAL) {
          double rm = xlo(0, ie) + Dl, rp = xhi(0, ie) + Dl;
          vol_new = (rp * rp * rp - rm * rm * rm) / 3.0 * (std::cos(th_lo(je)) - std::cos(th_hi(je))) *
                    (ph_hi(ke) - ph_lo(ke));
        }
        double acc[16], Uc[16], Wc[16];
        for (int v = 0; v < nv; ++v) {
          acc[v] = 0.0;
          Uc[v] = U[(size_t)v * nc + iidx(i, j, k)];
        }
        cons_to_prim(eos, Uc, Wc);
        double Flo[3][16], Fhi[3][16], Slo[3], Shi[3];
        double A1 = 0.0, A2 = 0.0;  // sums of u_f e_f dS and u_f dS (dual energy)
        for (int d = 0; d < dim; ++d) {
          long stride = d == 0 ? 1 : d == 1 ? m(0) : (long)m(0) * m(1);
          Slo[d] = moving ? dS_avg(d, 0, ie, je, ke, Dl) : dS(d, 0, ie, je, ke);
          Shi[d] = moving ? dS_avg(d, 1, ie, je, ke, Dl) : dS(d, 1, ie, je, ke);
          for (int v = 0; v < nv; ++v) {
            Flo[d][v] = Fl[d][(size_t)v * ne + e - stride];
            Fhi[d][v] = Fl[d][(size_t)v * ne + e];
            acc[v] += Flo[d][v] * Slo[d];
            acc[v] -= Fhi[d][v] * Shi[d];
          }
          if (eps_dual > 0.0) {
            A1 += Q1[d][(size_t)(e - stride)] * Slo[d] - Q1[d][(size_t)e] * Shi[d];
            A2 += Q2[d][(size_t)(e - stride)] * Slo[d] - Q2[d][(size_t)e] * Shi[d];
          }
        }
        double Unew[16];
        for (int v = 0; v < nv; ++v) Unew[v] = Uc[v] + dt / vol * acc[v];

        if (coords == ORC_SPHERICAL) {
          double rm = xlo(0, ie), rp = xhi(0, ie);
          /* pressure of the half-step cell state (reading R5) */
          double Uh[16], Wh[16];
          for (int v = 0; v < nv; ++v) Uh[v] = Uc[v] + dUc[(size_t)v * ne + e];
          cons_to_prim(eos, Uh, Wh);
          double P = (Wh[0] > 0.0 && Wh[1 + dim] > 0.0) ? Wh[1 + dim] : Wc[1 + dim];
          double rfac = (rp - rm) / ((rp + rm + Dl) * vol);
          /* theta-direction and phi-direction momentum-flux means; cell
           * values (rho u^2 + P with the absent velocity zero) when the axis
           * is absent. */
          double Tth = dim >= 2 ? 0.5 * (Flo[1][2] + Fhi[1][2]) : P;
          double Tph = dim >= 3 ? 0.5 * (Flo[2][3] + Fhi[2][3]) : P;
          /* radial momentum: ((rho u_th^2+P) + (rho u_ph^2+P))/r */
          Unew[1] += dt * 0.5 * (Tth + Tph) * (Shi[0] - Slo[0]) / vol;
          if (dim >= 2) {
            /* theta momentum: -rho u_th u_r / r  (Eq. 14 form) + cot(th)(rho u_ph^2+P)/r */
            Unew[2] += dt * (-rfac * (Fhi[0][2] * Shi[0] + Flo[0][2] * Slo[0]) +
                             Tph * (Shi[1] - Slo[1]) / vol);
          }
          if (dim >= 3) {
            /* phi momentum: Eq. 14 */
            double sm = std::sin(xlo(1, je)), sp = std::sin(xhi(1, je));
            double sfac = (sp - sm) / ((sp + sm) * vol);
            Unew[3] += dt * (-rfac * (Fhi[0][3] * Shi[0] + Flo[0][3] * Slo[0]) -
                             sfac * (Fhi[1][3] * Shi[1] + Flo[1][3] * Slo[1]));
          }
        }

        if (gravity != ORC_GRAV_NONE) {
          double gv[3] = {0.0, 0.0, 0.0};
          if (gravity == ORC_GRAV_UNIFORM) {
            for (int d = 0; d < dim; ++d) gv[d] = g0[d];
          } else {
            double r = xc(0, ie);
            double M = gravity == ORC_GRAV_POINT ? Mc : Mshell[i];
            gv[0] = -G * M / (r * r);
          }
          for (int d = 0; d < dim; ++d) Unew[1 + d] += dt * Uc[0] * gv[d];
          double work = 0.0;
          for (int d = 0; d < dim; ++d) work += Uc[1 + d] * gv[d];
          Unew[1 + dim] += dt * work;
        }

        double dheat = 0.0;
        if (heating != ORC_HEAT_NONE) {
          double rfni = 0.0;
          if (heating == ORC_HEAT_NI56) rfni = Uc[2 + dim + (int)heat_prm[0]];
          dheat = dt * heating_rate(heating, heat_prm, t, rfni);
          Unew[1 + dim] += dheat;
        }

        /* dual energy (Sect. 2.5): where the internal energy is small against
         * the kinetic energy, blend the internal-energy change of the total-
         * energy update (delta1) with that of de/dt + div(u e) + P div(u) = 0
         * (delta2, plus the heating) by the weight alpha of the t^n state. */
        if (eps_dual > 0.0) {
          double ke0 = 0.0, ke1 = 0.0;
          for (int d = 0; d < dim; ++d) {
            ke0 += 0.5 * Uc[1 + d] * Uc[1 + d] / Uc[0];
            ke1 += 0.5 * Unew[1 + d] * Unew[1 + d] / Unew[0];
          }
          double e0 = Uc[1 + dim] - ke0;
          double crit = eps_dual * ke0;
          double alpha = e0 >= crit ? 1.0 : (e0 > 0.1 * crit ? (e0 / crit) * (e0 / crit) : 0.0);
          if (alpha < 1.0) {
            double d1 = (Unew[1 + dim] - ke1) - e0;
            double d2 = dt / vol * (A1 + Wc[1 + dim] * A2) + dheat;
            Unew[1 + dim] = e0 + alpha * d1 + (1.0 - alpha) * d2 + ke1;
          }
        }

        /* moving grid: the content of the old cell, now spread over the new one */
        if (moving && vol_new != vol)
          for (int v = 0; v < nv; ++v) Unew[v] *= vol / vol_new;
        for (int v = 0; v < nv; ++v) Un[(size_t)v * nc + iidx(i, j, k)] = Unew[v];
      }

  /* state checks on the result; on error the state is left unchanged */
  for (long c = 0; c < nc; ++c) {
    double u[16];
    for (int v = 0; v < nv; ++v) u[v] = Un[(size_t)v * nc + c];
    if (!all_finite(u, (size_t)nv)) return ORC_ERR_NONFINITE;
    if (!state_ok(eos, u)) return ORC_ERR_NEGATIVE_STATE;
  }
  U.swap(Un);
  t += dt;
  if (maxis >= 0 && wgrid != 0.0) {
    for (double& f : xf[maxis]) f += wgrid * dt;
    build_ext_faces();
  }
  return ORC_OK;
}

}  // namespace

struct orc_ctx {
  Solver s;
};

extern "C" {

int orc_create(int dim, const int* n, const double* faces, const int* bc, int coords,
               double gamma, int n_scalars, int riemann, int limiter_kind, orc_t* out) {
  if (dim < 1 || dim > 3 || !n || !faces || !bc || !out) return ORC_ERR_ARG;
  if (n_scalars < 0 || n_scalars > 8 || riemann < 0 || riemann > 2 || limiter_kind < 0 || limiter_kind > 3)
    return ORC_ERR_ARG;
  if (riemann == ORC_EXACT && n_scalars < 0) return ORC_ERR_ARG;
  orc_ctx* c = new orc_ctx();
  Solver& s = c->s;
  s.dim = dim;
  s.coords = coords;
  s.riemann = riemann;
  s.lim = limiter_kind;
  s.eos = {gamma, dim, n_scalars};
  const double* f = faces;
  for (int d = 0; d < 3; ++d) {
    s.n[d] = d < dim ? n[d] : 1;
    s.bc[d][0] = d < dim ? bc[2 * d] : ORC_PERIODIC;
    s.bc[d][1] = d < dim ? bc[2 * d + 1] : ORC_PERIODIC;
    if (d < dim) {
      if (s.n[d] < 2) { delete c; return ORC_ERR_ARG; }
      s.xf[d].assign(f, f + s.n[d] + 1);
      f += s.n[d] + 1;
    } else {
      s.xf[d] = {0.0, 1.0};
    }
  }
  s.build_ext_faces();
  s.U.assign((size_t)s.eos.nv() * s.ncell(), 0.0);
  *out = c;
  return ORC_OK;
}

void orc_destroy(orc_t h) { delete h; }

int orc_set_sources(orc_t h, int gravity, const double* g0, double G, double Mc, int heating,
                    const double* heat_params) {
  Solver& s = h->s;
  if (gravity >= ORC_GRAV_POINT && s.coords != ORC_SPHERICAL) return ORC_ERR_ARG;
  s.gravity = gravity;
  for (int d = 0; d < 3; ++d) s.g0[d] = g0 ? g0[d] : 0.0;
  s.G = G;
  s.Mc = Mc;
  s.heating = heating;
  for (int i = 0; i < 4; ++i) s.heat_prm[i] = heat_params ? heat_params[i] : 0.0;
  return ORC_OK;
}

int orc_set_dual_energy(orc_t h, double eps) {
  if (!(eps >= 0.0)) return ORC_ERR_ARG;
  if (eps > 0.0 && h->s.maxis >= 0) return ORC_ERR_ARG;  /* not with a moving grid */
  h->s.eps_dual = eps;
  return ORC_OK;
}

int orc_set_eos_radiation(orc_t h, double R, double a) {
  if (!(R > 0.0) || !(a >= 0.0) || h->s.riemann == ORC_EXACT) return ORC_ERR_ARG;
  h->s.eos.kind = 1;
  h->s.eos.R = R;
  h->s.eos.a = a;
  return ORC_OK;
}

int orc_eos_rad(double gamma, double R, double a, double rho, double e, double* T, double* P, double* c) {
  Eos eos = {gamma, 1, 0};
  eos.kind = 1;
  eos.R = R;
  eos.a = a;
  *T = rad_temperature(rho * R / (gamma - 1.0), a, e);
  *P = eos_pressure(eos, rho, e);
  *c = sound_speed(eos, rho, *P);
  return ORC_OK;
}

int orc_eos_rad_eint(double gamma, double R, double a, double rho, double P, double* T, double* e) {
  Eos eos = {gamma, 1, 0};
  eos.kind = 1;
  eos.R = R;
  eos.a = a;
  *T = rad_temperature(rho * R, a / 3.0, P);
  *e = eos_eint(eos, rho, P);
  return ORC_OK;
}

int orc_set_guess(orc_t h, int guess, const float* w) {
  h->s.guess = guess;
  if (w) h->s.mlpw.assign(w, w + MLP_NPARAM);
  return ORC_OK;
}

int orc_set_state(orc_t h, const double* U) {
  std::memcpy(h->s.U.data(), U, h->s.U.size() * sizeof(double));
  return ORC_OK;
}
int orc_get_state(orc_t h, double* U) {
  std::memcpy(U, h->s.U.data(), h->s.U.size() * sizeof(double));
  return ORC_OK;
}
int orc_set_time(orc_t h, double t) {
  h->s.t = t;
  return ORC_OK;
}
int orc_cfl_dt(orc_t h, double cfl, double* dt) { return h->s.cfl(cfl, dt); }
int orc_step(orc_t h, double dt) { return h->s.step(dt); }

int orc_totals(orc_t h, double* out) {
  /* a10: sum of U dV over the interior, FP64, fixed order. */
  Solver& s = h->s;
  int nv = s.eos.nv();
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int k = 0; k < s.n[2]; ++k)
      for (int j = 0; j < s.n[1]; ++j)
        for (int i = 0; i < s.n[0]; ++i)
          acc += s.U[(size_t)v * s.ncell() + s.iidx(i, j, k)] * s.dV(i + s.off(0), j + s.off(1), k + s.off(2));
    out[v] = acc;
  }
  return ORC_OK;
}

int orc_stats(orc_t h, long long* out) {
  out[0] = h->s.st_faces;
  out[1] = h->s.st_iters;
  out[2] = h->s.st_fallback;
  out[3] = h->s.st_mlp;
  return ORC_OK;
}

int orc_shell_mass(orc_t h, double* M) {
  std::vector<double> m;
  h->s.monopole_mass(m);
  for (size_t i = 0; i < m.size(); ++i) M[i] = m[i];
  return ORC_OK;
}

int orc_set_exchange(orc_t h, int axis, int side, const double* ghost_faces) {
  Solver& s = h->s;
  if (axis < 0 || axis >= s.dim || side < 0 || side > 1 || !ghost_faces) return ORC_ERR_ARG;
  if (s.xaxis >= 0 && s.xaxis != axis) return ORC_ERR_ARG;  /* slabs: one axis */
  if (s.maxis >= 0) return ORC_ERR_ARG;                      /* not with a moving grid */
  s.xaxis = axis;
  s.xch[side] = true;
  for (int l = 0; l < NG; ++l) s.xg[side][l] = ghost_faces[l];
  s.halo[side].assign((size_t)s.eos.nv() * NG * s.cross(axis), 0.0);
  s.build_ext_faces();
  return ORC_OK;
}

int orc_set_halo(orc_t h, int axis, int side, const double* halo) {
  Solver& s = h->s;
  if (axis != s.xaxis || side < 0 || side > 1 || !s.xch[side] || !halo) return ORC_ERR_ARG;
  std::copy(halo, halo + s.halo[side].size(), s.halo[side].begin());
  return ORC_OK;
}

int orc_get_boundary(orc_t h, int axis, int side, double* out) {
  Solver& s = h->s;
  if (axis < 0 || axis >= s.dim || side < 0 || side > 1 || !out) return ORC_ERR_ARG;
  const int nv = s.eos.nv();
  const long nx = s.cross(axis);
  for (int v = 0; v < nv; ++v)
    for (int l = 0; l < NG; ++l)
      for (int k = 0; k < s.n[2]; ++k)
        for (int j = 0; j < s.n[1]; ++j)
          for (int i = 0; i < s.n[0]; ++i) {
            int g = axis == 0 ? i : axis == 1 ? j : k;
            int want = side == 0 ? l : s.n[axis] - 1 - l;
            if (g != want) continue;
            out[((size_t)v * NG + l) * nx + s.cross_idx(axis, i, j, k)] =
                s.U[(size_t)v * s.ncell() + s.iidx(i, j, k)];
          }
  return ORC_OK;
}

int orc_set_moving_grid(orc_t h, int axis, double w) {
  Solver& s = h->s;
  if (axis < 0 || axis >= s.dim || !std::isfinite(w)) return ORC_ERR_ARG;
  if (s.coords == ORC_SPHERICAL && axis != 0) return ORC_ERR_ARG;       /* radial only */
  if (s.xaxis >= 0 || s.eps_dual > 0.0) return ORC_ERR_ARG;            /* not with slabs or dual energy */
  for (int side = 0; side < 2; ++side) {
    int b = s.bc[axis][side];
    if (b == ORC_REFLECTIVE || (b == ORC_PERIODIC && s.coords == ORC_SPHERICAL)) return ORC_ERR_ARG;
  }
  s.maxis = axis;
  s.wgrid = w;
  return ORC_OK;
}

int orc_get_faces(orc_t h, int axis, double* out) {
  Solver& s = h->s;
  if (axis < 0 || axis >= s.dim || !out) return ORC_ERR_ARG;
  for (size_t f = 0; f < s.xf[axis].size(); ++f) out[f] = s.xf[axis][f];
  return ORC_OK;
}

int orc_shell_masses(orc_t h, double* m) {
  std::vector<double> sm;
  h->s.shell_masses(sm);
  for (size_t i = 0; i < sm.size(); ++i) m[i] = sm[i];
  return ORC_OK;
}

int orc_set_inner_mass(orc_t h, double mass) {
  h->s.inner_mass = mass;
  return ORC_OK;
}

int orc_batch_run(const int* lengths, int ntubes, double* U, double gamma, int riemann,
                  int limiter_kind, double cfl, int nsteps, int guess, const float* mlp_weights,
                  int nthreads, long long* stats_out) {
  /* Independent 1D tubes on [0,1] with uniform cells and transmissive ends;
   * each takes nsteps steps at its own CFL time step. */
  std::vector<long> off(ntubes + 1, 0);
  for (int b = 0; b < ntubes; ++b) off[b + 1] = off[b] + lengths[b];
  long total = off[ntubes];
  int status = ORC_OK;
  long long faces = 0, iters = 0, fallbacks = 0, mlp = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : faces, iters, fallbacks, mlp)
#endif
  for (int b = 0; b < ntubes; ++b) {
    int nb = lengths[b];
    std::vector<double> xf(nb + 1);
    for (int i = 0; i <= nb; ++i) xf[i] = (double)i / nb;
    int nn[3] = {nb, 1, 1};
    int bcs[6] = {ORC_TRANSMISSIVE, ORC_TRANSMISSIVE, 0, 0, 0, 0};
    orc_t h = nullptr;
    orc_create(1, nn, xf.data(), bcs, ORC_CARTESIAN, gamma, 0, riemann, limiter_kind, &h);
    orc_set_guess(h, guess, mlp_weights);
    std::vector<double> u(3 * (size_t)nb);
    for (int v = 0; v < 3; ++v)
      for (int i = 0; i < nb; ++i) u[(size_t)v * nb + i] = U[(size_t)v * total + off[b] + i];
    orc_set_state(h, u.data());
    int st = ORC_OK;
    for (int k = 0; k < nsteps && st == ORC_OK; ++k) {
      double dt;
      st = orc_cfl_dt(h, cfl, &dt);
      if (st == ORC_OK) st = orc_step(h, dt);
    }
    if (st != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
      status = st;
    }
    orc_get_state(h, u.data());
    for (int v = 0; v < 3; ++v)
      for (int i = 0; i < nb; ++i) U[(size_t)v * total + off[b] + i] = u[(size_t)v * nb + i];
    faces += h->s.st_faces;
    iters += h->s.st_iters;
    fallbacks += h->s.st_fallback;
    mlp += h->s.st_mlp;
    orc_destroy(h);
  }
  if (stats_out) {
    stats_out[0] = faces;
    stats_out[1] = iters;
    stats_out[2] = fallbacks;
    stats_out[3] = mlp;
  }
  return status;
}

double orc_limiter(int kind, double dm, double dp) { return limiter(kind, dm, dp); }

int orc_flux_1d(int riemann, double gamma, int n_scalars, int dim, const double* UL,
                const double* UR, double* F) {
  /* Riemann flux through a face normal to axis 0 from conserved states. */
  Eos eos = {gamma, dim, n_scalars};
  double WL[16], WR[16];
  cons_to_prim(eos, UL, WL);
  cons_to_prim(eos, UR, WR);
  if (riemann == ORC_HLL) flux_hll(eos, WL, WR, 0, F);
  else if (riemann == ORC_HLLC) flux_hllc(eos, WL, WR, 0, F);
  else {
    ExactStats st;
    return flux_exact(eos, WL, WR, 0, ORC_GUESS_TORO, nullptr, F, &st);
  }
  return ORC_OK;
}

int orc_exact_star(double gamma, const double* WL, const double* WR, int guess,
                   const float* mlp_weights, double* pstar, double* ustar, int* iters) {
  ExactResult r = exact_star(gamma, WL, WR, guess, mlp_weights);
  *pstar = r.pstar;
  *ustar = r.ustar;
  *iters = r.iters;
  return r.status;
}

int orc_exact_sample(double gamma, const double* WL, const double* WR, double xi, double* W) {
  ExactResult r = exact_star(gamma, WL, WR, ORC_GUESS_TORO, nullptr);
  if (r.status != ORC_OK) return r.status;
  int side;
  exact_sample(gamma, WL, WR, r.pstar, r.ustar, xi, W, &side);
  return ORC_OK;
}

double orc_guess_toro(double gamma, const double* WL, const double* WR, int* kind) {
  return toro_guess(gamma, WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], kind);
}

int orc_mlp_features(double gamma, const double* WL, const double* WR, double* x6, double* pref) {
  mlp_features(gamma, WL, WR, x6, pref);
  return ORC_OK;
}

int orc_mlp_forward(const float* w, const double* x6, long n, double* y) {
  double z1[64], h1[64], z2[64], h2[64];
  for (long s = 0; s < n; ++s) y[s] = mlp_eval(w, x6 + 6 * s, z1, h1, z2, h2);
  return ORC_OK;
}

double orc_mlp_loss_grad(const float* w, const double* x6, const double* t, long n, double* grad) {
  /* Mean-squared error L = (1/n) sum (y - t)^2 and its gradient by
   * reverse-mode differentiation of the three layers. */
  for (int p = 0; p < MLP_NPARAM; ++p) grad[p] = 0.0;
  double loss = 0.0;
  double z1[64], h1[64], z2[64], h2[64], g2[64], g1[64];
  for (long s = 0; s < n; ++s) {
    const double* x = x6 + 6 * s;
    double y = mlp_eval(w, x, z1, h1, z2, h2);
    double r = y - t[s];
    loss += r * r;
    double gy = 2.0 * r / n;
    grad[OFF_B3] += gy;
    for (int i = 0; i < MLP_H; ++i) {
      grad[OFF_W3 + i] += gy * h2[i];
      g2[i] = gy * w[OFF_W3 + i] * dsilu(z2[i]);
    }
    for (int o = 0; o < MLP_H; ++o) {
      grad[OFF_B2 + o] += g2[o];
      for (int i = 0; i < MLP_H; ++i) grad[OFF_W2 + o * MLP_H + i] += g2[o] * h1[i];
    }
    for (int i = 0; i < MLP_H; ++i) {
      double a = 0.0;
      for (int o = 0; o < MLP_H; ++o) a += g2[o] * w[OFF_W2 + o * MLP_H + i];
      g1[i] = a * dsilu(z1[i]);
    }
    for (int o = 0; o < MLP_H; ++o) {
      grad[OFF_B1 + o] += g1[o];
      for (int i = 0; i < MLP_IN; ++i) grad[OFF_W1 + o * MLP_IN + i] += g1[o] * x[i];
    }
  }
  return loss / n;
}

int orc_adam_step(float* w, float* m, float* v, const double* grad, int nparam, int step,
                  double lr, double b1, double b2, double eps) {
  /* Adam (Kingma & Ba 2015), bias-corrected moments. */
  double c1 = 1.0 - std::pow(b1, step), c2 = 1.0 - std::pow(b2, step);
  for (int p = 0; p < nparam; ++p) {
    double mm = b1 * m[p] + (1.0 - b1) * grad[p];
    double vv = b2 * v[p] + (1.0 - b2) * grad[p] * grad[p];
    m[p] = (float)mm;
    v[p] = (float)vv;
    w[p] = (float)(w[p] - lr * (mm / c1) / (std::sqrt(vv / c2) + eps));
  }
  return ORC_OK;
}

double orc_sedov_xi0(double gamma) {
  /* Sedov-Taylor constant of Eq. 25, d_sh = xi0 (E t^2/rho0)^(1/5), for a
   * spherical point blast.  With u = Rdot U(xi), rho = rho0 D(xi),
   * p = rho0 Rdot^2 P(xi), xi = r/R, R ~ t^(2/5), the Euler equations reduce to
   *   (U-xi) D' + D (U' + 2U/xi) = 0
   *   (U-xi) U' + P'/D = 3U/2
   *   (U-xi)(P'/P - gamma D'/D) = 3
   * with strong-shock values at xi = 1.  Integrate inward (RK4) and use the
   * energy integral E = (16 pi/25) rho0 R^5/t^2 * I,
   * I = int_0^1 (D U^2/2 + P/(gamma-1)) xi^2 dxi, so xi0 = (25/(16 pi I))^(1/5). */
  double g = gamma;
  auto rhs = [g](double xi, const double* y, double* dy) {
    double D = y[0], Uu = y[1], P = y[2];
    double a = Uu - xi;
    double dU = (1.5 * Uu * a * D - 3.0 * P + 2.0 * g * P * Uu / xi) / (a * a * D - g * P);
    double dD = -D * (dU + 2.0 * Uu / xi) / a;
    double dP = 3.0 * P / a + g * P * dD / D;
    dy[0] = dD;
    dy[1] = dU;
    dy[2] = dP;
  };
  double y[3] = {(g + 1.0) / (g - 1.0), 2.0 / (g + 1.0), 2.0 / (g + 1.0)};
  const int NSTEP = 200000;
  double xi = 1.0, xi_end = 1e-6;
  double hstep = (xi_end - xi) / NSTEP;
  auto integrand = [g](double x, const double* yy) {
    return (0.5 * yy[0] * yy[1] * yy[1] + yy[2] / (g - 1.0)) * x * x;
  };
  double I = 0.0;
  for (int s = 0; s < NSTEP; ++s) {
    double k1[3], k2[3], k3[3], k4[3], yt[3];
    double f0 = integrand(xi, y);
    rhs(xi, y, k1);
    for (int q = 0; q < 3; ++q) yt[q] = y[q] + 0.5 * hstep * k1[q];
    rhs(xi + 0.5 * hstep, yt, k2);
    for (int q = 0; q < 3; ++q) yt[q] = y[q] + 0.5 * hstep * k2[q];
    rhs(xi + 0.5 * hstep, yt, k3);
    for (int q = 0; q < 3; ++q) yt[q] = y[q] + hstep * k3[q];
    rhs(xi + hstep, yt, k4);
    for (int q = 0; q < 3; ++q) y[q] += hstep / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
    xi += hstep;
    double f1 = integrand(xi, y);
    I += 0.5 * (f0 + f1) * (-hstep);  // trapezoid, integrating from xi_end up to 1
  }
  return std::pow(25.0 / (16.0 * PI * I), 0.2);
}

double orc_heating_rate(int heating, const double* heat_params, double t, double rho_f_ni) {
  double prm[4] = {0, 0, 0, 0};
  if (heat_params)
    for (int i = 0; i < 4; ++i) prm[i] = heat_params[i];
  return heating_rate(heating, prm, t, rho_f_ni);
}

}  // extern "C"
