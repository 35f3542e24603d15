"""Pins of the oracle's gas + radiation EoS (Sect. 2.3, Eq. 6-7).

- The temperature solve: the returned T satisfies Eq. 6 and both inversions
  (from e, from P) agree, over six decades of P_rad/P_gas.
- Limits: no radiation (a = 0) is the ideal gas of Eq. 5, state for state and
  step for step; radiation-dominated states have P -> e/3 and c^2 -> (4/3) P/rho.
- The sound speed of Eq. 7 equals sqrt(dP/drho) along an adiabat of the
  EoS, integrated independently (d e = (e + P) d rho / rho, RK4).
- A stationary contact (pressure equilibrium, different temperatures) stays
  exactly at rest under HLLC; a periodic box conserves mass, momentum and
  energy to roundoff.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl

G = 5.0 / 3.0


@pytest.mark.parametrize("alpha_target", [1e-6, 1e-2, 1.0, 1e2, 1e6])
def test_temperature_solves_eq6_and_inversions_agree(alpha_target):
    R, a, rho = 1.0, 1.0, 0.7
    # pick T so that P_rad/P_gas = alpha_target: a T^3 / (3 rho R) = alpha
    T0 = (3.0 * rho * R * alpha_target / a) ** (1.0 / 3.0)
    e0 = rho * R * T0 / (G - 1.0) + a * T0 ** 4
    T, P, c = O.eos_rad(G, R, a, rho, e0)
    assert abs(T - T0) <= 1e-13 * T0
    assert abs(P - (rho * R * T0 + a * T0 ** 4 / 3.0)) <= 1e-13 * P
    T2, e2 = O.eos_rad_eint(G, R, a, rho, P)
    assert abs(T2 - T0) <= 1e-13 * T0 and abs(e2 - e0) <= 1e-13 * e0


def test_no_radiation_is_the_ideal_gas():
    for rho, e in [(1.0, 2.5), (0.125, 0.25), (3.0, 1e-6), (1e-4, 7.0)]:
        T, P, c = O.eos_rad(1.4, 2.0, 0.0, rho, e)
        assert abs(P - 0.4 * e) <= 1e-15 * P
        assert abs(c - math.sqrt(1.4 * P / rho)) <= 1e-15 * c
    # a Sod step with the radiation EoS at a = 0 equals the ideal-gas step
    case = wl.sod(200)
    ideal = O.solver_from_case(case)
    rad = O.solver_from_case(dict(case, eos_rad=(1.0, 0.0)))
    for _ in range(20):
        dt = ideal.cfl_dt(0.8)
        assert abs(rad.cfl_dt(0.8) - dt) <= 1e-14 * dt
        ideal.step(dt)
        rad.step(dt)
    A, B = ideal.get_state(), rad.get_state()
    assert np.abs(A - B).sum() <= 1e-13 * np.abs(A).sum()


def test_radiation_dominated_limit():
    R, a, rho = 1.0, 1.0, 1e-9
    e = 10.0
    T, P, c = O.eos_rad(G, R, a, rho, e)
    assert abs(P - e / 3.0) <= 1e-7 * P
    assert abs(c * c - 4.0 / 3.0 * P / rho) <= 1e-7 * c * c


def _adiabat_c2(R, a, rho, e, h=1e-3):
    """dP/drho along the adiabat through (rho, e), by RK4 in ln rho and a
    five-point derivative (independent of Eq. 7)."""
    def de(r, ee):
        return (ee + O.eos_rad(G, R, a, r, ee)[1]) / r

    def step(r, ee, dr, n=40):
        hh = dr / n
        for _ in range(n):
            k1 = de(r, ee)
            k2 = de(r + hh / 2, ee + hh / 2 * k1)
            k3 = de(r + hh / 2, ee + hh / 2 * k2)
            k4 = de(r + hh, ee + hh * k3)
            ee += hh / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            r += hh
        return ee

    P = []
    for k in (-2, -1, 1, 2):
        r = rho * (1 + k * h)
        P.append(O.eos_rad(G, R, a, r, step(rho, e, r - rho))[1])
    dr = rho * h
    return (P[0] - 8 * P[1] + 8 * P[2] - P[3]) / (12 * dr)


@pytest.mark.parametrize("e", [0.3, 3.0, 30.0, 300.0])
def test_sound_speed_is_the_adiabatic_derivative(e):
    R, a, rho = 1.0, 1.0, 0.5
    T, P, c = O.eos_rad(G, R, a, rho, e)
    assert abs(_adiabat_c2(R, a, rho, e) - c * c) <= 1e-8 * c * c


def _contact_tube(n=64):
    """Pressure equilibrium, rho 1 | 0.2, at rest: the temperatures differ."""
    R, a = 1.0, 1.0
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.5, 1.0, 0.2)
    P = 2.0
    e = np.array([O.eos_rad_eint(G, R, a, r, P)[1] for r in rho])
    U = np.stack([rho, np.zeros(n), e])
    case = dict(dim=1, n=[n, 1, 1], faces=[np.linspace(0, 1, n + 1)], bc=[(wl.PERIODIC, wl.PERIODIC)],
                coords=wl.CARTESIAN, gamma=G, n_scalars=0, riemann=wl.HLLC, limiter=wl.MINMOD,
                sources=None, U=U.reshape(3, 1, 1, n), eos_rad=(R, a))
    return case


def test_stationary_contact_is_kept_by_hllc():
    case = _contact_tube()
    s = O.solver_from_case(case)
    U0 = s.get_state()
    for _ in range(10):
        s.step(0.5 * s.cfl_dt(0.8))
    U = s.get_state()
    assert np.max(np.abs(U[1])) <= 1e-13
    assert np.max(np.abs(U - U0)) <= 1e-12 * np.max(np.abs(U0))


def test_periodic_box_conserves_totals():
    case = wl.smooth_random(2, [24, 20], 0, seed=4, riemann=wl.HLLC)
    case = dict(case, eos_rad=(1.0, 0.5))
    s = O.solver_from_case(case)
    t0 = s.totals()
    for _ in range(30):
        s.step(s.cfl_dt(0.4))
    t1 = s.totals()
    scale = np.abs(t0).max()
    assert np.max(np.abs(t1 - t0)) <= 1e-13 * scale
