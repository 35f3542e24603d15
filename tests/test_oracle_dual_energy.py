"""Pins of the oracle's dual-energy correction (Sect. 2.5).

- Off (eps = 0), or where every cell has e >= eps e_k, the step is the plain
  step bit for bit (alpha = 1 leaves the total energy untouched).
- Hypersonic uniform-pressure advection (Mach ~ 800): the exact solution keeps
  P and u fixed.  With the correction in force (alpha = 0) the pressure stays
  at its value to roundoff, as the paper intends; mass and momentum remain
  conserved to roundoff with it.
- In the blend band eps e_k/10 < e < eps e_k the result lies between the two
  estimates: the step with the correction differs from both pure forms.
"""
import numpy as np

import oracle as O
from paper_2503_04428_gb300 import workloads as wl


def _advection(n=128, u=1000.0, p=1.0):
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * x)
    U = wl.conserved(1.4, rho, [np.full(n, u)], np.full(n, p))
    return dict(name="adv", dim=1, n=[n, 1, 1], faces=[np.linspace(0, 1, n + 1)],
                bc=[(wl.PERIODIC, wl.PERIODIC)], coords=wl.CARTESIAN, gamma=1.4, n_scalars=0,
                riemann=wl.HLLC, limiter=wl.VANLEER, cfl=0.4, sources=None, U=U.reshape(3, 1, 1, n))


def _pressure(U, g=1.4):
    return (g - 1.0) * (U[2] - 0.5 * U[1] ** 2 / U[0])


def test_off_or_subsonic_is_the_plain_step():
    case = wl.smooth_random(2, [30, 24], 1, seed=3)
    a = O.solver_from_case(case)
    b = O.solver_from_case(dict(case, dual_energy=1e-6))
    for _ in range(5):
        dt = a.cfl_dt(0.4)
        a.step(dt)
        b.step(dt)
    assert np.array_equal(a.get_state(), b.get_state())


def test_hypersonic_advection_keeps_pressure():
    """P and u stay at their values to the precision with which E ~ rho u^2/2
    (5e5 here) can hold P = 1: a few units in the last place of E."""
    case = _advection()
    s = O.solver_from_case(dict(case, dual_energy=1.0))
    t0 = s.totals()
    for _ in range(100):
        s.step(s.cfl_dt(0.4))
    U = s.get_state()[:, 0, 0]
    ulp_e = np.spacing(U[2].max()) * 0.4
    assert np.max(np.abs(_pressure(U) - 1.0)) <= 8 * ulp_e
    assert np.max(np.abs(U[1] / U[0] - 1000.0)) < 1e-10
    t1 = s.totals()
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0]) and abs(t1[1] - t0[1]) <= 1e-13 * abs(t0[1])


def test_internal_energy_equation_closed_form():
    """With first-order states and every face supersonic to the right, the face
    quantities are those of the left cell, and with alpha = 0 the internal
    energy obeys e_i' = e + dt/dx (e + P)(u_{i-1} - u_i) for uniform rho, P."""
    n = 64
    x = (np.arange(n) + 0.5) / n
    u = 20.0 + 3.0 * np.sin(2 * np.pi * x)
    U = wl.conserved(1.4, np.ones(n), [u], np.ones(n))
    case = dict(name="div", dim=1, n=[n, 1, 1], faces=[np.linspace(0, 1, n + 1)],
                bc=[(wl.PERIODIC, wl.PERIODIC)], coords=wl.CARTESIAN, gamma=1.4, n_scalars=0,
                riemann=wl.HLLC, limiter=wl.FIRST_ORDER, cfl=0.4, sources=None,
                U=U.reshape(3, 1, 1, n), dual_energy=1.0)
    s = O.solver_from_case(case)
    dt = 0.2 * s.cfl_dt(0.4)
    s.step(dt)
    V = s.get_state()[:, 0, 0]
    e_new = V[2] - 0.5 * V[1] ** 2 / V[0]
    e_expect = 2.5 + dt * n * 3.5 * (np.roll(u, 1) - u)
    assert np.max(np.abs(e_new - e_expect)) < 1e-11


def test_blend_band_lies_between_the_two_estimates():
    # e / e_k ~ 5e-3 * ... choose eps so that eps e_k/10 < e < eps e_k in every cell
    case = _advection(n=64, u=30.0, p=1.0)  # e = 2.5, e_k = rho * 450 in [225, 675]
    eps = 0.02                              # eps e_k in [4.5, 13.5], a tenth in [0.45, 1.35]
    plain = O.solver_from_case(case)
    full = O.solver_from_case(dict(case, dual_energy=1e3))   # alpha = 0 everywhere
    blend = O.solver_from_case(dict(case, dual_energy=eps))
    dt = plain.cfl_dt(0.4)
    for s in (plain, full, blend):
        s.step(dt)
    e = [s.get_state()[2, 0, 0] - 0.5 * s.get_state()[1, 0, 0] ** 2 / s.get_state()[0, 0, 0]
         for s in (plain, full, blend)]
    lo, hi = np.minimum(e[0], e[1]), np.maximum(e[0], e[1])
    assert np.all(e[2] >= lo - 1e-12) and np.all(e[2] <= hi + 1e-12)
    assert not np.array_equal(e[2], e[0]) and not np.array_equal(e[2], e[1])
