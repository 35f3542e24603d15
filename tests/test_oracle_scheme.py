"""Pins of the oracle's full time step (HERACLES++ Sect. 3.2, Eq. 17-19) against
exact solutions, closed forms, conservation, symmetry and the spherical
source terms (Eq. 13-16)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _run(s, t_end, cfl, max_steps=100000):
    t = 0.0
    k = 0
    while t < t_end * (1 - 1e-14) and k < max_steps:
        dt = min(s.cfl_dt(cfl), t_end - t)
        s.step(dt)
        t += dt
        k += 1
    return k


def _sod_l1(n, riemann=O.HLLC, limiter=O.MINMOD):
    case = wl.sod(n, riemann=riemann, limiter=limiter)
    s = O.solver_from_case(case)
    _run(s, 0.2, 0.8)
    rho = s.get_state()[0, 0, 0]
    x = 0.5 * (case["faces"][0][1:] + case["faces"][0][:-1])
    ex = np.array([O.exact_sample(1.4, [1, 0, 1], [0.125, 0, 0.1], (xx - 0.5) / 0.2)[0] for xx in x])
    return np.mean(np.abs(rho - ex))


def test_sod_converges_to_exact_solution():
    e = [_sod_l1(n) for n in (100, 200, 400)]
    assert e[0] < 0.01
    assert e[1] < e[0] and e[2] < e[1]
    order = math.log(e[0] / e[2], 4.0)
    assert 0.5 < order < 1.2  # discontinuities limit the order to about one


@pytest.mark.parametrize("riemann", [O.HLL, O.EXACT])
def test_sod_other_solvers(riemann):
    assert _sod_l1(200, riemann=riemann) < 0.01


def test_smooth_advection_second_order():
    errs = []
    for n in (32, 64, 128):
        case = wl.advection1d(n, limiter=O.VANLEER)
        s = O.solver_from_case(case)
        _run(s, 1.0, 0.4)
        x = 0.5 * (case["faces"][0][1:] + case["faces"][0][:-1])
        # exact: translated by one period; cell averages of 1 + 0.2 sin(2 pi x)
        xf = case["faces"][0]
        ex = 1.0 - 0.2 * (np.cos(2 * math.pi * xf[1:]) - np.cos(2 * math.pi * xf[:-1])) / (2 * math.pi * (xf[1:] - xf[:-1]))
        errs.append(np.mean(np.abs(s.get_state()[0, 0, 0] - ex)))
        del x
    o1 = math.log2(errs[0] / errs[1])
    o2 = math.log2(errs[1] / errs[2])
    assert o2 > 1.6 and o1 > 1.4, errs


def test_periodic_conservation_kh():
    case = wl.kh2d(32, 64)
    s = O.solver_from_case(case)
    T0 = s.totals()
    for _ in range(60):
        s.step(s.cfl_dt(0.4))
    T1 = s.totals()
    scale = np.abs(T0) + np.abs(T1).max()
    assert np.all(np.abs(T1 - T0) <= 1e-13 * scale), (T1 - T0) / scale


@pytest.mark.parametrize("bc", [O.PERIODIC, O.TRANSMISSIVE, O.REFLECTIVE])
def test_uniform_state_is_steady(bc):
    n = 12
    f = np.linspace(0, 1, n + 1)
    s = O.Solver(3, [n, n, n], [f, f, f], [(bc, bc)] * 3, O.CARTESIAN, 1.4, 1, O.HLLC, O.VANLEER)
    U = wl.conserved(1.4, np.ones((n, n, n)), [np.zeros((n, n, n))] * 3, np.ones((n, n, n)),
                     [np.full((n, n, n), 0.3)])
    s.set_state(U)
    s.step(0.01)
    assert np.abs(s.get_state() - U).max() < 1e-15


def test_liska_wendroff_mirror_symmetry():
    case = wl.liska_wendroff(32)
    s = O.solver_from_case(case)
    for _ in range(25):
        s.step(s.cfl_dt(0.4))
    U = s.get_state()[:, 0]
    # mirror x <-> z: rho and E transpose, momenta swap
    assert np.abs(U[0] - U[0].T).max() < 1e-12
    assert np.abs(U[3] - U[3].T).max() < 1e-12 * np.abs(U[3]).max()
    assert np.abs(U[1] - U[2].T).max() < 1e-12 * (np.abs(U[1]).max() + 1e-300)


def test_uniform_gravity_closed_form():
    """Uniform gas, periodic box, uniform g: m_n = n dt rho g, E_n = E0 + rho g^2 dt^2 n(n-1)/2."""
    n = 8
    f = np.linspace(0, 1, n + 1)
    s = O.Solver(2, [n, n], [f, f], [(O.PERIODIC, O.PERIODIC)] * 2, O.CARTESIAN, 1.4, 0, O.HLLC, O.MINMOD)
    rho, p, g, dt = 1.3, 2.0, -0.7, 1e-3
    U = wl.conserved(1.4, np.full((n, n), rho), [np.zeros((n, n))] * 2, np.full((n, n), p))
    s.set_state(U)
    s.set_sources(O.GRAV_UNIFORM, g0=(0.0, g, 0.0))
    E0 = U[3].mean()
    N = 20
    for _ in range(N):
        s.step(dt)
    V = s.get_state()[:, 0]
    assert np.abs(V[2] - N * dt * rho * g).max() < 1e-13
    assert np.abs(V[1]).max() < 1e-14
    assert np.abs(V[3] - (E0 + rho * g * g * dt * dt * N * (N - 1) / 2)).max() < 1e-12


def test_constant_heating_closed_form():
    n = 6
    f = np.linspace(0, 1, n + 1)
    s = O.Solver(1, [n], [f], [(O.PERIODIC, O.PERIODIC)], O.CARTESIAN, 1.4, 0, O.HLLC, O.MINMOD)
    U = wl.conserved(1.4, np.ones(n), [np.zeros(n)], np.ones(n))
    s.set_state(U)
    s.set_sources(heating=O.HEAT_CONST, heat_params=(0.25,))
    for _ in range(10):
        s.step(0.01)
    assert np.abs(s.get_state()[2, 0, 0] - (U[2] + 10 * 0.01 * 0.25)).max() < 1e-14


def test_ni56_heating_rate_physics():
    """Eq. 8-9: at t=0 only Ni decays; integrated over all time each Ni nucleus
    releases Q_Ni + Q_Co (per 56 m_u of Ni mass)."""
    from scipy.integrate import quad
    m_u, MeV, day = 1.66053906660e-24, 1.602176634e-6, 86400.0
    rf = 1e-10
    r0 = O.heating_rate(O.HEAT_NI56, (0,), 0.0, rf)
    assert abs(r0 - rf * 1.75 * MeV / (56 * m_u * 8.8 * day)) < 1e-12 * r0
    tot, _ = quad(lambda t: O.heating_rate(O.HEAT_NI56, (0,), t, rf), 0, 5000 * day, limit=400)
    assert abs(tot - rf * (1.75 + 3.73) * MeV / (56 * m_u)) < 1e-6 * tot


def test_ni56_heating_in_the_step():
    n = 4
    f = np.linspace(0, 1, n + 1)
    s = O.Solver(1, [n], [f], [(O.PERIODIC, O.PERIODIC)], O.CARTESIAN, 5 / 3, 1, O.HLLC, O.MINMOD)
    U = wl.conserved(5 / 3, np.full(n, 1e-9), [np.zeros(n)], np.full(n, 1e-3), [np.full(n, 0.1)])
    s.set_state(U)
    s.set_sources(heating=O.HEAT_NI56, heat_params=(0,))
    t0, dt = 86400.0 * 3, 60.0
    s.set_time(t0)
    s.step(dt)
    expect = U[2] + dt * O.heating_rate(O.HEAT_NI56, (0,), t0, 1e-10)
    assert np.abs(s.get_state()[2, 0, 0] - expect).max() < 1e-13 * np.abs(expect).max()


def test_cfl_closed_form():
    n = 10
    fx = np.linspace(0, 2, n + 1)
    fy = np.linspace(0, 1, n + 1)
    s = O.Solver(2, [n, n], [fx, fy], [(O.PERIODIC, O.PERIODIC)] * 2, O.CARTESIAN, 1.4, 0, O.HLLC, O.MINMOD)
    rho, u, v, p = 2.0, 0.5, -0.25, 3.0
    s.set_state(wl.conserved(1.4, np.full((n, n), rho), [np.full((n, n), u), np.full((n, n), v)], np.full((n, n), p)))
    c = math.sqrt(1.4 * p / rho)
    expect = 0.4 / ((abs(u) + c) / 0.2 + (abs(v) + c) / 0.1)
    assert abs(s.cfl_dt(0.4) - expect) < 1e-14 * expect


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_spherical_static_uniform_state(dim):
    case = wl.sphere_state(8, 6, 5, uniform=True, dim=dim, n_scalars=1)
    s = O.solver_from_case(case)
    U0 = s.get_state()
    for _ in range(3):
        s.step(0.01)
    assert np.abs(s.get_state() - U0).max() < 1e-14


def test_spherical_angular_momentum_conserved():
    """L_z = sum r_i s_j (rho u_phi) dV telescopes under the Eq. 14 weights."""
    case = wl.sphere_state(10, 8, 12, rotating=True)
    s = O.solver_from_case(case)
    rf, tf, pf = case["faces"]
    rc = 0.5 * (rf[1:] + rf[:-1])
    sc = 0.5 * (np.sin(tf[1:]) + np.sin(tf[:-1]))
    dV = ((rf[1:] ** 3 - rf[:-1] ** 3) / 3)[None, None, :] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :, None] \
        * (pf[1:] - pf[:-1])[:, None, None]
    w = rc[None, None, :] * sc[None, :, None] * dV

    def Lz():
        return float(np.sum(w * s.get_state()[3]))
    L0 = Lz()
    for _ in range(30):
        s.step(s.cfl_dt(0.4))
    assert abs(Lz() - L0) < 1e-13 * abs(L0)
    # and the radial momentum is NOT conserved (geometric sources act)
    assert abs(np.sum(s.get_state()[1] * dV)) > 1e-6


def test_wedge_equals_1d_spherical_for_radial_flow():
    """A 3D wedge with purely radial structure evolves like the 1D spherical run."""
    nr = 24
    rf = np.linspace(0.5, 2.0, nr + 1)
    rc = 0.5 * (rf[1:] + rf[:-1])
    rho = 1.0 + 0.5 * np.exp(-((rc - 1.2) / 0.2) ** 2)
    p = 1.0 + 1.0 * np.exp(-((rc - 1.0) / 0.15) ** 2)
    U1 = wl.conserved(1.4, rho, [np.zeros(nr)], p)
    s1 = O.Solver(1, [nr], [rf], [(O.REFLECTIVE, O.TRANSMISSIVE)], O.SPHERICAL, 1.4, 0, O.HLLC, O.MINMOD)
    s1.set_state(U1)
    nt, npf = 6, 5
    tf = np.linspace(1.2, 1.9, nt + 1)
    pf = np.linspace(0.0, 0.6, npf + 1)
    sh = (npf, nt, nr)
    U3 = wl.conserved(1.4, np.broadcast_to(rho, sh), [np.zeros(sh)] * 3, np.broadcast_to(p, sh))
    s3 = O.Solver(3, [nr, nt, npf], [rf, tf, pf], [(O.REFLECTIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                                                   (O.REFLECTIVE, O.REFLECTIVE)], O.SPHERICAL, 1.4, 0, O.HLLC, O.MINMOD)
    s3.set_state(U3)
    for _ in range(10):
        dt = s1.cfl_dt(0.4)
        s1.step(dt)
        s3.step(dt)
    A, B = s1.get_state(), s3.get_state()
    for k in range(npf):
        for j in range(nt):
            assert np.abs(B[0, k, j] - A[0, 0, 0]).max() < 1e-12
            assert np.abs(B[1, k, j] - A[1, 0, 0]).max() < 1e-12
            assert np.abs(B[4, k, j] - A[2, 0, 0]).max() < 1e-12
    assert np.abs(B[2]).max() < 1e-12 and np.abs(B[3]).max() < 1e-12


def test_monopole_enclosed_mass_closed_form():
    """Cell densities chosen so that each full-sphere shell holds 4 pi rho0 dr:
    M_i = Mc + 4 pi rho0 (r_i- - r_in + dr_i/2)."""
    nr, nt = 12, 4
    rf = np.geomspace(1.0, 10.0, nr + 1)
    tf = np.linspace(1.0, 2.0, nt + 1)
    rho0, Mc = 0.7, 2.5
    rho = rho0 * (rf[1:] - rf[:-1]) / ((rf[1:] ** 3 - rf[:-1] ** 3) / 3)
    sh = (1, nt, nr)
    U = wl.conserved(1.4, np.broadcast_to(rho, sh)[0], [np.zeros(sh[1:])] * 2, np.ones(sh[1:]))
    s = O.Solver(2, [nr, nt], [rf, tf], [(O.REFLECTIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE)],
                 O.SPHERICAL, 1.4, 0, O.HLLC, O.MINMOD)
    s.set_state(U)
    s.set_sources(O.GRAV_POINT_MONOPOLE, G=1.0, Mc=Mc)
    M = s.shell_mass()
    expect = Mc + 4 * math.pi * rho0 * (rf[:-1] - rf[0] + 0.5 * (rf[1:] - rf[:-1]))
    assert np.abs(M - expect).max() < 1e-13 * expect.max()


def test_sedov_constant_quadrature():
    for line in open(os.path.join(GOLD, "sedov_xi0.txt")):
        if line.startswith("#"):
            continue
        g, xi, tol = map(float, line.split())
        assert abs(O.sedov_xi0(g) - xi) < tol


def test_sedov_1d_spherical_shock_radius():
    """App. C.4 setup: the shock radius follows Eq. 25 with xi0(1.4)."""
    case = wl.sedov1d_spherical(200)
    s = O.solver_from_case(case)
    t_end = 0.5
    _run(s, t_end, 0.4)
    rho = s.get_state()[0, 0, 0]
    rf = case["faces"][0]
    rc = 0.5 * (rf[1:] + rf[:-1])
    r_shock = rc[np.argmax(rho)]
    r_exact = O.sedov_xi0(1.4) * (t_end ** 2) ** 0.2
    assert abs(r_shock - r_exact) < 4 * (rf[1] - rf[0]), (r_shock, r_exact)
    assert rho.max() > 2.5  # compression toward (g+1)/(g-1) = 6


def test_fallback_keeps_state_positive():
    """A strong rarefaction into near-vacuum triggers the first-order fallback
    and the state stays physical."""
    n = 64
    f = np.linspace(0, 1, n + 1)
    x = 0.5 * (f[1:] + f[:-1])
    u = np.where(x < 0.5, -2.5, 2.5)
    s = O.Solver(1, [n], [f], [(O.TRANSMISSIVE, O.TRANSMISSIVE)], O.CARTESIAN, 1.4, 0, O.HLL, O.VANLEER)
    s.set_state(wl.conserved(1.4, np.ones(n), [u], np.full(n, 0.4)))
    for _ in range(20):
        s.step(s.cfl_dt(0.5))
    W = s.get_state()[:, 0, 0]
    assert np.all(W[0] > 0)


def test_spherical_closed_wedge_conserves_mass_and_energy():
    """Reflective r/theta walls and periodic phi: nothing crosses the boundary."""
    case = wl.sphere_state(10, 8, 12, rotating=True, n_scalars=1)
    s = O.solver_from_case(case)
    T0 = s.totals()
    for _ in range(30):
        s.step(s.cfl_dt(0.4))
    T1 = s.totals()
    for v in (0, 4, 5):  # mass, energy, scalar
        assert abs(T1[v] - T0[v]) < 1e-13 * abs(T0[v])


def test_point_gravity_closed_form():
    """Static uniform gas on a spherical wedge with a point mass: after one step
    the flux differences and the pressure source cancel, so m_r = -dt rho G Mc/r_i^2
    and the energy is unchanged (u = 0 at t^n)."""
    case = wl.sphere_state(12, 5, 4, uniform=True, dim=3, r_range=(2.0, 5.0))
    s = O.solver_from_case(case)
    s.set_sources(O.GRAV_POINT, G=0.3, Mc=7.0)
    dt = 1e-3
    s.step(dt)
    rf = case["faces"][0]
    rc = 0.5 * (rf[1:] + rf[:-1])
    U = s.get_state()
    expect = -dt * 1.0 * 0.3 * 7.0 / rc ** 2
    assert np.abs(U[1] - expect[None, None, :]).max() < 1e-13
    assert np.abs(U[4] - case["U"][4]).max() < 1e-13


def test_totals_of_uniform_state_equal_wedge_volume():
    """sum U dV of a uniform state = value x exact volume of the wedge."""
    r0, r1, t0, t1, p0, p1 = 1.0, 3.0, 0.6, 2.4, 0.0, 2 * math.pi
    case = wl.sphere_state(9, 7, 5, uniform=True, dim=3, r_range=(r0, r1), th_range=(t0, t1), ph_range=(p0, p1))
    s = O.solver_from_case(case)
    vol = (r1 ** 3 - r0 ** 3) / 3 * (math.cos(t0) - math.cos(t1)) * (p1 - p0)
    T = s.totals()
    assert abs(T[0] - vol) < 1e-13 * vol
    assert abs(T[4] - vol / (5 / 3 - 1)) < 1e-13 * vol / (5 / 3 - 1)
