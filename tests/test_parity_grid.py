"""GPU grid path vs the FP64 oracle, element by element, one step at a time.

Bars per conserved component and step (tests/parity.py): FP64 relative L1
<= 1e-12 and element-wise max|B - A| <= 1e-11 of the component's scale;
FP32 relative L1 <= 2e-5 and element-wise <= 1e-4 (the oracle is given the
FP32-rounded input, so this measures the step's FP32 arithmetic; eps_32 =
6e-8 times the O(100) rounding steps on the path of one value).  Sizes span
several tiles with ragged tails along every axis and several z-chunks in 3D.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

from parity import ELEM_TOL, L1_TOL, check

TOL = L1_TOL


def rel_l1(A, B, dim, gamma=1.4):
    """Relative L1 error per conserved component (B against the oracle's A),
    on the scales of tests/parity.py."""
    from parity import errors
    return errors(A, B, dim, gamma)[0]


def step_compare(hydro_lib, case, precision, steps=1, tol=None, dt=None):
    H = hydro_lib
    if precision == 32:
        case = dict(case)
        case["U"] = case["U"].astype(np.float32).astype(np.float64)
    s = O.solver_from_case(case)
    g = H.Grid.from_case(case, precision)
    tol = TOL[precision] if tol is None else tol
    elem = ELEM_TOL[precision] * tol / TOL[precision]
    worst = 0.0
    for _ in range(steps):
        d = dt if dt is not None else s.cfl_dt(case["cfl"])
        s.step(d)
        g.step(d)
        A = s.get_state()
        B = g.get_state()
        err, _ = check(A, B, case["dim"], case["gamma"], precision, l1=tol, elem=elem, label=case["name"])
        worst = max(worst, err.max())
        if precision == 32:  # restart both from the oracle's state each step
            g.set_state(A.astype(np.float32))
            s.set_state(A.astype(np.float32).astype(np.float64))
    g.close()
    return worst


BCS = [(O.PERIODIC, O.PERIODIC), (O.TRANSMISSIVE, O.REFLECTIVE), (O.REFLECTIVE, O.TRANSMISSIVE)]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("riemann", [O.HLL, O.HLLC, O.EXACT])
@pytest.mark.parametrize("limiter", [O.FIRST_ORDER, O.MINMOD, O.VANLEER, O.VANALBADA])
def test_1d_matrix(hydro_lib, precision, riemann, limiter):
    for bi, bc in enumerate(BCS):
        ns = (bi + limiter) % 4
        case = wl.smooth_random(1, [600], ns, seed=3 + bi, bc=[bc], riemann=riemann, limiter=limiter)
        step_compare(hydro_lib, case, precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("riemann", [O.HLL, O.HLLC, O.EXACT])
def test_2d_matrix(hydro_lib, precision, riemann):
    for limiter in (O.MINMOD, O.VANLEER, O.VANALBADA):
        for ns in (0, 1, 3):
            bc = [BCS[(limiter + ns) % 3], BCS[(limiter + 2 * ns + 1) % 3]]
            case = wl.smooth_random(2, [70, 45], ns, seed=10 * limiter + ns, bc=bc, riemann=riemann,
                                    limiter=limiter)
            step_compare(hydro_lib, case, precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("riemann", [O.HLL, O.HLLC, O.EXACT])
@pytest.mark.parametrize("ns", [0, 1, 2, 3])
def test_3d_matrix(hydro_lib, precision, riemann, ns):
    bc = [BCS[ns % 3], BCS[(ns + 1) % 3], BCS[(ns + 2) % 3]]
    case = wl.smooth_random(3, [37, 23, 40], ns, seed=100 + ns, bc=bc, riemann=riemann,
                            limiter=[O.MINMOD, O.VANLEER, O.VANALBADA, O.MINMOD][ns])
    step_compare(hydro_lib, case, precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("riemann", [O.HLLC, O.EXACT, O.HLL])
def test_spherical(hydro_lib, precision, dim, riemann):
    case = wl.sphere_state(37, 21, 19, dim=dim, riemann=riemann, n_scalars=dim - 1)
    step_compare(hydro_lib, case, precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("gravity", [O.GRAV_POINT, O.GRAV_POINT_MONOPOLE])
def test_spherical_gravity(hydro_lib, precision, gravity):
    case = wl.sphere_state(40, 12, 10, dim=3, rotating=True, r_range=(1.0, 20.0), n_scalars=1,
                           bc=[(O.REFLECTIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                               (O.PERIODIC, O.PERIODIC)])
    case["sources"] = dict(gravity=gravity, G=0.01, Mc=2.0)
    step_compare(hydro_lib, case, precision, steps=3)


@pytest.mark.parametrize("precision", [64, 32])
def test_uniform_gravity_and_heating(hydro_lib, precision):
    case = wl.rt2d(40, 96, riemann=O.HLLC)
    step_compare(hydro_lib, case, precision, steps=3)
    case = wl.smooth_random(2, [33, 20], 1, seed=5)
    case["sources"] = dict(gravity=O.GRAV_UNIFORM, g0=(0.3, -0.2, 0.0), heating=O.HEAT_CONST,
                           heat_params=(0.05,))
    step_compare(hydro_lib, case, precision, steps=2)


def test_ni56_heating(hydro_lib):
    """Ni-56 decay heating (Eq. 8-9, CGS) in a 1D ejecta-like state."""
    n = 300
    case = wl.smooth_random(1, [n], 2, seed=8)
    x = np.linspace(0, 1, n)
    rho = 1e-9 * (1 + 0.3 * np.sin(6 * x))
    case["U"] = wl.conserved(5 / 3, rho, [1e5 * np.sin(4 * x)], 1e-3 * (1 + 0.2 * np.cos(5 * x)),
                             [np.full(n, 0.5), 0.1 + 0.05 * np.sin(3 * x)]).reshape(4 + 1, 1, 1, n)
    case["gamma"] = 5 / 3
    case["sources"] = dict(heating=O.HEAT_NI56, heat_params=(1,))
    s = O.solver_from_case(case)
    s.set_time(86400.0 * 5)
    g = hydro_lib.Grid.from_case(case, 64)
    g.set_time(86400.0 * 5)
    dt = s.cfl_dt(0.4)
    U0 = s.get_state()
    s.step(dt)
    g.step(dt)
    assert np.abs(s.get_state()[2] - U0[2]).max() > 1e-6 * np.abs(U0[2]).max()  # heating acts
    check(s.get_state(), g.get_state(), 1, 5 / 3, 64)


@pytest.mark.parametrize("precision", [64, 32])
def test_minimum_sizes(hydro_lib, precision):
    """n = 2 along an axis (the smallest allowed) and thin slabs."""
    for n, dim in (([2], 1), ([2, 2], 2), ([2, 3, 2], 3), ([65, 2], 2), ([2, 2, 33], 3)):
        case = wl.smooth_random(dim, n, 1, seed=sum(n),
                                bc=[BCS[d % 3] for d in range(dim)])
        step_compare(hydro_lib, case, precision, steps=2)


def test_device_dt_run_matches_oracle_sod(hydro_lib):
    """hydro_run (device CFL time step, graph replay) to t=0.2 on the Sod tube."""
    case = wl.sod(1000)
    s = O.solver_from_case(case)
    t, k = 0.0, 0
    while t < 0.2 * (1 - 1e-14):
        dt = min(s.cfl_dt(0.8), 0.2 - t)
        s.step(dt)
        t += dt
        k += 1
    g = hydro_lib.Grid.from_case(case, 64)
    t_gpu = g.run(k + 5, 0.8, t_end=0.2)
    assert abs(t_gpu - 0.2) < 1e-14
    assert g.stats()["steps"] == k
    # (a whole run: the per-step bars times the ~250 steps; the shocks' cells
    # carry the largest differences)
    check(s.get_state(), g.get_state(), 1, 1.4, 64, l1=1e-10, elem=1e-9)


@pytest.mark.parametrize("precision", [64, 32])
def test_totals_and_cfl(hydro_lib, precision):
    case = wl.sphere_state(30, 10, 12, n_scalars=2)
    s = O.solver_from_case(case)
    g = hydro_lib.Grid.from_case(case, precision)
    tol = 1e-14 if precision == 64 else 1e-6
    assert np.all(np.abs(g.totals() - s.totals()) <= tol * np.abs(s.totals()).max())
    assert abs(g.cfl_dt(0.4) - s.cfl_dt(0.4)) <= tol * 10 * s.cfl_dt(0.4)


def test_invalid_states_are_rejected(hydro_lib):
    H = hydro_lib
    case = wl.smooth_random(2, [20, 12], 0, seed=1)
    g = H.Grid.from_case(case, 64)
    before = g.get_state()
    bad = case["U"].copy()
    bad[3, 0, 4, 5] = 0.0  # energy below kinetic: negative pressure
    with pytest.raises(H.HydroError) as e:
        g.set_state(bad)
    assert e.value.status == H.HYDRO_ERR_NEGATIVE_STATE
    bad = case["U"].copy()
    bad[0, 0, 2, 2] = np.nan
    with pytest.raises(H.HydroError) as e:
        g.set_state(bad)
    assert e.value.status == H.HYDRO_ERR_NONFINITE
    assert np.array_equal(g.get_state(), before)


def test_failed_step_rolls_back(hydro_lib):
    H = hydro_lib
    case = wl.sod(200)
    g = H.Grid.from_case(case, 64)
    g.step(g.cfl_dt(0.5))
    before = g.get_state()
    with pytest.raises(H.HydroError) as e:
        g.step(50.0)  # far beyond the CFL limit: the update goes non-physical
    assert e.value.status in (H.HYDRO_ERR_NEGATIVE_STATE, H.HYDRO_ERR_NONFINITE)
    assert np.array_equal(g.get_state(), before)
    assert g.stats()["steps"] == 1
    g.step(g.cfl_dt(0.5))  # the handle keeps working
    assert g.stats()["steps"] == 2


def test_bad_arguments(hydro_lib):
    H = hydro_lib
    with pytest.raises(H.HydroError):
        H.Grid(1, [1], [np.array([0.0, 1.0])], [(0, 0)], 0, 1.4, 0, 1, 1)  # n < 2
    with pytest.raises(H.HydroError):
        H.Grid(1, [4], [np.array([0.0, 1.0, 0.5, 2.0, 3.0])], [(1, 1)], 0, 1.4, 0, 1, 1)  # faces
    with pytest.raises(H.HydroError):
        H.Grid(1, [4], [np.linspace(0, 1, 5)], [(1, 1)], 0, 1.4, 4, 1, 1)  # too many scalars
    g = H.Grid(1, [4], [np.linspace(0, 1, 5)], [(1, 1)], 0, 1.4, 0, 1, 1)
    with pytest.raises(H.HydroError):
        g.step(-1.0)
    with pytest.raises(H.HydroError):
        g.set_sources(gravity=H.HYDRO_GRAV_POINT, G=1.0, Mc=1.0)  # needs spherical


# ---- full-size configurations, in the launch configuration of the bench ----

def test_rt2d_full_size(hydro_lib):
    """512 x 1536 Rayleigh-Taylor: one FP64 and one FP32 step against the oracle."""
    case = wl.rt2d()
    for precision in (64, 32):
        step_compare(hydro_lib, case, precision, steps=1)


@pytest.mark.parametrize("precision", [64, 32])
def test_sedov_full_size_window(hydro_lib, precision):
    """256^3 Sedov, one step with hydro_run (autotuned, graph): a 36^3 window
    around the blast is recomputed by the oracle; its interior (3 cells in,
    beyond the one-step stencil reach) must match."""
    case = wl.sedov3d(256)
    U0 = case["U"].astype(np.float32 if precision == 32 else np.float64)
    g = hydro_lib.Grid.from_case(dict(case, U=U0), precision)
    g.run(1, case["cfl"])
    dt = g.stats()["last_dt"]
    B = g.get_state()
    lo, hi = 110, 146
    f = case["faces"][0][lo:hi + 1]
    win = O.Solver(3, [hi - lo] * 3, [f, f, f], [(O.TRANSMISSIVE, O.TRANSMISSIVE)] * 3, O.CARTESIAN,
                   1.4, 0, case["riemann"], case["limiter"])
    win.set_state(U0[:, lo:hi, lo:hi, lo:hi].astype(np.float64))
    win.step(dt)
    A = win.get_state()[:, 3:-3, 3:-3, 3:-3]
    Bw = B[:, lo + 3:hi - 3, lo + 3:hi - 3, lo + 3:hi - 3]
    check(A, Bw, 3, 1.4, precision)
    # far field untouched in one step, and the blast is octant-symmetric
    assert np.array_equal(B[:, :100, :100, :100], U0[:, :100, :100, :100])
    assert np.abs(B[0] - B[0][::-1, ::-1, ::-1]).max() <= (1e-12 if precision == 64 else 1e-5)


def test_wedge_full_size_window(hydro_lib):
    """1024x128x128 spherical wedge (FP32 bulk), one step without gravity:
    windows at the inner and outer radius recomputed by the oracle."""
    case = wl.wedge()
    case["sources"] = None
    U0 = case["U"].astype(np.float32)
    g = hydro_lib.Grid.from_case(dict(case, U=U0), 32)
    g.run(1, case["cfl"])
    dt = g.stats()["last_dt"]
    B = g.get_state()
    rf, tf, pf = case["faces"]
    for r0, r1 in ((0, 30), (990, 1024)):
        j0, j1, k0, k1 = 0, 24, 100, 128
        bc = [(O.REFLECTIVE if r0 == 0 else O.TRANSMISSIVE, O.TRANSMISSIVE if r1 == 1024 else O.TRANSMISSIVE),
              (O.REFLECTIVE, O.TRANSMISSIVE), (O.TRANSMISSIVE, O.REFLECTIVE)]
        win = O.Solver(3, [r1 - r0, j1 - j0, k1 - k0], [rf[r0:r1 + 1], tf[j0:j1 + 1], pf[k0:k1 + 1]], bc,
                       O.SPHERICAL, case["gamma"], 3, case["riemann"], case["limiter"])
        win.set_state(U0[:, k0:k1, j0:j1, r0:r1].astype(np.float64))
        win.step(dt)
        A = win.get_state()
        # keep cells 3 away from every window edge that is not a true boundary
        ri = slice(0 if r0 == 0 else 3, (r1 - r0) if r1 == 1024 else (r1 - r0 - 3))
        sl = (slice(None), slice(3, k1 - k0), slice(0, j1 - j0 - 3), ri)
        Bw = B[:, k0:k1, j0:j1, r0:r1][sl]
        check(A[sl], Bw, 3, case["gamma"], 32)


@pytest.mark.parametrize("precision", [64, 32])
def test_runs_are_deterministic(hydro_lib, precision):
    """Two identical runs give bitwise identical states (the only atomics are
    the order-independent speed maximum and counters)."""
    case = wl.smooth_random(3, [37, 23, 40], 1, seed=5, riemann=O.HLLC)
    outs = []
    for _ in range(2):
        g = hydro_lib.Grid.from_case(case, precision)
        g.run(5, 0.4)
        outs.append(g.get_state())
        g.close()
    assert np.array_equal(outs[0], outs[1])


def test_fp32_periodic_conservation(hydro_lib):
    """FP32 bulk with FP64/Kahan totals: mass, momentum and energy of a periodic
    KH box stay constant to FP32 rounding of the state over 50 steps."""
    case = wl.kh2d(128, 256)
    g = hydro_lib.Grid.from_case(dict(case, U=case["U"].astype(np.float32)), 32)
    T0 = g.totals()
    g.run(50, 0.4)
    T1 = g.totals()
    scale = np.abs(T0).max()
    assert np.all(np.abs(T1 - T0) <= 2e-6 * scale), (T1 - T0) / scale


@pytest.mark.parametrize("precision", [64, 32])
def test_runs_with_totals_and_monopole_are_deterministic(hydro_lib, precision):
    """Also with the conserved totals accumulated in the step and with the
    monopole's FP64 shell sums (a spherical wedge): two runs of the same
    device-side CFL steps give the same state and totals, bit for bit."""
    cases = [wl.sedov3d(48), dict(wl.sphere_state(40, 12, 10, dim=3, rotating=True, n_scalars=3),
                                  sources=dict(gravity=O.GRAV_POINT_MONOPOLE, G=0.01, Mc=2.0))]
    for case in cases:
        out = []
        for _ in range(2):
            g = hydro_lib.Grid.from_case(case, precision)
            g.set_step_totals(True)
            g.run(6, case.get("cfl", 0.4))
            out.append((g.get_state(), g.step_totals(), g.stats()["steps"]))
            g.close()
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
        assert out[0][2] == out[1][2] == 6


def test_beyond_32bit_element_offsets(hydro_lib):
    """Maximum sizes: a 256 x 256 x 6600 FP32 grid (4.3e8 cells, 2.2e9 state
    values per buffer, past 32-bit element offsets) whose state varies along
    z only, periodic everywhere, so that every one of its columns must
    advance exactly like the column of a 16 x 16 x 6600 grid with the same
    face spacing (8.4e6 values); one step with the same dt gives the same
    bits in all 65536 columns, and that column agrees with the oracle's
    2 x 2 x 6600 step."""
    import torch
    H = hydro_lib
    n2, nb = 6600, 256
    z = (np.arange(n2) + 0.5) / n2
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * z)
    p = 1.0 + 0.1 * np.cos(2 * np.pi * z)
    vel = [np.full(n2, 0.05), np.full(n2, -0.02), 0.3 * np.sin(4 * np.pi * z)]
    col = wl.conserved(1.4, rho, vel, p).astype(np.float32)  # (5, n2)
    per = [(wl.PERIODIC, wl.PERIODIC)] * 3

    def case(nxy, U):
        f = np.arange(nxy + 1) / nb
        return dict(dim=3, n=[nxy, nxy, n2], faces=[f, f, np.linspace(0.0, 1.0, n2 + 1)], bc=per,
                    coords=wl.CARTESIAN, gamma=1.4, n_scalars=0, riemann=wl.HLL, limiter=wl.MINMOD,
                    sources=None, U=U)

    small = H.Grid.from_case(case(16, np.ascontiguousarray(
        np.broadcast_to(col[:, :, None, None], (5, n2, 16, 16)))), 32)
    dt = small.cfl_dt(0.4)
    small.step(dt)
    ref = small.get_state()[:, :, 0, 0]
    small.close()
    Ub = torch.from_numpy(col).cuda().view(5, n2, 1, 1).expand(5, n2, nb, nb).contiguous()
    big = H.Grid.from_case(case(nb, Ub), 32)
    assert big.cfl_dt(0.4) == dt
    big.step(dt)
    out = torch.empty_like(Ub)
    big.get_state(out)
    big.close()
    del Ub
    refd = torch.from_numpy(np.ascontiguousarray(ref)).cuda().view(5, n2, 1, 1)
    same = bool(torch.eq(out, refd).all())
    worst = float((out - refd).abs().max()) if not same else 0.0
    del out
    assert same, worst
    o = O.solver_from_case(case(2, np.ascontiguousarray(
        np.broadcast_to(col.astype(np.float64)[:, :, None, None], (5, n2, 2, 2)))))
    o.step(dt)
    check(o.get_state()[:, :, 0, 0], ref.astype(np.float64), 3, 1.4, 32)
