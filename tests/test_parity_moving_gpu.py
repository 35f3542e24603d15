"""GPU moving grid (Sect. 3.1.1, reading R16) against the FP64 oracle, step by step.

The oracle takes the flux through a moving face by sampling the Riemann
solution on the face's path x/t = w; the library takes the fixed-face flux
of the states seen from the frame that moves with the face and brings it
back to the lab frame -- two routes to the same number, so parity checks
both.  Cartesian grids move along each axis (transmissive and periodic
ends, HLL, HLLC and the exact solver); spherical grids move along r (1D and
3D, HLLC, with point-mass gravity in 3D), where the face areas are averaged
over the step and every cell's content is spread over its new volume.  Bars
per step as for the fixed grid (tests/parity.py); the faces must have moved
by w dt.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl
from parity import check

pytestmark = pytest.mark.gpu

CASES = [
    (1, [300], 0, O.EXACT, [(O.TRANSMISSIVE, O.TRANSMISSIVE)]),
    (1, [257], 0, O.HLL, [(O.PERIODIC, O.PERIODIC)]),
    (2, [70, 45], 0, O.HLLC, [(O.TRANSMISSIVE, O.TRANSMISSIVE), (O.PERIODIC, O.PERIODIC)]),
    (2, [41, 66], 1, O.EXACT, [(O.REFLECTIVE, O.TRANSMISSIVE), (O.TRANSMISSIVE, O.TRANSMISSIVE)]),
    (3, [37, 23, 40], 2, O.HLLC, [(O.PERIODIC, O.PERIODIC), (O.REFLECTIVE, O.TRANSMISSIVE),
                                  (O.PERIODIC, O.PERIODIC)]),
    (3, [33, 21, 19], 0, O.HLL, [(O.TRANSMISSIVE, O.TRANSMISSIVE), (O.PERIODIC, O.PERIODIC),
                                 (O.REFLECTIVE, O.REFLECTIVE)]),
]


def _run(H, case, precision, steps=3):
    if precision == 32:
        case = dict(case, U=case["U"].astype(np.float32).astype(np.float64))
    s = O.solver_from_case(case)
    g = H.Grid.from_case(case, precision)
    axis = case["moving"][0]
    for _ in range(steps):
        dt = s.cfl_dt(case["cfl"])
        assert abs(g.cfl_dt(case["cfl"]) - dt) <= (1e-13 if precision == 64 else 1e-6) * dt
        s.step(dt)
        g.step(dt)
        A = s.get_state()
        check(A, g.get_state(), case["dim"], case["gamma"], precision, label=case["name"])
        assert np.allclose(g.faces(axis), s.faces(axis), rtol=0, atol=1e-13)
        if precision == 32:
            g.set_state(A.astype(np.float32))
            s.set_state(A.astype(np.float32).astype(np.float64))
    g.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_cartesian_moving_axis(hydro_lib, precision, k):
    dim, n, axis, riemann, bc = CASES[k]
    case = wl.smooth_random(dim, n, 1, seed=40 + k, bc=bc, riemann=riemann)
    _run(hydro_lib, dict(case, moving=(axis, 0.31 if k % 2 else -0.23)), precision)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dim", [1, 3])
def test_spherical_radial_motion(hydro_lib, precision, dim):
    case = wl.sphere_state(45, 14, 12, dim=dim, rotating=True, r_range=(1.0, 4.0), n_scalars=1,
                           bc=[(O.TRANSMISSIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                               (O.PERIODIC, O.PERIODIC)][:dim])
    if dim == 3:
        case["sources"] = dict(gravity=O.GRAV_POINT, G=0.01, Mc=2.0)
    _run(hydro_lib, dict(case, moving=(0, 0.4)), precision)


def test_uniform_gas_stays_uniform_on_the_gpu(hydro_lib):
    """The geometric conservation law on the GPU: a uniform gas at rest on a
    3D spherical grid whose radial faces move stays uniform (FP64)."""
    case = wl.sphere_state(40, 10, 8, dim=3, uniform=True, r_range=(1.0, 3.0), ph_range=(0.0, 1.0),
                           bc=[(O.TRANSMISSIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                               (O.PERIODIC, O.PERIODIC)])
    g = hydro_lib.Grid.from_case(dict(case, moving=(0, 0.6)), 64)
    t = g.run(20, 0.4)
    U = g.get_state()
    U0 = case["U"]
    assert np.abs(U - U0).max() <= 1e-13 * np.abs(U0).max()
    assert g.stats()["steps"] == 20
    assert np.allclose(g.faces(0), np.asarray(case["faces"][0]) + 0.6 * t, rtol=0, atol=1e-12)
    g.close()


def test_moving_grid_rejections(hydro_lib):
    H = hydro_lib
    case = wl.sphere_state(20, 8, 6, dim=3, bc=[(O.REFLECTIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                                                (O.PERIODIC, O.PERIODIC)])
    g = H.Grid.from_case(case, 64)
    with pytest.raises(H.HydroError):
        g.set_moving_grid(0, 0.1)  # reflective inner end
    with pytest.raises(H.HydroError):
        g.set_moving_grid(1, 0.1)  # spherical: r only
    g.close()
