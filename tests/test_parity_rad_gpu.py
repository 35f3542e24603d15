"""GPU grid path with the gas + radiation EoS (Sect. 2.3, Eq. 6-7) against
the FP64 oracle, element by element, one step at a time.

The conserved state is read through Eq. 6 (e = rho R T/(gamma-1) + a T^4),
so with R = a = 1 the random test states have P_rad/P_gas between about 0.1
and 0.4.  Same bars as the ideal-gas parity tests: FP64 relative L1 per
component <= 1e-12 per step, FP32 <= 2e-5.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl

from test_parity_grid import step_compare

pytestmark = pytest.mark.gpu

RAD = (1.0, 1.0)  # R_gas, a_rad in code units


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("riemann", [O.HLL, O.HLLC])
def test_rad_1d(hydro_lib, precision, riemann):
    for ns, bc in ((0, (O.PERIODIC, O.PERIODIC)), (1, (O.TRANSMISSIVE, O.REFLECTIVE)), (3, (O.REFLECTIVE, O.TRANSMISSIVE))):
        case = wl.smooth_random(1, [600], ns, seed=21 + ns, bc=[bc], riemann=riemann)
        step_compare(hydro_lib, dict(case, eos_rad=RAD), precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("riemann", [O.HLL, O.HLLC])
def test_rad_2d(hydro_lib, precision, riemann):
    case = wl.smooth_random(2, [70, 37], 1, seed=5, riemann=riemann,
                            bc=[(O.PERIODIC, O.PERIODIC), (O.REFLECTIVE, O.TRANSMISSIVE)])
    step_compare(hydro_lib, dict(case, eos_rad=RAD), precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("ns", [0, 3])
def test_rad_3d(hydro_lib, precision, ns):
    case = wl.smooth_random(3, [37, 21, 35], ns, seed=9, riemann=O.HLLC,
                            bc=[(O.PERIODIC, O.PERIODIC), (O.TRANSMISSIVE, O.TRANSMISSIVE),
                                (O.REFLECTIVE, O.REFLECTIVE)])
    step_compare(hydro_lib, dict(case, eos_rad=RAD), precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
def test_rad_spherical_3d(hydro_lib, precision):
    case = wl.sphere_state(nr=20, nth=12, nph=10, seed=13, riemann=O.HLLC, n_scalars=1,
                           ph_range=(0.0, 0.6))
    step_compare(hydro_lib, dict(case, eos_rad=RAD), precision, steps=2)


def test_rad_stationary_contact_stays_at_rest(hydro_lib):
    n = 300
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.5, 1.0, 0.2)
    e = np.array([O.eos_rad_eint(5.0 / 3.0, 1.0, 1.0, r, 2.0)[1] for r in rho])
    U = np.stack([rho, np.zeros(n), e]).reshape(3, 1, 1, n)
    case = dict(name="contact", dim=1, n=[n, 1, 1], faces=[np.linspace(0, 1, n + 1)],
                bc=[(wl.PERIODIC, wl.PERIODIC)], coords=wl.CARTESIAN, gamma=5.0 / 3.0, n_scalars=0,
                riemann=wl.HLLC, limiter=wl.MINMOD, cfl=0.8, sources=None, U=U, eos_rad=(1.0, 1.0))
    g = hydro_lib.Grid.from_case(case, 64)
    g.run(50, 0.8)
    V = g.get_state()
    g.close()
    assert np.max(np.abs(V[1])) <= 1e-13
    assert np.max(np.abs(V - U)) <= 1e-12 * np.max(np.abs(U))


def test_rad_needs_hll_or_hllc(hydro_lib):
    case = wl.sod(64, riemann=wl.EXACT)
    g = hydro_lib.Grid.from_case(case, 64)
    with pytest.raises(hydro_lib.HydroError):
        g.set_eos_radiation(1.0, 1.0)
    g.close()
