"""GPU grid path with the dual-energy correction (Sect. 2.5) against the
FP64 oracle, one step at a time.  The test states are random smooth states
boosted to a bulk velocity of 30 (Mach ~ 25), so that e / e_k spans the
blend band eps e_k/10 < e < eps e_k (eps = 0.02) or lies below it (eps = 1).
Bars as for the other parity tests: FP64 <= 1e-12, FP32 <= 2e-5 relative L1
per component and step."""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl

from test_parity_grid import step_compare

pytestmark = pytest.mark.gpu


def _boost(case, v0=30.0):
    """Add v0 to the axis-0 velocity of every cell, keeping rho, e and scalars."""
    U = case["U"].copy()
    rho = U[0]
    dim = case["dim"]
    ux = U[1] / rho
    U[1 + dim] = U[1 + dim] + rho * v0 * ux + 0.5 * rho * v0 * v0
    U[1] = U[1] + rho * v0
    return dict(case, U=U)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("eps", [0.02, 1.0])
def test_dual_1d(hydro_lib, precision, eps):
    for ns in (0, 1):
        case = _boost(wl.smooth_random(1, [500], ns, seed=31 + ns, riemann=O.HLLC))
        step_compare(hydro_lib, dict(case, dual_energy=eps), precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
def test_dual_2d(hydro_lib, precision):
    case = _boost(wl.smooth_random(2, [70, 37], 1, seed=6, riemann=O.HLL))
    step_compare(hydro_lib, dict(case, dual_energy=0.02), precision, steps=2)


@pytest.mark.parametrize("precision", [64, 32])
def test_dual_3d(hydro_lib, precision):
    case = _boost(wl.smooth_random(3, [37, 21, 35], 0, seed=10, riemann=O.HLLC))
    step_compare(hydro_lib, dict(case, dual_energy=0.02), precision, steps=2)


def test_dual_with_radiation_eos(hydro_lib):
    case = _boost(wl.smooth_random(1, [400], 0, seed=17, riemann=O.HLLC))
    step_compare(hydro_lib, dict(case, dual_energy=0.02, eos_rad=(1.0, 1.0)), 64, steps=2)


def test_dual_off_is_bitwise_the_plain_step(hydro_lib):
    case = wl.smooth_random(2, [40, 30], 0, seed=2)
    a = hydro_lib.Grid.from_case(case, 64)
    b = hydro_lib.Grid.from_case(dict(case, dual_energy=1e-6), 64)
    a.run(5, 0.4)
    b.run(5, 0.4)
    assert np.array_equal(a.get_state(), b.get_state())
    a.close()
    b.close()
