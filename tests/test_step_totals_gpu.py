"""Conserved totals accumulated inside the step (FP32 bulk, FP64 conservation sums).

With hydro_set_step_totals on, every CTA of the fused sweep sums U dV of the
cells it updates in FP64 into its own partial, and hydro_step_totals sums the
partials in a fixed order.  Checked against what fixes them independently of
that code path: the oracle's totals of the same step's state (FP64: within
1e-12 of the largest total, the per-step parity bar applied to sums), the
library's separate totals pass over the same GPU state (FP64: 1e-13; FP32:
the Kahan-compensated FP32 partials of that pass against FP64 sums, 1e-6),
conservation on a periodic box (mass, momenta and energy unchanged to
roundoff), and determinism (two runs, the same bits).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


CASES = [
    ("sod_1d", lambda: wl.sod(500)),
    ("random_2d_periodic", lambda: wl.smooth_random(2, [70, 45], 1, seed=3, bc=[(O.PERIODIC, O.PERIODIC)] * 2,
                                                    riemann=O.HLLC)),
    ("random_3d", lambda: wl.smooth_random(3, [37, 23, 40], 1, seed=5, riemann=O.HLL,
                                           bc=[(O.TRANSMISSIVE, O.REFLECTIVE), (O.PERIODIC, O.PERIODIC),
                                               (O.PERIODIC, O.PERIODIC)])),
    ("wedge_3d_gravity", lambda: dict(wl.sphere_state(40, 12, 10, dim=3, rotating=True, n_scalars=3,
                                                      bc=[(O.REFLECTIVE, O.TRANSMISSIVE),
                                                          (O.REFLECTIVE, O.REFLECTIVE),
                                                          (O.PERIODIC, O.PERIODIC)]),
                                      sources=dict(gravity=O.GRAV_POINT, G=0.01, Mc=2.0))),
]


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("k", range(len(CASES)))
def test_step_totals_match_oracle_and_separate_pass(hydro_lib, precision, k):
    name, make = CASES[k]
    case = make()
    if precision == 32:
        case = dict(case, U=case["U"].astype(np.float32).astype(np.float64))
    s = O.solver_from_case(case)
    g = hydro_lib.Grid.from_case(case, precision)
    g.set_step_totals(True)
    for _ in range(3):
        dt = s.cfl_dt(case["cfl"])
        s.step(dt)
        g.step(dt)
        tg = g.step_totals()
        tp = g.totals()
        if precision == 64:
            assert _rel(tg, s.totals()) <= 1e-12, (name, tg, s.totals())
            assert _rel(tg, tp) <= 1e-13, (name, tg, tp)
        else:
            assert _rel(tg, tp) <= 1e-6, (name, tg, tp)
    g.close()


def test_step_totals_with_device_steps_conserve_on_a_periodic_box(hydro_lib):
    """hydro_run (device dt, graph): on a periodic box every total is
    conserved; the in-step totals after each run equal the separate pass."""
    case = wl.smooth_random(3, [32, 24, 28], 1, seed=9, riemann=O.HLLC, bc=[(O.PERIODIC, O.PERIODIC)] * 3)
    g = hydro_lib.Grid.from_case(case, 64)
    t0 = g.totals()
    g.set_step_totals(True)
    for _ in range(3):
        g.run(4, 0.4)
        tg = g.step_totals()
        assert _rel(tg, g.totals()) <= 1e-13
        scale = np.abs(t0).max()
        assert np.abs(tg - t0).max() <= 1e-12 * scale, (tg, t0)
    g.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_step_totals_are_deterministic(hydro_lib, precision):
    case = wl.smooth_random(3, [40, 33, 29], 1, seed=12, riemann=O.HLL)
    out = []
    for _ in range(2):
        g = hydro_lib.Grid.from_case(case, precision)
        g.set_step_totals(True)
        g.run(3, 0.4)
        out.append(g.step_totals())
        g.close()
    assert np.array_equal(out[0], out[1])


def test_step_totals_states_and_rejections(hydro_lib):
    H = hydro_lib
    case = wl.sod(300)
    g = H.Grid.from_case(case, 64)
    with pytest.raises(H.HydroError) as e:
        g.step_totals()  # off
    assert e.value.status == H.HYDRO_ERR_ARG
    g.set_step_totals(True)
    with pytest.raises(H.HydroError):
        g.step_totals()  # no step yet
    g.step(g.cfl_dt(0.8))
    t1 = g.step_totals()
    g.set_state(case["U"])
    with pytest.raises(H.HydroError):
        g.step_totals()  # the state was replaced
    g.step(g.cfl_dt(0.8))
    assert np.array_equal(g.step_totals(), t1)  # the same step from the same state
    with pytest.raises(H.HydroError) as e:
        g.set_moving_grid(0, 0.1)
    assert e.value.status == H.HYDRO_ERR_UNSUPPORTED
    g.set_step_totals(False)
    g.set_moving_grid(0, 0.1)
    with pytest.raises(H.HydroError) as e:
        g.set_step_totals(True)
    assert e.value.status == H.HYDRO_ERR_UNSUPPORTED
    g.close()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_fp32_step_totals_are_exact_sums_of_the_fp32_state(hydro_lib, k):
    """The FP32 3D form accumulates U dV as compensated FP32 column sums
    (exact FMA products, TwoSum pairs) scaled in FP64: its totals equal the
    FP64 sums of the very FP32 state it wrote to within 1e-12 of sum |U| dV,
    some five orders below what a plain FP32 accumulation allows."""
    if k < len(CASES):
        name, make = CASES[k]
        case = make()
    else:
        name = "random_3d_long_columns"
        case = wl.smooth_random(3, [48, 40, 150], 1, seed=21, riemann=O.HLLC,
                                bc=[(O.PERIODIC, O.PERIODIC)] * 3)
    case = dict(case, U=case["U"].astype(np.float32).astype(np.float64))
    g = hydro_lib.Grid.from_case(case, 32)
    g.set_step_totals(True)
    g.run(3, case["cfl"])
    tg = g.step_totals()
    U = g.get_state().astype(np.float64)
    g.close()
    exact = O.solver_from_case(dict(case, U=U)).totals()
    scale = O.solver_from_case(dict(case, U=np.abs(U))).totals()
    err = np.abs(tg - exact) / scale
    print(name, "worst |step total - FP64 sum| / sum |U| dV: %.2e" % err.max())
    assert err.max() <= 1e-12, (name, err)
