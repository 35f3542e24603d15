"""GPU exact Riemann sampling (hydro_exact_sample) and per-tube times
(hydro_batch_times), the pieces of the equal-accuracy check of the batched
workload (per-tube L1 error against the exact solution at the final time)."""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_exact_sample_matches_oracle(hydro_lib):
    g = 5.0 / 3.0
    WL, WR = wl.tube_states(64, 11)
    # sample every face across its whole wave fan, beyond both outer waves
    xi = np.linspace(-6.0, 6.0, 61)
    face_of = np.repeat(np.arange(64), len(xi))
    xs = np.tile(xi, 64)
    W = hydro_lib.hydro_exact_sample(WL, WR, g, face_of, xs)
    ref = np.array([O.exact_sample(g, WL[f], WR[f], x) for f, x in zip(face_of, xs)])
    scale = np.stack([ref[:, 0], np.sqrt(g * ref[:, 2] / ref[:, 0]), ref[:, 2]], 1)
    assert np.max(np.abs(W - ref) / scale) < 1e-11


def test_exact_sample_sod_star_region(hydro_lib):
    # Toro (2009) Table 4.3, test 1: p* = 0.30313, u* = 0.92745, rho*L = 0.42632
    # (x/t = 0.5: between the rarefaction tail and the contact), rho*R = 0.26557
    # (x/t = 1.2: between the contact and the shock)
    W = hydro_lib.hydro_exact_sample([1.0, 0.0, 1.0], [0.125, 0.0, 0.1], 1.4, [0, 0], [0.5, 1.2])
    assert np.all(np.abs(W[:, 2] - 0.30313) < 1e-5) and np.all(np.abs(W[:, 1] - 0.92745) < 1e-5)
    assert abs(W[0, 0] - 0.42632) < 1e-5 and abs(W[1, 0] - 0.26557) < 1e-5


def test_exact_sample_rejects_bad_face(hydro_lib):
    with pytest.raises(hydro_lib.HydroError):
        hydro_lib.hydro_exact_sample([1.0, 0.0, 1.0], [0.125, 0.0, 0.1], 1.4, [1], [0.0])


def _speed(U, lengths, g):
    """max_i (|u|+c) n_b per tube (FP64), the CFL speed of each tube."""
    rho, m, E = U
    u = m / rho
    p = (g - 1.0) * (E - 0.5 * rho * u * u)
    s = np.abs(u) + np.sqrt(g * p / rho)
    off = np.concatenate([[0], np.cumsum(lengths)])
    return np.array([s[off[b]:off[b + 1]].max() * lengths[b] for b in range(len(lengths))])


def test_batch_times_are_sums_of_own_cfl_steps(hydro_lib):
    w = wl.tubes(12, seed=5, lo=64, hi=300)
    g, cfl = w["gamma"], 0.8
    b = hydro_lib.Batch(w["lengths"], g, precision=64)
    b.set_state(w["U"])
    assert np.all(b.times() == 0.0)
    t_expect = cfl / _speed(w["U"], w["lengths"], g)
    b.run(1, cfl)
    assert np.allclose(b.times(), t_expect, rtol=1e-14, atol=0)
    U1 = b.get_state()
    t_expect = t_expect + cfl / _speed(U1, w["lengths"], g)
    b.run(1, cfl)
    assert np.allclose(b.times(), t_expect, rtol=1e-14, atol=0)
    b.close()
