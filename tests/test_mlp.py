"""The learned star-pressure guess: oracle pins (CPU) and GPU kernels vs oracle.

CPU pins: the oracle's backward pass agrees with central finite differences
of its own forward pass; a first Adam step has the closed form
w - lr g/(|g| + eps).
GPU: forward+backward gradients vs the oracle (FP32 vs FP64, relative
1e-4 of the gradient norm), one Adam step vs the oracle, the exact solver on
face lists vs the oracle, and the gain of the trained network over Toro's
guess (fewer Newton iterations on the faces where it is used).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 6))
    T = rng.normal(size=n)
    return X, T


def test_oracle_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    w = (0.3 * rng.standard_normal(O.MLP_NPARAM)).astype(np.float32)
    X, T = _samples(7, 2)
    _, g = O.mlp_loss_grad(w, X, T)
    # float32 weights limit the step size; check a sample of coordinates
    for p in list(range(0, 384, 37)) + list(range(448, 4544, 301)) + [4600, 4650, 4672]:
        wp = w.astype(np.float64).copy()
        h = 1e-3 * max(1.0, abs(wp[p]))
        wp[p] += h
        lp = np.mean((O.mlp_forward(wp.astype(np.float32), X) - T) ** 2)
        wm = w.astype(np.float64).copy()
        wm[p] -= h
        lm = np.mean((O.mlp_forward(wm.astype(np.float32), X) - T) ** 2)
        hh = float(np.float32(w[p] + h) - np.float32(w[p] - h))  # the step the float weights took
        fd = (lp - lm) / hh
        assert abs(fd - g[p]) <= 2e-3 * max(abs(g[p]), 1e-3), (p, fd, g[p])


def test_oracle_forward_special_cases():
    w = np.zeros(O.MLP_NPARAM, dtype=np.float32)
    w[-1] = 0.75
    assert np.allclose(O.mlp_forward(w, np.random.default_rng(0).normal(size=(4, 6))), 0.75)
    # one hidden path: y = w3_0 * silu(W2_00 * silu(W1_00 x_0))
    w[0] = 2.0
    w[384 + 64] = 1.5
    w[384 + 64 + 4096 + 64] = 0.5
    x = np.array([[0.3, 0, 0, 0, 0, 0]])
    silu = lambda z: z / (1 + np.exp(-z))
    assert abs(O.mlp_forward(w, x)[0] - (0.75 + 0.5 * silu(1.5 * silu(0.6)))) < 1e-12


def test_oracle_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    w = rng.normal(size=O.MLP_NPARAM).astype(np.float32)
    g = rng.normal(size=O.MLP_NPARAM)
    w1, m1, v1 = O.adam_step(w, np.zeros_like(w), np.zeros_like(w), g, 1, 1e-3)
    expect = w.astype(np.float64) - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.allclose(w1, expect, rtol=0, atol=2e-7 * np.abs(expect).max())


@pytest.mark.gpu
def test_gpu_gradient_matches_oracle(hydro_lib):
    rng = np.random.default_rng(4)
    w = (0.3 * rng.standard_normal(O.MLP_NPARAM)).astype(np.float32)
    for n in (1, 63, 64, 65, 1000):
        X, T = _samples(n, n)
        Xf = X.astype(np.float32).astype(np.float64)
        Tf = T.astype(np.float32).astype(np.float64)
        lo, go = O.mlp_loss_grad(w, Xf, Tf)
        lg, gg = hydro_lib.hydro_mlp_loss_grad(w, Xf, Tf)
        assert abs(lg - lo) <= 1e-5 * lo
        assert np.linalg.norm(gg - go) <= 1e-4 * np.linalg.norm(go), n


def _faces(ntubes, seed):
    WL, WR = wl.tube_states(ntubes, seed)
    return WL, WR


@pytest.mark.gpu
def test_gpu_exact_solver_matches_oracle(hydro_lib):
    WL, WR = _faces(2000, 31)
    ps, us, it = hydro_lib.hydro_exact_solve(WL, WR, 5 / 3, precision=64)
    for i in range(0, 2000, 7):
        p0, u0, i0 = O.exact_star(5 / 3, WL[i], WR[i])
        assert abs(ps[i] - p0) <= 1e-13 * p0 and abs(us[i] - u0) <= 1e-12 * (1 + abs(u0))
        assert abs(it[i] - i0) <= 1
    ps32, _, _ = hydro_lib.hydro_exact_solve(WL, WR, 5 / 3, precision=32)
    assert np.max(np.abs(ps32 - ps) / ps) < 1e-5


@pytest.mark.gpu
def test_gpu_adam_step_matches_oracle(hydro_lib):
    WL, WR = _faces(256, 32)
    faces = np.concatenate([WL, WR], axis=1)
    lp = np.log([O.exact_star(5 / 3, WL[i], WR[i])[0] for i in range(256)])
    rng = np.random.default_rng(5)
    w0 = (0.2 * rng.standard_normal(O.MLP_NPARAM)).astype(np.float32)
    b = hydro_lib.Batch([4, 4], 5 / 3)
    b.mlp_set(w0, False)
    b.mlp_train(faces, lp, epochs=1, batch=4096, lr=1e-3, seed=1)  # one full-batch step
    w1 = b.mlp_get()
    X = np.array([O.mlp_features(5 / 3, WL[i], WR[i])[0] for i in range(256)])
    pref = np.array([O.mlp_features(5 / 3, WL[i], WR[i])[1] for i in range(256)])
    tsrs = np.array([O.guess_toro(5 / 3, WL[i], WR[i])[1] == 2 and
                     max(WL[i, 2], WR[i, 2]) > 4 * min(WL[i, 2], WR[i, 2]) for i in range(256)])
    X32 = X.astype(np.float32).astype(np.float64)[tsrs]
    T32 = (lp - np.log(pref)).astype(np.float32).astype(np.float64)[tsrs]
    _, g = O.mlp_loss_grad(w0, X32, T32)
    we, _, _ = O.adam_step(w0, np.zeros_like(w0), np.zeros_like(w0), g, 1, 1e-3)
    # the first Adam step moves each weight by ~lr sign(g); FP32 gradients
    # only differ where |g| is tiny
    close = np.abs(w1 - we) <= 1e-6 + 1e-6 * np.abs(we)
    assert close.mean() > 0.99


@pytest.mark.gpu
def test_trained_network_reduces_newton_iterations(hydro_lib):
    """Train on the initial faces, partial-jump faces of the same state
    distribution and faces harvested from an FP64 run (seed 4 sampling);
    evaluate on a held-out harvest (seed 5): on the faces where the network is
    used (two-shock Toro estimate, pressure jump > 4) Newton needs fewer
    iterations than from Toro's guess, with identical p* after polishing."""
    H = hydro_lib
    w = wl.tubes(1024, seed=2)
    b = H.Batch(w["lengths"], w["gamma"], precision=64)
    b.set_state(w["U"])
    b.harvest_begin(400000, 1.0, 4)
    b.run(60, 0.8)
    harv = b.harvest_get(400000)
    tw = wl.tubes(512, seed=12)
    b2 = H.Batch(tw["lengths"], tw["gamma"], precision=64)
    b2.set_state(tw["U"])
    b2.harvest_begin(100000, 1.0, 5)
    b2.run(45, 0.8)
    test = b2.harvest_get(100000)
    train = np.concatenate([wl.partial_jump_faces(60000, 7), harv])
    assert len(harv) > 2000 and len(test) > 500
    ps, _, _ = H.hydro_exact_solve(train[:, :3], train[:, 3:], w["gamma"], precision=64)
    assert np.all(ps > 0)
    loss = b.mlp_train(train, np.log(ps), epochs=60, batch=256, lr=3e-3, seed=4)
    assert loss < 1e-4
    wts = b.mlp_get()
    p_t, _, it_t = H.hydro_exact_solve(test[:, :3], test[:, 3:], w["gamma"], precision=64)
    p_m, _, it_m = H.hydro_exact_solve(test[:, :3], test[:, 3:], w["gamma"], H.HYDRO_GUESS_MLP, wts, 64)
    assert np.all(np.abs(p_m - p_t) <= 1e-13 * p_t)
    assert it_m.mean() < 0.95 * it_t.mean(), (it_m.mean(), it_t.mean())
