"""Pins of the oracle's Riemann solvers and limiters against textbook values and
invariants (HERACLES++ Sect. 3.2; exact solver of App. C.1 / Toro 2009 ch. 4)."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        vals[k] = float(v)
    return vals


def _euler_flux(W, gamma):
    """Physical flux of the 1D Euler system (Eq. 1) from (rho, u, p)."""
    rho, u, p = W
    E = p / (gamma - 1) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, u * (E + p)])


def _cons(W, gamma):
    rho, u, p = W
    return np.array([rho, rho * u, p / (gamma - 1) + 0.5 * rho * u * u])


def test_sod_star_matches_toro_table():
    g = _golden("sod_star.txt")
    ps, us, it = O.exact_star(1.4, [1.0, 0.0, 1.0], [0.125, 0.0, 0.1])
    assert abs(ps - g["pstar"]) < 1e-5
    assert abs(us - g["ustar"]) < 1e-5
    assert it <= 10


def _random_problems(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        gamma = rng.choice([1.4, 5.0 / 3.0, 1.2])
        rL, rR = 10 ** rng.uniform(-2, 2, 2)
        pL, pR = 10 ** rng.uniform(-3, 3, 2)
        cL, cR = math.sqrt(gamma * pL / rL), math.sqrt(gamma * pR / rR)
        du_max = 2 * (cL + cR) / (gamma - 1)
        uL = rng.uniform(-2, 2)
        uR = uL + rng.uniform(-3, 0.8) * du_max / 2
        if uR - uL >= du_max * 0.95:
            continue
        out.append((gamma, np.array([rL, uL, pL]), np.array([rR, uR, pR])))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_solution_satisfies_jump_conditions(seed):
    """Across each wave the sampled star state satisfies Rankine-Hugoniot
    (shock) or the isentrope and Riemann invariant (rarefaction)."""
    for gamma, WL, WR in _random_problems(40, seed):
        ps, us, _ = O.exact_star(gamma, WL, WR)
        assert ps > 0
        eps = 1e-9 * (1 + abs(us))
        for side, WK in ((-1, WL), (1, WR)):
            # star density just beside the contact on this side
            Ws = O.exact_sample(gamma, WL, WR, us + side * eps)
            assert abs(Ws[1] - us) < 1e-9 * (1 + abs(us)) and abs(Ws[2] - ps) < 1e-9 * ps
            rK, uK, pK = WK
            rs = Ws[0]
            if ps > pK:  # shock
                S = (rs * us - rK * uK) / (rs - rK)
                m = rK * (uK - S)
                assert abs(m - rs * (us - S)) < 1e-8 * (abs(m) + rK)
                mom_K = rK * (uK - S) ** 2 + pK
                mom_s = rs * (us - S) ** 2 + ps
                assert abs(mom_K - mom_s) < 1e-8 * abs(mom_K)
                h_K = 0.5 * (uK - S) ** 2 + gamma * pK / ((gamma - 1) * rK)
                h_s = 0.5 * (us - S) ** 2 + gamma * ps / ((gamma - 1) * rs)
                assert abs(h_K - h_s) < 1e-8 * abs(h_K)
                # the sampled solution jumps exactly at S
                far = O.exact_sample(gamma, WL, WR, S - side * 1e-7 * (1 + abs(S)))
                near = O.exact_sample(gamma, WL, WR, S + side * 1e-7 * (1 + abs(S)))
                assert np.allclose(near, WK, rtol=1e-12) or np.allclose(far, WK, rtol=1e-12)
            else:  # rarefaction
                assert abs(ps / rs ** gamma - pK / rK ** gamma) < 1e-9 * pK / rK ** gamma
                cK, cs = math.sqrt(gamma * pK / rK), math.sqrt(gamma * ps / rs)
                J_K = uK - side * 2 * cK / (gamma - 1)
                J_s = us - side * 2 * cs / (gamma - 1)
                assert abs(J_K - J_s) < 1e-9 * (abs(J_K) + cK)
                # inside the fan the characteristic through the origin is xi = u -/+ c
                head = uK + side * cK
                tail = us + side * cs
                xi = 0.5 * (head + tail)
                Wf = O.exact_sample(gamma, WL, WR, xi)
                cf = math.sqrt(gamma * Wf[2] / Wf[0])
                assert abs(Wf[1] + side * cf - xi) < 1e-9 * (1 + abs(xi))
                assert abs(Wf[2] / Wf[0] ** gamma - pK / rK ** gamma) < 1e-9 * pK / rK ** gamma


def test_exact_newton_polish_independent_of_guess():
    """Newton is polished to roundoff, so a poor guess gives the same p*."""
    w = np.zeros(O.MLP_NPARAM, dtype=np.float32)
    for gamma, WL, WR in _random_problems(30, 9):
        ps0, us0, _ = O.exact_star(gamma, WL, WR)
        for b3 in (-3.0, 0.0, 2.0):  # MLP guess sqrt(pL pR) e^b3, used on two-shock faces
            w[-1] = b3
            ps1, us1, _ = O.exact_star(gamma, WL, WR, O.GUESS_MLP, w)
            assert abs(ps1 - ps0) <= 1e-13 * ps0
            assert abs(us1 - us0) <= 1e-12 * (abs(us0) + 1)


def test_exact_vacuum_is_an_error():
    with pytest.raises(O.OracleError) as e:
        O.exact_star(1.4, [1.0, -10.0, 1.0], [1.0, 10.0, 1.0])
    assert e.value.status == -8


def test_toro_guess_kinds():
    _, k = O.guess_toro(1.4, [1.0, 0.0, 1.0], [1.0, 0.01, 1.05])
    assert k == 0  # PVRS for nearby states
    _, k = O.guess_toro(1.4, [1.0, -2.0, 1.0], [1.0, 2.0, 1.0])
    assert k == 1  # two rarefactions
    _, k = O.guess_toro(1.4, [1.0, 0.0, 1000.0], [1.0, 0.0, 0.01])
    assert k == 2  # two shocks (strong pressure jump)


@pytest.mark.parametrize("solver", [O.HLL, O.HLLC, O.EXACT])
def test_flux_consistency(solver):
    """F(U, U) = F(U) for every solver (Eq. 1 flux)."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        W = np.array([10 ** rng.uniform(-1, 1), rng.uniform(-3, 3), 10 ** rng.uniform(-1, 1)])
        U = _cons(W, 1.4)
        F = O.flux_1d(solver, 1.4, U, U)
        assert np.allclose(F, _euler_flux(W, 1.4), rtol=1e-13, atol=1e-13 * np.abs(U).max())


@pytest.mark.parametrize("solver", [O.HLL, O.HLLC, O.EXACT])
def test_supersonic_upwinding(solver):
    WL = np.array([1.0, 5.0, 1.0])
    WR = np.array([0.5, 4.0, 0.8])
    F = O.flux_1d(solver, 1.4, _cons(WL, 1.4), _cons(WR, 1.4))
    assert np.allclose(F, _euler_flux(WL, 1.4), rtol=1e-14)
    F = O.flux_1d(solver, 1.4, _cons(-WL * [-1, 1, -1], 1.4), _cons(WR * [1, -1, 1], 1.4))
    assert np.allclose(F, _euler_flux(WR * [1, -1, 1], 1.4), rtol=1e-14)


def test_stationary_contact():
    """HLLC and the exact solver keep an isolated stationary contact; HLL diffuses it."""
    WL, WR = np.array([1.0, 0.0, 1.0]), np.array([0.1, 0.0, 1.0])
    for s in (O.HLLC, O.EXACT):
        F = O.flux_1d(s, 1.4, _cons(WL, 1.4), _cons(WR, 1.4))
        assert abs(F[0]) < 1e-15 and abs(F[1] - 1.0) < 1e-14 and abs(F[2]) < 1e-15
    F = O.flux_1d(O.HLL, 1.4, _cons(WL, 1.4), _cons(WR, 1.4))
    assert abs(F[0]) > 1e-3


def test_hllc_scalar_and_tangential_upwinded():
    """2D state with a scalar: HLLC carries tangential velocity and scalar by the contact."""
    g = 1.4
    WL = np.array([1.0, 0.3, 0.7, 1.0, 0.2])   # rho, u_n, u_t, p, f
    WR = np.array([0.8, 0.3, -0.4, 1.0, 0.9])
    def cons(W):
        rho, un, ut, p, f = W
        return np.array([rho, rho * un, rho * ut, p / (g - 1) + 0.5 * rho * (un * un + ut * ut), rho * f])
    F = O.flux_1d(O.HLLC, g, cons(WL), cons(WR), n_scalars=1, dim=2)
    # pure contact moving right at 0.3: flux is the left state's flux exactly
    rho, un, ut, p, f = WL
    E = p / (g - 1) + 0.5 * rho * (un * un + ut * ut)
    ref = np.array([rho * un, rho * un * un + p, rho * un * ut, un * (E + p), rho * un * f])
    assert np.allclose(F, ref, rtol=1e-13)


def test_limiters_reproduce_linear_data_and_are_tvd():
    rng = np.random.default_rng(5)
    for kind in (O.MINMOD, O.VANLEER, O.VANALBADA):
        for s in rng.normal(size=20):
            assert abs(O.limiter(kind, s, s) - s) <= 1e-15 * abs(s)  # linear data: exact slope
        for _ in range(200):
            a, b = rng.normal(size=2)
            sig = O.limiter(kind, a, b)
            if a * b <= 0:
                assert sig == 0.0  # extremum: no slope
            else:
                assert sig * a > 0  # same sign
                assert abs(sig) <= 2 * min(abs(a), abs(b)) + 1e-15  # TVD region
                assert abs(O.limiter(kind, b, a) - sig) <= 1e-15 * abs(sig)  # symmetric
    for _ in range(50):
        a, b = rng.normal(size=2)
        if a * b > 0:
            assert O.limiter(O.MINMOD, a, b) == (a if abs(a) < abs(b) else b)
    assert O.limiter(O.FIRST_ORDER, 1.0, 1.0) == 0.0
