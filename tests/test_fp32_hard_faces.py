"""FP32 exact-solver faces that are solved in FP64, and their neighbourhood, against the oracle.

The FP32 form solves a face in FP64 when its pressure ratio exceeds 1e6 or
its velocity jump du = u_R - u_L comes within 20 % of the vacuum limit
vac = 2 (c_L + c_R)/(gamma - 1), where the FP32 pressure functions lose
their digits (reading R12).  The FP32 form computes with gamma rounded to
FP32, so its star states are compared with the oracle's at that gamma (near
vacuum p* moves by ~1e-5 between gamma = 5/3 and its FP32 rounding).  The
workload's own jumps stop at a pressure ratio of 1e4, so these cases are
built here:

- star states of faces inside the FP64 band (ratio 2e6-1e8, or du between
  0.82 and 0.97 of vac): the FP64 Newton solve of the FP32-rounded data, so
  p* and u* must equal the oracle's solve of the same data up to the final
  rounding to FP32 (2 ulp);
- faces just outside the band, solved in FP32 (ratio 1e4-5e5, du from 0.40
  to 0.78 of vac), where the bound on p* follows from the rounding of the
  residual r(p) = f_L(p) + f_R(p) + du (Toro's pressure functions): k ulp of
  |f_L| + |f_R| + |du| move the root by kappa = (|f_L| + |f_R| + |du|) /
  (p* r'(p*)) times k eps32 relative (near vacuum the terms cancel to the
  margin vac - du, and kappa ~ vac/(z (vac - du)), z = (gamma-1)/(2 gamma)),
  on top of Newton's own FP32 stopping rule (1e-6, polished);
- whole FP32 tubes whose interface has a pressure ratio of 2e6-1e8, stepped
  against the oracle with the per-step FP32 bars of tests/parity.py, with
  the FP64 category of the solver counters showing that the FP64 path ran.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl
from parity import check

pytestmark = pytest.mark.gpu

G = 5.0 / 3.0
G32 = float(np.float32(G))  # the FP32 form's gamma
EPS32 = 2.0 ** -24


def _sound(W):
    return np.sqrt(G * W[:, 2] / W[:, 0])


def _faces(n, seed, ratio_lo, ratio_hi, vac_lo, vac_hi):
    """n faces: pressure ratio log-uniform in [ratio_lo, ratio_hi] (either
    side high), density ratio log-uniform in [1e-2, 1e2]; the second half has
    a pressure ratio of at most 10 and du a fraction in [vac_lo, vac_hi] of
    the vacuum limit instead.  FP32-representable values."""
    r = wl.uniform01(seed, 5 * n).reshape(5, n)
    rp = 10.0 ** (np.log10(ratio_lo) + (np.log10(ratio_hi) - np.log10(ratio_lo)) * r[0])
    rp = np.where(r[4] < 0.5, rp, 1.0 / rp)
    rr = 10.0 ** (-2.0 + 4.0 * r[1])
    h = n // 2
    rp[h:] = 10.0 ** (-1.0 + 2.0 * r[0, h:])
    WL = np.stack([np.sqrt(rr), np.zeros(n), np.sqrt(rp)], axis=1)
    WR = np.stack([1.0 / np.sqrt(rr), np.zeros(n), 1.0 / np.sqrt(rp)], axis=1)
    WL = WL.astype(np.float32).astype(np.float64)
    WR = WR.astype(np.float32).astype(np.float64)
    vac = 2.0 / (G - 1.0) * (_sound(WL) + _sound(WR))
    frac = vac_lo + (vac_hi - vac_lo) * r[2]
    du = np.where(np.arange(n) < h, -1.0 + 2.0 * r[3], frac * vac)
    WL[:, 1] = (-0.5 * du).astype(np.float32)
    WR[:, 1] = (0.5 * du).astype(np.float32)
    return WL, WR


def _kappa(W, p, gamma=G32):
    """|f_K(p)| and f_K'(p) of Toro's pressure function for the states W (n x 3)."""
    r, pk = W[:, 0], W[:, 2]
    c = np.sqrt(gamma * pk / r)
    A, B = 2.0 / ((gamma + 1.0) * r), (gamma - 1.0) / (gamma + 1.0) * pk
    shock = p > pk
    q = np.sqrt(A / (p + B))
    f = np.where(shock, (p - pk) * q, 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0))
    df = np.where(shock, q * (1.0 - 0.5 * (p - pk) / (B + p)),
                  (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (r * c))
    return np.abs(f), df


def _oracle(WL, WR, gamma=G32):
    out = np.array([O.exact_star(gamma, WL[i], WR[i])[:2] for i in range(len(WL))])
    return out[:, 0], out[:, 1]


def test_fp32_faces_in_the_fp64_band(hydro_lib):
    WL, WR = _faces(4000, 41, 2e6, 1e8, 0.82, 0.97)
    ps, us, it = hydro_lib.hydro_exact_solve(WL, WR, G, precision=32)
    po, uo = _oracle(WL, WR)
    assert np.all(it > 0) and np.all(ps > 0)
    scale_u = np.abs(uo) + _sound(WL) + _sound(WR)
    ep = np.abs(ps - po) / po
    eu = np.abs(us - uo) / scale_u
    print("FP64 band: worst relative p* error %.2e, u* %.2e" % (ep.max(), eu.max()))
    assert ep.max() <= 4 * EPS32
    assert eu.max() <= 4 * EPS32


def test_fp32_faces_next_to_the_fp64_band(hydro_lib):
    WL, WR = _faces(4000, 42, 1e4, 5e5, 0.40, 0.78)
    ps, us, it = hydro_lib.hydro_exact_solve(WL, WR, G, precision=32)
    po, uo = _oracle(WL, WR)
    assert np.all(it > 0), "Newton failed on %d faces" % int((it <= 0).sum())
    assert np.all(ps > 0)
    fl, dfl = _kappa(WL, po)
    fr, dfr = _kappa(WR, po)
    kappa = (fl + fr + np.abs(WR[:, 1] - WL[:, 1])) / (po * (dfl + dfr))
    bound = 1e-6 + 16.0 * EPS32 * kappa
    ep = np.abs(ps - po) / po
    print("next to the band: worst p* error / bound %.2e (worst relative %.2e)" % ((ep / bound).max(), ep.max()))
    assert np.all(ep <= bound)
    scale_u = np.abs(uo) + _sound(WL) + _sound(WR)
    assert (np.abs(us - uo) / scale_u).max() <= 1e-4


def test_fp32_tubes_with_fp64_faces(hydro_lib):
    n = 16
    r = wl.uniform01(43, 4 * n).reshape(4, n)
    rp = 10.0 ** (np.log10(2e6) + (8.0 - np.log10(2e6)) * r[0])
    rp = np.where(r[3] < 0.5, rp, 1.0 / rp)
    rr = 10.0 ** (-2.0 + 4.0 * r[1])
    du = -1.0 + 2.0 * r[2]
    lengths = (300 + (1700 * wl.uniform01(44, n))).astype(np.int32)
    WL = np.stack([np.sqrt(rr), -0.5 * du, np.sqrt(rp)], axis=1)
    WR = np.stack([1.0 / np.sqrt(rr), 0.5 * du, 1.0 / np.sqrt(rp)], axis=1)
    U = np.empty((3, int(lengths.sum())))
    off = 0
    for b, nb in enumerate(lengths):
        x = (np.arange(nb) + 0.5) / nb
        W = np.where((x < 0.5)[None, :], WL[b][:, None], WR[b][:, None])
        U[:, off:off + nb] = wl.conserved(G, W[0], [W[1]], W[2])
        off += nb
    # FP32, per step from the oracle's state
    U32 = U.astype(np.float32)
    b32 = hydro_lib.Batch(lengths, G, precision=32)
    for k in range(4):
        b32.set_state(U32)
        ref, _ = O.batch_run(lengths, U32.astype(np.float64), G, O.EXACT, O.MINMOD, 0.8, 1)
        b32.run(1, 0.8)
        check(ref, b32.get_state(), 1, G, 32, label="step %d" % (k + 1))
        U32 = ref.astype(np.float32)
    st = b32.stats()
    assert st["newton_faces"][2] >= n, st["newton_faces"]  # the interfaces, solved in FP64
    b32.close()
    # FP64 form, a run of 10 steps
    ref, _ = O.batch_run(lengths, U, G, O.EXACT, O.MINMOD, 0.8, 10)
    b64 = hydro_lib.Batch(lengths, G, precision=64)
    b64.set_state(U)
    b64.run(10, 0.8)
    check(ref, b64.get_state(), 1, G, 64, l1=1e-11, elem=1e-10)
    assert b64.stats()["newton_faces"][2] == 0
    b64.close()
