"""Element-wise and L1 comparison of a GPU state with the oracle's.

Two bars per conserved component v, both against the oracle's state A:

- relative L1: sum|B_v - A_v| / S1_v, the bar the accuracy target is stated
  in (1e-12 per FP64 step);
- element-wise: max|B_v - A_v| / Sinf_v, which a wrong value in a single
  cell (a wall, a tile seam, a z-chunk seam) cannot pass by being averaged
  over the grid.

Scales.  Density and energy are measured against their own norms (S1 =
sum|A_v|, Sinf = max|A_v|).  A momentum component is measured against at
least the acoustic momentum rho c of the same cells, a passive scalar
against at least the density: a momentum that is nearly zero somewhere (a
static state, or a transverse momentum created in one step) is not computed
to a relative accuracy of its own but to the accuracy of the momentum flux
rho u^2 + P that produces it, whose rounding error is eps P dt/dx = eps
(C/gamma) rho c at a CFL number C; likewise the scalar flux rho u f carries
the rounding of rho u whatever f is.  The same scales serve both bars:
S1 = max(sum|A_v|, sum rho c) and Sinf = max(max|A_v|, max rho c) for a
momentum; S1 = max(sum|A_v|, sum rho), Sinf = max(max|A_v|, max rho) for a
scalar.

Every comparison records its worst values under the running test's name;
the suite prints them at the end (tests/conftest.py).
"""
import os

import numpy as np

# per-step bars (FP64 / FP32)
L1_TOL = {64: 1e-12, 32: 2e-5}
ELEM_TOL = {64: 1e-11, 32: 1e-4}

WORST = {}


def _test_name():
    t = os.environ.get("PYTEST_CURRENT_TEST", "?")
    return t.split(" ")[0]


def scales(A, dim, gamma):
    """(S1, Sinf) per component of the oracle state A (shape (nv, ...))."""
    A = np.asarray(A, dtype=np.float64)
    nv = A.shape[0]
    rho = A[0]
    ke = 0.5 * sum(A[1 + d] ** 2 for d in range(dim)) / rho
    p = np.maximum((gamma - 1) * (A[1 + dim] - ke), 0.0)
    rc = np.sqrt(gamma * p * rho)
    s1, sinf = [], []
    for v in range(nv):
        a1, ainf = np.abs(A[v]).sum(), np.abs(A[v]).max()
        if 1 <= v <= dim:
            a1, ainf = max(a1, rc.sum()), max(ainf, rc.max())
        elif v > 1 + dim:
            a1, ainf = max(a1, np.abs(rho).sum()), max(ainf, np.abs(rho).max())
        s1.append(a1)
        sinf.append(ainf)
    return np.array(s1), np.array(sinf)


def errors(A, B, dim, gamma):
    """(relative L1, relative max) per component of B against A."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    assert A.shape == B.shape, (A.shape, B.shape)
    s1, sinf = scales(A, dim, gamma)
    d = np.abs(B - A).reshape(A.shape[0], -1)
    return d.sum(axis=1) / s1, d.max(axis=1) / sinf


def check(A, B, dim, gamma, precision=64, l1=None, elem=None, label=""):
    """Assert both bars (defaults: the per-step bars of `precision`) and
    record the worst values; returns (rel L1, rel max) per component."""
    l1 = L1_TOL[precision] if l1 is None else l1
    elem = ELEM_TOL[precision] if elem is None else elem
    e1, em = errors(A, B, dim, gamma)
    key = _test_name()
    w = WORST.setdefault(key, [0.0, 0.0, l1, elem])
    w[0] = max(w[0], float(e1.max()))
    w[1] = max(w[1], float(em.max()))
    w[2] = max(w[2], l1)
    w[3] = max(w[3], elem)
    assert np.all(e1 <= l1), ("relative L1 above %g" % l1, label, e1)
    assert np.all(em <= elem), ("element-wise error above %g of the component's scale" % elem, label, em)
    return e1, em
