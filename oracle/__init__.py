"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

The oracle is the plain, slow reference of the HERACLES++ cell update
(arXiv:2503.04428, Sect. 2-3) that the GPU library is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the GPU library never does.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

PERIODIC, TRANSMISSIVE, REFLECTIVE = 0, 1, 2
CARTESIAN, SPHERICAL = 0, 1
HLL, HLLC, EXACT = 0, 1, 2
FIRST_ORDER, MINMOD, VANLEER, VANALBADA = 0, 1, 2, 3
GRAV_NONE, GRAV_UNIFORM, GRAV_POINT, GRAV_POINT_MONOPOLE = 0, 1, 2, 3
HEAT_NONE, HEAT_CONST, HEAT_NI56 = 0, 1, 2
GUESS_TORO, GUESS_MLP = 0, 1
MLP_NPARAM = 64 * 6 + 64 + 64 * 64 + 64 + 64 + 1

_lib = None
_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I = C.POINTER(C.c_int)
_LL = C.POINTER(C.c_longlong)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("oracle %s failed with status %d" % (what, status))
        self.status = status


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_create.argtypes = [C.c_int, _I, _D, _I, C.c_int, C.c_double, C.c_int, C.c_int,
                                 C.c_int, C.POINTER(C.c_void_p)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_destroy.restype = None
        L.orc_set_sources.argtypes = [C.c_void_p, C.c_int, _D, C.c_double, C.c_double, C.c_int, _D]
        L.orc_set_guess.argtypes = [C.c_void_p, C.c_int, _F]
        L.orc_set_state.argtypes = [C.c_void_p, _D]
        L.orc_get_state.argtypes = [C.c_void_p, _D]
        L.orc_set_time.argtypes = [C.c_void_p, C.c_double]
        L.orc_cfl_dt.argtypes = [C.c_void_p, C.c_double, _D]
        L.orc_step.argtypes = [C.c_void_p, C.c_double]
        L.orc_totals.argtypes = [C.c_void_p, _D]
        L.orc_stats.argtypes = [C.c_void_p, _LL]
        L.orc_shell_mass.argtypes = [C.c_void_p, _D]
        L.orc_batch_run.argtypes = [_I, C.c_int, _D, C.c_double, C.c_int, C.c_int, C.c_double,
                                    C.c_int, C.c_int, _F, C.c_int, _LL]
        L.orc_limiter.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_limiter.restype = C.c_double
        L.orc_flux_1d.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, _D, _D, _D]
        L.orc_exact_star.argtypes = [C.c_double, _D, _D, C.c_int, _F, _D, _D, _I]
        L.orc_exact_sample.argtypes = [C.c_double, _D, _D, C.c_double, _D]
        L.orc_guess_toro.argtypes = [C.c_double, _D, _D, _I]
        L.orc_guess_toro.restype = C.c_double
        L.orc_mlp_features.argtypes = [C.c_double, _D, _D, _D, _D]
        L.orc_mlp_forward.argtypes = [_F, _D, C.c_long, _D]
        L.orc_mlp_loss_grad.argtypes = [_F, _D, _D, C.c_long, _D]
        L.orc_mlp_loss_grad.restype = C.c_double
        L.orc_adam_step.argtypes = [_F, _F, _F, _D, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_double, C.c_double]
        L.orc_sedov_xi0.argtypes = [C.c_double]
        L.orc_sedov_xi0.restype = C.c_double
        L.orc_heating_rate.argtypes = [C.c_int, _D, C.c_double, C.c_double]
        L.orc_heating_rate.restype = C.c_double
        L.orc_set_eos_radiation.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.orc_set_dual_energy.argtypes = [C.c_void_p, C.c_double]
        L.orc_eos_rad.argtypes = [C.c_double] * 5 + [_D, _D, _D]
        L.orc_eos_rad_eint.argtypes = [C.c_double] * 5 + [_D, _D]
        L.orc_set_exchange.argtypes = [C.c_void_p, C.c_int, C.c_int, _D]
        L.orc_set_halo.argtypes = [C.c_void_p, C.c_int, C.c_int, _D]
        L.orc_get_boundary.argtypes = [C.c_void_p, C.c_int, C.c_int, _D]
        L.orc_shell_masses.argtypes = [C.c_void_p, _D]
        L.orc_set_inner_mass.argtypes = [C.c_void_p, C.c_double]
        L.orc_set_moving_grid.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.orc_get_faces.argtypes = [C.c_void_p, C.c_int, _D]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _fp(a):
    return None if a is None else a.ctypes.data_as(_F)


def _check(st, what):
    if st != 0:
        raise OracleError(st, what)


class Solver:
    """One grid advanced by the oracle.  State arrays are (nv, nz, ny, nx)."""

    def __init__(self, dim, n, faces, bc, coords, gamma, n_scalars, riemann, limiter):
        self.dim = dim
        self.n = [int(n[d]) if d < dim else 1 for d in range(3)]
        self.nv = 2 + dim + n_scalars
        nn = np.array(self.n, dtype=np.int32)
        fc = np.ascontiguousarray(np.concatenate([np.asarray(faces[d], dtype=np.float64)
                                                  for d in range(dim)]))
        b = np.zeros(6, dtype=np.int32)
        for d in range(dim):
            b[2 * d], b[2 * d + 1] = bc[d]
        h = C.c_void_p()
        _check(lib().orc_create(dim, nn.ctypes.data_as(_I), _dp(fc), b.ctypes.data_as(_I), coords,
                                gamma, n_scalars, riemann, limiter, C.byref(h)), "create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    @property
    def shape(self):
        return (self.nv, self.n[2], self.n[1], self.n[0])

    def set_sources(self, gravity=GRAV_NONE, g0=(0.0, 0.0, 0.0), G=0.0, Mc=0.0,
                    heating=HEAT_NONE, heat_params=(0.0, 0.0, 0.0, 0.0)):
        g = np.asarray(g0, dtype=np.float64)
        hp = np.zeros(4)
        hp[:len(heat_params)] = heat_params
        _check(lib().orc_set_sources(self._h, gravity, _dp(g), G, Mc, heating, _dp(hp)), "set_sources")

    def set_eos_radiation(self, R, a):
        """Gas + radiation EoS (Sect. 2.3 Eq. 6-7), HLL/HLLC only."""
        _check(lib().orc_set_eos_radiation(self._h, R, a), "set_eos_radiation")

    def set_dual_energy(self, eps):
        """Dual-energy correction of Sect. 2.5 (eps = 0: off)."""
        _check(lib().orc_set_dual_energy(self._h, eps), "set_dual_energy")

    def set_guess(self, guess, weights=None):
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        self._w = w
        _check(lib().orc_set_guess(self._h, guess, _fp(w)), "set_guess")

    def set_state(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.shape)
        _check(lib().orc_set_state(self._h, _dp(U)), "set_state")

    def get_state(self):
        U = np.empty(self.shape)
        _check(lib().orc_get_state(self._h, _dp(U)), "get_state")
        return U

    def set_time(self, t):
        _check(lib().orc_set_time(self._h, t), "set_time")

    def cfl_dt(self, cfl):
        dt = C.c_double()
        _check(lib().orc_cfl_dt(self._h, cfl, C.byref(dt)), "cfl_dt")
        return dt.value

    def step(self, dt):
        _check(lib().orc_step(self._h, dt), "step")

    def totals(self):
        out = np.empty(self.nv)
        _check(lib().orc_totals(self._h, _dp(out)), "totals")
        return out

    def stats(self):
        out = np.zeros(4, dtype=np.int64)
        _check(lib().orc_stats(self._h, out.ctypes.data_as(_LL)), "stats")
        return dict(faces=int(out[0]), newton_iters=int(out[1]), fallbacks=int(out[2]),
                    mlp_faces=int(out[3]))

    def shell_mass(self):
        out = np.empty(self.n[0])
        _check(lib().orc_shell_mass(self._h, _dp(out)), "shell_mass")
        return out

    # --- domain decomposition (Sect. 3.3.1): exchanged sides of one axis ---
    def halo_shape(self, axis):
        """(nv, 2, cross section) of a halo of `axis` (the two other axes, lower fastest)."""
        other = [self.n[d] for d in range(3) if d != axis]
        return (self.nv, 2, other[1], other[0])

    def set_exchange(self, axis, side, ghost_faces):
        gf = np.ascontiguousarray(ghost_faces, dtype=np.float64)
        assert gf.shape == (2,)
        _check(lib().orc_set_exchange(self._h, axis, side, _dp(gf)), "set_exchange")

    def set_halo(self, axis, side, halo):
        a = np.ascontiguousarray(halo, dtype=np.float64).reshape(self.halo_shape(axis))
        _check(lib().orc_set_halo(self._h, axis, side, _dp(a)), "set_halo")

    def get_boundary(self, axis, side):
        out = np.empty(self.halo_shape(axis))
        _check(lib().orc_get_boundary(self._h, axis, side, _dp(out)), "get_boundary")
        return out

    def shell_masses(self):
        out = np.empty(self.n[0])
        _check(lib().orc_shell_masses(self._h, _dp(out)), "shell_masses")
        return out

    def set_inner_mass(self, mass):
        _check(lib().orc_set_inner_mass(self._h, float(mass)), "set_inner_mass")

    # --- moving grid (Sect. 3.1.1) ---
    def set_moving_grid(self, axis, w):
        _check(lib().orc_set_moving_grid(self._h, axis, float(w)), "set_moving_grid")

    def faces(self, axis):
        out = np.empty(self.n[axis] + 1)
        _check(lib().orc_get_faces(self._h, axis, _dp(out)), "get_faces")
        return out


def solver_from_case(case):
    """Build an oracle solver from a workload case (see the package's workloads module)."""
    s = Solver(case["dim"], case["n"], case["faces"], case["bc"], case["coords"], case["gamma"],
               case["n_scalars"], case["riemann"], case["limiter"])
    if case.get("eos_rad"):
        s.set_eos_radiation(*case["eos_rad"])
    if case.get("dual_energy"):
        s.set_dual_energy(case["dual_energy"])
    src = case.get("sources")
    if src:
        s.set_sources(**src)
    if case.get("moving"):
        s.set_moving_grid(*case["moving"])
    s.set_state(case["U"])
    return s


def batch_run(lengths, U, gamma, riemann, limiter, cfl, nsteps, guess=GUESS_TORO, weights=None,
              nthreads=0):
    """Advance concatenated tubes (U is (3, total) float64, modified copy returned)."""
    lengths = np.ascontiguousarray(lengths, dtype=np.int32)
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    st = np.zeros(4, dtype=np.int64)
    _check(lib().orc_batch_run(lengths.ctypes.data_as(_I), len(lengths), _dp(U), gamma, riemann,
                               limiter, cfl, nsteps, guess, _fp(w), nthreads,
                               st.ctypes.data_as(_LL)), "batch_run")
    return U, dict(faces=int(st[0]), newton_iters=int(st[1]), fallbacks=int(st[2]),
                   mlp_faces=int(st[3]))


def eos_rad(gamma, R, a, rho, e):
    """Gas + radiation EoS from (rho, e): (T, P, c)."""
    T, P, c = C.c_double(), C.c_double(), C.c_double()
    _check(lib().orc_eos_rad(gamma, R, a, rho, e, C.byref(T), C.byref(P), C.byref(c)), "eos_rad")
    return T.value, P.value, c.value


def eos_rad_eint(gamma, R, a, rho, P):
    """Gas + radiation EoS from (rho, P): (T, e)."""
    T, e = C.c_double(), C.c_double()
    _check(lib().orc_eos_rad_eint(gamma, R, a, rho, P, C.byref(T), C.byref(e)), "eos_rad_eint")
    return T.value, e.value


def limiter(kind, dm, dp):
    return lib().orc_limiter(kind, dm, dp)


def flux_1d(riemann, gamma, UL, UR, n_scalars=0, dim=1):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.empty_like(UL)
    _check(lib().orc_flux_1d(riemann, gamma, n_scalars, dim, _dp(UL), _dp(UR), _dp(F)), "flux_1d")
    return F


def exact_star(gamma, WL, WR, guess=GUESS_TORO, weights=None):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    ps, us, it = C.c_double(), C.c_double(), C.c_int()
    _check(lib().orc_exact_star(gamma, _dp(WL), _dp(WR), guess, _fp(w), C.byref(ps), C.byref(us),
                                C.byref(it)), "exact_star")
    return ps.value, us.value, it.value


def exact_sample(gamma, WL, WR, xi):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    out = np.empty(3)
    _check(lib().orc_exact_sample(gamma, _dp(WL), _dp(WR), xi, _dp(out)), "exact_sample")
    return out


def guess_toro(gamma, WL, WR):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    k = C.c_int()
    p = lib().orc_guess_toro(gamma, _dp(WL), _dp(WR), C.byref(k))
    return p, k.value


def mlp_features(gamma, WL, WR):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    x = np.empty(6)
    pref = C.c_double()
    _check(lib().orc_mlp_features(gamma, _dp(WL), _dp(WR), _dp(x), C.byref(pref)), "mlp_features")
    return x, pref.value


def mlp_forward(weights, X):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 6)
    y = np.empty(len(X))
    _check(lib().orc_mlp_forward(_fp(w), _dp(X), len(X), _dp(y)), "mlp_forward")
    return y


def mlp_loss_grad(weights, X, T):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 6)
    T = np.ascontiguousarray(T, dtype=np.float64)
    g = np.empty(MLP_NPARAM)
    loss = lib().orc_mlp_loss_grad(_fp(w), _dp(X), _dp(T), len(X), _dp(g))
    return loss, g


def adam_step(w, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    w = np.array(w, dtype=np.float32)
    m = np.array(m, dtype=np.float32)
    v = np.array(v, dtype=np.float32)
    g = np.ascontiguousarray(grad, dtype=np.float64)
    _check(lib().orc_adam_step(_fp(w), _fp(m), _fp(v), _dp(g), len(w), step, lr, beta1, beta2, eps),
           "adam_step")
    return w, m, v


def sedov_xi0(gamma):
    return lib().orc_sedov_xi0(gamma)


def heating_rate(kind, params, t, rho_f_ni):
    p = np.zeros(4)
    p[:len(params)] = params
    return lib().orc_heating_rate(kind, _dp(p), t, rho_f_ni)
