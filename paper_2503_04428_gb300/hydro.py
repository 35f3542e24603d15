"""ctypes binding of ``libhydro.so`` (the C ABI of ``include/hydro.h``).

Argument marshalling only: every step of the cell update runs in the
library's CUDA kernels.  The functions keep the C names (``hydro_create``,
``hydro_set_state``, ...); :class:`Grid` and :class:`Batch` wrap a handle for
convenience.  Arrays may be numpy arrays (host memory) or CUDA torch tensors
(device memory, passed by ``data_ptr()``).  If the library is missing the
import fails loudly: there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhydro.so")

HYDRO_OK = 0
HYDRO_ERR_ARG, HYDRO_ERR_CUDA, HYDRO_ERR_NEGATIVE_STATE, HYDRO_ERR_NONFINITE = -1, -2, -3, -4
HYDRO_ERR_NEWTON, HYDRO_ERR_TIMEOUT, HYDRO_ERR_OOM, HYDRO_ERR_VACUUM, HYDRO_ERR_UNSUPPORTED = -5, -6, -7, -8, -9
HYDRO_PERIODIC, HYDRO_TRANSMISSIVE, HYDRO_REFLECTIVE = 0, 1, 2
HYDRO_CARTESIAN, HYDRO_SPHERICAL = 0, 1
HYDRO_HLL, HYDRO_HLLC, HYDRO_EXACT = 0, 1, 2
HYDRO_FIRST_ORDER, HYDRO_MINMOD, HYDRO_VANLEER, HYDRO_VANALBADA = 0, 1, 2, 3
HYDRO_GRAV_NONE, HYDRO_GRAV_UNIFORM, HYDRO_GRAV_POINT, HYDRO_GRAV_POINT_MONOPOLE = 0, 1, 2, 3
HYDRO_HEAT_NONE, HYDRO_HEAT_CONST, HYDRO_HEAT_NI56 = 0, 1, 2
HYDRO_HOST, HYDRO_DEVICE = 0, 1
HYDRO_GUESS_TORO, HYDRO_GUESS_MLP = 0, 1
HYDRO_MAX_SCALARS = 3
HYDRO_MLP_NPARAM = 4673
HYDRO_NOALLOC_MAX_SAMPLES = 16384


class hydro_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("faces", C.POINTER(C.c_double) * 3),
                ("bc", (C.c_int * 2) * 3)]


class hydro_eos(C.Structure):
    _fields_ = [("gamma", C.c_double), ("n_scalars", C.c_int)]


class hydro_stats_t(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("faces", C.c_longlong), ("newton_iters", C.c_longlong),
                ("fallbacks", C.c_longlong), ("mlp_faces", C.c_longlong), ("t", C.c_double),
                ("last_dt", C.c_double), ("tile_x", C.c_int), ("tile_y", C.c_int),
                ("zchunk", C.c_int), ("threads", C.c_int), ("tuned_us_per_step", C.c_double),
                ("newton_faces", C.c_longlong * 3), ("newton_iters_by", C.c_longlong * 3)]


class HydroError(RuntimeError):
    def __init__(self, status, func, msg):
        super().__init__("%s failed (status %d): %s" % (func, status, msg))
        self.status = status


_lib = None
_VP = C.c_void_p
_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I = C.POINTER(C.c_int)

_SIGS = {
    "hydro_create": [C.POINTER(hydro_grid), C.c_int, C.POINTER(hydro_eos), C.c_int, C.c_int, C.c_int,
                     _VP, C.POINTER(_VP)],
    "hydro_set_sources": [_VP, C.c_int, _D, C.c_double, C.c_double, C.c_int, _D],
    "hydro_set_state": [_VP, _VP, C.c_int],
    "hydro_get_state": [_VP, _VP, C.c_int],
    "hydro_set_time": [_VP, C.c_double],
    "hydro_cfl_dt": [_VP, C.c_double, _D],
    "hydro_step": [_VP, C.c_double],
    "hydro_run": [_VP, C.c_int, C.c_double, C.c_double, _D],
    "hydro_totals": [_VP, _D],
    "hydro_stats": [_VP, C.POINTER(hydro_stats_t)],
    "hydro_batch_create": [_I, C.c_int, C.POINTER(hydro_eos), C.c_int, C.c_int, C.c_int, _VP,
                           C.POINTER(_VP)],
    "hydro_batch_run": [_VP, C.c_int, C.c_double],
    "hydro_batch_enqueue": [_VP, C.c_int, C.c_double],
    "hydro_harvest_begin": [_VP, C.c_long, C.c_double, C.c_ulonglong],
    "hydro_harvest_get": [_VP, _D, C.c_long, C.POINTER(C.c_long)],
    "hydro_mlp_set": [_VP, _F, C.c_int],
    "hydro_mlp_get": [_VP, _F],
    "hydro_mlp_train": [_VP, _D, _D, C.c_long, C.c_int, C.c_int, C.c_float, C.c_ulonglong, _D],
    "hydro_mlp_loss_grad": [_F, _D, _D, C.c_long, _D, _D],
    "hydro_exact_solve": [_D, _D, C.c_long, C.c_double, C.c_int, _F, C.c_int, _D, _D, _I],
    "hydro_mlp_loss_grad_device": [_VP, _VP, _VP, C.c_long, _VP, _VP, _VP],
    "hydro_destroy": [_VP],
    "hydro_fma_rate": [C.c_int, C.POINTER(C.c_double)],
    "hydro_wait_probe": [C.POINTER(C.c_double)],
    "hydro_set_eos_radiation": [_VP, C.c_double, C.c_double],
    "hydro_set_dual_energy": [_VP, C.c_double],
    "hydro_batch_run_host": [_VP, _VP, _VP, C.c_int, C.c_double, C.c_int],
    "hydro_exact_sample": [_D, _D, C.c_long, C.c_double, C.POINTER(C.c_longlong), _D, C.c_long, _D],
    "hydro_batch_times": [_VP, _D],
    "hydro_set_step_totals": [_VP, C.c_int],
    "hydro_step_totals": [_VP, _D],
    "hydro_batch_set_launch": [_VP, C.c_int, C.c_int, C.c_int],
    "hydro_set_exchange": [_VP, C.c_int, C.c_int, _D],
    "hydro_set_halo": [_VP, C.c_int, C.c_int, _VP, C.c_int],
    "hydro_get_boundary": [_VP, C.c_int, C.c_int, _VP, C.c_int],
    "hydro_shell_masses": [_VP, _D],
    "hydro_set_inner_mass": [_VP, C.c_double],
    "hydro_set_moving_grid": [_VP, C.c_int, C.c_double],
    "hydro_get_faces": [_VP, C.c_int, _D],
    "hydro_last_error": [],
}


def lib():
    """Load libhydro.so (built by ``paper_2503_04428_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhydro.so not found at %s: run __graft_entry__.build() "
                              "(there is no CPU fallback)" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = C.c_int
        L.hydro_destroy.restype = None
        L.hydro_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != HYDRO_OK:
        raise HydroError(st, name, lib().hydro_last_error().decode())
    return st


def _ptr(a):
    """(address, where, dtype) of a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        where = HYDRO_DEVICE if a.is_cuda else HYDRO_HOST
        return a.data_ptr(), where
    return a.ctypes.data, HYDRO_HOST


def _host_address(U, dtype, shape):
    """Address of a C-contiguous host array (numpy, or a CPU torch tensor) of
    the given dtype and shape; anything else is rejected."""
    if hasattr(U, "data_ptr"):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.float32
        if U.is_cuda or U.dtype != want or tuple(U.shape) != tuple(shape) or not U.is_contiguous():
            raise ValueError("need a contiguous CPU tensor of shape %s and dtype %s" % (shape, want))
        return U.data_ptr()
    if (not isinstance(U, np.ndarray) or U.dtype != dtype or U.shape != tuple(shape)
            or not U.flags.c_contiguous):
        raise ValueError("need a C-contiguous array of shape %s and dtype %s" % (shape, np.dtype(dtype).name))
    return U.ctypes.data


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


# ---- C-named functions -----------------------------------------------------

def hydro_create(grid, coords, eos, riemann, limiter, precision, stream):
    h = C.c_void_p()
    _call("hydro_create", C.byref(grid), coords, C.byref(eos), riemann, limiter, precision,
          stream, C.byref(h))
    return h


def hydro_set_sources(h, gravity, g0, G, Mc, heating, heat_params):
    g = (C.c_double * 3)(*g0)
    hp = (C.c_double * 4)(*(list(heat_params) + [0.0] * (4 - len(heat_params))))
    _call("hydro_set_sources", h, gravity, g, G, Mc, heating, hp)


def hydro_set_state(h, ptr, where):
    _call("hydro_set_state", h, ptr, where)


def hydro_get_state(h, ptr, where):
    _call("hydro_get_state", h, ptr, where)


def hydro_set_time(h, t):
    _call("hydro_set_time", h, t)


def hydro_cfl_dt(h, cfl):
    dt = C.c_double()
    _call("hydro_cfl_dt", h, cfl, C.byref(dt))
    return dt.value


def hydro_step(h, dt):
    _call("hydro_step", h, dt)


def hydro_run(h, nsteps, cfl, t_end=0.0):
    t = C.c_double()
    _call("hydro_run", h, nsteps, cfl, t_end, C.byref(t))
    return t.value


def hydro_totals(h, nv):
    out = np.empty(nv)
    _call("hydro_totals", h, out.ctypes.data_as(_D))
    return out


def hydro_stats(h):
    s = hydro_stats_t()
    _call("hydro_stats", h, C.byref(s))
    out = {k: getattr(s, k) for k, _ in hydro_stats_t._fields_}
    for k in ("newton_faces", "newton_iters_by"):
        out[k] = [int(x) for x in out[k]]
    return out


def hydro_batch_create(lengths, eos, riemann, limiter, precision, stream):
    ln = np.ascontiguousarray(lengths, dtype=np.int32)
    h = C.c_void_p()
    _call("hydro_batch_create", ln.ctypes.data_as(_I), len(ln), C.byref(eos), riemann, limiter,
          precision, stream, C.byref(h))
    return h


def hydro_batch_run(h, nsteps, cfl):
    _call("hydro_batch_run", h, nsteps, cfl)


def hydro_harvest_begin(h, capacity, keep_prob, seed):
    _call("hydro_harvest_begin", h, capacity, keep_prob, seed)


def hydro_harvest_get(h, cap):
    out = np.empty((cap, 6))
    n = C.c_long()
    _call("hydro_harvest_get", h, out.ctypes.data_as(_D), cap, C.byref(n))
    return out[:n.value].copy()


def hydro_mlp_set(h, weights, enable):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _call("hydro_mlp_set", h, w.ctypes.data_as(_F), int(enable))


def hydro_mlp_get(h):
    w = np.empty(HYDRO_MLP_NPARAM, dtype=np.float32)
    _call("hydro_mlp_get", h, w.ctypes.data_as(_F))
    return w


def hydro_mlp_train(h, faces6, log_pstar, epochs, batch, lr, seed):
    f = np.ascontiguousarray(faces6, dtype=np.float64).reshape(-1, 6)
    t = np.ascontiguousarray(log_pstar, dtype=np.float64)
    loss = C.c_double()
    _call("hydro_mlp_train", h, f.ctypes.data_as(_D), t.ctypes.data_as(_D), len(t), epochs, batch,
          lr, seed, C.byref(loss))
    return loss.value


def hydro_mlp_loss_grad(weights, x6, target):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    x = np.ascontiguousarray(x6, dtype=np.float64).reshape(-1, 6)
    t = np.ascontiguousarray(target, dtype=np.float64)
    g = np.empty(HYDRO_MLP_NPARAM)
    loss = C.c_double()
    _call("hydro_mlp_loss_grad", w.ctypes.data_as(_F), x.ctypes.data_as(_D), t.ctypes.data_as(_D),
          len(t), g.ctypes.data_as(_D), C.byref(loss))
    return loss.value, g


def hydro_mlp_loss_grad_device(weights, x6, target, n, grad_out, loss_out, stream=None):
    """Allocation-free gradient: every argument is a device address (int), e.g.
    a CUDA tensor's data_ptr(); queued on `stream`, not synchronised."""
    _call("hydro_mlp_loss_grad_device", weights, x6, target, n, grad_out, loss_out, stream)


def hydro_exact_solve(WL, WR, gamma, guess=HYDRO_GUESS_TORO, weights=None, precision=64):
    WL = np.ascontiguousarray(WL, dtype=np.float64).reshape(-1, 3)
    WR = np.ascontiguousarray(WR, dtype=np.float64).reshape(-1, 3)
    n = len(WL)
    ps, us = np.empty(n), np.empty(n)
    it = np.empty(n, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    _call("hydro_exact_solve", WL.ctypes.data_as(_D), WR.ctypes.data_as(_D), n, gamma, guess,
          None if w is None else w.ctypes.data_as(_F), precision, ps.ctypes.data_as(_D),
          us.ctypes.data_as(_D), it.ctypes.data_as(_I))
    return ps, us, it


def hydro_exact_sample(WL, WR, gamma, face_of, xi):
    """Exact Riemann solution (rho, u, P) of face face_of[k] at x/t = xi[k] (FP64, GPU)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64).reshape(-1, 3)
    WR = np.ascontiguousarray(WR, dtype=np.float64).reshape(-1, 3)
    face_of = np.ascontiguousarray(face_of, dtype=np.int64).ravel()
    xi = np.ascontiguousarray(xi, dtype=np.float64).ravel()
    if len(face_of) != len(xi):
        raise ValueError("face_of and xi differ in length")
    W = np.empty((len(xi), 3))
    _call("hydro_exact_sample", WL.ctypes.data_as(_D), WR.ctypes.data_as(_D), len(WL), gamma,
          face_of.ctypes.data_as(C.POINTER(C.c_longlong)), xi.ctypes.data_as(_D), len(xi),
          W.ctypes.data_as(_D))
    return W


def hydro_batch_times(h, ntubes):
    t = np.empty(ntubes)
    _call("hydro_batch_times", h, t.ctypes.data_as(_D))
    return t


HYDRO_FMA_F32X2 = 2


def hydro_fma_rate(precision=64):
    """Measured dense FMA peak of the current GPU in TFLOP/s (64: FP64, 32:
    FP32, HYDRO_FMA_F32X2: paired FP32 FMAs)."""
    out = C.c_double()
    _call("hydro_fma_rate", int(precision), C.byref(out))
    return out.value


def hydro_wait_probe():
    """(status, seconds) of a bounded device wait on an mbarrier that nothing
    completes: HYDRO_ERR_TIMEOUT is the expected status."""
    out = C.c_double()
    st = lib().hydro_wait_probe(C.byref(out))
    return st, out.value


def hydro_destroy(h):
    if h:
        lib().hydro_destroy(h)


# ---- convenience wrappers --------------------------------------------------

class Grid:
    """A grid handle.  State arrays are (nv, nz, ny, nx) in the handle's precision."""

    def __init__(self, dim, n, faces, bc, coords, gamma, n_scalars, riemann, limiter,
                 precision=64, stream=None):
        self.dim, self.precision = dim, precision
        self.n = [int(n[d]) if d < dim else 1 for d in range(3)]
        self.nv = 2 + dim + n_scalars
        self.dtype = np.float64 if precision == 64 else np.float32
        g = hydro_grid()
        g.dim = dim
        self._faces = []
        for d in range(3):
            g.n[d] = self.n[d]
            if d < dim:
                f = np.ascontiguousarray(faces[d], dtype=np.float64)
                self._faces.append(f)
                g.faces[d] = f.ctypes.data_as(_D)
                g.bc[d][0], g.bc[d][1] = bc[d]
        e = hydro_eos(gamma, n_scalars)
        self.h = hydro_create(g, coords, e, riemann, limiter, precision, _stream(stream))

    @classmethod
    def from_case(cls, case, precision=64, stream=None):
        g = cls(case["dim"], case["n"], case["faces"], case["bc"], case["coords"], case["gamma"],
                case["n_scalars"], case["riemann"], case["limiter"], precision, stream)
        if case.get("eos_rad"):
            g.set_eos_radiation(*case["eos_rad"])
        if case.get("dual_energy"):
            g.set_dual_energy(case["dual_energy"])
        src = case.get("sources")
        if src:
            g.set_sources(**src)
        if case.get("moving"):
            g.set_moving_grid(*case["moving"])
        g.set_state(case["U"])
        return g

    @property
    def shape(self):
        return (self.nv, self.n[2], self.n[1], self.n[0])

    def set_sources(self, gravity=HYDRO_GRAV_NONE, g0=(0.0, 0.0, 0.0), G=0.0, Mc=0.0,
                    heating=HYDRO_HEAT_NONE, heat_params=(0.0,)):
        hydro_set_sources(self.h, gravity, g0, G, Mc, heating, heat_params)

    def set_state(self, U):
        if hasattr(U, "data_ptr"):
            p, where = _ptr(U)
            hydro_set_state(self.h, p, where)
        else:
            a = np.ascontiguousarray(U, dtype=self.dtype).reshape(self.shape)
            hydro_set_state(self.h, a.ctypes.data, HYDRO_HOST)

    def get_state(self, out=None):
        if out is not None:
            p, where = _ptr(out)
            hydro_get_state(self.h, p, where)
            return out
        a = np.empty(self.shape, dtype=self.dtype)
        hydro_get_state(self.h, a.ctypes.data, HYDRO_HOST)
        return a

    def set_dual_energy(self, eps):
        """Internal-energy correction of Sect. 2.5 (eps = 0: off)."""
        _call("hydro_set_dual_energy", self.h, float(eps))

    def set_eos_radiation(self, R_gas, a_rad):
        """Gas + radiation EoS (Sect. 2.3 Eq. 6-7); call before set_state."""
        _call("hydro_set_eos_radiation", self.h, R_gas, a_rad)

    def set_time(self, t):
        hydro_set_time(self.h, t)

    def cfl_dt(self, cfl):
        return hydro_cfl_dt(self.h, cfl)

    def step(self, dt):
        hydro_step(self.h, dt)

    def run(self, nsteps, cfl, t_end=0.0):
        return hydro_run(self.h, nsteps, cfl, t_end)

    def totals(self):
        return hydro_totals(self.h, self.nv)

    def set_step_totals(self, on=True):
        """Accumulate the conserved totals inside every later step (hydro_set_step_totals)."""
        _call("hydro_set_step_totals", self.h, 1 if on else 0)

    def step_totals(self):
        """Totals of the current state from the last step's in-step partials (hydro_step_totals)."""
        out = np.empty(self.nv)
        _call("hydro_step_totals", self.h, out.ctypes.data_as(_D))
        return out

    def stats(self):
        return hydro_stats(self.h)

    # --- domain decomposition (Sect. 3.3.1): exchanged sides of one axis ---
    def halo_shape(self, axis):
        """(nv, 2, cross section) of a halo of `axis` (the two other axes, lower fastest)."""
        other = [self.n[d] for d in range(3) if d != axis]
        return (self.nv, 2, other[1], other[0])

    def set_exchange(self, axis, side, ghost_faces):
        gf = np.ascontiguousarray(ghost_faces, dtype=np.float64)
        if gf.shape != (2,):
            raise ValueError("ghost_faces: the two face coordinates beyond the side")
        _call("hydro_set_exchange", self.h, axis, side, gf.ctypes.data_as(_D))

    def set_halo(self, axis, side, halo):
        if hasattr(halo, "data_ptr"):
            p, where = _ptr(halo)
            _call("hydro_set_halo", self.h, axis, side, p, where)
        else:
            a = np.ascontiguousarray(halo, dtype=self.dtype).reshape(self.halo_shape(axis))
            _call("hydro_set_halo", self.h, axis, side, a.ctypes.data, HYDRO_HOST)

    def get_boundary(self, axis, side, out=None):
        if out is not None:
            p, where = _ptr(out)
            _call("hydro_get_boundary", self.h, axis, side, p, where)
            return out
        a = np.empty(self.halo_shape(axis), dtype=self.dtype)
        _call("hydro_get_boundary", self.h, axis, side, a.ctypes.data, HYDRO_HOST)
        return a

    def shell_masses(self):
        out = np.empty(self.n[0])
        _call("hydro_shell_masses", self.h, out.ctypes.data_as(_D))
        return out

    def set_inner_mass(self, mass):
        _call("hydro_set_inner_mass", self.h, float(mass))

    # --- moving grid (Sect. 3.1.1) ---
    def set_moving_grid(self, axis, w):
        _call("hydro_set_moving_grid", self.h, axis, float(w))

    def faces(self, axis):
        out = np.empty(self.n[axis] + 1)
        _call("hydro_get_faces", self.h, axis, out.ctypes.data_as(_D))
        return out

    def close(self):
        if getattr(self, "h", None):
            hydro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A batched-tube handle; the state is (3, total cells)."""

    def __init__(self, lengths, gamma, riemann=HYDRO_EXACT, limiter=HYDRO_MINMOD, precision=64,
                 stream=None):
        self.lengths = np.ascontiguousarray(lengths, dtype=np.int32)
        self.total = int(self.lengths.sum())
        self.precision = precision
        self.dtype = np.float64 if precision == 64 else np.float32
        self.h = hydro_batch_create(self.lengths, hydro_eos(gamma, 0), riemann, limiter, precision,
                                    _stream(stream))

    def set_state(self, U):
        if hasattr(U, "data_ptr"):
            p, where = _ptr(U)
            hydro_set_state(self.h, p, where)
        else:
            a = np.ascontiguousarray(U, dtype=self.dtype).reshape(3, self.total)
            hydro_set_state(self.h, a.ctypes.data, HYDRO_HOST)

    def get_state(self, out=None):
        if out is not None:
            p, where = _ptr(out)
            hydro_get_state(self.h, p, where)
            return out
        a = np.empty((3, self.total), dtype=self.dtype)
        hydro_get_state(self.h, a.ctypes.data, HYDRO_HOST)
        return a

    def run(self, nsteps, cfl):
        hydro_batch_run(self.h, nsteps, cfl)

    def enqueue(self, nsteps, cfl):
        """Queue nsteps steps without waiting (hydro_batch_enqueue); a device
        failure is reported by the next run()."""
        _call("hydro_batch_enqueue", self.h, nsteps, cfl)

    def stats(self):
        return hydro_stats(self.h)

    def run_host(self, U_in, U_out, nsteps, cfl, nparts=0):
        """Copy the host state U_in in, advance nsteps, copy the result to U_out
        (host arrays, pinned for overlap), pipelined over groups of tubes."""
        pin = _host_address(U_in, self.dtype, (3, self.total))
        pout = _host_address(U_out, self.dtype, (3, self.total))
        _call("hydro_batch_run_host", self.h, pin, pout, int(nsteps), float(cfl), int(nparts))

    def set_launch(self, warps_per_cta, item_cells, ctas_per_sm):
        """Fix the launch shape instead of autotuning it (hydro_batch_set_launch)."""
        _call("hydro_batch_set_launch", self.h, int(warps_per_cta), int(item_cells), int(ctas_per_sm))

    def times(self):
        """Simulation time of every tube (each advances at its own CFL step)."""
        return hydro_batch_times(self.h, len(self.lengths))

    def mlp_set(self, weights, enable=True):
        hydro_mlp_set(self.h, weights, enable)

    def mlp_get(self):
        return hydro_mlp_get(self.h)

    def mlp_train(self, faces6, log_pstar, epochs=20, batch=1024, lr=1e-3, seed=4):
        return hydro_mlp_train(self.h, faces6, log_pstar, epochs, batch, lr, seed)

    def harvest_begin(self, capacity, keep_prob, seed):
        hydro_harvest_begin(self.h, capacity, keep_prob, seed)

    def harvest_get(self, cap):
        return hydro_harvest_get(self.h, cap)

    def close(self):
        if getattr(self, "h", None):
            hydro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
