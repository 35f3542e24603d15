"""Seeded synthetic inputs for the hydro cell update (shared by tests, bench and smoke).

Every initial condition here is a definition taken from the paper's setups
(arXiv:2503.04428) or a synthetic stand-in with the same shapes, sizes and
structure.  The module holds none of the solver's arithmetic: it builds grids
and initial conserved states only (E = P/(gamma-1) + rho|u|^2/2 is the
initial-condition definition of Sect. 2.1/2.3 applied once to the input).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), a counter-based generator:
output k of stream `seed` is the SplitMix64 finaliser of seed + k * 0x9E3779B97F4A7C15
(see `splitmix64`).

A case is a dict with keys: name, dim, n (3 ints), faces (list of arrays),
bc (list of (lo, hi)), coords, gamma, n_scalars, riemann, limiter, cfl,
sources (dict or None), U (float64 array (nv, nz, ny, nx)), t_end.
"""
import math

import numpy as np

# Interface constants (values of the C ABI in include/hydro.h)
PERIODIC, TRANSMISSIVE, REFLECTIVE = 0, 1, 2
CARTESIAN, SPHERICAL = 0, 1
HLL, HLLC, EXACT = 0, 1, 2
FIRST_ORDER, MINMOD, VANLEER, VANALBADA = 0, 1, 2, 3
GRAV_NONE, GRAV_UNIFORM, GRAV_POINT, GRAV_POINT_MONOPOLE = 0, 1, 2, 3
HEAT_NONE, HEAT_CONST, HEAT_NI56 = 0, 1, 2

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed, count, offset=0):
    """`count` consecutive 64-bit outputs of SplitMix64 seeded with `seed`.

    State after k draws is seed + k*0x9E3779B97F4A7C15; each output is the
    published finaliser (shift-xor / multiply by 0xBF58476D1CE4E5B9 and
    0x94D049BB133111EB) of that state.
    """
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, count, offset=0):
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def conserved(gamma, rho, vel, p, scalars=()):
    """Stack primitive fields into conserved (rho, rho u_d, E, rho f_s)."""
    ke = 0.5 * rho * sum(v * v for v in vel)
    out = [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + ke] + [rho * f for f in scalars]
    return np.ascontiguousarray(np.stack(out).astype(np.float64))


def _centres(f):
    return 0.5 * (f[1:] + f[:-1])


def _case(name, dim, faces, bc, coords, gamma, n_scalars, riemann, limiter, cfl, U, sources=None,
          t_end=None):
    n = [len(faces[d]) - 1 if d < dim else 1 for d in range(3)]
    nv = 2 + dim + n_scalars
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(nv, n[2], n[1], n[0])
    return dict(name=name, dim=dim, n=n, faces=[np.asarray(f, dtype=np.float64) for f in faces],
                bc=bc, coords=coords, gamma=gamma, n_scalars=n_scalars, riemann=riemann,
                limiter=limiter, cfl=cfl, sources=sources, U=U, t_end=t_end)


# ---------------------------------------------------------------------------
# The five benchmark configurations
# ---------------------------------------------------------------------------

def sod(n=1000, riemann=HLLC, limiter=MINMOD):
    """1D Sod shock tube (App. C.1, Eq. 29): (1,0,1) | (0.125,0,0.1) at x=0.5, gamma 1.4."""
    xf = np.linspace(0.0, 1.0, n + 1)
    x = _centres(xf)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    U = conserved(1.4, rho, [np.zeros(n)], p)
    return _case("sod%d" % n, 1, [xf], [(TRANSMISSIVE, TRANSMISSIVE)], CARTESIAN, 1.4, 0, riemann,
                 limiter, 0.8, U, t_end=0.2)


def rt2d(nx=512, ny=1536, seed=1, riemann=HLLC, limiter=MINMOD):
    """2D Rayleigh-Taylor on [0,0.5]x[0,1.5], g=(0,-0.1), heavy (rho=2) over light (rho=1).

    Interface y=0.75; hydrostatic P = 2.5 + rho g (y-0.75) piecewise; v_y =
    0.01 U(-1,1) within 4 cells of the interface; one scalar = 1 in the heavy
    fluid.  Periodic x, reflective y.  Related to App. C.2 (random-seeded variant).
    """
    xf = np.linspace(0.0, 0.5, nx + 1)
    yf = np.linspace(0.0, 1.5, ny + 1)
    x, y = np.meshgrid(_centres(xf), _centres(yf), indexing="xy")
    g = -0.1
    heavy = y >= 0.75
    rho = np.where(heavy, 2.0, 1.0)
    p = 2.5 + rho * g * (y - 0.75)
    dy = 1.5 / ny
    band = np.abs(y - 0.75) < 4 * dy
    r = uniform01(seed, nx * ny).reshape(ny, nx)
    vy = np.where(band, 0.01 * (2.0 * r - 1.0), 0.0)
    f = np.where(heavy, 1.0, 0.0)
    U = conserved(1.4, rho, [np.zeros_like(x), vy], p, [f])
    src = dict(gravity=GRAV_UNIFORM, g0=(0.0, g, 0.0))
    return _case("rt2d_%dx%d" % (nx, ny), 2, [xf, yf], [(PERIODIC, PERIODIC), (REFLECTIVE, REFLECTIVE)],
                 CARTESIAN, 1.4, 1, riemann, limiter, 0.4, U, sources=src)


def rt2d_single_mode(nx=256, nz=512, riemann=HLLC, limiter=MINMOD):
    """Single-mode 2D Rayleigh-Taylor of App. C.2: x in [-0.5,0.5], z in [-1,1],
    g_z = -0.5, gamma = 1.4, rho = 2 above the interface z = h(x) = h0 cos(kappa x)
    (h0 = 0.01, kappa = 4 pi) and 1 below, smoothed into a tanh of width 0.005;
    hydrostatic P(z) = P0 + int_{-1}^z rho g dz with P0 = 10/7 + 1/4 (integrated
    exactly for the tanh profile); one scalar = 0 below and 1 above (same
    profile).  Periodic x, reflective z (the paper states no boundary kinds).
    Linear theory: amplitude h0 cosh(sqrt(A g kappa) t), Atwood number A = 1/3."""
    xf = np.linspace(-0.5, 0.5, nx + 1)
    zf = np.linspace(-1.0, 1.0, nz + 1)
    x, z = np.meshgrid(_centres(xf), _centres(zf), indexing="xy")
    g, h0, kappa, w = -0.5, 0.01, 4.0 * math.pi, 0.005
    h = h0 * np.cos(kappa * x)
    s = (z - h) / w
    rho = 1.5 + 0.5 * np.tanh(s)

    def lncosh(a):
        a = np.abs(a)
        return a + np.log1p(np.exp(-2.0 * a)) - math.log(2.0)

    # int_{-1}^{z} rho dz = 1.5 (z + 1) + 0.5 w [ln cosh s - ln cosh s(-1)]
    integral = 1.5 * (z + 1.0) + 0.5 * w * (lncosh(s) - lncosh((-1.0 - h) / w))
    p = 10.0 / 7.0 + 0.25 + g * integral
    f = 0.5 + 0.5 * np.tanh(s)
    U = conserved(1.4, rho, [np.zeros_like(x), np.zeros_like(x)], p, [f])
    src = dict(gravity=GRAV_UNIFORM, g0=(0.0, g, 0.0))
    return _case("rt2d_mode_%dx%d" % (nx, nz), 2, [xf, zf], [(PERIODIC, PERIODIC), (REFLECTIVE, REFLECTIVE)],
                 CARTESIAN, 1.4, 1, riemann, limiter, 0.4, U, sources=src)


def sedov3d(n=256, riemann=HLL, limiter=MINMOD):
    """3D Sedov blast on [-1,1]^3: rho=1, p=1e-5, E=1 over the central 2^3 cells (Sect. 4.3 style)."""
    f = np.linspace(-1.0, 1.0, n + 1)
    dx = 2.0 / n
    shape = (n, n, n)
    rho = np.ones(shape)
    p = np.full(shape, 1e-5)
    zero = np.zeros(shape)
    U = conserved(1.4, rho, [zero, zero, zero], p)
    c = n // 2
    U[4, c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] += 1.0 / (8.0 * dx ** 3)
    tb = (TRANSMISSIVE, TRANSMISSIVE)
    return _case("sedov3d_%d" % n, 3, [f, f, f], [tb, tb, tb], CARTESIAN, 1.4, 0, riemann, limiter,
                 0.4, U, t_end=0.05)


def tube_states(ntubes=4096, seed=2):
    """Left/right states of the batched shock tubes, normalised so that c_L c_R = gamma.

    Density ratio log-uniform in [1e-3,1e3], pressure ratio log-uniform in
    [1e-4,1e4], velocity jump uniform in [-2,2]; rho_L = sqrt(r), rho_R =
    1/sqrt(r) (same for p), u_L = -du/2, u_R = +du/2.
    """
    r = uniform01(seed, 3 * ntubes).reshape(3, ntubes)
    r_rho = 10.0 ** (-3.0 + 6.0 * r[0])
    r_p = 10.0 ** (-4.0 + 8.0 * r[1])
    du = -2.0 + 4.0 * r[2]
    WL = np.stack([np.sqrt(r_rho), -0.5 * du, np.sqrt(r_p)], axis=1)
    WR = np.stack([1.0 / np.sqrt(r_rho), 0.5 * du, 1.0 / np.sqrt(r_p)], axis=1)
    return WL, WR


def tube_lengths(ntubes=4096, seed=2, lo=256, hi=8192):
    """Cells per tube, uniform integers in [lo, hi] (a second stream of the same seed)."""
    r = uniform01(seed + 0x5bd1e995, ntubes)
    return (lo + np.floor(r * (hi - lo + 1))).astype(np.int32)


def tubes(ntubes=4096, seed=2, lo=256, hi=8192, gamma=5.0 / 3.0, perturb=0.0, tube_range=None):
    """Batched exact-Riemann workload: ragged SoA (3, total cells), interface at x=0.5 of [0,1].

    perturb > 0 multiplies density and pressure of every cell by
    1 + perturb U(-1,1) (a dense state in which no two neighbours are equal).
    tube_range = (b0, b1) keeps tubes b0..b1-1 of the ntubes-tube set (the
    same tubes and values as in the whole set)."""
    lengths = tube_lengths(ntubes, seed, lo, hi)
    WL, WR = tube_states(ntubes, seed)
    b0, b1 = (0, ntubes) if tube_range is None else (int(tube_range[0]), int(tube_range[1]))
    start = int(lengths[:b0].sum())
    total = int(lengths[b0:b1].sum())
    noise = None
    if perturb > 0:
        noise = 1.0 + perturb * (2.0 * uniform01(seed + 0x68E31DA4, 2 * int(lengths.sum()))
                                 .reshape(2, -1)[:, start:start + total] - 1.0)
    U = np.empty((3, total))
    off = 0
    for b in range(b0, b1):
        nb = int(lengths[b])
        x = (np.arange(nb) + 0.5) / nb
        left = x < 0.5
        rho = np.where(left, WL[b, 0], WR[b, 0])
        u = np.where(left, WL[b, 1], WR[b, 1])
        p = np.where(left, WL[b, 2], WR[b, 2])
        if noise is not None:
            rho = rho * noise[0, off:off + nb]
            p = p * noise[1, off:off + nb]
        U[:, off:off + nb] = conserved(gamma, rho, [u], p)
        off += nb
    return dict(name="tubes%d" % ntubes, lengths=lengths[b0:b1], U=U, gamma=gamma, WL=WL[b0:b1], WR=WR[b0:b1],
                riemann=EXACT, limiter=MINMOD, cfl=0.8)


def partial_jump_faces(n, seed):
    """Riemann problems from the tube-state distribution with partial jumps:
    (W_L, W_L + t (W_R - W_L)) for t uniform in [0, 1), plus the full jumps.
    Used (with harvested faces) as training inputs of the star-pressure guess."""
    WL, WR = tube_states(n, seed)
    t = uniform01(seed + 0x2545F491, n)[:, None]
    full = np.concatenate([WL, WR], axis=1)
    part = np.concatenate([WL, WL + t * (WR - WL)], axis=1)
    return np.concatenate([full, part])


def wedge(nr=1024, nth=128, nph=128, seed=3, riemann=HLLC, limiter=MINMOD):
    """Spherical wedge, supernova-shock-like synthetic stand-in (r, theta, phi).

    Log-spaced r in [1,1000]; theta in [pi/2-pi/12, pi/2+pi/12]; phi in
    [0, pi/6].  G=1, Mc=1; rho = rho0 r^-2 with rho0 = 1/(4 pi 999);
    P = 1e-4 rho G Mc / r; H/He/O mass-fraction shells (O r<10, He 10<=r<100,
    H r>=100); 1e-2 of the binding energy added uniformly per volume in the
    8 innermost shells; density x (1 + 0.005 U(-1,1)).  Reflective inner r and
    angular walls, transmissive outer r; point-mass plus monopole gravity.
    """
    gamma = 5.0 / 3.0
    rf = 10.0 ** (3.0 * np.arange(nr + 1) / nr)
    tf = np.linspace(0.5 * math.pi - math.pi / 12, 0.5 * math.pi + math.pi / 12, nth + 1)
    pf = np.linspace(0.0, math.pi / 6, nph + 1)
    rc = _centres(rf)
    G, Mc = 1.0, 1.0
    rho0 = 1.0 / (4.0 * math.pi * 999.0)
    # binding energy of the full-sphere envelope, FP64, fixed order
    dm = 4.0 * math.pi * rho0 * (rf[1:] - rf[:-1])
    below = np.concatenate([[0.0], np.cumsum(dm)[:-1]])
    Mi = Mc + below + 0.5 * dm
    E_bind = float(np.sum(G * Mi * dm / rc))
    V8 = 4.0 / 3.0 * math.pi * (rf[8] ** 3 - rf[0] ** 3)
    e_inj = 1e-2 * E_bind / V8
    shape = (nph, nth, nr)
    r3 = np.broadcast_to(rc[None, None, :], shape)
    pert = uniform01(seed, nr * nth * nph).reshape(shape)
    rho = rho0 / r3 ** 2 * (1.0 + 0.005 * (2.0 * pert - 1.0))
    p = 1e-4 * rho * G * Mc / r3
    fO = (r3 < 10.0).astype(np.float64)
    fHe = ((r3 >= 10.0) & (r3 < 100.0)).astype(np.float64)
    fH = (r3 >= 100.0).astype(np.float64)
    zero = np.zeros(shape)
    U = conserved(gamma, rho, [zero, zero, zero], p, [fH, fHe, fO])
    U[4, :, :, :8] += e_inj
    src = dict(gravity=GRAV_POINT_MONOPOLE, G=G, Mc=Mc)
    bc = [(REFLECTIVE, TRANSMISSIVE), (REFLECTIVE, REFLECTIVE), (REFLECTIVE, REFLECTIVE)]
    return _case("wedge_%dx%dx%d" % (nr, nth, nph), 3, [rf, tf, pf], bc, SPHERICAL, gamma, 3,
                 riemann, limiter, 0.4, U, sources=src)


# ---------------------------------------------------------------------------
# Test inputs
# ---------------------------------------------------------------------------

def smooth_random(dim, n, n_scalars=0, seed=7, coords=CARTESIAN, bc=None, riemann=HLLC,
                  limiter=MINMOD, gamma=1.4, amp=0.2, faces=None):
    """A random but positive state: rho, p in [1-amp, 1+amp] x ... , |u| < amp + noise.

    Each field is a smooth sinusoid plus per-cell noise, so that every limiter
    branch (smooth, extremum, sign change) occurs.
    """
    n = list(n) + [1] * (3 - len(n))
    if faces is None:
        faces = []
        for d in range(dim):
            # mildly non-uniform spacing exercises the centre-distance slopes
            s = np.arange(n[d] + 1) / n[d]
            faces.append(s + 0.02 * np.sin(2 * math.pi * s) / (2 * math.pi))
    shape = (n[2], n[1], n[0])
    ncell = n[0] * n[1] * n[2]
    nf = 2 + dim + n_scalars
    r = uniform01(seed, nf * ncell).reshape(nf, *shape)
    grids = np.meshgrid(*[np.arange(n[d]) / n[d] for d in (2, 1, 0)], indexing="ij")
    phase = 2 * math.pi * (grids[0] + 2 * grids[1] + 3 * grids[2])
    rho = 1.0 + amp * np.sin(phase) + 0.5 * amp * (2 * r[0] - 1)
    vel = [amp * np.cos(phase + d) + 0.5 * amp * (2 * r[1 + d] - 1) for d in range(dim)]
    p = 1.0 + amp * np.cos(2 * phase) + 0.5 * amp * (2 * r[1 + dim] - 1)
    sc = [0.5 + 0.4 * (2 * r[2 + dim + s] - 1) for s in range(n_scalars)]
    U = conserved(gamma, rho, vel, p, sc)
    if bc is None:
        bc = [(PERIODIC, PERIODIC)] * dim
    return _case("smooth%dd" % dim, dim, faces, bc, coords, gamma, n_scalars, riemann, limiter, 0.4, U)


def advection1d(n=128, riemann=HLLC, limiter=VANLEER):
    """rho = 1 + 0.2 sin(2 pi x), u = 1, p = 1 on a periodic unit interval."""
    xf = np.linspace(0.0, 1.0, n + 1)
    x = _centres(xf)
    U = conserved(1.4, 1.0 + 0.2 * np.sin(2 * math.pi * x), [np.ones(n)], np.ones(n))
    return _case("adv%d" % n, 1, [xf], [(PERIODIC, PERIODIC)], CARTESIAN, 1.4, 0, riemann, limiter, 0.4, U)


def kh2d(nx=64, nz=128, riemann=HLLC, limiter=MINMOD):
    """Kelvin-Helmholtz initial state of Sect. 4.1 (Lecoanet et al. 2016), fully periodic.

    Domain [0,1] x [0,2] (z1=0.5, z2=1.5), a=0.05, sigma=0.2, P0=10, gamma=5/3,
    with a passive scalar marking the shear layer.
    """
    xf = np.linspace(0.0, 1.0, nx + 1)
    zf = np.linspace(0.0, 2.0, nz + 1)
    x, z = np.meshgrid(_centres(xf), _centres(zf), indexing="xy")
    a, s, z1, z2 = 0.05, 0.2, 0.5, 1.5
    prof = np.tanh((z - z1) / a) - np.tanh((z - z2) / a)
    rho = 1.0 + 0.5 * prof
    ux = prof
    uz = 0.01 * np.sin(math.pi * x) * (np.exp(-(z - z1) ** 2 / s ** 2) + np.exp(-(z - z2) ** 2 / s ** 2))
    p = np.full_like(x, 10.0)
    U = conserved(5.0 / 3.0, rho, [ux, uz], p, [0.5 * prof])
    return _case("kh%dx%d" % (nx, nz), 2, [xf, zf], [(PERIODIC, PERIODIC)] * 2, CARTESIAN, 5.0 / 3.0,
                 1, riemann, limiter, 0.4, U)


def liska_wendroff(n=64, riemann=HLLC, limiter=MINMOD, threshold=0.15):
    """Implosion of App. C.3 on [0,0.3]^2, reflective; (1,1) if x+z >= threshold else (0.14,0.125).

    The printed threshold 0.015 is read as 0.15 (Liska & Wendroff 2003).
    """
    f = np.linspace(0.0, 0.3, n + 1)
    x, z = np.meshgrid(_centres(f), _centres(f), indexing="xy")
    outer = x + z >= threshold
    rho = np.where(outer, 1.0, 0.14)
    p = np.where(outer, 1.0, 0.125)
    zero = np.zeros_like(x)
    U = conserved(1.4, rho, [zero, zero], p)
    rb = (REFLECTIVE, REFLECTIVE)
    return _case("lw%d" % n, 2, [f, f], [rb, rb], CARTESIAN, 1.4, 0, riemann, limiter, 0.4, U)


def sedov1d_spherical(n=400, riemann=HLLC, limiter=MINMOD):
    """1D spherical Sedov of App. C.4: r in [0,1], rho=1, E=1e-12, total energy 1 in the first cell."""
    rf = np.linspace(0.0, 1.0, n + 1)
    rho = np.ones(n)
    E = np.full(n, 1e-12)
    dV0 = 4.0 * math.pi / 3.0 * rf[1] ** 3
    E[0] = 1.0 / dV0
    U = np.stack([rho, np.zeros(n), E])
    return _case("sedov1d_sph%d" % n, 1, [rf], [(REFLECTIVE, TRANSMISSIVE)], SPHERICAL, 1.4, 0,
                 riemann, limiter, 0.4, U, t_end=0.7)


def sphere_state(nr=16, nth=12, nph=10, seed=11, rotating=True, riemann=HLLC, limiter=MINMOD,
                 r_range=(1.0, 3.0), th_range=(0.6, 2.4), ph_range=(0.0, 2 * math.pi), n_scalars=0,
                 bc=None, uniform=False, dim=3):
    """A spherical-grid test state (r, theta, phi).  uniform=True gives a static uniform gas."""
    rf = np.linspace(r_range[0], r_range[1], nr + 1)
    tf = np.linspace(th_range[0], th_range[1], nth + 1)
    pf = np.linspace(ph_range[0], ph_range[1], nph + 1)
    faces = [rf, tf, pf][:dim]
    n = [nr, nth, nph][:dim] + [1] * (3 - dim)
    shape = (n[2], n[1], n[0])
    if uniform:
        rho = np.ones(shape)
        p = np.ones(shape)
        vel = [np.zeros(shape) for _ in range(dim)]
    else:
        r = uniform01(seed, 5 * int(np.prod(shape))).reshape(5, *shape)
        rho = 1.0 + 0.3 * r[0]
        p = 1.0 + 0.3 * r[1]
        vel = [0.2 * (2 * r[2 + d] - 1) for d in range(dim)]
        if rotating and dim == 3:
            vel[2] = vel[2] + 0.3
    sc = [np.full(shape, 0.5) for _ in range(n_scalars)]
    U = conserved(5.0 / 3.0, rho, vel, p, sc)
    if bc is None:
        bc = [(REFLECTIVE, REFLECTIVE), (REFLECTIVE, REFLECTIVE), (PERIODIC, PERIODIC)][:dim]
    return _case("sphere%dd" % dim, dim, faces, bc, SPHERICAL, 5.0 / 3.0, n_scalars, riemann, limiter,
                 0.4, U)
