"""Pins of the oracle's moving grid (Sect. 3.1.1, reading R16).

The paper moves the grid along one axis ("shift the grid ... during the
simulation"; radially, to follow expanding ejecta) without printing the
discretisation.  The reading: every face of that axis moves with one
velocity w; the flux through a moving face is F - w U of the Riemann
solution on the face's path x/t = w; the Hancock predictor uses those fluxes
along the moving axis; face areas are averaged over the step; a cell's
content is spread over its new volume.  What fixes it independently of the
code:

- w = 0 is the fixed grid, bit for bit;
- Galilean invariance (Cartesian): a step on a grid moving with w equals the
  fixed-grid step of the same state seen from the moving frame (every
  velocity minus w), seen back from the lab frame -- up to rounding, for
  HLL, HLLC and the exact solver, along every axis;
- the geometric conservation law (spherical): a uniform gas at rest stays
  uniform while the radial faces move, because the averaged radial areas make
  the swept volumes add up to the change of every cell volume;
- conservation (spherical): the mass inside the moving grid changes exactly
  by the boundary fluxes, which for a gas at rest at both ends are
  -w rho through the moving faces.
"""
import math

import numpy as np

import oracle as O
from paper_2503_04428_gb300 import workloads as wl


def _boost(case, w, axis):
    """The same state with the axis-velocity shifted by w (conserved form)."""
    U = case["U"].copy()
    dim = case["dim"]
    rho = U[0]
    u = U[1 + axis] / rho
    U[1 + dim] = U[1 + dim] + rho * w * u + 0.5 * rho * w * w
    U[1 + axis] = U[1 + axis] + rho * w
    return dict(case, U=U)


def test_zero_velocity_is_the_fixed_grid():
    case = wl.smooth_random(2, [30, 22], 1, seed=4, riemann=O.HLLC)
    a = O.solver_from_case(case)
    b = O.solver_from_case(dict(case, moving=(0, 0.0)))
    for _ in range(3):
        dt = a.cfl_dt(0.4)
        a.step(dt)
        b.step(dt)
    assert np.array_equal(a.get_state(), b.get_state())


def test_galilean_invariance_cartesian():
    for dim, n, axis, riemann, bc in (
            (1, [80], 0, O.EXACT, [(O.TRANSMISSIVE, O.TRANSMISSIVE)]),
            (1, [64], 0, O.HLL, [(O.PERIODIC, O.PERIODIC)]),
            (2, [26, 20], 1, O.HLLC, [(O.PERIODIC, O.PERIODIC), (O.TRANSMISSIVE, O.TRANSMISSIVE)]),
            (3, [12, 10, 14], 2, O.HLLC, [(O.REFLECTIVE, O.TRANSMISSIVE), (O.PERIODIC, O.PERIODIC),
                                          (O.PERIODIC, O.PERIODIC)]),
            (3, [14, 9, 11], 0, O.EXACT, [(O.TRANSMISSIVE, O.TRANSMISSIVE), (O.PERIODIC, O.PERIODIC),
                                          (O.REFLECTIVE, O.REFLECTIVE)])):
        base = wl.smooth_random(dim, n, 1, seed=20 + dim, bc=bc, riemann=riemann)
        w = 0.37
        moving = O.solver_from_case(dict(base, moving=(axis, w)))
        # the same flow seen from the frame that moves with the faces
        frame = O.solver_from_case(_boost(base, -w, axis))
        elapsed = 0.0
        for _ in range(3):
            dt = moving.cfl_dt(0.4)
            assert abs(dt - frame.cfl_dt(0.4)) <= 1e-13 * dt  # |u - w| + c, the same speeds
            moving.step(dt)
            frame.step(dt)
            elapsed += dt
        back = _boost(dict(base, U=frame.get_state()), w, axis)["U"]
        got = moving.get_state()
        scale = np.abs(back).reshape(back.shape[0], -1).max(axis=1)
        err = (np.abs(got - back).reshape(back.shape[0], -1).max(axis=1) / scale).max()
        assert err <= 1e-13, (dim, axis, riemann, err)
        # the faces moved by w times the elapsed time
        f0 = np.asarray(base["faces"][axis])
        assert np.allclose(moving.faces(axis), f0 + w * elapsed, rtol=0, atol=1e-14)


def _sph_uniform(nr, dim, r_range=(1.0, 3.0)):
    case = wl.sphere_state(nr, 8, 6, dim=dim, uniform=True, r_range=r_range, ph_range=(0.0, 1.0),
                           bc=[(O.TRANSMISSIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                               (O.PERIODIC, O.PERIODIC)][:dim])
    return case


def test_uniform_gas_at_rest_stays_uniform_while_radial_faces_move():
    for dim in (1, 3):
        case = _sph_uniform(40, dim)
        s = O.solver_from_case(dict(case, moving=(0, 0.6)))
        U0 = case["U"]
        for _ in range(6):
            s.step(s.cfl_dt(0.4))
        U = s.get_state()
        scale = np.abs(U0).reshape(U0.shape[0], -1).max(axis=1)
        err = (np.abs(U - U0).reshape(U0.shape[0], -1).max(axis=1) / np.maximum(scale, 1.0)).max()
        assert err <= 1e-13, (dim, err)


def test_mass_changes_by_the_boundary_fluxes_only():
    """A density bump in the middle, gas at rest and uniform at both ends: the
    mass in the moving grid changes only through its two boundary faces,
    by dt w (rho_out S_out - rho_in S_in), S the areas averaged over the step."""
    nr = 60
    rf = np.linspace(1.0, 4.0, nr + 1)
    rc = 0.5 * (rf[1:] + rf[:-1])
    rho = 1.0 + 0.5 * np.exp(-((rc - 2.5) / 0.3) ** 2)
    U = wl.conserved(5.0 / 3.0, rho, [np.zeros(nr)], np.ones(nr)).reshape(3, 1, 1, nr)
    case = dict(name="bump", dim=1, n=[nr, 1, 1], faces=[rf], bc=[(O.TRANSMISSIVE, O.TRANSMISSIVE)],
                coords=O.SPHERICAL, gamma=5.0 / 3.0, n_scalars=0, riemann=O.HLLC, limiter=O.MINMOD,
                cfl=0.4, sources=None, U=U)
    w = 0.25
    s = O.solver_from_case(dict(case, moving=(0, w)))

    def mass():
        f = s.faces(0)
        vol = 4.0 * math.pi / 3.0 * (f[1:] ** 3 - f[:-1] ** 3)
        return float((s.get_state()[0, 0, 0] * vol).sum()), f

    m0, f0 = mass()
    dt = s.cfl_dt(0.4)
    s.step(dt)
    m1, f1 = mass()
    D = w * dt
    sbar = lambda r: 4.0 * math.pi * (r * r + r * D + D * D / 3.0)
    r_in, r_out = U[0, 0, 0, 0], U[0, 0, 0, -1]  # the edge densities (the bump's tails are ~1e-11)
    expected = m0 + dt * w * (r_out * sbar(f0[-1]) - r_in * sbar(f0[0]))
    assert np.allclose(f1, f0 + D, rtol=0, atol=1e-14)
    assert abs(m1 - expected) <= 1e-14 * m0, (m1, expected)
