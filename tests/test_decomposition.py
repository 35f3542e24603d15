"""Domain decomposition of the oracle (CPU): a grid cut into slabs along one
axis, stepped with exchanged ghost layers, equals the whole grid bit for bit.

The paper runs one subdomain per MPI process, with ghost layers exchanged
between neighbouring subdomains and a global reduction of the time step
(Sect. 3.3.1; App. B).  A slab's cut sides carry the neighbour's two boundary
layers as ghosts and the neighbour's cells' geometry, so every cell does the
arithmetic it does in the whole grid; the global time step is the minimum of
the slabs' (a maximum of signal speeds, independent of order); a monopole
(Eq. 4) on a grid cut along r starts each slab's enclosed-mass sum at the
running sum of the slabs inside it, which is the whole grid's sum at that
radius.  So the split run must reproduce the whole run exactly:

- in one process, 2-3 slabs along z (Cartesian 3D: transmissive and
  periodic z, with reflective and periodic walls on the other axes), along
  x (2D), and along r of a spherical wedge with point-mass + monopole
  gravity and scalars;
- as two gloo ranks on CPU, one slab each, halos and shell masses as
  messages, the time step as an all-reduce.

Face coordinates are multiples of a power of two where a periodic axis is
cut (the ghosts across a periodic end sit at the first face minus the widths
of the last cells, a computation that is exact only then); the wedge's
log-spaced radii are cut inside the grid, where the ghost faces are the grid's
own.
"""
import os
import socket

import numpy as np

import oracle as O
from paper_2503_04428_gb300 import workloads as wl


def _slab(n, world, rank):
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _beyond(f, side, lo, hi):
    """Two faces beyond a cut, nearest first (periodic ends: the wrapped
    ghosts' positions, first face minus the last widths and vice versa)."""
    n = len(f) - 1
    out = []
    for k in (1, 2):
        i = lo - k if side == 0 else hi + k
        if 0 <= i <= n:
            out.append(f[i])
        elif i < 0:
            prev = out[-1] if out else f[0]
            out.append(prev - (f[i + n + 1] - f[i + n]))
        else:
            prev = out[-1] if out else f[n]
            out.append(prev + (f[i - n] - f[i - n - 1]))
    return np.array(out)


def _cut_sides(case, axis, world, rank):
    n = case["n"][axis]
    lo, hi = _slab(n, world, rank)
    periodic = case["bc"][axis][0] == O.PERIODIC
    f = np.asarray(case["faces"][axis])
    cuts = []
    if rank > 0 or periodic:
        cuts.append((0, _beyond(f, 0, lo, hi), (rank - 1) % world))
    if rank < world - 1 or periodic:
        cuts.append((1, _beyond(f, 1, lo, hi), (rank + 1) % world))
    return (lo, hi), cuts


def _slab_solver(case, axis, world, rank):
    (lo, hi), cuts = _cut_sides(case, axis, world, rank)
    dim = case["dim"]
    faces = [np.asarray(case["faces"][d]) for d in range(dim)]
    faces[axis] = faces[axis][lo:hi + 1]
    n = [case["n"][d] for d in range(dim)]
    n[axis] = hi - lo
    bc = [tuple(case["bc"][d]) for d in range(dim)]
    if case["bc"][axis][0] == O.PERIODIC:
        bc[axis] = (O.TRANSMISSIVE, O.TRANSMISSIVE)
    s = O.Solver(dim, n, faces, bc, case["coords"], case["gamma"], case["n_scalars"], case["riemann"],
                 case["limiter"])
    if case.get("sources"):
        s.set_sources(**case["sources"])
    for side, gf, _ in cuts:
        s.set_exchange(axis, side, gf)
    sl = [slice(None)] * 4
    sl[3 - axis] = slice(lo, hi)
    s.set_state(case["U"][tuple(sl)])
    return s, cuts


def _split_run(case, axis, world, nsteps):
    slabs = [_slab_solver(case, axis, world, r) for r in range(world)]
    mono = bool(case.get("sources")) and case["sources"].get("gravity") == O.GRAV_POINT_MONOPOLE
    for _ in range(nsteps):
        dt = min(s.cfl_dt(case["cfl"]) for s, _ in slabs)
        bnd = [{side: s.get_boundary(axis, side) for side, _, _ in cuts} for s, cuts in slabs]
        for r, (s, cuts) in enumerate(slabs):
            for side, _, nb in cuts:
                s.set_halo(axis, side, bnd[nb][1 - side])
        if mono:
            inner = 0.0
            for s, _ in slabs:
                s.set_inner_mass(inner)
                for m in s.shell_masses():
                    inner += m
        for s, _ in slabs:
            s.step(dt)
    return np.concatenate([s.get_state() for s, _ in slabs], axis=3 - axis)


def _whole_run(case, nsteps):
    s = O.solver_from_case(case)
    for _ in range(nsteps):
        s.step(s.cfl_dt(case["cfl"]))
    return s.get_state()


def _dyadic(case):
    """The same case on faces that are multiples of 2^-k (exact widths)."""
    out = dict(case)
    out["faces"] = [np.round(np.asarray(f) * 1024.0) / 1024.0 for f in case["faces"]]
    return out


def test_cartesian_3d_slabs_along_z():
    for bc, world in (([(O.REFLECTIVE, O.TRANSMISSIVE), (O.PERIODIC, O.PERIODIC), (O.TRANSMISSIVE, O.TRANSMISSIVE)], 3),
                      ([(O.PERIODIC, O.PERIODIC), (O.REFLECTIVE, O.REFLECTIVE), (O.PERIODIC, O.PERIODIC)], 2),
                      ([(O.PERIODIC, O.PERIODIC), (O.TRANSMISSIVE, O.REFLECTIVE), (O.PERIODIC, O.PERIODIC)], 3)):
        case = _dyadic(wl.smooth_random(3, [12, 10, 17], 1, seed=7, bc=bc, riemann=O.HLLC))
        whole = _whole_run(case, 4)
        split = _split_run(case, 2, world, 4)
        assert np.array_equal(whole, split), np.abs(whole - split).max()


def test_cartesian_2d_slabs_along_x_exact_solver():
    case = _dyadic(wl.smooth_random(2, [30, 14], 0, seed=9, riemann=O.EXACT,
                                    bc=[(O.PERIODIC, O.PERIODIC), (O.REFLECTIVE, O.TRANSMISSIVE)]))
    assert np.array_equal(_whole_run(case, 5), _split_run(case, 0, 3, 5))


def test_spherical_wedge_slabs_along_r_with_monopole():
    case = wl.sphere_state(36, 10, 8, dim=3, rotating=True, r_range=(1.0, 20.0), n_scalars=1,
                           bc=[(O.REFLECTIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                               (O.PERIODIC, O.PERIODIC)])
    case["sources"] = dict(gravity=O.GRAV_POINT_MONOPOLE, G=0.01, Mc=2.0)
    whole = _whole_run(case, 3)
    for world in (2, 3):
        split = _split_run(case, 0, world, 3)
        assert np.array_equal(whole, split), (world, np.abs(whole - split).max())


def test_a_wrong_halo_is_seen():
    """The halo enters the step: a slab given a perturbed neighbour layer
    differs from the whole run (so the equality above is not vacuous)."""
    case = _dyadic(wl.smooth_random(3, [10, 8, 12], 0, seed=3, riemann=O.HLL,
                                    bc=[(O.TRANSMISSIVE, O.TRANSMISSIVE)] * 3))
    s, cuts = _slab_solver(case, 2, 2, 0)
    other, _ = _slab_solver(case, 2, 2, 1)
    halo = other.get_boundary(2, 0)
    s.set_halo(2, 1, halo)
    dt = min(s.cfl_dt(case["cfl"]), other.cfl_dt(case["cfl"]))
    s.step(dt)
    good = s.get_state()
    s2, _ = _slab_solver(case, 2, 2, 0)
    halo[:, 1] *= 1.01  # the second ghost layer only
    s2.set_halo(2, 1, halo)
    s2.step(dt)
    assert not np.array_equal(good, s2.get_state())


# ---- the same over two gloo ranks ----

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, case, axis, nsteps, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s, cuts = _slab_solver(case, axis, world, rank)
    mono = bool(case.get("sources")) and case["sources"].get("gravity") == O.GRAV_POINT_MONOPOLE
    for _ in range(nsteps):
        dt = torch.tensor([s.cfl_dt(case["cfl"])], dtype=torch.float64)
        dist.all_reduce(dt, op=dist.ReduceOp.MIN)
        reqs, recv = [], []
        for side, _, nb in cuts:
            send = torch.from_numpy(s.get_boundary(axis, side))
            reqs.append(dist.isend(send, dst=nb, tag=1 - side))
            r = torch.empty_like(send)
            reqs.append(dist.irecv(r, src=nb, tag=side))
            recv.append((side, r, send))
        for q in reqs:
            q.wait()
        for side, r, _ in recv:
            s.set_halo(axis, side, r.numpy())
        if mono:
            m = torch.from_numpy(s.shell_masses())
            sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
            dist.all_gather(sizes, torch.tensor([len(m)]))
            nmax = int(max(x.item() for x in sizes))
            pad = torch.zeros(nmax, dtype=torch.float64)
            pad[:len(m)] = m
            allm = [torch.empty_like(pad) for _ in range(world)]
            dist.all_gather(allm, pad)
            inner = 0.0
            for r in range(rank):
                for x in allm[r][:int(sizes[r].item())].numpy():
                    inner += float(x)
            s.set_inner_mass(inner)
        s.step(float(dt.item()))
    out[rank] = s.get_state()
    dist.destroy_process_group()


def _gloo_split(case, axis, world, nsteps):
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, case, axis, nsteps, out), nprocs=world, join=True)
        parts = [out[r] for r in range(world)]
    return np.concatenate(parts, axis=3 - axis)


def test_two_gloo_ranks_equal_the_whole_grid():
    case = _dyadic(wl.smooth_random(3, [10, 9, 14], 1, seed=11, riemann=O.HLLC,
                                    bc=[(O.TRANSMISSIVE, O.REFLECTIVE), (O.PERIODIC, O.PERIODIC),
                                        (O.PERIODIC, O.PERIODIC)]))
    assert np.array_equal(_whole_run(case, 3), _gloo_split(case, 2, 2, 3))
    wedge = wl.sphere_state(24, 8, 6, dim=3, rotating=True, r_range=(1.0, 10.0), n_scalars=0,
                            bc=[(O.REFLECTIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                                (O.PERIODIC, O.PERIODIC)])
    wedge["sources"] = dict(gravity=O.GRAV_POINT_MONOPOLE, G=0.01, Mc=2.0)
    assert np.array_equal(_whole_run(wedge, 2), _gloo_split(wedge, 0, 2, 2))
