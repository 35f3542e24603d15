"""Slab decomposition of one grid over several processes (one GPU each).

The paper distributes a grid as MPI subdomains, one per process, with ghost
layers exchanged between neighbouring subdomains every step and a global
reduction of the time step (Sect. 3.3.1; the weak-scaling runs of App. B).
Here a grid is cut along one axis into contiguous slabs, one per rank of a
torch.distributed process group.  Each rank holds its slab in a library
handle whose cut sides are marked as exchanged (hydro_set_exchange); before
every step the ranks

  1. send the two boundary layers at each cut side to the neighbour across
     it (hydro_get_boundary) and install the neighbour's as their halo
     (hydro_set_halo), through point-to-point messages;
  2. with monopole gravity (Eq. 4) on a grid cut along r, gather every
     slab's shell masses and start each slab's enclosed-mass sum at the mass
     of the slabs inside it (hydro_shell_masses, hydro_set_inner_mass);
  3. take the minimum of the slabs' CFL time steps (an all-reduce);

and then advance one step (hydro_step).  With the gloo backend the halos
travel through host memory; with NCCL they are device tensors.  The slab of
a rank is the same arithmetic, cell for cell, as the whole grid: the ghosts
of a cut side carry the neighbour's values and geometry.
"""
import numpy as np

from . import hydro as H


def slab_range(n, world, rank):
    """Cells [lo, hi) of `rank` when n cells are cut into `world` slabs (the
    first n % world slabs take one cell more)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def ghost_faces(f, side, lo, hi, periodic):
    """The two face coordinates beyond side `side` of the slab [lo, hi) of
    an axis with faces f (n + 1 values), nearest first.  Across a periodic
    end they are the positions of the wrapped cells' ghosts: the first face
    minus the widths of the last cells (or the last face plus those of the
    first cells)."""
    n = len(f) - 1
    out = []
    for k in (1, 2):
        i = lo - k if side == 0 else hi + k
        if 0 <= i <= n:
            out.append(f[i])
        elif not periodic:
            raise ValueError("a non-periodic end is not cut")
        elif i < 0:
            out.append(out[-1] - (f[i + n + 1] - f[i + n]) if out else f[0] - (f[n] - f[n - 1]))
        else:
            out.append(out[-1] + (f[i - n] - f[i - n - 1]) if out else f[n] + (f[1] - f[0]))
    return np.array(out, dtype=np.float64)


def slab_case(case, axis, world, rank):
    """This rank's slab of a workload case: faces, state and boundary kinds
    of the slab, and its cut sides as (side, the two face coordinates beyond
    it, neighbour rank).  A periodic axis is cut on both ends of every slab;
    a non-periodic axis keeps its boundary kinds at the ends of the grid."""
    n = case["n"][axis]
    lo, hi = slab_range(n, world, rank)
    if hi - lo < 2:
        raise ValueError("every slab needs at least 2 cells along the cut axis")
    f = np.asarray(case["faces"][axis], dtype=np.float64)
    periodic = case["bc"][axis][0] == H.HYDRO_PERIODIC
    faces = list(case["faces"])
    faces[axis] = f[lo:hi + 1].copy()
    bc = [tuple(b) for b in case["bc"]]
    cuts = []
    if world > 1 and (rank > 0 or periodic):
        cuts.append((0, ghost_faces(f, 0, lo, hi, periodic), (rank - 1) % world))
    if world > 1 and (rank < world - 1 or periodic):
        cuts.append((1, ghost_faces(f, 1, lo, hi, periodic), (rank + 1) % world))
    if periodic and world > 1:
        # both ends of every slab are cut: a placeholder kind until the
        # exchange replaces it
        bc[axis] = (H.HYDRO_TRANSMISSIVE, H.HYDRO_TRANSMISSIVE)
    sl = [slice(None)] * 4
    sl[3 - axis] = slice(lo, hi)
    sub = dict(case)
    sub.update(n=[hi - lo if d == axis else case["n"][d] for d in range(len(case["n"]))], faces=faces, bc=bc,
               U=np.ascontiguousarray(case["U"][tuple(sl)]))
    return sub, cuts, (lo, hi)


class SlabRun:
    """One rank's slab of a grid cut along `axis`, stepped in lockstep with
    the other ranks of `group` (default: the whole world)."""

    def __init__(self, case, axis, precision=64, group=None, stream=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.axis = axis
        sub, self.cuts, self.range = slab_case(case, axis, self.world, self.rank)
        self.grid = H.Grid(sub["dim"], sub["n"], sub["faces"], sub["bc"], sub["coords"], sub["gamma"],
                           sub["n_scalars"], sub["riemann"], sub["limiter"], precision, stream)
        if sub.get("eos_rad"):
            self.grid.set_eos_radiation(*sub["eos_rad"])
        if sub.get("dual_energy"):
            self.grid.set_dual_energy(sub["dual_energy"])
        src = sub.get("sources")
        self.monopole = bool(src) and src.get("gravity") == H.HYDRO_GRAV_POINT_MONOPOLE
        if self.monopole and axis != 0:
            raise ValueError("monopole gravity needs whole shells on every rank: cut along r (axis 0)")
        if src:
            self.grid.set_sources(**src)
        for side, beyond, _ in self.cuts:
            self.grid.set_exchange(axis, side, beyond)
        self.grid.set_state(sub["U"])
        self.backend = dist.get_backend(group)

    def _tensor(self, a):
        import torch
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.cuda() if self.backend == "nccl" else t

    def exchange_halos(self):
        """Send the boundary layers at every cut side to the neighbour across
        it and install the neighbour's as the halo of that side (message tag
        = the receiving side)."""
        import torch
        reqs, recv = [], []
        g = self.grid
        for side, _, nb in self.cuts:
            buf = self._tensor(g.get_boundary(self.axis, side))
            reqs.append(self.dist.isend(buf, dst=self._global(nb), group=self.group, tag=1 - side))
            r = torch.empty_like(buf)
            reqs.append(self.dist.irecv(r, src=self._global(nb), group=self.group, tag=side))
            recv.append((side, r, buf))
        for q in reqs:
            q.wait()
        for side, r, _ in recv:
            g.set_halo(self.axis, side, r if r.is_cuda else r.numpy())

    def _global(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def exchange_mass(self):
        """Monopole on an r-cut grid: start this slab's enclosed-mass sum at
        the mass of every slab inside it (summed in radial order)."""
        import torch
        m = self.grid.shell_masses()
        n = torch.tensor([len(m)], dtype=torch.int64)
        counts = [torch.zeros(1, dtype=torch.int64) for _ in range(self.world)]
        if self.backend == "nccl":
            n, counts = n.cuda(), [c.cuda() for c in counts]
        self.dist.all_gather(counts, n, group=self.group)
        nmax = int(max(int(c.item()) for c in counts))
        pad = np.zeros(nmax)
        pad[:len(m)] = m
        mine = self._tensor(pad)
        allm = [torch.empty_like(mine) for _ in range(self.world)]
        self.dist.all_gather(allm, mine, group=self.group)
        inner = 0.0
        for r in range(self.rank):
            for x in allm[r][:int(counts[r].item())].cpu().numpy():
                inner += float(x)
        self.grid.set_inner_mass(inner)

    def cfl_dt(self, cfl):
        """The minimum over all slabs of cfl / max sum_d (|u_d|+c)/h_d."""
        import torch
        dt = torch.tensor([self.grid.cfl_dt(cfl)], dtype=torch.float64)
        if self.backend == "nccl":
            dt = dt.cuda()
        self.dist.all_reduce(dt, op=self.dist.ReduceOp.MIN, group=self.group)
        return float(dt.item())

    def step(self, dt):
        self.exchange_halos()
        if self.monopole:
            self.exchange_mass()
        self.grid.step(dt)

    def run(self, nsteps, cfl):
        """nsteps steps of the global CFL time step."""
        for _ in range(nsteps):
            self.step(self.cfl_dt(cfl))

    def get_state(self):
        return self.grid.get_state()

    def close(self):
        self.grid.close()
