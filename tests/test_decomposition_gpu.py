"""Slab decomposition of the GPU library over two ranks (gloo, host-staged halos).

Two processes, one slab each, on the same GPU: each holds its slab in a
library handle with exchanged cut sides (hydro_set_exchange) and steps it in
lockstep with the other through paper_2503_04428_gb300.decomp.SlabRun --
halos as point-to-point messages through host memory, the time step as an
all-reduce, shell masses for the monopole as an all-gather.  No kernel waits
on another process: every exchange happens on the host between steps.  The
result must equal the whole grid run by the library in one handle, and the
oracle's whole run within the per-step parity bars times the steps taken
(tests/parity.py).  Against the whole grid on the GPU the bar is 1e-14
(relative L1) and 1e-13 (element-wise) in FP64, 1e-6 and 1e-5 in FP32:
the 3D sweep's CTAs march z in chunks, which start at other planes in a
slab than in the whole grid (the test prints whether the states still agree
bit for bit, and their largest difference); the monopole's enclosed-mass sum
is also associated differently in a slab (its scan starts from the inner
slabs' total).  The oracle's slabs equal its whole grid bit for bit
(tests/test_decomposition.py).
"""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl
from parity import check

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, case, axis, nsteps, precision, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2503_04428_gb300 import decomp
    run = decomp.SlabRun(case, axis, precision=precision)
    run.run(nsteps, case["cfl"])
    out[rank] = run.get_state()
    run.close()
    dist.destroy_process_group()


def _split(case, axis, world, nsteps, precision):
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, case, axis, nsteps, precision, out), nprocs=world, join=True)
        parts = [out[r] for r in range(world)]
    return np.concatenate(parts, axis=3 - axis)


def _whole_gpu(H, case, nsteps, precision):
    g = H.Grid.from_case(case, precision)
    for _ in range(nsteps):
        g.step(g.cfl_dt(case["cfl"]))
    out = g.get_state()
    g.close()
    return out


def _whole_oracle(case, nsteps):
    s = O.solver_from_case(case)
    for _ in range(nsteps):
        s.step(s.cfl_dt(case["cfl"]))
    return s.get_state()


def _dyadic(case):
    out = dict(case)
    out["faces"] = [np.round(np.asarray(f) * 1024.0) / 1024.0 for f in case["faces"]]
    return out


@pytest.mark.parametrize("precision", [64, 32])
def test_two_slabs_along_z(hydro_lib, precision):
    case = _dyadic(wl.smooth_random(3, [37, 23, 40], 1, seed=13, riemann=O.HLLC,
                                    bc=[(O.TRANSMISSIVE, O.REFLECTIVE), (O.PERIODIC, O.PERIODIC),
                                        (O.PERIODIC, O.PERIODIC)]))
    if precision == 32:
        case["U"] = case["U"].astype(np.float32).astype(np.float64)
    nsteps = 4
    split = _split(case, 2, 2, nsteps, precision)
    whole = _whole_gpu(hydro_lib, case, nsteps, precision)
    print("z slabs, FP%d: split == whole bit for bit: %s, max |difference| %.3e"
          % (precision, np.array_equal(split, whole), np.abs(split - whole).max()))
    check(whole, split, 3, case["gamma"], 64, l1=1e-14 if precision == 64 else 1e-6,
          elem=1e-13 if precision == 64 else 1e-5)
    if precision == 64:
        check(_whole_oracle(case, nsteps), split, 3, case["gamma"], 64, l1=nsteps * 1e-12, elem=nsteps * 1e-11)


def test_three_slabs_along_r_with_monopole(hydro_lib):
    case = wl.sphere_state(48, 12, 10, dim=3, rotating=True, r_range=(1.0, 20.0), n_scalars=1,
                           bc=[(O.REFLECTIVE, O.TRANSMISSIVE), (O.REFLECTIVE, O.REFLECTIVE),
                               (O.PERIODIC, O.PERIODIC)])
    case["sources"] = dict(gravity=O.GRAV_POINT_MONOPOLE, G=0.01, Mc=2.0)
    nsteps = 3
    split = _split(case, 0, 3, nsteps, 64)
    whole = _whole_gpu(hydro_lib, case, nsteps, 64)
    check(whole, split, 3, case["gamma"], 64, l1=1e-14, elem=1e-13)
    check(_whole_oracle(case, nsteps), split, 3, case["gamma"], 64, l1=nsteps * 1e-12, elem=nsteps * 1e-11)


def test_exchanged_grid_rejects_device_side_runs(hydro_lib):
    H = hydro_lib
    case = wl.smooth_random(2, [16, 12], 0, seed=2)
    g = H.Grid(case["dim"], case["n"], case["faces"], case["bc"], case["coords"], case["gamma"],
               case["n_scalars"], case["riemann"], case["limiter"], 64)
    f = np.asarray(case["faces"][0])
    g.set_exchange(0, 1, [f[-1] + 0.1, f[-1] + 0.2])
    with pytest.raises(H.HydroError) as e:
        g.set_exchange(1, 0, [-0.2, -0.1][::-1])  # a second axis
    assert e.value.status == H.HYDRO_ERR_ARG
    g.set_state(case["U"])
    with pytest.raises(H.HydroError) as e:
        g.run(1, 0.4)
    assert e.value.status == H.HYDRO_ERR_UNSUPPORTED
    g.close()
