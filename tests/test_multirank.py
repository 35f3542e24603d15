"""The multi-rank bench path on CPU: world_size 2 over gloo.

Each rank builds its own tube set (no data exchange); the whole-job rate uses
the slowest rank's time and the cells of all ranks."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2503_04428_gb300 import workloads as wl
    lengths = wl.tube_lengths(64, bench.rank_seed(rank))
    cells = int(lengths.sum())
    elapsed = 1.0 + rank  # rank 1 is the slow one
    rate, t = bench.job_rate(elapsed, cells, 10, dist, "cpu")
    out[rank] = (rate, t, cells)
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    cells = [res[r][2] for r in range(world)]
    assert cells[0] != cells[1]  # each rank has its own tubes
    for r in range(world):
        rate, t, _ = res[r]
        assert t == 2.0  # max over ranks
        assert np.isclose(rate, sum(cells) * 10 / 2.0)


def test_single_process_rate():
    import bench
    rate, t = bench.job_rate(0.5, 1000, 4)
    assert t == 0.5 and rate == 8000.0
