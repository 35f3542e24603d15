"""The multi-rank bench path on CPU: world_size 2 over gloo.

The job at N ranks is N x 4096 tubes of the workload's distribution (one
seed), cut into N contiguous ranges of about equal cell counts; each rank
builds only its own range (no data exchange).  The whole-job rate uses the
slowest rank's time and the cells of all ranks."""
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
    w = bench.rank_tubes(world, rank, ntubes=64)
    cells = int(w["lengths"].sum())
    elapsed = 1.0 + rank  # rank 1 is the slow one
    rate, t = bench.job_rate(elapsed, cells, 10, dist, "cpu")
    out[rank] = (rate, t, cells, w["U"][:, :5].copy(), w["lengths"].copy())
    dist.destroy_process_group()


def test_two_ranks_partition_and_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    from paper_2503_04428_gb300 import workloads as wl
    whole = wl.tubes(64 * world, seed=2)
    cells = [res[r][2] for r in range(world)]
    # the two ranges are the whole tube set, in order, with no tube twice
    assert np.array_equal(np.concatenate([res[0][4], res[1][4]]), whole["lengths"])
    assert sum(cells) == int(whole["lengths"].sum())
    # the second range starts where the first ends, with the same values
    assert np.array_equal(res[1][3], whole["U"][:, cells[0]:cells[0] + 5])
    # balanced to within one tube
    assert abs(cells[0] - cells[1]) <= int(whole["lengths"].max())
    for r in range(world):
        rate, t, _, _, _ = res[r]
        assert t == 2.0  # max over ranks
        assert np.isclose(rate, sum(cells) * 10 / 2.0)


def test_partition_by_cells_covers_and_balances():
    import bench
    from paper_2503_04428_gb300 import workloads as wl
    for world in (1, 2, 3, 4, 8):
        ln = wl.tube_lengths(4096 * world, 2)
        parts = bench.partition_by_cells(ln, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(ln)
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        cells = [int(ln[a:b].sum()) for a, b in parts]
        assert max(cells) - min(cells) <= 2 * int(ln.max())
    # one rank: exactly the 4096-tube workload
    w = bench.rank_tubes(1, 0, ntubes=4096)
    ref = wl.tubes(4096, seed=2)
    assert np.array_equal(w["lengths"], ref["lengths"]) and np.array_equal(w["U"], ref["U"])


def test_trajectory_windows():
    """The timed steps: windows of consecutive steps inside the 200-step run,
    k steps in all, whose mean step is the run's mean step (99.5)."""
    import bench
    assert bench.trajectory_windows(200) == [(0, 200)]
    assert bench.trajectory_windows(250) == [(0, 250)]
    assert bench.trajectory_windows(20) == [(45, 10), (145, 10)]
    for k in (1, 5, 7, 9, 10, 11, 20, 33, 150, 199):
        win = bench.trajectory_windows(k)
        steps = bench.window_steps(win)
        assert len(steps) == k and len(set(steps)) == k
        assert min(steps) >= 0 and max(steps) < 200
        assert abs(np.mean(steps) - 99.5) <= 0.5, (k, win)
        assert all(win[i][0] + win[i][1] <= win[i + 1][0] for i in range(len(win) - 1))


def test_single_process_rate():
    import bench
    rate, t = bench.job_rate(0.5, 1000, 4)
    assert t == 0.5 and rate == 8000.0
