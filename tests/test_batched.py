"""Batched tubes (thousands of independent 1D shock tubes, exact solver) on the GPU vs the FP64 oracle.

Bars (tests/parity.py: relative L1 and element-wise, per component):
FP64: L1 <= 1e-11 and element-wise <= 1e-10 after the 5-20 steps of a run
(the per-step bars 1e-12 / 1e-11, accumulated); FP32: per step L1 <= 2e-5
and element-wise <= 1e-4, with both sides restarted from the oracle's state
each step.  The MLP guess must not change the answer (Newton is polished to
roundoff).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl
from parity import check, errors

pytestmark = pytest.mark.gpu

G53 = 5.0 / 3.0
RUN64 = dict(l1=1e-11, elem=1e-10)  # FP64 after a run of up to 20 steps


def small_tubes(ntubes=12, seed=21, lo=256, hi=1100):
    return wl.tubes(ntubes, seed=seed, lo=lo, hi=hi)


def rel_l1(A, B, gamma=G53):
    """Per-component relative L1 on the scales of tests/parity.py."""
    return errors(A, B, 1, gamma)[0]


def tube_slices(lengths):
    off = np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.int64))])
    return [slice(int(off[t]), int(off[t + 1])) for t in range(len(lengths))]


def test_fp64_matches_oracle(hydro_lib):
    w = small_tubes()
    ref, st = O.batch_run(w["lengths"], w["U"], w["gamma"], O.EXACT, O.MINMOD, 0.8, 20)
    b = hydro_lib.Batch(w["lengths"], w["gamma"], precision=64)
    b.set_state(w["U"])
    b.run(20, 0.8)
    check(ref, b.get_state(), 1, G53, 64, **RUN64)
    s = b.stats()
    assert s["steps"] == 20
    assert s["faces"] == st["faces"]
    # faces with identical states skip Newton on the GPU (their flux is the
    # state's own); every other face iterates as in the oracle
    assert 0 < s["newton_iters"] <= st["newton_iters"]


def test_fp64_mlp_guess_changes_nothing(hydro_lib):
    """Random (untrained) network weights: a poor guess, same polished answer."""
    w = small_tubes(6, seed=22)
    rng = np.random.default_rng(0)
    weights = (0.1 * rng.standard_normal(O.MLP_NPARAM)).astype(np.float32)
    ref, _ = O.batch_run(w["lengths"], w["U"], w["gamma"], O.EXACT, O.MINMOD, 0.8, 15)
    b = hydro_lib.Batch(w["lengths"], w["gamma"], precision=64)
    b.mlp_set(weights, True)
    b.set_state(w["U"])
    b.run(15, 0.8)
    check(ref, b.get_state(), 1, G53, 64, **RUN64)
    assert b.stats()["mlp_faces"] > 0


def test_fp32_per_step(hydro_lib):
    w = small_tubes(8, seed=23)
    U = w["U"].astype(np.float32)
    b = hydro_lib.Batch(w["lengths"], w["gamma"], precision=32)
    for _ in range(5):
        b.set_state(U)
        ref, _ = O.batch_run(w["lengths"], U.astype(np.float64), w["gamma"], O.EXACT, O.MINMOD, 0.8, 1)
        b.run(1, 0.8)
        check(ref, b.get_state(), 1, G53, 32)
        U = ref.astype(np.float32)


def test_ragged_and_minimum_tubes(hydro_lib):
    lengths = np.array([2, 3, 511, 512, 513, 1024, 7, 130], dtype=np.int32)
    WL, WR = wl.tube_states(len(lengths), 24)
    total = int(lengths.sum())
    U = np.empty((3, total))
    off = 0
    for bi, nb in enumerate(lengths):
        x = (np.arange(nb) + 0.5) / nb
        left = x < 0.5
        W = np.where(left[None, :], WL[bi][:, None], WR[bi][:, None])
        U[:, off:off + nb] = wl.conserved(5 / 3, W[0], [W[1]], W[2])
        off += nb
    ref, _ = O.batch_run(lengths, U, 5 / 3, O.EXACT, O.VANLEER, 0.6, 10)
    b = hydro_lib.Batch(lengths, 5 / 3, limiter=hydro_lib.HYDRO_VANLEER, precision=64)
    b.set_state(U)
    b.run(10, 0.6)
    check(ref, b.get_state(), 1, 5 / 3, 64, **RUN64)
    # FP32: the same ragged set (total not a multiple of the 16-byte slab
    # quantum, tubes shorter than one segment) per step, through the host and
    # the device copy paths
    torch = pytest.importorskip("torch")
    U32 = U.astype(np.float32)
    b32 = hydro_lib.Batch(lengths, 5 / 3, limiter=hydro_lib.HYDRO_VANLEER, precision=32)
    for k in range(4):
        if k % 2:
            b32.set_state(torch.from_numpy(U32).cuda())
        else:
            b32.set_state(U32)
        ref, _ = O.batch_run(lengths, U32.astype(np.float64), 5 / 3, O.EXACT, O.VANLEER, 0.6, 1)
        b32.run(1, 0.6)
        G = b32.get_state()
        check(ref, G, 1, 5 / 3, 32)
        U32 = G


def test_full_size_sampled(hydro_lib):
    """All 4096 tubes (~1.73e7 cells) in the bench's launch configuration;
    8 tubes recomputed by the oracle."""
    w = wl.tubes()
    b = hydro_lib.Batch(w["lengths"], w["gamma"], precision=64)
    b.set_state(w["U"])
    b.run(5, 0.8)
    G = b.get_state()
    off = np.concatenate([[0], np.cumsum(w["lengths"])])
    for t in (0, 1, 517, 1234, 2047, 3000, 4094, 4095):
        sl = slice(off[t], off[t + 1])
        ref, _ = O.batch_run(w["lengths"][t:t + 1], w["U"][:, sl], w["gamma"], O.EXACT, O.MINMOD, 0.8, 5)
        check(ref, G[:, sl], 1, w["gamma"], 64, l1=1e-11, elem=1e-10, label="tube %d" % t)


def test_rejects_bad_input(hydro_lib):
    H = hydro_lib
    with pytest.raises(H.HydroError):
        H.Batch([1, 5], 1.4)
    with pytest.raises(H.HydroError) as e:
        H.hydro_batch_create(np.array([8]), H.hydro_eos(1.4, 0), H.HYDRO_HLLC, H.HYDRO_MINMOD, 64, None)
    assert e.value.status == H.HYDRO_ERR_UNSUPPORTED
    b = H.Batch([8, 9], 1.4)
    U = np.ones((3, 17))
    U[2] = -1.0
    with pytest.raises(H.HydroError) as e:
        b.set_state(U)
    assert e.value.status == H.HYDRO_ERR_NEGATIVE_STATE


@pytest.mark.parametrize("precision", [64, 32])
def test_uniform_tubes_are_unchanged(hydro_lib, precision):
    """Tubes holding one state everywhere: every face is trivial and every step
    returns the state bit for bit (the uniform-window path and the full path
    both give U + 0)."""
    lengths = np.array([100, 57, 3000, 28, 29, 56], dtype=np.int32)
    total = int(lengths.sum())
    rho = np.repeat(np.array([1.0, 0.5, 2.0, 1e-3, 3.0, 0.7]), lengths)
    u = np.repeat(np.array([0.3, -1.0, 0.0, 2.0, -0.5, 0.1]), lengths)
    p = np.repeat(np.array([1.0, 0.2, 5.0, 1e-4, 0.9, 1.1]), lengths)
    U = wl.conserved(5 / 3, rho, [u], p)
    dt = np.float64 if precision == 64 else np.float32
    U0 = U.astype(dt)
    b = hydro_lib.Batch(lengths, 5 / 3, precision=precision)
    b.set_state(U0)
    b.run(3, 0.8)
    assert np.array_equal(b.get_state(), U0)
    assert b.stats()["newton_iters"] == 0


@pytest.mark.parametrize("precision", [64, 32])
def test_run_host_equals_set_run_get(hydro_lib, precision):
    """hydro_batch_run_host (copies pipelined with the steps of other groups
    of tubes) gives the state, the per-tube times and the handle state of
    set_state + run + get_state, bit for bit."""
    import torch
    w = wl.tubes(40, seed=8, lo=100, hi=2000)
    dt = np.float32 if precision == 32 else np.float64
    U = np.ascontiguousarray(w["U"].astype(dt))
    b = hydro_lib.Batch(w["lengths"], w["gamma"], precision=precision)
    rng = np.random.default_rng(1)
    b.mlp_set((0.05 * rng.standard_normal(hydro_lib.HYDRO_MLP_NPARAM)).astype(np.float32), True)
    b.set_state(U)
    b.run(3, 0.8)
    ref, tref = b.get_state(), b.times()
    out = np.empty_like(U)
    b.run_host(U, out, 3, 0.8, nparts=5)
    assert np.array_equal(out, ref)
    assert np.array_equal(b.times(), tref)
    assert np.array_equal(b.get_state(), ref)
    # pinned tensors, more parts than tubes
    pin_in = torch.from_numpy(U).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    b.run_host(pin_in, pin_out, 3, 0.8, nparts=100)
    assert np.array_equal(pin_out.numpy(), ref)
    # pinned buffers again (the captured graph is replayed) and after a
    # change of input contents, with other buffers, and with another step count
    b.run_host(pin_in, pin_out, 3, 0.8, nparts=100)
    assert np.array_equal(pin_out.numpy(), ref)
    pin_in.copy_(torch.from_numpy(ref))
    b.set_state(ref)
    b.run(2, 0.8)
    ref2 = b.get_state()
    b.run_host(pin_in, pin_out, 2, 0.8, nparts=100)
    assert np.array_equal(pin_out.numpy(), ref2)
    pin_out2 = torch.empty_like(pin_in).pin_memory()
    b.run_host(pin_in, pin_out2, 2, 0.8, nparts=3)
    assert np.array_equal(pin_out2.numpy(), ref2)
    # an invalid input state is reported
    bad = U.copy()
    bad[0, 5] = -1.0
    with pytest.raises(hydro_lib.HydroError):
        b.run_host(bad, out, 1, 0.8)
    b.close()


def test_tune_cache_round_trip(tmp_path):
    """A launch shape stored in the autotuner's cache file comes back as
    stored, including work items longer than 999 cells (HYDRO_TUNE_CACHE is
    read when a process first tunes a batch)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    prog = ("import json, sys; sys.path.insert(0, %r)\n"
            "from paper_2503_04428_gb300 import hydro as H, workloads as wl\n"
            "w = wl.tubes(16, seed=5, lo=4000, hi=8000)\n"
            "b = H.Batch(w['lengths'], w['gamma'], precision=32)\n"
            "b.set_state(w['U']); b.run(1, 0.8)\n"
            "import torch; sms = torch.cuda.get_device_properties(0).multi_processor_count\n"
            "s = b.stats(); print(json.dumps([s['tile_x'], s['tile_y'], s['zchunk'], sms]))\n" % root)
    env = dict(os.environ, HYDRO_TUNE_CACHE=str(cache))
    run = lambda: subprocess.run([sys.executable, "-c", prog], env=env, capture_output=True, text=True,
                                 timeout=300, check=True).stdout.strip().splitlines()[-1]
    import json
    json.loads(run())
    key, _, us = cache.read_text().splitlines()[0].split()
    # 8 warps per CTA, 3584-cell items, one CTA per SM
    cache.write_text("%s %d %s\n" % (key, (8 * 10000 + 3584) * 100 + 1, us))
    item, nw, grid, sms = json.loads(run())
    assert (item, nw, grid) == (3584, 8, sms)


@pytest.mark.parametrize("precision", [64, 32])
def test_one_launch_equals_single_steps(hydro_lib, precision):
    """A launch of several steps (a tube's step waits only for its own previous
    step) gives exactly what one-step launches give, with and without the
    network; two queued launches equal one."""
    w = small_tubes(10, seed=31)
    U = w["U"].astype(np.float32) if precision == 32 else w["U"]
    rng = np.random.default_rng(3)
    weights = (0.1 * rng.standard_normal(O.MLP_NPARAM)).astype(np.float32)
    for mlp in (False, True):
        runs = []
        for mode in ("one", "single", "queued"):
            b = hydro_lib.Batch(w["lengths"], w["gamma"], precision=precision)
            if mlp:
                b.mlp_set(weights, True)
            b.set_state(U)
            if mode == "one":
                b.run(9, 0.8)
            elif mode == "single":
                for _ in range(9):
                    b.run(1, 0.8)
            else:
                b.enqueue(4, 0.8)
                b.enqueue(5, 0.8)
                b.run(0, 0.8)
            assert b.stats()["steps"] == 9
            runs.append((b.get_state(), b.times()))
            b.close()
        for G, T in runs[1:]:
            assert np.array_equal(G, runs[0][0]) and np.array_equal(T, runs[0][1])


def test_failed_step_leaves_each_tube_at_its_last_good_step(hydro_lib):
    """One tube whose Riemann problem generates vacuum fails its first step;
    the launch stops, and every tube is left at the last step it completed:
    the failing tube at its initial state and time 0, each other tube at the
    oracle's state after the k steps it completed (k may differ between tubes,
    0..6), its time 0 exactly when k = 0.  The handle then runs on."""
    H = hydro_lib
    w = small_tubes(8, seed=33)
    n_vac = 300
    x = (np.arange(n_vac) + 0.5) / n_vac
    Uv = wl.conserved(w["gamma"], np.ones(n_vac), [np.where(x < 0.5, -5.0, 5.0)], np.full(n_vac, 0.1))
    lengths = list(w["lengths"][:3]) + [n_vac] + list(w["lengths"][3:])
    sl = tube_slices(w["lengths"])
    U = np.concatenate([w["U"][:, sl[t]] for t in range(3)] + [Uv] + [w["U"][:, sl[t]] for t in range(3, 8)],
                       axis=1)
    b = H.Batch(lengths, w["gamma"], precision=64)
    b.set_state(U)
    with pytest.raises(H.HydroError) as e:
        b.run(6, 0.8)
    assert e.value.status == H.HYDRO_ERR_VACUUM
    G, T = b.get_state(), b.times()
    slb = tube_slices(lengths)
    assert np.array_equal(G[:, slb[3]], U[:, slb[3]]) and T[3] == 0.0
    assert b.stats()["steps"] == 0
    for t in range(len(lengths)):
        if t == 3:
            continue
        Ut = U[:, slb[t]]
        best, kbest = np.inf, -1
        for k in range(7):
            ref = Ut if k == 0 else O.batch_run([lengths[t]], Ut, w["gamma"], O.EXACT, O.MINMOD, 0.8, k)[0]
            err = max(errors(ref, G[:, slb[t]], 1, G53)[0])
            if err < best:
                best, kbest = err, k
        assert best <= 1e-11, (t, kbest, best)
        assert (T[t] == 0.0) == (kbest == 0), (t, kbest, T[t])
    # with the vacuum tube replaced, the handle runs on from the new state
    U2 = U.copy()
    U2[:, slb[3]] = wl.conserved(w["gamma"], np.ones(n_vac), [np.zeros(n_vac)], np.ones(n_vac))
    b.set_state(U2)
    b.run(3, 0.8)
    ref, _ = O.batch_run(lengths, U2, w["gamma"], O.EXACT, O.MINMOD, 0.8, 3)
    check(ref, b.get_state(), 1, G53, 64, **RUN64)
    b.close()


def test_beyond_32bit_element_offsets(hydro_lib):
    """Maximum sizes: 100000 tubes of 7200 cells (7.2e8 cells, 2.16e9 values
    per buffer, past 32-bit element offsets), FP32, two steps: the first,
    middle and last tubes equal, bit for bit, the same tubes advanced in a
    batch of their own (tubes are independent, and the kernel's results do
    not depend on the launch shape or on which warp takes which segment)."""
    import torch
    H = hydro_lib
    nt, n, g = 100000, 7200, 5.0 / 3.0
    WL, WR = wl.tube_states(nt, seed=17)
    UL = wl.conserved(g, WL[:, 0], [WL[:, 1]], WL[:, 2]).astype(np.float32)  # (3, nt)
    UR = wl.conserved(g, WR[:, 0], [WR[:, 1]], WR[:, 2]).astype(np.float32)
    left = torch.from_numpy((np.arange(n) + 0.5) / n < 0.5).cuda()
    U = torch.where(left[None, None, :], torch.from_numpy(UL).cuda()[:, :, None],
                    torch.from_numpy(UR).cuda()[:, :, None]).reshape(3, nt * n)
    big = H.Batch(np.full(nt, n, dtype=np.int32), g, precision=32)
    big.set_launch(8, 7224, 2)  # whole-tube items, no autotuning (the small batch autotunes)
    big.set_state(U)
    big.run(2, 0.8)
    out = torch.empty_like(U)
    big.get_state(out)
    times = big.times()
    big.close()
    del U
    sample = [0, 1, nt // 2, nt - 2, nt - 1]
    Us = np.concatenate([np.where(((np.arange(n) + 0.5) / n < 0.5)[None, :], UL[:, t, None], UR[:, t, None])
                         for t in sample], axis=1)
    small = H.Batch(np.full(len(sample), n, dtype=np.int32), g, precision=32)
    small.set_state(np.ascontiguousarray(Us))
    small.run(2, 0.8)
    ref = small.get_state()
    tref = small.times()
    small.close()
    for q, t in enumerate(sample):
        got = out[:, t * n:(t + 1) * n].cpu().numpy()
        assert np.array_equal(got, ref[:, q * n:(q + 1) * n]), (t, np.abs(got - ref[:, q * n:(q + 1) * n]).max())
        assert times[t] == tref[q]
