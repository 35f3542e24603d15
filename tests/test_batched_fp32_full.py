"""The FP32 batched form in the configuration the benchmark times, against the FP64 oracle.

All 4096 tubes (256-8192 cells, 1.73e7 cells), the autotuned launch shape
and a fixed shape of 1792-cell work items (so that most tubes span several
items), and a network trained by the benchmark's own recipe
(bench.train_mlp): the form whose rate is the headline.  Tubes are independent, so the oracle
recomputes a sample of them: the longest and the shortest tube and tubes
that span two or three work items.  Three regimes, each compared step by
step with both sides restarted from the oracle's state (FP32-rounded):

  (i)   steps 1-3 from the initial state (waves just leaving the interface);
  (ii)  three steps from the oracle's own state after 150 steps (wide fans,
        plateaus and shocks: Newton on hundreds of faces per tube);
  (iii) three steps of the dense state (density and pressure x (1 + 0.01
        U(-1,1)) in every cell: every face iterates).

Bars per step (tests/parity.py): relative L1 <= 2e-5, element-wise <= 1e-4
of the component's scale.  The oracle runs Toro's guess; the GPU runs the
trained network on its gated faces: Newton's polishing step makes the
answers agree whatever the guess.
"""
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_2503_04428_gb300 import workloads as wl
from parity import check

pytestmark = pytest.mark.gpu

CFL = 0.8
G53 = 5.0 / 3.0


@pytest.fixture(scope="module")
def trained_weights(hydro_lib):
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    w, info = bench.train_mlp(hydro_lib, torch, G53, 2)
    return w


def _sample(lengths, item_len):
    """Tube indices: longest, shortest, and tubes spanning 2 and 3 work items."""
    ln = np.asarray(lengths)
    pick = [int(np.argmax(ln)), int(np.argmin(ln))]
    for lo, hi in ((item_len + 1, 2 * item_len), (2 * item_len + 1, 3 * item_len)):
        idx = np.nonzero((ln >= lo) & (ln <= hi))[0]
        pick += [int(i) for i in idx[:: max(1, len(idx) // 3)][:3]]
    pick += [0, len(ln) // 2, len(ln) - 1]
    return sorted(set(pick))


def _slices(lengths):
    off = np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.int64))])
    return off


def _compare_steps(H, b, w, U32, picks, nsteps, label):
    """Per-step comparison of the sampled tubes; both sides restart from the
    oracle's (FP32-rounded) state of the sampled tubes each step; the other
    tubes keep the GPU's state."""
    off = _slices(w["lengths"])
    worst = 0.0
    U = U32.copy()
    for k in range(nsteps):
        b.set_state(U)
        b.run(1, CFL)
        G = b.get_state()
        for t in picks:
            sl = slice(int(off[t]), int(off[t + 1]))
            ref, _ = O.batch_run(w["lengths"][t:t + 1], U[:, sl].astype(np.float64), G53, O.EXACT, O.MINMOD,
                                 CFL, 1)
            e1, em = check(ref, G[:, sl], 1, G53, 32, label="%s tube %d (n=%d) step %d"
                           % (label, t, w["lengths"][t], k + 1))
            worst = max(worst, float(em.max()))
            G[:, sl] = ref.astype(np.float32)
        U = G
    return worst


@pytest.mark.parametrize("shape", ["tuned", "items_1792"])
def test_fp32_full_size_sampled(hydro_lib, trained_weights, shape):
    """The autotuned launch shape (as in the benchmark), and a fixed shape of
    1792-cell items (8 warps per CTA, 2 CTAs per SM) under which the long
    tubes span several items whichever shape the autotuner picks."""
    H = hydro_lib
    w = wl.tubes()
    U0 = w["U"].astype(np.float32)
    b = H.Batch(w["lengths"], G53, precision=32)
    b.mlp_set(trained_weights, True)
    if shape != "tuned":
        b.set_launch(8, 1792, 2)
    b.set_state(U0)
    b.run(1, CFL)  # autotunes the launch shape (unless fixed), as in the benchmark
    item_len = b.stats()["tile_x"]
    picks = _sample(w["lengths"], item_len)
    if shape != "tuned":
        assert item_len == 1792 and max(w["lengths"][picks]) > 2 * item_len, (item_len, picks)
    s0 = b.stats()
    # (i) from the initial state
    worst_i = _compare_steps(H, b, w, U0, picks, 3, "initial")
    # (ii) from the oracle's state after 150 steps of the sampled tubes
    off = _slices(w["lengths"])
    U150 = U0.copy()
    for t in picks:
        sl = slice(int(off[t]), int(off[t + 1]))
        ref, _ = O.batch_run(w["lengths"][t:t + 1], U0[:, sl].astype(np.float64), G53, O.EXACT, O.MINMOD, CFL,
                             150)
        U150[:, sl] = ref.astype(np.float32)
    worst_ii = _compare_steps(H, b, w, U150, picks, 3, "after 150 steps")
    s1 = b.stats()
    assert s1["mlp_faces"] > s0["mlp_faces"], "the trained network was used on no face"
    # (iii) the dense state: every face runs Newton
    wd = wl.tubes(perturb=0.01)
    worst_iii = _compare_steps(H, b, wd, wd["U"].astype(np.float32), picks, 3, "dense")
    print("item_len %d, sampled tubes %s; worst element-wise error: initial %.2e, step 150 %.2e, dense %.2e"
          % (item_len, picks, worst_i, worst_ii, worst_iii))
    b.close()
