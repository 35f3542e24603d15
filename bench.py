"""Benchmark of the batched exact-Riemann workload (4096 tubes, 256-8192 cells each).

One step = one MUSCL-Hancock time step of every tube (primitive recovery,
limited reconstruction, Hancock predictor, exact Riemann solve with the
learned or Toro guess, conservative update, per-tube CFL speed).  One
persistent launch of the batched kernel runs any number of steps: a tube's
step waits only for the tube's own previous step, so there is no grid-wide
barrier between steps.

The workload runs every tube for K = 200 of its own CFL steps, and the cost
of a step changes along that run (the waves spread from each interface, and
with them the faces that run Newton).  So the `--steps` timed steps are
windows of consecutive steps of the 200-step run, each window one launch
timed with CUDA events: two windows centred in the two halves of the run
(one for fewer than 10 steps; the whole run from 200 steps on), so that the
timed steps' mean position is the run's; the run is advanced untimed (one
launch) between them.

Headline (`value`): FP32 bulk + MLP star-pressure guess, in cell-updates/s
over all ranks, inputs resident in HBM, over those steps.  Beside it, over
the same steps: the plain FP64 + Toro-guess form of the same kernel
(`fp64_plain`), the FP32 form without the network (`mlp_gain`), and the
end-to-end rate through the C ABI with host buffers (`e2e`, every step its
own call with its copies in and out); then the HBM roofline of the kernel,
the whole 200-step run as one launch (`whole_run`), the first steps alone
(`early_window`), a dense state on which every face iterates
(`dense_state`), the 3D grid sweeps, and the FP64 CPU oracle on a bounded
sample (`cpu_baseline`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun the job is N x 4096 tubes of the workload's distribution
(one seed), cut into N contiguous ranges of about equal cell counts, one per
rank (weak scaling, no data exchange); timing is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFL = 0.8
NTUBES = 4096
METRIC = "cell-updates/s"
WORKLOAD = "batched exact-Riemann: 4096 1D shock tubes, 256-8192 cells (1.73e7 cells), gamma=5/3, minmod"
KERNEL_SOURCES = ["paper_2503_04428_gb300/csrc/batched.cuh", "paper_2503_04428_gb300/csrc/physics.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "batched_fp32_mlp_4096tubes.traffic.json")
SWEEP_SOURCES = ["paper_2503_04428_gb300/csrc/sweep.cuh", "paper_2503_04428_gb300/csrc/physics.cuh"]
SWEEP_FLOPS_FILE = os.path.join(ROOT, "profiles", "sweep_sedov3d_fp64.flops.json")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash(sources=KERNEL_SOURCES):
    """Hash of the kernels' code (comments and whitespace removed), so that a
    profiled figure stays attached to the code it was measured on."""
    h = hashlib.sha256()
    for f in sources:
        src = open(os.path.join(ROOT, f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def sweep_fp64_flops_per_cell():
    """FP64 flops per cell-update of the FP64 Sedov sweep (DFMA = 2, DADD and
    DMUL = 1) from the committed ncu counts, if they match this kernel."""
    if not os.path.exists(SWEEP_FLOPS_FILE):
        return None
    d = json.load(open(SWEEP_FLOPS_FILE))
    if d.get("kernel_hash") != kernel_hash(SWEEP_SOURCES):
        return None
    return float(d["fp64_flops_per_cell"])


def alu_peaks(H):
    """Dense FMA peaks of this GPU, measured now by the library's FMA-chain kernel."""
    return {"fp64_tflops": H.hydro_fma_rate(64), "fp32_tflops": H.hydro_fma_rate(32),
            "fp32x2_tflops": H.hydro_fma_rate(H.HYDRO_FMA_F32X2),
            "source": "hydro_fma_rate: 8 independent FMA chains per thread (float2 chains of paired FMAs "
                      "for fp32x2), 8 CTAs of 256 per SM"}


def profiled_traffic(item_len):
    """DRAM bytes per step from the committed ncu summary (the captured
    launch's bytes over its steps), if it matches this kernel and the
    work-item length in effect (item boundaries re-fetch halos)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    d = json.load(open(TRAFFIC_FILE))
    if d.get("kernel_hash") != kernel_hash() or d.get("item_len") != item_len:
        return None
    return float(d["dram_bytes_per_launch"]) / float(d.get("steps_per_launch", 1))


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader",
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax = float(f[2].split()[0])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


TRAJ = 200  # steps every tube takes in the workload


def partition_by_cells(lengths, world):
    """Contiguous tube ranges [b0, b1) of about equal cell counts, one per
    rank: range r starts at the first tube whose cumulative cell count
    reaches r/world of the total."""
    cum = np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.int64))])
    total = int(cum[-1])
    bounds = [int(np.searchsorted(cum, r * total / world, side="left")) for r in range(world)] + [len(lengths)]
    for r in range(1, world + 1):
        bounds[r] = max(bounds[r], bounds[r - 1])
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def rank_tubes(world, rank, perturb=0.0, ntubes=NTUBES):
    """This rank's share of the job: world x ntubes tubes of the workload's
    distribution (seed 2; at world = 1 exactly the 4096-tube workload), cut
    by cumulative cell count."""
    from paper_2503_04428_gb300 import workloads as wl
    n = ntubes * world
    b0, b1 = partition_by_cells(wl.tube_lengths(n, 2), world)[rank]
    return wl.tubes(n, seed=2, perturb=perturb, tube_range=(b0, b1))


def trajectory_windows(k, length=TRAJ):
    """The k timed steps as windows of consecutive steps of the workload's
    run, each window one launch (a launch runs any number of steps, with no
    grid-wide barrier between them): the whole run when k >= length, else
    two windows (one, centred, when k < 10) about a quarter of the run either
    side of its middle, placed so that the timed steps' mean position is the
    run's.  [(first step, count)]."""
    if k >= length:
        return [(0, k)]
    mid = 0.5 * (length - 1)
    if k < 10:
        return [(int(round(mid - 0.5 * (k - 1))), k)]
    w0, w1 = (k + 1) // 2, k // 2
    # centres mid -/+ d0/d1 with w0 d0 = w1 d1 (about a quarter of the run each way)
    c0, c1 = mid - 0.5 * length * w1 / k, mid + 0.5 * length * w0 / k
    return [(int(round(c0 - 0.5 * (w0 - 1))), w0), (int(round(c1 - 0.5 * (w1 - 1))), w1)]


def window_steps(windows):
    """Every step index of the windows, in order."""
    return [p + i for p, w in windows for i in range(w)]


def job_rate(elapsed_local, cells_local, steps, dist=None, device=None):
    """Whole-job rate: cells of all ranks x steps / the slowest rank's time.

    With a process group the elapsed time is max-reduced and the cells are
    sum-reduced (timing only: no data-path collective)."""
    if dist is None:
        return cells_local * steps / elapsed_local, elapsed_local
    import torch
    t = torch.tensor([elapsed_local], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(c.item()) * steps / float(t.item()), float(t.item())


def train_mlp(H, torch, gamma, seed):
    """Harvest gated faces from an FP64 run, add partial-jump faces of the
    workload's state distribution, label them with the FP64 exact solver and
    train the guess network with the library's own kernels (untimed)."""
    from paper_2503_04428_gb300 import workloads as wl
    t0 = time.time()
    w = wl.tubes(1024, seed=seed)
    b = H.Batch(w["lengths"], gamma, precision=64)
    b.set_state(w["U"])
    b.harvest_begin(400000, 1.0, 4)
    b.run(60, CFL)
    faces = np.concatenate([wl.partial_jump_faces(60000, 7), b.harvest_get(400000)])
    ps, _, _ = H.hydro_exact_solve(faces[:, :3], faces[:, 3:], gamma, precision=64)
    keep = ps > 0
    loss = b.mlp_train(faces[keep], np.log(ps[keep]), epochs=60, batch=512, lr=3e-3, seed=4)
    wts = b.mlp_get()
    b.close()
    return wts, {"faces": int(keep.sum()), "loss": loss, "train_s": round(time.time() - t0, 2)}


def work_stream(torch):
    """A dedicated stream, made torch's current one: every handle is created
    on it, every tensor is made on it, and the timing events are recorded on
    it -- the stream the kernels are launched on.  (The legacy default
    stream would not do: a handle given a null stream makes its own.)"""
    s = torch.cuda.Stream()
    torch.cuda.set_stream(s)
    return s


def time_trajectory(torch, stream, b, U, windows, cfl=CFL):
    """From state U, advance the batch through the run and time each window
    of consecutive steps (trajectory_windows) as one launch: CUDA events on
    the launching stream around it, queued without a host round trip
    (hydro_batch_enqueue) behind the untimed launch that advances the run to
    the window, so that the events bracket the window's kernel and nothing
    else.  Returns the summed device time in seconds and the solver counters
    accumulated over the whole run (steps 0 .. the last window's end)."""
    b.set_state(U)
    s0 = b.stats()
    cur = 0
    evs = []
    torch.cuda.synchronize()
    for p, w in windows:
        if p > cur:
            b.enqueue(p - cur, cfl)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if not evs and p == 0:
            # nothing queued ahead: keep the device busy while the host
            # queues the first timed launch, so that e0 fires right before it
            torch.cuda._sleep(100000)
        e0.record(stream)
        b.enqueue(w, cfl)
        e1.record(stream)
        evs.append((e0, e1, w))
        cur = p + w
    b.run(0, cfl)  # waits, and reports a failed step
    torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1, _ in evs]
    t = sum(ms) / 1000.0
    s1 = b.stats()
    c = counters(s0, s1)
    c["step_us"] = {"windows": [[p, w] for p, w in windows],
                    "us_per_step": [round(1000.0 * m / w, 1) for m, (_, _, w) in zip(ms, evs)]}
    return t, c


def counters(s0, s1):
    """Exact-solver counters between two stats() snapshots: iterations per
    face (all faces), and per Newton face by guess category."""
    faces = max(s1["faces"] - s0["faces"], 1)
    nf = [a - b for a, b in zip(s1["newton_faces"], s0["newton_faces"])]
    ni = [a - b for a, b in zip(s1["newton_iters_by"], s0["newton_iters_by"])]
    out = {"steps": s1["steps"] - s0["steps"],
           "newton_iters_per_face": (s1["newton_iters"] - s0["newton_iters"]) / faces,
           "newton_face_fraction": sum(nf) / faces}
    for k, name in enumerate(("toro", "mlp", "fp64_fallback")):
        out[name] = {"faces": nf[k], "face_fraction": nf[k] / faces,
                     "iters_per_face": (ni[k] / nf[k]) if nf[k] else None}
    return out


def timed_steps(torch, stream, fn, steps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0


def cpu_baseline(steps_sample=4, tubes_sample=NTUBES):
    """The FP64 oracle (as it stands, all host cores) on a bounded sample of the
    workload: every tube for 4 steps (~20 s of CPU time on 16 cores), and on
    one core over the first 256 tubes."""
    import oracle as O
    from paper_2503_04428_gb300 import workloads as wl
    w = wl.tubes(NTUBES, seed=2)
    ln = w["lengths"][:tubes_sample]
    U = w["U"][:, :int(ln.sum())]
    cores = os.cpu_count() or 1
    t0 = time.time()
    O.batch_run(ln, U, w["gamma"], O.EXACT, O.MINMOD, CFL, steps_sample, nthreads=cores)
    dt = time.time() - t0
    cells = int(ln.sum()) * steps_sample
    # the same oracle on one core, over the first quarter of the sample
    ln1 = ln[:256]
    t0 = time.time()
    O.batch_run(ln1, U[:, :int(ln1.sum())], w["gamma"], O.EXACT, O.MINMOD, CFL, steps_sample, nthreads=1)
    v1 = int(ln1.sum()) * steps_sample / (time.time() - t0)
    return {"value": cells / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": "%d of 4096 tubes (%d cells) x %d steps from the initial state, FP64 Toro guess, "
                      "OpenMP over tubes"
                      % (tubes_sample, int(ln.sum()), steps_sample),
            "single_core": {"value": v1, "sample": "%d tubes (%d cells) x %d steps"
                                                   % (len(ln1), int(ln1.sum()), steps_sample)}}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle as O
    from paper_2503_04428_gb300 import workloads as wl
    w = wl.tubes(NTUBES, seed=2)
    ntub = 1024  # a quarter of the tubes per step: ~0.1 s of 16 host cores
    ln = w["lengths"][:ntub]
    U = w["U"][:, :int(ln.sum())].copy()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        U, _ = O.batch_run(ln, U, w["gamma"], O.EXACT, O.MINMOD, CFL, 1, nthreads=cores)
    t0 = time.time()
    for _ in range(args.steps):
        U, _ = O.batch_run(ln, U, w["gamma"], O.EXACT, O.MINMOD, CFL, 1, nthreads=cores)
    dt = time.time() - t0
    cells = int(ln.sum())
    value = cells * args.steps / dt
    sample = "%d of 4096 tubes (%d cells) per step, FP64 Toro guess, OpenMP over tubes" % (ntub, cells)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "tubes_per_gpu": NTUBES, "cells_per_gpu": int(w["lengths"].sum()),
                   "form": "FP64 CPU oracle (the reference arm), Toro guess", "sample": sample},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=TRAJ,
                    help="timed steps, spread evenly over the workload's 200-step run")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tubes", type=int, default=NTUBES, help="tubes per GPU (profiling a smaller case)")
    ap.add_argument("--skip-fp64", action="store_true", help="do not time the plain FP64 form")
    ap.add_argument("--skip-e2e", action="store_true", help="do not time the host-buffer path")
    ap.add_argument("--skip-grids", action="store_true", help="do not time the 3D grid sweeps")
    ap.add_argument("--skip-extras", action="store_true",
                    help="time only the headline form (profiling): no FP64, no-network, e2e, dense or grids")
    ap.add_argument("--grid-only", choices=["sedov3d_fp32", "sedov3d_fp64", "wedge_fp32", "wedge_fp32_rad"],
                    help="time one grid sweep only (profiling)")
    ap.add_argument("--grid-n", type=int, default=0, help="cells per axis for --grid-only sedov3d")
    ap.add_argument("--dense-only", action="store_true",
                    help="time only the headline form on the dense state (every face iterates), without the "
                         "network (profiling)")
    ap.add_argument("--profile-range", action="store_true",
                    help="with --grid-only or --dense-only: after the timing, run one more step between "
                         "cudaProfilerStart and cudaProfilerStop (for ncu --profile-from-start off)")
    ap.add_argument("--item-len", type=int, default=0,
                    help="fix the headline's work-item length (cells; 8 warps per CTA, 2 CTAs per SM) "
                         "instead of autotuning it (measurements of particular shapes)")
    args = ap.parse_args()
    if args.skip_extras:
        args.skip_fp64 = args.skip_e2e = args.skip_grids = True
    if args.grid_only:
        import torch
        from paper_2503_04428_gb300 import hydro as H
        print(json.dumps(time_grids(H, torch, work_stream(torch), args, only=args.grid_only,
                                    alu=alu_peaks(H))))
        return
    if args.dense_only:
        import torch
        from paper_2503_04428_gb300 import hydro as H
        print(json.dumps(time_dense(H, torch, work_stream(torch), args, 1, 0, None)))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2503_04428_gb300 import hydro as H

    w = rank_tubes(ws, rank, ntubes=args.tubes)
    total = int(w["lengths"].sum())
    gamma = w["gamma"]
    stream = work_stream(torch)
    weights, train_info = train_mlp(H, torch, gamma, 2)
    windows = trajectory_windows(args.steps)
    ksteps = sum(n for _, n in windows)
    dist_or_none = torch.distributed if ws > 1 else None

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # --- headline: FP32 + MLP guess, persistent batched launches of several steps
    U32 = torch.from_numpy(w["U"].astype(np.float32)).cuda()
    b32 = H.Batch(w["lengths"], gamma, precision=32, stream=stream.cuda_stream)
    b32.mlp_set(weights, True)
    if args.item_len:
        b32.set_launch(8, args.item_len, 2)
    b32.set_state(U32)
    b32.run(max(3, args.warmup), CFL)  # includes the autotuner on first use
    clocks = Clocks(local)
    barrier()
    clocks.start()
    t32, c32 = time_trajectory(torch, stream, b32, U32, windows)
    clk = clocks.stop()
    barrier()
    value, t32 = job_rate(t32, total, ksteps, dist_or_none, "cuda")
    ms = 1000.0 * t32 / ksteps
    extras = {}
    # the workload's whole 200-step run as one launch (hydro_batch_run(200)),
    # and the state it ends in, for the accuracy comparison
    out32 = times32 = None
    if not args.skip_fp64:
        tw, cw = time_trajectory(torch, stream, b32, U32, [(0, TRAJ)])
        out32 = b32.get_state().astype(np.float64)
        times32 = b32.times()
        vw, tw = job_rate(tw, total, TRAJ, dist_or_none, "cuda")
        extras["whole_run"] = {"value": vw, "unit": METRIC, "ms_per_step": 1000.0 * tw / TRAJ,
                               "steps": "all %d steps of the run in one launch" % TRAJ, "counters": cw}
    # the first steps alone (the easy regime: waves near the interfaces)
    k0 = min(ksteps, 20)
    te, ce = time_trajectory(torch, stream, b32, U32, [(0, k0)])
    ve, te = job_rate(te, total, k0, dist_or_none, "cuda")
    extras["early_window"] = {"value": ve, "unit": METRIC, "ms_per_step": 1000.0 * te / k0,
                              "steps": "1-%d of the run" % k0, "counters": ce}
    if not args.skip_fp64:
        # the FP32 form without the network, same steps
        b32.mlp_set(weights, False)
        tn, cn = time_trajectory(torch, stream, b32, U32, windows)
        b32.mlp_set(weights, True)
        vn, tn = job_rate(tn, total, ksteps, dist_or_none, "cuda")
        extras["mlp_gain"] = {"value_with_network": value, "value_without_network": vn,
                              "gain": value / vn, "counters_without_network": cn}
        extras["fp64_plain"], extras["accuracy"] = time_fp64(H, torch, stream, w, windows, ws, total, value,
                                                            out32, times32)
    e2e = None
    if not args.skip_e2e:
        e2e = time_e2e(H, torch, b32, w, window_steps(windows), ws, total, barrier)
    alu = None
    if not args.skip_fp64:
        extras["dense_state"] = time_dense(H, torch, stream, args, ws, rank, weights)
        alu = alu_peaks(H)
        extras["alu_peaks"] = alu
    if not args.skip_grids:
        extras["grid_sweep"] = time_grids(H, torch, stream, args, alu=alu)
    return report(args, ws, rank, b32, value, ms, t32, windows, total, e2e, clk, train_info, c32, extras)


def time_grids(H, torch, stream, args, only=None, alu=None):
    """The fused grid sweep on the 3D configurations: Sedov 256^3 (HLL, NV=5) in
    FP32 and FP64 and the spherical wedge 1024x128x128 (HLLC, NV=8, point +
    monopole gravity) in FP32; device-side CFL steps replayed as a graph."""
    from paper_2503_04428_gb300 import workloads as wl
    peak, _ = load_peaks()
    out = {}
    runs = (("sedov3d_fp32", lambda: wl.sedov3d(args.grid_n or 256), 32, 20),
            ("sedov3d_fp64", lambda: wl.sedov3d(args.grid_n or 256), 64, 5),
            ("wedge_fp32", wl.wedge, 32, 10),
            # the same wedge read through the gas + radiation EoS (Eq. 6-7) with
            # R = 1 and a = 2.5e8 in code units: P_rad/P_gas ~ 1 at r = 1, ~1e-3 at r = 1000
            ("wedge_fp32_rad", lambda: dict(wl.wedge(), eos_rad=(1.0, 2.5e8)), 32, 10))
    for name, make, prec, k in runs:
        if only and name != only:
            continue
        if only:
            k = args.steps
        case = make()
        name = "%s_%s" % (case["name"], name.split("_", 1)[1])
        dt = np.float32 if prec == 32 else np.float64
        g = H.Grid.from_case(dict(case, U=case["U"].astype(dt)), prec, stream=stream.cuda_stream)
        g.run(2, case["cfl"])  # autotuner on first use
        s0 = g.stats()
        t = timed_steps(torch, stream, lambda n: g.run(n, case["cfl"]), k)
        if only and args.profile_range:
            profiled_step(torch, lambda: g.run(1, case["cfl"]))
        cells = int(np.prod(case["n"]))
        nv = case["U"].shape[0]
        bytes_cell = 2 * nv * (4 if prec == 32 else 8)
        st = g.stats()
        t_its = (st["newton_iters"] - s0["newton_iters"]) / (cells * k) if case.get("eos_rad") else None
        g.close()
        gbs = bytes_cell * cells * k / t / 1e9
        out[name] = {"value": cells * k / t, "unit": METRIC, "ms_per_step": 1000.0 * t / k, "steps": k,
                     "hbm_gbs": gbs, "hbm_frac": gbs / peak, "tile": [st["tile_x"], st["tile_y"]],
                     "threads": st["threads"], "zchunk": st["zchunk"],
                     "gpu_launches_per_step": 3 if name.startswith("wedge") else 1,
                     "eos": "gas + radiation (Eq. 6-7)" if case.get("eos_rad") else "ideal gas (Eq. 5)"}
        if name.startswith("sedov") and prec == 32 and not only:
            # the same steps with the conserved totals accumulated in the step
            g = H.Grid.from_case(dict(case, U=case["U"].astype(dt)), prec, stream=stream.cuda_stream)
            g.set_step_totals(True)
            g.run(2, case["cfl"])
            tt = timed_steps(torch, stream, lambda n: g.run(n, case["cfl"]), k)
            tot = g.step_totals()
            g.close()
            out[name]["with_step_totals"] = {"ms_per_step": 1000.0 * tt / k, "cost": tt / t - 1.0,
                                             "totals_fp64": [float(x) for x in tot]}
        if t_its is not None:
            out[name]["temperature_newton"] = {
                "iters_per_cell_update": t_its,
                "note": "every EoS call's Newton iterations (15 calls per cell-update: the staged cells, "
                        "6 limited and 6 predicted face states and the new state), summed by the sweep"}
        fpc = sweep_fp64_flops_per_cell() if (prec == 64 and name.startswith("sedov")) else None
        if fpc is not None and alu is not None:
            ach = fpc * cells * k / t / 1e12
            out[name]["roofline"] = {"bound": "fp64", "achieved": ach, "peak": alu["fp64_tflops"],
                                     "unit": "TFLOP/s", "frac": ach / alu["fp64_tflops"],
                                     "flops_per_cell": fpc, "peak_kind": "measured (hydro_fma_rate)"}
        del case
    return out


def profiled_step(torch, fn):
    """One more step between cudaProfilerStart and cudaProfilerStop, so that
    ncu --profile-from-start off captures exactly this launch."""
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    fn()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


def time_dense(H, torch, stream, args, ws, rank, weights):
    """The headline form on a dense state: every cell's density and pressure
    perturbed by 1 %, so that no face has two identical states and every face
    runs the Newton iteration; with and without the network (weights None:
    without only)."""
    w = rank_tubes(ws, rank, perturb=0.01, ntubes=args.tubes)
    total = int(w["lengths"].sum())
    U = torch.from_numpy(w["U"].astype(np.float32)).cuda()
    b = H.Batch(w["lengths"], w["gamma"], precision=32, stream=stream.cuda_stream)
    if weights is not None:
        b.mlp_set(weights, True)
    b.set_state(U)
    b.run(2, CFL)
    k = min(max(5, args.steps // 4), 20)
    out = {"state": "every cell's rho and P x (1 + 0.01 U(-1,1))", "steps": "1-%d" % k}
    if weights is None:
        t, c = time_trajectory(torch, stream, b, U, [(0, k)])
        rate, t = job_rate(t, total, k, None, "cuda")
        out.update({"value": rate, "unit": METRIC, "ms_per_step": 1000.0 * t / k, "counters": c,
                    "tubes": args.tubes, "cells": total})
        if args.profile_range:
            b.set_state(U)
            profiled_step(torch, lambda: b.run(1, CFL))
        b.close()
        return out
    for on in (True, False):
        b.mlp_set(weights, on)
        t, c = time_trajectory(torch, stream, b, U, [(0, k)])
        rate, t = job_rate(t, total, k, torch.distributed if ws > 1 else None, "cuda")
        key = "with_network" if on else "without_network"
        out[key] = {"value": rate, "unit": METRIC, "ms_per_step": 1000.0 * t / k, "counters": c}
    out["value"] = out["with_network"]["value"]
    out["mlp_gain"] = out["with_network"]["value"] / out["without_network"]["value"]
    b.close()
    return out


def exact_l1_rho(H, w, rho, times):
    """Mean over tubes of the L1 density error against the exact Riemann
    solution at each tube's own time (sum_i |rho_i - rho_exact(x_i)| / n_b),
    the exact solution sampled by the library (hydro_exact_sample, FP64)."""
    lengths = np.asarray(w["lengths"], dtype=np.int64)
    face_of = np.repeat(np.arange(len(lengths), dtype=np.int64), lengths)
    start = np.repeat(np.cumsum(lengths) - lengths, lengths)
    i = np.arange(int(lengths.sum()), dtype=np.int64) - start
    nb = lengths[face_of].astype(np.float64)
    xi = ((i + 0.5) / nb - 0.5) / np.asarray(times)[face_of]
    ex = H.hydro_exact_sample(w["WL"], w["WR"], w["gamma"], face_of, xi)[:, 0]
    err = np.abs(np.asarray(rho, dtype=np.float64) - ex) / nb
    return float(np.bincount(face_of, weights=err).mean())


def time_fp64(H, torch, stream, w, windows, ws, total, value32, out32, times32):
    """The plain FP64 form of the same kernel (Toro guess) over the same steps
    of the run, and the accuracy of both forms after the workload's 200 steps."""
    gamma = w["gamma"]
    U64 = torch.from_numpy(w["U"]).cuda()
    b64 = H.Batch(w["lengths"], gamma, precision=64, stream=stream.cuda_stream)
    b64.set_state(U64)
    b64.run(3, CFL)
    k = sum(n for _, n in windows)
    t64, c64 = time_trajectory(torch, stream, b64, U64, windows)
    value64, t64 = job_rate(t64, total, k, torch.distributed if ws > 1 else None, "cuda")
    peak, _ = load_peaks()
    ach64 = 2 * 3 * 8 * total / (t64 / k) / 1e9
    fp64 = {"value": value64, "unit": METRIC, "ms_per_step": 1000.0 * t64 / k,
            "hbm_frac": ach64 / peak, "counters": c64, "speedup_of_headline": value32 / value64,
            "steps": "the headline's steps of the run"}
    # equal stated accuracy: both forms' per-tube L1(rho) error against the
    # exact solution after the workload's 200 steps, averaged over tubes
    tw, _ = time_trajectory(torch, stream, b64, U64, [(0, TRAJ)])
    vw, _ = job_rate(tw, total, TRAJ, torch.distributed if ws > 1 else None, "cuda")
    fp64["whole_run"] = {"value": vw, "unit": METRIC, "ms_per_step": 1000.0 * tw / TRAJ}
    out64 = b64.get_state()
    times64 = b64.times()
    b64.close()
    e32 = exact_l1_rho(H, w, out32[0], times32)
    e64 = exact_l1_rho(H, w, out64[0], times64)
    acc = {"rho_rel_l1_fp32mlp_vs_fp64": float(np.abs(out32[0] - out64[0]).sum() / np.abs(out64[0]).sum()),
           "l1_rho_vs_exact": {"fp32_mlp": e32, "fp64_toro": e64, "relative_difference": abs(e32 - e64) / e64,
                               "steps": TRAJ,
                               "definition": "mean over tubes of sum_i |rho_i - rho_exact(x_i, t_b)| / n_b"}}
    return fp64, acc


def time_e2e(H, torch, b32, w, positions, ws, total, barrier):
    """Same metric through the C ABI with pinned host buffers, at the same
    steps of the run: each timed step copies that step's state in from host
    memory, advances one step and copies the result out
    (hydro_batch_run_host: the copies of one group of tubes overlap the steps
    of the others); wall-clock time of the call.  The state for the next
    timed step is prepared untimed.  Also the unpipelined sequence set_state
    + run + get_state at the same steps."""
    host_in = torch.from_numpy(w["U"].astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    U0 = host_in.clone()
    b32.run_host(host_in, host_out, 1, CFL)  # captures the host-run graph
    ts = tu = 0.0
    b32.set_state(U0)
    cur = 0
    barrier()
    for p in positions:
        if p > cur:
            b32.run(p - cur, CFL)
        b32.get_state(host_in)  # this step's input, in host memory (untimed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b32.run_host(host_in, host_out, 1, CFL)
        ts += time.perf_counter() - t0
        # the plain sequence on the same input (the handle then holds the same result)
        t0 = time.perf_counter()
        b32.set_state(host_in)
        b32.run(1, CFL)
        b32.get_state(host_out)
        tu += time.perf_counter() - t0
        cur = p + 1
    barrier()
    rate, ts = job_rate(ts, total, len(positions), torch.distributed if ws > 1 else None, "cuda")
    rate_u, _ = job_rate(tu, total, len(positions), torch.distributed if ws > 1 else None, "cuda")
    nbytes = 3 * total * 4
    return {"value": rate, "unit": METRIC, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "api": "hydro_batch_run_host (8 groups of tubes, pinned buffers), the headline's steps of the run",
            "unpipelined_value": rate_u}


def report(args, ws, rank, b32, value, ms, t32, windows, total, e2e, clk, train_info, c32, extras):
    ksteps = sum(n for _, n in windows)
    peak, peak_kind = load_peaks()
    alg_bytes = 2 * 3 * 4 * total  # read U^n and write U^{n+1} every step, FP32
    per_launch = ksteps / len(windows)  # steps per timed launch
    achieved = alg_bytes / (t32 / ksteps) / 1e9
    st = b32.stats()
    tr = profiled_traffic(st["tile_x"])
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None if tr is None else tr * per_launch, "peak_kind": peak_kind,
            "kernel": "batched_kernel<float>", "algorithmic_bytes_per_launch": alg_bytes * per_launch,
            "steps_per_launch": per_launch,
            "window": "the headline's timed windows (one launch of several steps each)"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": ksteps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.tubes == NTUBES else "%d-tube subset of: %s" % (args.tubes, WORKLOAD),
                       "tubes_per_gpu": len(b32.lengths), "cells_per_gpu": total,
                       "form": "FP32 bulk + MLP p* guess (two-shock faces, jump > 4) + persistent batched kernel, "
                               "one launch per window of steps (per-tube step dependencies, no grid-wide barrier)",
                       "cfl": CFL, "l2": "state 208 MB per buffer > 129 MB L2 (no flush needed)",
                       "timing": "%d steps of the workload's 200-step run (one pass from the initial state) in "
                                 "windows of consecutive steps %s ([first step, count]), each window one launch "
                                 "timed with CUDA events, an untimed launch advancing the run between them"
                                 % (ksteps, json.dumps([[p, n] for p, n in windows])),
                       "partition": "the job is %d x 4096 tubes (seed 2) cut into %d ranges of about equal cells"
                                    % (ws, ws),
                       "launch": {"item_cells": st["tile_x"], "warps_per_cta": st["tile_y"], "ctas": st["zchunk"]}},
            "e2e": e2e,
            "gpu_launches": len(windows),
            "clocks": clk,
            "roofline": roof,
            "cpu_baseline": cpu,
            "solver": c32,
            "mlp": train_info,
        }
        line.update(extras)
        print(json.dumps(line))
    b32.close()


if __name__ == "__main__":
    main()
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed
        torch.distributed.destroy_process_group()
