"""Benchmark of the batched exact-Riemann workload (4096 tubes, 256-8192 cells each).

One step = one MUSCL-Hancock time step of every tube (primitive recovery,
limited reconstruction, Hancock predictor, exact Riemann solve with the
learned or Toro guess, conservative update, per-tube CFL speed), i.e. one
persistent launch of the batched kernel replayed from a CUDA graph.

Headline (`value`): FP32 bulk + MLP star-pressure guess + batched/graph, in
cell-updates/s over all ranks, inputs resident in HBM.  Beside it: the plain
FP64 + Toro-guess form of the same kernel (`fp64_plain`), the end-to-end rate
through the C ABI with host buffers (`e2e`), the HBM roofline of the kernel,
and the FP64 CPU oracle on a bounded sample (`cpu_baseline`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank advances its own 4096 tubes (weak scaling, no data
exchange); timing is the max over ranks.
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
            "source": "hydro_fma_rate: 8 independent FMA chains per thread, 8 CTAs of 256 per SM"}


def profiled_traffic(item_len):
    """DRAM bytes per launch from the committed ncu summary, if it matches this
    kernel and the work-item length in effect (item boundaries re-fetch halos)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    d = json.load(open(TRAFFIC_FILE))
    if d.get("kernel_hash") != kernel_hash() or d.get("item_len") != item_len:
        return None
    return float(d["dram_bytes_per_launch"])


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


def rank_seed(rank):
    """Each rank advances its own 4096 tubes (weak scaling): a seed per rank."""
    return 2 + 1000 * rank


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
    ap.add_argument("--steps", type=int, default=200, help="steps per timed pass (the workload's K = 200)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed passes, each from the initial state (the state reset is not timed)")
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tubes", type=int, default=NTUBES, help="tubes per GPU (profiling a smaller case)")
    ap.add_argument("--skip-fp64", action="store_true", help="do not time the plain FP64 form")
    ap.add_argument("--skip-e2e", action="store_true", help="do not time the host-buffer path")
    ap.add_argument("--skip-grids", action="store_true", help="do not time the 3D grid sweeps")
    ap.add_argument("--grid-only", choices=["sedov3d_fp32", "sedov3d_fp64", "wedge_fp32", "wedge_fp32_rad"],
                    help="time one grid sweep only (profiling)")
    ap.add_argument("--grid-n", type=int, default=0, help="cells per axis for --grid-only sedov3d")
    args = ap.parse_args()
    if args.grid_only:
        import torch
        from paper_2503_04428_gb300 import hydro as H
        print(json.dumps(time_grids(H, torch, torch.cuda.current_stream(), args, only=args.grid_only,
                                    alu=alu_peaks(H))))
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
    from paper_2503_04428_gb300 import workloads as wl

    seed = rank_seed(rank)
    w = wl.tubes(args.tubes, seed=seed)
    total = int(w["lengths"].sum())
    gamma = w["gamma"]
    stream = torch.cuda.current_stream()
    weights, train_info = train_mlp(H, torch, gamma, seed)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # --- headline: FP32 + MLP guess, batched persistent launch replayed as a graph
    U32 = torch.from_numpy(w["U"].astype(np.float32)).cuda()
    b32 = H.Batch(w["lengths"], gamma, precision=32, stream=stream.cuda_stream)
    b32.mlp_set(weights, True)
    b32.set_state(U32)
    b32.run(args.warmup, CFL)  # includes the autotuner on first use
    clocks = Clocks(local)
    t32 = 0.0
    it_acc = mlp_acc = face_acc = 0
    barrier()
    clocks.start()
    for _ in range(args.repeats):
        b32.set_state(U32)
        s0 = b32.stats()
        t32 += timed_steps(torch, stream, lambda k: b32.run(k, CFL), args.steps)
        s1 = b32.stats()
        face_acc += s1["faces"] - s0["faces"]
        it_acc += s1["newton_iters"] - s0["newton_iters"]
        mlp_acc += s1["mlp_faces"] - s0["mlp_faces"]
    clk = clocks.stop()
    barrier()
    nsteps = args.steps * args.repeats
    value, t32 = job_rate(t32, total, nsteps, torch.distributed if ws > 1 else None, "cuda")
    it32 = it_acc / max(face_acc, 1)
    mlp_frac = mlp_acc / max(face_acc, 1)
    ms = 1000.0 * t32 / nsteps
    out32 = b32.get_state().astype(np.float64)
    times32 = b32.times()

    value64 = t64 = it64 = rho_rel = None
    k64 = 0
    accuracy = {"rho_rel_l1_fp32mlp_vs_fp64": None}
    if not args.skip_fp64:
        value64, t64, k64, it64, rho_rel, out64, times64 = time_fp64(H, torch, stream, w, args, ws, total,
                                                                       out32)
        # equal stated accuracy: both forms' per-tube L1(rho) error against the
        # exact solution at the final time, averaged over tubes
        e32 = exact_l1_rho(H, w, out32[0], times32)
        e64 = exact_l1_rho(H, w, out64[0], times64)
        accuracy = {"rho_rel_l1_fp32mlp_vs_fp64": rho_rel,
                    "l1_rho_vs_exact": {"fp32_mlp": e32, "fp64_toro": e64,
                                        "relative_difference": abs(e32 - e64) / e64,
                                        "steps": args.steps,
                                        "definition": "mean over tubes of sum_i |rho_i - rho_exact(x_i, t_b)| / n_b"}}
    e2e = None
    if not args.skip_e2e:
        e2e = time_e2e(H, torch, b32, w, args, ws, total, barrier)
    dense = None
    if not args.skip_fp64:
        dense = time_dense(H, torch, stream, args, ws, weights)
    alu = alu_peaks(H)
    grids = None
    if not args.skip_grids:
        grids = time_grids(H, torch, stream, args, alu=alu)
    return report(args, ws, rank, b32, value, ms, t32, total, e2e, clk, train_info, it32, mlp_frac,
                  value64, t64, k64, it64, accuracy, dense, grids, alu)


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
        t = timed_steps(torch, stream, lambda n: g.run(n, case["cfl"]), k)
        cells = int(np.prod(case["n"]))
        nv = case["U"].shape[0]
        bytes_cell = 2 * nv * (4 if prec == 32 else 8)
        st = g.stats()
        g.close()
        gbs = bytes_cell * cells * k / t / 1e9
        out[name] = {"value": cells * k / t, "unit": METRIC, "ms_per_step": 1000.0 * t / k, "steps": k,
                     "hbm_gbs": gbs, "hbm_frac": gbs / peak, "tile": [st["tile_x"], st["tile_y"]],
                     "threads": st["threads"], "zchunk": st["zchunk"],
                     "gpu_launches_per_step": 3 if name.startswith("wedge") else 1,
                     "eos": "gas + radiation (Eq. 6-7)" if case.get("eos_rad") else "ideal gas (Eq. 5)"}
        fpc = sweep_fp64_flops_per_cell() if (prec == 64 and name.startswith("sedov")) else None
        if fpc is not None and alu is not None:
            ach = fpc * cells * k / t / 1e12
            out[name]["roofline"] = {"bound": "fp64", "achieved": ach, "peak": alu["fp64_tflops"],
                                     "unit": "TFLOP/s", "frac": ach / alu["fp64_tflops"],
                                     "flops_per_cell": fpc, "peak_kind": "measured (hydro_fma_rate)"}
        del case
    return out


def time_dense(H, torch, stream, args, ws, weights):
    """The headline form on a dense state: every cell's density and pressure
    perturbed by 1 %, so that no face has two identical states and every face
    runs the Newton iteration."""
    from paper_2503_04428_gb300 import workloads as wl
    w = wl.tubes(args.tubes, seed=rank_seed(dist_info()[1]), perturb=0.01)
    total = int(w["lengths"].sum())
    U = torch.from_numpy(w["U"].astype(np.float32)).cuda()
    b = H.Batch(w["lengths"], w["gamma"], precision=32, stream=stream.cuda_stream)
    b.mlp_set(weights, True)
    b.set_state(U)
    b.run(2, CFL)
    b.set_state(U)
    k = max(5, args.steps // 2)
    s0 = b.stats()
    t = timed_steps(torch, stream, lambda n: b.run(n, CFL), k)
    s1 = b.stats()
    rate, t = job_rate(t, total, k, torch.distributed if ws > 1 else None, "cuda")
    it = (s1["newton_iters"] - s0["newton_iters"]) / max(s1["faces"] - s0["faces"], 1)
    b.close()
    return {"value": rate, "unit": METRIC, "ms_per_step": 1000.0 * t / k, "newton_iters_per_face": it,
            "state": "every cell's rho and P x (1 + 0.01 U(-1,1))"}


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


def time_fp64(H, torch, stream, w, args, ws, total, out32):
    """The plain FP64 form of the same kernel (Toro guess), and the difference
    of its density field from the headline form's after the same steps."""
    gamma = w["gamma"]
    U64 = torch.from_numpy(w["U"]).cuda()
    b64 = H.Batch(w["lengths"], gamma, precision=64, stream=stream.cuda_stream)
    b64.set_state(U64)
    b64.run(max(2, args.warmup // 2), CFL)
    b64.set_state(U64)
    k64 = max(5, args.steps // 2)  # FP64 is ~15x slower: half a pass
    r0 = b64.stats()
    t64 = timed_steps(torch, stream, lambda k: b64.run(k, CFL), k64)
    r1 = b64.stats()
    it64 = (r1["newton_iters"] - r0["newton_iters"]) / max(r1["faces"] - r0["faces"], 1)
    value64, t64 = job_rate(t64, total, k64, torch.distributed if ws > 1 else None, "cuda")
    # same number of steps from the same start for an accuracy comparison
    b64.set_state(U64)
    b64.run(args.steps, CFL)
    out64 = b64.get_state()
    times64 = b64.times()
    rho_rel = float(np.abs(out32[0] - out64[0]).sum() / np.abs(out64[0]).sum())
    b64.close()
    return value64, t64, k64, it64, rho_rel, out64, times64


def time_e2e(H, torch, b32, w, args, ws, total, barrier):
    """Same metric through the C ABI with pinned host buffers: every step
    copies the state in from host memory, advances one step and copies it
    out (hydro_batch_run_host: the copies of one group of tubes overlap the
    steps of the others).  Also the unpipelined sequence set_state + run +
    get_state for reference."""
    host_in = torch.from_numpy(w["U"].astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ke = max(3, args.steps // 5)
    b32.run_host(host_in, host_out, 1, CFL)
    barrier()
    te0 = time.perf_counter()
    for _ in range(ke):
        b32.run_host(host_in, host_out, 1, CFL)
    torch.cuda.synchronize()
    te = time.perf_counter() - te0
    rate, te = job_rate(te, total, ke, torch.distributed if ws > 1 else None, "cuda")
    barrier()
    ts0 = time.perf_counter()
    for _ in range(ke):
        b32.set_state(host_in)
        b32.run(1, CFL)
        b32.get_state(host_out)
    torch.cuda.synchronize()
    ts = time.perf_counter() - ts0
    nbytes = 3 * total * 4
    return {"value": rate, "unit": METRIC, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "api": "hydro_batch_run_host (8 groups of tubes, pinned buffers)",
            "unpipelined_value": ws * total * ke / ts}


def report(args, ws, rank, b32, value, ms, t32, total, e2e, clk, train_info, it32, mlp_frac,
           value64, t64, k64, it64, accuracy, dense=None, grids=None, alu=None):
    peak, peak_kind = load_peaks()
    nsteps = args.steps * args.repeats
    alg_bytes = 2 * 3 * 4 * total  # read U^n and write U^{n+1}, FP32
    achieved = alg_bytes / (t32 / nsteps) / 1e9
    st = b32.stats()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": profiled_traffic(st["tile_x"]), "peak_kind": peak_kind, "kernel": "batched_kernel<float>",
            "algorithmic_bytes_per_launch": alg_bytes}
    fp64 = None
    if value64 is not None:
        ach64 = 2 * 3 * 8 * total / (t64 / k64) / 1e9
        fp64 = {"value": value64, "unit": METRIC, "ms_per_step": 1000.0 * t64 / k64, "hbm_frac": ach64 / peak,
                "fp64_peak_tflops": alu["fp64_tflops"] if alu else None,
                "newton_iters_per_face": it64, "speedup_of_headline": value / value64}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": nsteps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.tubes == NTUBES else "%d-tube subset of: %s" % (args.tubes, WORKLOAD),
                       "tubes_per_gpu": args.tubes, "cells_per_gpu": total,
                       "form": "FP32 bulk + MLP p* guess (two-shock faces, jump > 4) + persistent batched kernel + CUDA graph",
                       "cfl": CFL, "l2": "state 208 MB per buffer > 129 MB L2 (no flush needed)",
                       "timing": "%d passes of %d steps from the initial state (state reset untimed)"
                                 % (args.repeats, args.steps),
                       "launch": {"chunk": st["tile_x"], "ctas": st["zchunk"]}},
            "e2e": e2e,
            "gpu_launches": nsteps,
            "clocks": clk,
            "roofline": roof,
            "cpu_baseline": cpu,
            "fp64_plain": fp64,
            "dense_state": dense,
            "grid_sweep": grids,
            "alu_peaks": alu,
            "newton_iters_per_face": {"fp32_mlp": it32, "fp64_toro": it64},
            "mlp": dict(train_info, guessed_face_fraction=mlp_frac),
            "accuracy": accuracy,
        }))
    b32.close()


if __name__ == "__main__":
    main()
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed
        torch.distributed.destroy_process_group()
