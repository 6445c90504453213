"""Benchmark: one channel-flow step (Poisson + three z-implicit Helmholtz
solves, FP64) on the 512 x 384 x 384 tanh(1.8) grid, through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is the whole hot path over one synthetic input set already resident in
HBM: packed x rFFT, y FFT, z Thomas, inverse y and x transforms (the five
kernels of cfs_poisson_solve, launched stage by stage so that each kernel is
timed by CUDA events inside the timed region), then three Algorithm 2 solves
(u and v cell-centred, w face-located).  Every field (604 MB) is larger than
L2, so no flush is needed between steps.

Metric: ns per grid point per step (lower is better).  With N GPUs each rank
runs its own replica of the step (the solves share nothing), and the value is
the max-over-ranks time divided by all ranks' points.  Rank 0 prints one JSON
line.  `--impl reference` times the CPU oracle on a bounded sample instead.

After the timed steps, the line's "mixed" object compares FP32 solves with
FP64 iterative refinement (tolerance 1e-10) against the FP64 solve on the
1024 x 768 x 512 uniform workload (`--no-mixed` skips it).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2502_06296_gb300 import synth  # noqa: E402

METRIC = "Poisson+Helmholtz ns/grid-pt, % HBM peak; mixed vs FP64 at 1e-10; p99 latency"
UNIT = "ns/grid-pt"
CFG = synth.CHANNEL
STAGES = ["x_forward", "y_forward", "z_thomas", "y_inverse", "x_inverse", "helm_u", "helm_v",
          "helm_w"]
HELM_STAGES = ("helm_u", "helm_v", "helm_w")
KERNEL_OF_STAGE = {"x_forward": "rfft_x_kernel<false>", "y_forward": "fft_y_kernel<false>",
                   "z_thomas": "thomas_kernel", "y_inverse": "fft_y_kernel<true>",
                   "x_inverse": "rfft_x_kernel<true>", "helm_u": "pcr_kernel",
                   "helm_v": "pcr_kernel", "helm_w": "pcr_kernel"}
SOURCE_OF_STAGE = {"x_forward": "fft_x.cu", "x_inverse": "fft_x.cu", "y_forward": "fft_y.cu",
                   "y_inverse": "fft_y.cu", "z_thomas": "thomas.cu", "helm_u": "pcr.cu",
                   "helm_v": "pcr.cu", "helm_w": "pcr.cu"}


class nvtx_range:
    """An NVTX range (profilers can restrict a capture to it: ncu --nvtx
    --nvtx-include "<name>/"); nothing if NVTX is unavailable."""

    def __init__(self, name: str):
        self.name = name

    def __enter__(self):
        try:
            import torch
            torch.cuda.nvtx.range_push(self.name)
            self.on = True
        except Exception:
            self.on = False
        return self

    def __exit__(self, *exc):
        if self.on:
            import torch
            torch.cuda.nvtx.range_pop()


def set_helm_method(thomas: bool):
    """The Helmholtz stages run Algorithm 2 (pcr_kernel) or Thomas sweeps
    (helm_thomas_kernel), as the plan's option says."""
    for s in HELM_STAGES:
        KERNEL_OF_STAGE[s] = "helm_thomas_kernel" if thomas else "pcr_kernel"
        SOURCE_OF_STAGE[s] = "helm_thomas.cu" if thomas else "pcr.cu"


# ----------------------------------------------------------------------------
# Algorithmic work per launch (5 N log2 N flops per complex FFT of length N,
# half that for a real FFT; 16 bytes per point read + written)
# ----------------------------------------------------------------------------

def stage_work(stage: str, nx: int, ny: int, nz: int):
    npts = nx * ny * nz
    if stage.startswith("x_"):
        flops = ny * nz * 2.5 * nx * np.log2(nx)
    elif stage.startswith("y_"):
        flops = (nx // 2) * nz * 5.0 * ny * np.log2(ny)
    elif stage == "z_thomas":
        flops = 5.0 * npts  # forward: 2 mul + 1 add, backward: 1 mul + 1 add
    elif KERNEL_OF_STAGE[stage] == "helm_thomas_kernel":
        flops = 5.0 * npts  # forward: 1 mul + 1 FMA, backward: 1 FMA
    else:
        flops = 9.0 * npts  # Algorithm 2: 2 + 2 (Step 2) + 5 (Step 4)
    return float(flops), 16.0 * npts


def fp64_peak_tflops(sm_count: int = 152, clock_mhz: float = 2070.0) -> float:
    """Two FP64 FMA lanes per SM per clock (the GB300 rate: 1.25 TFLOP/s
    nominal), counted as 2 flops each, at the maximum SM clock."""
    return sm_count * 2 * 2 * clock_mhz * 1e6 / 1e12


def run_fma_probe(chanfs, device_index: int, reps: int = 5) -> dict:
    """FP64 and FP32 FMA rates of this GPU (cfs_probe_fma), with the SM clock
    sampled meanwhile: the evidence for the FP64 unit count in the peak."""
    with ClockSampler(device_index) as clk:
        r64 = [chanfs.probe_fma(64, 1 << 14) for _ in range(reps)]
        r32 = [chanfs.probe_fma(32, 1 << 20) for _ in range(reps)]
    clock = clk.summary() or {}
    import torch
    nsm = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz = clock.get("sm_mhz") or 0.0
    f64 = statistics.median(r for r, _ in r64)
    f32 = statistics.median(r for r, _ in r32)
    out = {"fp64_fma_per_s": f64, "fp32_fma_per_s": f32, "sms": nsm,
           "launch_ms_fp64": round(statistics.median(m for _, m in r64), 3),
           "launch_ms_fp32": round(statistics.median(m for _, m in r32), 3),
           "sm_mhz_median": mhz, "clock_samples": clock.get("samples"),
           "reasons": clock.get("reasons"), "reps": reps,
           "how": "cfs_probe_fma: one full wave of 256-thread blocks, 16 independent FMA chains per "
                  "thread, CUDA events; median of reps"}
    if mhz:
        out["fp64_fma_per_sm_per_clk"] = f64 / (nsm * mhz * 1e6)
        out["fp32_fma_per_sm_per_clk"] = f32 / (nsm * mhz * 1e6)
    return out


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def profiled_traffic(stage: str):
    """Bytes per launch from the committed ncu summary of this stage's kernel,
    or None if there is none or the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{stage}_channel_512x384x384.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    if not m or not h:
        return None
    src = os.path.join(ROOT, "paper_2502_06296_gb300", "csrc", SOURCE_OF_STAGE[stage])
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return float(m.group(1)) if cur == h.group(1) else None


# ----------------------------------------------------------------------------
# Clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------
# Distributed helpers (replicas only; the data path has no collective)
# ----------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, device=None) -> float:
    """Max over ranks of a host scalar (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(max_ms_total: float, steps: int, npts_per_rank: int, world: int) -> dict:
    """Whole-job figures from the max-over-ranks elapsed time of `steps` steps."""
    ms_per_step = max_ms_total / steps
    ns_per_pt = ms_per_step * 1e6 / (npts_per_rank * world)
    return {"ms_per_step": ms_per_step, "value": ns_per_pt}


# ----------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ----------------------------------------------------------------------------

def oracle_sample_step(nz_sample: int):
    """The channel step on the full x-y planes and nz_sample tanh(1.8) cells:
    one Poisson and three Helmholtz solves by the CPU oracle.  Returns
    (seconds, points)."""
    import oracle
    nx, ny = CFG["nx"], CFG["ny"]
    dz = synth.tanh_dz(nz_sample, CFG["beta"])
    shape = (nz_sample, ny, nx)
    f = synth.remove_weighted_mean(synth.normal(CFG["seed"], shape), dz)
    rhs = [synth.normal(CFG["seed"] + 1 + i, shape) for i in range(3)]
    t0 = time.perf_counter()
    oracle.poisson_solve(f, CFG["lx"], CFG["ly"], dz, oracle.NEUMANN)
    for r, loc in zip(rhs, (oracle.CENTER, oracle.CENTER, oracle.FACE)):
        oracle.helmholtz_solve(r, dz, synth.CHANNEL_C, loc, oracle.THOMAS)
    return time.perf_counter() - t0, nx * ny * nz_sample


def cpu_baseline(nz_sample: int = 96):
    secs, npts = oracle_sample_step(nz_sample)
    return {"value": secs * 1e9 / npts, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one step (Poisson + 3 Helmholtz) on {CFG['nx']}x{CFG['ny']}x{nz_sample} "
                      f"(full x-y planes, {nz_sample} tanh(1.8) cells), single-threaded FP64 C, "
                      f"{secs:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    nz_s = 24
    for _ in range(args.warmup):
        oracle_sample_step(nz_s)
    tot, npts = 0.0, 0
    for _ in range(args.steps):
        s, n = oracle_sample_step(nz_s)
        tot += s
        npts = n
    ns = tot * 1e9 / (npts * args.steps)
    line = {"metric": METRIC, "value": ns, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": CFG["name"], "sample_nz": nz_s, "parallelism": "cpu_1core"},
            "cpu_baseline": {"value": ns, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: Poisson + 3 Helmholtz on {CFG['nx']}x{CFG['ny']}x{nz_s}"},
            "e2e": {"value": ns, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# FP32 solves + FP64 refinement against the FP64 solve (1024 x 768 x 512)
# ----------------------------------------------------------------------------

def run_mixed(chanfs, torch, device, reps: int = 5, warmup: int = 3, nz: int = 0):
    """Poisson solve of the 1024 x 768 x 512 uniform workload by an FP64 plan
    and by a CFS_F32_REFINED plan (tolerance 1e-10, at most 4 FP32 solves),
    each timed by CUDA events over `reps` solves after `warmup`; the refined
    result is compared with the FP64 one.  Fields are 3.2 GB (larger than L2)."""
    cfg = dict(synth.PRECISION)
    if nz:  # reduced wall-normal size (profiling captures only)
        cfg.update(nz=nz, name=f"poisson_uniform_{cfg['nx']}x{cfg['ny']}x{nz}")
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    npts = nx * ny * nz
    dz = synth.grid_dz(cfg)
    f = torch.from_numpy(synth.precision_rhs(cfg)).to(device)
    stream = torch.cuda.current_stream(device)
    out, res = {}, {}
    for name, dtype in (("f64", chanfs.F64), ("f32_refined", chanfs.F32_REFINED)):
        with chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, chanfs.NEUMANN, dtype) as plan:
            tuned = plan.autotune()  # kernel shapes by measurement, for both plans
            p = torch.empty_like(f)
            for _ in range(warmup):
                plan.poisson_solve(f, out=p)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
            iters = []
            with nvtx_range(f"solve_{name}"):
                ev[0].record(stream)
                for r in range(reps):
                    plan.poisson_solve(f, out=p)
                    ev[r + 1].record(stream)
                    if dtype == chanfs.F32_REFINED:
                        iters.append(plan.last_info())
                torch.cuda.synchronize()
            ms = [ev[r].elapsed_time(ev[r + 1]) for r in range(reps)]
            entry = {"ms": round(statistics.median(ms), 4),
                     "ns_per_pt": statistics.median(ms) * 1e6 / npts,
                     "device_status": plan.check(), "kernel_shapes": tuned}
            if iters:
                entry["fp32_solves"] = max(i for i, _ in iters)
                entry["rel_residual"] = max(r for _, r in iters)
            out[name] = entry
            res[name] = p
    err = float((res["f32_refined"] - res["f64"]).abs().max() / res["f64"].abs().max())
    out.update({"workload": cfg["name"], "tol": 1e-10, "rel_err_vs_f64": err,
                "speedup": out["f64"]["ms"] / out["f32_refined"]["ms"], "reps": reps,
                "timing": "median of CUDA-event times of single solves on the launching stream; "
                          "refined solves include their host reads of the residual norm"})
    return out


# ----------------------------------------------------------------------------
# Fully implicit 3-D Helmholtz (Eq. 8) on the channel workload
# ----------------------------------------------------------------------------

def run_helmholtz3d(chanfs, torch, device, plan, rhs, outs, reps: int = 5):
    """u, v (centred) and w (face) fully implicit solves with the channel's
    alpha nu dt, FP64, on the channel plan; median over reps of the three."""
    c = synth.CHANNEL_C
    locs = (chanfs.CENTER, chanfs.CENTER, chanfs.FACE)
    for loc in (chanfs.CENTER, chanfs.FACE):
        plan.helmholtz3d_prepare(c, loc)

    def three():
        for r, o, loc in zip(rhs, outs, locs):
            plan.helmholtz3d_solve(c, r, loc, out=o)

    three()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        three()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    npts = rhs[0].numel()
    t = statistics.median(ms)
    return {"workload": CFG["name"], "solves": "u, v centred + w face, Dirichlet, c = alpha nu dt",
            "ms_three_solves": round(t, 4), "ns_per_pt_per_solve": t * 1e6 / (3 * npts),
            "launches_per_solve": 5, "precision": "f64"}


# ----------------------------------------------------------------------------
# Walls in y (DCT-II / DST-II) on the channel workload
# ----------------------------------------------------------------------------

def run_ywalls(chanfs, torch, device, f, dz, reps: int = 5):
    """The channel's Poisson solve with Neumann or Dirichlet walls in y
    instead of periodicity, FP64, median of reps solves each."""
    nz, ny, nx = f.shape
    out = {"workload": CFG["name"], "precision": "f64"}
    p = torch.empty_like(f)
    for name, ybc in (("neumann", chanfs.Y_NEUMANN), ("dirichlet", chanfs.Y_DIRICHLET)):
        with chanfs.Plan(nx, ny, nz, CFG["lx"], CFG["ly"], dz, chanfs.NEUMANN, chanfs.F64,
                         ybc) as plan:
            plan.poisson_solve(f, out=p)
            torch.cuda.synchronize()
            ms = []
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                plan.poisson_solve(f, out=p)
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            t = statistics.median(ms)
            out[name] = {"ms": round(t, 4), "ns_per_pt": t * 1e6 / f.numel(),
                         "device_status": plan.check()}
    return out


# ----------------------------------------------------------------------------
# Batched ensemble: 48 boxes, grouped FP32 + FP64-refined solves vs per box
# ----------------------------------------------------------------------------

def run_ensemble(chanfs, torch, device, reps: int = 3):
    """One ensemble step = per box a Poisson solve (Neumann) and three
    Helmholtz solves (u, v centred, w face; the box's own alpha nu dt).
    Grouped (one launch per stage for all boxes, autotuned shapes) against
    the same work box by box in FP64 and box by box refined."""
    cfg = synth.ENSEMBLE
    boxes = synth.ensemble_boxes(cfg)
    gen = torch.Generator(device=device)
    gen.manual_seed(cfg["seed"])
    plans32, plans64, f, rhs = [], [], [], []
    t0 = time.perf_counter()
    for nx, ny, nz, beta, c in boxes:
        dz = synth.tanh_dz(nz, beta)
        p32 = chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, chanfs.NEUMANN, chanfs.F32_REFINED)
        p32.autotune()
        p64 = chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, chanfs.NEUMANN, chanfs.F64)
        p64.autotune()
        plans32.append(p32)
        plans64.append(p64)
        f.append(torch.randn(nz, ny, nx, dtype=torch.float64, device=device, generator=gen))
        rhs.append([torch.randn(nz, ny, nx, dtype=torch.float64, device=device, generator=gen)
                    for _ in range(3)])
    setup_s = time.perf_counter() - t0
    npts = sum(nx * ny * nz for nx, ny, nz, _, _ in boxes)
    cs = [b[4] for b in boxes]
    locs = (chanfs.CENTER, chanfs.CENTER, chanfs.FACE)
    p = [torch.empty_like(x) for x in f]
    u = [[torch.empty_like(x) for x in r] for r in rhs]
    group = chanfs.Group(plans32)

    def grouped():
        group.poisson_solve(f, p)
        for k in range(3):
            group.helmholtz_solve(cs, [r[k] for r in rhs], [locs[k]] * len(boxes), [x[k] for x in u])

    def per_box(plans):
        def step():
            for b, pl in enumerate(plans):
                pl.poisson_solve(f[b], out=p[b])
                for k in range(3):
                    pl.helmholtz_solve(cs[b], rhs[b][k], locs[k], out=u[b][k])
        return step

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    grouped()  # a launch shape is captured as a graph at its second solve
    t_group = timed(grouped)
    with nvtx_range("ensemble_grouped_step"):  # one more step, for profilers
        grouped()
        torch.cuda.synchronize()
    info = group.last_info()
    group.set_graphs(False)  # the same launches, refinement loop on the host
    t_group_host = timed(grouped)
    with nvtx_range("ensemble_grouped_step_direct"):  # kernel by kernel, for profilers
        grouped()
        torch.cuda.synchronize()
    group.set_graphs(True)
    # Idle time between a grouped step's nodes: the device time of each copy
    # and kernel (direct launches, one event pair each), summed, against the
    # graph-launched step.  Best of reps.
    group.set_trace(True)
    sums, launches = [], 0
    for _ in range(reps):
        traced = []
        group.poisson_solve(f, p)
        traced += group.trace()
        for k in range(3):
            group.helmholtz_solve(cs, [r[k] for r in rhs], [locs[k]] * len(boxes), [x[k] for x in u])
            traced += group.trace()
        sums.append(sum(traced))
        launches = len(traced)
    group.set_trace(False)
    t64 = timed(per_box(plans64))
    t32 = timed(per_box(plans32))
    group.close()
    opts = {}
    for (nx, ny, nz, _, _), pl in zip(boxes, plans32):
        opts[f"{nx}x{ny}x{nz}"] = [pl.get_option(o) for o in (
            chanfs.OPT_X_LINES, chanfs.OPT_Y_TILE, chanfs.OPT_THOMAS_TILE, chanfs.OPT_PCR_PARTS,
            chanfs.OPT_HELM_FP64, chanfs.OPT_HELM_THOMAS, chanfs.OPT_HELM_THOMAS32)]
    for pl in plans32 + plans64:
        pl.close()
    return {"workload": cfg["name"], "boxes": len(boxes), "points": npts,
            "step": "per box: Poisson (Neumann) + 3 Helmholtz (u, v centred, w face)",
            "grouped_refined_ms": round(t_group, 3),
            "grouped_refined_host_loop_ms": round(t_group_host, 3),
            "grouped": "one CUDA graph per solve (refinement loop in a conditional WHILE node); "
                       "host_loop: the same launches with one host wait per iteration",
            "per_box_f64_ms": round(t64, 3),
            "per_box_refined_ms": round(t32, 3),
            "grouped_ns_per_pt": t_group * 1e6 / npts, "per_box_f64_ns_per_pt": t64 * 1e6 / npts,
            "speedup_vs_per_box_f64": t64 / t_group,
            "launch_trace": {"copies_and_kernels": launches,
                             "device_ms_sum": round(min(sums), 3),
                             "graph_step_ms": round(t_group, 3),
                             "idle_ms": round(t_group - min(sums), 3),
                             "how": "cfs_group_set_trace: an event pair around every copy and "
                                    "kernel of one step launched directly, summed (best of "
                                    "reps); idle = graph-launched step - sum"},
            "max_fp32_solves_last_helmholtz": max(i for i, _ in info),
            "max_rel_residual_last_helmholtz": max(r for _, r in info),
            "autotuned": "per refined box size: x_lines, y_tile, thomas_tile, pcr_parts, "
                         "helm_fp64, helm_thomas, helm_thomas32 (Thomas sweeps vs Algorithm 2)",
            "options": opts, "setup_s": round(setup_s, 1),
            "timing": f"median of {reps} CUDA-event timings of whole steps; fields larger than "
                      "L2 in total (no flush between steps)"}


HELM_SIZES = [(128, 96, 64, 2.2, 1e-4), (192, 192, 128, 2.0, 3e-5), (256, 192, 192, 1.8, 1e-5),
              (512, 384, 384, 1.8, 9.615e-9)]


def run_refined_helmholtz(chanfs, torch, device, reps: int = 7, sizes=HELM_SIZES):
    """z-implicit Helmholtz per size (ensemble and serving shapes): FP64
    Algorithm 2, FP64 Thomas sweeps, and the refined solves of a
    CFS_F32_REFINED plan -- one pass over the field (FP32 Algorithm 2 and
    double-float residuals on chip) at each partition count it runs with,
    and the loop with FP32 Thomas inner solves -- median CUDA-event times."""
    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    out = []
    gen = torch.Generator(device=device)
    gen.manual_seed(1234)
    for nx, ny, nz, beta, c in sizes:
        dz = synth.tanh_dz(nz, beta)
        r = torch.randn(nz, ny, nx, dtype=torch.float64, device=device, generator=gen)
        u = torch.empty_like(r)
        row = {"size": f"{nx}x{ny}x{nz}", "c": c}
        with chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, chanfs.NEUMANN, chanfs.F64) as p64:
            for th, name in ((0, "f64_algorithm2_ms"), (1, "f64_thomas_ms")):
                p64.set_option(chanfs.OPT_HELM_THOMAS, th)
                row[name] = round(timed(lambda: p64.helmholtz_solve(c, r, 0, out=u)), 4)
        with chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, chanfs.NEUMANN, chanfs.F32_REFINED) as p32:
            one = {}
            for parts in (8, 16, 32):
                try:
                    p32.set_option(chanfs.OPT_PCR_PARTS, parts)
                except chanfs.ChanfsError:
                    continue
                if (nz + parts - 1) // parts > 32:
                    continue  # more rows per partition than the one-pass kernel holds
                with nvtx_range(f"refined_helmholtz_{nx}x{ny}x{nz}_p{parts}"):
                    t = timed(lambda: p32.helmholtz_solve(c, r, 0, out=u))
                it, rho = p32.last_info()
                one[str(parts)] = {"ms": round(t, 4), "fp32_solves": it, "rel_residual": rho}
            row["refined_one_pass"] = one
            p32.set_option(chanfs.OPT_PCR_PARTS, 0)
            p32.set_option(chanfs.OPT_HELM_THOMAS32, 1)
            row["refined_thomas_loop_ms"] = round(timed(lambda: p32.helmholtz_solve(c, r, 0, out=u)), 4)
        out.append(row)
    return {"what": "median CUDA-event ms per Helmholtz solve, rhs N(0,1), Dirichlet centred",
            "sizes": out}


def run_cufft_comparison(torch, f, stage_ms, reps: int = 5):
    """cuFFT (through torch.fft) D2Z / Z2D over (y, x) of the FP64 channel
    field, timed for comparison only (the library does not use it), beside
    the x + y stages of the solve (packed real FFT along x, complex FFT along
    y of the half spectrum)."""
    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)
    nz, ny, nx = f.shape
    spec = torch.fft.rfft2(f)
    t_fwd = timed(lambda: torch.fft.rfft2(f))
    t_inv = timed(lambda: torch.fft.irfft2(spec, s=(ny, nx)))
    del spec
    ours_fwd = stage_ms["x_forward"] + stage_ms["y_forward"]
    ours_inv = stage_ms["y_inverse"] + stage_ms["x_inverse"]
    return {"what": "torch.fft.rfft2 / irfft2 (cuFFT D2Z / Z2D) over (y, x) of the FP64 "
                    f"{nx}x{ny}x{nz} field, comparison only",
            "cufft_forward_ms": round(t_fwd, 4), "cufft_inverse_ms": round(t_inv, 4),
            "ours_forward_ms": round(ours_fwd, 4), "ours_inverse_ms": round(ours_inv, 4),
            "ours_vs_cufft": round((t_fwd + t_inv) / (ours_fwd + ours_inv), 3)}


def run_stress(chanfs, torch, device, reps: int = 3):
    """The paper's per-GPU weak-scaling box shape, 3456 x 3072 x 30 (318.5 M
    points, a thin wall-normal direction), on one GPU: FP64 Poisson solve and
    the three Helmholtz solves of the channel step (tanh 1.8 grid, the
    channel's alpha nu dt), shapes from the tuner; Helmholtz by Algorithm 2
    and by the tuner's choice."""
    cfg = dict(synth.STRESS)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    npts = nx * ny * nz
    dz = synth.grid_dz(cfg)
    c = synth.CHANNEL_C
    gen = torch.Generator(device=device)
    gen.manual_seed(cfg["seed"])
    f = torch.randn(nz, ny, nx, dtype=torch.float64, device=device, generator=gen)
    w = torch.from_numpy(dz).to(device)
    f -= (f.sum(dim=(1, 2)) * w).sum() / (w.sum() * nx * ny)  # zero dz-weighted mean
    r = torch.randn(nz, ny, nx, dtype=torch.float64, device=device, generator=gen)
    out = torch.empty_like(f)
    locs = (chanfs.CENTER, chanfs.CENTER, chanfs.FACE)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    with chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, chanfs.NEUMANN) as plan:
        tuned = plan.autotune()
        thomas = plan.get_option(chanfs.OPT_HELM_THOMAS)
        t_p = timed(lambda: plan.poisson_solve(f, out=out))
        plan.set_option(chanfs.OPT_HELM_THOMAS, 0)
        t_pcr = timed(lambda: [plan.helmholtz_solve(c, r, loc, out=out) for loc in locs])
        plan.set_option(chanfs.OPT_HELM_THOMAS, 1)
        t_th = timed(lambda: [plan.helmholtz_solve(c, r, loc, out=out) for loc in locs])
        status = plan.check()
    del f, r, out
    return {"workload": cfg["name"], "points": npts, "precision": "f64",
            "poisson_ms": round(t_p, 4), "poisson_ns_per_pt": t_p * 1e6 / npts,
            "helmholtz3_algorithm2_ms": round(t_pcr, 4),
            "helmholtz3_thomas_ms": round(t_th, 4),
            "step_ms_algorithm2": round(t_p + t_pcr, 4),
            "step_ns_per_pt_algorithm2": (t_p + t_pcr) * 1e6 / npts,
            "tuner_helmholtz": "thomas" if thomas else "algorithm2",
            "kernel_shapes": tuned, "device_status": status,
            "timing": f"median of {reps} CUDA-event timings; fields 2.5 GB (larger than L2)"}


# ----------------------------------------------------------------------------
# Serving stream: Poisson arrivals of Poisson/Helmholtz requests from 32 runs
# ----------------------------------------------------------------------------

def run_serving(chanfs, torch, device, nreq: int = 0, workers: int = 4, max_batch: int = 32,
                slots: int = 2, rates=(2000.0, 3500.0)):
    """The serving stream through cfs_server_*: the seeded arrivals at each
    offered rate in `rates` (the stream's own 2000/s, then its arrival times
    scaled to a rate near capacity), p50/p99 latency, solves/s and batching;
    then capacity (requests submitted at once) against per-request FP64."""
    cfg = dict(synth.SERVING)
    if nreq:
        cfg["nreq"] = nreq
    runs, reqs = synth.serving_stream(cfg)
    gen = torch.Generator(device=device)
    gen.manual_seed(cfg["seed"])
    srv = chanfs.Server(int(cfg["budget_gb"] * 2**30), workers, max_batch, autotune=True,
                        slots_per_run=slots)
    # per run: one right-hand side and `slots` outputs (requests of one run
    # in flight at the same time write different outputs)
    fields = []
    for nx, ny, nz, beta, _ in runs:
        srv.add_run(nx, ny, nz, cfg["lx"], cfg["ly"], synth.tanh_dz(nz, beta), chanfs.NEUMANN)
        x = torch.randn(nz, ny, nx, dtype=torch.float64, device=device, generator=gen)
        fields.append((x, [torch.empty_like(x) for _ in range(slots)]))
    torch.cuda.synchronize()
    nth = [0] * len(runs)

    def submit(r, kind, ci, loc):
        out = fields[r][1][nth[r] % slots]
        nth[r] += 1
        return srv.submit(r, kind, fields[r][0], out, runs[r][4][ci], loc)

    # warm the plans (creation, tuning, the Helmholtz sets of each run), every slot
    t0 = time.perf_counter()
    for _ in range(slots):
        warm = []
        for r, (nx, ny, nz, beta, cs) in enumerate(runs):
            warm.append(submit(r, chanfs.REQ_POISSON, 0, 0))
            for ci in range(len(cs)):
                for loc in (chanfs.CENTER, chanfs.FACE):
                    warm.append(submit(r, chanfs.REQ_HELMHOLTZ, ci, loc))
        for t in warm:
            srv.wait(t)
    warm_s = time.perf_counter() - t0
    pts = np.array([runs[r][0] * runs[r][1] * runs[r][2] for _, r, _, _, _ in reqs], dtype=np.float64)

    def stream(rate):
        scale = cfg["rate"] / rate
        before = srv.stats()
        tickets = []
        start = time.perf_counter()
        for arrival, r, kind, ci, loc in reqs:
            due = start + arrival * scale
            while True:
                lag = due - time.perf_counter()
                if lag <= 0:
                    break
                if lag > 2e-4:
                    time.sleep(lag - 1e-4)
            tickets.append(submit(r, kind, ci, loc))
        lat, failed, statuses = [], 0, {}
        for t in tickets:
            status, l = srv.wait(t)
            lat.append(l)
            failed += status != 0
            if status:
                key = chanfs.status_string(status)
                statuses[key] = statuses.get(key, 0) + 1
        span = time.perf_counter() - start
        after = srv.stats()
        lat = np.array(lat)
        nb = after["batches"] - before["batches"]
        return {"offered_rate_per_s": rate, "arrival_span_s": reqs[-1][0] * scale,
                "solves_per_s": len(reqs) / span, "wall_s": span,
                "p50_latency_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_latency_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_latency_ms": float(lat.mean() * 1e3), "failed": int(failed),
                "failures": statuses, "grid_points_per_s": float(pts.sum() / span),
                "mean_batch": (after["completed"] - before["completed"]) / max(nb, 1)}

    streams = [stream(rate) for rate in rates]
    # capacity: the first `ncap` requests of the stream submitted at once
    ncap = min(4000, len(reqs))
    t0 = time.perf_counter()
    cap_tickets = [submit(r, kind, ci, loc) for _, r, kind, ci, loc in reqs[:ncap]]
    for t in cap_tickets:
        srv.wait(t)
    cap_s = time.perf_counter() - t0
    after = srv.stats()
    srv.close()
    # the same requests as plain per-request FP64 solves, one after another
    plans64 = []
    for nx, ny, nz, beta, _ in runs:
        pl = chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], synth.tanh_dz(nz, beta), chanfs.NEUMANN)
        pl.autotune()
        plans64.append(pl)

    def fp64(sub):
        for _, r, kind, ci, loc in sub:
            if kind == 0:
                plans64[r].poisson_solve(fields[r][0], out=fields[r][1][0])
            else:
                plans64[r].helmholtz_solve(runs[r][4][ci], fields[r][0], loc, out=fields[r][1][0])

    fp64(reqs[:200])  # Helmholtz sets and warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fp64(reqs[:ncap])
    torch.cuda.synchronize()
    f64_s = time.perf_counter() - t0
    for pl in plans64:
        pl.close()
    out = {"workload": cfg["name"], "requests": len(reqs), "runs": len(runs),
           "poisson_requests": sum(1 for q in reqs if q[2] == 0)}
    out.update(streams[0])
    out["streams"] = streams
    out.update({"max_batch": after["max_batch_seen"], "plans_created": after["plans_created"],
                "plans_evicted": after["plans_evicted"], "plan_bytes": after["bytes_in_use"],
                "workers": workers, "slots_per_run": slots, "budget_gb": cfg["budget_gb"],
                "warm_s": round(warm_s, 1),
                "capacity_solves_per_s": ncap / cap_s,
                "per_request_f64_solves_per_s": ncap / f64_s,
                "capacity_vs_per_request_f64": f64_s / cap_s,
                "capacity_sample": f"first {ncap} requests of the stream submitted at once, against "
                                   "the same requests solved one after another by FP64 plans",
                "precision": "Poisson: FP32 solves + FP64 refinement to 1e-10 (at most 4 FP32 "
                             "solves); Helmholtz: per size the faster of that and FP64 Algorithm 2 "
                             "(autotuner), both within 1e-10",
                "latency": "host clock from submission (at the scheduled arrival) to completion; "
                           "plans warmed before the streams; the second stream is the same "
                           "arrivals with their times scaled to the higher rate"})
    return out


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_mixed_only(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs
    mixed = run_mixed(chanfs, torch, torch.device("cuda", 0), reps=args.steps, warmup=args.warmup,
                      nz=args.mixed_nz)
    print(json.dumps({"mixed": mixed}), flush=True)
    return 0


def run_zsolve_only(args):
    """The refined Poisson solve of the 1024 x 768 x nz uniform workload with
    each z-solve kernel of FP32 spectra: the partitioned solve
    (CFS_OPT_THOMAS_TILE 1) and the streaming sweep (-1); median CUDA-event
    ms per solve over --steps solves after one warm-up solve each."""
    import torch
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs
    cfg = dict(synth.PRECISION)
    if args.mixed_nz:
        cfg.update(nz=args.mixed_nz)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    f = torch.from_numpy(synth.precision_rhs(cfg)).to(device)
    p = torch.empty_like(f)
    out = {"workload": f"poisson_uniform_{nx}x{ny}x{nz}"}
    with chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], synth.grid_dz(cfg), chanfs.NEUMANN,
                     chanfs.F32_REFINED) as plan:
        for tw, name in ((1, "partitioned"), (-1, "streaming")):
            plan.set_option(chanfs.OPT_THOMAS_TILE, tw)
            plan.poisson_solve(f, out=p)
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                with nvtx_range(f"refined_solve_{name}"):
                    plan.poisson_solve(f, out=p)
                b.record()
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            it, rho = plan.last_info()
            out[name] = {"ms": round(statistics.median(ms), 4), "fp32_solves": it,
                         "rel_residual": rho}
    print(json.dumps({"zsolve": out}), flush=True)
    return 0


def run_helmholtz_only(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs
    sizes = HELM_SIZES
    if args.helm_size:
        nx, ny, nz = (int(v) for v in args.helm_size.split("x"))
        sizes = [(nx, ny, nz, 1.8, 1e-5)]
    out = run_refined_helmholtz(chanfs, torch, torch.device("cuda", 0), reps=args.steps,
                                sizes=sizes)
    print(json.dumps({"refined_helmholtz": out}), flush=True)
    return 0


def run_probe_only(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs
    print(json.dumps({"fma_probe": run_fma_probe(chanfs, 0, reps=args.steps)}), flush=True)
    return 0


def run_f64_adds_sweep(args):
    """The FP64 transforms of the channel Poisson solve with each level of
    integer-unit butterfly additions (CFS_OPT_F64_ADDS_X / _Y): median
    CUDA-event ms per stage over --steps solves (stage by stage, both options
    at the level), the bits of each solve against level 0's, and the pair
    rates of the FP64 pipe and of the integer-unit additions."""
    import torch
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs
    cfg = dict(CFG)
    if args.nz:
        cfg.update(nz=args.nz)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    f_h, _ = synth.channel_fields(cfg)
    f = torch.from_numpy(f_h).to(device)
    p = torch.empty_like(f)
    stream = torch.cuda.current_stream(device)
    out = {"workload": f"channel_{nx}x{ny}x{nz}_tanh1.8", "levels": {}}
    order = (chanfs.X_FORWARD, chanfs.Y_FORWARD, chanfs.Z_SOLVE, chanfs.Y_INVERSE,
             chanfs.X_INVERSE)
    names = ("x_forward", "y_forward", "z_thomas", "y_inverse", "x_inverse")
    with chanfs.Plan(nx, ny, nz, CFG["lx"], CFG["ly"], synth.grid_dz(cfg), chanfs.NEUMANN) as plan:
        ref = None
        for level in range(5):
            plan.set_option(chanfs.OPT_F64_ADDS_X, level)
            plan.set_option(chanfs.OPT_F64_ADDS_Y, level)
            times = {n: [] for n in names}
            for rep in range(args.warmup + args.steps):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
                ev[0].record(stream)
                src = f
                for i, st in enumerate(order):
                    plan.poisson_stage(st, src, out=p)
                    src = p
                    ev[i + 1].record(stream)
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    for i, n in enumerate(names):
                        times[n].append(ev[i].elapsed_time(ev[i + 1]))
            if ref is None:
                ref = p.clone()
            out["levels"][str(level)] = {
                "stage_ms": {n: round(statistics.median(v), 4) for n, v in times.items()},
                "stage_ms_min": {n: round(min(v), 4) for n, v in times.items()},
                "bits_equal_level0": bool(torch.equal(p, ref))}
        out["device_status"] = plan.check()
    for emu in (False, True):
        r = [chanfs.probe_addsub(emu, 1 << 14) for _ in range(3)]
        out["pairs_per_s_" + ("integer" if emu else "fp64_pipe")] = statistics.median(
            v for v, _ in r)
    out["selfcheck_mismatches"] = chanfs.selfcheck_f64_addsub(1 << 24)
    print(json.dumps({"f64_adds_sweep": out}), flush=True)
    return 0


def run_extras_only(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs
    dev = torch.device("cuda", 0)
    out = {}
    if not args.no_stress:
        out["stress"] = run_stress(chanfs, torch, dev)
    if not args.no_ensemble:
        out["ensemble"] = run_ensemble(chanfs, torch, dev)
    if not args.no_serving:
        out["serving"] = run_serving(chanfs, torch, dev, args.serve_requests)
    print(json.dumps(out), flush=True)
    return 0


def run_slab(args):
    """The paper's weak-scaling layout (Sec. 3: p_y = 1, p_z = number of GPUs):
    one z-slab of 384 planes of a 512 x 384 x (384 N) tanh(1.8) channel per
    GPU, the step (Poisson + three Helmholtz solves) by P-TDMA with one NCCL
    all-gather of the boundary values per solve.  Each rank's fields are its
    own seeded N(0,1) draws."""
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs, slab

    nx, ny, nzl = CFG["nx"], CFG["ny"], CFG["nz"]
    nz = nzl * world
    dz = synth.tanh_dz(nz, CFG["beta"])
    c = synth.CHANNEL_C
    solver = slab.SlabSolver(nx, ny, nz, CFG["lx"], CFG["ly"], dz, chanfs.NEUMANN)
    gen = torch.Generator(device=device)
    gen.manual_seed(CFG["seed"] + 1000 * rank)
    shape = solver.shape
    f = torch.randn(*shape, dtype=torch.float64, device=device, generator=gen)
    rhs = [torch.randn(*shape, dtype=torch.float64, device=device, generator=gen) for _ in range(3)]
    p = torch.empty_like(f)
    us = [torch.empty_like(f) for _ in range(3)]
    w = torch.empty_like(f)
    locs = (chanfs.CENTER, chanfs.CENTER, chanfs.FACE)

    def step():
        solver.poisson_solve(f, out=p, work=p)
        for i in range(3):
            solver.helmholtz_solve(c, rhs[i], locs[i], out=us[i], work=w)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(device)
    with ClockSampler(local) as clk:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            step()
        b.record()
        torch.cuda.synchronize()
    barrier(device)
    max_ms = reduce_max(a.elapsed_time(b), device)
    npts = nx * ny * shape[0]
    agg = aggregate(max_ms, args.steps, nx * ny * nzl, world)
    solver.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": agg["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": agg["ms_per_step"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"channel_zslab_{nx}x{ny}x{nz}_tanh1.8", "nx": nx, "ny": ny,
                   "nz": nz, "planes_per_gpu": nzl, "parallelism": f"zslab{world}",
                   "method": "P-TDMA: local x/y transforms, Algorithm 2 Step 2 per slab, NCCL "
                             "all-gather of 2 values per column per rank, reduced solve and "
                             "reconstruction per slab",
                   "l2": f"inputs larger than L2 ({npts * 8 / 1e6:.0f} MB fields per GPU)"},
        "e2e": None, "gpu_launches": None, "roofline": None, "cpu_baseline": None,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)

    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs

    cfg = dict(CFG)
    if args.nz:  # reduced wall-normal size for profiling captures
        cfg.update(nz=args.nz, name=f"channel_{CFG['nx']}x{CFG['ny']}x{args.nz}_tanh1.8")
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    npts = nx * ny * nz
    dz = synth.grid_dz(cfg)
    c = synth.CHANNEL_C
    f_h, rhs_h = synth.channel_fields(cfg)
    plan = chanfs.Plan(nx, ny, nz, CFG["lx"], CFG["ly"], dz, chanfs.NEUMANN)
    tuned = plan.autotune() if not args.nparts else None  # kernel shapes by measurement
    # the workload's Helmholtz solves are Algorithm 2 (pre-processed PCR),
    # whatever the tuner found for the Thomas alternative
    helm_thomas_tuned = plan.get_option(chanfs.OPT_HELM_THOMAS)
    plan.set_option(chanfs.OPT_HELM_THOMAS, 0)
    set_helm_method(False)
    for loc in (chanfs.CENTER, chanfs.FACE):
        plan.helmholtz_prepare(c, loc, args.nparts)
    f = torch.from_numpy(f_h).to(device)
    rhs = [torch.from_numpy(r).to(device) for r in rhs_h]
    p = torch.empty_like(f)
    us = [torch.empty_like(f) for _ in range(3)]
    locs = (chanfs.CENTER, chanfs.CENTER, chanfs.FACE)
    stream = torch.cuda.current_stream(device)

    # the stage sequence is cfs_poisson_solve's: check it gives the same bits
    plan.poisson_solve(f, out=p)
    ref_bits = p.clone()

    def step(events=None):
        def mark(i):
            if events is not None:
                events[i].record(stream)
        mark(0)
        plan.poisson_stage(chanfs.X_FORWARD, f, out=p)
        mark(1)
        plan.poisson_stage(chanfs.Y_FORWARD, p, out=p)
        mark(2)
        plan.poisson_stage(chanfs.Z_SOLVE, p, out=p)
        mark(3)
        plan.poisson_stage(chanfs.Y_INVERSE, p, out=p)
        mark(4)
        plan.poisson_stage(chanfs.X_INVERSE, p, out=p)
        mark(5)
        for i in range(3):
            plan.helmholtz_solve(c, rhs[i], locs[i], out=us[i])
            mark(6 + i)

    step()
    torch.cuda.synchronize()
    assert torch.equal(p, ref_bits), "stage-by-stage step differs from cfs_poisson_solve"

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(9)] for _ in range(args.steps)]
    barrier(device)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk, nvtx_range("timed_steps"):
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for k in range(args.steps):
            step(events[k])
        stop.record(stream)
        torch.cuda.synchronize()
    barrier(device)
    elapsed_ms = start.elapsed_time(stop)
    status = plan.check()
    stage_ms = {s: [] for s in STAGES}
    for ev in events:
        for i, s in enumerate(STAGES):
            stage_ms[s].append(ev[i].elapsed_time(ev[i + 1]))
    max_ms = reduce_max(elapsed_ms, device)
    agg = aggregate(max_ms, args.steps, npts, world)

    # end to end through the host-buffer entry points: pinned host -> device,
    # solve, device -> host, every step
    f_pin = torch.from_numpy(f_h).pin_memory()
    rhs_pin = [torch.from_numpy(r).pin_memory() for r in rhs_h]
    out_pin = [torch.empty_like(f_pin).pin_memory() for _ in range(4)]

    jobs = [(chanfs.REQ_POISSON, 0.0, 0, f_pin, out_pin[0])]
    jobs += [(chanfs.REQ_HELMHOLTZ, c, locs[i], rhs_pin[i], out_pin[1 + i]) for i in range(3)]

    def e2e_step(chunks):  # one call: the four solves, copies overlapped with the solves
        plan.set_option(chanfs.OPT_STREAM_CHUNKS, chunks)
        t = time.perf_counter()
        plan.solve_batch_host(jobs)  # returns once every result is in host memory
        return (time.perf_counter() - t) * 1e3

    # the library's default (fields streamed in chunks) and, interleaved with
    # it call by call, the same calls moving and solving whole fields; the
    # host link's speed drifts and stalls now and then, so each figure is the
    # median over its calls
    e2e_step(0)
    e2e_step(1)
    e2e_steps = max(3, min(args.steps, 10))
    times = {0: [], 1: []}
    barrier(device)
    for k in range(e2e_steps):
        for chunks in ((0, 1) if k % 2 == 0 else (1, 0)):
            times[chunks].append(e2e_step(chunks))
    torch.cuda.synchronize()
    plan.set_option(chanfs.OPT_STREAM_CHUNKS, 0)
    stream_chunks = plan.get_option(chanfs.OPT_STREAM_CHUNKS)  # the automatic count
    e2e_ms = reduce_max(statistics.median(times[0]), device)
    whole_ms = reduce_max(statistics.median(times[1]), device)
    barrier(device)
    e2e = aggregate(e2e_ms, 1, npts, world)
    e2e_whole = aggregate(whole_ms, 1, npts, world)
    e2e_mean = {c: statistics.mean(v) for c, v in times.items()}
    field_bytes = npts * 8

    if rank != 0:
        plan.close()
        return 0

    # roofline of the kernel with the largest time per step
    mean_ms = {s: float(np.mean(v)) for s, v in stage_ms.items()}
    per_kernel = {}
    for s in STAGES:
        k = KERNEL_OF_STAGE[s]
        per_kernel.setdefault(k, 0.0)
        per_kernel[k] += mean_ms[s]
    dom_stage = max(STAGES, key=lambda s: mean_ms[s])
    flops, nbytes = stage_work(dom_stage, nx, ny, nz)
    dur_s = mean_ms[dom_stage] * 1e-3
    peaks = read_peaks()
    clock = clk.summary()
    peak_tf = fp64_peak_tflops()
    roof = {"bound": "alu", "achieved": flops / dur_s / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": flops / dur_s / 1e12 / peak_tf, "traffic": profiled_traffic(dom_stage),
            "kernel": KERNEL_OF_STAGE[dom_stage], "stage": dom_stage,
            "launch_ms": mean_ms[dom_stage], "flops_per_launch": flops,
            "algorithmic_bytes_per_launch": nbytes,
            "hbm_gbs": nbytes / dur_s / 1e9,
            "hbm_frac": nbytes / dur_s / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
            "peak_source": "FP64: 152 SMs x 2 DFMA/clk x 2 flops x 2070 MHz (1.26 TFLOP/s), the "
                           "2 DFMA/clk/SM measured by cfs_probe_fma (line's fma_probe; "
                           "profiles/fp64_fma_probe.md); HBM: MEASURED_PEAKS.json hbm_gbs"}
    line = {
        "metric": METRIC, "value": agg["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": agg["ms_per_step"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "nx": nx, "ny": ny, "nz": nz, "lx": CFG["lx"],
                   "ly": CFG["ly"], "z_grid": "tanh(1.8) faces", "poisson_bc": "neumann",
                   "helmholtz_c": c, "helmholtz": "u,v centred + w face, Dirichlet, Algorithm 2",
                   "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 ({npts * 8 / 1e6:.0f} MB fields, L2 129 MB)",
                   "pcr_partitions": args.nparts or plan.get_option(chanfs.OPT_PCR_PARTS),
                   "kernel_shapes": tuned or "fixed by --nparts",
                   "helmholtz_tuner_choice": "thomas" if helm_thomas_tuned else "algorithm2"},
        "e2e": {"value": e2e["value"], "unit": UNIT, "h2d_bytes_per_step": 4 * field_bytes,
                "d2h_bytes_per_step": 4 * field_bytes, "steps": e2e_steps,
                "api": "cfs_solve_batch_host (Poisson + 3 Helmholtz, host<->device copies "
                       "overlapped with the solves), pinned host buffers",
                "stream_chunks": stream_chunks,
                "ms_per_step": e2e["ms_per_step"], "mean_ms_per_step": e2e_mean[0],
                "timing": "host clock around each call (it returns once every result is in "
                          "host memory); median over the calls, interleaved call by call "
                          "with the whole-field calls",
                "whole_fields": {"value": e2e_whole["value"],
                                 "ms_per_step": e2e_whole["ms_per_step"],
                                 "mean_ms_per_step": e2e_mean[1],
                                 "how": "the same calls with CFS_OPT_STREAM_CHUNKS 1 (each "
                                        "field copied and solved whole)"}},
        "gpu_launches": 8 * args.steps,
        "roofline": roof,
        "stage_ms": {s: round(v, 4) for s, v in mean_ms.items()},
        "stage_ms_min": {s: round(float(np.min(v)), 4) for s, v in stage_ms.items()},
        "kernel_ms_per_step": {k: round(v, 4) for k, v in per_kernel.items()},
        "clocks": clock,
        "device_status": status,
    }
    line["fma_probe"] = run_fma_probe(chanfs, local)
    line["helmholtz3d"] = run_helmholtz3d(chanfs, torch, device, plan, rhs, us)
    line["ywalls"] = run_ywalls(chanfs, torch, device, f, dz)
    line["cufft_comparison"] = run_cufft_comparison(torch, f, mean_ms)
    plan.close()
    del f, rhs, p, us, ref_bits
    if not args.no_stress:
        line["stress"] = run_stress(chanfs, torch, device)
    if not args.no_mixed:
        line["refined_helmholtz"] = run_refined_helmholtz(chanfs, torch, device)
        line["mixed"] = run_mixed(chanfs, torch, device)
    if not args.no_ensemble:
        line["ensemble"] = run_ensemble(chanfs, torch, device)
    if not args.no_serving:
        line["serving"] = run_serving(chanfs, torch, device, args.serve_requests)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    else:
        line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nparts", type=int, default=0, help="PCR partitions (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the FP32-refined vs FP64 comparisons (Helmholtz per size and "
                         "the 1024x768x512 workload)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 48-box ensemble")
    ap.add_argument("--no-stress", action="store_true",
                    help="skip the 3456x3072x30 single-GPU box")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream")
    ap.add_argument("--serve-requests", type=int, default=0,
                    help="requests of the serving stream (0: the full 20,000)")
    ap.add_argument("--extras-only", action="store_true",
                    help="run only the stress box, ensemble and serving measurements")
    ap.add_argument("--mixed-nz", type=int, default=0,
                    help="wall-normal size of the mixed comparison (profiling captures only)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="run only the FP32-refined vs FP64 comparison and print its object")
    ap.add_argument("--zsolve-only", action="store_true",
                    help="time the refined Poisson solve with each FP32 z-solve kernel "
                         "(1024 x 768 x --mixed-nz, default 512)")
    ap.add_argument("--helmholtz-only", action="store_true",
                    help="time only the FP64 and refined Helmholtz solves per size")
    ap.add_argument("--helm-size", default="",
                    help="with --helmholtz-only: one size NXxNYxNZ (stretching 1.8, c = 1e-5)")
    ap.add_argument("--probe-only", action="store_true",
                    help="measure only the FP64 and FP32 FMA rates (--steps repetitions)")
    ap.add_argument("--f64-adds-sweep", action="store_true",
                    help="time the FP64 transforms at each level of integer-unit butterfly "
                         "additions (CFS_OPT_F64_ADDS_X / _Y) and check their bits")
    ap.add_argument("--slab", action="store_true",
                    help="N > 1: one z-slab of the channel per GPU, solved by P-TDMA with an "
                         "NCCL all-gather (the default runs independent replicas)")
    ap.add_argument("--nz", type=int, default=0,
                    help="override the wall-normal size (profiling captures only)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.mixed_only:
        return run_mixed_only(args)
    if args.probe_only:
        return run_probe_only(args)
    if args.f64_adds_sweep:
        return run_f64_adds_sweep(args)
    if args.helmholtz_only:
        return run_helmholtz_only(args)
    if args.zsolve_only:
        return run_zsolve_only(args)
    if args.slab:
        return run_slab(args)
    if args.extras_only:
        return run_extras_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
