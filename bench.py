#!/usr/bin/env python
"""Benchmark of the GBEM hot path on GB300.

One step = one full capacitance extraction of the 2x2 crossing bus
(N = 6264 edge-graded panels, 4 conductors, eps_r 3.9): Galerkin assembly
(Sec. 3.4, Eq. "matrix"), Cholesky factorisation (Sec. 3.2), solve with one
right-hand side per conductor plus FP64 refinement (Eq. "lineareq1") and the
charge reduction to the Maxwell matrix (Eq. "electriccharge").

metric: panel-pair integrals/s = N(N+1)/2 unique pair integrals of the
extraction per second of the whole extraction (the paper's Table 2 setting:
all entries, then the solve, timed together).  ``value`` runs with the panel
geometry already resident on the device; ``e2e`` meshes on the host and
uploads every step, and reads the capacitance matrix back.

Multi-GPU: independent extractions per rank (replicas, weak scaling), no
collective on the data path.  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "crossing_bus_2x2"
METRIC = "panel-pair integrals/s"
UNIT = "pairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 30; 10 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-pairs", type=int, default=200000)
    ap.add_argument("--workload", default="crossing_bus_2x2", choices=["crossing_bus_2x2", "batch512", "serving"],
                    help="crossing_bus_2x2: the headline line; batch512 / serving: the batched and served forms")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--serve-count", type=int, default=120)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    ap.add_argument("--profile", default=None, choices=["mixed", "fp64"],
                    help="one warm-up and one extraction in that precision, nothing else "
                         "(for ncu captures)")
    ap.add_argument("--profile-workload", default="crossing_bus_2x2",
                    choices=["crossing_bus_2x2", "two_bars", "bus_3layer_5x5x5"],
                    help="structure of the --profile run (two_bars: a small case for pass counts)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else 30
    return args


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_start(world: int, backend: str = "nccl"):
    """One process per GPU under torchrun: join the process group (the ranks
    exchange only timings, never data of the extraction)."""
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def dist_stop(world: int):
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of every rank's x (a time): the whole job ends with its
    slowest rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed (each rank the same number) per second of
    the slowest rank."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons every 50 ms, each
    row time-stamped, so that the rows taken inside the timed region
    (begin() .. end()) are the ones reported.  The GPU is addressed by its PCI
    bus id (nvidia-smi's index order need not match CUDA's), else by index."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def _target(self):
        try:
            import torch
            p = torch.cuda.get_device_properties(self.index)
            bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
            r = subprocess.run(["nvidia-smi", f"--id={bus}", "--query-gpu=index", "--format=csv,noheader"],
                               capture_output=True, timeout=20)
            if r.returncode == 0 and r.stdout.strip():
                return bus
        except Exception:
            pass
        return str(self.index)

    def start(self):
        """Start sampling; give nvidia-smi time to take its first sample."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self._target()}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except (OSError, FileNotFoundError):
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, parts[1:]))
        os.unlink(self.path)
        inside = [r for ts, r in rows if ts is not None and self.t0 is not None and self.t1 is not None
                  and self.t0 <= ts <= self.t1]
        # a region shorter than the interval may hold no sample: then the
        # samples of the 0.5 s around it (the warm-up runs just before)
        window = "timed region"
        if not inside:
            inside = [r for ts, r in rows if ts is not None and self.t0 is not None and self.t1 is not None
                      and self.t0 - 0.5 <= ts <= self.t1 + 0.5]
            window = "timed region +- 0.5 s"
        if not inside:
            inside = [r for _, r in rows]
            window = "whole sampler run"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = sorted(v for v in (num(r[1]) for r in inside) if v is not None)
        mx = max((v for v in (num(r[2]) for r in inside) if v is not None), default=None)
        reasons = sorted({self.NAMES[k] for r in inside for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(inside), "window": window}


# ---------------------------------------------------------------- CPU baseline (oracle)

def cpu_baseline(n_sample: int):
    """Time the FP64 oracle on a bounded sample: its assembly rate on random
    entries of the workload's matrix, plus a full-size Cholesky factorisation
    and solve (scipy LAPACK, as the oracle solves), scaled to one extraction."""
    import numpy as np
    import scipy.linalg as sla
    from oracle import oracle as O
    from paper_2203_11733_gb300 import workloads as W
    boxes, params = getattr(W, WORKLOAD)()
    a, g, c = O.mesh_boxes(boxes, **params)
    n = len(a)
    rng = np.random.default_rng(1)
    I = rng.integers(0, n, n_sample)
    J = rng.integers(0, n, n_sample)
    t0 = time.perf_counter()
    O.entries(a, g, I, J)
    t_entries = time.perf_counter() - t0
    rate = n_sample / t_entries
    # factor + solve at full size on an SPD matrix of the same order
    M = rng.standard_normal((n, 64))
    A = M @ M.T / 64 + np.eye(n)
    B, _ = O.rhs(c)
    t0 = time.perf_counter()
    cf = sla.cho_factor(A, lower=True)
    sla.cho_solve(cf, B)
    t_solve = time.perf_counter() - t0
    pairs = n * (n + 1) / 2
    t_extract = pairs / rate + t_solve
    return {
        "value": pairs / t_extract, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
        "sample": (f"{n_sample} random entries of the {n}-panel matrix in {t_entries:.1f} s "
                   f"({rate:.0f} entries/s) plus a full {n}x{n} Cholesky and {B.shape[1]}-RHS "
                   f"solve ({t_solve:.2f} s); one extraction estimated at {t_extract:.0f} s"),
        "extraction_s": t_extract,
    }


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    per_step = max(500, args.cpu_sample_pairs // 4)
    for _ in range(args.warmup):
        cpu_baseline(200)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(per_step)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n_panels": 6264, "n_cond": 4,
                                        "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm

def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_start(world)
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem, workloads as W
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    lib = gbem.load()
    boxes, params = getattr(W, args.profile_workload if args.profile else WORKLOAD)()
    eps_r = W.EPS_R_SIO2
    ctx = gbem.Context(local)
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    mesh = gbem.gbem_mesh(ctx, boxes, params)
    n, nc = mesh.n, mesh.n_cond
    pairs = n * (n + 1) / 2

    def step(prec):
        mat = gbem.gbem_assemble(mesh, prec, stream)
        C, _ = gbem.gbem_capacitance(mesh, mat, eps_r, stream, want_residual=False)
        mat.close()
        return C

    if args.profile:
        prec = gbem.GBEM_MIXED if args.profile == "mixed" else gbem.GBEM_FP64
        step(prec)
        torch.cuda.synchronize()
        C = step(prec)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile": args.profile, "n_panels": n, "C": C.tolist()}))
        mesh.close()
        ctx.close()
        return

    def timed(fn, k, flush_between=True):
        """k steps timed with CUDA events on the launching stream, L2 flushed
        (untimed) before each; returns total ms, max over ranks."""
        total = 0.0
        for _ in range(k):
            if flush_between:
                with torch.cuda.stream(stream):
                    flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return max_over_ranks(total, world), out

    # ---- mixed precision (the headline path)
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step(gbem.GBEM_MIXED)
    barrier()
    gbem.set_timing(ctx, 1)
    stats = gbem.get_stats(ctx, reset=True)
    clocks.begin()
    ms_total, C_mixed = timed(lambda: step(gbem.GBEM_MIXED), args.steps)
    clocks.end()
    clk = clocks.stop()
    barrier()
    stats = gbem.get_stats(ctx, reset=True)
    ms_step = ms_total / args.steps
    value = whole_job_rate(pairs * args.steps, world, ms_total * 1e-3)

    # ---- the same steps again with an event pair around every launch of the
    # traced kernels (kept out of the headline timing: the events cost time)
    gbem.set_timing(ctx, 2)
    gbem.get_kernel_stats(ctx, reset=True)
    ms_traced, _ = timed(lambda: step(gbem.GBEM_MIXED), args.steps)
    kst = gbem.get_kernel_stats(ctx, reset=True)
    gbem.set_timing(ctx, 0)
    gbem.get_stats(ctx, reset=True)

    # the final relative residual of the refinement (one extra, untimed extraction)
    mat_r = gbem.gbem_assemble(mesh, gbem.GBEM_MIXED, stream)
    _, ir_residual = gbem.gbem_capacitance(mesh, mat_r, eps_r, stream, want_residual=True)
    mat_r.close()

    # ---- FP64 path on the same GPU
    step(gbem.GBEM_FP64)
    barrier()
    gbem.set_timing(ctx, 1)
    gbem.get_stats(ctx, reset=True)
    ms64, C_fp64 = timed(lambda: step(gbem.GBEM_FP64), args.fp64_steps)
    stats64 = gbem.get_stats(ctx, reset=True)
    gbem.set_timing(ctx, 0)
    ms64_step = ms64 / args.fp64_steps

    # ---- end to end: host boxes -> mesh + upload -> ... -> C on the host
    def step_e2e():
        return gbem.extract(ctx, boxes, params, eps_r, precision=gbem.GBEM_MIXED, stream=stream)[0]
    step_e2e()
    barrier()
    ms_e2e, _ = timed(step_e2e, args.steps)
    value_e2e = whole_job_rate(pairs * args.steps, world, ms_e2e * 1e-3)
    h2d = n * (5 * 8 + 1 + 4)
    d2h = nc * nc * 8

    # ---- accuracy against the stored oracle result
    gold_path = os.path.join(ROOT, "tests", "golden", f"{WORKLOAD}_capacitance.json")
    err_mixed = err_fp64 = None
    if os.path.exists(gold_path):
        C_ref = np.array(json.load(open(gold_path))["C"])
        scale = np.max(np.abs(C_ref))
        err_mixed = float(np.max(np.abs(C_mixed - C_ref)) / scale)
        err_fp64 = float(np.max(np.abs(C_fp64 - C_ref)) / scale)

    roof, kern = roofline(kst, args.steps, ms_traced / args.steps)
    # the same pairs over the assembly phase alone (its CUDA-event time)
    asm_ms = stats["ms"][PHASES.index("assemble")] / args.steps
    asm_rate = world * pairs / (asm_ms * 1e-3) if asm_ms > 0 else None
    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(args.cpu_sample_pairs)
            cpu.pop("extraction_s", None)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} (2x2 crossing bus, 0.1 um wires, edge-graded)",
                       "n_panels": n, "n_cond": nc, "eps_r": eps_r, "precision": "mixed",
                       "l2": "flushed (512 MB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "extractions_per_s": world * 1e3 / ms_step,
            "assembly_pairs_per_s": asm_rate,
            "phase_ms_per_step": {k: v / args.steps for k, v in zip(PHASES, stats["ms"])},
            "fp64": {"value": world * pairs / (ms64_step * 1e-3), "ms_per_step": ms64_step,
                     "extractions_per_s": world * 1e3 / ms64_step,
                     "phase_ms_per_step": {k: v / args.fp64_steps for k, v in zip(PHASES, stats64["ms"])},
                     "cap_rel_err_vs_oracle": err_fp64},
            "mixed_over_fp64": ms64_step / ms_step,
            "cap_rel_err_vs_oracle": err_mixed,
            "ir_residual": ir_residual,
            "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": ms_e2e / args.steps},
            "gpu_launches": int(stats["launches"]),
            "roofline": roof,
            "kernels": kern,
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    mesh.close()
    ctx.close()
    dist_stop(world)


PHASES = ["mesh_upload", "assemble", "factor", "solve", "reduce"]


KERNEL_NAMES = {
    "assemble": "assemble_tiles<mixed>: Galerkin entries, one CTA per 32x32 lower tile",
    "factor": "factor_step: one launch per elimination step (panel rows, strip update, next diagonal "
              "block factor+inverse, tcgen05 3xTF32 trailing tiles)",
    "sweep": "sweep_fwd_f32/sweep_bwd_f32: persistent cooperative triangular sweeps (x_b = z_b - M_b x_p)",
    "residual": "residual_df: R = B - A X, compensated FP32 over float-pair storage",
}
FP64_PEAK_TF = 1.25   # nominal GB300 FP64 (non-tensor) rate


def traffic_per_launch(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (dram__bytes_read.sum + dram__bytes_write.sum over one factorisation's
    launches, divided by their number), or None."""
    p = os.path.join(ROOT, "profiles", f"traffic_{WORKLOAD}_mixed.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = [x.strip() for x in line.strip().strip("|").split("|")]
        if len(parts) >= 3 and parts[0] == kernel:
            try:
                return float(parts[2])
            except ValueError:
                return None
    return None


def roofline(kst, steps, ms_traced_step):
    """Roofline of the kernel with the largest device time in the traced
    pass.  achieved = its algorithmic bytes (or flops) per launch, as the
    library reports them for every launch, over its average CUDA-event
    launch duration on the launching stream."""
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peaks = json.load(open(p))
    kern = {}
    for k, d in kst.items():
        if d["launches"] == 0:
            continue
        t = d["ms"] / d["launches"] * 1e-3
        kern[k] = {"ms_per_step": d["ms"] / steps, "launches_per_step": d["launches"] / steps,
                   "us_per_launch": t * 1e6,
                   "gb_per_s": d["bytes"] / d["launches"] / t / 1e9,
                   "tflop_per_s": d["flops"] / d["launches"] / t / 1e12}
    kern["traced_ms_per_step"] = ms_traced_step
    names = [k for k in kst if kst[k]["launches"] > 0]
    dom = max(names, key=lambda k: kst[k]["ms"])
    d = kst[dom]
    t = d["ms"] / d["launches"] * 1e-3
    out = {"kernel": KERNEL_NAMES[dom], "share_of_traced_step": d["ms"] / steps / ms_traced_step,
           "launches_per_step": d["launches"] / steps, "us_per_launch": t * 1e6}
    if dom == "residual":
        out.update({"bound": "alu", "achieved": d["flops"] / d["launches"] / t / 1e12, "peak": FP64_PEAK_TF,
                    "unit": "TFLOP/s", "peak_source": "nominal FP64 rate (no measured FP64 peak)",
                    "work_per_launch": d["flops"] / d["launches"], "traffic": None})
    else:
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
        out.update({"bound": "hbm", "achieved": d["bytes"] / d["launches"] / t / 1e9, "peak": hbm,
                    "unit": "GB/s", "peak_source": src, "work_per_launch": d["bytes"] / d["launches"],
                    "traffic": traffic_per_launch(dom)})
    out["frac"] = out["achieved"] / out["peak"]
    return out, kern


def run_batch(args):
    """512 independent 2-6 bar structures (N log-uniform in [200, 3000]):
    the autotuned batch (groups of structures whose graphs run concurrently,
    fewest refinement passes that meet the tolerance) against the untuned one
    and against one-at-a-time extractions (mixed and FP64) of the same
    structures on the same GPU."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_start(world)
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem, workloads as W
    B.build()
    # each rank its own structures: independent problems, no data exchanged
    structs = W.batch_small_structures(seed=4242 + rank, count=args.batch_count)
    ctx = gbem.Context(local)
    meshes = [ctx.mesh(b, p) for b, p in structs]
    ns = np.array([m.n for m in meshes])
    stream = torch.cuda.current_stream()

    def timed_runs(batch, k):
        total = 0.0
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = batch.run(W.EPS_R_SIO2, stream)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return total / k, out

    # the untuned batch (one group, three refinement passes) for comparison
    t0 = time.perf_counter()
    base = gbem.Batch(ctx, meshes, iters=3)
    t_create = time.perf_counter() - t0
    for _ in range(args.warmup):
        base.run(W.EPS_R_SIO2, stream)
    ms_base, _ = timed_runs(base, args.steps)
    base.close()
    # the autotuned batch (groups and refinement passes), cache in a temporary file
    cache = os.path.join(tempfile.mkdtemp(), "batch_tuning.txt")
    t0 = time.perf_counter()
    batch, choice = gbem.Batch.autotune(ctx, meshes, max_iters=3, cache_path=cache)
    t_tune = time.perf_counter() - t0
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        batch.run(W.EPS_R_SIO2, stream)
    gbem.get_stats(ctx, reset=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    ms_batch, (Cs, res) = timed_runs(batch, args.steps)
    clocks.end()
    clk = clocks.stop()
    ms_batch = max_over_ranks(ms_batch, world)
    st = gbem.get_stats(ctx, reset=True)
    # one at a time, same structures, same GPU
    def one_at_a_time(prec, idx):
        t = 0.0
        out = []
        for i in idx:
            m = meshes[i]
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mat = gbem.gbem_assemble(m, prec, stream)
            C, _ = gbem.gbem_capacitance(m, mat, W.EPS_R_SIO2, stream, want_residual=False)
            e1.record(stream)
            e1.synchronize()
            mat.close()
            t += e0.elapsed_time(e1)
            out.append(C)
        return t, out
    idx = list(range(len(meshes)))
    one_at_a_time(gbem.GBEM_MIXED, idx[:4])
    t_mixed, C_mixed = one_at_a_time(gbem.GBEM_MIXED, idx)
    sub = idx[::8]                      # FP64 one at a time on every 8th structure (time bound)
    t64, C64 = one_at_a_time(gbem.GBEM_FP64, sub)
    err_vs_fp64 = max(float(np.max(np.abs(Cs[i] - C)) / np.max(np.abs(C))) for i, C in zip(sub, C64))
    err_vs_single = max(float(np.max(np.abs(Cs[i] - C)) / np.max(np.abs(C))) for i, C in zip(idx, C_mixed))
    n_ext = len(meshes)
    line = {
        "metric": "extractions/s", "value": whole_job_rate(n_ext, world, ms_batch * 1e-3), "unit": "extractions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
        "data": "synthetic",
        "config": {"workload": f"batch{n_ext}: 2-6 parallel/crossing bars, N log-uniform [200,3000]",
                   "n_structures": n_ext, "n_panels_total": int(ns.sum()), "n_min": int(ns.min()),
                   "n_max": int(ns.max()), "refinement_passes": choice["iters"], "groups": choice["groups"],
                   "graph_kernels_per_launch": int(st["launches"] / args.steps)},
        "autotune": {"choice": choice, "tune_s": t_tune, "untuned_ms_per_step": ms_base,
                     "untuned_config": {"groups": 1, "refinement_passes": 3}},
        "pairs_per_s": whole_job_rate(float((ns * (ns + 1) / 2).sum()), world, ms_batch * 1e-3),
        "one_at_a_time_mixed": {"extractions_per_s": n_ext / (t_mixed * 1e-3), "ms_total": t_mixed},
        "one_at_a_time_fp64": {"extractions_per_s": len(sub) / (t64 * 1e-3), "structures": len(sub)},
        "batch_over_single_mixed": t_mixed / ms_batch,
        "batch_over_single_fp64": (t64 / len(sub) * n_ext) / ms_batch,
        "cap_rel_err_vs_fp64_gpu": err_vs_fp64, "cap_rel_err_vs_single_mixed": err_vs_single,
        "max_residual": float(np.max(res)), "batch_create_s": t_create, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    batch.close()
    ctx.close()
    dist_stop(world)


def run_serving(args):
    """Poisson stream of 2-15 conductor bus extractions (N log-uniform in
    [500, 30000]) through the continuous-batching server, at 0.8x the
    capacity measured on a burst; against one-at-a-time FP64 and mixed loops
    on the first requests."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_start(world)
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem, workloads as W
    B.build()
    budget = int(args.serve_budget_gb * (1 << 30))

    def run_stream(reqs, rate_scale=None):
        srv = gbem.Server(local, hbm_budget=budget, slots=args.serve_slots)
        got = {}
        t0 = time.perf_counter()
        for k, (t_arr, boxes, params) in enumerate(reqs):
            if rate_scale is not None:
                while time.perf_counter() - t0 < t_arr * rate_scale:
                    for info, C in srv.poll(wait_ms=1):
                        got[info["id"]] = (info, C)
            srv.submit(k, boxes, params, W.EPS_R_SIO2)
        while len(got) < len(reqs):
            for info, C in srv.poll(wait_ms=20):
                got[info["id"]] = (info, C)
        stats = srv.stats()
        srv.close()
        return got, stats

    # capacity: a burst of requests submitted at once
    cal = W.serving_requests(seed=2024 + rank, count=24, rate_per_s=1.0)
    got, _ = run_stream(cal)
    t_first = min(i["submit_s"] for i, _ in got.values())
    t_last = max(i["done_s"] for i, _ in got.values())
    capacity = len(cal) / (t_last - t_first)
    rate = 0.8 * capacity
    reqs = W.serving_requests(seed=777 + rank, count=args.serve_count, rate_per_s=1.0)
    # the generator's arrival times are for rate 1/s: scale them to `rate`
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    clocks.begin()
    got, stats = run_stream(reqs, rate_scale=1.0 / rate)
    clocks.end()
    clk = clocks.stop()
    infos = [got[k][0] for k in range(len(reqs))]
    lat = np.array([i["done_s"] - i["submit_s"] for i in infos]) * 1e3
    wait = np.array([i["start_s"] - i["submit_s"] for i in infos]) * 1e3
    span = max_over_ranks(max(i["done_s"] for i in infos) - min(i["submit_s"] for i in infos), world)
    ok = all(i["status"] == 0 for i in infos)
    failed = [{"id": int(i["id"]), "status": int(i["status"]), "n_panels": int(i["n_panels"]),
               "residual": float(i["residual"])} for i in infos if i["status"] != 0]
    ns = np.array([i["n_panels"] for i in infos])
    # one at a time on the same GPU: the first requests, FP64 then mixed
    ctx = gbem.Context(local)
    def loop(prec, k_max, t_cap):
        t = []
        Cs = []
        for k in range(k_max):
            _, boxes, params = reqs[k]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C, _ = gbem.extract(ctx, boxes, params, W.EPS_R_SIO2, precision=prec)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
            Cs.append(C)
            if sum(t) > t_cap:
                break
        return np.array(t), Cs
    t64, C64 = loop(gbem.GBEM_FP64, 8, 40.0)
    tmx, Cmx = loop(gbem.GBEM_MIXED, len(t64), 1e9)
    err = max(float(np.max(np.abs(got[k][1] - C64[k])) / np.max(np.abs(C64[k]))) for k in range(len(C64)))
    ctx.close()
    line = {
        "metric": "extractions/s", "value": whole_job_rate(len(reqs), world, span), "unit": "extractions/s",
        "n_gpus": world,
        "steps": len(reqs), "warmup": len(cal), "ms_per_step": 1e3 * span / len(reqs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {len(reqs)} 2-15 conductor buses, N log-uniform [500,30000]",
                   "rate_per_s": rate, "capacity_per_s": capacity, "slots": args.serve_slots,
                   "hbm_budget_gb": args.serve_budget_gb, "n_max": int(ns.max()), "n_median": int(np.median(ns))},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "queue_wait_p50_ms": float(np.percentile(wait, 50)),
        "queue_wait_p99_ms": float(np.percentile(wait, 99)), "all_ok": ok, "failed": failed,
        "peak_reserved_gb": stats["peak_reserved"] / (1 << 30),
        "one_at_a_time_fp64": {"requests": len(t64), "extractions_per_s": len(t64) / float(t64.sum()),
                               "p50_ms": float(np.percentile(t64, 50) * 1e3)},
        "one_at_a_time_mixed": {"requests": len(tmx), "extractions_per_s": len(tmx) / float(tmx.sum())},
        "cap_rel_err_vs_fp64_gpu": err, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    dist_stop(world)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch512":
        run_batch(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
