#!/usr/bin/env python
"""Benchmark of the GBEM hot path on GB300.

One step = one full capacitance extraction of the three-layer 5x5x5 crossing
bus (N = 23172 edge-graded panels, 15 conductors, eps_r 3.9), the largest
single-GPU workload: Galerkin assembly (Sec. 3.4, Eq. "matrix"), Cholesky
factorisation (Sec. 3.2), the solve with one right-hand side per conductor
plus FP64 refinement (Eq. "lineareq1") and the charge reduction to the
Maxwell matrix (Eq. "electriccharge").  The 2x2 crossing bus (N = 6264, 4
conductors) is measured the same way and reported under ``secondary``.

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
import platform
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "bus_3layer_5x5x5"
SECONDARY = "crossing_bus_2x2"
DESCRIPTION = {
    "bus_3layer_5x5x5": "three-layer 5x5x5 crossing bus, 15 conductors, edge-graded",
    "crossing_bus_2x2": "2x2 crossing bus, 0.1 um wires, edge-graded",
}
METRIC = "panel-pair integrals/s"
UNIT = "pairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 20; 10 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--secondary-steps", type=int, default=30)
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=24,
                    help="whole matrix rows the all-core oracle evaluates for the CPU baseline")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "batch512", "serving", "partition", "unit_rates", "stack", "sphere",
                             "stack_partition"],
                    help="headline: the three-layer bus (and the 2x2 bus as secondary); "
                         "batch512 / serving: the batched and served forms; unit_rates: the "
                         "arithmetic-unit rates that bound the assembly, nothing else; stack: the "
                         "multi-dielectric system of a layered stack; sphere: flat triangles")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--serve-count", type=int, default=1000)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=96.0)
    ap.add_argument("--serve-rates", default="0.5,0.8,1.0,1.2",
                    help="comma-separated arrival rates as fractions of the measured capacity")
    ap.add_argument("--serve-fp64-loop", type=int, default=120,
                    help="requests of the stream (a seeded uniform sample) the one-at-a-time FP64 loop "
                         "runs (-1: all)")
    ap.add_argument("--profile", default=None, choices=["mixed", "fp64"],
                    help="one warm-up and one extraction in that precision, nothing else "
                         "(for ncu captures)")
    ap.add_argument("--profile-workload", default="crossing_bus_2x2",
                    choices=["crossing_bus_2x2", "two_bars", "bus_3layer_5x5x5", "bus_3layer_mid"],
                    help="structure of the --profile run (two_bars: a small case for pass counts; "
                         "bus_3layer_mid: the three-layer bus at h 70 nm, N = 10938, matrices of 1.5 GB, "
                         "for full-section ncu captures)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else 20
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

def cpu_model() -> str:
    """Model name of the host CPU (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _oracle_rows(O, a, g, rows, threads):
    """Seconds the oracle takes for the whole matrix rows `rows` (every
    pair class appears in a row in its proportion of the whole matrix)."""
    import numpy as np
    n = len(a)
    I = np.repeat(np.asarray(rows, dtype=np.int64), n)
    J = np.tile(np.arange(n), len(rows))
    t0 = time.perf_counter()
    O.entries(a, g, I, J, nthreads=threads)
    return time.perf_counter() - t0


def _lapack_factor_solve(n: int, nrhs: int, n_max: int):
    """LAPACK dpotrf + dpotrs (scipy, the oracle's own solver) on an SPD
    matrix of order m = min(n, n_max); returns (m, factor s, solve s), the
    times scaled to order n by (n/m)^3 and (n/m)^2 when m < n."""
    import numpy as np
    import scipy.linalg as sla
    m = min(n, n_max)
    rng = np.random.default_rng(1)
    M = rng.standard_normal((m, 64))
    A = M @ M.T / 64 + np.eye(m)
    B = rng.standard_normal((m, nrhs))
    t0 = time.perf_counter()
    cf = sla.cho_factor(A, lower=True, overwrite_a=True, check_finite=False)
    t1 = time.perf_counter()
    sla.cho_solve(cf, B, check_finite=False)
    t2 = time.perf_counter()
    return m, (t1 - t0) * (n / m) ** 3, (t2 - t1) * (n / m) ** 2


def cpu_baseline(workload: str, rows_all: int, rows_single: int, lapack_max: int = 12000):
    """The FP64 oracle timed on the host cores on a bounded sample of one
    extraction of `workload`: its entry rate on whole random rows of the
    matrix with all threads and with one thread, plus LAPACK's Cholesky and
    solve (scipy; scaled from order `lapack_max` when N is larger), summed
    into the time of one extraction."""
    import numpy as np
    from oracle import oracle as O
    from paper_2203_11733_gb300 import workloads as W
    boxes, params = getattr(W, workload)()
    a, g, c = O.mesh_boxes(boxes, **params)
    n = len(a)
    nc = len(np.unique(c))
    threads = O.max_threads()
    rng = np.random.default_rng(5)
    rows = rng.choice(n, size=rows_all, replace=False)
    t_all = _oracle_rows(O, a, g, rows, threads)
    rate_all = rows_all * n / t_all
    t_one = _oracle_rows(O, a, g, rows[:rows_single], 1) if rows_single > 0 else None
    _oracle_rows(O, a, g, rows[:1][:0], threads)    # leave the oracle's thread count at all cores
    rate_one = rows_single * n / t_one if t_one else None
    m, t_f, t_s = _lapack_factor_solve(n, nc, lapack_max)
    pairs = n * (n + 1) / 2
    t_extract = pairs / rate_all + t_f + t_s
    out = {
        "value": pairs / t_extract, "unit": UNIT, "cores": threads, "kind": "oracle",
        "sample": (f"{rows_all} whole random rows of the {n}-panel matrix ({rows_all * n} entries) in "
                   f"{t_all:.1f} s on {threads} threads ({rate_all:.0f} entries/s), plus LAPACK dpotrf "
                   f"{'at order ' + str(m) + ' scaled by (N/m)^3' if m < n else 'at full order'} "
                   f"({t_f:.1f} s) and the {nc}-RHS solve ({t_s:.2f} s); one extraction estimated at "
                   f"{t_extract:.0f} s"),
        "cpu_model": cpu_model(),
        "assembly_pairs_per_s_all_cores": rate_all,
        "lapack": {"order_timed": m, "dpotrf_s_at_N": t_f, "dpotrs_s_at_N": t_s,
                   "dpotrf_gflop_per_s": n ** 3 / 3 / t_f / 1e9},
        "extraction_s": t_extract,
    }
    if rate_one:
        out["single_thread"] = {"assembly_pairs_per_s": rate_one, "rows": rows_single,
                                "seconds": t_one,
                                "assembly_s_estimate": pairs / rate_one}
    return out


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores; each
    step a bounded sample (two whole rows and a scaled LAPACK Cholesky) of
    one extraction of the headline workload."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    for _ in range(args.warmup):
        cpu_baseline(WORKLOAD, 1, 0, lapack_max=2048)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(WORKLOAD, 2, 0, lapack_max=4096)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"{WORKLOAD} ({DESCRIPTION[WORKLOAD]})",
                                        "n_panels": 23172, "n_cond": 15, "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"], "cpu_model": last["cpu_model"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- rooflines

PHASES = ["mesh_upload", "assemble", "factor", "solve", "reduce"]

KERNEL_NAMES = {
    "assemble": "assemble_tiles<mixed>: Galerkin entries, one CTA per 32x32 lower tile",
    "factor": "the FP32 factorisation, one span: factor_step (one launch per elimination step: panel "
              "rows, strip update, next diagonal block factor+inverse, tcgen05 3xFP16 tiles of the panel's "
              "columns) beside rest_update (second stream: warp-specialised tcgen05 3xFP16 tiles of the "
              "trailing matrix beyond the panel, K = 256 per panel of four steps)",
    "sweep": "sweep_fwd_f32/sweep_bwd_f32: persistent cooperative triangular sweeps (x_b = z_b - M_b x_p)",
    "residual": "residual_df: R = B - A X, compensated FP32 over float-pair storage",
}
# FP64 cost of one corner term of the near-field closed forms, in DFMA
# equivalents of the library calls' rates measured on the GPU at hand
# (gbem_unit_rates): F = 2 log + 1 atan + 1 sqrt + about 25 arithmetic
# operations; H = 3 log + 3 atan + 1 sqrt + about 40 (16 corner terms per pair)
def term_dfma(rates):
    eq = {k: rates["dfma"] / rates[k] for k in ("dsqrt", "dlog", "datan")}
    f = 2 * eq["dlog"] + eq["datan"] + eq["dsqrt"] + 25
    h = 3 * eq["dlog"] + 3 * eq["datan"] + eq["dsqrt"] + 40
    return f, h, eq


# FP64 far-field evaluation (FP64 mode): 3 differences, r^2 (3), the rsqrt
# estimate and its Newton step (4), the weighted sum (1)
FAR_EVAL_DFMA_FP64 = 11.0
# the trailing updates run in 3xFP16 on the tensor cores (kind::f16, the
# dense BF16/FP16 rate): three FP16 products per useful flop


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "MEASURED_PEAKS.json (of measured)"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "recipe fallback 6.8 TB/s, 1.9 PF bf16 (of fallback)"}


def traffic_per_launch(workload, kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    profiles/traffic_<workload>_mixed.md (dram__bytes_read.sum +
    dram__bytes_write.sum over one factorisation's launches, divided by
    their number), or None."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}_mixed.md")
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


def assembly_work(cls, rates, mixed=True):
    """Algorithmic work of one assembly from its 14 class counts: far-field
    1/r evaluations (n^4 per pair of order n) and FP64 corner-term work of
    the near pairs, with the time each needs at the unit rates `rates`
    (gbem_unit_rates, operations per second)."""
    f_term, h_term, _ = term_dfma(rates)
    far_evals = sum(n ** 4 * (int(cls[2 * n]) + int(cls[2 * n + 1])) for n in range(1, 7))
    near_dfma = 16 * (f_term * int(cls[0]) + h_term * int(cls[1]))
    if mixed:
        t_far = far_evals / rates["mufu_rsqrt"]
        t_near = near_dfma / rates["dfma"]
    else:
        t_far = 0.0
        t_near = (near_dfma + FAR_EVAL_DFMA_FP64 * far_evals) / rates["dfma"]
    return {"far_evaluations": far_evals, "near_pairs_parallel": int(cls[0]),
            "near_pairs_perpendicular": int(cls[1]), "near_fp64_dfma_equiv": near_dfma,
            "t_far_bound_ms": 1e3 * t_far, "t_near_bound_ms": 1e3 * t_near}


def kernel_table(kst, steps, n, cls, peaks, workload, rates):
    """Per traced kernel: time per step and launch, its algorithmic work rate
    and the fraction of the bound that applies to it."""
    out = {}
    useful = n ** 3 / 3.0                                   # Cholesky, per factorisation
    f16 = peaks["bf16_tflops"]
    for k, d in kst.items():
        if d["launches"] == 0:
            continue
        t = d["ms"] / d["launches"] * 1e-3
        e = {"ms_per_step": d["ms"] / steps, "launches_per_step": d["launches"] / steps,
             "us_per_launch": t * 1e6}
        if k == "factor":
            per_launch = useful / (d["launches"] / steps)
            e.update({"bound": "tensor", "unit": "TFLOP/s", "achieved": per_launch / t / 1e12,
                      "peak": f16 / 3.0,
                      "peak_source": f"dense bf16/fp16 {peaks['bf16_tflops']:.1f} TF/s / 3 "
                                     f"(3xFP16 products per useful flop), {peaks['source']}",
                      "work_per_launch": per_launch, "work": "N^3/3 useful flop per factorisation",
                      "method_bytes_per_launch": 4.0 * n * n / (d["launches"] / steps),
                      "traffic": traffic_per_launch(workload, "factor")})
        elif k == "assemble":
            w = assembly_work(cls, rates)
            t_bound = max(w["t_far_bound_ms"], w["t_near_bound_ms"]) * 1e-3
            e.update({"bound": "alu", "unit": "1/r evaluations/s",
                      "achieved": w["far_evaluations"] / t, "peak": rates["mufu_rsqrt"],
                      "peak_source": "MUFU rsqrt rate measured on this GPU before the timed region "
                                     "(gbem_unit_rates)",
                      "frac_of_alu_bound": t_bound / t, "work": w, "traffic": None,
                      "work_per_launch": w["far_evaluations"]})
        else:
            e.update({"bound": "hbm", "unit": "GB/s", "achieved": d["bytes"] / d["launches"] / t / 1e9,
                      "peak": peaks["hbm_gbs"], "peak_source": peaks["source"],
                      "work_per_launch": d["bytes"] / d["launches"], "traffic": None})
        e["frac"] = e["achieved"] / e["peak"] if k != "assemble" else e["frac_of_alu_bound"]
        out[k] = e
    return out


def roofline(kern, kst, steps, ms_traced_step):
    """The roofline object of the kernel with the largest device time."""
    dom = max((k for k in kern if k in kst), key=lambda k: kst[k]["ms"])
    e = kern[dom]
    out = {"kernel": KERNEL_NAMES[dom], "share_of_traced_step": e["ms_per_step"] / ms_traced_step,
           "launches_per_step": e["launches_per_step"], "us_per_launch": e["us_per_launch"]}
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic", "peak_source", "work_per_launch",
                "work", "method_bytes_per_launch"):
        if key in e:
            out[key] = e[key]
    return out


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
    gbem.load()
    eps_r = W.EPS_R_SIO2
    ctx = gbem.Context(local)
    stream = torch.cuda.Stream()
    # unit rates of this GPU, the assembly's roofline (measured outside the timed region)
    rates = ctx.unit_rates(stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def step(mesh, prec):
        mat = gbem.gbem_assemble(mesh, prec, stream)
        C, _ = gbem.gbem_capacitance(mesh, mat, eps_r, stream, want_residual=False)
        mat.close()
        return C

    if args.profile:
        if args.profile_workload == "bus_3layer_mid":
            boxes, params = W.bus_3layer_5x5x5(h=0.07, h_min=0.014)
        else:
            boxes, params = getattr(W, args.profile_workload)()
        mesh = gbem.gbem_mesh(ctx, boxes, params)
        prec = gbem.GBEM_MIXED if args.profile == "mixed" else gbem.GBEM_FP64
        step(mesh, prec)
        torch.cuda.synchronize()
        C = step(mesh, prec)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile": args.profile, "n_panels": mesh.n, "C": C.tolist()}))
        mesh.close()
        ctx.close()
        return

    def timed(fn, k, flush_between=True):
        """k steps timed with CUDA events on the launching stream, L2 flushed
        (untimed) before each; returns total ms, max over ranks."""
        total = 0.0
        out = None
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

    def measure(workload, steps, fp64_steps, clocks=None):
        """Mixed extractions (timed, then traced), the FP64 extraction on the
        same GPU, the end-to-end form and the error against the stored
        oracle result, for one workload."""
        boxes, params = getattr(W, workload)()
        mesh = gbem.gbem_mesh(ctx, boxes, params)
        n, nc = mesh.n, mesh.n_cond
        pairs = n * (n + 1) / 2
        for _ in range(args.warmup):
            step(mesh, gbem.GBEM_MIXED)
        barrier()
        gbem.set_timing(ctx, 1)
        gbem.get_stats(ctx, reset=True)
        if clocks:
            clocks.begin()
        ms_total, C_mixed = timed(lambda: step(mesh, gbem.GBEM_MIXED), steps)
        if clocks:
            clocks.end()
        barrier()
        stats = gbem.get_stats(ctx, reset=True)
        ms_step = ms_total / steps
        # the same steps again with an event pair around every launch of the
        # traced kernels (kept out of the headline timing: the events cost time)
        gbem.set_timing(ctx, 2)
        gbem.get_kernel_stats(ctx, reset=True)
        ms_traced, _ = timed(lambda: step(mesh, gbem.GBEM_MIXED), steps)
        kst = gbem.get_kernel_stats(ctx, reset=True)
        gbem.set_timing(ctx, 0)
        gbem.get_stats(ctx, reset=True)
        # class counts and the final refinement residual (one extra, untimed extraction)
        mat = gbem.gbem_assemble(mesh, gbem.GBEM_MIXED, stream)
        cls = mat.class_counts()
        _, ir_residual = gbem.gbem_capacitance(mesh, mat, eps_r, stream, want_residual=True)
        mat.close()
        # FP64 path on the same GPU
        step(mesh, gbem.GBEM_FP64)
        barrier()
        gbem.set_timing(ctx, 1)
        gbem.get_stats(ctx, reset=True)
        ms64, C_fp64 = timed(lambda: step(mesh, gbem.GBEM_FP64), fp64_steps)
        stats64 = gbem.get_stats(ctx, reset=True)
        gbem.set_timing(ctx, 0)
        ms64_step = ms64 / fp64_steps
        mesh.close()
        # end to end: host boxes -> mesh + upload -> ... -> C on the host
        def step_e2e():
            return gbem.extract(ctx, boxes, params, eps_r, precision=gbem.GBEM_MIXED, stream=stream)[0]
        step_e2e()
        barrier()
        ms_e2e, _ = timed(step_e2e, steps)
        gold_path = os.path.join(ROOT, "tests", "golden", f"{workload}_capacitance.json")
        err_mixed = err_fp64 = None
        if os.path.exists(gold_path):
            C_ref = np.array(json.load(open(gold_path))["C"])
            scale = np.max(np.abs(C_ref))
            err_mixed = float(np.max(np.abs(C_mixed - C_ref)) / scale)
            err_fp64 = float(np.max(np.abs(C_fp64 - C_ref)) / scale)
        peaks = _peaks()
        kern = kernel_table(kst, steps, n, cls, peaks, workload, rates)
        kern["traced_ms_per_step"] = ms_traced / steps
        asm_ms = stats["ms"][PHASES.index("assemble")] / steps
        return {
            "n": n, "nc": nc, "pairs": pairs, "ms_step": ms_step, "ms_total": ms_total,
            "value": whole_job_rate(pairs * steps, world, ms_total * 1e-3),
            "extractions_per_s": world * 1e3 / ms_step,
            "assembly_pairs_per_s": world * pairs / (asm_ms * 1e-3) if asm_ms > 0 else None,
            "phase_ms_per_step": {k: v / steps for k, v in zip(PHASES, stats["ms"])},
            "launches": int(stats["launches"]),
            "fp64": {"value": world * pairs / (ms64_step * 1e-3), "ms_per_step": ms64_step,
                     "extractions_per_s": world * 1e3 / ms64_step,
                     "phase_ms_per_step": {k: v / fp64_steps for k, v in zip(PHASES, stats64["ms"])},
                     "cap_rel_err_vs_oracle": err_fp64},
            "mixed_over_fp64": ms64_step / ms_step,
            "cap_rel_err_vs_oracle": err_mixed, "ir_residual": ir_residual,
            "e2e": {"value": whole_job_rate(pairs * steps, world, ms_e2e * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": n * (5 * 8 + 1 + 4), "d2h_bytes_per_step": nc * nc * 8,
                    "ms_per_step": ms_e2e / steps},
            "kernels": kern, "kst": kst, "ms_traced_step": ms_traced / steps,
            "class_counts": [int(x) for x in cls],
        }

    clocks = ClockSampler(local)
    clocks.start()
    head = measure(WORKLOAD, args.steps, args.fp64_steps, clocks)
    clk = clocks.stop()
    sec = None
    if not args.no_secondary:
        sec = measure(SECONDARY, args.secondary_steps, max(2, args.fp64_steps))
    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(WORKLOAD, args.cpu_rows, 2)
            cpu.pop("extraction_s", None)
        kern = dict(head["kernels"])
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} ({DESCRIPTION[WORKLOAD]})",
                       "n_panels": head["n"], "n_cond": head["nc"], "eps_r": eps_r, "precision": "mixed",
                       "l2": "flushed (512 MB write) before every timed step; matrices of 6.5 GB exceed L2",
                       "parallelism": f"replicas x{world}"},
            "extractions_per_s": head["extractions_per_s"],
            "assembly_pairs_per_s": head["assembly_pairs_per_s"],
            "phase_ms_per_step": head["phase_ms_per_step"],
            "fp64": head["fp64"], "mixed_over_fp64": head["mixed_over_fp64"],
            "cap_rel_err_vs_oracle": head["cap_rel_err_vs_oracle"], "ir_residual": head["ir_residual"],
            "e2e": head["e2e"],
            "gpu_launches": head["launches"],
            "roofline": roofline(kern, head["kst"], args.steps, head["ms_traced_step"]),
            "kernels": kern,
            "assembly_class_counts": head["class_counts"],
            "unit_rates_per_s": rates,
            "clocks": clk,
        }
        if sec is not None:
            line["secondary"] = {
                "workload": f"{SECONDARY} ({DESCRIPTION[SECONDARY]})", "n_panels": sec["n"], "n_cond": sec["nc"],
                "steps": args.secondary_steps, "metric": METRIC, "value": sec["value"], "unit": UNIT,
                "ms_per_step": sec["ms_step"], "extractions_per_s": sec["extractions_per_s"],
                "assembly_pairs_per_s": sec["assembly_pairs_per_s"], "phase_ms_per_step": sec["phase_ms_per_step"],
                "fp64": sec["fp64"], "mixed_over_fp64": sec["mixed_over_fp64"],
                "cap_rel_err_vs_oracle": sec["cap_rel_err_vs_oracle"], "ir_residual": sec["ir_residual"],
                "e2e": sec["e2e"], "roofline": roofline(sec["kernels"], sec["kst"], args.secondary_steps,
                                                         sec["ms_traced_step"]),
                "kernels": sec["kernels"], "gpu_launches": sec["launches"]}
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    ctx.close()
    dist_stop(world)


def stack_cpu_baseline(spec, rows_all: int = 16, rows_single: int = 2):
    """The multi-dielectric oracle timed on the host cores on a bounded sample
    of one extraction: its rate of single- and double-layer entries on whole
    random rows of the system (all threads, and one thread), plus LAPACK's LU
    and solve (scipy) at the full order, summed into one extraction."""
    import numpy as np
    import scipy.linalg as sla
    from oracle import dielectric as D
    from oracle import oracle as O
    st = D.Stack(spec["lo"], spec["hi"], spec["z"], spec["eps_r"], spec["face_bc"])
    m = D.mesh_stack(st, spec["boxes"], spec["h"], spec["h_outer"])
    rows, _, _, ids = D.layout(m)
    ra, rb = m["region_a"], m["region_b"]
    regions = [np.nonzero((ra == a) | (rb == a))[0] for a in range(len(spec["eps_r"]))]
    pairs = sum(len(P) ** 2 for P in regions)
    rng = np.random.default_rng(11)
    threads = O.max_threads()

    def rate(nrows, nthreads):
        I, K = [], []
        for r in rng.integers(0, len(rows), nrows):
            a, i = rows[r]
            I.append(np.full(len(regions[a]), i))
            K.append(regions[a])
        I, K = np.concatenate(I), np.concatenate(K)
        t0 = time.perf_counter()
        D.slayer_entries(m["axis"], m["geo"], I, K, nthreads)
        D.dlayer_entries(m["axis"], m["geo"], I, K, nthreads)
        return len(I) / (time.perf_counter() - t0), len(I), time.perf_counter() - t0

    r_all, e_all, s_all = rate(rows_all, threads)
    r_one, e_one, s_one = rate(rows_single, 1)
    n = len(rows)
    A = np.random.default_rng(3).standard_normal((n, n)) + n * np.eye(n)
    t0 = time.perf_counter()
    f = sla.lu_factor(A, check_finite=False)
    t_lu = time.perf_counter() - t0
    t0 = time.perf_counter()
    sla.lu_solve(f, np.ones((n, len(ids))), check_finite=False)
    t_solve = time.perf_counter() - t0
    t_ext = pairs / r_all + t_lu + t_solve
    return {"value": 1.0 / t_ext, "unit": "extractions/s", "cores": threads, "kind": "oracle",
            "sample": f"{rows_all} whole random rows of the {n}-equation system ({e_all} pairs, single and "
                      f"double layer) in {s_all:.1f} s on {threads} threads, plus LAPACK getrf/getrs at order {n} "
                      f"({t_lu:.2f} + {t_solve:.2f} s); one extraction estimated at {t_ext:.0f} s",
            "cpu_model": platform.processor() or platform.machine(),
            "pairs_per_s_all_cores": r_all, "lapack_getrf_s": t_lu,
            "single_thread": {"pairs_per_s": r_one, "rows": rows_single, "seconds": s_one}}


def run_stack(args):
    """The multi-dielectric path (Sec. 4) on a layered stack: per step the
    assembly of the per-layer system, its LU factorisation with partial
    pivoting, the solve for every conductor and the charges, timed with CUDA
    events on the stream (the 2 x 244 MB of matrices exceed L2, and L2 is
    flushed before each step as well); end to end adds the mesh from the host
    boxes, its upload and the copy of C back."""
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
    gbem.load()
    ctx = gbem.Context(local)
    stream = torch.cuda.Stream()
    spec = W.stack_3layer_5wires()

    def make():
        return gbem.Stack(ctx, spec["lo"], spec["hi"], spec["z"], spec["eps_r"], spec["face_bc"], spec["boxes"],
                          spec["h"], spec["h_outer"])

    S = make()
    if args.profile:
        # one warm-up and one extraction in that precision, nothing else
        prec = gbem.GBEM_MIXED if args.profile == "mixed" else gbem.GBEM_FP64
        for _ in range(2):
            S.assemble(prec, stream)
            C, resid = S.capacitance(stream)
        if rank == 0:
            print(json.dumps({"profile": args.profile, "n_eq": S.n_eq, "residual": resid, "C": C.tolist()}))
        S.close()
        ctx.close()
        return
    rates = ctx.unit_rates(stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        S.assemble(gbem.GBEM_MIXED, stream)
        return S.capacitance(stream)

    def timed(fn, k):
        total = 0.0
        out = None
        for _ in range(k):
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

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = gbem.get_stats(ctx)["launches"]
    clocks.begin()
    ms_total, (C, resid) = timed(step, args.steps)
    clocks.end()
    clk = clocks.stop()
    launches = (gbem.get_stats(ctx)["launches"] - launches0) // args.steps
    ms_step = ms_total / args.steps
    # per-span device times (assembly, LU, sweeps, residual)
    gbem.set_timing(ctx, 2)
    gbem.get_kernel_stats(ctx, reset=True)
    ms_traced, _ = timed(step, args.steps)
    kst = gbem.get_kernel_stats(ctx, reset=True)
    gbem.set_timing(ctx, 0)

    iters_mixed = S.iterations()

    # the same extraction in FP64 (entries and LU), on the same GPU
    def step64():
        S.assemble(gbem.GBEM_FP64, stream)
        return S.capacitance(stream)

    step64()
    ms64, (C64, resid64) = timed(step64, max(1, min(args.steps, 3)))
    ms64_step = ms64 / max(1, min(args.steps, 3))

    def step_e2e():
        T = make()
        try:
            T.assemble(gbem.GBEM_MIXED, stream)
            return T.capacitance(stream)
        finally:
            T.close()

    step_e2e()
    ms_e2e, _ = timed(step_e2e, args.steps)
    np_ = (S.n_eq + 63) // 64 * 64
    names = {"assemble": "stack_assemble<mixed>: single- and double-layer entries of every layer's rows (FP64 "
                         "closed forms near, FP32 Gauss-Legendre far)",
             "factor": "the FP32 LU factorisation, one span: lu_panel (one CTA, partial pivoting), lu_swap, "
                       "lu_trsm and lu_gemm_f32 (128 x 128 tiles) per block of 64 columns",
             "sweep": "the refinement corrections: FP32 triangular sweeps (tri_block / tri_update per block)",
             "residual": "residual_partial / residual_finish: B - M0 X in FP64"}
    kern = {}
    for k, d in kst.items():
        if d["launches"] == 0:
            continue
        t = d["ms"] / d["launches"] * 1e-3
        e = {"ms_per_step": d["ms"] / args.steps, "launches_per_step": d["launches"] / args.steps}
        if k == "factor":
            e.update({"bound": "alu", "unit": "TFLOP/s", "achieved": 2.0 * np_ ** 3 / 3.0 / t / 1e12,
                      "peak": 2.0 * rates["ffma"] / 1e12,
                      "peak_source": "2 x the FFMA rate measured on this GPU (gbem_unit_rates): the FP32 LU",
                      "work_per_launch": 2.0 * np_ ** 3 / 3.0, "work": "2 np^3 / 3 flop per factorisation"})
        else:
            e.update({"bound": "hbm", "unit": "GB/s", "achieved": d["bytes"] / d["launches"] / t / 1e9,
                      "peak": _peaks()["hbm_gbs"], "peak_source": _peaks()["source"],
                      "work_per_launch": d["bytes"] / d["launches"]})
        e["frac"] = e["achieved"] / e["peak"]
        kern[k] = e
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    roof = {"kernel": names[dom], "share_of_traced_step": kern[dom]["ms_per_step"] / (ms_traced / args.steps)}
    for key in ("bound", "achieved", "peak", "unit", "frac", "peak_source", "work_per_launch", "work"):
        if key in kern[dom]:
            roof[key] = kern[dom][key]
    roof["traffic"] = None
    if rank == 0:
        p = S.panels()
        line = {
            "metric": "extractions/s", "value": whole_job_rate(args.steps, world, ms_total * 1e-3),
            "unit": "extractions/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": {"workload": "stack_3layer_5wires (12 x 12 x 4 um, eps_r 3.9 / 2.5 / 7.0, five wires, "
                                   "grounded top and bottom, insulating sides)",
                       "n_panels": S.n, "n_eq": S.n_eq, "n_cond": S.n_cond,
                       "panels_by_kind": {k: int(np.sum(p["kind"] == v)) for k, v in
                                          (("conductor", 0), ("face", 1), ("interface", 2))},
                       "l2": "flushed (512 MB write) before every timed step; the two matrices (2 x 244 MB) "
                             "exceed L2", "parallelism": f"replicas x{world}"},
            "residual": resid, "refinement_iterations": iters_mixed,
            "capacitance_aF": (C * 1e18).round(4).tolist(),
            "fp64": {"ms_per_step": ms64_step, "value": world * 1e3 / ms64_step, "residual": resid64,
                     "mixed_vs_fp64_rel": float(np.abs(C - C64).max() / np.abs(C64).max())},
            "e2e": {"value": whole_job_rate(args.steps, world, ms_e2e * 1e-3), "unit": "extractions/s",
                    "ms_per_step": ms_e2e / args.steps,
                    # the stack's geometry and layout (62 B per panel, 4 per row,
                    # the layer tables) and the quadrature nodes; C, the
                    # residual norms and the status back
                    "h2d_bytes_per_step": 62 * S.n + 4 * S.n_eq + 20 * (len(spec["eps_r"]) + 1) + 672,
                    "d2h_bytes_per_step": 8 * S.n_cond * S.n_cond + 16 * S.n_cond + 4},
            "gpu_launches": int(launches), "roofline": roof, "kernels": kern,
            "unit_rates_per_s": rates, "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = stack_cpu_baseline(spec)
        print(json.dumps(line))
    S.close()
    ctx.close()
    dist_stop(world)


# FP64 cost of the triangle entries in DFMA equivalents at the measured
# library rates: a potential evaluation is three edges of 2 logs, 2 atans,
# 2 square roots and about 40 arithmetic operations.  Mixed mode: 25 x 25
# tanh-sinh nodes per touching pair, 36 per near pair, the far rules in FP32
# (not counted); FP64: 39 x 39, 256, and about 14 operations per far-rule
# evaluation.
def tri_work(counts, rates, mixed=True):
    eq = term_dfma(rates)[2]
    pot = 3 * (2 * eq["dlog"] + 2 * eq["datan"] + 2 * eq["dsqrt"] + 40)
    if mixed:
        return counts[1] * 25 * 25 * pot + counts[2] * 36 * pot
    return counts[1] * 39 * 39 * pot + counts[2] * 256 * pot + sum(counts[k] * k ** 4 * 14 for k in range(3, 7))


def run_sphere(args):
    """Flat triangles (general conductors): the capacitance of a sphere of
    radius 1 um from a level-4 icosphere (5120 triangles), per step the
    assembly (FP64 entries, stored for the mixed factor), the FP32 factor with
    refinement and the charge; against 4 pi eps0 R and the FP64 run."""
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
    gbem.load()
    ctx = gbem.Context(local)
    stream = torch.cuda.Stream()
    rates = ctx.unit_rates(stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tris = W.icosphere(1.0, 4)
    cond = np.zeros(len(tris), np.int32)
    n = len(tris)
    pairs = n * (n + 1) / 2
    c_exact = 4 * math.pi * 8.8541878128e-12 * 1e-6
    mesh = ctx.mesh_from_triangles(tris, cond)

    def step(prec):
        mat = mesh.assemble(prec, stream)
        try:
            return gbem.gbem_capacitance(mesh, mat, 1.0, stream)
        finally:
            mat.close()

    def timed(fn, k):
        total = 0.0
        out = None
        for _ in range(k):
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

    for _ in range(args.warmup):
        step(gbem.GBEM_MIXED)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = gbem.get_stats(ctx)["launches"]
    clocks.begin()
    ms, (C, resid) = timed(lambda: step(gbem.GBEM_MIXED), args.steps)
    clocks.end()
    clk = clocks.stop()
    launches = (gbem.get_stats(ctx)["launches"] - l0) // args.steps
    gbem.set_timing(ctx, 2)
    gbem.get_kernel_stats(ctx, reset=True)
    ms_traced, _ = timed(lambda: step(gbem.GBEM_MIXED), args.steps)
    kst = gbem.get_kernel_stats(ctx, reset=True)
    gbem.set_timing(ctx, 0)
    mat = mesh.assemble(gbem.GBEM_MIXED, stream)
    counts = mat.class_counts()
    mat.close()
    k64 = max(1, min(args.steps, 2))
    ms64, (C64, _) = timed(lambda: step(gbem.GBEM_FP64), k64)

    def e2e():
        m = ctx.mesh_from_triangles(tris, cond)
        try:
            mat = m.assemble(gbem.GBEM_MIXED, stream)
            try:
                return gbem.gbem_capacitance(m, mat, 1.0, stream)
            finally:
                mat.close()
        finally:
            m.close()

    e2e()
    ms_e2e, _ = timed(e2e, args.steps)
    ms_step = ms / args.steps
    work = tri_work([int(x) for x in counts[:7]], rates)
    kern = {}
    for k, d in kst.items():
        if d["launches"] == 0:
            continue
        t = d["ms"] / d["launches"] * 1e-3
        e = {"ms_per_step": d["ms"] / args.steps, "launches_per_step": d["launches"] / args.steps}
        if k == "assemble":
            e.update({"bound": "alu", "unit": "DFMA-eq/s", "achieved": work / t, "peak": rates["dfma"],
                      "peak_source": "DFMA rate measured on this GPU (gbem_unit_rates)", "work_per_launch": work,
                      "work": "FP64 work of the touching and near pairs (exact potentials under tanh-sinh and "
                              "Gauss-Legendre rules) in DFMA equivalents; the FP32 far rules are not counted"})
        elif k == "factor":
            np_ = (n + 127) // 128 * 128
            e.update({"bound": "tensor", "unit": "TFLOP/s", "achieved": np_ ** 3 / 3.0 / t / 1e12,
                      "peak": _peaks()["bf16_tflops"] / 3.0,
                      "peak_source": "dense bf16/fp16 / 3 (3xFP16 products per useful flop), " + _peaks()["source"],
                      "work_per_launch": np_ ** 3 / 3.0, "work": "N^3/3 useful flop per factorisation"})
        else:
            e.update({"bound": "hbm", "unit": "GB/s", "achieved": d["bytes"] / d["launches"] / t / 1e9,
                      "peak": _peaks()["hbm_gbs"], "peak_source": _peaks()["source"],
                      "work_per_launch": d["bytes"] / d["launches"]})
        e["frac"] = e["achieved"] / e["peak"]
        kern[k] = e
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    roof = {"kernel": dom, "share_of_traced_step": kern[dom]["ms_per_step"] / (ms_traced / args.steps),
            "traffic": None}
    for key in ("bound", "achieved", "peak", "unit", "frac", "peak_source", "work_per_launch", "work"):
        if key in kern[dom]:
            roof[key] = kern[dom][key]
    if rank == 0:
        line = {
            "metric": "extractions/s", "value": whole_job_rate(args.steps, world, ms * 1e-3),
            "unit": "extractions/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed): FP32 far rules, FP64 near entries, FP32 factor refined in FP64",
            "data": "synthetic",
            "config": {"workload": "sphere of radius 1 um, level-4 icosphere", "n_panels": n,
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{world}"},
            "pairs_per_s": whole_job_rate(pairs * args.steps, world, ms * 1e-3),
            "c_over_4pi_eps_r": float(C[0, 0] / c_exact), "residual": resid,
            "fp64": {"ms_per_step": ms64 / k64, "mixed_vs_fp64_rel": float(abs(C[0, 0] / C64[0, 0] - 1.0))},
            "class_counts": [int(x) for x in counts[:7]],
            "e2e": {"value": whole_job_rate(args.steps, world, ms_e2e * 1e-3), "unit": "extractions/s",
                    "ms_per_step": ms_e2e / args.steps, "h2d_bytes_per_step": n * (72 + 4),
                    "d2h_bytes_per_step": 8 + 8},
            "gpu_launches": int(launches), "roofline": roof, "kernels": kern, "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            from oracle import oracle as O
            from oracle import triangles as T
            rng = np.random.default_rng(9)
            rows = rng.integers(0, n, 8)
            I, J = np.repeat(rows, n), np.tile(np.arange(n), len(rows))
            t0 = time.perf_counter()
            T.tri_entries(tris, I, J)
            r_all = len(I) / (time.perf_counter() - t0)
            import scipy.linalg as sla
            A = np.eye(n) * n + np.random.default_rng(1).standard_normal((n, n)) * 0.01
            A = 0.5 * (A + A.T)
            t0 = time.perf_counter()
            sla.cho_factor(A)
            t_chol = time.perf_counter() - t0
            t_ext = pairs / r_all + t_chol
            line["cpu_baseline"] = {"value": 1.0 / t_ext, "unit": "extractions/s", "cores": O.max_threads(),
                                    "kind": "oracle",
                                    "sample": f"8 whole random rows ({len(I)} triangle pairs) on {O.max_threads()} "
                                              f"threads, plus LAPACK dpotrf at order {n} ({t_chol:.2f} s); one "
                                              f"extraction estimated at {t_ext:.0f} s"}
        print(json.dumps(line))
    mesh.close()
    ctx.close()
    dist_stop(world)


def run_stack_partition(args):
    """Panels for accuracy on a layered stack (Sec. 3.3 and Sec. 4): net 0's
    column of C in FP64 from uniform meshes and from the paper's partition for
    net 0, against the partition at p1 = 0.025.  Two 3 x 0.5 x 0.5 um wires
    0.5 um apart in the middle of three layers (eps_r 3.9 / 2.5 / 7.0) of a
    16 x 16 x 4 um enclosure, grounded top and bottom, insulating sides.  One
    JSON line."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    B.build()
    ctx = gbem.Context(0)
    lo, hi, z, eps = [-8, -8, 0], [8, 8, 4], [0, 1.5, 2.5, 4], [3.9, 2.5, 7.0]
    bc = [gbem.FACE_NEUMANN] * 4 + [gbem.FACE_GROUND] * 2
    boxes = [([-1.5, -0.25, 1.75], [1.5, 0.25, 2.25], 0), ([-1.5, 0.75, 1.75], [1.5, 1.25, 2.25], 1)]

    def column(h, h_outer, graded=None):
        S = gbem.Stack(ctx, lo, hi, z, eps, bc, boxes, h, h_outer, graded=graded)
        try:
            S.assemble(gbem.GBEM_FP64)
            C, _ = S.capacitance()
            return S.n, np.asarray(C)[:, 0]
        finally:
            S.close()

    n_ref, ref = column(0.25, 8.0, (0, 0.025, 4.0, 1.0, 1.0))
    rows = []
    for label, kw in (("uniform h=0.5 h_outer=4", (0.5, 4.0, None)), ("uniform h=0.25 h_outer=2", (0.25, 2.0, None)),
                      ("uniform h=0.25 h_outer=1", (0.25, 1.0, None)),
                      ("partition p1=0.25", (0.5, 8.0, (0, 0.25, 4.0, 1.0, 1.0))),
                      ("partition p1=0.1", (0.5, 8.0, (0, 0.1, 4.0, 1.0, 1.0))),
                      ("partition p1=0.05", (0.5, 8.0, (0, 0.05, 4.0, 1.0, 1.0)))):
        n, c = column(*kw)
        rows.append({"mesh": label, "panels": n, "err_C00": float(abs(c[0] / ref[0] - 1.0)),
                     "err_C10": float(abs(c[1] / ref[1] - 1.0))})
    print(json.dumps({"workload": "stack_partition", "reference_panels": n_ref, "C00_aF": float(ref[0] * 1e18),
                      "C10_aF": float(ref[1] * 1e18), "rows": rows}))
    ctx.close()


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
    """Poisson streams of 2-15 conductor bus extractions (N log-uniform in
    [500, 30000]) through the continuous-batching server, at a sweep of
    arrival rates given as fractions of the capacity measured on a burst;
    against one-at-a-time mixed extractions of every request of the stream
    and one-at-a-time FP64 extractions of the same requests (all of them, or
    a seeded uniform sample of them: --serve-fp64-loop)."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_start(world)
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem, workloads as W
    B.build()
    budget = int(args.serve_budget_gb * (1 << 30))

    def run_stream(reqs, arrival_scale=None):
        srv = gbem.Server(local, hbm_budget=budget, slots=args.serve_slots)
        got = {}
        t0 = time.perf_counter()
        for k, (t_arr, boxes, params) in enumerate(reqs):
            if arrival_scale is not None:
                while time.perf_counter() - t0 < t_arr * arrival_scale:
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
    cal = W.serving_requests(seed=2024 + rank, count=48, rate_per_s=1.0)
    got, _ = run_stream(cal)
    t_first = min(i["submit_s"] for i, _ in got.values())
    t_last = max(i["done_s"] for i, _ in got.values())
    capacity = len(cal) / (t_last - t_first)
    reqs = W.serving_requests(seed=777 + rank, count=args.serve_count, rate_per_s=1.0)
    ns = np.array([0] * len(reqs))
    sweep = []
    served = None
    clk = None
    for frac in [float(x) for x in args.serve_rates.split(",")]:
        rate = frac * capacity
        clocks = ClockSampler(local)
        clocks.start()
        if world > 1:
            torch.distributed.barrier()
        clocks.begin()
        # the generator's arrival times are for rate 1/s: scale them to `rate`
        got, stats = run_stream(reqs, arrival_scale=1.0 / rate)
        clocks.end()
        c = clocks.stop()
        infos = [got[k][0] for k in range(len(reqs))]
        lat = np.array([i["done_s"] - i["submit_s"] for i in infos]) * 1e3
        wait = np.array([i["start_s"] - i["submit_s"] for i in infos]) * 1e3
        span = max_over_ranks(max(i["done_s"] for i in infos) - min(i["submit_s"] for i in infos), world)
        ns = np.array([i["n_panels"] for i in infos])
        entry = {"rate_fraction_of_capacity": frac, "rate_per_s": rate,
                 "extractions_per_s": whole_job_rate(len(reqs), world, span), "span_s": span,
                 "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                 "mean_ms": float(lat.mean()), "queue_wait_p50_ms": float(np.percentile(wait, 50)),
                 "queue_wait_p99_ms": float(np.percentile(wait, 99)),
                 "all_ok": all(i["status"] == 0 for i in infos),
                 "failed": [{"id": int(i["id"]), "status": int(i["status"]), "n_panels": int(i["n_panels"])}
                            for i in infos if i["status"] != 0],
                 "max_residual": float(max(i["residual"] for i in infos)),
                 "peak_reserved_gb": stats["peak_reserved"] / (1 << 30), "clocks": c}
        sweep.append(entry)
        if served is None or abs(frac - 0.8) < abs(served[0] - 0.8):
            served = (frac, got, entry)
            clk = c
    frac_h, got_h, head = served
    # one at a time on the same GPU: every request mixed, then FP64 on all of
    # them or on a seeded uniform sample
    ctx = gbem.Context(local)

    def loop(prec, idx):
        t = []
        Cs = {}
        for k in idx:
            _, boxes, params = reqs[k]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C, _ = gbem.extract(ctx, boxes, params, W.EPS_R_SIO2, precision=prec)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
            Cs[k] = C
        return np.array(t), Cs

    all_idx = list(range(len(reqs)))
    tmx, _ = loop(gbem.GBEM_MIXED, all_idx)
    if args.serve_fp64_loop < 0 or args.serve_fp64_loop >= len(reqs):
        sub = all_idx
    else:
        rng = np.random.default_rng(99)
        sub = sorted(rng.choice(len(reqs), size=args.serve_fp64_loop, replace=False).tolist())
    t64, C64 = loop(gbem.GBEM_FP64, sub)
    ctx.close()
    err = max(float(np.max(np.abs(got_h[k][1] - C64[k])) / np.max(np.abs(C64[k]))) for k in sub)
    fp64_per_s = len(sub) / float(t64.sum())
    line = {
        "metric": "extractions/s", "value": head["extractions_per_s"], "unit": "extractions/s", "n_gpus": world,
        "steps": len(reqs), "warmup": len(cal), "ms_per_step": 1e3 * head["span_s"] / len(reqs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
        "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {len(reqs)} 2-15 conductor buses, N log-uniform [500,30000]",
                   "rate_per_s": head["rate_per_s"], "rate_fraction_of_capacity": frac_h,
                   "capacity_per_s": capacity, "slots": args.serve_slots, "hbm_budget_gb": args.serve_budget_gb,
                   "n_max": int(ns.max()), "n_median": int(np.median(ns))},
        "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"], "mean_ms": head["mean_ms"],
        "queue_wait_p50_ms": head["queue_wait_p50_ms"], "queue_wait_p99_ms": head["queue_wait_p99_ms"],
        "all_ok": head["all_ok"], "failed": head["failed"], "peak_reserved_gb": head["peak_reserved_gb"],
        "rate_sweep": sweep,
        "one_at_a_time_mixed": {"requests": len(all_idx), "extractions_per_s": len(all_idx) / float(tmx.sum()),
                                "p50_ms": float(np.percentile(tmx, 50) * 1e3)},
        "one_at_a_time_fp64": {"requests": len(sub),
                               "sample": "all requests of the stream" if len(sub) == len(reqs) else
                               f"{len(sub)} requests drawn uniformly (seed 99) from the stream",
                               "extractions_per_s": fp64_per_s, "p50_ms": float(np.percentile(t64, 50) * 1e3)},
        "served_over_fp64_one_at_a_time": head["extractions_per_s"] / fp64_per_s,
        "cap_rel_err_vs_fp64_gpu": err, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    dist_stop(world)


def run_partition(args):
    """Panels for accuracy (Sec. 3.3): the column of the Maxwell matrix that
    belongs to net 0, in FP64, from uniform meshes, edge-graded meshes and the
    paper's distance-graded partition for main net 0, each against the same
    column from a fine mesh of the same structure.  One JSON line per
    structure; the paper's Table 2 geometry (two crossing bars in a grounded
    40 x 40 x 10 um box, eps_r = 1) adds its printed converged values."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem, workloads as W
    B.build()
    ctx = gbem.Context(0)

    def column(mesh, eps_r):
        mat = gbem.gbem_assemble(mesh, gbem.GBEM_FP64)
        try:
            C, _ = gbem.gbem_capacitance(mesh, mat, eps_r)
        finally:
            mat.close()
        return np.asarray(C)[:, 0]

    def graded(boxes, p1, p5, encl, h_max=0.0):
        return gbem.gbem_mesh_graded(ctx, boxes, 0, p1, 4.0, 1.0, p5, h_max=h_max, enclosure=encl)

    def net0_density(mesh, mat):
        """Charge density of net 0's solve on each panel (X / |I|)."""
        a, g, c, ids = mesh.panels()
        B = torch.tensor((c == ids[0]).astype(np.float64), device="cuda")
        X, _ = gbem.gbem_solve(mat, B)
        return X[:, 0].cpu().numpy() / ((g[:, 2] - g[:, 1]) * (g[:, 4] - g[:, 3]))

    def adaptive(start, eps_r, theta=0.5, max_panels=4000, max_steps=8):
        """Sec. 3.2's estimate driving the mesh: solve, indicators from the
        density of net 0, bisect the panels within theta of the largest."""
        out, mesh = [], start
        for _ in range(max_steps):
            mat = gbem.gbem_assemble(mesh, gbem.GBEM_FP64)
            try:
                C, _ = gbem.gbem_capacitance(mesh, mat, eps_r)
                dens = net0_density(mesh, mat)
            finally:
                mat.close()
            out.append((mesh.n, np.asarray(C)[:, 0]))
            if mesh.n >= max_panels:
                break
            new, _, marked = gbem.gbem_mesh_refine(mesh, dens, theta)
            mesh.close()
            mesh = new
        mesh.close()
        return out

    bars, box = W.paper_two_bars()
    studies = [
        # name, boxes, enclosure, eps_r, reference mesh maker, uniform meshes, edge-graded meshes,
        # the paper's p1 values (p2 = 4, p3 = 1), p5
        ("two_bars", W.two_bars()[0], None, W.EPS_R_SIO2,
         ("edge_graded", dict(h=0.01, ratio=1.3, h_min=0.002)),
         [0.2, 0.1, 0.05, 0.03], [0.2, 0.15, 0.1, 0.06], [0.02, 0.01, 0.005, 0.0025, 0.00125], 0.1),
        ("crossing_bus_2x2", W.crossing_bus_2x2()[0], None, W.EPS_R_SIO2,
         ("edge_graded", dict(h=0.015, ratio=1.3, h_min=0.002)),
         [0.1, 0.05, 0.03, 0.02], [0.15, 0.1, 0.06, 0.04], [0.004, 0.002, 0.001, 0.0005, 0.00025], 0.1),
        ("paper_table2", bars, box, 1.0, ("paper_graded", dict(p1=0.02, p5=1.0)),
         [4.0, 2.0, 1.0], [], [3.0, 1.5, 0.75, 0.375, 0.1875], 1.0),
    ]
    for name, boxes, encl, eps_r, (ref_kind, ref_p), hs_u, hs_g, p1s, p5 in studies:
        if ref_kind == "edge_graded":
            mesh = gbem.gbem_mesh(ctx, boxes, ref_p)
        else:
            mesh = graded(boxes, ref_p["p1"], ref_p["p5"], encl)
        n_ref = mesh.n
        ref = column(mesh, eps_r)
        mesh.close()
        rows = []

        def add(kind, param, mesh):
            col = column(mesh, eps_r)
            rows.append({"mesh": kind, "param": param, "panels": mesh.n,
                         "c00_aF": float(col[0] * 1e18), "c10_aF": float(col[1] * 1e18),
                         "err_c00": float(abs(col[0] - ref[0]) / abs(ref[0])),
                         "err_column": float(np.max(np.abs(col - ref)) / abs(ref[0]))})
            mesh.close()
        for h in hs_u:
            if encl is None:
                add("uniform", {"h": h}, gbem.gbem_mesh(ctx, boxes, dict(h=h, ratio=1.0, h_min=0.0)))
            else:   # no area bound, edges capped at h: a uniform grid of nets and walls
                add("uniform", {"h": h}, graded(boxes, 1e9, p5, encl, h_max=h))
        for h in hs_g:
            add("edge_graded", {"h": h, "ratio": 1.5, "h_min": h / 6},
                gbem.gbem_mesh(ctx, boxes, dict(h=h, ratio=1.5, h_min=h / 6)))
        for p1 in p1s:
            add("paper_graded", {"p1": p1, "p2": 4.0, "p3": 1.0, "p5": p5, "main": 0}, graded(boxes, p1, p5, encl))
        # error-driven refinement (Sec. 3.2), from the coarsest uniform mesh
        # or, inside the grounded box, from the coarsest partition
        start = (gbem.gbem_mesh(ctx, boxes, dict(h=hs_u[0], ratio=1.0, h_min=0.0)) if encl is None
                 else graded(boxes, p1s[0], p5, encl))
        for n_k, col in adaptive(start, eps_r):
            rows.append({"mesh": "adaptive", "param": {"theta": 0.5, "start": "uniform h %g" % hs_u[0]
                                                       if encl is None else "partition p1 %g" % p1s[0]},
                         "panels": n_k, "c00_aF": float(col[0] * 1e18), "c10_aF": float(col[1] * 1e18),
                         "err_c00": float(abs(col[0] - ref[0]) / abs(ref[0])),
                         "err_column": float(np.max(np.abs(col - ref)) / abs(ref[0]))})
        # fewest panels within 5 % and 1 % on the column, per kind
        best = {}
        for tol in (0.05, 0.01):
            for kind in ("uniform", "edge_graded", "paper_graded", "adaptive"):
                ok = [r["panels"] for r in rows if r["mesh"] == kind and r["err_column"] <= tol]
                best[f"{kind}_within_{int(tol * 100)}pct"] = min(ok) if ok else None
        out = {"study": "panels_for_accuracy", "structure": name, "net": 0, "precision": "fp64", "eps_r": eps_r,
               "reference": {"mesh": ref_kind, **ref_p, "panels": n_ref,
                             "c00_aF": float(ref[0] * 1e18), "c10_aF": float(ref[1] * 1e18)},
               "fewest_panels": best, "rows": rows}
        if name == "paper_table2":
            out["paper_converged_aF"] = {"C11": 226.0, "C21": -58.7, "panels": 594}
        print(json.dumps(out), flush=True)
    ctx.close()


def run_unit_rates():
    """One JSON line: the rates gbem_unit_rates measures on cuda:0, the SM
    clock around the call, and each FP64 library call in DFMA equivalents."""
    import torch
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    B.build()
    gbem.load()
    torch.cuda.set_device(0)
    ctx = gbem.Context(0)
    stream = torch.cuda.Stream()
    ctx.unit_rates(stream)                     # warm the clocks
    clocks = ClockSampler(0)
    clocks.start()
    clocks.begin()
    rates = ctx.unit_rates(stream)
    clocks.end()
    clk = clocks.stop()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz")
    per_sm_clk = {k: v / (sms * mhz * 1e6) for k, v in rates.items()} if mhz else None
    print(json.dumps({"unit_rates_per_s": rates, "per_sm_per_clock": per_sm_clk, "sms": sms,
                      "dfma_equivalents": term_dfma(rates)[2], "clocks": clk}))
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch512":
        run_batch(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "partition":
        run_partition(args)
    elif args.workload == "unit_rates":
        run_unit_rates()
    elif args.workload == "stack":
        run_stack(args)
    elif args.workload == "sphere":
        run_sphere(args)
    elif args.workload == "stack_partition":
        run_stack_partition(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
