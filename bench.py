"""Benchmark of the coupled cathode LBM step on GB300.

Default workload: the 4096 x 1024 production-shaped cathode in FP32 storage
(40/55/5 % channel/GDL/catalyst rows, GDL porosity and permeability drawn
per 32 x 32 block, volumetric catalyst, Re 50, 343 K, 0.5 V).  A step is one
coupled update of every cell (D2Q9 MRT flow + three D2Q5 scalars +
catalyst reaction).  The metric is MLUPS (million lattice-cell updates per
second), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) each rank steps an independent replica of the
workload on its own GPU (weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2103_01444_gb300 import workloads  # noqa: E402

METRIC = "coupled MLUPS"
UNIT = "MLUPS"
NX, NY = 4096, 1024
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16", "fp16"])
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the batched operating-point sweep measurement")
    ap.add_argument("--sweep-cases", type=int, default=64)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=20000)
    ap.add_argument("--sweep-steps", type=int, default=256)
    ap.add_argument("--workload", default="blocks",
                    choices=["blocks", "grains", "cavity", "porous-cavity", "kang"],
                    help="blocks: 4096x1024 GDL blocks + volumetric catalyst; grains: "
                         "8192x2048 pore-scale grains + thin film; cavity, porous-cavity, "
                         "kang: the validation set-ups of Sec. 3 (2048x2048 cavities at "
                         "Ra 1e6, clear with a heated bottom or porous with Da 1e-2; "
                         "a 4096x1024 surface-reaction box), their own line")
    ap.add_argument("--interface", type=int, default=1, choices=[0, 1],
                    help="0: Eq. 10 as printed (per-cell b, alpha C continuous across the "
                         "GDL/channel interface); 1: Fickian interfaces (the default)")
    ap.add_argument("--advection", default="relative", choices=["printed", "relative"],
                    help="flux moments of the D2Q5 equilibria: u C as printed in Eq. 10, or "
                         "u (C - C_in) relative to the inlet values (the default)")
    ap.add_argument("--residual-every", type=int, default=128,
                    help="steps between the residual checks inside the timed region")
    ap.add_argument("--inlet", default="velocity", choices=["velocity", "pressure"],
                    help="drive of the flow: parabolic inlet velocity at Re, or the pressure "
                         "difference of Sec. 4 (--dp-in, lattice units)")
    ap.add_argument("--dp-in", type=float, default=2e-3)
    ap.add_argument("--to-residual", type=float, default=0.0, metavar="TOL",
                    help="instead of the throughput bench: step the workload from reset until "
                         "the residual (checked every 100 steps) is below TOL, or until "
                         "--max-seconds of stepping; one JSON line with steps and wall time")
    ap.add_argument("--max-seconds", type=float, default=240.0)
    ap.add_argument("--cavity-study", action="store_true",
                    help="steady differentially heated cavities (Sec. 3) at Ra 1e3..1e5 on "
                         "three grids: wall Nusselt numbers, their agreement and grid "
                         "convergence; its own line")
    ap.add_argument("--rounding", default="nearest", choices=["nearest", "stochastic"],
                    help="16-bit storage: round to nearest even, or stochastic rounding")
    ap.add_argument("--precision-errors", type=int, default=0, metavar="NSTEPS",
                    help="instead of the throughput bench: run the workload NSTEPS steps with "
                         "FP32, BF16 and FP16 storage and report per-field relative L2 errors "
                         "of the 16-bit runs against the FP32 run (default workload: grains)")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(value: float, pg, device=None) -> float:
    """Max of a float over all ranks (identity without a process group)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg, device=None):
    if pg is not None:
        import torch
        t = torch.zeros(1, device=device)
        pg.all_reduce(t)


def workload(args):
    if args.workload == "grains":
        nx = args.nx if args.nx != NX else 8192
        ny = args.ny if args.ny != NY else 2048
        case = workloads.cathode_grains(nx=nx, ny=ny)
    else:
        case = workloads.cathode_blocks(nx=args.nx, ny=args.ny)
    if getattr(args, "inlet", "velocity") == "pressure":
        case = dict(case, inlet="pressure", dp_in=args.dp_in)
    if getattr(args, "advection", "printed") == "relative":
        case = dict(case, scalar_advection=1)
    return case


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            j = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBps", "copy_gbs"):
                if k in j:
                    return float(j[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; entering
    waits (at most 5 s) for the first sample so that sampling is live when
    the timed region starts."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.out.name) > 0:
                break
            time.sleep(0.05)
        self.start_bytes = os.path.getsize(self.out.name)
        return self

    def mark(self):
        """Drops the samples taken so far (the timed region starts now)."""
        if self.proc is not None and self.out is not None:
            self.out.flush()
            self.start_bytes = os.path.getsize(self.out.name)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return None
        self.out.flush()
        text = open(self.out.name).read()
        os.unlink(self.out.name)
        # samples taken before the timed region started are dropped
        timed = text[getattr(self, "start_bytes", 0):]
        rows = [r.split(",") for r in (timed if timed.strip() else text).strip().splitlines()
                if r.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profiles(workload="cathode-4096x1024", precision="fp32"):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary of a workload and storage, if one exists for the current kernel."""
    path = os.path.join(ROOT, "profiles", f"k_step_{workload}-{precision}.json")
    if os.path.exists(path):
        try:
            j = json.load(open(path))
            if j.get("kernel_source_hash") == kernel_source_hash(precision):
                return float(j["dram_bytes_per_launch"])
        except Exception:
            pass
    return None


STEP_SOURCES = ("lbm_core.cuh", "lbm_step.cuh")
STORAGE_UNIT = {"fp32": "kernels_f32.cu", "fp64": "kernels_f64.cu", "bf16": "kernels_bf16.cu",
                "fp16": "kernels_fp16.cu"}


def kernel_source_hash(precision="fp32"):
    """Hash of the sources that make the step kernel of one storage type (its
    device code, its launcher and its launch shapes): a committed DRAM count
    is used only while these are unchanged."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_01444_gb300", "csrc")
    for name in STEP_SOURCES + (STORAGE_UNIT[precision],):
        h.update(open(os.path.join(csrc, name), "rb").read())
    launch = open(os.path.join(csrc, "lbm_launch.h")).read()
    shapes = re.search(r"kStepShapes\[kStepVariants\] = \{[^;]*;", launch)
    h.update(shapes.group(0).encode() if shapes else b"")
    return h.hexdigest()[:16]


def cpu_baseline(case, seconds_target=15.0, interface_mode=0):
    """The FP64 oracle as it stands, on the host cores, over a bounded number
    of steps of the same workload; returns (MLUPS, cores, sample text)."""
    from oracle import Oracle
    from oracle.params import lattice_problem
    params, material, solid = lattice_problem(case, interface_mode=interface_mode)
    o = Oracle(params, material, solid)
    cells = case["nx"] * case["ny"]
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    n = max(1, int(seconds_target / max(t1 - t0, 1e-6)) - 1)
    n = min(n, 50)
    t2 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t2
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    return cells * n / dt / 1e6, cores, f"{n} oracle steps of the {case['nx']}x{case['ny']} lattice after 1 warm-up step"


_SINGLE_CORE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
from oracle import Oracle
from oracle.params import lattice_problem
from paper_2103_01444_gb300 import workloads
out = {{}}
for name, case, n in (("cathode-1024x256-blocks", workloads.cathode_blocks(1024, 256), 6),
                      ("cathode-200x40 (the 5000-step FP64 case)", workloads.cathode_200x40(), 400)):
    o = Oracle(*lattice_problem(case))
    o.step(1)
    t = time.perf_counter()
    o.step(n)
    out[name] = [case["nx"] * case["ny"] * n / (time.perf_counter() - t) / 1e6, n]
print(json.dumps(out))
"""


def cpu_baseline_extra():
    """The oracle on one host core (OMP_NUM_THREADS=1, a child process) and
    on all cores for the small FP64 case: bounded samples, MLUPS."""
    import subprocess
    out = {}
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", _SINGLE_CORE.format(root=ROOT)], env=env,
                           capture_output=True, text=True, timeout=120)
        for name, (v, n) in json.loads(r.stdout.strip().splitlines()[-1]).items():
            out[f"single_core {name}"] = {"value": v, "unit": UNIT, "cores": 1,
                                          "sample": f"{n} oracle steps after 1 warm-up step"}
    except Exception as e:   # the extra figures never fail the run
        out["single_core"] = {"error": str(e)[:200]}
    from oracle import Oracle
    from oracle.params import lattice_problem
    case = workloads.cathode_200x40()
    o = Oracle(*lattice_problem(case))
    o.step(1)
    t = time.perf_counter()
    o.step(1000)
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    out["all_cores cathode-200x40"] = {"value": 200 * 40 * 1000 / (time.perf_counter() - t) / 1e6,
                                       "unit": UNIT, "cores": cores,
                                       "sample": "1000 oracle steps after 1 warm-up step"}
    return out


def reference_sample(args, budget_s=90.0):
    """Largest lattice of the same recipe (halving nx and ny from the bench
    size) whose W + K oracle steps fit the time budget."""
    from oracle import Oracle
    from oracle.params import lattice_problem
    nx, ny = args.nx, args.ny
    total = max(args.warmup, 3) + max(args.steps, 1)
    while True:
        case = workloads.cathode_blocks(nx=nx, ny=ny)
        if args.advection == "relative":
            case = dict(case, scalar_advection=1)
        params, material, solid = lattice_problem(case, interface_mode=args.interface)
        o = Oracle(params, material, solid)
        t0 = time.perf_counter()
        o.step(1)
        t = time.perf_counter() - t0
        if t * total <= budget_s or (nx <= 128 and ny <= 64):
            return case, o
        nx, ny = max(128, nx // 2), max(64, ny // 2)


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    W, K = max(args.warmup, 3), max(args.steps, 1)
    case, o = reference_sample(args)
    cells = case["nx"] * case["ny"]
    o.step(W)
    t0 = time.perf_counter()
    o.step(K)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    v = cells * K / dt / 1e6
    sample = (f"each step one FP64 oracle step of a {case['nx']}x{case['ny']} lattice of the "
              f"same recipe as the {args.nx}x{args.ny} workload (host cores)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": dt / K * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"cathode-{args.nx}x{args.ny}-blocks",
                       "sample_nx": case["nx"], "sample_ny": case["ny"], "storage": "fp64",
                       "interface_mode": args.interface,
                       "scalar_advection": ("u (C - C_in)" if args.advection == "relative"
                                            else "u C (Eq. 10 as printed)")},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    world, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2103_01444_gb300.build import build
    if rank == 0:
        build()
    barrier(pg, dev)
    build()
    from paper_2103_01444_gb300.lbm import Domain
    case = workload(args)
    cells = case["nx"] * case["ny"]
    stream = torch.cuda.Stream(device=dev)
    d = Domain.from_case(case, precision=args.precision, stream=stream.cuda_stream,
                         interface_mode=args.interface, rounding=args.rounding)
    variant, tune_ms = d.tune(20)       # launch shape of the step kernel
    W, K = max(args.warmup, 3), max(args.steps, 1)
    with ClockSampler(local) as clk:
        # the warm-up runs after the sampler has started (starting it leaves
        # the GPU idle for a while), so that the timed steps start on a busy
        # GPU; only samples taken from the timed region on are kept
        warm_up(d, W)
        torch.cuda.synchronize()
        barrier(pg, dev)
        torch.cuda.synchronize()
        clk.mark()
        ms, launches = timed_steps(d, K, stream, args.residual_every)
    torch.cuda.synchronize()
    barrier(pg, dev)
    ms_max = max_over_ranks(ms, pg, dev)
    clocks = clk.summary()
    # state after the timed run: reaction and the residual over 100 more steps
    i_avg, heat, _ = d.current_density(profile=False)
    d.residual()
    d.step(100)
    res = d.residual()

    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(case, args.precision, K, stream, args.interface)
        e2e_s = max_over_ranks(e2e.pop("seconds"), pg, dev)
        e2e["value"] = world * cells * K / e2e_s / 1e6

    if rank != 0:
        return
    ms_step = ms_max / K
    value = world * cells * K / (ms_max * 1e-3) / 1e6
    bpc = d.bytes_per_cell()
    achieved = bpc * cells / (ms_step * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": case["name"], "nx": case["nx"], "ny": case["ny"],
                   "storage": args.precision + ("" if args.rounding == "nearest"
                                                else ", stochastic rounding"),
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (two population buffers of "
                         f"{24 * cells * d_esize(args.precision) / 1e6:.0f} MB)",
                   "reaction": ("volumetric catalyst rows" if case["reaction_mode"] == 1
                                else "thin catalyst film"),
                   "interface_mode": args.interface,
                   "scalar_advection": ("u (C - C_in)" if case.get("scalar_advection")
                                        else "u C (Eq. 10 as printed)"),
                   "step_variant": variant,
                   "V_op": case["V_op"],
                   "inlet": (f"pressure, dp_in {case['dp_in']:g}" if case.get("inlet") == "pressure"
                             else f"velocity, Re {case['Re']:g}"),
                   "T_in": case["T_in"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (traffic_from_profiles(precision=args.precision)
                                 if args.workload == "blocks" and (args.nx, args.ny) == (NX, NY)
                                 else None),
                     "peak_source": peak_kind, "bytes_per_cell": bpc,
                     "kernel": "k_step (coupled collide+stream)"},
        "gpu_launches": launches,
        "step": ("coupled update of every cell (a1-a7) with the per-step current-density and "
                 f"heat reduction copied to the host (a8), and the residual every "
                 f"{args.residual_every} steps"),
        "clocks": clocks,
        "state_check": {"i_avg_A_cm2": i_avg, "heat_W_cm2": heat, "residual": res},
    }
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_sweep and args.workload == "blocks":
        line["sweep"] = sweep(args, stream)
    if not args.no_adjoint and args.workload == "blocks":
        line["adjoint"] = adjoint_ratio(args, stream)
    if world == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_baseline(case, interface_mode=args.interface)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample, "other_samples": cpu_baseline_extra()}
    print(json.dumps(line), flush=True)


def warm_up(d, W):
    """W untimed steps through the calls the timed region makes (observed
    steps and a residual), so that their first-call set-up (observation
    slots, side stream, step graphs, residual snapshot) happens before the
    timing starts."""
    i_buf, h_buf = np.zeros(W), np.zeros(W)
    d.step_observe(W, i_buf, h_buf)
    d.residual()


def timed_steps(d, K, stream, residual_every):
    """K steps of the whole hot path, timed with CUDA events on the domain's
    stream: each step's coupled update, its current-density and heat
    reduction copied to pinned host memory as the step completes
    (lbm_step_observe), and the steady-state residual every residual_every
    steps.  Returns (ms, kernel launches)."""
    import torch
    i_buf = torch.zeros(K, dtype=torch.float64).pin_memory().numpy()
    h_buf = torch.zeros(K, dtype=torch.float64).pin_memory().numpy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    done, checks = 0, 0
    while done < K:
        n = min(residual_every, K - done)
        d.step_observe(n, i_buf[done:done + n], h_buf[done:done + n])
        done += n
        if n == residual_every:
            d.residual()
            checks += 1
    e1.record(stream)
    e1.synchronize()
    assert np.isfinite(i_buf).all()
    # per step: the step kernel, the catalyst reduction and its column sum;
    # per check: the residual kernel and its block sum
    return e0.elapsed_time(e1), 3 * K + 2 * checks


def sweep_run(cases, args, stream):
    """Cases x steps per second for the tuned batched schedule, for one
    launch per case and step (same kernel, no graph), and their ratio."""
    from paper_2103_01444_gb300.lbm import Batch, Domain
    sa = 1 if args.advection == "relative" else 0
    doms = [Domain.from_case(dict(c, scalar_advection=sa), precision=args.precision,
                             stream=stream.cuda_stream, interface_mode=args.interface)
            for c in cases]
    cells = sum(c["nx"] * c["ny"] for c in cases)
    b = Batch(doms)
    sched, var, _ = b.tune(5)
    K = args.sweep_steps
    b.step(16)
    t_best = b.time_steps(K) / 1e3
    names = ["graph", "persistent", "per-case", "concurrent"]
    b.set_schedule("per-case", variant=var)
    b.step(4)
    t_naive = b.time_steps(K) / 1e3
    n = len(cases)
    others = {}
    for other in ("graph", "persistent", "concurrent"):
        if other != names[sched]:
            b.set_schedule(other, variant=var if other != "persistent" else 6)
            b.step(4)
            others[other] = n * K / (b.time_steps(K) / 1e3)
    out = {"unit": "cases*steps/s", "cases": n, "cells": cells, "steps": K,
           "value": n * K / t_best, "schedule": names[sched],
           "variant": var, "mlups": cells * K / t_best / 1e6,
           "per_case_launches": n * K / t_naive,
           "other_schedules": others,
           "speedup_vs_per_case": t_naive / t_best}
    b.close()
    for d in doms:
        d.close()
    return out


def sweep(args, stream):
    """The operating-point sweep: ncases cathodes of uneven size (512..2048
    x 128..512, V, T, Re, K drawn from a seed) advanced together, and the
    same sweep over 256 small cathodes (128..512 x 32..128), where one launch
    per case leaves most of the GPU idle."""
    out = sweep_run(workloads.sweep_cases(args.sweep_cases), args, stream)
    small = workloads.sweep_cases(256, seed=2103, nx_range=(128, 512), ny_range=(32, 128),
                                  re_range=(5.0, 20.0))
    out["small_cases"] = sweep_run(small, args, stream)
    out["small_cases"]["workload"] = "256 cathodes 128..512 x 32..128, Re 5..20"
    return out


def adjoint_ratio(args, stream):
    """The adjoint on the 1024 x 256 cathode: gradient of the mean current
    density after N steps w.r.t. per-cell phi, K, D_O2 and u_in, checkpoint
    segments of ceil(sqrt N), timed against N forward steps."""
    import torch
    from paper_2103_01444_gb300.lbm import Domain
    case = workloads.cathode_blocks(nx=1024, ny=256, seed=4)
    if args.advection == "relative":
        case = dict(case, scalar_advection=1)
    d = Domain.from_case(case, precision=args.precision, stream=stream.cuda_stream,
                         interface_mode=args.interface)
    d.tune(10)
    N = args.adjoint_steps
    d.step(20)
    torch.cuda.synchronize()
    t_fwd = d.time_steps(N) / 1e3
    t0 = time.perf_counter()
    J, g = d.grad(0, N)
    t_adj = time.perf_counter() - t0
    assert np.isfinite(J) and all(np.isfinite(g[k]).all() for k in ("phi", "K", "D_O2"))
    # the same gradient with every segment recomputed from its checkpoint
    # (no stored reverse records beyond two segments)
    d.set_grad_memory(0)
    t0 = time.perf_counter()
    J_ck, g_ck = d.grad(0, N)
    t_ck = time.perf_counter() - t0
    diff = max(float(np.max(np.abs(g_ck[k] - g[k])) / max(np.max(np.abs(g[k])), 1e-300))
               for k in ("phi", "K", "D_O2"))
    d.close()
    return {"unit": "adjoint/forward time", "value": t_adj / t_fwd, "steps": N,
            "segment": int(np.ceil(np.sqrt(N))), "forward_s": t_fwd, "adjoint_s": t_adj,
            # lbm_grad runs the forward sweep itself (the N steps that give J, with the
            # reverse records of every stored segment); what it adds is the reverse sweep
            "reverse_sweep_over_forward": (t_adj - t_fwd) / t_fwd,
            "records": "every step's reverse records kept from the forward sweep "
                       "(lbm_set_grad_memory -1, the default)",
            "recomputed": {"value": t_ck / t_fwd, "adjoint_s": t_ck,
                           "max_rel_diff_vs_stored": diff, "J_equal": bool(J_ck == J),
                           "records": "every segment recomputed from its checkpoint "
                                      "(lbm_set_grad_memory 0)"},
            "workload": "cathode-1024x256-blocks", "objective": "mean current density"}


def d_esize(precision):
    return {"fp64": 8, "fp32": 4, "bf16": 2, "fp16": 2}[precision]


def end_to_end(case, precision, K, stream, interface_mode=0):
    """The user's job through the public API with host buffers: upload the
    material from pinned host memory, reset, then K observed steps (each
    step's current density and heat copied to pinned host arrays as it
    completes, lbm_step_observe), and a final read of the fields.  MLUPS
    over the wall-clock of the whole job.

    The job runs twice on one domain.  The first run also makes what a
    domain keeps between jobs: the device arrays the material and the fields
    pass through, and the library's work space made at first use (palette
    build scratch, observation slots and side stream).  The second run, the
    reported one, repeats every step of the job itself on that domain."""
    import torch
    from paper_2103_01444_gb300.units import cathode_params
    from paper_2103_01444_gb300.lbm import Domain
    params, fields, geo = cathode_params(case, interface_mode=interface_mode)
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in fields.items()}
    cells = case["nx"] * case["ny"]
    d = Domain(precision=precision, stream=stream.cuda_stream, **geo)
    d.set_params(params)
    fields_host = torch.empty((6, case["ny"], case["nx"]), dtype=torch.float64).pin_memory()
    i_avg = torch.zeros(K, dtype=torch.float64).pin_memory().numpy()
    heat = torch.zeros(K, dtype=torch.float64).pin_memory().numpy()
    dev, out = {}, None

    def job():
        nonlocal out
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the material goes up as six copies from pinned memory; the library
        # builds the palette from them on the device (lbm_set_fields, on_device)
        with torch.cuda.stream(stream):
            for k, v in pinned.items():
                if k not in dev:
                    dev[k] = torch.empty(v.shape, dtype=v.dtype, device="cuda")
                dev[k].copy_(v, non_blocking=True)
        d.set_fields(**dev)
        d.reset()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        d.step_observe(K, i_avg, heat)      # every step's reaction copied to the host
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        assert np.isfinite(i_avg).all() and i_avg[-1] > 0
        with torch.cuda.stream(stream):
            if out is None:
                out = torch.empty((6, case["ny"], case["nx"]), dtype=torch.float64,
                                  device="cuda")
            d.fields(out=out)                 # written on the domain's stream
            fields_host.copy_(out, non_blocking=True)
        stream.synchronize()
        t3 = time.perf_counter()
        assert torch.isfinite(fields_host[3]).all()
        return t3 - t0, {"upload_and_reset": t1 - t0, "steps_with_reads": t2 - t1,
                         "fields_read": t3 - t2}

    first_s, first_breakdown = job()
    dt, breakdown = job()
    h2d = 6 * 8 * cells                   # the six material arrays
    d2h = K * 2 * 8 + 6 * 8 * cells
    d.close()
    return {"seconds": dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
            "breakdown_s": breakdown,
            "first_job": {"value": cells * K / first_s / 1e6, "breakdown_s": first_breakdown,
                          "includes": "the same job on a new domain, with the device arrays "
                                      "and the library's first-use work space made inside"},
            "includes": "material upload from pinned memory (palette built on the device), "
                        "reset, per-step current-density and heat copy to the host "
                        "(lbm_step_observe), final fields read into pinned memory; a job on "
                        "a domain that has run one before"}


def run_cavity_study(args):
    """The clear cavity of Sec. 3 with the left wall hot, the right wall cold
    and the top and bottom insulated, run to a steady state in FP64 storage
    (residual below 1e-10, checked every 1000 steps, at most 40 diffusion
    times L^2/alpha; FP32 storage drifts away from the steady state over
    millions of steps in the closed cavity) on
    grids of 32, 64 and 128 cells for Ra 1e3 and of 64, 128 and 256 cells
    for Ra 1e4 and 1e5: the mean Nusselt numbers of the hot and the cold wall
    (equal at a steady state), the largest velocities in units of alpha / L,
    and the observed order of convergence of Nu between the grids; then the
    porous cavity (porosity 0.6, Darcy number 1e-2) at Ra 1e4 and 1e5."""
    import torch
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Domain, LbmError
    build()
    out = []
    runs = [(1e3, None, (32, 64, 128)), (1e4, None, (64, 128, 256)), (1e5, None, (64, 128, 256)),
            (1e4, 1e-2, (32, 64, 128)), (1e5, 1e-2, (64, 128, 256))]
    for Ra, Da, grids in runs:
        row = {"Ra": Ra, "Da": Da, "phi": 0.6 if Da else 1.0, "grids": []}
        for n in grids:
            case = (workloads.natural_convection_cavity(n, Ra=Ra) if Da is None else
                    workloads.natural_convection_cavity(n, Ra=Ra, Da=Da, phi=0.6))
            d = Domain.from_case(case, precision="fp64")
            alpha = d.params["nu"] / case["Pr"]
            dT = case["T_hot"] - case["T_cold"]
            cap = int(40 * n * n / alpha)
            t0 = time.perf_counter()
            d.residual()
            steps, r = 0, float("inf")
            try:
                while steps < cap and r >= 1e-10:
                    d.step(1000)
                    steps += 1000
                    r = d.residual()
            except LbmError as e:       # diverged: reported, not fatal
                row["grids"].append({"n": n, "steps": steps, "error": str(e)})
                d.close()
                continue
            b = d.balances()
            f = d.fields()
            torch.cuda.synchronize()
            row["grids"].append({
                "n": n, "steps": steps, "residual": r, "wall_s": time.perf_counter() - t0,
                "Nu_hot": b["in_T"] / (alpha * dT), "Nu_cold": -b["out_T"] / (alpha * dT),
                "u_max": float(np.abs(f["ux"]).max()) * n / alpha,
                "v_max": float(np.abs(f["uy"]).max()) * n / alpha})
            d.close()
        nu = [g.get("Nu_hot", float("nan")) for g in row["grids"]]
        if np.all(np.isfinite(nu)) and abs(nu[2] - nu[1]) > 0 and abs(nu[1] - nu[0]) > 0:
            row["observed_order"] = float(np.log2(abs(nu[1] - nu[0]) / abs(nu[2] - nu[1])))
            row["Nu_extrapolated"] = nu[2] + (nu[2] - nu[1]) / (2 ** row["observed_order"] - 1)
        out.append(row)
    print(json.dumps({"metric": "steady cavity Nusselt numbers", "storage": "fp64",
                      "Pr": 0.71, "results": out}), flush=True)


def run_to_residual(args):
    """The separate run of the production cathode to residual < TOL: steps
    and wall time from reset, the residual r = max over (u_x, u_y, T - T_in,
    C_O2, C_H2O) of ||X^n - X^{n-100}|| / ||X^n|| checked every 100 steps
    (FP64 accumulation), and its trace.  Stops at TOL or after max-seconds
    of stepping and says which."""
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Domain, LbmError
    build()
    case = workload(args)
    d = Domain.from_case(case, precision=args.precision, interface_mode=args.interface)
    d.tune(10)
    d.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, r, trace = 0, float("inf"), []
    d.residual()                       # snapshot of the reset state
    while True:
        d.step(100)
        steps += 100
        try:
            r = d.residual()
        except LbmError as e:          # diverged: report it
            r = float("nan")
            trace.append([steps, str(e)])
            break
        if steps % 10000 == 0 or r < args.to_residual:
            trace.append([steps, r])
        if r < args.to_residual or time.perf_counter() - t0 > args.max_seconds:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    i_avg, heat, _ = d.current_density(profile=False)
    cells = case["nx"] * case["ny"]
    print(json.dumps({
        "metric": "steps to residual", "tol": args.to_residual,
        "reached": bool(r < args.to_residual), "steps": steps, "wall_s": wall,
        "final_residual": r, "mlups_incl_checks": cells * steps / wall / 1e6,
        "i_avg_A_cm2": i_avg, "heat_W_cm2": heat,
        "config": {"workload": f"cathode-{case['nx']}x{case['ny']}-{args.workload}",
                   "storage": args.precision, "check_every": 100},
        "trace": trace}))
    d.close()


def run_precision_errors(args):
    """Reduced-precision storage at full size: the workload stepped NSTEPS
    times from reset with FP32, BF16 and FP16 populations (FP32 arithmetic
    in all), the 16-bit ones with round-to-nearest and with stochastic
    rounding; per-field relative L2 errors of the 16-bit runs against the
    FP32 run over the fluid cells, and the current density of each.
    The FP64 oracle is far too slow for this size; the comparison against
    it is made on small grain cathodes by the tests."""
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Domain
    build()
    case = workload(args)
    N = args.precision_errors
    out, ref, live = {}, None, None
    runs = [("fp32", "nearest")] + [(p, r) for p in ("bf16", "fp16")
                                    for r in ("nearest", "stochastic")]
    for prec, rounding in runs:
        d = Domain.from_case(case, precision=prec, interface_mode=args.interface,
                             rounding=rounding)
        d.tune(5)
        d.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.step(N)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        f = d.fields()
        i_avg = d.current_density(profile=False)[0]
        if live is None:
            live = (d.mask() & 3) != 3
        fields = {"u": np.stack([f["ux"], f["uy"]]), "T-T_in": f["T"] - case["T_in"],
                  "C_O2": f["C_O2"], "C_H2O": f["C_H2O"]}
        row = {"i_avg_A_cm2": i_avg, "glups": case["nx"] * case["ny"] * N / wall / 1e9}
        if ref is None:
            ref = (fields, i_avg)
        else:
            for k, v in fields.items():
                m = np.broadcast_to(live, v.shape)
                row[k] = float(np.linalg.norm((v - ref[0][k])[m]) / np.linalg.norm(ref[0][k][m]))
            row["i_avg"] = abs(i_avg - ref[1]) / abs(ref[1])
        out[prec if prec == "fp32" else f"{prec}-{rounding}"] = row
        d.close()
    print(json.dumps({"metric": "per-field relative L2 error of 16-bit storage vs FP32",
                      "steps": N, "config": {"workload": case["name"], "nx": case["nx"],
                                             "ny": case["ny"], "interface_mode": args.interface},
                      "results": out}))


def validation_case(args):
    if args.workload == "cavity":
        n = args.nx if args.nx != NX else 2048
        return workloads.natural_convection_cavity(n, Ra=1e6, heated_bottom=True)
    if args.workload == "porous-cavity":
        n = args.nx if args.nx != NX else 2048
        return workloads.natural_convection_cavity(n, Ra=1e6, Da=1e-2, phi=0.6)
    return workloads.kang_surface_reaction(nx=args.nx, ny=args.ny, Da=1.0)


def run_validation(args):
    """MLUPS of the step on a validation set-up of Sec. 3 (the extended
    step instantiation: closed ends, fixed wall values, buoyancy), with the
    wall balances of the state it reaches."""
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2103_01444_gb300.build import build
    build()
    from paper_2103_01444_gb300.lbm import Domain
    case = validation_case(args)
    cells = case["nx"] * case["ny"]
    stream = torch.cuda.Stream(device=dev)
    d = Domain.from_case(case, precision=args.precision, stream=stream.cuda_stream)
    variant, _ = d.tune(20)
    W, K = max(args.warmup, 3), max(args.steps, 1)
    d.step(W)
    torch.cuda.synchronize()
    barrier(pg, dev)
    with ClockSampler(local) as clk:
        ms = d.time_steps(K)
    launches = K   # one step kernel per step (no reductions in the timed region)
    torch.cuda.synchronize()
    ms_max = max_over_ranks(ms, pg, dev)
    b = d.balances()
    if rank != 0:
        return
    ms_step = ms_max / K
    bpc = d.bytes_per_cell()
    achieved = bpc * cells / (ms_step * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    state = {k: b[k] for k in ("in_T", "out_T", "J", "in_O2")}
    if case["kind"] == "cavity":
        alpha = d.params["nu"] / case["Pr"]
        dT = case["T_hot"] - case["T_cold"]
        # wall-averaged Nusselt numbers of the state reached (not steady)
        state["Nu_left"] = b["in_T"] / (alpha * dT)
        state["Nu_right"] = -b["out_T"] / (alpha * dT)
    line = {
        "metric": METRIC, "value": world * cells * K / (ms_max * 1e-3) / 1e6, "unit": UNIT,
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}-{case['nx']}x{case['ny']}",
                   "nx": case["nx"], "ny": case["ny"], "storage": args.precision,
                   "parallelism": f"replicas{world}", "step_variant": variant,
                   "l2": "inputs larger than L2 (two population buffers of "
                         f"{24 * cells * d_esize(args.precision) / 1e6:.0f} MB)",
                   **{k: case[k] for k in ("Ra", "Pr", "Da", "phi", "heated_bottom", "D")
                      if k in case}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (traffic_from_profiles("cavity-2048x2048", "fp32")
                                 if args.workload == "cavity" and args.precision == "fp32"
                                 and case["nx"] == 2048 else None),
                     "peak_source": peak_kind,
                     "bytes_per_cell": bpc,
                     "kernel": "k_step, extended instantiation (" +
                               ("128 x 2" if variant <= 2 else "64 x 2") + " threads per block)"},
        "gpu_launches": launches,
        "step": ("coupled update of every cell (a1-a7) with the per-step current-density and "
                 f"heat reduction copied to the host (a8), and the residual every "
                 f"{args.residual_every} steps"), "clocks": clk.summary(), "state_check": state,
    }
    if world == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_baseline(case, interface_mode=args.interface)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload in ("cavity", "porous-cavity", "kang"):
        run_validation(a)
    elif a.cavity_study:
        run_cavity_study(a)
    elif a.to_residual > 0:
        run_to_residual(a)
    elif a.precision_errors > 0:
        if a.workload == "blocks" and a.nx == NX and a.ny == NY:
            a.workload = "grains"
        run_precision_errors(a)
    else:
        run_ours(a)
