"""The bounds-checked build of the library (memory-checker substitute).

libpemlbm_checked.so tests the index of every population, mask,
material-index and palette access of the step kernels, and the lambda and
record accesses of the adjoint kernels, against the extent of its buffer; it
skips and records an access outside it, and never traps.  A child process
loads it (PEMLBM_LIB) and runs every set-up and call of the API on small
lattices with ragged edges: steps in all storage types and both roundings,
the validation set-ups, x-slabs and their halo exchange, every batch
schedule, the read-outs, checkpoints and the adjoint.  No access may be
recorded.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import torch
from paper_2103_01444_gb300 import lbm, workloads
from paper_2103_01444_gb300.lbm import Batch, Domain, bounds_check
from paper_2103_01444_gb300.slabs import SlabLattice

def check(what):
    v = bounds_check()
    assert v == 0, f"{what}: out-of-range access at site {v >> 48}, index {v & ((1 << 48) - 1)}"

cases = {
    "film": workloads.small_cathode(nx=70, ny=18, reaction_mode=0, V_op=0.45, seed=1),
    "vol": workloads.small_cathode(nx=77, ny=20, reaction_mode=1, V_op=0.4, seed=5),
    "grains": workloads.small_cathode(nx=70, ny=24, reaction_mode=0, grains=True, seed=9),
    "film-p": dict(workloads.small_cathode(nx=66, ny=18, reaction_mode=0, seed=2),
                   inlet="pressure", dp_in=1e-3),
    "grains-p-bv": dict(workloads.small_cathode(nx=70, ny=24, reaction_mode=0, grains=True,
                                                V_op=0.95, seed=9),
                        inlet="pressure", dp_in=1e-3, alpha_a=0.5),
}
bounds_check()                                   # clears the record
for name, case in cases.items():
    for prec in ("fp64", "fp32", "bf16", "fp16"):
        for mode in (0, 1):
            d = Domain.from_case(case, precision=prec, interface_mode=mode)
            d.step(40)
            d.step_observe(5)
            d.current_density()
            d.fields()
            d.balances()
            d.residual()
            blob = d.save_state()
            d.load_state(blob)
            if prec in ("bf16", "fp16"):
                s = Domain.from_case(case, precision=prec, interface_mode=mode,
                                     rounding="stochastic")
                s.step(20)
                s.close()
            snap = torch.zeros((5, d.ny, d.nx), device="cuda",
                               dtype=torch.float64 if prec == "fp64" else torch.float32)
            d.residual_noalloc(snap)
            live = (d.mask() & 3) != 3
            lam = np.random.default_rng(0).standard_normal((24, d.ny, d.nx)) * live
            d.vjp(lam)
            d.grad(0, 12, segment=5)
            d.set_grad_memory(0)
            d.grad(1, 12, segment=5)
            d.close()
            check(f"{name} {prec} interface {mode}")
for case in (workloads.natural_convection_cavity(40, Ra=1e4),
             workloads.natural_convection_cavity(36, Ra=1e4, Da=1e-2, phi=0.6),
             workloads.kang_surface_reaction(48, 20, Da=1.0)):
    d = Domain.from_case(case, precision="fp32")
    d.step(30)
    d.fields()
    d.balances()
    d.close()
    check("validation set-ups")
for prec in ("fp64", "fp32", "bf16"):
    lat = SlabLattice(cases["film-p"], 3, precision=prec)
    lat.step(25)
    lat.fields()
    lat.current_density()
    for d in lat.slabs:
        d.close()
    check(f"x-slabs {prec}")
doms = [Domain.from_case(c, precision="fp32") for c in (cases["film"], cases["vol"], cases["grains"])]
b = Batch(doms)
b.tune(2)                                        # (between the reset and the first step)
for sched in ("graph", "persistent", "per-case", "concurrent"):
    b.set_schedule(sched)
    b.step(10)
b.close()
for d in doms:
    d.close()
check("batch schedules")
print("BOUNDS_OK")
'''


def test_checked_build_records_no_out_of_range_access():
    from paper_2103_01444_gb300.build import build
    lib = build(bounds_check=True)
    env = dict(os.environ, PEMLBM_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "BOUNDS_OK" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
