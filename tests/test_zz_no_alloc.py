"""lbm_residual_noalloc: the residual for callers that must not allocate.

Real-time loops (a cudaMalloc can stall the device's streams for an
unbounded time) and hosts that hand out all device memory from their own
pool cannot let the library allocate when they ask for the steady-state
residual.  lbm_residual_noalloc keeps its scratch in a static device array
and takes the snapshot from the caller; it must give the same residual as
lbm_residual, call after call, and must not allocate.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _domain(case, precision):
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Domain
    build()
    return Domain.from_case(case, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_residual_matches_lbm_residual_on_two_calls(precision):
    import torch
    from paper_2103_01444_gb300 import workloads
    case = workloads.small_cathode(nx=300, ny=64, reaction_mode=1, V_op=0.45)
    d = _domain(case, precision)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    snap = torch.zeros((5, d.ny, d.nx), dtype=dtype, device="cuda")
    torch.cuda.synchronize()
    # first call: the snapshot of the reset state (the domain took its own)
    r0 = d.residual_noalloc(snap)
    assert r0 == pytest.approx(1.0)
    for _ in range(2):
        d.step(60)
        r_ref = d.residual()
        r_new = d.residual_noalloc(snap)
        assert np.isfinite(r_new) and r_new > 0
        assert r_new == pytest.approx(r_ref, rel=1e-12, abs=0)
    # the caller's snapshot now holds the current moments
    r_same = d.residual_noalloc(snap)
    assert r_same == 0.0


def test_noalloc_residual_allocates_nothing(monkeypatch):
    """With the library's allocation-failure hook armed on its first
    allocation, the call still succeeds and gives lbm_residual's value,
    twice; a call that does allocate (a new domain) fails under the same
    hook, which shows it was armed."""
    import torch
    from paper_2103_01444_gb300 import workloads
    from paper_2103_01444_gb300.lbm import LbmError
    case = workloads.small_cathode(nx=130, ny=40, reaction_mode=0, V_op=0.45)
    d = _domain(case, "fp32")
    snap = torch.zeros((5, d.ny, d.nx), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    d.residual_noalloc(snap)
    monkeypatch.setenv("PEMLBM_FAIL_ALLOC", "1")
    for _ in range(2):
        d.step(40)
        r_ref = d.residual()
        r_new = d.residual_noalloc(snap)
        assert r_new == pytest.approx(r_ref, rel=1e-12, abs=0) and r_new > 0
    with pytest.raises(LbmError, match="ENOMEM"):
        _domain(case, "fp32")
    monkeypatch.delenv("PEMLBM_FAIL_ALLOC")


def test_noalloc_residual_rejects_lattices_beyond_its_scratch():
    from paper_2103_01444_gb300 import workloads
    from paper_2103_01444_gb300.lbm import LbmError
    import torch
    case = workloads.cathode_blocks(nx=4224, ny=1024)      # 16896 blocks > 16384
    d = _domain(case, "bf16")
    snap = torch.zeros((5, d.ny, d.nx), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(LbmError, match="EINVAL.*16384"):
        d.residual_noalloc(snap)
