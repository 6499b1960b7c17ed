"""Failure paths on the GPU without any device fault: allocations made to
fail on the host (PEMLBM_FAIL_ALLOC, the library's fault-injection hook)
must come back as LBM_ENOMEM from whichever call made them, leave no
half-built object behind, and leave the CUDA context usable."""
import numpy as np
import pytest

from paper_2103_01444_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_01444_gb300.build import build
    build()


def session(case):
    """A short use of most of the API; returns normally or raises LbmError."""
    from paper_2103_01444_gb300.lbm import Batch, Domain
    d = Domain.from_case(case, precision="fp32")
    d.step(130)                      # graph capture and replay
    d.step_observe(70)               # observation slots and streams
    d.fields()                       # read-out scratch
    d.grad(0, 6, segment=3)          # adjoint workspace and checkpoints
    b = Batch([d])
    b.set_schedule("concurrent", variant=7)
    b.step(2)
    b.close()
    d.close()


def test_allocation_failures_return_enomem_and_the_context_survives(monkeypatch):
    from paper_2103_01444_gb300.lbm import Domain, LbmError
    case = workloads.small_cathode(nx=40, ny=12)
    failed = []
    for n in range(1, 41):
        monkeypatch.setenv("PEMLBM_FAIL_ALLOC", str(n))
        try:
            session(case)
        except LbmError as e:
            assert "ENOMEM" in str(e), (n, str(e))
            failed.append(n)
        finally:
            monkeypatch.delenv("PEMLBM_FAIL_ALLOC")
    # every allocation of the session can fail; the first fifteen or so are
    # the domain's own
    assert len(failed) >= 15, failed
    assert failed[:13] == list(range(1, 14)), failed
    d = Domain.from_case(case, precision="fp32")
    d.step(50)
    i, _, _ = d.current_density()
    assert np.isfinite(i) and i > 0
