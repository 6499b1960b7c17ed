"""Full-size parity: the 4096 x 1024 production-shaped cathode in the launch
configuration the benchmark times.

The oracle cannot run thousands of steps of 4.2 M cells, but one step of a
cell depends only on its own column and the two neighbouring columns.  So
for sampled columns (including the inlet and the outlet) the oracle
recomputes one step from a full-height three-column window of the GPU's
state, and the result must match the GPU's next state population by
population.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle.params import lattice_problem
from paper_2103_01444_gb300 import workloads

pytestmark = pytest.mark.gpu


def window_case(case, x0):
    w = dict(case)
    w["nx"] = 3
    w["phi"] = case["phi"][:, x0:x0 + 3]
    w["K_cm2"] = case["K_cm2"][:, x0:x0 + 3]
    if case.get("solid") is not None:
        w["solid"] = case["solid"][:, x0:x0 + 3]
    return w


@pytest.mark.parametrize("precision,mode,tol", [("fp32", 0, 3e-6), ("fp32", 1, 3e-6)])
def test_sampled_columns_one_step(precision, mode, tol):
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Domain
    build()
    case = workloads.cathode_blocks(nx=4096, ny=1024)
    nx, ny = case["nx"], case["ny"]
    d = Domain.from_case(case, precision=precision, interface_mode=mode)
    d.step(300)
    s0 = d.state()
    d.step(1)
    s1 = d.state()
    rng = np.random.default_rng(11)
    cols = sorted(set([0, 1, 31, 32, 33, nx // 2, nx - 2, nx - 1] +
                      list(rng.integers(0, nx, 24))))
    scale = np.abs(s1).reshape(24, -1).max(axis=1)
    worst = 0.0
    for xc in cols:
        x0 = min(max(xc - 1, 0), nx - 3)
        k = xc - x0                           # column of xc inside the window
        params, material, solid = lattice_problem(window_case(case, x0), interface_mode=mode)
        o = Oracle(params, material, solid)
        o.f = np.ascontiguousarray(s0[:9, :, x0:x0 + 3])
        o.g = np.ascontiguousarray(s0[9:, :, x0:x0 + 3].reshape(3, 5, ny, 3))
        o.step(1)
        ref = np.concatenate([o.f, o.g.reshape(15, ny, 3)])[:, :, k]
        got = s1[:, :, xc]
        err = (np.abs(got - ref).max(axis=1) / scale).max()
        worst = max(worst, err)
        assert err < tol, (xc, err)
    print(f"worst scaled one-step difference over {len(cols)} columns: {worst:.3e}")


@pytest.mark.parametrize("kind", ["cavity", "kang"])
def test_validation_setups_sampled_columns_one_step(kind):
    """The same column check for the validation set-ups at the benchmark's
    sizes and tuned launch shape (the extended step instantiation): a
    2048 x 2048 cavity at Ra 1e6 with a heated bottom, and the 4096 x 1024
    surface-reaction box.  The window's own x ends are walls; only columns
    whose neighbours lie inside the window, or that sit on the lattice's
    real walls, are compared."""
    from paper_2103_01444_gb300.build import build
    from paper_2103_01444_gb300.lbm import Domain
    build()
    if kind == "cavity":
        case = workloads.natural_convection_cavity(2048, Ra=1e6, heated_bottom=True)
    else:
        case = workloads.kang_surface_reaction(nx=4096, ny=1024, Da=1.0)
    nx, ny = case["nx"], case["ny"]
    d = Domain.from_case(case, precision="fp32")
    d.tune(5)
    d.step(300)
    s0 = d.state()
    d.step(1)
    s1 = d.state()
    params, material, _ = lattice_problem(case)
    rng = np.random.default_rng(12)
    cols = sorted(set([0, 1, 63, 64, nx // 2, nx - 2, nx - 1] + list(rng.integers(0, nx, 16))))
    scale = np.abs(s1).reshape(24, -1).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)   # the cavity's H2O planes are exactly zero
    worst = 0.0
    for xc in cols:
        x0 = min(max(xc - 1, 0), nx - 3)
        k = xc - x0
        win = {key: (v[:, x0:x0 + 3] if isinstance(v, np.ndarray) and v.ndim == 2 else v)
               for key, v in material.items()}
        o = Oracle(dict(params, nx=3), win, None)
        o.f = np.ascontiguousarray(s0[:9, :, x0:x0 + 3])
        o.g = np.ascontiguousarray(s0[9:, :, x0:x0 + 3].reshape(3, 5, ny, 3))
        o.step(1)
        ref = np.concatenate([o.f, o.g.reshape(15, ny, 3)])[:, :, k]
        err = (np.abs(s1[:, :, xc] - ref).max(axis=1) / scale).max()
        worst = max(worst, err)
        assert err < 3e-6, (xc, err)
    print(f"{kind}: worst scaled one-step difference over {len(cols)} columns: {worst:.3e}")
