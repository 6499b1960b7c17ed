"""The validation set-ups of Sec. 3 on the CUDA path, against the oracle:
natural convection in a clear cavity heated from the left and the bottom,
in a porous cavity heated from the left (Darcy-Forchheimer force with the
buoyancy), and Kang's diffusion with a first-order surface reaction.  They
run the extended step instantiation (closed x ends, fixed wall values,
buoyancy); FP64 storage must match the oracle to round-off, FP32 storage
within relative L2 1e-5, and the wall balances must equal the oracle's.
"""
import numpy as np
import pytest

from oracle import Oracle
from oracle.oracle import DIAG
from oracle.params import lattice_problem
from paper_2103_01444_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_01444_gb300.build import build
    build()


def gpu_domain(case, precision="fp64"):
    from paper_2103_01444_gb300.lbm import Domain
    return Domain.from_case(case, precision=precision)


def oracle_of(case):
    return Oracle(*lattice_problem(case))


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (den if den > 0 else 1.0)


CASES = {
    "cavity-heated-bottom-24": lambda: workloads.natural_convection_cavity(
        24, Ra=1e4, heated_bottom=True),
    "cavity-ragged-70x70": lambda: workloads.natural_convection_cavity(70, Ra=1e5),
    "porous-cavity-20": lambda: workloads.natural_convection_cavity(20, Ra=1e4, Da=1e-2, phi=0.6),
    "kang-30x12": lambda: workloads.kang_surface_reaction(30, 12, Da=2.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mask_bit_exact(name):
    case = CASES[name]()
    np.testing.assert_array_equal(gpu_domain(case).mask(), oracle_of(case).mask)


@pytest.mark.parametrize("name,steps", [("cavity-heated-bottom-24", 600),
                                        ("cavity-ragged-70x70", 300),
                                        ("porous-cavity-20", 600), ("kang-30x12", 600)])
def test_fp64_state_matches_oracle(name, steps):
    case = CASES[name]()
    d, o = gpu_domain(case), oracle_of(case)
    d.step(steps)
    o.step(steps)
    st = d.state()
    ref = np.concatenate([o.f, o.g.reshape(15, o.ny, o.nx)], axis=0)
    for q in range(24):
        scale = max(np.abs(ref[q]).max(), 1e-300)
        np.testing.assert_allclose(st[q], ref[q], rtol=0, atol=1e-11 * scale,
                                   err_msg=f"population plane {q}")
    fg, fo = d.fields(), o.fields()
    for k in ("ux", "uy", "T", "C_O2", "C_H2O"):
        assert rel_l2(fg[k], fo[k]) < 1e-11, k
    if case["kind"] == "cavity":
        assert np.abs(fo["uy"]).max() > 1e-3          # the buoyancy drives a flow
    # balances of the last step: the heat through the held x walls and, for
    # Kang's case, the reaction and the reactant entering at the left wall
    b, dg = d.balances(), o.diag
    for key in ("in_T", "out_T", "in_O2", "out_O2"):
        # T flows are differences of populations of about 343 K each
        tol = 1e-10 if key.endswith("_T") else 1e-14
        assert b[key] == pytest.approx(dg[DIAG[key]], rel=1e-9, abs=tol), key
    assert b["J"] == pytest.approx(dg[DIAG["J"]], rel=1e-9, abs=1e-16)


@pytest.mark.parametrize("name,steps", [("cavity-heated-bottom-24", 2000),
                                        ("porous-cavity-20", 2000), ("kang-30x12", 2000)])
def test_fp32_fields_within_tolerance(name, steps):
    """FP32 storage within relative L2 1e-4: FP32 rounding of a per-step
    increment that keeps its sign adds up linearly over the run, so 2000
    steps allow about 2000 x 2^-24 = 1.2e-4 (measured: up to 2.3e-5 for the
    cavity's velocity, whose buoyancy feeds the temperature's rounding back
    into a developing flow, and 1.5e-5 for Kang's reactant)."""
    case = CASES[name]()
    d, o = gpu_domain(case, "fp32"), oracle_of(case)
    d.step(steps)
    o.step(steps)
    fg, fo = d.fields(), o.fields()
    err = {k: rel_l2(fg[k], fo[k]) for k in ("ux", "uy", "T", "C_O2")}
    assert max(err.values()) < 1e-4, err
    if case["kind"] == "kang":
        # the left wall holds T at the reference (initial) value: no heat
        # crosses it in exact arithmetic; in FP32 what remains is the
        # collision's rounding, below 1e-7 K per wall link and step (the
        # wall link's two large products alone left about 5e-6)
        assert abs(d.balances()["in_T"]) < 1e-7 * case["ny"]


def test_cavity_256_fp32_matches_oracle():
    """A 256 x 256 cavity (several launch tiles, Ra 1e6) after 150 steps."""
    case = workloads.natural_convection_cavity(256, Ra=1e6, heated_bottom=True)
    d, o = gpu_domain(case, "fp32"), oracle_of(case)
    d.step(150)
    o.step(150)
    fg, fo = d.fields(), o.fields()
    err = {k: rel_l2(fg[k], fo[k]) for k in ("ux", "uy", "T")}
    assert err["T"] < 1e-5 and err["ux"] < 1e-4 and err["uy"] < 1e-4, err


def test_validation_setups_are_refused_where_not_covered():
    from paper_2103_01444_gb300.lbm import Batch, Domain, LbmError
    case = CASES["cavity-heated-bottom-24"]()
    d = gpu_domain(case)
    d.step(2)
    with pytest.raises(LbmError, match="EINVAL.*adjoint"):
        d.grad(0, 4)
    with pytest.raises(LbmError, match="EINVAL"):
        Batch([d])
    p = dict(d.params)
    with pytest.raises(LbmError, match="EINVAL.*thin film"):
        d.set_params(dict(p, wall_dirichlet=p["wall_dirichlet"] | (1 << 7)))
    # fixed right-wall values need closed ends
    k = workloads.small_cathode(nx=40, ny=12)
    e = Domain.from_case(k, precision="fp64", reset=False)
    with pytest.raises(LbmError, match="EINVAL.*closed_x"):
        e.set_params(dict(e.params, wall_dirichlet=1 << 3))
    with pytest.raises(LbmError, match="EINVAL.*periodic"):
        Domain(16, 8, periodic_x=1, closed_x=1)
