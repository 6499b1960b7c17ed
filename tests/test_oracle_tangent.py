"""The oracle's tangent (forward-mode derivative, oracle/lbm_oracle_tangent.cc).

The tangent build compiles lbm_oracle.c unchanged with dual numbers.  Two
pins tie it to the plain FP64 oracle:
1. its value parts are the plain oracle's numbers, bit for bit;
2. its derivative parts are the derivative of the plain oracle's steps:
   they agree with central differences of the plain build along the same
   direction (state, material fields, inlet drive), to the accuracy of the
   differences.
The GPU adjoint is then checked against this tangent (tests/test_gpu_adjoint.py).
"""
import numpy as np
import pytest

from oracle import Oracle, TangentOracle
from oracle.params import lattice_problem
from paper_2103_01444_gb300 import workloads


def case_of(name):
    if name == "film":
        return workloads.small_cathode(nx=30, ny=12, reaction_mode=0, V_op=0.45, seed=21)
    if name == "vol":
        return workloads.small_cathode(nx=28, ny=16, reaction_mode=1, V_op=0.4, seed=22)
    if name == "grains-p":
        return dict(workloads.small_cathode(nx=32, ny=14, reaction_mode=0, V_op=0.45,
                                            grains=True, seed=23), inlet="pressure", dp_in=1e-3)
    if name == "film-bv":
        return dict(workloads.small_cathode(nx=30, ny=12, reaction_mode=0, V_op=0.85, seed=21),
                    alpha_a=0.5)
    if name == "vol-sa":
        return dict(workloads.small_cathode(nx=28, ny=16, reaction_mode=1, V_op=0.4, seed=22),
                    scalar_advection=1)
    raise KeyError(name)


def drive_key(case):
    return "dp_in" if case.get("inlet") == "pressure" else "u_in_avg"


def state_of(o):
    return np.concatenate([o.f, o.g.reshape(15, o.ny, o.nx)])


CASES = [("film", 0), ("film", 1), ("vol", 1), ("grains-p", 0), ("film-bv", 1), ("vol-sa", 0)]


@pytest.mark.parametrize("name,mode", CASES)
def test_tangent_values_are_the_oracle_bit_for_bit(name, mode):
    case = case_of(name)
    params, mat, solid = lattice_problem(case, interface_mode=mode)
    o = Oracle(params, mat, solid).step(12)
    rng = np.random.default_rng(2)
    t = TangentOracle(params, mat, solid,
                      dmaterial={"phi": rng.standard_normal((case["ny"], case["nx"]))}).step(12)
    np.testing.assert_array_equal(t.f[..., 0], o.f)
    np.testing.assert_array_equal(t.g[..., 0], o.g)
    np.testing.assert_array_equal(t.Jx[:, 0], o.Jx)
    fo, ft = o.fields(), t.fields()
    for k in ("ux", "uy", "T", "C_O2", "C_H2O"):
        np.testing.assert_array_equal(ft[k][0], fo[k])


@pytest.mark.parametrize("name,mode", CASES)
def test_tangent_is_the_derivative_of_the_oracle_steps(name, mode):
    """Along one direction at a time (the state, phi, K, D_O2, alpha_T over
    the GDL, the inlet drive), the tangent's derivative of the state and of
    the current density after 10 steps matches central differences of the
    plain oracle."""
    case = case_of(name)
    N = 10
    params, mat, solid = lattice_problem(case, interface_mode=mode)
    base = Oracle(params, mat, solid).step(15)     # a state away from rest
    s0 = state_of(base)
    ny, nx = case["ny"], case["nx"]
    live = (base.mask & 3) != 3
    gdl = np.zeros((ny, nx), bool)
    gdl[case["ny_cl"]:case["ny_cl"] + case["ny_gdl"]] = True
    gdl &= live
    rng = np.random.default_rng(11)

    def run(material, p, state):
        o = Oracle(p, material, solid)
        o.f[...] = state[:9]
        o.g[...] = state[9:].reshape(3, 5, ny, nx)
        o.step(N)
        return state_of(o), o.current_density()[0]

    directions = [("state", rng.standard_normal(s0.shape) * live * 1e-3)]
    for key in ("phi", "K", "D_O2", "alpha_T"):
        directions.append((key, np.where(gdl, rng.standard_normal((ny, nx)) * mat[key], 0.0)))
    directions.append(("drive", params[drive_key(case)]))
    for key, w in directions:
        dm, dp = {}, {}
        if key == "state":
            t = TangentOracle(params, mat, solid)
            t.set_state(s0[:9], s0[9:].reshape(3, 5, ny, nx), w[:9], w[9:].reshape(3, 5, ny, nx))
        else:
            if key == "drive":
                dp = {drive_key(case): w}
            else:
                dm = {key: w}
            t = TangentOracle(params, mat, solid, dparams=dp, dmaterial=dm)
            t.set_state(s0[:9], s0[9:].reshape(3, 5, ny, nx))
        t.step(N)
        d_state = np.concatenate([t.f[..., 1], t.g[..., 1].reshape(15, ny, nx)])
        d_i = t.current_density()[1]
        h = {"state": 1e-3, "drive": 1e-5}.get(key, 1e-4)

        def shifted(sign):
            if key == "state":
                return run(mat, params, s0 + sign * h * w)
            if key == "drive":
                k = drive_key(case)
                return run(mat, dict(params, **{k: params[k] + sign * h * w}), s0)
            return run(dict(mat, **{key: mat[key] + sign * h * w}), params, s0)
        (sp, ip), (sm, im) = shifted(+1), shifted(-1)
        fd_state = (sp - sm) / (2 * h)
        fd_i = (ip - im) / (2 * h)
        scale = max(np.abs(fd_state).max(), 1e-300)
        err = np.abs(d_state - fd_state).max()
        assert err <= 2e-5 * scale, (key, err, scale)
        # (i_avg sums the reaction of every catalyst cell after N steps: its
        # round-off is about 1e-11 of i_avg, so a central difference carries
        # about 1e-11 |i_avg| / h, which matters for directions the current
        # barely feels)
        assert abs(d_i - fd_i) <= 1e-4 * abs(fd_i) + 1e-10 * abs(ip) / h, (key, d_i, fd_i)
