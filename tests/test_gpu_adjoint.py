"""Discrete adjoint of the coupled step.

1. One transposed step against finite differences of the FP64 GPU step and
   of the independent FP64 oracle's step (dot-product test) in state and
   parameter directions, and against the oracle's own derivative of its
   step (its tangent, the step run in dual numbers) to rounding.
2. Gradients of the objectives (mean current density, hottest catalyst-row
   temperature) after N steps against FP64 central finite differences of the
   independent oracle, within 1e-3 relative, and against the oracle's
   tangent through the same steps, within 1e-9.
"""
import numpy as np
import pytest

from oracle import Oracle, TangentOracle
from oracle.params import lattice_problem
from paper_2103_01444_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2103_01444_gb300.build import build
    build()


def case_of(name):
    if name == "film":
        return workloads.small_cathode(nx=40, ny=14, reaction_mode=0, V_op=0.45, seed=21)
    if name == "vol":
        return workloads.small_cathode(nx=36, ny=20, reaction_mode=1, V_op=0.4, seed=22)
    if name == "grains":
        return workloads.small_cathode(nx=44, ny=16, reaction_mode=0, V_op=0.45, grains=True,
                                       seed=23)
    if name == "film-bv":      # Butler-Volmer near open circuit
        return dict(workloads.small_cathode(nx=40, ny=14, reaction_mode=0, V_op=1.05, seed=21),
                    alpha_a=0.5)
    if name == "vol-bv":
        return dict(workloads.small_cathode(nx=36, ny=20, reaction_mode=1, V_op=1.05, seed=22),
                    alpha_a=0.5)
    if name == "film-bv1":     # Butler-Volmer, anodic branch about 1 % of the flux
        return dict(workloads.small_cathode(nx=40, ny=14, reaction_mode=0, V_op=1.0, seed=21),
                    alpha_a=0.5)
    if name == "vol-bv1":
        return dict(workloads.small_cathode(nx=36, ny=20, reaction_mode=1, V_op=1.0, seed=22),
                    alpha_a=0.5)
    if name.endswith("-sa"):   # scalars advected relative to their inlet values
        return dict(case_of(name[:-3]), scalar_advection=1)
    if name.endswith("-p"):    # the pressure-driven inlet of Sec. 4
        return dict(case_of(name[:-2]), inlet="pressure", dp_in=1e-3)
    raise KeyError(name)


def drive_key(case):
    """The inlet drive that du_in differentiates by."""
    return "dp_in" if case.get("inlet") == "pressure" else "u_in_avg"


def gpu(case, precision="fp64", mode=0):
    from paper_2103_01444_gb300.lbm import Domain
    return Domain.from_case(case, precision=precision, interface_mode=mode)


@pytest.mark.parametrize("name", ["film", "vol", "grains", "film-bv", "vol-bv", "film-p",
                                  "grains-p", "film-sa", "vol-sa", "grains-p-sa"])
@pytest.mark.parametrize("mode", [0, 1])
def test_one_step_transpose_dot_product(name, mode):
    """<lam, (step(s + e v) - step(s - e v)) / 2e> = <step^T lam, v>, and the
    same for the parameters phi, K, D_O2 and the inlet drive (u_in_avg, or
    dp_in with the pressure inlet) (FP64 storage)."""
    from paper_2103_01444_gb300.units import cathode_params
    case = case_of(name)
    d = gpu(case, mode=mode)
    d.step(25)
    s0 = d.state()
    live = (d.mask() & 3) != 3
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(s0.shape) * live
    lam_prev, g = d.vjp(lam)

    def step_from(state, fields=None, params=None):
        if params is not None:
            d.set_params(params)
        if fields is not None:
            d.set_fields(**fields)
        d.set_state(state)
        d.step(1)
        out = d.state()
        return out

    v = rng.standard_normal(s0.shape) * live * 1e-3
    eps = 1e-4
    fd = np.sum(lam * (step_from(s0 + eps * v) - step_from(s0 - eps * v))) / (2 * eps)
    ad = np.sum(lam_prev * v)
    assert abs(fd - ad) <= 1e-7 * (abs(fd) + np.abs(lam_prev * v).sum()), (fd, ad)

    # the same directional derivative from the independent FP64 oracle's step
    o_params, o_mat, o_solid = lattice_problem(case, interface_mode=mode)

    def oracle_step_from(state, material=None):
        o = Oracle(o_params, material if material is not None else o_mat, o_solid)
        o.f[...] = state[:9]
        o.g[...] = state[9:].reshape(3, 5, *state.shape[1:])
        o.step(1)
        return np.concatenate([o.f, o.g.reshape(15, *state.shape[1:])]) * live

    fdo = np.sum(lam * (oracle_step_from(s0 + eps * v) - oracle_step_from(s0 - eps * v))) / (2 * eps)
    assert abs(fdo - ad) <= 1e-7 * (abs(fdo) + np.abs(lam_prev * v).sum()), (fdo, ad)

    params, fields, _ = cathode_params(case, interface_mode=mode)
    gdl = np.zeros((case["ny"], case["nx"]), bool)
    gdl[case["ny_cl"]:case["ny_cl"] + case["ny_gdl"]] = True
    gdl &= live
    for key, gkey in (("phi", "phi"), ("K", "K"), ("D_O2", "D_O2")):
        base = fields[key]
        vv = np.where(gdl, rng.standard_normal(base.shape) * np.where(gdl, base, 0.0), 0.0)
        h = 1e-5
        fp = dict(fields, **{key: base + h * vv})
        fm = dict(fields, **{key: base - h * vv})
        # difference the states first: the temperature populations are large
        diff = step_from(s0, fields=fp) - step_from(s0, fields=fm)
        fdp = np.sum(lam * diff) / (2 * h)
        adp = np.sum(g[gkey] * vv)
        assert abs(fdp - adp) <= 1e-4 * max(abs(fdp), abs(adp), 1e-12), (key, fdp, adp)
        # the oracle keeps full values (T populations near 70 K), so its
        # central difference takes a wider step to stay above their round-off
        base_o, ho = o_mat[key], 1e-4
        diff_o = (oracle_step_from(s0, dict(o_mat, **{key: base_o + ho * vv})) -
                  oracle_step_from(s0, dict(o_mat, **{key: base_o - ho * vv})))
        fdo = np.sum(lam * diff_o) / (2 * ho)
        assert abs(fdo - adp) <= 1e-4 * max(abs(fdo), abs(adp), 1e-12), (key, fdo, adp)
    d.set_fields(**fields)
    key = drive_key(case)
    h = 1e-6 * params[key]
    diff = (step_from(s0, params=dict(params, **{key: params[key] + h})) -
            step_from(s0, params=dict(params, **{key: params[key] - h})))
    fdu = np.sum(lam * diff) / (2 * h)
    assert abs(fdu - g["u_in"]) <= 1e-4 * max(abs(fdu), 1e-12), (fdu, g["u_in"])


def tangent_direction(case, params, mat, live, rng):
    """A direction over the GDL's phi, K and D_O2 (relative to each field)
    and the inlet drive (relative to its value).  The GDL lies below the
    channel, whose clear fluid holds each scalar's largest diffusivity, so the
    direction leaves the Fickian mode's per-scalar b fixed, as the adjoint
    treats it."""
    gdl = np.zeros((case["ny"], case["nx"]), bool)
    gdl[case["ny_cl"]:case["ny_cl"] + case["ny_gdl"]] = True
    gdl &= live
    w = {k: np.where(gdl, rng.standard_normal(gdl.shape) * mat[k], 0.0)
         for k in ("phi", "K", "D_O2")}
    w["u_in"] = params[drive_key(case)]
    return w


@pytest.mark.parametrize("name", ["film", "vol", "grains", "film-bv", "vol-bv", "film-p",
                                  "grains-p", "film-sa", "vol-sa", "grains-p-sa"])
@pytest.mark.parametrize("mode", [0, 1])
def test_one_step_transpose_is_the_transpose_of_the_oracle_tangent(name, mode):
    """<lam, J w> from the oracle's own derivative of its step (its tangent:
    the step run in dual numbers) equals <J^T lam, w> from lbm_vjp, with w a
    direction in the state, phi, K, D_O2 and the inlet drive at once (FP64
    storage): the transposed step is the transpose of the oracle's step to
    rounding, not only to a finite difference's accuracy."""
    case = case_of(name)
    d = gpu(case, mode=mode)
    d.step(25)
    s0 = d.state()
    ny, nx = case["ny"], case["nx"]
    live = (d.mask() & 3) != 3
    rng = np.random.default_rng(17)
    lam = rng.standard_normal(s0.shape) * live
    lam_prev, g = d.vjp(lam)
    params, mat, solid = lattice_problem(case, interface_mode=mode)
    w = tangent_direction(case, params, mat, live, rng)
    ws = rng.standard_normal(s0.shape) * live
    t = TangentOracle(params, mat, solid, dparams={drive_key(case): w["u_in"]},
                      dmaterial={k: w[k] for k in ("phi", "K", "D_O2")})
    t.set_state(s0[:9], s0[9:].reshape(3, 5, ny, nx), ws[:9], ws[9:].reshape(3, 5, ny, nx))
    t.step(1)
    Jw = np.concatenate([t.f[..., 1], t.g[..., 1].reshape(15, ny, nx)]) * live
    lhs = np.sum(lam * Jw)
    terms = [lam_prev * ws] + [g[k] * w[k] for k in ("phi", "K", "D_O2")]
    rhs = sum(float(np.sum(x)) for x in terms) + g["u_in"] * w["u_in"]
    scale = sum(float(np.abs(x).sum()) for x in terms) + abs(g["u_in"] * w["u_in"])
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("name,mode,objective", [("film", 0, 0), ("film", 1, 1), ("vol", 1, 0),
                                                 ("grains", 0, 1), ("film-bv1", 0, 0),
                                                 ("vol-bv1", 1, 0), ("film-p", 1, 0),
                                                 ("grains-p", 1, 1), ("vol-p-sa", 1, 1)])
def test_gradient_is_the_oracle_tangent_of_the_objective(name, mode, objective):
    """lbm_grad over 40 steps (checkpoint segments of 7, records recomputed
    and kept) against the oracle's tangent through the same 40 steps from the
    same state: <grad, w> equals the objective's derivative along w, for w
    over the GDL's phi, K, D_O2 and the inlet drive, to 1e-9."""
    case = case_of(name)
    N = 40
    d = gpu(case, mode=mode)
    s0 = d.state()
    ny, nx = case["ny"], case["nx"]
    live = (d.mask() & 3) != 3
    params, mat, solid = lattice_problem(case, interface_mode=mode)
    rng = np.random.default_rng(23)
    w = tangent_direction(case, params, mat, live, rng)
    t = TangentOracle(params, mat, solid, dparams={drive_key(case): w["u_in"]},
                      dmaterial={k: w[k] for k in ("phi", "K", "D_O2")})
    t.set_state(s0[:9], s0[9:].reshape(3, 5, ny, nx))
    t.step(N)
    if objective == 0:
        Jt, dJ = t.current_density()
    else:
        T, dT = t.fields()["T"]
        xs = int(np.argmax(T[0]))
        Jt, dJ = T[0, xs], dT[0, xs]
    for limit in (-1, 0):          # records kept, and every segment recomputed
        d.set_grad_memory(limit)
        J, g = d.grad(objective, N, segment=7)
        assert J == pytest.approx(Jt, rel=1e-9)
        terms = [float(np.sum(g[k] * w[k])) for k in ("phi", "K", "D_O2")]
        terms.append(g["u_in"] * w["u_in"])
        scale = sum(float(np.abs(g[k] * w[k]).sum()) for k in ("phi", "K", "D_O2"))
        scale += abs(g["u_in"] * w["u_in"])
        assert abs(sum(terms) - dJ) <= 1e-9 * max(abs(dJ), scale), (sum(terms), dJ, scale)


def oracle_objective(case, mode, objective, N, material=None, drive=None, x_star=None):
    params, mat0, solid = lattice_problem(case, interface_mode=mode)
    base = Oracle(params, mat0, solid)          # the initial state is held fixed
    p = dict(params)
    if drive is not None:
        p[drive_key(case)] = drive
    o = Oracle(p, material if material is not None else mat0, solid)
    o.f[...] = base.f
    o.g[...] = base.g
    o.step(N)
    if objective == 0:
        return o.current_density()[0], None
    T = o.fields()["T"][0]
    xs = int(np.argmax(T)) if x_star is None else x_star
    return T[xs], xs


@pytest.mark.parametrize("name,mode,objective", [("film", 0, 0), ("film", 1, 1), ("vol", 0, 0),
                                                 ("vol", 1, 0), ("grains", 0, 1),
                                                 ("film-bv1", 0, 0), ("vol-bv1", 1, 0),
                                                 ("film-bv1", 0, 1), ("film-p", 0, 0),
                                                 ("grains-p", 1, 1), ("vol-p", 0, 0),
                                                 ("film-sa", 1, 0), ("vol-p-sa", 1, 1)])
def test_gradient_matches_oracle_finite_differences(name, mode, objective):
    """Gradients of the objective after 40 steps (checkpoint segments of 7)
    w.r.t. phi, K, D_O2 (random directions over the GDL and on single cells)
    and the inlet drive against FP64 central differences of the oracle: 1e-3
    relative."""
    case = case_of(name)
    N = 40
    d = gpu(case, mode=mode)
    J, g = d.grad(objective, N, segment=7)
    J0, xs = oracle_objective(case, mode, objective, N)
    assert J == pytest.approx(J0, rel=1e-9)
    params, mat0, _ = lattice_problem(case, interface_mode=mode)
    live = (d.mask() & 3) != 3
    gdl = np.zeros((case["ny"], case["nx"]), bool)
    gdl[case["ny_cl"]:case["ny_cl"] + case["ny_gdl"]] = True
    gdl &= live
    rng = np.random.default_rng(9)
    cells = np.argwhere(gdl)
    picks = cells[rng.choice(len(cells), 3, replace=False)]
    for key in ("phi", "K", "D_O2"):
        base = mat0[key]
        dirs = [np.where(gdl, rng.standard_normal(base.shape) * np.where(gdl, base, 0.0), 0.0)]
        for (yy, xx) in picks:
            e = np.zeros(base.shape)
            e[yy, xx] = base[yy, xx]
            dirs.append(e)
        for vv in dirs:
            # near open circuit the current is small (~1e-6 A/cm2) and the
            # oracle's central difference is in round-off below h = 3e-4; at
            # h = 1e-3 it is converged to about 3e-4 in every direction
            h = 1e-3 if "bv" in name else 1e-5
            Jp, _ = oracle_objective(case, mode, objective, N, dict(mat0, **{key: base + h * vv}),
                                     x_star=xs)
            Jm, _ = oracle_objective(case, mode, objective, N, dict(mat0, **{key: base - h * vv}),
                                     x_star=xs)
            fd = (Jp - Jm) / (2 * h)
            ad = float(np.sum(g[key] * vv))
            # directions whose effect is below the finite difference's noise
            # (about 1e-4 of J0 per unit h near open circuit) count as zero
            scale = max(abs(fd), abs(ad), (1e-3 if "bv" in name else 1e-5) * abs(J0))
            assert abs(fd - ad) <= 1e-3 * scale, (key, fd, ad)
    u0 = params[drive_key(case)]
    hu = (1e-5 if "bv" in name else 1e-6) * u0
    Jp, _ = oracle_objective(case, mode, objective, N, drive=u0 + hu, x_star=xs)
    Jm, _ = oracle_objective(case, mode, objective, N, drive=u0 - hu, x_star=xs)
    fdu = (Jp - Jm) / (2 * hu)
    assert abs(fdu - g["u_in"]) <= 1e-3 * max(abs(fdu), 1e-5 * abs(J0) / u0), (fdu, g["u_in"])


def test_fp32_adjoint_close_to_fp64():
    case = case_of("vol")
    J64, g64 = gpu(case, "fp64").grad(0, 60)
    J32, g32 = gpu(case, "fp32").grad(0, 60)
    assert J32 == pytest.approx(J64, rel=1e-4)
    for k in ("phi", "K", "D_O2"):
        err = np.linalg.norm(g32[k] - g64[k]) / np.linalg.norm(g64[k])
        assert err < 1e-3, (k, err)
    assert g32["u_in"] == pytest.approx(g64["u_in"], rel=1e-3)


def test_grad_leaves_state_and_autograd_function():
    import torch
    from paper_2103_01444_gb300.lbm import cathode_objective
    from paper_2103_01444_gb300.units import cathode_params
    case = case_of("film")
    d = gpu(case)
    d.step(10)
    s = d.state()
    d.grad(0, 20)
    np.testing.assert_array_equal(d.state(), s)
    params, fields, _ = cathode_params(case)
    phi = torch.tensor(fields["phi"], dtype=torch.float64, requires_grad=True)
    K = torch.tensor(fields["K"], dtype=torch.float64, requires_grad=True)
    D = torch.tensor(fields["D_O2"], dtype=torch.float64, requires_grad=True)
    u = torch.tensor(params["u_in_avg"], dtype=torch.float64, requires_grad=True)
    f = cathode_objective()
    J = f.apply(phi, K, D, u, d, fields, params, 0, 20, 0)
    (2.0 * J).backward()
    d2 = gpu(case)
    _, g = d2.grad(0, 20)
    np.testing.assert_allclose(phi.grad.numpy(), 2 * g["phi"], rtol=1e-12)
    np.testing.assert_allclose(D.grad.numpy(), 2 * g["D_O2"], rtol=1e-12)
    assert u.grad.item() == pytest.approx(2 * g["u_in"], rel=1e-12)


def test_autograd_on_cuda_tensors_matches_host_gradients():
    """cathode_objective on CUDA tensors: the binding passes the material and
    the gradient buffers to the library as device pointers (lbm_set_fields
    and lbm_grad with on_device = 1: no host copy of a field), and the
    per-cell gradients equal those of the host-pointer lbm_grad bit for
    bit."""
    import torch
    from paper_2103_01444_gb300.lbm import cathode_objective
    from paper_2103_01444_gb300.units import cathode_params
    case = dict(case_of("vol-p"), scalar_advection=1)
    params, fields, _ = cathode_params(case, interface_mode=1)
    dev = torch.device("cuda")
    leaf = lambda a: torch.tensor(a, dtype=torch.float64, device=dev, requires_grad=True)  # noqa
    phi, K, D = leaf(fields["phi"]), leaf(fields["K"]), leaf(fields["D_O2"])
    u = leaf(params["dp_in"])
    d = gpu(case, mode=1)
    J = cathode_objective().apply(phi, K, D, u, d, fields, params, 0, 30, 0)
    (3.0 * J).backward()
    assert J.is_cuda and phi.grad.is_cuda and D.grad.is_cuda
    J_h, g = gpu(case, mode=1).grad(0, 30)
    assert J.item() == J_h
    np.testing.assert_array_equal(phi.grad.cpu().numpy(), 3.0 * g["phi"])
    np.testing.assert_array_equal(K.grad.cpu().numpy(), 3.0 * g["K"])
    np.testing.assert_array_equal(D.grad.cpu().numpy(), 3.0 * g["D_O2"])
    # the drive gradient is an FP64 atomic sum over cells: equal to rounding
    assert u.grad.item() == pytest.approx(3.0 * g["u_in"], rel=1e-12)


@pytest.mark.parametrize("name,mode,objective,precision",
                         [("film", 0, 0, "fp64"), ("vol", 1, 1, "fp64"),
                          ("grains-p", 0, 0, "fp64"), ("vol-p-sa", 1, 0, "fp32")])
def test_stored_and_recomputed_records_give_the_same_gradient(name, mode, objective, precision):
    """The reverse sweep reads each step's records either from the forward
    sweep (stored segments) or from a recompute of the segment from its
    checkpoint: the same kernel writes both, so the gradient must not depend
    on how much memory lbm_grad may use (all stored, a few, none)."""
    case = case_of(name)
    N, seg = 45, 7
    d = gpu(case, precision, mode)
    from paper_2103_01444_gb300.lbm import LbmError
    with pytest.raises(LbmError):
        d.set_grad_memory(-2)
    ref = None
    for limit in (-1, 0, 200_000, 2_000_000, 8_000_000):
        d.set_grad_memory(limit)
        J, g = d.grad(objective, N, segment=seg)
        if ref is None:
            ref = (J, g)
            continue
        assert J == ref[0]
        for k in ("phi", "K", "D_O2"):
            np.testing.assert_array_equal(g[k], ref[1][k], err_msg=f"{k} at limit {limit}")
        # (the inlet drive's gradient is summed with FP64 atomics in any order)
        assert g["u_in"] == pytest.approx(ref[1]["u_in"], rel=1e-12)
