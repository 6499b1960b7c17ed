"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, textbook definitions of the moment bases, Guo's velocity-space
forcing, closed-form steady solutions (Poiseuille, Brinkman, linear and
exponential diffusion profiles, the cosh reaction-diffusion profile) and
exact discrete invariants (stoichiometric and energy balances).
"""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from oracle.oracle import DIAG
from oracle.params import base_params, uniform_material, bruggeman, alpha_eff, lattice_problem
from paper_2103_01444_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            vals[k] = float(v)
    return vals


# Eq. 2 velocity formula, evaluated independently of the oracle's tables.
def d2q9_velocities():
    e = [(0, 0)]
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        e.append((round(math.cos(a)), round(math.sin(a))))
    for i in range(5, 9):
        a = (i - 5) * math.pi / 2 + math.pi / 4
        e.append((round(math.sqrt(2) * math.cos(a)), round(math.sqrt(2) * math.sin(a))))
    return np.array(e, float)


def matrices(L):
    M = np.zeros((9, 9)); Mi = np.zeros((9, 9)); N = np.zeros((5, 5)); Ni = np.zeros((5, 5))
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    L.orc_matrices(p(M), p(Mi), p(N), p(Ni))
    return M, Mi, N, Ni


def dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------ algebra

def test_moment_basis_matches_textbook_polynomials(oracle_lib):
    """Rows of M (Eq. 3) are the Lallemand-Luo moment polynomials of the
    Eq. 2 velocities; rows of N (Eq. 10) the D2Q5 ones."""
    M, Mi, N, Ni = matrices(oracle_lib)
    e = d2q9_velocities()
    ex, ey = e[:, 0], e[:, 1]
    e2 = ex ** 2 + ey ** 2
    rows = [np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2 ** 2, ex, (-5 + 3 * e2) * ex, ey,
            (-5 + 3 * e2) * ey, ex ** 2 - ey ** 2, ex * ey]
    np.testing.assert_array_equal(M, np.array(rows))
    e5 = e[:5]
    rows5 = [np.ones(5), e5[:, 0], e5[:, 1], -4 + 5 * (e5 ** 2).sum(1), e5[:, 0] ** 2 - e5[:, 1] ** 2]
    np.testing.assert_array_equal(N, np.array(rows5))
    np.testing.assert_allclose(M @ Mi, np.eye(9), atol=1e-14)
    np.testing.assert_allclose(N @ Ni, np.eye(5), atol=1e-14)


@pytest.mark.parametrize("phi", [1.0, 0.6, 0.4])
def test_equilibrium_consistent_with_pressure_and_velocity(oracle_lib, phi):
    """f_eq = M^-1 m_eq (Eq. 5) carries momentum rho0 u and gives back p
    through Eq. 8; the rest state f = w rho0 is the equilibrium of p = 1/(3 phi)."""
    M, Mi, _, _ = matrices(oracle_lib)
    rng = np.random.default_rng(1)
    for _ in range(5):
        p, ux, uy = 1 / (3 * phi) + 0.01 * rng.standard_normal(), *(0.05 * rng.standard_normal(2))
        meq = np.zeros(9)
        oracle_lib.orc_flow_meq(phi, p, ux, uy, dptr(meq))
        feq = Mi @ meq
        e = d2q9_velocities()
        assert abs(feq.sum() - 1.0) < 1e-14
        np.testing.assert_allclose(e.T @ feq, [ux, uy], atol=1e-14)
        p_back = 0.6 / phi * feq[1:].sum() - 6 * (ux * ux + uy * uy) / (15 * phi * phi)
        assert abs(p_back - p) < 1e-14
    meq = np.zeros(9)
    oracle_lib.orc_flow_meq(phi, 1 / (3 * phi), 0.0, 0.0, dptr(meq))
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    np.testing.assert_allclose(Mi @ meq, w, atol=1e-15)


def test_forcing_moments_equal_guo_velocity_space_forcing(oracle_lib):
    """M^-1 G equals Guo's forcing w_i rho0 [3 e.F + 9 (e.u)(e.F)/phi - 3 u.F/phi]
    (pins the sign of G7 and the form of G8, which Eq. 6 prints garbled)."""
    _, Mi, _, _ = matrices(oracle_lib)
    e = d2q9_velocities()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rng = np.random.default_rng(2)
    for _ in range(10):
        phi = rng.uniform(0.3, 1.0)
        ux, uy, Fx, Fy = 0.1 * rng.standard_normal(4)
        G = np.zeros(9)
        oracle_lib.orc_flow_G(phi, ux, uy, Fx, Fy, dptr(G))
        eu = e @ [ux, uy]
        eF = e @ [Fx, Fy]
        guo = w * (3 * eF + 9 * eu * eF / phi - 3 * (ux * Fx + uy * Fy) / phi)
        np.testing.assert_allclose(Mi @ G, guo, atol=1e-15)


def test_d2q5_equilibrium_moments_and_diffusivity(oracle_lib):
    """Sum g_eq = C, sum e g_eq = u C, sum e_x^2 g_eq = (4+b) C/10, and the
    relaxation rates of Eq. 10 with b = 20 sqrt3 alpha - 4 give diffusivity
    c_s^2 (1/s_1 - 1/2) = alpha."""
    e5 = d2q9_velocities()[:5]
    Q = np.zeros(5)
    oracle_lib.orc_scalar_Q(dptr(Q))
    for alpha in (0.005, 0.03, 0.1, 0.14):
        b = oracle_lib.orc_b_of_alpha(alpha)
        geq = np.zeros(5)
        C, ux, uy = 0.7, 0.03, -0.02
        oracle_lib.orc_d2q5_eq(C, ux, uy, b, dptr(geq))
        assert abs(geq.sum() - C) < 1e-15
        np.testing.assert_allclose(e5.T @ geq, [ux * C, uy * C], atol=1e-15)
        assert abs((e5[:, 0] ** 2) @ geq - (4 + b) * C / 10) < 1e-15
        cs2 = (4 + b) / 10
        assert abs(cs2 * (1 / Q[1] - 0.5) - alpha) < 1e-15
    # Eq. 10 rates: magic products of the flux and energy rates
    assert abs((1 / Q[1] - 0.5) * (1 / Q[3] - 0.5) - 1 / 6) < 1e-15


def test_flow_relaxation_rates(oracle_lib):
    """Sec. 2.1: s_q = 8(2 - 1/tau)/(8 - 1/tau) gives Lambda = 3/16 for any tau;
    nu = (tau - 1/2)/3."""
    for tau in (0.55, 0.65, 1.0, 1.7):
        S = np.zeros(9)
        oracle_lib.orc_flow_S(tau, dptr(S))
        assert S[1] == S[2] == S[7] == S[8] == pytest.approx(1 / tau)
        assert S[3] == S[5] == 0
        lam = (1 / S[7] - 0.5) * (1 / S[4] - 0.5)
        assert abs(lam - 3 / 16) < 1e-14


def test_implicit_velocity_solves_darcy_forchheimer(oracle_lib):
    """Eq. 8 u = v/(l0 + sqrt(l0^2 + l1 |v|)) solves v = u - F(u)/2 with the
    Eq. 7 drag F = -phi nu u/K - phi F_phi |u| u/sqrt(K)."""
    P = Oracle(base_params(4, 4), uniform_material(4, 4)).P
    rng = np.random.default_rng(3)
    for _ in range(20):
        phi = rng.uniform(0.3, 1.0)
        K = 10 ** rng.uniform(-3, 2)
        c = np.zeros(5)
        oracle_lib.orc_porous(ctypes.byref(P), phi, K, dptr(c))
        vx, vy = 0.05 * rng.standard_normal(2)
        ux = ctypes.c_double(); uy = ctypes.c_double()
        oracle_lib.orc_velocity(c[3], c[4], vx, vy, ctypes.byref(ux), ctypes.byref(uy))
        u = np.array([ux.value, uy.value])
        Fphi = 0.143 * phi ** -1.5
        F = -phi * P.nu / K * u - phi * Fphi / math.sqrt(K) * np.linalg.norm(u) * u
        np.testing.assert_allclose(u - 0.5 * F, [vx, vy], rtol=1e-13, atol=1e-16)


# ------------------------------------------------------------- closures

def test_kinetics_special_cases_and_heat_identity(oracle_lib):
    """Eq. 17 at its reference temperature returns the Nomenclature value;
    Eq. 15 with Eq. 16 reduces to Q = -j (V_op - 0.2329) at any T; a hand
    evaluation of Eqs. 13-17 at 0.6 V and 343 K."""
    gv = golden()
    P = Oracle(base_params(4, 4, aj0_ref=gv["aj0_ref_A_cm3"]), uniform_material(4, 4)).P
    assert oracle_lib.orc_aj0(ctypes.byref(P), gv["T_ref_kin_K"]) == pytest.approx(1e-4, rel=1e-15)
    for T in (323.0, 343.0, 353.0, 373.0):
        j = oracle_lib.orc_tafel_j(ctypes.byref(P), 0.21, T)
        Q = oracle_lib.orc_heat_Q(ctypes.byref(P), j, T)
        assert Q == pytest.approx(-j * (P.V_op - gv["U0_intercept_V"]), rel=1e-13)
    # hand evaluation at V = 0.6 V, T = 343 K, C = C_ref
    assert oracle_lib.orc_U0(ctypes.byref(P), 343.0) == pytest.approx(1.0904, abs=1e-12)
    assert oracle_lib.orc_eta(ctypes.byref(P), 343.0) == pytest.approx(-0.4904, abs=1e-12)
    assert oracle_lib.orc_aj0(ctypes.byref(P), 343.0) == pytest.approx(2.5185e-5, rel=2e-4)
    j = oracle_lib.orc_tafel_j(ctypes.byref(P), 0.21, 343.0)
    assert j == pytest.approx(-404.79, rel=2e-4)
    # cathodic: the rate grows as the voltage drops
    P.V_op = 0.3
    assert oracle_lib.orc_tafel_j(ctypes.byref(P), 0.21, 343.0) < j


def test_bruggeman_matches_fig5_caption_and_tables():
    """Eq. 18 at phi = 0.4 gives the Fig. 5 caption's D_O2,eff; Table 1 has one
    Re/U_avg ratio and Table 2 one K/Da ratio, the latter fixing the GDL
    thickness used by the workloads."""
    gv = golden()
    D = bruggeman(gv["phi_gdl"], gv["D_O2_cm2_s"])
    assert round(D, 4) == pytest.approx(gv["D_O2_eff_fig5_cm2_s"], abs=1e-12)
    ratios = [gv[f"table1_re{k}"] / gv[f"table1_u{k}"] for k in (1, 2, 3)]
    assert max(ratios) / min(ratios) - 1 < 5e-4
    kd = [gv[f"table2_K{k}_cm2"] / gv[f"table2_Da{k}"] for k in (1, 2, 3)]
    assert max(kd) / min(kd) - 1 < 5e-3
    assert math.sqrt(np.mean(kd)) == pytest.approx(workloads.H_GDL_CM, rel=2e-3)
    # Eq. 19: solid conduction raises, solid heat capacity lowers alpha_eff
    assert alpha_eff(1.0, 0.07) == pytest.approx(0.07)
    assert alpha_eff(0.4, 0.07) < 0.07


# ------------------------------------------------------------ geometry

def test_mask_layout():
    case = workloads.small_cathode(nx=16, ny=12, reaction_mode=1, random_material=False)
    params, material, solid = lattice_problem(case)
    o = Oracle(params, material, solid)
    m = o.mask
    ny_cl, ny_gdl = case["ny_cl"], case["ny_gdl"]
    assert (m[:ny_cl] & 3 == 2).all()
    assert (m[ny_cl:ny_cl + ny_gdl] & 3 == 1).all()
    assert (m[ny_cl + ny_gdl:] & 3 == 0).all()
    assert (m[:, 0] & 4).all() and not (m[:, 1:] & 4).any()
    assert (m[:, -1] & 8).all() and not (m[:, :-1] & 8).any()
    assert (m[-1] & 16).all() and (m[0] & 32).all()
    inlet = (m & 64) != 0
    assert inlet[ny_cl + ny_gdl:, 0].all() and inlet.sum() == case["ny"] - ny_cl - ny_gdl
    solid = np.zeros((12, 16), np.uint8)
    solid[5, 7] = 1
    o = Oracle(params, material, solid)
    near = (o.mask & 128) != 0
    assert o.mask[5, 7] & 3 == 3
    assert near.sum() == 8 and near[4:7, 6:9].sum() == 8


# ----------------------------------------------------- steady solutions

def test_rest_state_is_a_fixed_point():
    for phi, K in ((1.0, math.inf), (0.4, 0.3), (0.7, 20.0)):
        o = Oracle(base_params(6, 8), uniform_material(6, 8, phi=phi, K=K))
        f0, g0 = o.f.copy(), o.g.copy()
        o.step(50)
        np.testing.assert_allclose(o.f, f0, atol=1e-15)
        np.testing.assert_allclose(o.g, g0, rtol=1e-14)


def test_perturbations_decay():
    """Small random perturbations of the rest state die out (the mass moment
    relaxes at 1/tau; with the printed s_0 = 0 this grows without bound)."""
    o = Oracle(base_params(8, 8), uniform_material(8, 8, phi=0.8, K=2.0))
    w = o.f.copy()
    o.f = o.f + 1e-6 * np.random.default_rng(0).standard_normal(o.f.shape)
    o.step(1)
    d0 = np.abs(o.f - w).max()
    o.step(800)
    assert np.abs(o.f - w).max() < 0.05 * d0


def test_poiseuille_exact():
    """Clear channel, periodic x, bounce-back walls, body force g: the steady
    profile is g/(2 nu) y (H - y) from the halfway walls, exact up to O(u^2)."""
    nx, ny, g, nu = 4, 16, 1e-7, 0.05
    o = Oracle(base_params(nx, ny, body_force_x=g, nu=nu), uniform_material(nx, ny))
    o.step(12000)
    u = o.fields()["ux"][:, 0]
    y = np.arange(ny) + 0.5
    ex = g / (2 * nu) * y * (ny - y)
    assert np.abs(u - ex).max() / ex.max() < 1e-8


def test_pressure_driven_poiseuille_exact():
    """The paper's drive (Sec. 4): no body force, inlet pressure phi p =
    1/3 + dp at the virtual column -1, 1/3 at the virtual column nx.  The
    pressure falls linearly over nx + 1 spacings, G = dp/(nx + 1), and the
    steady profile is G/(2 nu) y (H - y) in every column, with no transverse
    velocity."""
    nx, ny, dp, nu = 10, 12, 2e-5, 0.05
    p = base_params(nx, ny, nu=nu, periodic_x=0, inlet_mode=1, dp_in=dp)
    o = Oracle(p, uniform_material(nx, ny))
    o.step(30000)
    f = o.fields()
    y = np.arange(ny) + 0.5
    ex = dp / (nx + 1) / (2 * nu) * y * (ny - y)
    for x in (0, nx // 2, nx - 1):
        assert np.abs(f["ux"][:, x] - ex).max() / ex.max() < 1e-8, x
    # transverse velocity at round-off of the populations (~1e-12 absolute)
    assert np.abs(f["uy"]).max() < 1e-7 * ex.max()
    # the pressure falls linearly between the two virtual columns
    pc = f["p"][ny // 2]
    assert np.allclose(np.diff(pc), -dp / (nx + 1), rtol=1e-6, atol=0)
    # mass balance: what enters through the inlet links equals the column
    # flux and leaves through the outlet
    d = f["diag"]
    flux = f["ux"][:, nx // 2].sum()
    assert d[DIAG["in_mass"]] == pytest.approx(flux, rel=1e-9)
    assert d[DIAG["out_mass"]] == pytest.approx(-flux, rel=1e-9)
    # the same with the inlet disabled (velocity mode, zero velocity): no flow
    o0 = Oracle(base_params(nx, ny, nu=nu, periodic_x=0, inlet_mode=0, dp_in=dp),
                uniform_material(nx, ny))
    o0.step(2000)
    assert np.abs(o0.fields()["ux"]).max() < 1e-14


def brinkman_error(H, phi=0.5):
    g, nu = 1e-6, 0.05
    K = phi * H * H / 16.0
    o = Oracle(base_params(4, H, body_force_x=g, forchheimer=0),
               uniform_material(4, H, phi=phi, K=K))
    o.step(int(14 * H * H))
    u = o.fields()["ux"][:, 0]
    y = np.arange(H) + 0.5
    r = math.sqrt(phi / K)
    ex = g * K / nu * (1 - np.cosh(r * (y - H / 2)) / np.cosh(r * H / 2))
    return np.abs(u - ex).max() / ex.max()


def test_brinkman_second_order():
    """Fully porous channel with Darcy drag (Eq. 7 without the Forchheimer
    term): u = (gK/nu)[1 - cosh(r(y - H/2))/cosh(rH/2)], r = sqrt(phi/K)."""
    e16, e32 = brinkman_error(16), brinkman_error(32)
    assert e32 < 3e-4
    assert 3.5 < e16 / e32 < 4.5


def scalar_case(H, reaction_mode=0, **kw):
    p = base_params(4, H, reaction_mode=reaction_mode, top_dirichlet=1, C_O2_top=1.0,
                    V_op=0.2329, E_act=0.0, **kw)
    return p


def test_linear_diffusion_and_surface_reaction_exact(oracle_lib):
    """No flow, Dirichlet C = 1 at the top wall, reactive bottom wall with
    rate k (Tafel, linear in C): C = C_w + (k C_w / D) y with
    C_w = 1/(1 + k H/D); k -> infinity is the linear Dirichlet profile."""
    for H, aj0, D in ((8, 1e30, 0.03), (12, 1e-4, 0.05), (12, 3e-5, 0.02)):
        p = scalar_case(H, aj0_ref=aj0)
        o = Oracle(p, uniform_material(4, H, D_O2=D))
        k = oracle_lib.orc_k_surface(ctypes.byref(o.P), 343.0)
        o.step(int(12 * H * H / D))
        C = o.fields()["C_O2"][:, 0]
        Cw = 1 / (1 + k * H / D)
        y = np.arange(H) + 0.5
        np.testing.assert_allclose(C, Cw + k * Cw / D * y, atol=1e-12)


def test_layered_diffusion_alpha_C_linear():
    """Per-cell b with a fixed Q (Eq. 10 as printed): the steady diffusive
    flux is -d(alpha C)/dy, so alpha C is linear across two layers."""
    for H in (8, 12):
        a1, a2 = 0.02, 0.05
        mat = uniform_material(4, H, D_O2=a2)
        mat["D_O2"][: H // 2] = a1
        o = Oracle(scalar_case(H, aj0_ref=1e30), mat)
        o.step(int(10 * H * H / a1))
        C = o.fields()["C_O2"][:, 0]
        y = np.arange(H) + 0.5
        np.testing.assert_allclose(mat["D_O2"][:, 0] * C, a2 * y / H, atol=1e-12)


def test_layered_diffusion_fickian_mode():
    """Fickian interface mode: one b per scalar, diffusivity through the
    flux rate, so C and the flux -alpha dC/dy are continuous: C is piecewise
    linear with slopes J/alpha_1 and J/alpha_2."""
    for H in (8, 12):
        a1, a2 = 0.02, 0.05
        mat = uniform_material(4, H, D_O2=a2)
        mat["D_O2"][: H // 2] = a1
        o = Oracle(scalar_case(H, aj0_ref=1e30, interface_mode=1), mat)
        o.step(int(10 * H * H / a1))
        C = o.fields()["C_O2"][:, 0]
        s = np.arange(H) + 0.5
        J = 1 / ((H / 2) * (1 / a1 + 1 / a2))
        ex = np.where(s < H / 2, J * s / a1, J * (H / 2) / a1 + J * (s - H / 2) / a2)
        np.testing.assert_allclose(C, ex, atol=1e-12)


def advection_profile(H, Pe, scalar_advection=0):
    a = 0.05
    mat = uniform_material(4, H, D_O2=a)
    ui = np.zeros((2, H, 4))
    ui[1] = Pe * a / H
    mat["u_imposed"] = ui
    o = Oracle(scalar_case(H, aj0_ref=1e30, scalar_advection=scalar_advection), mat)
    o.step(int(6 * H * H / a))
    return o.fields()["C_O2"][:, 0]


def advection_error(H, Pe, scalar_advection=0):
    C = advection_profile(H, Pe, scalar_advection)
    s = (np.arange(H) + 0.5) / H
    ex = (np.exp(Pe * s) - 1) / (np.exp(Pe) - 1)
    return np.abs(C - ex).max()


@pytest.mark.parametrize("scalar_advection", [0, 1])
@pytest.mark.parametrize("Pe", [4.0, -4.0])
def test_advection_diffusion_second_order(Pe, scalar_advection):
    """Uniform imposed u_y, C = 0 and 1 on the walls:
    C = (exp(Pe s) - 1)/(exp(Pe) - 1), Pe = u H/alpha; with the flux taken
    relative to the inlet value (0.21 here) too."""
    e16 = advection_error(16, Pe, scalar_advection)
    e32 = advection_error(32, Pe, scalar_advection)
    assert e32 < 2.5e-3
    assert 3.3 < e16 / e32 < 4.5


def test_relative_advection_equals_eq10_for_a_solenoidal_flow():
    """Where div u = 0 exactly (a uniform imposed velocity), advecting C or
    C - C_in gives the same discrete solution: the constant flux u C_in
    streams through unchanged."""
    for Pe in (4.0, -2.0):
        np.testing.assert_allclose(advection_profile(16, Pe, 1), advection_profile(16, Pe, 0),
                                   rtol=0, atol=1e-13)


def test_relative_advection_keeps_uniform_inlet_values():
    """A gas entering at uniform T_in and mole fractions, with no reaction,
    is a steady solution of the continuum scalar equations for any flow.
    Advected relative to the inlet values, the scalars stay exactly uniform
    through the channel and the porous layer; with the flux u C of Eq. 10 as
    printed, the small divergence of the lattice flow acts as a source
    C_in div u and moves them away from the inlet values.  (Fickian
    interfaces: with Eq. 10's per-cell b, alpha C diffuses, so a uniform C
    over a varying diffusivity is not steady.)"""
    case = workloads.small_cathode(nx=48, ny=16, reaction_mode=0)
    dev = {}
    for sa in (0, 1):
        params, material, solid = lattice_problem(dict(case, scalar_advection=sa),
                                                  interface_mode=1)
        params["aj0_ref"] = 0.0
        o = Oracle(params, material, solid).step(1500)
        fl = o.fields()
        live = (o.mask & 3) != 3
        dev[sa] = max(np.abs(fl["T"] - params["T_in"])[live].max() / params["T_in"],
                      np.abs(fl["C_O2"] - params["C_O2_in"])[live].max() / params["C_O2_in"],
                      np.abs(fl["C_H2O"])[live].max())
        assert np.abs(fl["ux"]).max() > 1e-3               # the gas does flow
    assert dev[1] < 1e-13
    assert dev[0] > 1e-6


def cosh_error(H, oracle_lib):
    D = 0.05
    p = scalar_case(H, reaction_mode=1, ny_cl=H, aj0_ref=1e-4)
    kv0 = oracle_lib.orc_k_volume(ctypes.byref(Oracle(p, uniform_material(4, H)).P), 343.0)
    p["dt_s"] *= (4.0 * D / (H * H)) / kv0
    o = Oracle(p, uniform_material(4, H, D_O2=D))
    kv = oracle_lib.orc_k_volume(ctypes.byref(o.P), 343.0)
    o.step(int(6 * H * H / D))
    C = o.fields()["C_O2"][:, 0]
    y = np.arange(H) + 0.5
    m = math.sqrt(kv / (1 + kv) / D)
    return np.abs(C - np.cosh(m * y) / np.cosh(m * H)).max()


def test_volumetric_reaction_cosh_profile(oracle_lib):
    """Catalyst rows with first-order volumetric sink, insulated bottom,
    C = 1 on top: C = cosh(m y)/cosh(m H), m = sqrt(k_eff/D), k_eff = k/(1+k)."""
    e16, e32 = cosh_error(16, oracle_lib), cosh_error(32, oracle_lib)
    assert e32 < 6e-5
    assert 3.5 < e16 / e32 < 4.5


def bv_box(mode, oracle_lib, k_target, nx=4, ny=8, alpha_a=0.5):
    """Closed periodic box at rest, insulated walls, no heat (rho_cp_f huge)
    and no Arrhenius factor: the temperature stays at T_in, eta = -0.02 V.
    The time step is scaled so that the cathodic lattice rate is k_target."""
    p = base_params(nx, ny, reaction_mode=mode, ny_cl=ny if mode else 0, V_op=0.98,
                    U0_0=1.0, dU0dT=0.0, E_act=0.0, aj0_ref=1e-4, alpha_a=alpha_a,
                    rho_cp_f=1e30)
    rate = oracle_lib.orc_k_volume if mode else oracle_lib.orc_k_surface
    k0 = rate(ctypes.byref(Oracle(p, uniform_material(nx, ny)).P), p["T_in"])
    p["dt_s"] *= k_target / k0
    return p


def nernst_equilibrium(p):
    """O2 mole fraction at which the Butler-Volmer current is zero:
    (C/C_ref) exp(-alpha_c F eta/RT) = exp(alpha_a F eta/RT)."""
    eta = p["V_op"] - (p["dU0dT"] * p["T_in"] + p["U0_0"])
    return p["x_ref"] * math.exp((p["alpha_a"] + p["alpha_c"]) * p["F"] * eta /
                                 (p["R"] * p["T_in"]))


def test_butler_volmer_volumetric_relaxation_exact(oracle_lib):
    """Butler-Volmer kinetics in a uniform catalyst box: each cell's sink is
    the backward Euler step of dC/dt = k_a - k_v C, so C_n = C* + (C_0 - C*)
    (1 + k_v)^-n exactly, and C* = k_a/k_v is the mole fraction at which the
    current of the two branches cancels."""
    p = bv_box(1, oracle_lib, 0.05)
    o = Oracle(p, uniform_material(4, 8, D_O2=0.05))
    kv = oracle_lib.orc_k_volume(ctypes.byref(o.P), p["T_in"])   # T stays T_in
    ka = oracle_lib.orc_k_volume_anodic(ctypes.byref(o.P), p["T_in"])
    Cs = nernst_equilibrium(p)
    assert ka / kv == pytest.approx(Cs, rel=1e-13)
    assert 0.01 < kv < 1 and 0.02 < Cs < 0.2
    C0 = p["C_O2_in"]
    o2 = Oracle(p, uniform_material(4, 8, D_O2=0.05))
    done = 0
    for n in (1, 7, 40):
        o2.step(n - done)
        done = n
        C = o2.g[1].sum(axis=0)        # after n sink steps (post-collision state)
        np.testing.assert_allclose(C, Cs + (C0 - Cs) * (1 + kv) ** -n, rtol=1e-13)
    # two H2O per O2 (Eq. 12) in both directions of the reaction
    np.testing.assert_allclose(o2.g[2].sum(axis=0), p["C_H2O_in"] + 2 * (C0 - C), atol=1e-14)


def test_butler_volmer_thin_film_equilibrium(oracle_lib):
    """Butler-Volmer at the reacting bottom wall of a closed box: the O2
    field relaxes to the uniform mole fraction at which the net wall current
    is zero."""
    p = bv_box(0, oracle_lib, 0.01)
    o = Oracle(p, uniform_material(4, 8, D_O2=0.05))
    o.step(40000)
    np.testing.assert_allclose(o.fields()["C_O2"], nernst_equilibrium(p), rtol=1e-10)


def test_butler_volmer_off_is_tafel():
    """alpha_a = 0 removes the anodic branch: Eq. 13 as printed."""
    case = workloads.small_cathode(nx=30, ny=12, reaction_mode=0, V_op=0.45)
    p, m, s = lattice_problem(case)
    a = Oracle(p, m, s).step(50)
    b = Oracle(dict(p, alpha_a=0.0), m, s).step(50)
    np.testing.assert_array_equal(a.g, b.g)
    c = Oracle(dict(p, alpha_a=0.5), m, s).step(50)
    assert np.abs(c.g - a.g).max() > 0


# --------------------------------------------------------------- balances

@pytest.mark.parametrize("scalar_advection", [0, 1])
@pytest.mark.parametrize("alpha_a", [0.0, 0.5])
@pytest.mark.parametrize("mode", [0, 1])
def test_closed_box_stoichiometric_and_energy_invariants(mode, alpha_a, scalar_advection,
                                                         oracle_lib):
    """Periodic x, insulated walls, reaction on: every O2 consumed makes two
    H2O (Eq. 12) and releases Eq. 15's heat, so sum(C_H2O + 2 C_O2) and
    sum(T + h C_O2) stay constant, and so does the flow mass."""
    nx, ny = 12, 10
    p = base_params(nx, ny, reaction_mode=mode, ny_cl=3 if mode else 0, V_op=0.5,
                    aj0_ref=1e-4, dt_s=2e-5, dx_cm=2e-3, body_force_x=1e-5, alpha_a=alpha_a,
                    scalar_advection=scalar_advection)
    o = Oracle(p, uniform_material(nx, ny, phi=0.6, K=1.0, D_O2=0.03, D_H2O=0.04,
                                   alpha_T=0.02))
    h = oracle_lib.orc_heat_per_O2(ctypes.byref(o.P), 343.0)
    tot = lambda: (o.g[2].sum() + 2 * o.g[1].sum(), o.g[0].sum() + h * o.g[1].sum(),  # noqa
                   o.f.sum())
    a0 = tot()
    o.step(200)
    a1 = tot()
    assert o.g[1].sum() < 0.99 * 0.21 * nx * ny  # the reaction did consume O2
    for x0, x1 in zip(a0, a1):
        assert abs(x1 - x0) <= 1e-12 * abs(x0)


@pytest.mark.parametrize("mode", [0, 1])
def test_open_cathode_balances_per_step(mode):
    """With inlet and outlet: per step, the change of each total equals the
    inflow at the inlet plus the outlet plus the reaction terms."""
    case = workloads.small_cathode(nx=40, ny=16, reaction_mode=mode, V_op=0.4)
    params, material, solid = lattice_problem(case)
    o = Oracle(params, material, solid)
    o.step(30)
    for _ in range(5):
        g0 = o.g.sum(axis=(1, 2, 3))
        o.step(1)
        d = o.diag
        g1 = o.g.sum(axis=(1, 2, 3))
        J, heat = d[DIAG["J"]], d[DIAG["heat"]]
        assert J > 0
        np.testing.assert_allclose(g1[1] - g0[1], d[DIAG["in_O2"]] + d[DIAG["out_O2"]] - J,
                                   rtol=0, atol=1e-12 * g0[1])
        np.testing.assert_allclose(g1[2] - g0[2],
                                   d[DIAG["in_H2O"]] + d[DIAG["out_H2O"]] + 2 * J,
                                   rtol=0, atol=1e-12 * max(g0[1], 1))
        np.testing.assert_allclose(g1[0] - g0[0], d[DIAG["in_T"]] + d[DIAG["out_T"]] + heat,
                                   rtol=0, atol=1e-12 * g0[0])


def test_clear_channel_inlet_outlet():
    """A clear channel fed by the parabolic inlet and left at the outlet
    pressure: the steady flow is the Poiseuille parabola with the inlet's
    flux in every column, the pressure level does not drift, and the inlet
    values of the scalars stay uniform."""
    nx, ny = 48, 12
    p = base_params(nx, ny, periodic_x=0, u_in_avg=0.02, reaction_mode=0, aj0_ref=0.0)
    o = Oracle(p, uniform_material(nx, ny, alpha_T=0.04, D_O2=0.05, D_H2O=0.06))
    o.step(9000)
    fl = o.fields()
    for k, v in (("T", 343.0), ("C_O2", 0.21)):
        np.testing.assert_allclose(fl[k], v, rtol=1e-3)
    np.testing.assert_allclose(fl["C_H2O"], 0.0, atol=1e-14)
    p0 = fl["p"].copy()
    o.step(200)
    assert np.abs(o.fields()["p"] - p0).max() < 1e-9
    flux = fl["ux"].sum(axis=0)
    assert np.abs(flux[2:-2] / flux[nx // 2] - 1).max() < 1e-6
    y = np.arange(ny) + 0.5
    par = y * (ny - y)
    u = fl["ux"][:, nx // 2]
    np.testing.assert_allclose(u / u.sum(), par / par.sum(), atol=2e-3)
    assert np.abs(fl["uy"][:, nx // 2]).max() < 1e-6


# ------------------------------------------- validation set-ups (Sec. 3)
def test_fixed_walls_conduction_exact():
    """Closed box at rest, T held at the halfway x walls, top and bottom
    insulated: the steady profile is linear between the wall values, and
    the heat through each wall is alpha dT ny / nx (the discrete flux of a
    linear profile is exact).  The same with the bottom and top held
    (bottom wall bit, top_dirichlet): linear in y.  A fixed O2 value on the
    left wall with the rest closed fills the box with that value."""
    nx, ny, a = 12, 5, 0.1
    p = base_params(nx, ny, periodic_x=0, closed_x=1, wall_dirichlet=1 | (1 << 1) | (1 << 3),
                    C_wall=[350.0, 0.3, 0.0, 340.0, 0.0, 0.0, 0.0, 0.0, 0.0], T_in=345.0)
    o = Oracle(p, uniform_material(nx, ny, alpha_T=a, D_O2=a))
    o.step(20000)
    f = o.fields()
    x = np.arange(nx) + 0.5
    assert np.abs(f["T"] - (350.0 - 10.0 * x / nx)).max() < 1e-9
    assert np.abs(f["C_O2"] - 0.3).max() < 1e-12
    assert np.abs(f["ux"]).max() == 0.0 and np.abs(f["uy"]).max() == 0.0
    d = f["diag"]
    assert d[DIAG["in_T"]] == pytest.approx(a * 10.0 * ny / nx, rel=1e-10)
    assert d[DIAG["out_T"]] == pytest.approx(-a * 10.0 * ny / nx, rel=1e-10)
    assert d[DIAG["in_mass"]] == 0.0 and abs(d[DIAG["out_mass"]]) < 1e-15
    # vertical: bottom held by the wall bit, top by top_dirichlet
    nx, ny = 4, 10
    p = base_params(nx, ny, periodic_x=1, wall_dirichlet=1 << 6, C_wall=[0.0] * 6 + [330.0, 0, 0],
                    top_dirichlet=1, T_top=350.0, T_in=345.0)
    o = Oracle(p, uniform_material(nx, ny, alpha_T=a))
    o.step(20000)
    y = np.arange(ny) + 0.5
    assert np.abs(o.fields()["T"][:, 0] - (330.0 + 20.0 * y / ny)).max() < 1e-9


def buoyant_slot(H, phi=1.0, K=math.inf):
    """Periodic slot with the bottom at Tb and the top at Tt, gravity along
    x: T is linear in y and the flow obeys nu u'' - (phi nu / K) u +
    phi gamma (T - T_buoy) = 0 with no-slip halfway walls."""
    Tb, Tt, Tr, gam, nu, a = 350.0, 340.0, 343.0, 1e-5, 0.1, 0.1
    p = base_params(4, H, periodic_x=1, wall_dirichlet=1 << 6, C_wall=[0.0] * 6 + [Tb, 0.21, 0],
                    top_dirichlet=1, T_top=Tt, T_in=345.0, nu=nu, buoy_gx=gam, T_buoy=Tr,
                    forchheimer=0)
    o = Oracle(p, uniform_material(4, H, phi=phi, K=K, alpha_T=a))
    o.step(40 * H * H)
    f = o.fields()
    s = np.arange(H) + 0.5
    G = lambda s: gam * (Tb + (Tt - Tb) * s / H - Tr)  # noqa: E731
    if math.isinf(K):
        eta = s / H
        A, B = G(0.0), gam * (Tt - Tb)
        u = H * H / nu * (A * eta * (1 - eta) / 2 + B * eta * (1 - eta ** 2) / 6)
    else:
        r = math.sqrt(phi / K)
        c1 = -(K / nu) * G(0.0)
        c2 = (-(K / nu) * G(float(H)) - c1 * math.cosh(r * H)) / math.sinh(r * H)
        u = (K / nu) * G(s) + c1 * np.cosh(r * s) + c2 * np.sinh(r * s)
    T_err = np.abs(f["T"][:, 0] - (Tb + (Tt - Tb) * s / H)).max() / (Tb - Tt)
    return np.abs(f["ux"][:, 0] - u).max() / np.abs(u).max(), T_err, np.abs(f["uy"]).max()


def test_buoyant_slot_closed_forms():
    """Boussinesq buoyancy along a periodic slot between held walls: the
    clear slot has the cubic profile (H^2/nu)[A eta(1-eta)/2 +
    B eta(1-eta^2)/6] (A = gamma (Tb - T_buoy), B = gamma (Tt - Tb)); the
    porous slot (Darcy drag, no Forchheimer) the Brinkman solution
    (K/nu) G(y) + c1 cosh(ry) + c2 sinh(ry), r = sqrt(phi/K), converging at
    second order."""
    eu, eT, uy = buoyant_slot(8)
    assert eu < 1e-4 and eT < 5e-5 and uy < 1e-6
    e8, _, _ = buoyant_slot(8, phi=0.6, K=0.6 * 8 * 8 / 16)
    e16, eT16, _ = buoyant_slot(16, phi=0.6, K=0.6 * 16 * 16 / 16)
    assert e16 < 2e-3 and eT16 < 1e-4
    assert 3.0 < e8 / e16 < 4.5


def test_cavity_point_symmetry_and_heat_balance():
    """Differentially heated cavity (left +1/2, right -1/2, top and bottom
    insulated, buoyancy gamma T along y): the set-up is invariant under the
    half turn about the centre with T -> -T and u -> -u, and so is every
    discrete step, so the state stays symmetric to round-off.  At the steady
    state the heat entering through the hot wall leaves through the cold one,
    and convection raises it above conduction (Nu > 1)."""
    n, nu, a, Ra = 12, 0.071, 0.1, 1e4
    gam = Ra * nu * a / n ** 3
    p = base_params(n, n, periodic_x=0, closed_x=1, reaction_mode=1,
                    wall_dirichlet=1 | (1 << 3), C_wall=[0.5, 0.21, 0, -0.5, 0.21, 0, 0, 0, 0],
                    T_in=0.0, nu=nu, buoy_gy=gam, T_buoy=0.0)
    o = Oracle(p, uniform_material(n, n, alpha_T=a))
    o.step(1500)
    f = o.fields()
    umax = np.abs(f["uy"]).max()
    assert umax > 1e-3
    assert np.abs(f["T"] + f["T"][::-1, ::-1]).max() < 1e-13
    assert np.abs(f["ux"] + f["ux"][::-1, ::-1]).max() < 1e-13 * umax * 1e3
    assert np.abs(f["uy"] + f["uy"][::-1, ::-1]).max() < 1e-13 * umax * 1e3
    o.step(20000)
    d = o.diag
    assert d[DIAG["in_T"]] == pytest.approx(-d[DIAG["out_T"]], rel=1e-9)
    Nu = d[DIAG["in_T"]] / (a * 1.0 * n / n)
    assert 1.2 < Nu < 4.0
    # no buoyancy: pure conduction, Nu = 1 exactly
    o0 = Oracle(dict(p, buoy_gy=0.0), uniform_material(n, n, alpha_T=a))
    o0.step(20000)
    assert o0.diag[DIAG["in_T"]] / (a * n / n) == pytest.approx(1.0, rel=1e-10)


def kang_series(nx, ny, k, D, C0, terms=80):
    """C(x, y) = C0 sum_n A_n cos(l_n (Ly - y)) cosh(l_n (Lx - x)) /
    cosh(l_n Lx): D dC/dy = k C at the bottom (l tan(l Ly) = k/D), dC/dy = 0
    at the top, C = C0 at x = 0, dC/dx = 0 at x = Lx; A_n by orthogonality.
    Coordinates from the halfway walls (cell centres at +1/2)."""
    from scipy.optimize import brentq
    Lx, Ly = float(nx), float(ny)
    lam = np.array([brentq(lambda v: v * math.tan(v * Ly) - k / D,
                           j * math.pi / Ly + 1e-12, (j + 0.5) * math.pi / Ly - 1e-12)
                    for j in range(terms)])
    A = (np.sin(lam * Ly) / lam) / (Ly / 2 + np.sin(2 * lam * Ly) / (4 * lam))
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    return C0 * sum(A[j] * np.cos(lam[j] * (Ly - Y)) * np.cosh(lam[j] * (Lx - X)) /
                    np.cosh(lam[j] * Lx) for j in range(terms))


@pytest.mark.parametrize("Da", [0.5, 4.0])
def test_kang_surface_reaction_series(Da):
    """Diffusion with first-order consumption on the bottom wall, the
    reactant held on the left wall (the surface-reaction case of Sec. 3):
    the steady field matches the separable series solution, within 1.5e-3
    of C0 away from the corner where the held wall meets the reactive one
    (the series and the lattice both resolve that corner coarsely)."""
    from paper_2103_01444_gb300 import workloads
    case = workloads.kang_surface_reaction(nx=24, ny=12, Da=Da, D=0.1, C0=0.2)
    p, mat, solid = lattice_problem(case)
    o = Oracle(p, mat, solid)
    o.step(20000)
    C = o.fields()["C_O2"]
    k = Da * 0.1 / 12
    err = np.abs(C - kang_series(24, 12, k, 0.1, 0.2)) / 0.2
    away = np.ones_like(err, bool)
    away[:2, :2] = False
    assert err[away].max() < 1.5e-3, err[away].max()
    assert err.max() < 2e-2
    # at the steady state the consumption equals what enters through the
    # held wall
    d = o.diag
    assert d[DIAG["J"]] == pytest.approx(d[DIAG["in_O2"]], rel=1e-5)


# --------------------------------------------- physical units (Eq. 13-17)
# The reaction terms are the only place where the oracle leaves lattice
# units.  These pins evaluate Eq. 13-17 by hand from the printed constants
# (tests/golden/paper_values.txt) and check the oracle's lattice rates, its
# heat per unit O2 and its current and heat outputs against Fick's and
# Fourier's laws in physical units, so that a lost factor 4 (electrons per
# O2), a misplaced catalyst thickness or a wrong dx/dt scale fails.

def hand_kinetics(V, T):
    """Eq. 13, 14, 16, 17 evaluated from the printed constants: the
    volumetric current magnitude per unit O2 mole fraction (A/cm^3)."""
    gv = golden()
    aj0 = gv["aj0_ref_A_cm3"] * math.exp(-gv["E_act_K"] * (1 / T - 1 / gv["T_ref_kin_K"]))
    U0 = gv["U0_slope_V_K"] * T + gv["U0_intercept_V"]
    eta = V - U0
    return aj0 * math.exp(-gv["alpha_c"] * gv["F_C_mol"] * eta / (gv["R_J_molK"] * T)) / 0.21


def physical_scales(dx_cm, D_lat=0.05):
    """Lattice time step that maps the lattice O2 diffusivity onto the
    printed D_O2, and the total gas concentration C_O2,ref / 0.21."""
    gv = golden()
    dt = D_lat * dx_cm ** 2 / gv["D_O2_cm2_s"]
    c_tot = gv["C_O2_ref_mol_cm3"] / 0.21
    return dt, c_tot


def test_lattice_rate_constants_hand_evaluated(oracle_lib):
    """At 0.6 V and 343 K: the film's lattice rate is the Tafel current of a
    catalyst of thickness delta per unit mole fraction, divided by the charge
    4 F c_tot per unit mole fraction and volume (Eq. 12: four electrons per
    O2), times dt/dx; the volumetric rate is the same without delta/dx; the
    heat per unit O2 consumed is 4 F c_tot (V - 0.2329)/(rho c_p)_f (Eq. 15
    with Eq. 16, whose T dU0/dT terms cancel)."""
    gv = golden()
    F = gv["F_C_mol"]
    dx = 0.05
    dt, c_tot = physical_scales(dx)
    rho_cp = 29.3 * c_tot
    delta = 10e-4
    p = base_params(4, 4, V_op=0.6, aj0_ref=gv["aj0_ref_A_cm3"], dx_cm=dx, dt_s=dt,
                    c_tot=c_tot, rho_cp_f=rho_cp, delta_cl_cm=delta)
    P = ctypes.byref(Oracle(p, uniform_material(4, 4)).P)
    j1 = hand_kinetics(0.6, 343.0)
    assert j1 * 0.21 == pytest.approx(404.79, rel=2e-4)      # A/cm^3 at C = C_ref
    k_s = j1 * delta / (4 * F * c_tot) * dt / dx
    k_v = j1 / (4 * F * c_tot) * dt
    h = 4 * F * c_tot * (0.6 - gv["U0_intercept_V"]) / rho_cp
    assert oracle_lib.orc_k_surface(P, 343.0) == pytest.approx(k_s, rel=1e-13)
    assert oracle_lib.orc_k_volume(P, 343.0) == pytest.approx(k_v, rel=1e-13)
    assert oracle_lib.orc_heat_per_O2(P, 343.0) == pytest.approx(h, rel=1e-13)
    # the same numbers written out (dx = 0.05 cm, dt = 2.3948e-3 s)
    assert k_s == pytest.approx(2.82086e-3, rel=1e-5)
    assert k_v == pytest.approx(0.141043, rel=1e-5)
    assert h == pytest.approx(4835.55, rel=1e-5)
    # the heat per unit O2 does not depend on T (Eq. 15-16)
    assert oracle_lib.orc_heat_per_O2(P, 360.0) == pytest.approx(h, rel=1e-13)


def steady_column(reaction_mode, H=16, ny_cl=0, dx=0.05, sigma=50.0, alpha_T=0.1, steps=60000):
    """A column at rest (periodic x), held at C_O2 = 0.21 and T = 343 K on the
    halfway top wall, the catalyst at the bottom (film or rows), run to its
    steady state.  Physical scales from the printed constants."""
    gv = golden()
    dt, c_tot = physical_scales(dx)
    p = base_params(4, H, reaction_mode=reaction_mode, ny_cl=ny_cl, top_dirichlet=1,
                    C_O2_top=0.21, T_top=343.0, V_op=0.6, aj0_ref=gv["aj0_ref_A_cm3"],
                    dx_cm=dx, dt_s=dt, c_tot=c_tot, rho_cp_f=29.3 * c_tot)
    m = uniform_material(4, H, alpha_T=alpha_T, D_O2=0.05, D_H2O=0.05)
    m["sigma"] = np.full((H, 4), sigma)
    o = Oracle(p, m)
    o.step(steps)
    assert o.residual() == 0.0 or o.step(1).residual() < 1e-13    # steady
    return o, dict(dx=dx, dt=dt, c_tot=c_tot, H=H, sigma=sigma, alpha_T=alpha_T)


def wall_value(col, y0, y1, y):
    """Value at height y of the line through two cells' values (cell j at
    height j + 1/2)."""
    s = (col[y1] - col[y0]) / (y1 - y0)
    return col[y0] + s * (y - (y0 + 0.5)), s


def test_thin_film_current_obeys_fick_tafel_fourier_and_eq15():
    """Steady column with the catalyst film on the bottom wall:
    - Fick: i = 4 F D_O2 c_tot (x_top - x_w)/L, with the printed D_O2;
    - Eq. 13 at the wall: i = aj0(T) delta (x_w/x_ref) exp(-alpha_c F eta/(R T));
    - Eq. 15-16: heat = i (V - 0.2329);
    - Fourier: heat = k_eff (T_w - T_top)/L, k_eff = alpha sigma (rho c_p)_f.
    All in physical units (A/cm^2, W/cm^2)."""
    gv = golden()
    o, s = steady_column(0)
    F, H, dx = gv["F_C_mol"], s["H"], s["dx"]
    L = H * dx
    fl = o.fields()
    C, T = fl["C_O2"][:, 0], fl["T"][:, 0]
    x_w, sl = wall_value(C, 0, 1, 0.0)
    x_top, _ = wall_value(C, H - 2, H - 1, H)
    assert x_top == pytest.approx(0.21, rel=1e-11)
    T_w, _ = wall_value(T, 0, 1, 0.0)
    i_avg, heat, ix = o.current_density()
    assert 0.1 < x_w / 0.21 < 0.9        # neither transport- nor kinetics-free
    assert i_avg == pytest.approx(4 * F * gv["D_O2_cm2_s"] * s["c_tot"] * (x_top - x_w) / L,
                                  rel=1e-9)
    T_c = T[0]                           # the rate takes the catalyst cell's T
    delta = 10e-4
    assert i_avg == pytest.approx(hand_kinetics(0.6, T_c) * delta * x_w, rel=1e-9)
    assert heat == pytest.approx(i_avg * (0.6 - gv["U0_intercept_V"]), rel=1e-12)
    alpha_phys = s["alpha_T"] * dx ** 2 / s["dt"]
    k_eff = alpha_phys * s["sigma"] * 29.3 * s["c_tot"]
    T_top, _ = wall_value(T, H - 2, H - 1, H)
    assert T_top == pytest.approx(343.0, rel=1e-12)
    assert heat == pytest.approx(k_eff * (T_w - T_top) / L, rel=1e-9)
    assert T_w - T_top > 1.0


def test_volumetric_current_obeys_fick_and_tafel():
    """Steady column whose bottom rows are catalyst: the current equals the
    O2 flux through the gas above them by Fick's law, and the sum over the
    catalyst rows of Eq. 13 per unit volume times the row height, at the
    backward-Euler concentration C/(1 + k_v) of each cell (k_v the lattice
    rate of the hand evaluation)."""
    gv = golden()
    ny_cl = 4
    o, s = steady_column(1, ny_cl=ny_cl)
    F, H, dx, dt, c_tot = gv["F_C_mol"], s["H"], s["dx"], s["dt"], s["c_tot"]
    fl = o.fields()
    C = fl["C_O2"][:, 0]
    _, sl = wall_value(C, ny_cl + 2, ny_cl + 5, 0.0)
    i_avg, heat, _ = o.current_density()
    assert i_avg == pytest.approx(4 * F * gv["D_O2_cm2_s"] * c_tot * sl / dx, rel=1e-9)
    mom = o.state_moments()                  # post-collision sums of the step
    i_tafel = 0.0
    for y in range(ny_cl):
        T_c, C_c = mom[2][y, 0], mom[3][y, 0]
        j1 = hand_kinetics(0.6, T_c)
        k_v = j1 / (4 * F * c_tot) * dt
        i_tafel += j1 * C_c / (1 + k_v) * dx
    assert i_avg == pytest.approx(i_tafel, rel=1e-9)
    assert heat == pytest.approx(i_avg * (0.6 - gv["U0_intercept_V"]), rel=1e-12)


# ---------------------------------------------------- residual (reading)

def test_residual_special_cases():
    """The steady-state residual max_X ||X - X_prev|| / ||X|| over
    X = (j_x, j_y, T - T_in, C_O2, C_H2O): zero for an unchanged state; a
    field scaled by 1 + a changes by a/(1 + a) of its new norm; a field that
    was zero and is not has residual 1; the largest of the five is taken;
    the snapshot is replaced on every call."""
    case = workloads.small_cathode(nx=24, ny=10, reaction_mode=0, V_op=0.4)
    params, material, solid = lattice_problem(case)
    o = Oracle(params, material, solid)
    assert o.residual() == 0.0                      # same state as at reset
    # at reset T = T_in, j = 0 and C_H2O = 0: heating by 0.5 K gives T - T_in
    # residual 1 (0.5 against 0); scaling O2 by 1.5 gives 1/3
    o.g[1] *= 1.5
    assert o.residual() == pytest.approx(1 / 3, rel=1e-14)
    o.g[0] += 0.5 * o.g[0] / o.g[0].sum(axis=0)      # T -> T + 0.5 in every cell
    assert o.residual() == pytest.approx(1.0, rel=1e-14)
    assert o.residual() == 0.0
    o.step(40)
    o.residual()
    o.g[1] *= 1.25                                  # O2: 0.2
    o.g[2] *= 1.5                                   # H2O: 1/3
    assert o.residual() == pytest.approx(1 / 3, rel=1e-13)
    # momentum: reversing the flow changes j by 2 j
    o.f[[1, 2, 3, 4, 5, 6, 7, 8]] = o.f[[3, 4, 1, 2, 7, 8, 5, 6]]
    assert o.residual() == pytest.approx(2.0, rel=1e-13)
