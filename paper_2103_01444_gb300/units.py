"""Physical cathode description -> lattice parameters and per-cell material.

Constants from arXiv 2103.01444 (Nomenclature, Eqs. 13-19); lattice scales
where the paper gives none:
  * gas viscosity nu = 0.05 (tau = 0.65) and O2 diffusivity 0.05 in lattice
    units (Schmidt number 1), H2O diffusivity 1.3 x O2, Prandtl number 0.7;
  * dx = GDL thickness / GDL rows, dt = 0.05 dx^2 / D_O2 (D_O2 = 5.2197e-2
    cm^2/s, Nomenclature);
  * solid/gas heat-capacity ratio 1500 and conductivity ratio 1.5/0.026
    (Nomenclature) in Eq. 19; the reaction heat is divided by the same
    effective heat capacity (rho_cp_ratio per cell); catalyst film 10 um;
  * c_tot = C_O2,ref / 0.21 with C_O2,ref = 17.808e-6 mol/cm^3, and a gas
    molar heat capacity of 29.3 J/(mol K);
  * Eq. 17's reference temperature 353.15 K.
"""
from __future__ import annotations

import numpy as np

PAPER = dict(
    aj0_ref=1.0e-4,        # A/cm^3 (exchange current density x area)
    C_O2_ref=17.808e-6,    # mol/cm^3
    alpha_c=1.0,
    F=96487.0,
    R=8.314,
    D_O2_cm2_s=5.2197e-2,
    k_f=0.026, k_s=1.5,    # W/(m K)
    E_act=16456.0, T_ref_kin=353.15,   # Eq. 17
    dU0dT=0.0025, U0_0=0.2329,         # Eq. 16
)

LATTICE = dict(nu=0.05, D_O2=0.05, h2o_over_o2=1.3, prandtl=0.7, heat_capacity_ratio=1500.0,
               delta_cl_cm=10e-4, gas_cp_J_molK=29.3, x_ref=0.21)


def effective_diffusivity(phi, D):
    """Bruggeman correlation, Eq. 18."""
    return D * phi ** 1.5


def effective_thermal_diffusivity(phi, alpha_gas):
    """Eq. 19 with the gas diffusivity k_f/(rho c_p)_f factored out."""
    kr = PAPER["k_s"] / PAPER["k_f"]
    cr = LATTICE["heat_capacity_ratio"]
    return alpha_gas * (phi + kr * (1.0 - phi)) / (phi + cr * (1.0 - phi))


def cathode_params(case: dict, forchheimer: int = 1, interface_mode: int = 0):
    """Returns (params dict matching lbm_params, fields dict of [ny][nx]
    float64 arrays phi, K, alpha_T, D_O2, D_H2O, geometry dict).  The
    validation cases (case["kind"]) go to validation_params."""
    if case.get("kind"):
        return validation_params(case, forchheimer, interface_mode)
    nx, ny = int(case["nx"]), int(case["ny"])
    ny_cl, ny_gdl = int(case["ny_cl"]), int(case["ny_gdl"])
    L = LATTICE
    dx = case["h_gdl_cm"] / ny_gdl
    dt = L["D_O2"] * dx ** 2 / PAPER["D_O2_cm2_s"]
    c_tot = PAPER["C_O2_ref"] / L["x_ref"]
    channel_rows = ny - ny_cl - ny_gdl
    phi = np.ascontiguousarray(case["phi"], dtype=np.float64)
    K_cm2 = np.asarray(case["K_cm2"], dtype=np.float64)
    K = np.ascontiguousarray(np.where(np.isfinite(K_cm2), K_cm2 / dx ** 2, np.inf))
    alpha_gas = L["nu"] / L["prandtl"]
    fields = dict(
        phi=phi, K=K,
        alpha_T=np.ascontiguousarray(effective_thermal_diffusivity(phi, alpha_gas)),
        D_O2=np.ascontiguousarray(effective_diffusivity(phi, L["D_O2"])),
        D_H2O=np.ascontiguousarray(effective_diffusivity(phi, L["h2o_over_o2"] * L["D_O2"])),
        rho_cp_ratio=np.ascontiguousarray(phi + LATTICE["heat_capacity_ratio"] * (1.0 - phi)),
    )
    params = dict(
        nu=L["nu"], u_in_avg=case["Re"] * L["nu"] / channel_rows, body_force_x=0.0,
        V_op=case["V_op"], T_in=case["T_in"], C_O2_in=case["C_O2_in"], C_H2O_in=case["C_H2O_in"],
        T_top=case["T_in"], C_O2_top=case["C_O2_in"], C_H2O_top=case["C_H2O_in"],
        aj0_ref=PAPER["aj0_ref"], T_ref_kin=PAPER["T_ref_kin"], E_act=PAPER["E_act"],
        alpha_c=PAPER["alpha_c"], F=PAPER["F"], R=PAPER["R"], dU0dT=PAPER["dU0dT"],
        U0_0=PAPER["U0_0"], x_ref=L["x_ref"], dx_cm=dx, dt_s=dt, delta_cl_cm=L["delta_cl_cm"],
        c_tot=c_tot, rho_cp_f=L["gas_cp_J_molK"] * c_tot, forchheimer=forchheimer,
        top_dirichlet=0, interface_mode=interface_mode,
        # the drive: inlet velocity at Re (default) or the pressure difference
        # of Sec. 4 (case["inlet"] == "pressure", excess dp_in in lattice units)
        inlet_mode=1 if case.get("inlet") == "pressure" else 0,
        dp_in=float(case.get("dp_in", 0.0)),
        # kinetics: Tafel (Eq. 13) unless an anodic transfer coefficient is
        # given for the Butler-Volmer branch
        alpha_a=float(case.get("alpha_a", 0.0)),
        # advective flux of the scalars in Eq. 10: u C as printed (0) or
        # relative to the inlet values, u (C - C_in) (1)
        scalar_advection=int(case.get("scalar_advection", 0)),
    )
    geometry = dict(nx=nx, ny=ny, ny_cl=ny_cl, ny_gdl=ny_gdl,
                    reaction_mode=int(case["reaction_mode"]),
                    periodic_x=int(case.get("periodic_x", 0)), solid=case.get("solid"))
    return params, fields, geometry


# Lattice scales of the validation cases (Sec. 3): the buoyant velocity
# scale alpha sqrt(Ra Pr) / L is held at 0.05 (Mach number about 0.09), with
# the diffusivity capped at 0.1; the heat capacity ratio is 1.
CAVITY_U = 0.05
CAVITY_ALPHA_MAX = 0.1


def _lattice_base(nx, ny, forchheimer, interface_mode, **kw):
    """lbm_params for a case given in lattice units: no drive, no reaction
    heat (V_op = U0_0), temperature-independent kinetics (E_act = alpha_c =
    0) whose lattice rate constant is aj0_ref (x_ref = 4 F c_tot = delta =
    dx = dt = 1)."""
    p = dict(nu=0.1, u_in_avg=0.0, body_force_x=0.0, V_op=0.0, T_in=343.0, C_O2_in=0.21,
             C_H2O_in=0.0, T_top=343.0, C_O2_top=0.21, C_H2O_top=0.0, aj0_ref=0.0,
             T_ref_kin=343.0, E_act=0.0, alpha_c=0.0, F=0.25, R=PAPER["R"], dU0dT=0.0, U0_0=0.0,
             x_ref=1.0, dx_cm=1.0, dt_s=1.0, delta_cl_cm=1.0, c_tot=1.0, rho_cp_f=1.0,
             forchheimer=forchheimer, top_dirichlet=0, interface_mode=interface_mode,
             inlet_mode=0, dp_in=0.0, alpha_a=0.0, buoy_gx=0.0, buoy_gy=0.0, T_buoy=343.0,
             wall_dirichlet=0, C_wall=[[0.0] * 3 for _ in range(3)], scalar_advection=0)
    p.update(kw)
    return p


def validation_params(case: dict, forchheimer: int = 1, interface_mode: int = 0):
    """The validation cases of Sec. 3 -> (params, fields, geometry), as
    cathode_params.
      cavity: L = n cells between the halfway walls, dT = T_hot - T_cold,
        alpha = min(0.1, 0.05 L / sqrt(Ra Pr)), nu = Pr alpha, and the
        buoyancy gamma = Ra nu alpha / (dT L^3) (Ra = g beta dT L^3/(nu
        alpha)); the porous cavity has K = Da L^2 and porosity phi
        everywhere; the walls hold T_hot (left, and the bottom if heated)
        and T_cold (right); T_buoy and the initial T are the mean.
      kang: k = Da D / ny on the bottom film, C0 held on the left wall."""
    nx, ny = int(case["nx"]), int(case["ny"])
    full = lambda v: np.full((ny, nx), float(v))  # noqa: E731
    sa = int(case.get("scalar_advection", 0))
    if case["kind"] == "cavity":
        L = float(nx)
        dT = case["T_hot"] - case["T_cold"]
        Tm = 0.5 * (case["T_hot"] + case["T_cold"])
        alpha = min(CAVITY_ALPHA_MAX, CAVITY_U * L / np.sqrt(case["Ra"] * case["Pr"]))
        nu = case["Pr"] * alpha
        porous = case.get("Da") is not None
        fields = dict(phi=full(case["phi"] if porous else 1.0),
                      K=full(case["Da"] * L * L if porous else np.inf),
                      alpha_T=full(alpha), D_O2=full(alpha), D_H2O=full(alpha),
                      rho_cp_ratio=full(1.0))
        bits = (1 << 0) | (1 << 3) | ((1 << 6) if case["heated_bottom"] else 0)
        wall = [[case["T_hot"], 0.21, 0.0], [case["T_cold"], 0.21, 0.0],
                [case["T_hot"], 0.21, 0.0]]
        params = _lattice_base(nx, ny, forchheimer, interface_mode, nu=nu, T_in=Tm, T_top=Tm,
                               buoy_gy=case["Ra"] * nu * alpha / (dT * L ** 3), T_buoy=Tm,
                               wall_dirichlet=bits, C_wall=wall, scalar_advection=sa)
        geometry = dict(nx=nx, ny=ny, ny_cl=0, ny_gdl=ny if porous else 0, reaction_mode=0,
                        periodic_x=0, closed_x=1, solid=None)
        return params, fields, geometry
    if case["kind"] == "kang":
        D = case["D"]
        fields = dict(phi=full(1.0), K=full(np.inf), alpha_T=full(D), D_O2=full(D),
                      D_H2O=full(D), rho_cp_ratio=full(1.0))
        params = _lattice_base(nx, ny, forchheimer, interface_mode, C_O2_in=case["C0"],
                               C_O2_top=case["C0"], aj0_ref=case["Da"] * D / ny,
                               wall_dirichlet=0b111, C_wall=[[343.0, case["C0"], 0.0],
                                                             [0.0] * 3, [0.0] * 3],
                               scalar_advection=sa)
        geometry = dict(nx=nx, ny=ny, ny_cl=0, ny_gdl=0, reaction_mode=0, periodic_x=0,
                        closed_x=1, solid=None)
        return params, fields, geometry
    raise ValueError(f"unknown case kind {case['kind']!r}")
