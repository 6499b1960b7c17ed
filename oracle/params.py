"""The oracle's own mapping from a physical cathode description to lattice
parameters (test infrastructure; independent of the product's unit helper).

Paper constants come from the Nomenclature and Eqs. 13-19 of arXiv
2103.01444.  Where the paper gives no lattice scales the readings are:
  - lattice viscosity nu = 0.05 (tau = 0.65) and lattice O2 diffusivity
    0.05 in the clear gas (Schmidt number 1);
  - dx = GDL thickness / GDL rows; dt from matching the O2 diffusivity
    D_O2 = 5.2197e-2 cm^2/s: dt = D_lat dx^2 / D_O2;
  - D_H2O = 1.3 D_O2 (not in the paper); Prandtl number 0.7 in the gas;
  - (rho c_p)_s / (rho c_p)_f = 1500; k_s/k_f = 1.5/0.026 (Nomenclature);
    the reaction heat enters the temperature equation divided by the
    effective heat capacity of Eq. 19, like the conduction does;
  - catalyst film thickness 10 um; total gas concentration
    c_tot = C_O2,ref / 0.21 (C_O2,ref read as mol/cm^3);
    (rho c_p)_f = 29.3 J/(mol K) * c_tot;
  - Eq. 17's reference temperature is taken as 353.15 K.
"""
from __future__ import annotations

import math

import numpy as np

# Nomenclature and Eqs. 13-17
AJ0_REF = 1e-4            # A/cm^3
C_O2_REF_MOLAR = 17.808e-6  # mol/cm^3
ALPHA_C = 1.0
FARADAY = 96487.0
R_GAS = 8.314
D_O2_PHYS = 5.2197e-2     # cm^2/s
K_FLUID = 0.026           # W/(m K)
K_SOLID = 1.5             # W/(m K)
E_ACT = 16456.0           # K (Eq. 17)
T_REF_KIN = 353.15        # K (Eq. 17)
DU0_DT = 0.0025           # V/K (Eq. 16)
U0_0 = 0.2329             # V (Eq. 16)
X_REF = 0.21

# Readings for the lattice scales
NU_LAT = 0.05
D_O2_LAT = 0.05
D_H2O_RATIO = 1.3
PRANDTL = 0.7
RHOCP_RATIO = 1500.0
DELTA_CL_CM = 10e-4
C_TOT = C_O2_REF_MOLAR / X_REF
RHO_CP_F = 29.3 * C_TOT


def bruggeman(phi, D):
    """Eq. 18: effective diffusivity of the porous layer."""
    return np.power(phi, 1.5) * D


def alpha_eff(phi, alpha_f, ks_over_kf=K_SOLID / K_FLUID, rc=RHOCP_RATIO):
    """Eq. 19 divided through by (rho c_p)_f: thermal diffusivity of the
    porous layer from the gas diffusivity alpha_f = k_f/(rho c_p)_f."""
    return alpha_f * (phi + (1.0 - phi) * ks_over_kf) / (phi + (1.0 - phi) * rc)


def heat_capacity_ratio(phi, rc=RHOCP_RATIO):
    """(rho c_p)_eff / (rho c_p)_f of Eq. 19."""
    return phi + (1.0 - phi) * rc


def lattice_problem(case: dict, forchheimer: int = 1, interface_mode: int = 0):
    """Physical workload dict -> (params dict, material dict, solid); the
    validation cases of Sec. 3 (case["kind"]) go to validation_problem."""
    if case.get("kind"):
        return validation_problem(case, forchheimer, interface_mode)
    nx, ny = case["nx"], case["ny"]
    ny_cl, ny_gdl = case["ny_cl"], case["ny_gdl"]
    dx = case["h_gdl_cm"] / ny_gdl
    dt = D_O2_LAT * dx * dx / D_O2_PHYS
    h_ch = ny - ny_cl - ny_gdl
    phi = np.asarray(case["phi"], np.float64)
    Kc = np.asarray(case["K_cm2"], np.float64)
    K_lat = np.where(np.isinf(Kc), np.inf, Kc / (dx * dx))
    alpha_f = NU_LAT / PRANDTL
    material = dict(
        phi=phi, K=K_lat,
        alpha_T=alpha_eff(phi, alpha_f),
        D_O2=bruggeman(phi, D_O2_LAT),
        D_H2O=bruggeman(phi, D_H2O_RATIO * D_O2_LAT),
        sigma=heat_capacity_ratio(phi),
    )
    params = dict(
        nx=nx, ny=ny, ny_cl=ny_cl, ny_gdl=ny_gdl, reaction_mode=case["reaction_mode"],
        periodic_x=case.get("periodic_x", 0), forchheimer=forchheimer, top_dirichlet=0,
        interface_mode=interface_mode,
        nu=NU_LAT, u_in_avg=case["Re"] * NU_LAT / h_ch, body_force_x=0.0,
        V_op=case["V_op"], T_in=case["T_in"], C_O2_in=case["C_O2_in"],
        C_H2O_in=case["C_H2O_in"], T_top=case["T_in"], C_O2_top=case["C_O2_in"],
        C_H2O_top=case["C_H2O_in"],
        aj0_ref=AJ0_REF, T_ref_kin=T_REF_KIN, E_act=E_ACT, alpha_c=ALPHA_C, F=FARADAY,
        R=R_GAS, dU0dT=DU0_DT, U0_0=U0_0, x_ref=X_REF,
        dx_cm=dx, dt_s=dt, delta_cl_cm=DELTA_CL_CM, c_tot=C_TOT, rho_cp_f=RHO_CP_F,
        # drive of the flow: a parabolic inlet velocity at Re (default), or
        # the paper's pressure difference (Sec. 4): phi p = 1/3 + dp_in at
        # the inlet, 1/3 at the outlet, dp_in in lattice units
        inlet_mode=1 if case.get("inlet") == "pressure" else 0,
        dp_in=float(case.get("dp_in", 0.0)),
        # kinetics: Tafel (Eq. 13) unless the case gives an anodic transfer
        # coefficient for the Butler-Volmer branch
        alpha_a=float(case.get("alpha_a", 0.0)),
        # advective flux of the scalars: u C as printed in Eq. 10 (0), or
        # relative to the inlet values, u (C - C_in) (1)
        scalar_advection=int(case.get("scalar_advection", 0)),
    )
    return params, material, case.get("solid")


def base_params(nx, ny, **kw):
    """Parameter dict for the closed-form tests (no reaction by default)."""
    p = dict(nx=nx, ny=ny, ny_cl=0, ny_gdl=0, reaction_mode=0, periodic_x=1, forchheimer=1,
             top_dirichlet=0, interface_mode=0, nu=NU_LAT, u_in_avg=0.0, body_force_x=0.0, V_op=0.6,
             T_in=343.0, C_O2_in=0.21, C_H2O_in=0.0, T_top=343.0, C_O2_top=0.21,
             C_H2O_top=0.0, aj0_ref=0.0, T_ref_kin=T_REF_KIN, E_act=E_ACT, alpha_c=ALPHA_C,
             F=FARADAY, R=R_GAS, dU0dT=DU0_DT, U0_0=U0_0, x_ref=X_REF, dx_cm=1e-3,
             dt_s=1e-6, delta_cl_cm=DELTA_CL_CM, c_tot=C_TOT, rho_cp_f=RHO_CP_F,
             inlet_mode=0, dp_in=0.0, alpha_a=0.0, closed_x=0, wall_dirichlet=0, buoy_gx=0.0,
             buoy_gy=0.0, T_buoy=343.0, C_wall=[0.0] * 9, scalar_advection=0)
    p.update(kw)
    return p


def uniform_material(nx, ny, phi=1.0, K=math.inf, alpha_T=0.05, D_O2=0.05, D_H2O=0.05):
    full = lambda v: np.full((ny, nx), float(v))  # noqa: E731
    return dict(phi=full(phi), K=full(K), alpha_T=full(alpha_T), D_O2=full(D_O2),
                D_H2O=full(D_H2O))


# Readings for the validation cases (Sec. 3 gives only their dimensionless
# groups): the buoyant velocity scale alpha sqrt(Ra Pr)/L is 0.05 in lattice
# units, alpha at most 0.1; sigma = 1.
BUOYANT_VELOCITY = 0.05
ALPHA_CAP = 0.1


def validation_problem(case: dict, forchheimer: int = 1, interface_mode: int = 0):
    """Cavity (natural convection, clear or porous) and Kang's surface
    reaction -> (params, material, solid).

    Cavity of side L = n cells (walls halfway outside the end cells):
    Ra = g beta dT L^3 / (nu alpha) and Pr = nu / alpha fix
    gamma = g beta = Ra nu alpha / (dT L^3); Da = K / L^2 in the porous
    cavity.  Left wall T_hot, right wall T_cold, bottom T_hot when heated,
    the rest insulated; gravity along -y, so the buoyancy per unit mass is
    +gamma (T - T_mean) along y.

    Kang: fluid at rest, C0 on the left wall, first-order consumption
    k C_w on the bottom wall with Da = k ny / D.  The kinetics are made
    linear and heat-free: no activation energy, alpha_c = 0, V = U0, and
    unit scales so that the film's lattice rate is aj0_ref."""
    nx, ny = case["nx"], case["ny"]
    p = base_params(nx, ny, periodic_x=0, closed_x=1, reaction_mode=0,
                    forchheimer=forchheimer, interface_mode=interface_mode,
                    E_act=0.0, alpha_c=0.0, dU0dT=0.0, U0_0=0.0, V_op=0.0, T_ref_kin=343.0,
                    x_ref=1.0, F=0.25, c_tot=1.0, delta_cl_cm=1.0, dx_cm=1.0, dt_s=1.0,
                    rho_cp_f=1.0, scalar_advection=int(case.get("scalar_advection", 0)))
    ones = np.ones((ny, nx))
    if case["kind"] == "cavity":
        L = float(nx)
        hot, cold = case["T_hot"], case["T_cold"]
        mean = 0.5 * (hot + cold)
        Ra, Pr = case["Ra"], case["Pr"]
        alpha = min(ALPHA_CAP, BUOYANT_VELOCITY * L / math.sqrt(Ra * Pr))
        nu = Pr * alpha
        p.update(nu=nu, T_in=mean, T_top=mean, buoy_gx=0.0, buoy_gy=Ra * nu * alpha / ((hot - cold) * L ** 3),
                 T_buoy=mean, C_O2_in=0.21, C_H2O_in=0.0,
                 wall_dirichlet=1 | (1 << 3) | ((1 << 6) if case["heated_bottom"] else 0),
                 C_wall=[hot, 0.21, 0.0, cold, 0.21, 0.0, hot, 0.21, 0.0])
        if case.get("Da") is not None:
            p["ny_gdl"] = ny
            mat = dict(phi=case["phi"] * ones, K=case["Da"] * L * L * ones)
        else:
            mat = dict(phi=ones, K=np.full((ny, nx), np.inf))
        mat.update(alpha_T=alpha * ones, D_O2=alpha * ones, D_H2O=alpha * ones, sigma=ones)
        return p, mat, None
    if case["kind"] == "kang":
        D = case["D"]
        p.update(nu=0.1, T_in=343.0, C_O2_in=case["C0"], C_O2_top=case["C0"], C_H2O_in=0.0,
                 aj0_ref=case["Da"] * D / ny, wall_dirichlet=0b111,
                 C_wall=[343.0, case["C0"], 0.0] + [0.0] * 6)
        mat = dict(phi=ones, K=np.full((ny, nx), np.inf), alpha_T=D * ones, D_O2=D * ones,
                   D_H2O=D * ones, sigma=ones)
        return p, mat, None
    raise ValueError(case["kind"])
