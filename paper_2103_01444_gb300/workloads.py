"""Seeded synthetic cathode workloads.

This module only draws inputs: lattice sizes, row splits, per-cell porosity
and permeability, solid grains and operating points.  It holds none of the
method's arithmetic (no closures, no unit mapping, no lattice constants), so
it can feed both the CUDA path and the FP64 oracle.

A workload is a plain dict:
  nx, ny, ny_cl, ny_gdl : lattice size and row split (rows from the bottom;
                          the channel takes the remaining top rows)
  reaction_mode         : 0 thin catalyst film on the bottom wall,
                          1 volumetric catalyst in the bottom ny_cl rows
  periodic_x            : 0 inlet/outlet, 1 periodic (closed-form tests)
  h_gdl_cm              : physical GDL thickness (sets the lattice spacing)
  phi                   : (ny, nx) porosity, 1 in the channel
  K_cm2                 : (ny, nx) permeability in cm^2, +inf in the channel
  solid                 : (ny, nx) uint8 pore-scale solid cells, or None
  V_op, T_in, Re        : operating point (V, K, channel Reynolds number)
  C_O2_in, C_H2O_in     : inlet mole fractions
The validation cases at the end carry kind="cavity" or kind="kang" and
their dimensionless groups instead.
"""
from __future__ import annotations

import numpy as np

# Thickness of the GDL on which the paper's Darcy numbers are based: the
# ratio K/Da of Table 2 is 6.47e-4 cm^2, i.e. h = 254.4 um.
H_GDL_CM = 254.4e-4


def _layered(nx, ny, ny_cl, ny_gdl, phi_gdl, K_gdl_cm2, phi_cl=0.4, K_cl_cm2=1e-8):
    phi = np.ones((ny, nx))
    K = np.full((ny, nx), np.inf)
    phi[ny_cl:ny_cl + ny_gdl] = phi_gdl
    K[ny_cl:ny_cl + ny_gdl] = K_gdl_cm2
    if ny_cl:
        phi[:ny_cl] = phi_cl
        K[:ny_cl] = K_cl_cm2
    return phi, K


def cathode_200x40(steps_hint: int = 5000) -> dict:
    """200 x 40 cathode: GDL rows 0-19 (phi 0.6, Da 1e-3 on the 20-row GDL),
    channel rows 20-39, parabolic inlet at Re 20, 343 K, O2 0.21, 0.6 V,
    thin-film catalyst on the bottom wall."""
    nx, ny, ny_gdl = 200, 40, 20
    dx = H_GDL_CM / ny_gdl
    K = 1e-3 * (ny_gdl * dx) ** 2
    phi, Kf = _layered(nx, ny, 0, ny_gdl, 0.6, K)
    return dict(name="cathode-200x40", nx=nx, ny=ny, ny_cl=0, ny_gdl=ny_gdl,
                reaction_mode=0, periodic_x=0, h_gdl_cm=H_GDL_CM, phi=phi, K_cm2=Kf,
                solid=None, V_op=0.6, T_in=343.0, Re=20.0, C_O2_in=0.21, C_H2O_in=0.0,
                steps=steps_hint)


def split_rows(ny: int):
    """40/55/5 % channel/GDL/catalyst split, catalyst and GDL from the bottom."""
    ny_cl = max(1, int(round(0.05 * ny)))
    ny_gdl = int(round(0.55 * ny))
    return ny_cl, ny_gdl


def cathode_blocks(nx: int = 4096, ny: int = 1024, seed: int = 210301444,
                   V_op: float = 0.5, Re: float = 50.0, T_in: float = 343.0,
                   block: int = 32) -> dict:
    """Production-shaped cathode: 40/55/5 % channel/GDL/catalyst rows, GDL
    porosity uniform in [0.4, 0.8] and permeability log-uniform in
    [1e-12, 1e-10] m^2, both drawn per block x block tile in row-major tile
    order; volumetric catalyst rows (phi 0.4, K 1e-12 m^2)."""
    ny_cl, ny_gdl = split_rows(ny)
    rng = np.random.default_rng(seed)
    bx, by = -(-nx // block), -(-ny // block)
    phi_b = rng.uniform(0.4, 0.8, size=(by, bx))
    K_b = 10.0 ** rng.uniform(-12.0, -10.0, size=(by, bx)) * 1e4  # m^2 -> cm^2
    phi_full = np.repeat(np.repeat(phi_b, block, 0), block, 1)[:ny, :nx]
    K_full = np.repeat(np.repeat(K_b, block, 0), block, 1)[:ny, :nx]
    phi, K = _layered(nx, ny, ny_cl, ny_gdl, 1.0, 1.0, phi_cl=0.4, K_cl_cm2=1e-8)
    rows = slice(ny_cl, ny_cl + ny_gdl)
    phi[rows] = phi_full[rows]
    K[rows] = K_full[rows]
    return dict(name=f"cathode-{nx}x{ny}-blocks", nx=nx, ny=ny, ny_cl=ny_cl, ny_gdl=ny_gdl,
                reaction_mode=1, periodic_x=0, h_gdl_cm=H_GDL_CM, phi=phi, K_cm2=K,
                solid=None, V_op=V_op, T_in=T_in, Re=Re, C_O2_in=0.21, C_H2O_in=0.0)


def cathode_grains(nx: int = 8192, ny: int = 2048, seed: int = 7, solid_fraction: float = 0.3,
                   grain: int = 4) -> dict:
    """Pore-scale GDL: channel on the top 40 % of rows, below it a GDL whose
    grain x grain tiles are solid with the given probability (clear fluid
    elsewhere), thin-film catalyst on the bottom wall.  Grains are kept off
    the first and the last two columns (inlet and outlet)."""
    ny_gdl = ny - int(round(0.4 * ny))
    rng = np.random.default_rng(seed)
    gx, gy = nx // grain, ny_gdl // grain
    tiles = rng.random((gy, gx)) < solid_fraction
    solid = np.zeros((ny, nx), np.uint8)
    s = np.repeat(np.repeat(tiles, grain, 0), grain, 1).astype(np.uint8)
    solid[:s.shape[0], :s.shape[1]] = s
    solid[:, :grain] = 0
    solid[:, nx - grain:] = 0
    phi = np.ones((ny, nx))
    K = np.full((ny, nx), np.inf)
    return dict(name=f"cathode-{nx}x{ny}-grains", nx=nx, ny=ny, ny_cl=0, ny_gdl=ny_gdl,
                reaction_mode=0, periodic_x=0, h_gdl_cm=H_GDL_CM, phi=phi, K_cm2=K,
                solid=solid, V_op=0.6, T_in=343.0, Re=50.0, C_O2_in=0.21, C_H2O_in=0.0)


def sweep_cases(n: int = 64, seed: int = 1444, nx_range=(512, 2048), ny_range=(128, 512),
                steps: int = 20000, re_range=(10.0, 100.0)) -> list:
    """Operating-point sweep: cell voltage U[0.3, 0.9] V, temperature
    U[333, 363] K, Re log-uniform over re_range (default [10, 100]), GDL
    permeability one of 1e-12/1e-11/1e-10 m^2, grid sizes U{nx_range} x
    U{ny_range} rounded down to multiples of 32, 40/55/5 % split, volumetric
    catalyst.  Small channels need a smaller Re to keep the inlet Mach
    number low."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1)) // 32 * 32
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1)) // 32 * 32
        V = float(rng.uniform(0.3, 0.9))
        T = float(rng.uniform(333.0, 363.0))
        Re = float(10.0 ** rng.uniform(np.log10(re_range[0]), np.log10(re_range[1])))
        Kg = float(rng.choice([1e-12, 1e-11, 1e-10])) * 1e4
        ny_cl, ny_gdl = split_rows(ny)
        phi, K = _layered(nx, ny, ny_cl, ny_gdl, 0.6, Kg, phi_cl=0.4, K_cl_cm2=1e-8)
        out.append(dict(name=f"sweep-{k}", nx=nx, ny=ny, ny_cl=ny_cl, ny_gdl=ny_gdl,
                        reaction_mode=1, periodic_x=0, h_gdl_cm=H_GDL_CM, phi=phi, K_cm2=K,
                        solid=None, V_op=V, T_in=T, Re=Re, C_O2_in=0.21, C_H2O_in=0.0,
                        steps=steps))
    return out


def small_cathode(nx: int = 64, ny: int = 16, reaction_mode: int = 0, seed: int = 3,
                  V_op: float = 0.5, Re: float = 10.0, grains: bool = False,
                  random_material: bool = True) -> dict:
    """Small cathode for parity tests: a few tiles wide with ragged edges,
    optional per-cell random porosity/permeability and optional solid grains."""
    rng = np.random.default_rng(seed)
    if reaction_mode == 1:
        ny_cl, ny_gdl = split_rows(ny)
    else:
        ny_cl, ny_gdl = 0, ny // 2
    phi, K = _layered(nx, ny, ny_cl, ny_gdl, 0.6, 1e-8)
    if random_material:
        rows = slice(ny_cl, ny_cl + ny_gdl)
        phi[rows] = rng.uniform(0.4, 0.8, size=(ny_gdl, nx))
        K[rows] = 10.0 ** rng.uniform(-12.0, -10.0, size=(ny_gdl, nx)) * 1e4
    solid = None
    if grains:
        solid = np.zeros((ny, nx), np.uint8)
        t = rng.random((ny_gdl // 2, nx // 2)) < 0.25
        s = np.repeat(np.repeat(t, 2, 0), 2, 1)
        solid[ny_cl:ny_cl + s.shape[0], :s.shape[1]] = s
        solid[:, :2] = 0
        solid[:, nx - 3:] = 0
    return dict(name=f"small-{nx}x{ny}-m{reaction_mode}", nx=nx, ny=ny, ny_cl=ny_cl,
                ny_gdl=ny_gdl, reaction_mode=reaction_mode, periodic_x=0, h_gdl_cm=H_GDL_CM,
                phi=phi, K_cm2=K, solid=solid, V_op=V_op, T_in=343.0, Re=Re, C_O2_in=0.21,
                C_H2O_in=0.0)


# ------------------------------------------------- validation workloads
# The validation cases of Sec. 3, described by their dimensionless groups
# (the paper plots them for ranges of these numbers; no lattice sizes are
# given).  Both the product and the oracle map them to lattice parameters
# with their own code.

def natural_convection_cavity(n: int = 64, Ra: float = 1e4, Pr: float = 0.71,
                              heated_bottom: bool = False, Da: float | None = None,
                              phi: float = 1.0, T_hot: float = 348.0,
                              T_cold: float = 338.0) -> dict:
    """Square cavity of n x n cells with no-slip walls all round: the left
    wall hot, the right wall cold, the top insulated; the bottom hot with
    heated_bottom (the clear-media case of Sec. 3), else insulated (the
    porous-media case, with Darcy number Da = K / L^2 and porosity phi over
    the whole cavity).  Gravity points down."""
    return dict(kind="cavity", nx=n, ny=n, Ra=float(Ra), Pr=float(Pr),
                heated_bottom=bool(heated_bottom), Da=None if Da is None else float(Da),
                phi=float(phi), T_hot=float(T_hot), T_cold=float(T_cold))


def kang_surface_reaction(nx: int = 96, ny: int = 48, Da: float = 1.0, D: float = 0.1,
                          C0: float = 0.2) -> dict:
    """Diffusion with a first-order surface reaction in a rectangle (the
    third case of Sec. 3): fluid at rest, the reactant held at C0 on the left
    wall, consumed on the bottom wall at the rate k C with Damkohler number
    Da = k ny / D, the other walls closed.  D is the lattice diffusivity."""
    return dict(kind="kang", nx=nx, ny=ny, Da=float(Da), D=float(D), C0=float(C0))
