/*
 * FP64 CPU oracle of the coupled lattice-Boltzmann PEMFC-cathode time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it is used by the tests, by the package smoke check and by
 * the benchmark's CPU-baseline leg, nowhere else.  It shares no code, header,
 * table or constant with the CUDA library.
 *
 * What it computes, in the paper's order and notation (arXiv 2103.01444):
 *   stream  : f_i(x, t+1) <- f*_i(x - e_i, t)               (Eq. 1 LHS, Eq. 2)
 *             g_i(x, t+1) <- g*_i(x - e_i, t)               (Eq. 9, Eq. 10 LHS)
 *             with the boundary links of Sec. 4 (bounce-back walls, inlet,
 *             outlet, catalyst-layer reaction, Eq. 12-17)
 *   macros  : v = sum e_i f_i / rho0, u = v / (l0 + sqrt(l0^2 + l1 |v|)),
 *             p = (0.6/phi) sum_{i>=1} f_i - 6 rho0 |u|^2 / (15 phi^2)  (Eq. 8)
 *             C = sum_i g_i                                          (Eq. 11)
 *   collide : m = M f;  m* = m - S (m - m_eq) + (I - S/2) G;  f* = M^-1 m*
 *                                                             (Eq. 1, 3-7)
 *             n = N g;  n* = n - Q (n - n_eq);  g* = N^-1 n*  (Eq. 10)
 *             + volumetric catalyst sink when the catalyst layer has rows.
 *   outputs : current density and heat of the reaction links (Eq. 13, 15)
 *             and the steady-state residual of the moments (orc_residual).
 *
 * Readings taken where the paper is silent or garbled (each listed in the
 * design notes):
 *   - Eq. 6 prints G7 with a minus sign and G8 = (ux Fx + uy Fy)/phi; the
 *     moments of Guo's velocity-space forcing give G7 = +2 rho0 (ux Fx -
 *     uy Fy)/phi and G8 = rho0 (ux Fy + uy Fx)/phi.  The derived form is used.
 *   - The inlet carries a parabolic velocity (Ladd moving-wall bounce-back,
 *     velocity taken where the link crosses the inlet plane) over the
 *     channel rows; GDL/CL rows at the inlet are walls.  Scalars:
 *     anti-bounce-back Dirichlet at the inlet channel rows.
 *   - Pressure inlet (inlet_mode 1, the drive of Sec. 4): the channel rows
 *     pull from a virtual column -1 that repeats column 0 with its
 *     equilibrium pressure part moved to phi p = rho0/3 + dp_in.
 *   - Outlet: fully developed (the virtual column nx repeats column nx-1);
 *     for the flow, the virtual cell's equilibrium pressure part is moved to
 *     the specified outlet pressure phi p = rho0/3 (Sec. 5), which anchors
 *     the pressure level.
 *   - The mass moment relaxes at s_0 = 1/tau, like e and zeta: the printed S
 *     has s_0 = 0, with which sum_{i>=1} f_i (the pressure invariant of the
 *     incompressible equilibrium of Eq. 5/8) is not conserved and the scheme
 *     is linearly unstable.
 *   - Surface reaction (thin catalyst film at y = -1/2): the Tafel rate is
 *     linear in C, J = k(T) C_w with C_w = (g_down* + g_up)/(2 w), solved
 *     implicitly: g_up = g_down* (1 - kappa)/(1 + kappa), kappa = k/(2w).
 *     Water gets +2J (Eq. 12); temperature gets the heat of Eq. 15.
 *   - Volumetric catalyst rows: backward-Euler sink S = -k_v C/(1 + k_v),
 *     added after collision as w_i(b) S.
 *   - Butler-Volmer (alpha_a > 0): an anodic branch aj0(T) exp(alpha_a F
 *     eta/(RT)) at unit reactant activity is subtracted from the O2 flux,
 *     J = k C_w - k_a; the implicit link becomes g_up = (g_down* (1 - kappa)
 *     + k_a)/(1 + kappa), the sink S = (k_va - k_v C)/(1 + k_v).
 *   - k(T), C and T in the reaction terms use the cell's previous
 *     post-collision sums (C^n = sum g*(x)).
 *   - Optionally (scalar_advection 1) the flux moments of the D2Q5
 *     equilibria carry u (C - C_in) instead of u C: the same continuum
 *     equation where div u = 0, without the source C_in div u that the weakly
 *     compressible flow's small divergence would add.
 *   - Eq. 10 with a per-cell b and fixed Q (the default) diffuses alpha C,
 *     so alpha C, not C, is continuous across the GDL/channel interface; an
 *     optional Fickian interface mode keeps one b per scalar and sets each
 *     cell's diffusivity through the flux-moment rate instead.
 *   - The validation cases of Sec. 3: closed x ends (no-slip walls), scalars
 *     held at fixed values on walls by anti-bounce-back at the halfway wall,
 *     and the Boussinesq buoyancy gamma (T - T_buoy) added like the uniform
 *     body force (half a step in Eq. 8's velocity, times phi in the force),
 *     with T the cell's post-stream sum.
 *
 * Storage: f[q][y][x] (9 planes), g[s][q][y][x] (3 scalars x 5 planes),
 * s = 0 temperature, 1 O2 mole fraction, 2 H2O mole fraction.  Full values,
 * never deviations.  Built with plain gcc, no fast-math.  Every real number
 * has the type `real` (double here; see below).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The arithmetic type.  This file is plain C in double precision; the
 * oracle's tangent (lbm_oracle_tangent.cc) compiles the same source as C++
 * with `real` a forward-mode dual number, a value and its derivative along
 * one direction of the inputs, and defines ORC_REAL_DEFINED. */
#ifndef ORC_REAL_DEFINED
typedef double real;
#endif

/* ---------------------------------------------------------------- lattices */

/* D2Q9 velocity set, Eq. 2: rest, four axis links, four diagonals. */
static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const real W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* D2Q5 velocity set, Eq. 9. */
static const int EX5[5] = {0, 1, 0, -1, 0};
static const int EY5[5] = {0, 0, 1, 0, -1};

/* Transformation matrix M, Eq. 3. */
static const real M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

/* Transformation matrix N, Eq. 10. */
static const real N5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1}};

static int opposite9(int i) {
  for (int j = 0; j < 9; ++j)
    if (EX9[j] == -EX9[i] && EY9[j] == -EY9[i]) return j;
  return -1;
}
static int opposite5(int i) {
  for (int j = 0; j < 5; ++j)
    if (EX5[j] == -EX5[i] && EY5[j] == -EY5[i]) return j;
  return -1;
}

/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix. */
static int invert(int n, const real *a, real *inv) {
  real w[9 * 18];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c)
      w[r * 2 * n + c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(w[r * 2 * n + c]) > fabs(w[piv * 2 * n + c])) piv = r;
    if (fabs(w[piv * 2 * n + c]) < 1e-12) return -1;
    if (piv != c)
      for (int k = 0; k < 2 * n; ++k) {
        real t = w[c * 2 * n + k];
        w[c * 2 * n + k] = w[piv * 2 * n + k];
        w[piv * 2 * n + k] = t;
      }
    real d = w[c * 2 * n + c];
    for (int k = 0; k < 2 * n; ++k) w[c * 2 * n + k] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      real s = w[r * 2 * n + c];
      for (int k = 0; k < 2 * n; ++k) w[r * 2 * n + k] -= s * w[c * 2 * n + k];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) inv[r * n + c] = w[r * 2 * n + n + c];
  return 0;
}

static real MINV9[9][9];
static real NINV5[5][5];
static int g_inverted = 0;

static void ensure_inverses(void) {
  if (g_inverted) return;
  invert(9, &M9[0][0], &MINV9[0][0]);
  invert(5, &N5[0][0], &NINV5[0][0]);
  g_inverted = 1;
}

/* ------------------------------------------------------------- problem */

/* Operating point, constants and flags (lattice units unless noted). */
typedef struct {
  int32_t nx, ny;
  int32_t ny_cl, ny_gdl;    /* rows counted from the bottom (y = 0) */
  int32_t reaction_mode;    /* 0 thin-film surface at y=-1/2, 1 volumetric CL rows */
  int32_t periodic_x;       /* 1: x wraps (closed-form tests), 0: inlet/outlet */
  int32_t forchheimer;      /* 1: Eq. 7 with the Forchheimer term, 0: Darcy only */
  int32_t top_dirichlet;    /* scalars at the top wall: 0 insulated, 1 Dirichlet */
  int32_t interface_mode;   /* 0: per-cell b, fixed Q (Eq. 10 as printed);
                               1: Fickian: one b per scalar, per-cell flux rate */
  int32_t inlet_mode;       /* 0: parabolic velocity inlet; 1: pressure inlet (Sec. 4) */
  int32_t closed_x;         /* 1: no-slip walls at both x ends (the cavities of Sec. 3) */
  int32_t wall_dirichlet;   /* bit 3k+s: scalar s held at C_wall[3k+s] on wall k
                               (0 the x = 0 end outside inlet rows, 1 the x = nx-1 end,
                               2 the bottom); otherwise insulated */
  real nu;                /* kinematic viscosity; 3 nu = tau - 1/2 (Eq. 8) */
  real u_in_avg;          /* mean inlet velocity over the channel rows */
  real body_force_x;      /* uniform body force per unit mass (tests only) */
  real V_op, T_in, C_O2_in, C_H2O_in;
  real T_top, C_O2_top, C_H2O_top;
  real aj0_ref;           /* A/cm^3 at T_ref_kin (Eq. 13, 17) */
  real T_ref_kin, E_act;  /* 353.15 K, 16456 K (Eq. 17) */
  real alpha_c, F, R;     /* Eq. 13 */
  real dU0dT, U0_0;       /* Eq. 16 */
  real x_ref;             /* reference O2 mole fraction (C_O2,ref) */
  real dx_cm, dt_s, delta_cl_cm, c_tot, rho_cp_f;
  real dp_in;             /* pressure inlet: phi p there is rho0/3 + dp_in */
  real alpha_a;           /* anodic transfer coefficient of the Butler-Volmer
                               branch; 0 = Tafel kinetics, Eq. 13 as printed */
  real buoy_gx, buoy_gy;  /* Boussinesq buoyancy of the natural-convection cases
                               (Sec. 3): force per unit mass (buoy_gx, buoy_gy)(T - T_buoy) */
  real T_buoy;
  real C_wall[9];         /* wall values of wall_dirichlet, [wall][scalar] */
  int32_t scalar_advection; /* flux moments of the D2Q5 equilibria (Eq. 10):
                               0 u C as printed; 1 u (C - C_in), relative to the
                               scalar's inlet value */
} orc_params;

/* Per-cell material, lattice units. K = +inf marks clear fluid.  sigma is
 * (rho c_p)_eff / (rho c_p)_f of Eq. 19 (NULL = 1): the reaction heat enters
 * the temperature equation, whose diffusivity is k_eff/(rho c_p)_eff,
 * divided by the same effective heat capacity. */
typedef struct {
  const real *phi, *K, *alpha_T, *D_O2, *D_H2O;
  const real *u_imposed; /* optional [2][ny][nx]: freeze flow (tests) */
  const real *sigma;     /* optional [ny][nx] heat-capacity ratio */
} orc_material;

/* Mask bits (one byte per cell). */
enum {
  REG_CLEAR = 0, REG_POROUS = 1, REG_CATALYST = 2, REG_SOLID = 3,
  B_XLO = 1 << 2, B_XHI = 1 << 3, B_YHI = 1 << 4, B_YLO = 1 << 5,
  B_INLET = 1 << 6, B_NEAR_SOLID = 1 << 7
};

#define IDX(x, y) ((size_t)(y) * (size_t)nx + (size_t)(x))

/* Node types from the geometry: rows [0, ny_cl) catalyst (volumetric mode),
 * [ny_cl, ny_cl + ny_gdl) porous GDL, the rest clear channel; explicit
 * solid cells override.  Boundary bits follow the cell's position. */
void orc_build_mask(const orc_params *P, const uint8_t *solid, uint8_t *mask) {
  int nx = P->nx, ny = P->ny;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int reg;
      if (solid && solid[IDX(x, y)]) reg = REG_SOLID;
      else if (y < P->ny_cl) reg = REG_CATALYST;
      else if (y < P->ny_cl + P->ny_gdl) reg = REG_POROUS;
      else reg = REG_CLEAR;
      uint8_t m = (uint8_t)reg;
      if (x == 0) m |= B_XLO;
      if (x == nx - 1) m |= B_XHI;
      if (y == ny - 1) m |= B_YHI;
      if (y == 0) m |= B_YLO;
      if (reg == REG_CLEAR && x == 0 && !P->periodic_x && !P->closed_x) m |= B_INLET;
      mask[IDX(x, y)] = m;
    }
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if ((mask[IDX(x, y)] & 3) == REG_SOLID) continue;
      for (int i = 1; i < 9; ++i) {
        int sx = x - EX9[i], sy = y - EY9[i];
        if (sy < 0 || sy >= ny) continue;
        if (P->periodic_x) sx = (sx + nx) % nx;
        if (sx < 0 || sx >= nx) continue;
        if ((mask[IDX(sx, sy)] & 3) == REG_SOLID) mask[IDX(x, y)] |= B_NEAR_SOLID;
      }
    }
}

/* ------------------------------------------------------- closures (Sec. 4) */

/* Eq. 16 */
real orc_U0(const orc_params *P, real T) { return P->dU0dT * T + P->U0_0; }
/* Eq. 14 */
real orc_eta(const orc_params *P, real T) { return P->V_op - orc_U0(P, T); }
/* Eq. 17 */
real orc_aj0(const orc_params *P, real T) {
  return P->aj0_ref * exp(-P->E_act * (1.0 / T - 1.0 / P->T_ref_kin));
}
/* Eq. 13: volumetric current density (A/cm^3, negative = cathodic) at O2
 * mole fraction x and temperature T. */
real orc_tafel_j(const orc_params *P, real x, real T) {
  return -orc_aj0(P, T) * (x / P->x_ref) *
         exp(-P->alpha_c * P->F / (P->R * T) * orc_eta(P, T));
}
/* Anodic branch of Butler-Volmer kinetics, the reverse of Eq. 12 (water
 * oxidation), taken at unit reactant activity: aj0(T) exp(alpha_a F eta/(RT))
 * in A/cm^3; zero when alpha_a = 0 (Tafel, Eq. 13 alone).  The full current
 * is j = orc_tafel_j + orc_anodic_j. */
real orc_anodic_j(const orc_params *P, real T) {
  if (P->alpha_a == 0.0) return 0.0;
  return orc_aj0(P, T) * exp(P->alpha_a * P->F / (P->R * T) * orc_eta(P, T));
}
/* Eq. 15: heat per unit volume (W/cm^3) released by current j at T. */
real orc_heat_Q(const orc_params *P, real j, real T) {
  return -j * (orc_eta(P, T) + T * P->dU0dT);
}

/* Lattice rate constant of the thin film: O2 mole-fraction flux per step
 * through one wall link, per unit wall mole fraction. */
static real k_surface(const orc_params *P, real T) {
  real j1 = -orc_tafel_j(P, P->x_ref, T) / P->x_ref; /* A/cm^3 per unit x */
  real flux = j1 * P->delta_cl_cm / (4.0 * P->F * P->c_tot); /* cm/s */
  return flux * P->dt_s / P->dx_cm;
}
/* Lattice rate of the volumetric catalyst: fraction of O2 per step. */
static real k_volume(const orc_params *P, real T) {
  real j1 = -orc_tafel_j(P, P->x_ref, T) / P->x_ref;
  return j1 / (4.0 * P->F * P->c_tot) * P->dt_s;
}
/* The anodic branch as O2 mole fraction produced per step: through one
 * wall link of the thin film, and per cell of the volumetric catalyst. */
static real k_surface_anodic(const orc_params *P, real T) {
  return orc_anodic_j(P, T) * P->delta_cl_cm / (4.0 * P->F * P->c_tot) * P->dt_s / P->dx_cm;
}
static real k_volume_anodic(const orc_params *P, real T) {
  return orc_anodic_j(P, T) / (4.0 * P->F * P->c_tot) * P->dt_s;
}
/* Temperature rise (K) per unit of O2 mole fraction consumed, Eq. 15 with
 * j = -4 F c_tot (consumed flux). */
static real heat_per_O2(const orc_params *P, real T) {
  return 4.0 * P->F * P->c_tot * (orc_eta(P, T) + T * P->dU0dT) / P->rho_cp_f;
}

/* ------------------------------------------------- moment-space pieces */

/* b of Eq. 10 for diffusivity alpha */
real orc_b_of_alpha(real alpha) { return 20.0 * sqrt(3.0) * alpha - 4.0; }

/* D2Q5 coefficients of one cell and scalar: the b of its equilibrium and
 * the relaxation rate of the flux moments.  Eq. 10 as printed sets b from
 * the cell's own diffusivity with the fixed rate 6/(3 + sqrt 3).  In the
 * Fickian interface mode every cell takes the b of the largest diffusivity
 * of that scalar (alpha_max) and the cell's diffusivity enters through the
 * flux rate instead: alpha = c_s^2 (1/s_1 - 1/2), c_s^2 = (4 + b)/10. */
typedef struct { real b, q1; } scalar_coef;
static scalar_coef scalar_coefficients(const orc_params *P, real alpha, real alpha_max) {
  scalar_coef r;
  if (P->interface_mode == 1) {
    r.b = orc_b_of_alpha(alpha_max);
    real cs2 = (4.0 + r.b) / 10.0;
    r.q1 = 1.0 / (alpha / cs2 + 0.5);
  } else {
    r.b = orc_b_of_alpha(alpha);
    r.q1 = 6.0 / (3.0 + sqrt(3.0));
  }
  return r;
}

/* Largest diffusivity of each scalar over the fluid cells. */
static void max_diffusivities(const orc_params *P, const orc_material *mat, const uint8_t *mask,
                              real amax[3]) {
  size_t n = (size_t)P->nx * P->ny;
  amax[0] = amax[1] = amax[2] = 0.0;
  for (size_t c = 0; c < n; ++c) {
    if ((mask[c] & 3) == REG_SOLID) continue;
    if (mat->alpha_T[c] > amax[0]) amax[0] = mat->alpha_T[c];
    if (mat->D_O2[c] > amax[1]) amax[1] = mat->D_O2[c];
    if (mat->D_H2O[c] > amax[2]) amax[2] = mat->D_H2O[c];
  }
}

/* D2Q5 equilibrium populations N^-1 n_eq for value C, velocity u, b. */
static void d2q5_equilibrium(real C, real ux, real uy, real b, real geq[5]) {
  real neq[5] = {C, ux * C, uy * C, b * C, 0.0};
  for (int i = 0; i < 5; ++i) {
    geq[i] = 0;
    for (int k = 0; k < 5; ++k) geq[i] += NINV5[i][k] * neq[k];
  }
}

/* Eq. 5 equilibrium moments. */
static void flow_meq(real phi, real p, real ux, real uy, real meq[9]) {
  const real rho0 = 1.0;
  real u2 = ux * ux + uy * uy;
  meq[0] = rho0;
  meq[1] = -4 * rho0 + 6 * phi * p + 3 * rho0 * u2 / phi;
  meq[2] = 4 * rho0 - 9 * phi * p - 3 * rho0 * u2 / phi;
  meq[3] = rho0 * ux;
  meq[4] = -rho0 * ux;
  meq[5] = rho0 * uy;
  meq[6] = -rho0 * uy;
  meq[7] = rho0 * (ux * ux - uy * uy) / phi;
  meq[8] = rho0 * ux * uy / phi;
}

/* Eq. 6 forcing moments (G7, G8 in the form derived from Guo's forcing). */
static void flow_G(real phi, real ux, real uy, real Fx, real Fy, real G[9]) {
  const real rho0 = 1.0;
  real uF = ux * Fx + uy * Fy;
  G[0] = 0;
  G[1] = 6 * rho0 * uF / phi;
  G[2] = -6 * rho0 * uF / phi;
  G[3] = rho0 * Fx;
  G[4] = -rho0 * Fx;
  G[5] = rho0 * Fy;
  G[6] = -rho0 * Fy;
  G[7] = 2 * rho0 * (ux * Fx - uy * Fy) / phi;
  G[8] = rho0 * (ux * Fy + uy * Fx) / phi;
}

/* Relaxation rates S (Sec. 2.1) for relaxation time tau.  The printed S has
 * s_0 = 0, but Eq. 5 sets m_0^eq = rho0, which differs from m_0 = sum f in
 * this pressure-based incompressible model; with s_0 = 0 the scheme is
 * linearly unstable (von Neumann amplification 1.43 at tau = 0.65).  The
 * mass moment relaxes at 1/tau instead, as in the BGK limit of the same
 * incompressible equilibrium. */
static void flow_S(real tau, real S[9]) {
  real sq = 8.0 * (2.0 - 1.0 / tau) / (8.0 - 1.0 / tau);
  real s[9] = {1 / tau, 1 / tau, 1 / tau, 0, sq, 0, sq, 1 / tau, 1 / tau};
  memcpy(S, s, sizeof s);
}

/* Q of Eq. 10. */
static void scalar_Q(real Q[5]) {
  real a = 6.0 / (3.0 + sqrt(3.0)), c = 6.0 / (3.0 + 2.0 * sqrt(3.0));
  real q[5] = {0, a, a, c, c};
  memcpy(Q, q, sizeof q);
}

/* Darcy-Forchheimer coefficients of Eq. 7/8 for one cell. */
typedef struct { real phi, darcy, forch, l0, l1; } porous_coef;
static porous_coef porous(const orc_params *P, real phi, real K) {
  porous_coef c;
  c.phi = phi;
  if (isinf(K)) {
    c.darcy = 0; c.forch = 0;
  } else {
    real Fphi = 0.143 * pow(phi, -1.5);
    c.darcy = phi * P->nu / K;
    c.forch = P->forchheimer ? phi * Fphi / sqrt(K) : 0.0;
  }
  /* l0 = (2K + phi nu dt)/(4K), l1 = phi dt F_phi/(2 sqrt K), dt = 1 */
  c.l0 = 0.5 + 0.25 * c.darcy;
  c.l1 = 0.5 * c.forch;
  return c;
}

/* Eq. 8: velocity from the auxiliary velocity v. */
void orc_velocity(real l0, real l1, real vx, real vy, real *ux, real *uy) {
  real vn = sqrt(vx * vx + vy * vy);
  real den = l0 + sqrt(l0 * l0 + l1 * vn);
  *ux = vx / den;
  *uy = vy / den;
}

/* Inlet velocity profile: parabola over the channel rows, mean u_in_avg,
 * evaluated at height y (cell centres at integer y, channel from y0 - 1/2
 * to ny - 1/2); zero outside the channel. */
static real inlet_u(const orc_params *P, real y) {
  int y0 = P->ny_cl + P->ny_gdl;
  real h = P->ny - y0;
  real s = (y - y0 + 0.5) / h;
  if (s <= 0.0 || s >= 1.0) return 0.0;
  return 6.0 * P->u_in_avg * s * (1.0 - s);
}

/* Whether scalar s is held at a fixed value on wall k (0 the x = 0 end,
 * 1 the x = nx-1 end, 2 the bottom). */
static int wall_fixed(const orc_params *P, int k, int s) {
  return (P->wall_dirichlet >> (3 * k + s)) & 1;
}

/* Body force per unit mass at temperature T: the uniform force along x of
 * the closed-form tests plus the Boussinesq buoyancy of Sec. 3's
 * natural-convection cases, gamma (T - T_buoy). */
static void body_force(const orc_params *P, real T, real *Gx, real *Gy) {
  *Gx = P->body_force_x + P->buoy_gx * (T - P->T_buoy);
  *Gy = P->buoy_gy * (T - P->T_buoy);
}

/* --------------------------------------------------------------- state */

/* Initial state: f = w rho0 (rest), g = D2Q5 equilibrium of the inlet values
 * at rest with the cell's own b. */
void orc_init(const orc_params *P, const orc_material *mat, const uint8_t *mask,
              real *f, real *g) {
  ensure_inverses();
  int nx = P->nx, ny = P->ny;
  size_t n = (size_t)nx * ny;
  real Cin[3] = {P->T_in, P->C_O2_in, P->C_H2O_in}, amax[3];
  max_diffusivities(P, mat, mask, amax);
  for (size_t c = 0; c < n; ++c) {
    if ((mask[c] & 3) == REG_SOLID) {
      for (int i = 0; i < 9; ++i) f[i * n + c] = 0;
      for (int k = 0; k < 15; ++k) g[k * n + c] = 0;
      continue;
    }
    for (int i = 0; i < 9; ++i) f[i * n + c] = W9[i];
    real alpha[3] = {mat->alpha_T[c], mat->D_O2[c], mat->D_H2O[c]};
    for (int s = 0; s < 3; ++s) {
      real geq[5];
      d2q5_equilibrium(Cin[s], 0, 0, scalar_coefficients(P, alpha[s], amax[s]).b, geq);
      for (int i = 0; i < 5; ++i) g[(s * 5 + i) * n + c] = geq[i];
    }
  }
}

/* d f_i^eq / d(phi p) of the Eq. 5 equilibrium (M^-1 applied to the p
 * column of m_eq): 1/3 on axis links, 1/12 on diagonals. */
static real pressure_weight(int i) {
  real dm[9] = {0, 6, -9, 0, 0, 0, 0, 0, 0}, v = 0;
  for (int k = 0; k < 9; ++k) v += MINV9[i][k] * dm[k];
  return v;
}
/* phi p of a cell's post-collision populations (Eq. 8 applied to f*). */
static real post_pressure(real phi, const real *fs, size_t n, size_t c) {
  real jx = 0, jy = 0, s18 = 0;
  for (int k = 0; k < 9; ++k) {
    jx += EX9[k] * fs[k * n + c];
    jy += EY9[k] * fs[k * n + c];
    if (k >= 1) s18 += fs[k * n + c];
  }
  return phi * (0.6 / phi * s18 - 6.0 * (jx * jx + jy * jy) / (15.0 * phi * phi));
}

/* Diagnostics of one stream: index layout of the diag[] vector. */
enum {
  D_J = 0,          /* O2 consumed by reaction, sum over the catalyst (lattice) */
  D_HEAT = 1,       /* temperature added by reaction heat (lattice K) */
  D_IN = 2,         /* 2..5: net inflow at the inlet  (mass, T, O2, H2O) */
  D_OUT = 6,        /* 6..9: net inflow at the outlet (mass, T, O2, H2O) */
  D_NDIAG = 10
};

/* Stream with boundary links (f, g post-collision at t -> post-stream at t+1).
 * Also records the reaction terms applied in this stream: the surface
 * fluxes go into the incoming links; the volumetric sinks (S per cell and
 * scalar) are returned in src[3][ny][nx] for the collision to add. */
static void stream(const orc_params *P, const orc_material *mat, const uint8_t *mask,
                   const real *fs, const real *gs, real *f, real *g,
                   real *src, real *diag, real *Jx, real *qx) {
  int nx = P->nx, ny = P->ny;
  size_t n = (size_t)nx * ny;
  real Cin[3] = {P->T_in, P->C_O2_in, P->C_H2O_in};
  real Ctop[3] = {P->T_top, P->C_O2_top, P->C_H2O_top}, amax[3];
  max_diffusivities(P, mat, mask, amax);
  for (int k = 0; k < D_NDIAG; ++k) diag[k] = 0;
  if (Jx) for (int x = 0; x < nx; ++x) Jx[x] = 0;
  if (qx) for (int x = 0; x < nx; ++x) qx[x] = 0;
  memset(src, 0, sizeof(real) * 3 * n);

  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = IDX(x, y);
      uint8_t m = mask[c];
      if ((m & 3) == REG_SOLID) {
        for (int i = 0; i < 9; ++i) f[i * n + c] = 0;
        for (int k = 0; k < 15; ++k) g[k * n + c] = 0;
        continue;
      }
      /* previous post-collision sums at this cell (C^n, T^n) */
      real Cn[3];
      for (int s = 0; s < 3; ++s) {
        Cn[s] = 0;
        for (int i = 0; i < 5; ++i) Cn[s] += gs[(s * 5 + i) * n + c];
      }
      real bcell[3] = {scalar_coefficients(P, mat->alpha_T[c], amax[0]).b,
                         scalar_coefficients(P, mat->D_O2[c], amax[1]).b,
                         scalar_coefficients(P, mat->D_H2O[c], amax[2]).b};

      /* ---- D2Q9 flow links */
      for (int i = 0; i < 9; ++i) {
        int sx = x - EX9[i], sy = y - EY9[i], io = opposite9(i);
        real val;
        if (sy < 0 || sy >= ny) {
          val = fs[io * n + c];                               /* wall */
        } else {
          if (P->periodic_x) sx = (sx + nx) % nx;
          if (sx < 0) {
            if ((m & B_INLET) && P->inlet_mode == 1) {
              /* pressure inlet: the virtual column -1 repeats column 0 (fully
               * developed), with its equilibrium pressure part moved to
               * phi p = rho0/3 + dp_in; the outlet stays at rho0/3, so the
               * pressure difference drives the flow (Sec. 4).  A source row
               * outside the channel is the GDL's end wall. */
              size_t cv = IDX(0, sy);
              if (mask[cv] & B_INLET) {
                val = fs[i * n + cv] +
                      pressure_weight(i) * (1.0 / 3.0 + P->dp_in - post_pressure(mat->phi[cv], fs, n, cv));
                diag[D_IN + 0] += val - fs[io * n + c];
              } else {
                val = fs[io * n + c];
              }
            } else if (m & B_INLET) {                         /* moving-wall inlet */
              /* link crosses the inlet plane at height y - e_iy/2 */
              real uin = inlet_u(P, y - 0.5 * EY9[i]);
              val = fs[io * n + c] + 6.0 * W9[i] * 1.0 * (EX9[i] * uin);
              diag[D_IN + 0] += val - fs[io * n + c];
            } else {
              val = fs[io * n + c];
            }
          } else if (sx >= nx && P->closed_x) {
            val = fs[io * n + c];                              /* end wall */
            diag[D_OUT + 0] += val;
          } else if (sx >= nx) {
            /* outlet: the virtual column nx repeats column nx-1 (fully
             * developed flow), with its equilibrium pressure part moved to
             * the specified outlet pressure phi p = rho0/3 (Sec. 5) */
            size_t cv = IDX(nx - 1, sy);
            val = fs[i * n + cv] + pressure_weight(i) * (1.0 / 3.0 - post_pressure(mat->phi[cv], fs, n, cv));
            diag[D_OUT + 0] += val;
          } else if ((mask[IDX(sx, sy)] & 3) == REG_SOLID) {
            val = fs[io * n + c];
          } else {
            val = fs[i * n + IDX(sx, sy)];
          }
        }
        f[i * n + c] = val;
      }

      /* populations leaving through the outlet */
      if (!P->periodic_x) {
        for (int i = 0; i < 9; ++i) {
          int dx = x + EX9[i], dy = y + EY9[i];
          if (dy < 0 || dy >= ny) continue;
          if (dx >= nx) diag[D_OUT + 0] -= fs[i * n + c];
        }
      }

      /* ---- reaction rate at this cell (uses T^n and C^n) */
      real kS = 0, kV = 0, kSa = 0, kVa = 0;
      int surface = (P->reaction_mode == 0) && (m & B_YLO);
      int volume = (P->reaction_mode == 1) && ((m & 3) == REG_CATALYST);
      if (surface) { kS = k_surface(P, Cn[0]); kSa = k_surface_anodic(P, Cn[0]); }
      if (volume) { kV = k_volume(P, Cn[0]); kVa = k_volume_anodic(P, Cn[0]); }
      real hpo = (surface || volume) ? heat_per_O2(P, Cn[0]) : 0.0;   /* gas K per O2 */
      real sig = mat->sigma ? mat->sigma[c] : 1.0;

      /* ---- D2Q5 scalar links */
      real Jsurf = 0;
      for (int s = 0; s < 3; ++s) {
        real w1 = (4.0 + bcell[s]) / 20.0;
        for (int i = 0; i < 5; ++i) {
          int sx = x - EX5[i], sy = y - EY5[i], io = opposite5(i);
          const real *gq = gs + (size_t)(s * 5) * n;
          real own_out = gq[io * n + c];
          real val;
          if (sy < 0) {
            if (wall_fixed(P, 2, s)) {
              /* fixed bottom value (anti-bounce-back at the halfway wall) */
              val = -own_out + 2.0 * w1 * P->C_wall[6 + s];
            } else if (surface) {
              if (s == 1) {
                /* net O2 flux J = kS C_w - kSa with the wall value
                 * C_w = (own_out + val)/(2 w1) and J = own_out - val */
                real kappa = kS / (2.0 * w1);
                val = (own_out * (1.0 - kappa) + kSa) / (1.0 + kappa);
                Jsurf = own_out - val;
              } else {
                val = own_out; /* completed after O2 below */
              }
            } else {
              val = own_out;
            }
          } else if (sy >= ny) {
            if (P->top_dirichlet) val = -own_out + 2.0 * w1 * Ctop[s];
            else val = own_out;
          } else {
            if (P->periodic_x) sx = (sx + nx) % nx;
            if (sx < 0) {
              if (m & B_INLET) {
                val = -own_out + 2.0 * w1 * Cin[s];
                diag[D_IN + 1 + s] += val - own_out;
              } else if (wall_fixed(P, 0, s)) {
                val = -own_out + 2.0 * w1 * P->C_wall[s];
                diag[D_IN + 1 + s] += val - own_out;
              } else {
                val = own_out;
              }
            } else if (sx >= nx && P->closed_x) {
              val = wall_fixed(P, 1, s) ? -own_out + 2.0 * w1 * P->C_wall[3 + s] : own_out;
              diag[D_OUT + 1 + s] += val;
            } else if (sx >= nx) {
              int x2 = nx - 2, tx = x2 - EX5[i], ty = y - EY5[i];
              size_t c2 = IDX(x2, y);
              if ((mask[IDX(tx, ty)] & 3) == REG_SOLID) val = gq[io * n + c2];
              else val = gq[i * n + IDX(tx, ty)];
              diag[D_OUT + 1 + s] += val;
            } else if ((mask[IDX(sx, sy)] & 3) == REG_SOLID) {
              val = own_out;
            } else {
              val = gq[i * n + IDX(sx, sy)];
            }
          }
          g[(s * 5 + i) * n + c] = val;
        }
        if (!P->periodic_x) {
          for (int i = 0; i < 5; ++i) {
            const real *gq = gs + (size_t)(s * 5) * n;
            if (x + EX5[i] >= nx) diag[D_OUT + 1 + s] -= gq[i * n + c];
          }
        }
      }
      if (surface) {
        /* Eq. 12: two H2O per O2; Eq. 15: heat into the temperature link */
        int up = 2; /* the D2Q5 link arriving from below, e = (0, 1) */
        g[(2 * 5 + up) * n + c] += 2.0 * Jsurf;
        g[(0 * 5 + up) * n + c] += hpo / sig * Jsurf;
        diag[D_J] += Jsurf;
        diag[D_HEAT] += hpo / sig * Jsurf;
        if (Jx) Jx[x] += Jsurf;
        if (qx) qx[x] += hpo * Jsurf;
      }
      if (volume) {
        /* backward Euler for dC/dt = kVa - kV C */
        real S = (kVa - kV * Cn[1]) / (1.0 + kV);
        src[0 * n + c] = -S * hpo / sig;
        src[1 * n + c] = S;
        src[2 * n + c] = -2.0 * S;
        diag[D_J] += -S;
        diag[D_HEAT] += -S * hpo / sig;
        if (Jx) Jx[x] += -S;
        if (qx) qx[x] += -S * hpo;
      }
    }
}

/* Macroscopic fields of a post-stream state (Eq. 8, 11).  out may be NULL. */
typedef struct { real ux, uy, p, C[3], usx, usy; } cell_macro;

static cell_macro macros_at(const orc_params *P, const orc_material *mat, size_t n, size_t c,
                            const real *f, const real *g) {
  cell_macro r;
  porous_coef pc = porous(P, mat->phi[c], mat->K[c]);
  const real rho0 = 1.0;
  real vx = 0, vy = 0, s18 = 0;
  for (int i = 0; i < 9; ++i) {
    vx += EX9[i] * f[i * n + c] / rho0;
    vy += EY9[i] * f[i * n + c] / rho0;
    if (i >= 1) s18 += f[i * n + c];
  }
  /* the force enters Eq. 8's auxiliary velocity with half a time step; the
   * buoyancy takes the cell's temperature after streaming */
  real T = 0, Gx, Gy;
  for (int i = 0; i < 5; ++i) T += g[(0 * 5 + i) * n + c];
  body_force(P, T, &Gx, &Gy);
  vx += 0.5 * pc.phi * Gx;
  vy += 0.5 * pc.phi * Gy;
  orc_velocity(pc.l0, pc.l1, vx, vy, &r.ux, &r.uy);
  /* velocity carried by the scalars: the flow's, or an imposed one (tests) */
  r.usx = mat->u_imposed ? mat->u_imposed[c] : r.ux;
  r.usy = mat->u_imposed ? mat->u_imposed[n + c] : r.uy;
  real u2 = r.ux * r.ux + r.uy * r.uy;
  r.p = 0.6 / pc.phi * s18 - 6.0 * rho0 * u2 / (15.0 * pc.phi * pc.phi);
  for (int s = 0; s < 3; ++s) {
    r.C[s] = 0;
    for (int i = 0; i < 5; ++i) r.C[s] += g[(s * 5 + i) * n + c];
  }
  return r;
}

/* One coupled time step: (fs, gs) post-collision at t -> (fo, go) at t+1.
 * diag[D_NDIAG], Jx[nx], qx[nx] may be NULL. */
void orc_step(const orc_params *P, const orc_material *mat, const uint8_t *mask,
              const real *fs, const real *gs, real *fo, real *go, real *diag,
              real *Jx, real *qx) {
  ensure_inverses();
  int nx = P->nx, ny = P->ny;
  size_t n = (size_t)nx * ny;
  real *f = (real *)malloc(sizeof(real) * 9 * n);
  real *g = (real *)malloc(sizeof(real) * 15 * n);
  real *src = (real *)malloc(sizeof(real) * 3 * n);
  real dloc[D_NDIAG];
  stream(P, mat, mask, fs, gs, f, g, src, dloc, Jx, qx);
  if (diag) memcpy(diag, dloc, sizeof dloc);

  real tau = 3.0 * P->nu + 0.5, S[9], Q[5], amax[3];
  const real Cin[3] = {P->T_in, P->C_O2_in, P->C_H2O_in};
  flow_S(tau, S);
  scalar_Q(Q);
  max_diffusivities(P, mat, mask, amax);

#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = IDX(x, y);
      if ((mask[c] & 3) == REG_SOLID) {
        for (int i = 0; i < 9; ++i) fo[i * n + c] = 0;
        for (int k = 0; k < 15; ++k) go[k * n + c] = 0;
        continue;
      }
      cell_macro mc = macros_at(P, mat, n, c, f, g);
      porous_coef pc = porous(P, mat->phi[c], mat->K[c]);
      /* Eq. 7 force plus phi times the body force (uniform and buoyant) */
      real un = sqrt(mc.ux * mc.ux + mc.uy * mc.uy), Gx, Gy;
      body_force(P, mc.C[0], &Gx, &Gy);
      real Fx = -pc.darcy * mc.ux - pc.forch * un * mc.ux + pc.phi * Gx;
      real Fy = -pc.darcy * mc.uy - pc.forch * un * mc.uy + pc.phi * Gy;
      /* Eq. 1 in moment space */
      real m[9], meq[9], G[9], ms[9];
      for (int k = 0; k < 9; ++k) {
        m[k] = 0;
        for (int i = 0; i < 9; ++i) m[k] += M9[k][i] * f[i * n + c];
      }
      flow_meq(pc.phi, mc.p, mc.ux, mc.uy, meq);
      flow_G(pc.phi, mc.ux, mc.uy, Fx, Fy, G);
      for (int k = 0; k < 9; ++k)
        ms[k] = m[k] - S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * G[k];
      for (int i = 0; i < 9; ++i) {
        real v = 0;
        for (int k = 0; k < 9; ++k) v += MINV9[i][k] * ms[k];
        fo[i * n + c] = v;
      }
      /* Eq. 10 for T, O2, H2O */
      real alpha[3] = {mat->alpha_T[c], mat->D_O2[c], mat->D_H2O[c]};
      for (int s = 0; s < 3; ++s) {
        scalar_coef sc = scalar_coefficients(P, alpha[s], amax[s]);
        real b = sc.b, Qs[5] = {Q[0], sc.q1, sc.q1, Q[3], Q[4]};
        real C = mc.C[s];
        /* the advected value: C itself (Eq. 10 as printed) or its excess over
         * the inlet value; the two give the same continuum equation where
         * div u = 0, which the flow of Sec. 2.1 is built to satisfy */
        real Ca = P->scalar_advection ? C - Cin[s] : C;
        real nv[5], neq[5] = {C, mc.usx * Ca, mc.usy * Ca, b * C, 0.0}, ns[5];
        for (int k = 0; k < 5; ++k) {
          nv[k] = 0;
          for (int i = 0; i < 5; ++i) nv[k] += N5[k][i] * g[(s * 5 + i) * n + c];
        }
        for (int k = 0; k < 5; ++k) ns[k] = nv[k] - Qs[k] * (nv[k] - neq[k]);
        real wsrc[5] = {(1.0 - b) / 5.0, (4.0 + b) / 20.0, (4.0 + b) / 20.0,
                          (4.0 + b) / 20.0, (4.0 + b) / 20.0};
        for (int i = 0; i < 5; ++i) {
          real v = 0;
          for (int k = 0; k < 5; ++k) v += NINV5[i][k] * ns[k];
          go[(s * 5 + i) * n + c] = v + wsrc[i] * src[s * n + c];
        }
      }
    }
  free(f);
  free(g);
  free(src);
}

/* Fields after a step, from the state before it: stream (fs, gs) and take the
 * macroscopic values the collision of that step uses.
 * out: [6][ny][nx] = ux, uy, p, T, C_O2, C_H2O.  Solid cells give zeros. */
void orc_fields(const orc_params *P, const orc_material *mat, const uint8_t *mask,
                const real *fs, const real *gs, real *out, real *diag, real *Jx,
                real *qx) {
  ensure_inverses();
  int nx = P->nx, ny = P->ny;
  size_t n = (size_t)nx * ny;
  real *f = (real *)malloc(sizeof(real) * 9 * n);
  real *g = (real *)malloc(sizeof(real) * 15 * n);
  real *src = (real *)malloc(sizeof(real) * 3 * n);
  real dloc[D_NDIAG];
  stream(P, mat, mask, fs, gs, f, g, src, dloc, Jx, qx);
  if (diag) memcpy(diag, dloc, sizeof dloc);
  for (size_t c = 0; c < n; ++c) {
    if ((mask[c] & 3) == REG_SOLID) {
      for (int k = 0; k < 6; ++k) out[k * n + c] = 0;
      continue;
    }
    cell_macro mc = macros_at(P, mat, n, c, f, g);
    out[0 * n + c] = mc.ux;
    out[1 * n + c] = mc.uy;
    out[2 * n + c] = mc.p;
    for (int s = 0; s < 3; ++s) out[(3 + s) * n + c] = mc.C[s];
  }
  free(f);
  free(g);
  free(src);
}

/* Moments of a post-collision state used by the steady-state residual:
 * out [5][ny][nx] = sum e_x f*, sum e_y f*, sum g*_T, sum g*_O2, sum g*_H2O. */
void orc_state_moments(const orc_params *P, const uint8_t *mask, const real *fs,
                       const real *gs, real *out) {
  int nx = P->nx, ny = P->ny;
  size_t n = (size_t)nx * ny;
  for (size_t c = 0; c < n; ++c) {
    real jx = 0, jy = 0, C[3] = {0, 0, 0};
    if ((mask[c] & 3) != REG_SOLID) {
      for (int i = 0; i < 9; ++i) {
        jx += EX9[i] * fs[i * n + c];
        jy += EY9[i] * fs[i * n + c];
      }
      for (int s = 0; s < 3; ++s)
        for (int i = 0; i < 5; ++i) C[s] += gs[(s * 5 + i) * n + c];
    }
    out[0 * n + c] = jx;
    out[1 * n + c] = jy;
    for (int s = 0; s < 3; ++s) out[(2 + s) * n + c] = C[s];
  }
}

/* Steady-state residual (the paper reports steady states and states no
 * convergence test; reading): the moments X of the post-collision state,
 * X in {sum e_x f*, sum e_y f*, T - T_in, C_O2, C_H2O} (solid cells 0), are
 * compared with the moments of the previous call, held in snapshot
 * [5][ny][nx]; r = max over the five of ||X - X_prev||_2 / ||X||_2, with
 * 0/0 read as 0 and x/0 (x > 0) as +inf.  The snapshot is then replaced by
 * the current moments.  Sums in FP64, cell by cell in row-major order. */
real orc_residual(const orc_params *P, const uint8_t *mask, const real *fs,
                    const real *gs, real *snapshot) {
  int nx = P->nx, ny = P->ny;
  size_t n = (size_t)nx * ny;
  real *X = (real *)malloc(sizeof(real) * 5 * n);
  orc_state_moments(P, mask, fs, gs, X);
  for (size_t c = 0; c < n; ++c)
    if ((mask[c] & 3) != REG_SOLID) X[2 * n + c] -= P->T_in;
  real r = 0.0;
  for (int k = 0; k < 5; ++k) {
    real num = 0.0, den = 0.0;
    for (size_t c = 0; c < n; ++c) {
      real d = X[k * n + c] - snapshot[k * n + c];
      num += d * d;
      den += X[k * n + c] * X[k * n + c];
    }
    real rk = den > 0 ? sqrt(num / den) : (num > 0 ? INFINITY : 0.0);
    if (rk > r || isnan(rk)) r = rk;
  }
  memcpy(snapshot, X, sizeof(real) * 5 * n);
  free(X);
  return r;
}

/* ----------------------------------------- exposed pieces for the pins */

void orc_matrices(real *M, real *Minv, real *N, real *Ninv) {
  ensure_inverses();
  memcpy(M, M9, sizeof M9);
  memcpy(Minv, MINV9, sizeof MINV9);
  memcpy(N, N5, sizeof N5);
  memcpy(Ninv, NINV5, sizeof NINV5);
}
void orc_flow_meq(real phi, real p, real ux, real uy, real *meq) {
  flow_meq(phi, p, ux, uy, meq);
}
void orc_flow_G(real phi, real ux, real uy, real Fx, real Fy, real *G) {
  flow_G(phi, ux, uy, Fx, Fy, G);
}
void orc_flow_S(real tau, real *S) { flow_S(tau, S); }
void orc_scalar_Q(real *Q) { scalar_Q(Q); }
void orc_d2q5_eq(real C, real ux, real uy, real b, real *geq) {
  ensure_inverses();
  d2q5_equilibrium(C, ux, uy, b, geq);
}
real orc_k_surface(const orc_params *P, real T) { return k_surface(P, T); }
real orc_k_volume(const orc_params *P, real T) { return k_volume(P, T); }
real orc_heat_per_O2(const orc_params *P, real T) { return heat_per_O2(P, T); }
real orc_k_surface_anodic(const orc_params *P, real T) { return k_surface_anodic(P, T); }
real orc_k_volume_anodic(const orc_params *P, real T) { return k_volume_anodic(P, T); }
void orc_porous(const orc_params *P, real phi, real K, real *out5) {
  porous_coef c = porous(P, phi, K);
  out5[0] = c.phi; out5[1] = c.darcy; out5[2] = c.forch; out5[3] = c.l0; out5[4] = c.l1;
}
