/*
 * pemlbm: coupled lattice-Boltzmann time step of a PEM fuel-cell cathode
 * (gas channel over a porous gas-diffusion layer over a catalyst layer) on
 * one GB300 GPU (sm_103a).
 *
 * Method: arXiv 2103.01444, "Simulation of Coupled Heat and Mass Transport
 * With Reaction in PEM Fuel Cell Cathode using Lattice Boltzmann Method".
 *   flow     : D2Q9 MRT generalized lattice-Boltzmann equation for porous
 *              media with the Darcy-Forchheimer force (Sec. 2.1, Eq. 1-8)
 *   scalars  : three D2Q5 MRT advection-diffusion lattices for temperature,
 *              O2 and H2O mole fractions (Sec. 2.2, Eq. 9-11)
 *   reaction : Tafel oxygen reduction at the catalyst layer with its heat
 *              release (Sec. 4, Eq. 12-17); Bruggeman and effective thermal
 *              diffusivity (Eq. 18-19) are the caller's material inputs.
 *
 * Conventions of every entry point:
 *   - Returns an lbm_status; no C++ exception crosses the ABI.  On failure
 *     lbm_last_error() gives a message (thread-local, valid until the next
 *     call on the same thread).
 *   - Inputs are copied: the caller keeps ownership of every pointer passed.
 *     Outputs go to caller-allocated buffers.
 *   - Host arrays over the lattice are row-major [ny][nx], x (the flow
 *     direction, inlet at x = -1/2) fastest, y = 0 the bottom row next to
 *     the catalyst wall, y = ny-1 the top row under the channel wall.
 *   - A domain owns all its device memory; work runs asynchronously on the
 *     domain's stream.  Calls that return host values synchronise it.
 *   - Lattice units: dx = dt = 1, rho0 = 1.
 */
#ifndef PEMLBM_H
#define PEMLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* invalid argument or parameter outside the stable range */
  LBM_ENOMEM = 2,    /* device or host allocation failed */
  LBM_ECUDA = 3,     /* a CUDA runtime call failed */
  LBM_ESTATE = 4,    /* call not valid in the domain's current state */
  LBM_EDIVERGED = 5, /* non-finite values found in the state */
  LBM_ETIMEOUT = 6   /* a bounded device-side wait gave up */
} lbm_status;

/* Storage type of the 24 populations per cell; arithmetic is FP64 for
 * LBM_FP64 and FP32 otherwise. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_BF16 = 2, LBM_FP16 = 3 } lbm_precision;

/* Geometry of one cathode lattice (Sec. 4, Fig. 4). */
typedef struct {
  int32_t nx, ny;          /* lattice cells; nx >= 4, ny >= 3 */
  int32_t ny_cl;           /* catalyst rows at the bottom (volumetric mode only, else 0) */
  int32_t ny_gdl;          /* porous GDL rows above them; the channel takes the rest */
  int32_t reaction_mode;   /* 0: thin catalyst film on the bottom wall (the paper's
                              negligible-thickness layer); 1: volumetric catalyst rows */
  int32_t periodic_x;      /* 1: x is periodic (closed-form tests); 0: inlet/outlet */
  int32_t closed_x;        /* 1: both x ends are no-slip walls (the cavities of Sec. 3):
                              no inlet, no outlet; the scalars there are insulated
                              unless lbm_params.wall_dirichlet fixes them.  Excludes
                              periodic_x; lbm_grad and lbm_vjp need 0. */
  int32_t precision;       /* lbm_precision */
  int32_t rounding;        /* how a step stores 16-bit populations (LBM_BF16, LBM_FP16):
                              0 round to nearest even; 1 stochastic rounding, unbiased,
                              with random bits from a counter-based hash of the cell, the
                              link and a device step counter (reset by lbm_reset), so runs
                              from reset are reproducible.  Small per-step increments of a
                              large deviation (slow heating, water production) survive
                              in expectation instead of being rounded away.  Must be 0 for
                              FP32/FP64; lbm_grad, lbm_vjp, batches, closed_x,
                              buoyancy and fixed wall values need 0. */
  const uint8_t *solid;    /* optional host [ny][nx] pore-scale solid cells (1 = solid);
                              NULL = none.  Solids may not touch column 0 or the last
                              two columns. */
  void *cuda_stream;       /* borrowed cudaStream_t; NULL = the library's own stream */
  int32_t x_begin, x_end;  /* x-slab decomposition of a long channel (the geometry of Sec. 4,
                              Fig. 4): with x_end > 0 the domain holds only the columns
                              [x_begin, x_end) of the nx-column lattice described here
                              (at least 4 of them).  Positions, the inlet and outlet
                              columns, solid cells (solid is the whole [ny][nx] lattice)
                              and, in lbm_set_fields, the material arrays and the
                              palette are the whole lattice's, so that neighbouring
                              slabs agree cell for cell.  A side inside the lattice
                              borders a neighbour slab: its pulls read a ghost column
                              that lbm_halo_exchange (same device) or lbm_halo_unpack
                              fills before each step.  Per-cell arrays of the other
                              calls cover the slab's own columns.  Not with
                              periodic_x, lbm_grad, lbm_vjp, batches or device
                              material.  0, 0: the whole lattice. */
} lbm_domain_desc;

/* Operating point and closure constants.  Lattice units unless a unit is
 * given.  Physical constants enter only the reaction terms. */
typedef struct {
  double nu;                   /* kinematic viscosity, 3 nu = tau - 1/2 (Eq. 8); > 0 */
  double u_in_avg;             /* mean inlet velocity over the channel rows (parabola) */
  double body_force_x;         /* uniform body force per unit mass (tests; 0 in use) */
  double V_op;                 /* cell operating potential, V (Eq. 14) */
  double T_in, C_O2_in, C_H2O_in;   /* inlet temperature (K) and mole fractions */
  double T_top, C_O2_top, C_H2O_top; /* top-wall values when top_dirichlet = 1 */
  double aj0_ref;              /* A/cm^3 at T_ref_kin (Eq. 13, 17) */
  double T_ref_kin;            /* K, reference temperature of Eq. 17 */
  double E_act;                /* K, activation temperature of Eq. 17 (16456) */
  double alpha_c, F, R;        /* transfer coefficient, C/mol, J/(mol K) (Eq. 13) */
  double dU0dT, U0_0;          /* Eq. 16: U0 = dU0dT T + U0_0 (V/K, V) */
  double x_ref;                /* reference O2 mole fraction (C_O2,ref of Eq. 13) */
  double dx_cm, dt_s;          /* lattice spacing (cm) and time step (s) */
  double delta_cl_cm;          /* catalyst film thickness (cm), thin-film mode */
  double c_tot;                /* total gas concentration, mol/cm^3 */
  double rho_cp_f;             /* gas volumetric heat capacity, J/(cm^3 K) */
  int32_t forchheimer;         /* 1: Eq. 7 with the Forchheimer term; 0: Darcy only */
  int32_t top_dirichlet;       /* scalars at the top wall: 0 insulated, 1 fixed values */
  int32_t interface_mode;      /* 0: Eq. 10 as printed, b from each cell's own diffusivity
                                  with fixed Q (alpha C is continuous across layers);
                                  1: Fickian, one b per scalar (that of its largest
                                  diffusivity) and each cell's diffusivity set through
                                  the flux-moment rate (C and -alpha grad C continuous) */
  int32_t inlet_mode;          /* drive of the flow: 0 parabolic inlet velocity u_in_avg over
                                  the channel rows (Ladd moving wall); 1 the pressure
                                  difference of Sec. 4: the channel rows pull from a virtual
                                  column -1 that repeats column 0 with its equilibrium
                                  pressure moved to phi p = 1/3 + dp_in, against 1/3 at the
                                  outlet (u_in_avg is then unused; the du_in of lbm_grad
                                  and lbm_vjp is then the derivative by dp_in). */
  double dp_in;                /* inlet pressure excess of inlet_mode 1, lattice units,
                                  |dp_in| < 0.01 */
  double alpha_a;              /* kinetics: 0 Tafel, Eq. 13 as printed; > 0 (at most 4)
                                  Butler-Volmer, with the anodic branch
                                  aj0(T) exp(alpha_a F eta/(R T)) at unit reactant
                                  activity subtracted from the O2 consumption */
  double buoy_gx, buoy_gy;     /* Boussinesq buoyancy (the natural-convection cases of
                                  Sec. 3): body force per unit mass
                                  (buoy_gx, buoy_gy) (T - T_buoy), lattice units per K,
                                  with T the cell's temperature after streaming.  Like the
                                  uniform body force it enters Eq. 8's velocity and, times
                                  phi, the force F of Eq. 7 (the generalised porous model
                                  Eq. 7-8 come from).  lbm_grad and lbm_vjp need 0. */
  double T_buoy;               /* K, reference temperature of the buoyancy */
  int32_t wall_dirichlet;      /* bit 3 k + s: scalar s (0 T, 1 O2, 2 H2O) is held at
                                  C_wall[k][s] on wall k (0 the x = 0 end outside the inlet
                                  rows, 1 the x = nx - 1 end, closed_x only, 2 the bottom)
                                  instead of insulated.  With the thin film (reaction_mode
                                  0) the bottom's O2 and H2O bits must be 0; the film's
                                  heat adds to a fixed bottom temperature.  lbm_grad and
                                  lbm_vjp need 0. */
  double C_wall[3][3];         /* wall values of wall_dirichlet: K and mole fractions */
  int32_t scalar_advection;    /* flux moments of the D2Q5 equilibria of Eq. 10: 0 u C as
                                  printed; 1 u (C - C_in), each scalar advected relative to
                                  its inlet value.  Both give the same continuum equation
                                  where div u = 0, which the incompressible flow of Sec. 2.1
                                  satisfies; 1 drops the source C_in div u that the lattice
                                  flow's small divergence adds (a uniform field at the inlet
                                  value then stays exactly uniform), and keeps the flux
                                  populations small in the deviation storage. */
} lbm_params;

typedef struct lbm_domain lbm_domain; /* opaque */

/* Allocates a domain (two population buffers, node mask, material palette,
 * reduction scratch) and builds the node mask on the device.  The state is
 * undefined until lbm_set_params, lbm_set_fields and lbm_reset are called.
 * EINVAL: bad sizes, rounding outside {0, 1} or 1 with FP32/FP64 storage,
 * solids on the inlet/outlet columns (or on the end walls' columns with
 * closed_x), closed_x outside {0, 1} or together with periodic_x.
 * ENOMEM: device allocation failed. */
lbm_status lbm_create_domain(const lbm_domain_desc *desc, lbm_domain **out);

/* Frees every resource of d (synchronises its stream first).  NULL is OK. */
lbm_status lbm_destroy_domain(lbm_domain *d);

/* Copies the operating point (Sec. 4-5).  EINVAL unless nu > 0,
 * sqrt(3) * 1.5 * u_in_avg < 0.3 (inlet_mode 0), |dp_in| < 0.01 (inlet_mode
 * 1), 0 <= alpha_a <= 4, T_in > 0, dx_cm > 0, dt_s > 0, wall_dirichlet
 * within bits 0..8 (the right wall's only with closed_x, the bottom's O2
 * and H2O bits 0 with the thin film), finite buoyancy. */
lbm_status lbm_set_params(lbm_domain *d, const lbm_params *p);

/* Per-cell material, arrays [ny][nx] of doubles, lattice units:
 *   phi           porosity, 0 < phi <= 1 (Eq. 5, 7)
 *   K             permeability; +INFINITY marks clear fluid (no drag) (Eq. 7)
 *   alpha_T       effective thermal diffusivity (Eq. 19)
 *   D_O2          effective O2 diffusivity (Eq. 18)
 *   D_H2O         effective H2O diffusivity
 *   rho_cp_ratio  (rho c_p)_eff / (rho c_p)_f of Eq. 19, >= 1e-6; the
 *                 reaction heat enters the temperature equation divided by
 *                 it.  NULL = 1 everywhere.
 * on_device = 0: host arrays.  on_device = 1: device arrays on the domain's
 * device, read on the domain's stream (ordered after work already queued
 * there); the material palette is then built by kernels, and only the
 * palette (at most 65535 tuples) is copied to the host.  Both give the same
 * palette, entry for entry.  Each diffusivity must lie in
 * (0, 5/(20 sqrt 3)] so that the D2Q5 rest weight (1-b)/5 of Eq. 10 is
 * non-negative.  Solid cells are ignored.  Distinct material tuples are
 * collected into a palette of at most 65535 entries (EINVAL beyond that).
 * EINVAL leaves the domain's previous material unchanged.  Synchronises
 * the stream. */
lbm_status lbm_set_fields(lbm_domain *d, const double *phi, const double *K,
                          const double *alpha_T, const double *D_O2, const double *D_H2O,
                          const double *rho_cp_ratio, int32_t on_device);

/* Initial state: f_i = w_i rho0 (rest), g = D2Q5 equilibrium of the inlet
 * values at rest with each cell's own b.  Step counter := 0. */
lbm_status lbm_reset(lbm_domain *d);

/* Advances nsteps coupled steps (Eq. 1, 10 with the Sec. 4 boundary links):
 * stream with boundary links -> macroscopic values (Eq. 8, 11) ->
 * collisions -> catalyst sources.  Asynchronous on the domain's stream;
 * long runs are replayed from a captured CUDA graph. */
lbm_status lbm_step(lbm_domain *d, int64_t nsteps);

/* Reaction of the last step (Sec. 5 outputs): mean current density over the
 * catalyst (A/cm^2), mean heat release (W/cm^2) and, if profile_nx is not
 * NULL, the local current density i(x) along the catalyst (A/cm^2, nx
 * floats).  Accumulated in FP64.  Synchronises the stream.  ESTATE before
 * the first step. */
lbm_status lbm_current_density(lbm_domain *d, double *i_avg_A_cm2, double *heat_W_cm2,
                               float *profile_nx);

/* Observed stepping: advances nsteps steps like lbm_step and reports the
 * reaction of every step, i_avg[k] and heat[k] (host arrays of nsteps
 * doubles, A/cm^2 and W/cm^2 as lbm_current_density; either may be NULL,
 * not both).  Each step's FP64 sums are copied to the host as soon as that
 * step's reduction ends, without stopping the stream: chunks of 64 steps
 * are replayed from CUDA graphs while the host converts the previous
 * chunk.  Synchronises the stream before returning.  EINVAL for nsteps < 0
 * or two NULL arrays; ENOMEM if the observation slots cannot be
 * allocated. */
lbm_status lbm_step_observe(lbm_domain *d, int64_t nsteps, double *i_avg_A_cm2,
                            double *heat_W_cm2);

/* Steady-state residual: r = max over X in {j_x, j_y, T - T_in, C_O2, C_H2O}
 * (moments of the post-collision state) of ||X - X_prev|| / ||X||, where
 * X_prev is the snapshot taken by the previous call (or by lbm_reset); the
 * snapshot is then replaced.  FP64 accumulation.  EDIVERGED on non-finite
 * values. */
lbm_status lbm_residual(lbm_domain *d, double *res);

/* Balances of the last step (per-step reductions of Sec. 4's boundary
 * conditions and Eq. 12-15), lattice units, summed over the lattice, FP64:
 *   out[0] O2 consumed by the reaction (mole fraction per step),
 *   out[1] its heat, h J summed (temperature x mole fraction per step),
 *   out[2..5] net inflow through the inlet column of mass, T, O2, H2O,
 *   out[6..9] net inflow through the outlet column (negative = outflow).
 * With them, the change of each scalar total over the step is exact
 * (the D2Q5 collisions conserve C): O2 in + out - J, H2O in + out + 2 J;
 * the mass flows are those through the boundary links (the collision also
 * relaxes the flow's mass moment, Sec. 2.1).  With closed_x, out[2..5]
 * and out[6..9] are the flows through the walls at x = 0 and x = nx - 1
 * (non-zero only for scalars held at fixed wall values); a fixed bottom
 * value's flow is not listed.  Recomputed from the state before the last
 * step by the step's own boundary pulls (zeros for a periodic lattice).
 * out: host, 10 doubles.  ESTATE before the first step. */
lbm_status lbm_balances(lbm_domain *d, double *out);

/* Macroscopic fields of the last step (the values its collision used):
 * out = [6][ny][nx] doubles: u_x, u_y, p (Eq. 8), T, C_O2, C_H2O (Eq. 11);
 * zeros in solid cells.  on_device = 1: out is a device pointer written on
 * the domain's stream (asynchronous); 0: host pointer (synchronises). */
lbm_status lbm_get_fields(lbm_domain *d, double *out, int32_t on_device);

/* Current post-collision populations as full values (deviation storage
 * removed): out = [24][ny][nx] doubles, planes f_0..f_8, g_T0..4, g_O2 0..4,
 * g_H2O 0..4 (Eq. 2 and Eq. 9 orders).  Host pointer; synchronises. */
lbm_status lbm_get_state(lbm_domain *d, double *out);

/* Overwrites both population buffers with the given full values (same
 * layout as lbm_get_state); the step counter is kept. */
lbm_status lbm_set_state(lbm_domain *d, const double *in);

/* Node mask, [ny][nx] bytes: bits 0-1 region (0 channel, 1 GDL, 2 catalyst
 * rows, 3 solid); bit 2 x = 0; bit 3 x = nx-1; bit 4 y = ny-1; bit 5 y = 0;
 * bit 6 open inlet (x = 0 channel row, not periodic); bit 7 a D2Q9
 * neighbour is solid. */
lbm_status lbm_get_mask(lbm_domain *d, uint8_t *mask_host);

/* Number of steps taken since lbm_reset. */
lbm_status lbm_get_step(lbm_domain *d, int64_t *steps);

/* Checkpoint of the state: with buf == NULL, *bytes receives the size; else
 * writes an 80-byte header (sizes, precision, step) and the raw populations
 * of both buffers in the storage layout of the step: per buffer, five planes
 * of 4-value groups (link i = 0..4 of the flow, T, O2 and H2O, in that order,
 * for every cell) followed by the four planes of flow links 5-8; a plane
 * holds ny rows of the padded row length, x fastest, and every value is a
 * deviation from its direction's reference.  lbm_load_state restores a blob
 * taken from a domain of the same geometry and precision (EINVAL otherwise,
 * and for blobs of an earlier storage layout). */
lbm_status lbm_save_state(lbm_domain *d, void *buf, size_t *bytes);
lbm_status lbm_load_state(lbm_domain *d, const void *buf, size_t bytes);

/* Average device time per launch of the coupled-step kernel over the last
 * lbm_step call that was timed with lbm_time_steps (ms), for roofline
 * reporting: runs nsteps steps bracketed by CUDA events on the domain's
 * stream and returns the elapsed device time. */
lbm_status lbm_time_steps(lbm_domain *d, int64_t nsteps, double *elapsed_ms);

/* Launch shapes of the step kernel (cells per block along x and y, and the
 * minimum resident blocks per SM asked of the register allocator).
 * lbm_tune, called between lbm_reset and the first step, times every shape
 * over trial_steps launches of the same step (the state is left as reset
 * left it), keeps the fastest and returns its index and time per step (ms).
 * ESTATE after the first step.  lbm_set_variant selects one explicitly
 * (0 <= variant < 8; EINVAL otherwise).  All shapes give bit-identical
 * results.  Untuned, FP32 domains use variant 7 (64 x 2 cells, 8 blocks
 * per SM) and the others variant 0. */
lbm_status lbm_tune(lbm_domain *d, int32_t trial_steps, int32_t *variant, double *best_ms);
lbm_status lbm_set_variant(lbm_domain *d, int32_t variant);

/* Bytes the method must move per cell update for this domain's storage
 * (24 populations read and written once, plus the 1-byte node mask). */
lbm_status lbm_bytes_per_cell(lbm_domain *d, double *bytes);

/* Discrete adjoint of the coupled step (gradients for design studies of
 * the GDL, Sec. 5: porosity, permeability and effective O2 diffusivity).
 * Starting from the domain's current state s^0, held fixed, the domain is
 * advanced nsteps steps (in private buffers: the domain's own state is left
 * unchanged) and the objective is evaluated at step N = nsteps:
 *   objective 0: mean current density over the catalyst of step N (A/cm^2),
 *                the value lbm_current_density reports after N steps;
 *   objective 1: the largest temperature of the bottom row in the fields
 *                of step N (K; ties go to the smallest x).
 * Its gradient with respect to the per-cell phi, K and D_O2 of
 * lbm_set_fields (lattice units; K of clear cells gets 0) and to the inlet
 * drive (the lattice inlet velocity u_in_avg, or dp_in with inlet_mode 1)
 * is computed by the transposed step, applied from step N back to step 1.
 * The transpose of step n needs from the forward run only the step's
 * reverse records (per cell the Eq. 8 auxiliary velocity, the three scalar
 * sums and two O2 flux moments, 8 values; per edge or catalyst cell its
 * pulled values and own sums), a third of a population state.  The forward
 * sweep keeps the records of its last segments of `segment` steps (<= 0:
 * ceil(sqrt(nsteps))) in device memory, as many as the limit of
 * lbm_set_grad_memory allows (by default all that fits in the free device
 * memory but a reserve of max(1 GiB, 1/64 of the device)); every earlier
 * segment is recomputed from a checkpoint of its first state.  The records
 * are the same either way, so the result does not depend on the limit.
 * Memory: the stored segments' records, plus, when some segment is
 * recomputed, one population state per recomputed segment and two
 * segments' records.  The gradient of the
 * Fickian interface mode treats each scalar's b (that of its largest
 * diffusivity) as fixed.  dphi, dK, dD_O2 are [ny][nx] doubles (NULL to
 * skip): host memory with on_device = 0, device memory written on the
 * domain's stream with on_device = 1.  J and du_in (one double each) are
 * host values either way; the call synchronises the stream.  EINVAL for
 * objective outside {0, 1}, nsteps outside [2, 2^30], stochastic rounding
 * (lbm_domain_desc.rounding 1), closed_x, buoyancy or fixed wall values
 * (the natural-convection and validation set-ups); ENOMEM if the
 * checkpoints do not fit. */
lbm_status lbm_grad(lbm_domain *d, int32_t objective, int64_t nsteps, int32_t segment,
                    double *J, double *dphi, double *dK, double *dD_O2, double *du_in,
                    int32_t on_device);

/* Device memory lbm_grad may hold for the reverse records of stored
 * segments (bytes): -1 (the default) for what is free less the reserve, 0
 * to recompute every segment from its checkpoint.  The setting is the
 * domain's and applies to its later lbm_grad calls.  EINVAL for a null
 * domain or bytes < -1. */
lbm_status lbm_set_grad_memory(lbm_domain *d, int64_t bytes);

/* Self-check of the device code's indexing (no counterpart in the paper; it
 * stands in for a memory checker).  A library built with bounds checks
 * (paper_2103_01444_gb300.build.build(bounds_check=True), which compiles
 * with -DPEMLBM_BOUNDS_CHECK into libpemlbm_checked.so) tests the index of
 * every population, mask, material-index and palette access of the step
 * kernels, and the lambda, own-use, gradient and record accesses of the
 * adjoint kernels (directly, or through the cell index that bounds them),
 * against the extent of its buffer; an access outside it is skipped (no
 * trap) and the first one recorded.  This call waits for the device, writes
 * the first recorded access since the previous call to *first_bad (site <<
 * 48 | index; 0 for none) and clears the record.  EINVAL for a null
 * argument; ESTATE (and *first_bad = 0) in a library built without the
 * checks. */
lbm_status lbm_bounds_check(uint64_t *first_bad);

/* One transposed step at the current state s: given lam_next (host
 * [24][ny][nx], the adjoint of the state after one step), writes lam_prev =
 * (d step / d s)^T lam_next and the parameter gradients of
 * <lam_next, step(s)> (host, as in lbm_grad; NULL to skip).  EINVAL as
 * lbm_grad for the rounding and the set-ups it does not cover. */
lbm_status lbm_vjp(lbm_domain *d, const double *lam_next, double *lam_prev, double *dphi,
                   double *dK, double *dD_O2, double *du_in);

/* Batched stepping (operating-point sweeps over cases of uneven size).
 * lbm_create_batch groups ncases domains, each already set up and reset
 * (ESTATE otherwise), all of one precision and each a cathode set-up
 * without closed_x, buoyancy or fixed wall values (EINVAL otherwise); the batch
 * borrows them (they must outlive it) and works on their own buffers, so
 * fields, current density and checkpoints of each case stay available
 * through the per-domain calls.  The batch runs on the first domain's
 * stream, ordered after and before the other domains' streams by events.
 * Schedules (lbm_batch_set_schedule):
 *   0  one launch per step covering every case's tiles (launch shape
 *      `variant` of lbm_set_variant), long runs replayed from a CUDA graph;
 *   1  one persistent cooperative launch for all steps: co-resident blocks
 *      loop over the tiles and meet at a grid barrier between steps; each
 *      barrier wait gives up after spin_limit polls (<= 0 keeps the current
 *      limit, 2^24 by default) and the call returns ETIMEOUT, leaving the
 *      case states undefined (reset or load them);
 *   2  one launch per case and step, no graph (the unbatched reference);
 *   3  one stream per case, each case's steps a chain of single-domain
 *      launches (shape `variant`), the chains running concurrently; long
 *      runs replayed from one graph, captured again when a case was stepped
 *      on its own or its arguments changed.
 * All schedules give bit-identical states.  lbm_batch_tune, called between
 * lbm_reset and the first step of every case, times schedules 0 and 3 with
 * every launch shape and schedule 1 over trial_steps repetitions of the
 * first step, keeps the fastest and leaves the states as reset left them. */
typedef struct lbm_batch lbm_batch; /* opaque */
lbm_status lbm_create_batch(lbm_domain *const *domains, int32_t ncases, lbm_batch **out);
lbm_status lbm_destroy_batch(lbm_batch *b);
lbm_status lbm_batch_set_schedule(lbm_batch *b, int32_t schedule, int32_t variant,
                                  int64_t spin_limit);
lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, int32_t *schedule, int32_t *variant,
                          double *best_ms);
/* Advances every case by nsteps (0 <= nsteps <= 2^30). */
lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps);
/* lbm_batch_step bracketed by CUDA events on the batch stream; elapsed ms. */
lbm_status lbm_batch_time_steps(lbm_batch *b, int64_t nsteps, double *elapsed_ms);

/* x-slabs (lbm_domain_desc.x_begin, x_end).  The step pulls, at a slab side,
 * six populations per row from the neighbouring slab's edge column: the +x
 * movers (f1, f5, f8 and the D2Q5 link-1 populations of T, O2, H2O, Eq. 2
 * and 9 orders) enter through the low side, the -x movers (f3, f6, f7 and
 * the link-3 populations) through the high side.  After every step (and
 * after lbm_reset), before the next step, each side's ghost column must be
 * filled from the neighbour's state of the same step:
 *   lbm_halo_exchange(left, right): both directions between two slabs of one
 *     lattice on the same device (left's x_end = right's x_begin).  Ordered
 *     after both slabs' queued work by events; the copies run on left's
 *     stream and right's stream waits for them.  EINVAL unless they are
 *     neighbours with equal storage and deviation references (the same
 *     lattice arrays and parameters); ESTATE before reset or at different
 *     step counts.
 *   lbm_halo_pack(d, side, buf): writes the six populations leaving d through
 *     side (0 low x, 1 high x) into buf, device memory of [6][ny] values of
 *     the storage type, in the order above;
 *   lbm_halo_unpack(d, side, buf): fills side's ghost column from such an
 *     array packed by the neighbour on its facing side.
 *   Both are asynchronous on d's stream; for slabs in different processes
 *   the caller moves buf between them.  EINVAL for a side that borders no
 *   slab.  The values are the storage's deviations, which agree between
 *   slabs set up from the same lattice arrays and parameters.
 * Reductions are per slab: lbm_current_density averages over the slab's
 * columns (the lattice's mean weights each slab by its width),
 * lbm_balances reports zero flow through a slab side, lbm_residual compares
 * the slab's own moments. */
lbm_status lbm_halo_exchange(lbm_domain *left, lbm_domain *right);
lbm_status lbm_halo_pack(lbm_domain *d, int32_t side, void *buf);
lbm_status lbm_halo_unpack(lbm_domain *d, int32_t side, const void *buf);

/* The steady-state residual of lbm_residual, computed without allocating.
 * The paper has no counterpart of this entry point.  It is for callers that
 * must not let the library allocate device memory once they are running:
 * real-time loops, where a cudaMalloc can stall the device's streams for an
 * unbounded time, and host programs that hand out all device memory from a
 * pool of their own and account for every byte of it.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   snapshot  device memory owned by the caller, [5][ny][nx] values of the
 *             domain's arithmetic type (double for LBM_FP64, float otherwise):
 *             the moments of the previous call (zeros before the first one);
 *             read, then overwritten with the current moments.  The library
 *             cannot check this buffer: its type, size and device are the
 *             caller's responsibility.
 *   res       host: ||X - X_prev|| / ||X|| maximised over the five moments
 * The reduction's block partial sums live in one file-scope device array of
 * 16384 blocks x 10 doubles (1.31 MB), which every GPU that loads the library
 * holds until the process exits; lattices needing more than 16384 blocks of
 * 128 x 2 cells (about 4.19 M cells) are rejected with EINVAL.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current and keeps it; make that first call before any
 * stream capture.  All calls share the array, and it keeps the last call's
 * contents (each call clears the flag word that must start at zero): calls
 * that overlap on the GPU, on any domain, race.  The call is synchronous: it
 * waits for the domain's stream before it returns.  EDIVERGED on non-finite
 * values. */
lbm_status lbm_residual_noalloc(lbm_domain *d, void *snapshot, double *res);

const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PEMLBM_H */
