/*
 * lb3e.h -- C ABI of the B300 (sm_103a) three-phase electrohydrodynamic lattice
 * Boltzmann step: Onsager-variational phase-field model of Liu, Qian, Xiong and
 * Wang (three-phase dielectric fluid flows), D2Q9 discretisation of its Section 3.
 *
 * One time step (lb3e_step) is, in order:
 *   zeroth moments of the phase and charge populations (phi_i, sum l);
 *   property interpolation rho, sigma (Eq. 29) and eps (Eq. 30);
 *   isotropic stencils of Eq. 33 and the closed-form charge q = sum l + R/2;
 *   the pseudo-time LB potential solve of Eq. 42-45 (warm-started, to a residual);
 *   the chemical potential of Eq. 20, the force -sum phi_i grad mu_i + q E (Eq. 27b);
 *   flow moments (Eq. 41);
 *   collision + streaming of the phase (Eq. 34-36), flow (Eq. 37-40) and
 *   charge (Eq. 46-50) populations, with half-way walls and electrodes.
 *
 * Conventions for every entry point:
 *   - Device memory is owned by the caller.  lb3e_workspace_bytes() says how much;
 *     the caller allocates it (e.g. a torch tensor) and passes the pointer to
 *     lb3e_init(); it must stay alive and untouched until lb3e_destroy().
 *     The handle itself owns only host memory (and a small pinned host buffer).
 *   - All work is issued on the stream given to lb3e_init() (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream).  Functions that return host
 *     results synchronise that stream.
 *   - Arrays are C-ordered [..][ny][nx] (x fastest), double precision, in lattice
 *     units (dx = dt = 1).  Pointer arguments may be host or device memory
 *     (unified addressing decides); they are read or written before return.
 *   - Every function returns LB3E_OK (0) or a negative LB3E_ERR_* code; none
 *     aborts or prints.  lb3e_status_string() describes a code.
 */
#ifndef LB3E_H
#define LB3E_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LB3E_OK = 0,
    LB3E_ERR_PARAM = -1,          /* invalid parameter (sizes, tau <= 1/2, lambda_i <= 0, ...) */
    LB3E_ERR_WORKSPACE = -2,      /* workspace NULL, misaligned (256 B) or too small */
    LB3E_ERR_CUDA = -3,           /* a CUDA call failed; the handle may be unusable */
    LB3E_ERR_NOT_CONVERGED = -4,  /* potential solve hit max_iter above tol */
    LB3E_ERR_FIELD = -5,          /* unknown field id */
    LB3E_ERR_NULL = -6,           /* NULL handle or output pointer */
    LB3E_ERR_TOO_LARGE = -7,      /* lattice larger than lb3e_observables_noalloc's fixed scratch */
    LB3E_ERR_UNSUPPORTED = -8     /* no reverse mode for this configuration (see lb3e_adjoint_step) */
};

/* Field ids for lb3e_get_field.  "Last step" fields hold the values computed
 * during the most recent time step (after lb3e_init: the initial values). */
enum {
    LB3E_FIELD_PHI1 = 0,  /* phi_i used in the last step (moments at its start) */
    LB3E_FIELD_PHI2 = 1,
    LB3E_FIELD_PHI3 = 2,
    LB3E_FIELD_UX = 3,    /* velocity of the last step, Eq. 41 */
    LB3E_FIELD_UY = 4,
    LB3E_FIELD_P = 5,     /* pressure of the last step, Eq. 41 */
    LB3E_FIELD_Q = 6,     /* charge q = sum l + R/2 of the last step */
    LB3E_FIELD_PSI = 7,   /* potential, Eq. 45, of the current h */
    LB3E_FIELD_EX = 8,    /* E = -grad psi (+ E_ext) used in the last step */
    LB3E_FIELD_EY = 9,
    LB3E_FIELD_MU1 = 10,  /* chemical potentials (Eq. 20) of the last step */
    LB3E_FIELD_MU2 = 11,
    LB3E_FIELD_MU3 = 12,
    LB3E_FIELD_PHINOW1 = 13, /* phi_i = sum_j f^i_j of the current populations */
    LB3E_FIELD_PHINOW2 = 14,
    LB3E_FIELD_PHINOW3 = 15,
    LB3E_FIELD_QTILDE = 16,  /* sum_j l_j of the current populations */
    LB3E_FIELD_N1 = 17,      /* ion concentrations n_i = sum_j n^i_j of the current */
    LB3E_FIELD_N2 = 18,      /* ion populations (ions = 1 only) */
    LB3E_FIELD_UZ = 19,      /* three-dimensional lattices: velocity and field along z */
    LB3E_FIELD_EZ = 20,
    LB3E_FIELD_POP = 100     /* + 9*set + j; sets 0 g, 1-3 f^1..f^3, 4 l, 5 h,
                                6-7 the ion species (ions = 1 only); on
                                three-dimensional lattices + 15*set + j, sets 0-5 */
};

/* Largest lattice lb3e_init accepts (cells, nx * ny * nz on three-dimensional
 * lattices; 45 population planes are addressed with 32-bit offsets). */
#define LB3E_MAX_CELLS 40000000
#define LB3E_MAX_NY (65535 * 8)   /* tiles of 8 rows, at most 65535 of them along y */

/* Model and run parameters.  Index i of the per-phase arrays is phase i+1. */
typedef struct lb3e_params {
    int32_t nx, ny;               /* lattice, cells; both >= 2, nx * ny <= LB3E_MAX_CELLS, ny <= LB3E_MAX_NY; periodic in x */
    int32_t bc_y;                 /* 0 periodic, 1 half-way walls, 2 walls with electrodes */
    int32_t electric;             /* 1: solve the potential every step; 0: E = E_ext */
    int32_t precision;            /* 0 fp64; 1 fp32; 2 fp32 compute, fp16-stored populations;
                                     3 fp32 with 3 tangent directions; 4 fp64 with 1 tangent;
                                     5 fp32 compute, bf16-stored populations */
    int32_t _pad0;
    double rho[3];                /* phase densities, Eq. 29 */
    double visc[3];               /* phase dynamic viscosities, Eq. 29; all <= 0: use tau_g */
    double tau_g;                 /* flow relaxation time when visc is not given */
    double gamma12, gamma13, gamma23; /* surface tensions; lambda_i from Eq. 9 must be > 0 */
    double width_D;               /* interface width D, Eq. 7 */
    double tau_f;                 /* phase relaxation time; m0 = cs^2 (tau_f - 1/2) */
    double eps[3];                /* phase permittivities, Eq. 30 */
    double sigma[3];              /* phase conductivities, Eq. 29 (>= 0) */
    double eps_ref;               /* constant part of the permittivity split (Eq. 42); tau_h = 1/2 + eps_ref/cs^2 */
    double alpha;                 /* charge diffusivity; tau_l = 1/2 + alpha/cs^2 (Eq. 49) */
    double V_bottom, V_top;       /* electrode potentials at y = -1/2 and y = ny - 1/2 (bc_y = 2) */
    double E_ext[2];              /* uniform field added to -grad psi */
    double u_wall_bottom, u_wall_top; /* tangential wall speeds (bc_y >= 1) */
    int32_t charge_convection;    /* 1: velocity terms of Eq. 49-50 on */
    int32_t inner_phase;          /* 1-based phase whose indicator gives D_inner */
    int32_t matrix_phase;         /* 1-based phase; indicator 1 - phi gives D_outer */
    int32_t _pad1;
    double poisson_tol;           /* stop when the relative increments of psi and of
                                     sum_j c_j h_j between pseudo-iterations are <= tol */
    int32_t poisson_max_iter;     /* iteration cap per solve */
    int32_t poisson_check_every;  /* residual evaluated every this many iterations (solver 2:
                                     a coarse correction every this many, the residual
                                     max(2, this / 16) times in between) */
    int32_t poisson_fixed_iter;   /* > 0: exactly this many iterations, no residual */
    int32_t _pad2;
    /* precision 3 and 4 only: the parameter each tangent direction (3, or the
     * first only for precision 4) differentiates (-1 none; 0 V_top; 1, 2, 3 eps[0..2]; 4, 5, 6 gamma12,
     * gamma13, gamma23).  Fields are then available per direction (see
     * LB3E_TANGENT). */
    int32_t tangent_param[3];
    /* 0: the paper's pseudo-time LB potential solve (Eq. 42-45), h in the build's
     *    precision;
     * 1: geometric multigrid on the finite-difference form of Eq. 27d (5-point,
     *    harmonic-mean faces, half-cell Dirichlet electrodes; bc_y = 2, even nx,
     *    precision <= 2), FP64, V-cycles until the relative residual is <=
     *    poisson_tol (at most poisson_max_iter cycles); E is then the Eq. 33
     *    gradient of psi;
     * 2: the LB solve of Eq. 42-45 (same fixed point as 0) with h held as an FP64
     *    anchor plus a correction in the build's precision, and a multigrid coarse
     *    correction every poisson_check_every iterations (the increment is checked
     *    max(2, poisson_check_every / 16) times a cycle, the last check feeding it): the
     *    residual of the macroscopic equation, read from the LB increment, drives
     *    one FP32 V-cycle of the finite-difference operator whose solution enters h
     *    as its local equilibrium.  The stopping test is the LB increment of 0,
     *    taken in FP64 (bc_y = 2, even nx, precision <= 2);
     * 3: as 2 without the coarse correction (the plain pseudo-time iteration on an
     *    FP64 anchor; precision <= 2).
     * With poisson_fixed_iter > 0, solvers 2 and 3 run exactly that many plain
     * pseudo-iterations (no corrections).  Solvers 0, 2 and 3 stop, not converged,
     * when the residual stalls (no 1% gain over 32 checks; 8 for solver 2). */
    int32_t potential_solver;
    /* 1: two Nernst-Planck ion species (Eq. 52; Section 5.1's electro-osmotic
     * check) carry the charge, q = ion_charge * sum_i ion_z[i] n_i, in place of the
     * closure charge of Eq. 46-50 (whose populations still evolve, unread).  Each
     * species is a D2Q9 set of the charge scheme's form: equilibrium w_j n_i (1 +
     * c_j . v_i / cs^2) with v_i = u + ion_z[i] ion_beta ion_D[i] E, the backward-
     * difference source T_j of d/dt(n_i v_i), tau_i = 1/2 + ion_D[i]/cs^2, bounce-
     * back at walls.  Concentrations start at 0; set them with lb3e_set_ions.
     * Precisions 0-2, single lattices (not batches). */
    int32_t ions;
    int32_t _pad3;
    double ion_D[2];              /* diffusivities (> 0 when ions = 1) */
    double ion_z[2];              /* valences */
    double ion_beta;              /* e / (k_B T): inverse thermal voltage, lattice units */
    double ion_charge;            /* charge per unit concentration */
    /* >= 2: the three-dimensional step on the D3Q15 lattice (Eq. 32) over nx x ny x nz
     * cells, arrays [..][nz][ny][nx].  x and y are periodic; bc_y then gives the
     * boundary of the walls normal to z (at z = -1/2 and nz - 1/2; electrodes V_bottom,
     * V_top; wall speeds along x), E_ext = (along x, along z).  The potential source
     * is split evenly over the 14 moving directions.  Precisions 0 and 1, the LB
     * potential solve, no ions, no population noise, no snapshots, single lattices.
     * 0 or 1: the two-dimensional D2Q9 step. */
    int32_t nz;
    int32_t _pad4;
} lb3e_params;

/* Field id offset of tangent k (1..3) of a field in the tangent builds: field
 * f's derivative along direction k is field f + k * LB3E_TANGENT. */
#define LB3E_TANGENT 1000

typedef struct lb3e_observables_t {
    double mass[3];          /* sum phi_i of the last step */
    double charge;           /* sum q of the last step */
    double free_energy[4];   /* Eq. 18 parts: phase (bulk + gradient), electric, kinetic, charge */
    double max_sum_dev;      /* max |phi_1 + phi_2 + phi_3 - 1| */
    double D_inner, D_outer; /* deformation factors from second moments of the indicators */
    double poisson_residual; /* residual at the last check of the last solve (-1: none) */
    int64_t nonfinite;       /* non-finite phi, u or q values */
    int64_t step;            /* completed time steps */
    int32_t poisson_iters;   /* iterations of the last solve */
    int32_t poisson_converged; /* 1 reached poisson_tol (or a fixed count ran); 0 hit the
                                  iteration cap; -1 stopped on a stalled residual */
} lb3e_observables_t;

typedef struct lb3e_handle lb3e_handle;

/* Device bytes lb3e_init() needs for these parameters.  Errors: PARAM, NULL. */
int lb3e_workspace_bytes(const lb3e_params* params, size_t* bytes);

/* Validate params, lay out the workspace (256-byte aligned, >= the size above),
 * build the initial state and solve the initial potential (with the initial
 * charge).  Initial state: phi_i = phi_init ([3][ny][nx], required), u = u_init
 * ([2][ny][nx] or NULL = 0), q = q_init ([ny][nx] or NULL = 0), p = 0; phase
 * populations at equilibrium with mu_i of Eq. 20, flow at g_eq(p = 0, u), charge
 * at l_eq(q, u); then pop_noise ([5][9][ny][nx] for sets g, f1, f2, f3, l, or
 * NULL) is added.  Errors: PARAM, WORKSPACE, NULL, CUDA (a non-converged initial
 * solve is not an error; see lb3e_observables). */
int lb3e_init(const lb3e_params* params, void* workspace, size_t workspace_bytes,
              const double* phi_init, const double* u_init, const double* q_init,
              const double* pop_noise, void* stream, lb3e_handle** out);

/* Advance nsteps time steps.  A potential solve that reaches poisson_max_iter
 * does not stop the run; lb3e_observables() reports its iterations and
 * residual.  Errors: NULL, PARAM (nsteps < 0), CUDA. */
int lb3e_step(lb3e_handle* h, int32_t nsteps);

/* Run the potential solve alone (Eq. 42-45) for the permittivity of the last
 * step and the charge q (device or host [ny][nx], or NULL for the stored q),
 * updating h, psi and E.  Returns NOT_CONVERGED if max_iter was reached.
 * *iters and *residual (may be NULL) receive the iteration count and the last
 * residual. */
int lb3e_solve_potential(lb3e_handle* h, const double* q, double tol, int32_t max_iter,
                         int32_t check_every, int32_t* iters, double* residual);

/* Reductions over the last step's fields: per-cell terms in the build's
 * precision, every sum and the max in FP64.  Synchronises the stream. */
int lb3e_observables(lb3e_handle* h, lb3e_observables_t* out);

/* Copy one field (see the LB3E_FIELD_* ids) as doubles into dst ([ny][nx],
 * host or device).  Synchronises the stream.  Errors: NULL, FIELD, CUDA. */
int lb3e_get_field(lb3e_handle* h, int32_t field_id, double* dst);

/* Size of a full state snapshot (populations, potential populations, fields,
 * d/dt history, ion state when ions = 1, step counter) and save/load to caller
 * memory (host or device). */
int lb3e_state_bytes(const lb3e_handle* h, size_t* bytes);
int lb3e_save_state(lb3e_handle* h, void* dst);
int lb3e_load_state(lb3e_handle* h, const void* src);

/* Deformation factors D = (a - b)/(a + b) (Section 5.3's measure, radii from the
 * second moments of the indicator: a = 2 sqrt(Iyy) along the field, b = 2 sqrt(Ixx)
 * across it) of the phases of the current populations (phi_i = sum_j f^i_j, as the
 * PHINOW fields): D[0] of phi_inner, D[1] of 1 - phi_matrix.  In the tangent builds
 * (precision 3, 4) also their derivatives along each tangent direction: dD[3 k + t]
 * is dD[k]/d(parameter of direction t) (0 for directions a build does not carry);
 * plain builds set dD to 0.  dD may be NULL.  The moments are FP64 sums on the GPU;
 * D and dD are formed from them on the host.  Synchronises the stream.
 * Errors: NULL, PARAM (three-dimensional lattices), CUDA. */
int lb3e_deformation(lb3e_handle* h, double* D, double* dD);

/* Target interface shape: J = sum over the three phases and all cells of
 * (phi_i - phi_target_i)^2, phi_i of the current populations, phi_target
 * [3][ny][nx] doubles (host or device).  In the tangent builds also dJ[t] =
 * dJ/d(parameter of tangent direction t) = sum 2 (phi_i - phi_target_i)
 * dphi_i/dtheta_t, t = 0..2 (0 for directions a build does not carry; plain builds
 * set dJ to 0).  dJ may be NULL.  FP64 sums on the GPU.  Synchronises the stream.
 * Errors: NULL, PARAM (three-dimensional lattices), CUDA. */
int lb3e_shape_objective(lb3e_handle* h, const double* phi_target, double* J, double* dJ);

/* ---------------------------------------------------------------- reverse mode
 * The adjoint of the step: for an objective J of a later state, the derivative of J
 * with respect to the state before a step and to the model parameters, one step at a
 * time backwards (the chain rule through the step of Section 3 and the state's
 * creation).  Two-dimensional plain builds (precision 0 FP64, 1 FP32, 2 and 5 with
 * FP32 arithmetic) without ion transport, and, with electric = 1, the LB potential
 * (potential_solver 0) run for a fixed count of pseudo-time iterations
 * (poisson_fixed_iter > 0, Eq. 43): the count is part of the discrete step, while a
 * residual-controlled solve stops on a decision with no derivative.  Anything else
 * returns LB3E_ERR_UNSUPPORTED.
 *
 * The state vector X (device memory, 64 planes of N values in the build's
 * arithmetic type: double for precision 0, float otherwise; plane k is the [ny][nx]
 * array at offset k N):  g_j 0-8, f^i_j 9-35 (phase-major), l_j 36-44, h_j 45-53
 * (the potential populations the next solve starts from), E 54-55 (x, y; the field
 * the next step's charge closure reads), (phi_i u)^{n-1} 56-61 (x, y per phase),
 * (q u)^{n-1} 62-63.  The phase rest populations are the full f^i_0 (the storage's
 * deviation form rebuilt).  An adjoint a has the same layout: a = dJ/dX.
 *
 * Parameter slots of dparams (11 doubles, host, added to):  V_bottom, V_top,
 * eps_1, eps_2, eps_3, sigma_1, sigma_2, sigma_3, gamma_12, gamma_13, gamma_23.  The
 * electric field strength E0 enters through V_top = V_bottom + E0 ny.
 *
 * The adjoint needs a caller-owned device workspace (lb3e_adjoint_workspace_bytes,
 * 256-byte aligned): the re-computed intermediates of one step, every potential
 * iterate included, and the adjoint's scratch planes.  All calls run on the
 * handle's stream and synchronise it before returning. */

/* Bytes of the adjoint workspace of this handle's configuration.
 * Errors: NULL, UNSUPPORTED. */
int lb3e_adjoint_workspace_bytes(const lb3e_handle* h, size_t* bytes);

/* Write the current state vector X (layout above) to dst (device, 64 N values), in
 * stream order (no synchronisation).  *first = 1 while the handle's state is the
 * created one (its step has no d/dt terms), else 0.
 * Errors: NULL, UNSUPPORTED, CUDA. */
int lb3e_state_vector(lb3e_handle* h, void* dst);
int lb3e_is_first_step(const lb3e_handle* h, int32_t* first);

/* One step backwards.  saved_state: a snapshot of the state X^n before the step, as
 * lb3e_save_state wrote it (host or device), which replaces the handle's state; NULL
 * takes the handle's current state as X^n.  adj_in = dJ/dX^{n+1} and adj_out =
 * dJ/dX^n (device, 64 N values each, distinct buffers); dparams[11] += dJ/dtheta
 * through this step.  The step is re-run from X^n to recover its intermediates (the
 * moments, properties, stencils, charge, each potential iterate, the field, the
 * chemical potential, force and flow moments), then every statement of the step is
 * transposed in reverse order.
 * Errors: NULL, UNSUPPORTED, WORKSPACE, CUDA. */
int lb3e_adjoint_step(lb3e_handle* h, const void* saved_state, const void* adj_in, void* adj_out,
                      double* dparams, void* adj_workspace, size_t adj_bytes);

/* The same step backwards from a state vector X^n (device, as lb3e_state_vector
 * wrote it before the step) instead of a snapshot; first = 1 for the step from the
 * created state.  The handle's state is not touched.  dparams may be device memory
 * (11 doubles): it is then accumulated in stream order and the call returns without
 * synchronising, so a backward sweep needs no host round trip; a host dparams
 * synchronises as in lb3e_adjoint_step.  On a stream other than the legacy default
 * stream the step's kernels are captured once per (workspace, adj_in, adj_out,
 * first, dparams) as a CUDA graph (the last 8 are kept) and replayed.
 * Errors: NULL, UNSUPPORTED, WORKSPACE, CUDA. */
int lb3e_adjoint_step_x(lb3e_handle* h, const void* X, int32_t first, const void* adj_in, void* adj_out,
                        double* dparams, void* adj_workspace, size_t adj_bytes);

/* The state's creation backwards: with adj_in = dJ/dX^0, dparams[11] += dJ/dtheta
 * through the creation from phi_init (the initial populations at equilibrium with
 * phi, zero velocity and charge, the potential iterated poisson_fixed_iter times
 * from the linear electrode profile), and, if dphi_init is not NULL, dphi_init
 * [3][ny][nx] doubles (host or device) += dJ/dphi_init.  phi_init [3][ny][nx]
 * doubles, host or device, as given to lb3e_init.  The handle's state is left as it
 * was.  Errors: NULL, UNSUPPORTED, WORKSPACE, CUDA. */
int lb3e_adjoint_init(lb3e_handle* h, const double* phi_init, const void* adj_in, double* dparams,
                      double* dphi_init, void* adj_workspace, size_t adj_bytes);

/* Seeds of the two objectives of the current populations' phases: D of
 * lb3e_deformation (which = 0 inner, 1 outer) and the shape objective J of
 * lb3e_shape_objective; *D or *J gets the value and adj_out (device, 64 N values) the
 * state-vector adjoint dD/dX or dJ/dX (nonzero on the f planes only, since phi_i =
 * sum_j f^i_j).  Errors: NULL, PARAM (which), UNSUPPORTED, CUDA. */
int lb3e_deformation_seed(lb3e_handle* h, int32_t which, double* D, void* adj_out);
int lb3e_shape_seed(lb3e_handle* h, const double* phi_target, double* J, void* adj_out);

/* Potential solves since the previous call (or lb3e_init): how many ran, how many
 * ended above the tolerance (iteration cap or a stalled residual), and the largest
 * final residual among them (-1: none taken, e.g. fixed counts).  Host counters:
 * no synchronisation.  The counters are then cleared.  Errors: NULL. */
int lb3e_potential_stats(lb3e_handle* h, int64_t* solves, int64_t* not_converged, double* max_residual);

/* Diagnostic for the potential of the last solve: ||b - A psi|| / ||b|| (FP64) with
 * A psi = b the finite-difference form of div(eps grad psi) + q = 0 (5-point
 * stencil, harmonic-mean faces; electrodes as Dirichlet faces at half a cell, b = q
 * plus their 2 eps V terms; plain walls carry no flux), for this step's eps and q.
 * For the LB solvers it measures how close the LB fixed point is to that
 * discretisation (they differ at second order); for solver 1 it is the solve's own
 * residual.  Synchronises the stream.  Errors: NULL, PARAM (electric = 0, a tangent
 * build, or a three-dimensional lattice), CUDA. */
int lb3e_potential_fd_residual(lb3e_handle* h, double* residual);

/* Start the Nernst-Planck ion species (ions = 1) from the concentrations n_init
 * ([2][ny][nx] doubles, host or device; species-major): their charge replaces q,
 * the potential is solved for it as lb3e_init solves it, and each ion set starts at
 * its equilibrium with the initial u and that field.  Only before the first step.
 * Errors: NULL, PARAM (ions = 0, a step already taken, or a tangent build), CUDA. */
int lb3e_set_ions(lb3e_handle* h, const double* n_init);

/* Number of kernel launches issued since lb3e_init (for launch accounting). */
int64_t lb3e_launch_count(const lb3e_handle* h);

/* Pseudo-iterations of the potential solve (Eq. 43) executed since lb3e_init,
 * over all solves (a launch may run several). */
int64_t lb3e_potential_iterations(const lb3e_handle* h);

/* Pseudo-iterations of the LB potential solve (Eq. 43) per kernel launch: 1
 * (one launch per iteration), 2 (temporally blocked on a tile with a 2-cell
 * halo), 3..4 (4-cell halo; the default is 4) or 5..8 (8-cell halo).  The
 * per-cell arithmetic is the same for every choice (FP64 states agree bitwise);
 * the speed differs.  Dual-number precisions accept only 1.
 * Errors: NULL, PARAM (out of range). */
int lb3e_set_potential_chunk(lb3e_handle* h, int32_t iterations_per_launch);

/* Tile of the fused chemical-potential/force/collide/stream pass: blocks of 32 x rows
 * cells, rows 4 (the default in the FP32-compute precisions), 8 (the default
 * otherwise) or 16 (FP32-compute precisions only; 8 only in the tangent builds).  The per-cell arithmetic is the same for every tile (FP64
 * states agree bitwise); the speed differs.  Errors: NULL, PARAM (another height, a
 * three-dimensional lattice). */
int lb3e_set_fused_tile(lb3e_handle* h, int32_t rows);

/* Input staging of the three-dimensional (D3Q15) potential iteration (Eq. 43):
 * planes >= 1 (2 by default) copies each plane's 15 population boxes, eps and q into
 * shared memory with the tensor memory accelerator, each block walking `planes`
 * consecutive z planes of its 32 x 8 tile, where the lattice allows it (FP32, nx a
 * multiple of 4) and the iteration neither checks nor saves its increment; 0 loads
 * every input per thread.  The per-cell arithmetic is the same; the states agree
 * bitwise.  Errors: NULL, PARAM (planes outside 0..1024), UNSUPPORTED (a
 * two-dimensional lattice). */
int lb3e_set_staging(lb3e_handle* h, int32_t planes);

/* Kernel timing with CUDA events recorded on the simulation's stream around each
 * launch (off by default; costs two event records per launch).  Enabling or
 * disabling clears the totals. */
int lb3e_set_timing(lb3e_handle* h, int32_t enable);

/* Kernel classes reported by lb3e_kernel_times. */
enum {
    LB3E_KC_MOMENTS = 0,   /* zeroth moments of the phase and charge populations, with the
                              properties, stencils and closed-form charge in the same pass */
    LB3E_KC_PROLOGUE = 1,  /* properties and stencils alone (initialisation, batches) */
    LB3E_KC_POISSON = 2,   /* potential solve: LB pseudo-iterations (one or several per launch) or multigrid */
    LB3E_KC_REDUCE = 3,    /* FP64 reductions (residual, observables) */
    LB3E_KC_FIELDS = 4,    /* psi and E from the potential populations */
    LB3E_KC_FUSED = 5,     /* fused chemical potential, force, collide and stream */
    LB3E_KC_OTHER = 6,     /* initialisation and conversions */
    LB3E_KC_IONS = 7,      /* Nernst-Planck ion moments, collision and streaming */
    LB3E_KC_ANCHOR = 8,    /* potential solvers 2, 3: FP64 anchor refresh (fold, increment) */
    LB3E_KC_COARSE = 9,    /* potential solver 2: the multigrid coarse correction */
    LB3E_KC_COUNT = 10
};

/* Synchronise the stream and return, per kernel class, the summed event time in
 * milliseconds (ms[LB3E_KC_COUNT]) and the number of timed launches
 * (launches[LB3E_KC_COUNT]) since the last call; the totals are then cleared. */
int lb3e_kernel_times(lb3e_handle* h, double* ms, int64_t* launches);

/* ---- Batches: many lattices stepped together (parameter sweeps) ----
 * Instances of one precision, each with its own size and parameters, are
 * advanced in lockstep: every kernel of a time step is one launch over the tiles
 * of all instances, and pairs of steps are replayed as one CUDA graph.  Every
 * instance with electric = 1 must use the same poisson_fixed_iter (> 0): the
 * potential is iterated a fixed number of times per step, so all instances do
 * the same work and the graph is fixed (graphs are used only on a created stream:
 * the legacy default stream cannot be captured, and there every step is plain
 * launches).  Each instance starts as lb3e_init would
 * start it with u = q = 0 and no noise.  The device workspace is the caller's. */
typedef struct lb3e_batch lb3e_batch;

/* Device bytes for n instances (params[n]).  Errors: NULL, PARAM. */
int lb3e_batch_workspace_bytes(const lb3e_params* params, int32_t n, size_t* bytes);

/* Create and initialise n instances; phi_init[i] is instance i's [3][ny][nx]
 * phase field (host or device).  Errors: NULL, PARAM, WORKSPACE, CUDA. */
int lb3e_batch_create(const lb3e_params* params, int32_t n, const double* const* phi_init, void* workspace,
                      size_t workspace_bytes, void* stream, lb3e_batch** out);

/* Advance every instance nsteps time steps (synchronises the stream). */
int lb3e_batch_run(lb3e_batch* b, int32_t nsteps);

/* Observables of every instance into out[n] (D_inner, D_outer, ...). */
int lb3e_batch_observables(lb3e_batch* b, lb3e_observables_t* out);

/* One field of one instance, as lb3e_get_field. */
int lb3e_batch_get_field(lb3e_batch* b, int32_t instance, int32_t field_id, double* dst);

/* Pseudo-iterations of the potential per launch for this batch: 1 (one launch
 * per iteration) up to 8 (temporally blocked: several iterations on a tile held
 * in shared memory).  The result does not depend on it; the speed does.
 * Errors: NULL, PARAM (out of range), CUDA. */
int lb3e_batch_set_potential_chunk(lb3e_batch* b, int32_t iterations_per_launch);

/* Tile of the batch's fused chemical-potential/force/collide/stream pass: blocks of
 * 32 x rows cells, rows 4, 8 (the default) or 16 (FP32-compute precisions only).  The
 * result does not depend on it (the per-cell arithmetic is the same); the speed does
 * -- shared memory per block, blocks per SM and the halo overhead change with it.
 * Errors: NULL, PARAM (another height), CUDA. */
int lb3e_batch_set_fused_tile(lb3e_batch* b, int32_t rows);

/* Kernel launches issued for this batch (graph nodes counted per replay). */
int64_t lb3e_batch_launch_count(const lb3e_batch* b);

void lb3e_batch_destroy(lb3e_batch* b);

/* Largest lattice (nx * ny cells) lb3e_observables_noalloc accepts. */
#define LB3E_NOALLOC_MAX_CELLS (2048 * 2048)

/* The reductions of lb3e_observables for callers that cannot allocate device
 * memory -- for instance code running under a memory pool that must not grow,
 * inside an allocator owned by another framework, or in a monitoring hook that
 * must leave the caller's memory untouched.  The paper has no counterpart: this is
 * a deployment convenience around the same FP64 reductions.
 *
 * Inputs are the caller's FP64 device fields of one lattice: phi [3][ny][nx],
 * q [ny][nx], E [2][ny][nx], u [2][ny][nx]; params gives nx, ny, bc_y, the
 * phase properties, width_D and inner/matrix_phase.  No handle or workspace is
 * used and nothing is allocated: the scratch is a fixed array of the library
 * (about 2.5 MB per GPU that loads the library, held until the process exits).
 * Results are written to *out (host); poisson_* and step are left at -1 / 0.
 *
 * The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current); make that first call before
 * any stream capture.  All calls share the one array, so calls that overlap on
 * the GPU (different streams or threads, same device) race; serialise them.
 * Each call overwrites what the previous one left there.
 * params is checked as lb3e_init checks it; the arrays are not checked: each must
 * hold the stated number of doubles for params' nx and ny, on the current device.
 * Errors: NULL, PARAM (a field lb3e_init rejects, or nz >= 2), TOO_LARGE (nx * ny >
 * LB3E_NOALLOC_MAX_CELLS), CUDA.
 * Synchronises `stream`. */
int lb3e_observables_noalloc(const lb3e_params* params, const double* phi, const double* q,
                             const double* E, const double* u, void* stream,
                             lb3e_observables_t* out);

/* Release the host-side handle (the workspace stays the caller's). */
void lb3e_destroy(lb3e_handle* h);

/* Static description of a status code. */
const char* lb3e_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* LB3E_H */
