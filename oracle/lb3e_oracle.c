/*
 * lb3e_oracle.c -- plain FP64 CPU oracle of the three-phase EHD lattice Boltzmann
 * step (Liu, Qian, Xiong, Wang: Onsager-variational LB model for three-phase
 * dielectric fluid flows).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the GPU path computes.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header or constant
 * generator with the CUDA library.
 *
 * Everything is double precision, one cell at a time, in the order of the paper's
 * Section 3: moments, property interpolation (Eq. 29-30), isotropic stencils
 * (Eq. 33), the potential solve (Eq. 42-45), the chemical potential (Eq. 20), the
 * capillary + Coulomb force (Eq. 26/27b), flow moments (Eq. 41), then collision of
 * the phase (Eq. 34-36), flow (Eq. 37-40) and charge (Eq. 46-50) populations and
 * streaming.  Build with -ffp-contract=off so no multiply-add is fused.
 *
 * Readings where the paper is silent or garbled (each is listed in the design
 * notes):  chemical potential from Eq. 20, not the energy density printed in
 * Eq. 27c;  source F_j^i of Eq. 36 read as w_j c_j . [...] (the mobility part is a
 * flux, so it carries c_j);  the implicit charge q = sum l + R/2 solved in closed
 * form with the previous step's field;  d/dt terms as first-order backward
 * differences;  half-way walls at y = -1/2 and ny - 1/2 with mirrored stencil
 * ghosts;  electrodes applied by anti-bounce-back of the potential populations;
 * potential iterations stopped on the relative increments of the potential and
 * of the first moment of h (which carries the field).
 *
 * Optional ion transport (Eq. 52, the electro-osmotic validation of Section 5.1):
 * two species with concentrations n_i obey the Nernst-Planck equation.  Each is
 * carried by its own D2Q9 population set with the structure of the charge scheme of
 * Eq. 48-50: equilibrium w_j n_i (1 + c_j . v_i / cs2) with the drift velocity
 * v_i = u + z_i beta D_i E (advection plus migration along E), the same first-order
 * d/dt(n_i v_i) correction T_j, relaxation tau_i = 1/2 + D_i/cs2, and plain
 * bounce-back (no flux) at walls.  The charge is then q = e_q sum_i z_i n_i and
 * replaces the transported charge of Eq. 46-50.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- D2Q9 lattice, Eq. 31 ---------------- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#define CS2 (1.0 / 3.0) /* lattice sound speed squared, Section 3.1 */

/* parameter block; field meanings follow the paper's notation */
typedef struct orc_params {
    int32_t nx, ny;
    int32_t bc_y;              /* 0 periodic, 1 walls, 2 walls + electrodes */
    int32_t electric;          /* 1: potential solved each step */
    double rho[3], visc[3];    /* Eq. 29 */
    double tau_g;              /* used when every visc <= 0 */
    double gamma12, gamma13, gamma23; /* Eq. 9 */
    double width_D;            /* interface width D, Eq. 7 */
    double tau_f;              /* m0 = cs2 (tau_f - 1/2), Section 3.2 */
    double eps[3], sigma[3];   /* Eq. 29-30 */
    double eps_ref;            /* the constant part of the permittivity split, Eq. 42 */
    double alpha;              /* charge diffusivity, tau_l = 1/2 + alpha/cs2 */
    double V_bottom, V_top;    /* electrode potentials at y = -1/2 and ny - 1/2 */
    double E_ext[2];           /* uniform external field added to -grad psi */
    double u_wall_bottom, u_wall_top;
    int32_t charge_convection; /* 1: u-terms in l_eq and T_j (Eq. 49-50) */
    int32_t inner_phase, matrix_phase; /* 1-based, for the deformation factor */
    double poisson_tol;
    int32_t poisson_max_iter, poisson_check_every, poisson_fixed_iter;
    int32_t potential_solver;  /* 0: the LB pseudo-time solve (Eq. 42-45); 1: the
                                  finite-difference form of Eq. 27d solved directly */
    double debye_kappa2;       /* > 0: validation closure for the electro-osmotic channel
                                  (Section 5.1): the charge is the linearised Boltzmann
                                  (Debye-Hueckel) response q = -eps kappa^2 psi instead of
                                  the transported charge; 0: the method as stated */
    int32_t ions;              /* 1: two Nernst-Planck ion species carry the charge (Eq. 52) */
    double ion_D[2];           /* diffusivities D_i (lattice units) */
    double ion_z[2];           /* valences z_i */
    double ion_beta;           /* e / (k_B T) in lattice units: the inverse thermal voltage */
    double ion_charge;         /* charge per unit concentration: q = ion_charge sum_i z_i n_i */
} orc_params;

enum { F_PHI1 = 0, F_PHI2, F_PHI3, F_UX, F_UY, F_P, F_Q, F_PSI, F_EX, F_EY,
       F_MU1, F_MU2, F_MU3, F_PHINOW1, F_PHINOW2, F_PHINOW3, F_QTILDE, F_N1, F_N2, F_NFIELDS };
enum { POP_BASE = 100 }; /* POP_BASE + 9*set + j, sets: g, f1, f2, f3, l, h, n1, n2 */

typedef struct orc_state {
    orc_params p;
    int N;
    double lam[3], m0, tau_h, tau_l;
    /* populations at the start of a step (post-stream), and post-collision scratch */
    double *g, *f, *l, *h;       /* g[9N], f[27N] (set-major), l[9N], h[9N] */
    double *gs, *fs, *ls, *hs;
    /* fields of the last completed step */
    double *phi, *qt, *q, *rho, *sig, *eps, *lap, *geps, *gsig, *grho;
    double *E, *psi, *mu, *gmu, *F, *u, *pr, *R;
    double *prev_phiu, *prev_qu;  /* (phi_i u)^{n-1}, (q u)^{n-1} */
    double *ion, *ions_s;         /* ion populations n^i_j [18N] and post-collision scratch */
    double *nion, *prev_nv;       /* n_i [2N] of the step, (n_i v_i)^{n-1} [4N] */
    double tau_ion[2];
    double *psi_prev, *J_prev;    /* psi and J at the previous pseudo-iteration */
    int64_t step;
    int last_iters;
    double last_res;
    int last_converged;
} orc_state;

static double* alloc0(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

/* ---------------- grid helpers ---------------- */
static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* Stencil ghost rows: periodic in y, or the mirror image about a half-way wall
 * (zero normal gradient of every stencilled field). */
static int ghost_y(const orc_state* s, int y) {
    int ny = s->p.ny;
    if (s->p.bc_y == 0) return wrap(y, ny);
    if (y < 0) return -1 - y;
    if (y >= ny) return 2 * ny - 1 - y;
    return y;
}
static double at(const orc_state* s, const double* fld, int x, int y) {
    return fld[ghost_y(s, y) * s->p.nx + wrap(x, s->p.nx)];
}

/* Eq. 33: grad chi = sum_j w_j c_j chi(x + c_j) / cs2 */
static void grad_at(const orc_state* s, const double* fld, int x, int y, double* gx, double* gy) {
    double ax = 0.0, ay = 0.0;
    for (int j = 0; j < 9; ++j) {
        double v = at(s, fld, x + CX[j], y + CY[j]);
        ax += W[j] * CX[j] * v;
        ay += W[j] * CY[j] * v;
    }
    *gx = ax / CS2;
    *gy = ay / CS2;
}
/* Eq. 33: lap chi = sum_j 2 w_j [chi(x + c_j) - chi(x)] / cs2 */
static double lap_at(const orc_state* s, const double* fld, int x, int y) {
    double c = at(s, fld, x, y), a = 0.0;
    for (int j = 0; j < 9; ++j) a += 2.0 * W[j] * (at(s, fld, x + CX[j], y + CY[j]) - c);
    return a / CS2;
}

/* ---------------- closures ---------------- */
/* Eq. 30: eps = sum eps_i H(phi_i), H = phi^2 (3 - 2 phi) */
static double perm(const orc_params* p, const double* ph) {
    double e = 0.0;
    for (int i = 0; i < 3; ++i) e += p->eps[i] * ph[i] * ph[i] * (3.0 - 2.0 * ph[i]);
    return e;
}
static int use_visc(const orc_params* p) { return p->visc[0] > 0 && p->visc[1] > 0 && p->visc[2] > 0; }

/* gather phi_i(x) of the last moments into a small array */
static void phis(const orc_state* s, int c, double* ph) {
    for (int i = 0; i < 3; ++i) ph[i] = s->phi[i * s->N + c];
}

/* ---------------- potential solve, Eq. 42-45 ---------------- */
static double psi_moment(const orc_state* s, const double* h, int c) {
    double a = 0.0;
    for (int j = 1; j < 9; ++j) a += h[j * s->N + c];
    return a / (1.0 - W[0]);                       /* Eq. 45 */
}
static void gradpsi_moment(const orc_state* s, const double* h, int c, double epshat,
                           double* gx, double* gy) {
    double ax = 0.0, ay = 0.0;
    for (int j = 0; j < 9; ++j) {
        ax += CX[j] * h[j * s->N + c];
        ay += CY[j] * h[j * s->N + c];
    }
    double den = epshat + CS2 * s->tau_h;          /* Eq. 45 (Delta t = 1) */
    *gx = -ax / den;
    *gy = -ay / den;
}

/* stream post-collision populations `src` into `dst` (Section 3, streaming step),
 * periodic in x; in y periodic or half-way bounce-back.  kind: 0 plain
 * bounce-back, 1 flow (moving wall, needs rho), 2 potential (anti-bounce-back to the
 * electrode potential when bc_y == 2, plain bounce-back otherwise). */
static void stream(const orc_state* s, const double* src, double* dst, int kind) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            for (int j = 0; j < 9; ++j) {
                double v = src[j * N + c];
                int yt = y + CY[j];
                if (s->p.bc_y != 0 && (yt < 0 || yt >= ny)) {
                    int top = yt >= ny;
                    double out = v;
                    if (kind == 1) {
                        double uw = top ? s->p.u_wall_top : s->p.u_wall_bottom;
                        out = v - 2.0 * W[j] * s->rho[c] * (CX[j] * uw) / CS2;
                    } else if (kind == 2 && s->p.bc_y == 2) {
                        double vw = top ? s->p.V_top : s->p.V_bottom;
                        out = -v + 2.0 * W[j] * vw;
                    }
                    dst[OPP[j] * N + c] = out;
                } else {
                    int xt = wrap(x + CX[j], nx);
                    dst[j * N + wrap(yt, ny) * nx + xt] = v;
                }
            }
        }
}

/* One pseudo-time iteration of Eq. 43: collide every cell, then stream. */
static void poisson_iteration(orc_state* s) {
    const int N = s->N;
    const double th = s->tau_h;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; ++c) {
        double epshat = s->eps[c] - s->p.eps_ref;
        double psi = psi_moment(s, s->h, c);
        double gx, gy;
        gradpsi_moment(s, s->h, c, epshat, &gx, &gy);
        /* the Debye-Hueckel closure follows the current iterate of psi */
        double qc = s->p.debye_kappa2 > 0.0 ? -s->eps[c] * s->p.debye_kappa2 * psi : s->q[c];
        for (int j = 0; j < 9; ++j) {
            double heq = (j == 0) ? (W[0] - 1.0) * psi : W[j] * psi;      /* Eq. 44 */
            double varpi = (j == 0) ? 0.0 : 1.0 / 8.0;
            double hj = s->h[j * N + c];
            double cg = CX[j] * gx + CY[j] * gy;
            s->hs[j * N + c] = hj - (hj - heq) / th - (epshat / CS2) * W[j] * cg / th + varpi * qc;
        }
    }
    stream(s, s->hs, s->h, 2);
}

/* first moment J = sum_j c_j h_j (E = J / (epshat + cs2 tau_h), Eq. 45) */
static void first_moment(const orc_state* s, const double* h, int c, double* jx, double* jy) {
    double ax = 0.0, ay = 0.0;
    for (int j = 0; j < 9; ++j) {
        ax += CX[j] * h[j * s->N + c];
        ay += CY[j] * h[j * s->N + c];
    }
    *jx = ax;
    *jy = ay;
}

/* Iterate until the relative increments of psi and of the first moment J between
 * consecutive pseudo-iterations are both <= tol (checked every check_every
 * iterations, before the collision of that iteration), or a fixed number of
 * iterations.  A solve whose best residual has not fallen by 1% over 32
 * consecutive checks stops there, not converged (*converged = -1): a residual that
 * stalls (a drifting null mode on a lattice without electrodes, a rounding floor)
 * does not spin to the cap.  Returns the number of collide+stream iterations
 * applied. */
static int poisson_solve(orc_state* s, double tol, int max_iter, int fixed, int check,
                         double* res, int* converged) {
    const int N = s->N;
    int n = fixed > 0 ? fixed : max_iter;
    if (check < 1) check = 1;
    *res = -1.0;
    *converged = fixed > 0;
    double best = INFINITY;
    int since_best = 0;
    for (int k = 1; k <= n; ++k) {
        if (fixed <= 0 && k >= 2 && k % check == 0) {
            double dp = 0.0, pp = 0.0, dj = 0.0, jj = 0.0;
            for (int c = 0; c < N; ++c) {
                double pk = psi_moment(s, s->h, c), jx, jy;
                first_moment(s, s->h, c, &jx, &jy);
                double d = pk - s->psi_prev[c];
                double ex = jx - s->J_prev[c], ey = jy - s->J_prev[N + c];
                dp += d * d;
                pp += pk * pk;
                dj += ex * ex + ey * ey;
                jj += jx * jx + jy * jy;
            }
            double r1 = pp > 0.0 ? sqrt(dp) / sqrt(pp) : (dp > 0.0 ? INFINITY : 0.0);
            double r2 = jj > 0.0 ? sqrt(dj) / sqrt(jj) : (dj > 0.0 ? INFINITY : 0.0);
            double r = r1 > r2 ? r1 : r2;
            *res = r;
            if (r <= tol) { *converged = 1; return k - 1; }
            if (r < 0.99 * best) {
                best = r;
                since_best = 0;
            } else if (++since_best >= 32) {
                *converged = -1;
                return k - 1;
            }
        }
        if (fixed <= 0 && (k + 1) % check == 0)
            for (int c = 0; c < N; ++c) {
                s->psi_prev[c] = psi_moment(s, s->h, c);
                first_moment(s, s->h, c, &s->J_prev[c], &s->J_prev[N + c]);
            }
        poisson_iteration(s);
    }
    return n;
}

/* psi and E = -grad psi (+ external field) from the current potential populations */
static void potential_fields(orc_state* s) {
    for (int c = 0; c < s->N; ++c) {
        double gx, gy;
        s->psi[c] = psi_moment(s, s->h, c);
        gradpsi_moment(s, s->h, c, s->eps[c] - s->p.eps_ref, &gx, &gy);
        s->E[c] = -gx + s->p.E_ext[0];
        s->E[s->N + c] = -gy + s->p.E_ext[1];
    }
}

/* ---------------- finite-difference potential (alternative solver) ----------------
 * The same equation, div(eps grad psi) + q = 0 (Eq. 27d), discretised with the
 * 5-point stencil: face permittivity = harmonic mean of the two cells; a wall
 * carrying an electrode is a Dirichlet face at distance 1/2 (flux 2 eps_C (V - psi_C));
 * an insulating wall carries no flux; x (and y when bc_y = 0) is periodic.  The
 * symmetric system A psi = b is solved by conjugate gradients to a relative
 * residual of 1e-13 (with no Dirichlet face the mean of q is removed and psi has
 * zero mean).  E is the isotropic gradient of Eq. 33, with ghost cells 2V - psi at
 * electrodes and mirrors at insulating walls. */
static double hmean(double a, double b) { return 2.0 * a * b / (a + b); }

static void fd_apply(const orc_state* s, const double* x, double* Ax) {
    const int nx = s->p.nx, ny = s->p.ny;
    for (int y = 0; y < ny; ++y)
        for (int xx = 0; xx < nx; ++xx) {
            int c = y * nx + xx;
            double ec = s->eps[c], acc = 0.0;
            int nb[4][2] = {{xx + 1, y}, {xx - 1, y}, {xx, y + 1}, {xx, y - 1}};
            for (int k = 0; k < 4; ++k) {
                int yy = nb[k][1];
                if (s->p.bc_y != 0 && (yy < 0 || yy >= ny)) {
                    if (s->p.bc_y == 2) acc += 2.0 * ec * x[c];
                    continue;
                }
                int n = wrap(yy, ny) * nx + wrap(nb[k][0], nx);
                acc += hmean(ec, s->eps[n]) * (x[c] - x[n]);
            }
            Ax[c] = acc;
        }
}

static double dot(const double* a, const double* b, int n) {
    double r = 0.0;
    for (int i = 0; i < n; ++i) r += a[i] * b[i];
    return r;
}

static int fd_solve(orc_state* s, double* res_out) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
    double* b = alloc0(N);
    double* r = alloc0(N);
    double* d = alloc0(N);
    double* Ad = alloc0(N);
    for (int c = 0; c < N; ++c) b[c] = s->q[c];
    if (s->p.bc_y == 2)
        for (int x = 0; x < nx; ++x) {
            b[x] += 2.0 * s->eps[x] * s->p.V_bottom;
            b[(ny - 1) * nx + x] += 2.0 * s->eps[(ny - 1) * nx + x] * s->p.V_top;
        }
    else {
        double m = 0.0;
        for (int c = 0; c < N; ++c) m += b[c];
        for (int c = 0; c < N; ++c) b[c] -= m / N;
    }
    double* x = s->psi;
    fd_apply(s, x, Ad);
    for (int c = 0; c < N; ++c) { r[c] = b[c] - Ad[c]; d[c] = r[c]; }
    double bb = dot(b, b, N), rr = dot(r, r, N);
    int it = 0;
    const double tol2 = 1e-26 * (bb > 0 ? bb : 1.0);
    while (rr > tol2 && it < 100000) {
        fd_apply(s, d, Ad);
        double alpha = rr / dot(d, Ad, N);
        for (int c = 0; c < N; ++c) { x[c] += alpha * d[c]; r[c] -= alpha * Ad[c]; }
        double rr2 = dot(r, r, N);
        for (int c = 0; c < N; ++c) d[c] = r[c] + (rr2 / rr) * d[c];
        rr = rr2;
        ++it;
    }
    if (s->p.bc_y != 2) {
        double m = 0.0;
        for (int c = 0; c < N; ++c) m += x[c];
        for (int c = 0; c < N; ++c) x[c] -= m / N;
    }
    *res_out = bb > 0 ? sqrt(rr / bb) : 0.0;
    free(b); free(r); free(d); free(Ad);
    return it;
}

/* psi at a stencil ghost position: periodic, 2V - psi at electrodes, mirror at walls */
static double psi_at(const orc_state* s, int x, int y) {
    const int nx = s->p.nx, ny = s->p.ny;
    if (s->p.bc_y == 0 || (y >= 0 && y < ny)) return s->psi[wrap(y, ny) * nx + wrap(x, nx)];
    int ym = y < 0 ? -1 - y : 2 * ny - 1 - y;
    double v = s->psi[ym * nx + wrap(x, nx)];
    if (s->p.bc_y == 2) return 2.0 * (y < 0 ? s->p.V_bottom : s->p.V_top) - v;
    return v;
}

static void fd_fields(orc_state* s) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double ax = 0.0, ay = 0.0;
            for (int j = 0; j < 9; ++j) {
                double v = psi_at(s, x + CX[j], y + CY[j]);
                ax += W[j] * CX[j] * v;
                ay += W[j] * CY[j] * v;
            }
            int c = y * nx + x;
            s->E[c] = -(ax / CS2) + s->p.E_ext[0];
            s->E[N + c] = -(ay / CS2) + s->p.E_ext[1];
        }
}

/* ---------------- step pieces ---------------- */
/* S2 + S3: properties and their stencils from the phi fields */
static void properties_and_stencils(orc_state* s) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
    for (int c = 0; c < N; ++c) {
        double ph[3];
        phis(s, c, ph);
        s->rho[c] = ph[0] * s->p.rho[0] + ph[1] * s->p.rho[1] + ph[2] * s->p.rho[2];   /* Eq. 29 */
        s->sig[c] = ph[0] * s->p.sigma[0] + ph[1] * s->p.sigma[1] + ph[2] * s->p.sigma[2];
        s->eps[c] = perm(&s->p, ph);                                                  /* Eq. 30 */
    }
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            for (int i = 0; i < 3; ++i) s->lap[i * N + c] = lap_at(s, s->phi + i * N, x, y);
            grad_at(s, s->eps, x, y, &s->geps[c], &s->geps[N + c]);
            grad_at(s, s->sig, x, y, &s->gsig[c], &s->gsig[N + c]);
            grad_at(s, s->rho, x, y, &s->grho[c], &s->grho[N + c]);
        }
}

/* S6: chemical potential, Eq. 20 with eps'(phi_i) = 6 eps_i phi_i (1 - phi_i) */
static void chemical_potential(orc_state* s) {
    const int N = s->N;
    const double D = s->p.width_D;
    for (int c = 0; c < N; ++c) {
        double e2 = s->E[c] * s->E[c] + s->E[N + c] * s->E[N + c];
        for (int i = 0; i < 3; ++i) {
            double ph = s->phi[i * N + c];
            double bulk = 24.0 / D * s->lam[i] * ph * (ph - 0.5) * (ph - 1.0);
            double grad = 0.75 * D * s->lam[i] * s->lap[i * N + c];
            double deps = 6.0 * s->p.eps[i] * ph * (1.0 - ph);
            s->mu[i * N + c] = bulk - grad - 0.5 * deps * e2;
        }
    }
}

/* S12 ingredients: s_j(u), Eq. 40 */
static double s_j(int j, double ux, double uy) {
    double cu = CX[j] * ux + CY[j] * uy;
    double uu = ux * ux + uy * uy;
    return W[j] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

static double tau_g_at(const orc_state* s, int c) {
    if (!use_visc(&s->p)) return s->p.tau_g;
    double eta = 0.0;
    for (int i = 0; i < 3; ++i) eta += s->phi[i * s->N + c] * s->p.visc[i];
    return 0.5 + eta / (s->rho[c] * CS2);           /* mu = rho cs2 (tau_g - 1/2) */
}

/* S9: u and p from the flow populations, Eq. 41 */
static void flow_moments(orc_state* s) {
    const int N = s->N;
    for (int c = 0; c < N; ++c) {
        double mx = 0.0, my = 0.0, g1 = 0.0;
        for (int j = 0; j < 9; ++j) {
            double gj = s->g[j * N + c];
            mx += CX[j] * gj;
            my += CY[j] * gj;
            if (j) g1 += gj;
        }
        double ux = (mx + 0.5 * s->F[c]) / s->rho[c];
        double uy = (my + 0.5 * s->F[N + c]) / s->rho[c];
        double ugr = ux * s->grho[c] + uy * s->grho[N + c];
        s->u[c] = ux;
        s->u[N + c] = uy;
        s->pr[c] = CS2 / (1.0 - W[0]) * (g1 + 0.5 * ugr + s->rho[c] * s_j(0, ux, uy));
    }
}

/* S11-S13 collisions, then streaming (S14) */
static void collide_and_stream(orc_state* s, int first) {
    const int N = s->N;
    const double tf = s->p.tau_f, tl = s->tau_l, m0 = s->m0;
    const int cc = s->p.charge_convection;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; ++c) {
        double ph[3];
        phis(s, c, ph);
        double ux = s->u[c], uy = s->u[N + c], qc = s->q[c];
        /* S10: d/dt(phi_i u) and d/dt(q u), first-order backward differences */
        double dpu[3][2], dqu[2];
        for (int i = 0; i < 3; ++i) {
            dpu[i][0] = first ? 0.0 : ph[i] * ux - s->prev_phiu[(2 * i) * N + c];
            dpu[i][1] = first ? 0.0 : ph[i] * uy - s->prev_phiu[(2 * i + 1) * N + c];
        }
        dqu[0] = first ? 0.0 : qc * ux - s->prev_qu[c];
        dqu[1] = first ? 0.0 : qc * uy - s->prev_qu[N + c];

        /* phase populations, Eq. 34-36, mobility Eq. 28 */
        for (int i = 0; i < 3; ++i) {
            double Yx = 0.0, Yy = 0.0;
            double Mii = 0.0;
            for (int k = 0; k < 3; ++k)
                if (k != i) Mii += m0 * ph[i] * ph[k];
            for (int k = 0; k < 3; ++k) {
                double Mik = (k == i) ? (Mii - m0) : -m0 * ph[i] * ph[k];
                Yx += Mik * s->gmu[(2 * k) * N + c];
                Yy += Mik * s->gmu[(2 * k + 1) * N + c];
            }
            double Ax = dpu[i][0] / CS2 - Yx / m0;
            double Ay = dpu[i][1] / CS2 - Yy / m0;
            double mui = s->mu[i * N + c];
            for (int j = 0; j < 9; ++j) {
                double feq = (j == 0) ? ph[i] - (1.0 - W[0]) * mui
                                      : W[j] * mui + W[j] * (CX[j] * ph[i] * ux + CY[j] * ph[i] * uy) / CS2;
                double Fj = W[j] * (CX[j] * Ax + CY[j] * Ay);
                double fj = s->f[(9 * i + j) * N + c];
                s->fs[(9 * i + j) * N + c] = fj - (fj - feq) / tf + (1.0 - 1.0 / (2.0 * tf)) * Fj;
            }
        }

        /* flow populations, Eq. 37-40 */
        {
            double tg = tau_g_at(s, c);
            double rho = s->rho[c], p = s->pr[c];
            double Fx = s->F[c], Fy = s->F[N + c];
            double grx = s->grho[c], gry = s->grho[N + c];
            double ugr = ux * grx + uy * gry;
            for (int j = 0; j < 9; ++j) {
                double geq = (j == 0) ? (W[0] - 1.0) * p / CS2 + rho * s_j(0, ux, uy)
                                      : W[j] * p / CS2 + rho * s_j(j, ux, uy);
                double cu = CX[j] * ux + CY[j] * uy;
                double cgr = CX[j] * grx + CY[j] * gry;
                double cF = CX[j] * Fx + CY[j] * Fy;
                double G = W[j] * (ugr + cF / CS2 + (cu * cgr - CS2 * ugr) / CS2);
                double gj = s->g[j * N + c];
                s->gs[j * N + c] = gj - (gj - geq) / tg + (1.0 - 1.0 / (2.0 * tg)) * G;
            }
        }

        /* charge populations, Eq. 48-50 */
        {
            double Rc = s->R[c];
            for (int j = 0; j < 9; ++j) {
                double cu = CX[j] * ux + CY[j] * uy;
                double leq = cc ? W[j] * qc * (1.0 + cu / CS2) : W[j] * qc;
                double Sj = (1.0 - 1.0 / (2.0 * tl)) * W[j] * Rc;
                double Tj = cc ? (1.0 - 1.0 / (2.0 * tl)) * W[j] * (CX[j] * dqu[0] + CY[j] * dqu[1]) / CS2 : 0.0;
                double lj = s->l[j * N + c];
                s->ls[j * N + c] = lj - (lj - leq) / tl + Sj + Tj;
            }
        }
    }
    for (int i = 0; i < 3; ++i) stream(s, s->fs + 9 * i * N, s->f + 9 * i * N, 0);
    stream(s, s->gs, s->g, 1);
    stream(s, s->ls, s->l, 0);
}

/* Ion moments n_i = sum_j n^i_j and the charge they carry, q = e_q sum_i z_i n_i. */
static void ion_charge_from_populations(orc_state* s) {
    const int N = s->N;
    for (int c = 0; c < N; ++c) {
        double q = 0.0;
        for (int i = 0; i < 2; ++i) {
            double a = 0.0;
            for (int j = 0; j < 9; ++j) a += s->ion[(9 * i + j) * N + c];
            s->nion[i * N + c] = a;
            q += s->p.ion_z[i] * a;
        }
        s->q[c] = s->p.ion_charge * q;
    }
}

/* drift velocity of species i at cell c: v_i = u + z_i beta D_i E */
static void ion_velocity(const orc_state* s, int i, int c, double* vx, double* vy) {
    double m = s->p.ion_z[i] * s->p.ion_beta * s->p.ion_D[i];
    *vx = s->u[c] + m * s->E[c];
    *vy = s->u[s->N + c] + m * s->E[s->N + c];
}

/* Nernst-Planck populations (Eq. 52): collide with the u^n and E^n of this step,
 * then stream with bounce-back at walls. */
static void ions_collide_and_stream(orc_state* s, int first) {
    const int N = s->N;
    for (int i = 0; i < 2; ++i) {
        const double ti = s->tau_ion[i];
        for (int c = 0; c < N; ++c) {
            double n = s->nion[i * N + c], vx, vy;
            ion_velocity(s, i, c, &vx, &vy);
            double dx = first ? 0.0 : n * vx - s->prev_nv[(2 * i) * N + c];
            double dy = first ? 0.0 : n * vy - s->prev_nv[(2 * i + 1) * N + c];
            for (int j = 0; j < 9; ++j) {
                double cv = CX[j] * vx + CY[j] * vy;
                double neq = W[j] * n * (1.0 + cv / CS2);
                double Tj = (1.0 - 1.0 / (2.0 * ti)) * W[j] * (CX[j] * dx + CY[j] * dy) / CS2;
                double nj = s->ion[(9 * i + j) * N + c];
                s->ions_s[(9 * i + j) * N + c] = nj - (nj - neq) / ti + Tj;
            }
            s->prev_nv[(2 * i) * N + c] = n * vx;
            s->prev_nv[(2 * i + 1) * N + c] = n * vy;
        }
        stream(s, s->ions_s + 9 * i * N, s->ion + 9 * i * N, 0);
    }
}

/* The step in four phases (one_step runs them in order; the reverse mode below
 * re-runs the first three to recover the intermediates of a step). */

/* S1-S4: zeroth moments, properties and stencils, the charge of the step */
static void step_moments_closure(orc_state* s) {
    const int N = s->N;
    /* S1: zeroth moments of the current populations */
    for (int c = 0; c < N; ++c) {
        for (int i = 0; i < 3; ++i) {
            double a = 0.0;
            for (int j = 0; j < 9; ++j) a += s->f[(9 * i + j) * N + c];
            s->phi[i * N + c] = a;
        }
        double a = 0.0;
        for (int j = 0; j < 9; ++j) a += s->l[j * N + c];
        s->qt[c] = a;
    }
    /* S2, S3 */
    properties_and_stencils(s);
    if (s->p.ions) ion_charge_from_populations(s);
    /* S4: q = sum l + R/2 with R linear in q, field of the previous step */
    for (int c = 0; c < N && !s->p.ions; ++c) {
        double r = s->sig[c] / s->eps[c];
        double Ex = s->E[c], Ey = s->E[N + c];
        double src = r * (s->geps[c] * Ex + s->geps[N + c] * Ey) - (s->gsig[c] * Ex + s->gsig[N + c] * Ey);
        s->q[c] = (s->qt[c] + 0.5 * src) / (1.0 + 0.5 * r);
    }
}

/* S5: potential solve (warm-started from the current h, or the FD form) */
static void step_potential(orc_state* s) {
    const int N = s->N;
    if (s->p.electric && s->p.potential_solver == 1) {
        s->last_iters = fd_solve(s, &s->last_res);
        s->last_converged = 1;
        fd_fields(s);
    } else if (s->p.electric) {
        int conv;
        s->last_iters = poisson_solve(s, s->p.poisson_tol, s->p.poisson_max_iter, s->p.poisson_fixed_iter,
                                      s->p.poisson_check_every, &s->last_res, &conv);
        s->last_converged = conv;
        potential_fields(s);
    } else {
        for (int c = 0; c < N; ++c) {
            s->E[c] = s->p.E_ext[0];
            s->E[N + c] = s->p.E_ext[1];
            s->psi[c] = 0.0;
        }
    }
}

/* R^n, S6-S9: charge source, chemical potential and its gradient, force, flow moments */
static void step_forces(orc_state* s) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
    /* the Debye-Hueckel closure: charge from the solved potential */
    if (s->p.debye_kappa2 > 0.0)
        for (int c = 0; c < N; ++c) s->q[c] = -s->eps[c] * s->p.debye_kappa2 * s->psi[c];
    /* R^n of Eq. 47 with q^n and E^n */
    for (int c = 0; c < N; ++c) {
        double r = s->sig[c] / s->eps[c];
        double Ex = s->E[c], Ey = s->E[N + c];
        s->R[c] = -r * s->q[c] + r * (s->geps[c] * Ex + s->geps[N + c] * Ey) - (s->gsig[c] * Ex + s->gsig[N + c] * Ey);
    }
    /* S6, S7 */
    chemical_potential(s);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            for (int i = 0; i < 3; ++i) grad_at(s, s->mu + i * N, x, y, &s->gmu[(2 * i) * N + c], &s->gmu[(2 * i + 1) * N + c]);
        }
    /* S8: F = -sum phi_i grad mu_i + q E  (Eq. 27b) */
    for (int c = 0; c < N; ++c) {
        double Fx = 0.0, Fy = 0.0;
        for (int i = 0; i < 3; ++i) {
            Fx -= s->phi[i * N + c] * s->gmu[(2 * i) * N + c];
            Fy -= s->phi[i * N + c] * s->gmu[(2 * i + 1) * N + c];
        }
        s->F[c] = Fx + s->q[c] * s->E[c];
        s->F[N + c] = Fy + s->q[c] * s->E[N + c];
    }
    /* S9 */
    flow_moments(s);
}

/* S10-S14: collisions and streaming; the d/dt state for the next step */
static void step_collide(orc_state* s, int first) {
    const int N = s->N;
    collide_and_stream(s, first);
    if (s->p.ions) ions_collide_and_stream(s, first);
    for (int c = 0; c < N; ++c) {
        for (int i = 0; i < 3; ++i) {
            s->prev_phiu[(2 * i) * N + c] = s->phi[i * N + c] * s->u[c];
            s->prev_phiu[(2 * i + 1) * N + c] = s->phi[i * N + c] * s->u[N + c];
        }
        s->prev_qu[c] = s->q[c] * s->u[c];
        s->prev_qu[N + c] = s->q[c] * s->u[N + c];
    }
    s->step += 1;
}

static void one_step(orc_state* s) {
    const int first = s->step == 0;
    step_moments_closure(s);
    step_potential(s);
    step_forces(s);
    step_collide(s, first);
}

/* ---------------- reverse mode: the transposed step ----------------
 *
 * The step maps the state X^n = (g, f, l, h, E, (phi_i u)^{n-1}, (q u)^{n-1}) and the
 * parameters theta to X^{n+1}.  Given the adjoint a^{n+1} = dJ/dX^{n+1} of an
 * objective J, the routines below return a^n = (dX^{n+1}/dX^n)^T a^{n+1} and add
 * (dX^{n+1}/dtheta)^T a^{n+1} to dJ/dtheta.  Each is the literal transpose of the
 * forward statements above, taken in reverse order: a statement y = f(x) becomes
 * xbar += (df/dx)^T ybar, and a stencil or streaming gather becomes the matching
 * scatter.  The potential is differentiated through its fixed number of pseudo-time
 * iterations (Eq. 43), each transposed at the iterate it was applied to (a residual-
 * controlled solve stops on a decision that has no derivative).
 *
 * State vector planes (N cells each): g 0-8, f 9-35 (set-major), l 36-44, h 45-53,
 * E 54-55, (phi_i u)^{n-1} 56-61 (x, y per phase), (q u)^{n-1} 62-63.
 * Parameter slots: V_bottom, V_top, eps_1..3, sigma_1..3, gamma_12, gamma_13, gamma_23. */
void orc_destroy(orc_state* s);
orc_state* orc_create(const orc_params* p, const double* phi_init, const double* u_init,
                      const double* q_init, const double* noise, int* status);

enum { SV_G = 0, SV_F = 9, SV_L = 36, SV_H = 45, SV_E = 54, SV_PU = 56, SV_QU = 62, SV_N = 64 };
enum { AP_VB = 0, AP_VT, AP_EPS, AP_SIG = AP_EPS + 3, AP_GAM = AP_SIG + 3, AP_N = AP_GAM + 3 };

#define ORC_BUFFERS(X) X(g, 9) X(f, 27) X(l, 9) X(h, 9) X(gs, 9) X(fs, 27) X(ls, 9) X(hs, 9) \
    X(phi, 3) X(qt, 1) X(q, 1) X(rho, 1) X(sig, 1) X(eps, 1) X(lap, 3) X(geps, 2) X(gsig, 2) X(grho, 2) \
    X(E, 2) X(psi, 1) X(mu, 3) X(gmu, 6) X(F, 2) X(u, 2) X(pr, 1) X(R, 1) X(prev_phiu, 6) X(prev_qu, 2) \
    X(psi_prev, 1) X(J_prev, 2) X(ion, 18) X(ions_s, 18) X(nion, 2) X(prev_nv, 4)

/* deep copy of a state */
orc_state* orc_clone(const orc_state* s) {
    orc_state* t = (orc_state*)malloc(sizeof(orc_state));
    if (!t) return NULL;
    *t = *s;
    const size_t N = (size_t)s->N;
#define ORC_COPY(name, k) t->name = alloc0((k) * N); memcpy(t->name, s->name, (k) * N * sizeof(double));
    ORC_BUFFERS(ORC_COPY)
#undef ORC_COPY
    return t;
}

/* the state vector of the layout above: read (out) or write (in) */
static double* sv_plane(orc_state* s, int k) {
    const size_t N = (size_t)s->N;
    if (k < SV_F) return s->g + k * N;
    if (k < SV_L) return s->f + (k - SV_F) * N;
    if (k < SV_H) return s->l + (k - SV_L) * N;
    if (k < SV_E) return s->h + (k - SV_H) * N;
    if (k < SV_PU) return s->E + (k - SV_E) * N;
    if (k < SV_QU) return s->prev_phiu + (k - SV_PU) * N;
    return s->prev_qu + (k - SV_QU) * N;
}
void orc_get_state_vector(orc_state* s, double* out) {
    for (int k = 0; k < SV_N; ++k) memcpy(out + (size_t)k * s->N, sv_plane(s, k), s->N * sizeof(double));
}
void orc_set_state_vector(orc_state* s, const double* in) {
    for (int k = 0; k < SV_N; ++k) memcpy(sv_plane(s, k), in + (size_t)k * s->N, s->N * sizeof(double));
}

/* transpose of grad_at over the lattice: out(d) += sum over (c, j) with ghost(c + c_j)
 * = d of w_j c_j . gbar(c) / cs2;  gbar = (x plane, y plane) */
static void grad_T(const orc_state* s, const double* gbar, double* out) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            for (int j = 0; j < 9; ++j) {
                int d = ghost_y(s, y + CY[j]) * nx + wrap(x + CX[j], nx);
                out[d] += W[j] * (CX[j] * gbar[c] + CY[j] * gbar[N + c]) / CS2;
            }
        }
}
/* transpose of lap_at */
static void lap_T(const orc_state* s, const double* lbar, double* out) {
    const int nx = s->p.nx, ny = s->p.ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            for (int j = 0; j < 9; ++j) {
                int d = ghost_y(s, y + CY[j]) * nx + wrap(x + CX[j], nx);
                out[d] += 2.0 * W[j] * lbar[c] / CS2;
                out[c] -= 2.0 * W[j] * lbar[c] / CS2;
            }
        }
}
/* transpose of stream(): srcbar = (dst <- src)^T dstbar; the moving-wall term adds
 * to rhobar (kind 1), the electrode term to the V slots (kind 2) */
static void stream_T(const orc_state* s, const double* dstbar, double* srcbar, int kind, double* rhobar,
                     double* dpar) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            for (int j = 0; j < 9; ++j) {
                int yt = y + CY[j];
                if (s->p.bc_y != 0 && (yt < 0 || yt >= ny)) {
                    int top = yt >= ny;
                    double b = dstbar[OPP[j] * N + c];
                    if (kind == 1) {
                        double uw = top ? s->p.u_wall_top : s->p.u_wall_bottom;
                        srcbar[j * N + c] = b;
                        rhobar[c] += -2.0 * W[j] * (CX[j] * uw) / CS2 * b;
                    } else if (kind == 2 && s->p.bc_y == 2) {
                        srcbar[j * N + c] = -b;
                        dpar[top ? AP_VT : AP_VB] += 2.0 * W[j] * b;
                    } else {
                        srcbar[j * N + c] = b;
                    }
                } else {
                    srcbar[j * N + c] = dstbar[j * N + wrap(yt, ny) * nx + wrap(x + CX[j], nx)];
                }
            }
        }
}

/* transpose of one pseudo-time iteration (collide at the iterate hk, then stream):
 * hbar <- (iteration)^T hbar, adding to epsbar, qbar and the V slots */
static void poisson_iteration_T(const orc_state* s, const double* hk, double* hbar, double* tmp,
                                double* epsbar, double* qbar, double* dpar) {
    const int N = s->N;
    const double th = s->tau_h;
    stream_T(s, hbar, tmp, 2, NULL, dpar);
    for (int c = 0; c < N; ++c) {
        double epshat = s->eps[c] - s->p.eps_ref;
        double den = epshat + CS2 * th;
        double ax = 0.0, ay = 0.0;
        for (int j = 0; j < 9; ++j) {
            ax += CX[j] * hk[j * N + c];
            ay += CY[j] * hk[j * N + c];
        }
        double gx = -ax / den, gy = -ay / den;
        double apsi = 0.0, agx = 0.0, agy = 0.0, aeh = 0.0, aq = 0.0;
        for (int j = 0; j < 9; ++j) {
            double b = tmp[j * N + c];
            double coef = (j == 0) ? (W[0] - 1.0) : W[j];   /* h_eq = coef psi, Eq. 44 */
            double cg = CX[j] * gx + CY[j] * gy;
            hbar[j * N + c] = (1.0 - 1.0 / th) * b;
            apsi += coef * b / th;
            agx += -(epshat / CS2) * W[j] * CX[j] * b / th;
            agy += -(epshat / CS2) * W[j] * CY[j] * b / th;
            aeh += -(1.0 / CS2) * W[j] * cg * b / th;
            if (j) aq += b / 8.0;
        }
        /* g = -a / den, den = epshat + cs2 tau_h */
        double aax = -agx / den, aay = -agy / den;
        aeh += (agx * ax + agy * ay) / (den * den);
        for (int j = 0; j < 9; ++j)
            hbar[j * N + c] += CX[j] * aax + CY[j] * aay + (j ? apsi / (1.0 - W[0]) : 0.0);
        epsbar[c] += aeh;
        qbar[c] += aq;
    }
}

/* transpose of E = J(h) / (epshat + cs2 tau_h) + E_ext (potential_fields) into hbar
 * and epsbar */
static void fields_T(const orc_state* s, const double* h, const double* Ebar, double* hbar, double* epsbar) {
    const int N = s->N;
    for (int c = 0; c < N; ++c) {
        double den = s->eps[c] - s->p.eps_ref + CS2 * s->tau_h;
        double ax = 0.0, ay = 0.0;
        for (int j = 0; j < 9; ++j) {
            ax += CX[j] * h[j * N + c];
            ay += CY[j] * h[j * N + c];
        }
        for (int j = 0; j < 9; ++j) hbar[j * N + c] += (CX[j] * Ebar[c] + CY[j] * Ebar[N + c]) / den;
        epsbar[c] += -(ax * Ebar[c] + ay * Ebar[N + c]) / (den * den);
    }
}

/* transpose of the chemical potential (Eq. 20) into phibar, lapbar, Ebar, lambar and
 * the eps slots */
static void chemical_potential_T(const orc_state* s, const double* mubar, double* phibar, double* lapbar,
                                 double* Ebar, double* lambar, double* dpar) {
    const int N = s->N;
    const double D = s->p.width_D;
    for (int c = 0; c < N; ++c) {
        double Ex = s->E[c], Ey = s->E[N + c];
        double e2 = Ex * Ex + Ey * Ey;
        for (int i = 0; i < 3; ++i) {
            double ph = s->phi[i * N + c], mb = mubar[i * N + c];
            double deps = 6.0 * s->p.eps[i] * ph * (1.0 - ph);
            phibar[i * N + c] += mb * (24.0 / D * s->lam[i] * (3.0 * ph * ph - 3.0 * ph + 0.5)
                                       - 3.0 * s->p.eps[i] * (1.0 - 2.0 * ph) * e2);
            lapbar[i * N + c] += -0.75 * D * s->lam[i] * mb;
            Ebar[c] += -deps * Ex * mb;
            Ebar[N + c] += -deps * Ey * mb;
            lambar[i] += mb * (24.0 / D * ph * (ph - 0.5) * (ph - 1.0) - 0.75 * D * s->lap[i * N + c]);
            dpar[AP_EPS + i] += -3.0 * ph * (1.0 - ph) * e2 * mb;
        }
    }
}

/* transpose of the properties (Eq. 29-30) into phibar and the eps, sigma slots */
static void properties_T(const orc_state* s, const double* rhobar, const double* sigbar, const double* epsbar,
                         double* phibar, double* dpar) {
    const int N = s->N;
    for (int c = 0; c < N; ++c)
        for (int i = 0; i < 3; ++i) {
            double ph = s->phi[i * N + c];
            phibar[i * N + c] += s->p.rho[i] * rhobar[c] + s->p.sigma[i] * sigbar[c]
                               + s->p.eps[i] * 6.0 * ph * (1.0 - ph) * epsbar[c];
            dpar[AP_SIG + i] += ph * sigbar[c];
            dpar[AP_EPS + i] += ph * ph * (3.0 - 2.0 * ph) * epsbar[c];
        }
}

/* lambda_i of Eq. 9 are sums of the gamma_jk: their adjoints map back */
static void lambda_T(const double* lambar, double* dpar) {
    dpar[AP_GAM + 0] += lambar[0] + lambar[1] - lambar[2];
    dpar[AP_GAM + 1] += lambar[0] - lambar[1] + lambar[2];
    dpar[AP_GAM + 2] += -lambar[0] + lambar[1] + lambar[2];
}

static int adjoint_supported(const orc_params* p) {
    if (p->ions || p->debye_kappa2 > 0.0) return 0;
    if (p->electric && (p->potential_solver != 0 || p->poisson_fixed_iter <= 0)) return 0;
    return 1;
}

/* a_out = (dX^{n+1}/dX^n)^T a_in for the step that starts from the state s (left
 * unchanged); dpar[AP_N] += (dX^{n+1}/dtheta)^T a_in.  Returns -1 for a configuration
 * without a derivative here (ions, the Debye-Hueckel closure, the FD potential, a
 * residual-controlled potential). */
int orc_adjoint_step(const orc_state* s0, const double* a_in, double* a_out, double* dpar) {
    if (!adjoint_supported(&s0->p)) return -1;
    const int N = s0->N;
    const size_t n = (size_t)N;
    const int K = s0->p.electric ? s0->p.poisson_fixed_iter : 0;
    const int first = s0->step == 0;
    /* forward again on a copy, keeping the intermediates and the potential iterates */
    orc_state* t = orc_clone(s0);
    double* Eprev = alloc0(2 * n);
    memcpy(Eprev, t->E, 2 * n * sizeof(double));
    double* hk = alloc0((size_t)(K + 1) * 9 * n);
    step_moments_closure(t);
    if (t->p.electric) {
        for (int k = 0; k < K; ++k) {
            memcpy(hk + (size_t)k * 9 * n, t->h, 9 * n * sizeof(double));
            poisson_iteration(t);
        }
        memcpy(hk + (size_t)K * 9 * n, t->h, 9 * n * sizeof(double));
        potential_fields(t);
    } else {
        step_potential(t);
    }
    step_forces(t);

    const double tf = t->p.tau_f, tl = t->tau_l, m0 = t->m0;
    const int cc = t->p.charge_convection;
    double *a_fs = alloc0(27 * n), *a_gs = alloc0(9 * n), *a_ls = alloc0(9 * n);
    double *a_phi = alloc0(3 * n), *a_u = alloc0(2 * n), *a_q = alloc0(n), *a_mu = alloc0(3 * n);
    double *a_gmu = alloc0(6 * n), *a_rho = alloc0(n), *a_p = alloc0(n), *a_F = alloc0(2 * n);
    double *a_grho = alloc0(2 * n), *a_R = alloc0(n), *a_E = alloc0(2 * n), *a_sig = alloc0(n);
    double *a_eps = alloc0(n), *a_geps = alloc0(2 * n), *a_gsig = alloc0(2 * n), *a_lap = alloc0(3 * n);
    double *a_h = alloc0(9 * n), *tmp = alloc0(9 * n);
    double lambar[3] = {0.0, 0.0, 0.0};
    memset(a_out, 0, SV_N * n * sizeof(double));
    /* the field of this step is part of the state it leaves */
    memcpy(a_E, a_in + SV_E * n, 2 * n * sizeof(double));

    /* the d/dt state written at the end of the step: (phi_i u), (q u) */
    for (int c = 0; c < N; ++c) {
        double ux = t->u[c], uy = t->u[N + c];
        for (int i = 0; i < 3; ++i) {
            double bx = a_in[(SV_PU + 2 * i) * n + c], by = a_in[(SV_PU + 2 * i + 1) * n + c];
            a_phi[i * N + c] += ux * bx + uy * by;
            a_u[c] += t->phi[i * N + c] * bx;
            a_u[N + c] += t->phi[i * N + c] * by;
        }
        double bx = a_in[SV_QU * n + c], by = a_in[(SV_QU + 1) * n + c];
        a_q[c] += ux * bx + uy * by;
        a_u[c] += t->q[c] * bx;
        a_u[N + c] += t->q[c] * by;
    }
    /* streaming (S14) */
    for (int i = 0; i < 3; ++i) stream_T(t, a_in + (SV_F + 9 * i) * n, a_fs + 9 * i * n, 0, NULL, NULL);
    stream_T(t, a_in + SV_G * n, a_gs, 1, a_rho, NULL);
    stream_T(t, a_in + SV_L * n, a_ls, 0, NULL, NULL);

    /* collisions (S10-S13) */
    for (int c = 0; c < N; ++c) {
        double ph[3];
        phis(t, c, ph);
        double ux = t->u[c], uy = t->u[N + c], qc = t->q[c];
        double aux = 0.0, auy = 0.0, aqc = 0.0;
        /* phase populations, Eq. 34-36 */
        for (int i = 0; i < 3; ++i) {
            double aAx = 0.0, aAy = 0.0;
            for (int j = 0; j < 9; ++j) {
                double fb = a_fs[(9 * i + j) * n + c];
                a_out[(SV_F + 9 * i + j) * n + c] += (1.0 - 1.0 / tf) * fb;
                double feqb = fb / tf, Fjb = (1.0 - 1.0 / (2.0 * tf)) * fb;
                aAx += W[j] * CX[j] * Fjb;
                aAy += W[j] * CY[j] * Fjb;
                if (j == 0) {
                    a_phi[i * N + c] += feqb;
                    a_mu[i * N + c] += -(1.0 - W[0]) * feqb;
                } else {
                    a_mu[i * N + c] += W[j] * feqb;
                    double tq = W[j] * feqb / CS2;   /* d feq_j / d(phi_i u) = w_j c_j / cs2 */
                    a_phi[i * N + c] += tq * (CX[j] * ux + CY[j] * uy);
                    aux += tq * CX[j] * ph[i];
                    auy += tq * CY[j] * ph[i];
                }
            }
            /* A = d/dt(phi_i u) / cs2 - Y / m0,  Y = sum_k M_ik grad mu_k */
            double aYx = -aAx / m0, aYy = -aAy / m0;
            for (int k = 0; k < 3; ++k) {
                double Mii = 0.0;
                for (int kk = 0; kk < 3; ++kk)
                    if (kk != i) Mii += m0 * ph[i] * ph[kk];
                double Mik = (k == i) ? (Mii - m0) : -m0 * ph[i] * ph[k];
                a_gmu[(2 * k) * n + c] += Mik * aYx;
                a_gmu[(2 * k + 1) * n + c] += Mik * aYy;
                double aM = aYx * t->gmu[(2 * k) * n + c] + aYy * t->gmu[(2 * k + 1) * n + c];
                if (k != i) {
                    a_phi[i * N + c] += -m0 * ph[k] * aM;
                    a_phi[k * N + c] += -m0 * ph[i] * aM;
                } else {
                    for (int kk = 0; kk < 3; ++kk)
                        if (kk != i) {
                            a_phi[i * N + c] += m0 * ph[kk] * aM;
                            a_phi[kk * N + c] += m0 * ph[i] * aM;
                        }
                }
            }
            if (!first) {
                double adx = aAx / CS2, ady = aAy / CS2;
                a_phi[i * N + c] += ux * adx + uy * ady;
                aux += ph[i] * adx;
                auy += ph[i] * ady;
                a_out[(SV_PU + 2 * i) * n + c] -= adx;
                a_out[(SV_PU + 2 * i + 1) * n + c] -= ady;
            }
        }
        /* flow populations, Eq. 37-40 */
        {
            double tg = tau_g_at(t, c);
            double rho = t->rho[c], p = t->pr[c];
            double Fx = t->F[c], Fy = t->F[N + c];
            double grx = t->grho[c], gry = t->grho[N + c];
            double ugr = ux * grx + uy * gry;
            double atg = 0.0;
            for (int j = 0; j < 9; ++j) {
                double gb = a_gs[j * n + c];
                a_out[(SV_G + j) * n + c] += (1.0 - 1.0 / tg) * gb;
                double geqb = gb / tg, Gb = (1.0 - 1.0 / (2.0 * tg)) * gb;
                double sj = s_j(j, ux, uy);
                double cu = CX[j] * ux + CY[j] * uy;
                double cgr = CX[j] * grx + CY[j] * gry;
                if (use_visc(&t->p)) {
                    double geq = (j == 0) ? (W[0] - 1.0) * p / CS2 + rho * sj : W[j] * p / CS2 + rho * sj;
                    double cF = CX[j] * Fx + CY[j] * Fy;
                    double G = W[j] * (ugr + cF / CS2 + (cu * cgr - CS2 * ugr) / CS2);
                    atg += gb * ((t->g[j * n + c] - geq) + 0.5 * G) / (tg * tg);
                }
                a_p[c] += ((j == 0) ? (W[0] - 1.0) : W[j]) / CS2 * geqb;
                a_rho[c] += sj * geqb;
                /* d s_j / du = w_j (c_j / cs2 + (c_j.u) c_j / cs2^2 - u / cs2) */
                aux += rho * geqb * W[j] * (CX[j] / CS2 + cu * CX[j] / (CS2 * CS2) - ux / CS2);
                auy += rho * geqb * W[j] * (CY[j] / CS2 + cu * CY[j] / (CS2 * CS2) - uy / CS2);
                /* G_j: the u.grad rho terms cancel (coefficient w_j (1 - cs2/cs2) = 0) */
                a_F[c] += W[j] * CX[j] * Gb / CS2;
                a_F[N + c] += W[j] * CY[j] * Gb / CS2;
                aux += W[j] * CX[j] * cgr * Gb / CS2;
                auy += W[j] * CY[j] * cgr * Gb / CS2;
                a_grho[c] += W[j] * CX[j] * cu * Gb / CS2;
                a_grho[N + c] += W[j] * CY[j] * cu * Gb / CS2;
            }
            if (use_visc(&t->p)) {
                double eta = 0.0;
                for (int i = 0; i < 3; ++i) eta += ph[i] * t->p.visc[i];
                double aeta = atg / (rho * CS2);
                a_rho[c] += -atg * eta / (rho * rho * CS2);
                for (int i = 0; i < 3; ++i) a_phi[i * N + c] += t->p.visc[i] * aeta;
            }
        }
        /* charge populations, Eq. 48-50 */
        {
            double adqx = 0.0, adqy = 0.0;
            for (int j = 0; j < 9; ++j) {
                double lb = a_ls[j * n + c];
                a_out[(SV_L + j) * n + c] += (1.0 - 1.0 / tl) * lb;
                double leqb = lb / tl;
                a_R[c] += (1.0 - 1.0 / (2.0 * tl)) * W[j] * lb;
                if (cc) {
                    double cu = CX[j] * ux + CY[j] * uy;
                    aqc += W[j] * (1.0 + cu / CS2) * leqb;
                    aux += W[j] * qc * CX[j] / CS2 * leqb;
                    auy += W[j] * qc * CY[j] / CS2 * leqb;
                    adqx += (1.0 - 1.0 / (2.0 * tl)) * W[j] * CX[j] * lb / CS2;
                    adqy += (1.0 - 1.0 / (2.0 * tl)) * W[j] * CY[j] * lb / CS2;
                } else {
                    aqc += W[j] * leqb;
                }
            }
            if (cc && !first) {
                aqc += ux * adqx + uy * adqy;
                aux += qc * adqx;
                auy += qc * adqy;
                a_out[SV_QU * n + c] -= adqx;
                a_out[(SV_QU + 1) * n + c] -= adqy;
            }
        }
        a_u[c] += aux;
        a_u[N + c] += auy;
        a_q[c] += aqc;
    }

    /* S9: u = (m + F/2) / rho, p = cs2/(1 - w0) (g1 + ugr/2 + rho s_0(u)) */
    for (int c = 0; c < N; ++c) {
        double rho = t->rho[c], ux = t->u[c], uy = t->u[N + c];
        double grx = t->grho[c], gry = t->grho[N + c];
        double kp = CS2 / (1.0 - W[0]), ap = a_p[c];
        double ag1 = kp * ap, augr = 0.5 * kp * ap;
        a_rho[c] += kp * s_j(0, ux, uy) * ap;
        double aux = a_u[c] + kp * rho * ap * W[0] * (-ux / CS2);  /* d s_0 / du = -w0 u / cs2 */
        double auy = a_u[N + c] + kp * rho * ap * W[0] * (-uy / CS2);
        aux += grx * augr;
        auy += gry * augr;
        a_grho[c] += ux * augr;
        a_grho[N + c] += uy * augr;
        double amx = aux / rho, amy = auy / rho;
        a_F[c] += 0.5 * aux / rho;
        a_F[N + c] += 0.5 * auy / rho;
        a_rho[c] += -(ux * aux + uy * auy) / rho;
        for (int j = 0; j < 9; ++j) a_out[(SV_G + j) * n + c] += CX[j] * amx + CY[j] * amy + (j ? ag1 : 0.0);
    }
    /* S8: F = -sum phi_i grad mu_i + q E;  R = -r q + r geps.E - gsig.E, r = sig/eps */
    for (int c = 0; c < N; ++c) {
        double aFx = a_F[c], aFy = a_F[N + c];
        for (int i = 0; i < 3; ++i) {
            a_phi[i * N + c] += -(t->gmu[(2 * i) * n + c] * aFx + t->gmu[(2 * i + 1) * n + c] * aFy);
            a_gmu[(2 * i) * n + c] += -t->phi[i * N + c] * aFx;
            a_gmu[(2 * i + 1) * n + c] += -t->phi[i * N + c] * aFy;
        }
        double Ex = t->E[c], Ey = t->E[N + c], qc = t->q[c];
        a_q[c] += Ex * aFx + Ey * aFy;
        a_E[c] += qc * aFx;
        a_E[N + c] += qc * aFy;
        double r = t->sig[c] / t->eps[c], aR = a_R[c];
        double gex = t->geps[c], gey = t->geps[N + c], gsx = t->gsig[c], gsy = t->gsig[N + c];
        a_q[c] += -r * aR;
        double ar = (-qc + gex * Ex + gey * Ey) * aR;
        a_geps[c] += r * Ex * aR;
        a_geps[N + c] += r * Ey * aR;
        a_E[c] += (r * gex - gsx) * aR;
        a_E[N + c] += (r * gey - gsy) * aR;
        a_gsig[c] += -Ex * aR;
        a_gsig[N + c] += -Ey * aR;
        a_sig[c] += ar / t->eps[c];
        a_eps[c] += -ar * t->sig[c] / (t->eps[c] * t->eps[c]);
    }
    /* S7, S6 */
    for (int i = 0; i < 3; ++i) grad_T(t, a_gmu + 2 * i * n, a_mu + i * n);
    chemical_potential_T(t, a_mu, a_phi, a_lap, a_E, lambar, dpar);
    /* S5: E from the last iterate, then the iterations in reverse */
    for (size_t k = 0; k < 9 * n; ++k) a_h[k] = a_in[SV_H * n + k];
    if (t->p.electric) {
        fields_T(t, hk + (size_t)K * 9 * n, a_E, a_h, a_eps);
        for (int k = K - 1; k >= 0; --k) poisson_iteration_T(t, hk + (size_t)k * 9 * n, a_h, tmp, a_eps, a_q, dpar);
    }
    for (size_t k = 0; k < 9 * n; ++k) a_out[SV_H * n + k] = a_h[k];
    /* S4: q = (qt + src/2) / (1 + r/2), src = r geps.E' - gsig.E' with the previous E' */
    double* a_qt = tmp;
    for (int c = 0; c < N; ++c) {
        double r = t->sig[c] / t->eps[c], d = 1.0 + 0.5 * r, aq = a_q[c];
        double Ex = Eprev[c], Ey = Eprev[N + c];
        double gex = t->geps[c], gey = t->geps[N + c], gsx = t->gsig[c], gsy = t->gsig[N + c];
        a_qt[c] = aq / d;
        double asrc = 0.5 * aq / d;
        double ar = 0.5 * (-t->q[c] * aq / d) + (gex * Ex + gey * Ey) * asrc;
        a_geps[c] += r * Ex * asrc;
        a_geps[N + c] += r * Ey * asrc;
        a_gsig[c] += -Ex * asrc;
        a_gsig[N + c] += -Ey * asrc;
        a_out[SV_E * n + c] += (r * gex - gsx) * asrc;
        a_out[(SV_E + 1) * n + c] += (r * gey - gsy) * asrc;
        a_sig[c] += ar / t->eps[c];
        a_eps[c] += -ar * t->sig[c] / (t->eps[c] * t->eps[c]);
    }
    /* S3, S2 */
    for (int i = 0; i < 3; ++i) lap_T(t, a_lap + i * n, a_phi + i * n);
    grad_T(t, a_geps, a_eps);
    grad_T(t, a_gsig, a_sig);
    grad_T(t, a_grho, a_rho);
    properties_T(t, a_rho, a_sig, a_eps, a_phi, dpar);
    lambda_T(lambar, dpar);
    /* S1 */
    for (int c = 0; c < N; ++c) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 9; ++j) a_out[(SV_F + 9 * i + j) * n + c] += a_phi[i * N + c];
        for (int j = 0; j < 9; ++j) a_out[(SV_L + j) * n + c] += a_qt[c];
    }
    double* bufs[] = {Eprev, hk, a_fs, a_gs, a_ls, a_phi, a_u, a_q, a_mu, a_gmu, a_rho, a_p, a_F, a_grho,
                      a_R, a_E, a_sig, a_eps, a_geps, a_gsig, a_lap, a_h, tmp};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) free(bufs[k]);
    orc_destroy(t);
    return 0;
}

/* Transpose of orc_create: dpar[AP_N] += (dX^0/dtheta)^T a_in and, if dphi is not
 * NULL, dphi[3N] += (dX^0/dphi_init)^T a_in (the noise is additive and u_init, q_init
 * are held fixed).  Returns -1 as orc_adjoint_step does, or on bad parameters. */
int orc_adjoint_init(const orc_params* p, const double* phi_init, const double* u_init, const double* q_init,
                     const double* a_in, double* dpar, double* dphi) {
    if (!adjoint_supported(p)) return -1;
    int st;
    orc_state* t = orc_create(p, phi_init, u_init, q_init, NULL, &st);
    if (!t) return -1;
    const int N = t->N, nx = p->nx, ny = p->ny;
    const size_t n = (size_t)N;
    const int K = p->electric ? p->poisson_fixed_iter : 0;
    /* the intermediates of the creation: properties from phi_init, the iterates of the
     * potential from the linear electrode profile */
    memcpy(t->phi, phi_init, 3 * n * sizeof(double));
    memset(t->q, 0, n * sizeof(double));
    if (q_init) memcpy(t->q, q_init, n * sizeof(double));
    properties_and_stencils(t);
    double* hk = alloc0((size_t)(K + 1) * 9 * n);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            double psi0 = p->bc_y == 2 ? p->V_bottom + (p->V_top - p->V_bottom) * (y + 0.5) / ny : 0.0;
            for (int j = 0; j < 9; ++j) t->h[j * N + c] = (j == 0) ? (W[0] - 1.0) * psi0 : W[j] * psi0;
        }
    if (p->electric) {
        for (int k = 0; k < K; ++k) {
            memcpy(hk + (size_t)k * 9 * n, t->h, 9 * n * sizeof(double));
            poisson_iteration(t);
        }
        memcpy(hk + (size_t)K * 9 * n, t->h, 9 * n * sizeof(double));
        potential_fields(t);
    } else {
        for (int c = 0; c < N; ++c) {
            t->E[c] = p->E_ext[0];
            t->E[N + c] = p->E_ext[1];
        }
    }
    chemical_potential(t);

    double *a_phi = alloc0(3 * n), *a_mu = alloc0(3 * n), *a_lap = alloc0(3 * n), *a_E = alloc0(2 * n);
    double *a_rho = alloc0(n), *a_sig = alloc0(n), *a_eps = alloc0(n), *a_q = alloc0(n);
    double *a_h = alloc0(9 * n), *tmp = alloc0(9 * n);
    double lambar[3] = {0.0, 0.0, 0.0};
    const int cc = p->charge_convection;
    for (int c = 0; c < N; ++c) {
        double ux = t->u[c], uy = t->u[N + c];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 9; ++j) {
                double fb = a_in[(SV_F + 9 * i + j) * n + c];
                if (j == 0) {
                    a_phi[i * N + c] += fb;
                    a_mu[i * N + c] += -(1.0 - W[0]) * fb;
                } else {
                    a_mu[i * N + c] += W[j] * fb;
                    a_phi[i * N + c] += W[j] * (CX[j] * ux + CY[j] * uy) / CS2 * fb;
                }
            }
        for (int j = 0; j < 9; ++j) {
            a_rho[c] += s_j(j, ux, uy) * a_in[(SV_G + j) * n + c];
            double cu = CX[j] * ux + CY[j] * uy;
            a_q[c] += (cc ? W[j] * (1.0 + cu / CS2) : W[j]) * a_in[(SV_L + j) * n + c];
        }
        a_E[c] += a_in[SV_E * n + c];
        a_E[N + c] += a_in[(SV_E + 1) * n + c];
    }
    chemical_potential_T(t, a_mu, a_phi, a_lap, a_E, lambar, dpar);
    for (size_t k = 0; k < 9 * n; ++k) a_h[k] = a_in[SV_H * n + k];
    if (p->electric) {
        fields_T(t, hk + (size_t)K * 9 * n, a_E, a_h, a_eps);
        for (int k = K - 1; k >= 0; --k) poisson_iteration_T(t, hk + (size_t)k * 9 * n, a_h, tmp, a_eps, a_q, dpar);
        if (p->bc_y == 2)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int c = y * nx + x;
                    double apsi = 0.0, s = (y + 0.5) / ny;
                    for (int j = 0; j < 9; ++j) apsi += ((j == 0) ? (W[0] - 1.0) : W[j]) * a_h[j * N + c];
                    dpar[AP_VT] += apsi * s;
                    dpar[AP_VB] += apsi * (1.0 - s);
                }
    }
    for (int i = 0; i < 3; ++i) lap_T(t, a_lap + i * n, a_phi + i * n);
    properties_T(t, a_rho, a_sig, a_eps, a_phi, dpar);
    lambda_T(lambar, dpar);
    if (dphi)
        for (size_t k = 0; k < 3 * n; ++k) dphi[k] += a_phi[k];
    double* bufs[] = {hk, a_phi, a_mu, a_lap, a_E, a_rho, a_sig, a_eps, a_q, a_h, tmp};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) free(bufs[k]);
    orc_destroy(t);
    return 0;
}

/* ---------------- public (test-only) API ---------------- */
void orc_destroy(orc_state* s) {
    if (!s) return;
    double* bufs[] = {s->g, s->f, s->l, s->h, s->gs, s->fs, s->ls, s->hs, s->phi, s->qt, s->q, s->rho,
                      s->sig, s->eps, s->lap, s->geps, s->gsig, s->grho, s->E, s->psi, s->mu, s->gmu,
                      s->F, s->u, s->pr, s->R, s->prev_phiu, s->prev_qu, s->psi_prev, s->J_prev,
                      s->ion, s->ions_s, s->nion, s->prev_nv};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) free(bufs[k]);
    free(s);
}

/* status: 0 ok, -1 bad parameters, -2 out of memory */
orc_state* orc_create(const orc_params* p, const double* phi_init, const double* u_init,
                      const double* q_init, const double* noise, int* status) {
    *status = -1;
    if (p->nx < 2 || p->ny < 2 || p->bc_y < 0 || p->bc_y > 2 || p->potential_solver < 0 || p->potential_solver > 1)
        return NULL;
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5) || !(p->width_D > 0) || !(p->eps_ref > 0) || !(p->alpha > 0))
        return NULL;
    for (int i = 0; i < 3; ++i)
        if (!(p->rho[i] > 0) || !(p->eps[i] > 0) || p->sigma[i] < 0) return NULL;
    if (p->ions != 0 && (p->ions != 1 || !(p->ion_D[0] > 0) || !(p->ion_D[1] > 0) || p->debye_kappa2 > 0.0))
        return NULL;
    double lam[3] = {p->gamma12 + p->gamma13 - p->gamma23,   /* Eq. 9 */
                     p->gamma12 + p->gamma23 - p->gamma13,
                     p->gamma13 + p->gamma23 - p->gamma12};
    for (int i = 0; i < 3; ++i)
        if (!(lam[i] > 0)) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    *status = -2;
    if (!s) return NULL;
    s->p = *p;
    const int N = p->nx * p->ny;
    s->N = N;
    for (int i = 0; i < 3; ++i) s->lam[i] = lam[i];
    s->m0 = CS2 * (p->tau_f - 0.5);
    s->tau_h = 0.5 + p->eps_ref / CS2;
    s->tau_l = 0.5 + p->alpha / CS2;
    s->g = alloc0(9 * (size_t)N); s->f = alloc0(27 * (size_t)N); s->l = alloc0(9 * (size_t)N); s->h = alloc0(9 * (size_t)N);
    s->gs = alloc0(9 * (size_t)N); s->fs = alloc0(27 * (size_t)N); s->ls = alloc0(9 * (size_t)N); s->hs = alloc0(9 * (size_t)N);
    s->phi = alloc0(3 * (size_t)N); s->qt = alloc0(N); s->q = alloc0(N); s->rho = alloc0(N); s->sig = alloc0(N);
    s->eps = alloc0(N); s->lap = alloc0(3 * (size_t)N); s->geps = alloc0(2 * (size_t)N); s->gsig = alloc0(2 * (size_t)N);
    s->grho = alloc0(2 * (size_t)N); s->E = alloc0(2 * (size_t)N); s->psi = alloc0(N); s->mu = alloc0(3 * (size_t)N);
    s->gmu = alloc0(6 * (size_t)N); s->F = alloc0(2 * (size_t)N); s->u = alloc0(2 * (size_t)N); s->pr = alloc0(N);
    s->R = alloc0(N); s->prev_phiu = alloc0(6 * (size_t)N); s->prev_qu = alloc0(2 * (size_t)N); s->psi_prev = alloc0(N);
    s->J_prev = alloc0(2 * (size_t)N);
    s->ion = alloc0(18 * (size_t)N); s->ions_s = alloc0(18 * (size_t)N); s->nion = alloc0(2 * (size_t)N);
    s->prev_nv = alloc0(4 * (size_t)N);
    if (!s->J_prev || !s->prev_nv) { orc_destroy(s); return NULL; }
    for (int i = 0; i < 2; ++i) s->tau_ion[i] = 0.5 + p->ion_D[i] / CS2;

    memcpy(s->phi, phi_init, 3 * (size_t)N * sizeof(double));
    if (u_init) memcpy(s->u, u_init, 2 * (size_t)N * sizeof(double));
    if (q_init) memcpy(s->q, q_init, (size_t)N * sizeof(double));
    properties_and_stencils(s);

    /* potential populations start at equilibrium with the linear electrode profile */
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int c = y * p->nx + x;
            double psi0 = p->bc_y == 2 ? p->V_bottom + (p->V_top - p->V_bottom) * (y + 0.5) / p->ny : 0.0;
            for (int j = 0; j < 9; ++j) s->h[j * N + c] = (j == 0) ? (W[0] - 1.0) * psi0 : W[j] * psi0;
        }
    if (p->electric && p->potential_solver == 1) {
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                s->psi[y * p->nx + x] = p->bc_y == 2 ? p->V_bottom + (p->V_top - p->V_bottom) * (y + 0.5) / p->ny : 0.0;
        s->last_iters = fd_solve(s, &s->last_res);
        s->last_converged = 1;
        fd_fields(s);
    } else if (p->electric) {
        int conv;
        s->last_iters = poisson_solve(s, p->poisson_tol, p->poisson_max_iter, p->poisson_fixed_iter,
                                      p->poisson_check_every, &s->last_res, &conv);
        s->last_converged = conv;
        potential_fields(s);
    } else {
        for (int c = 0; c < N; ++c) {
            s->E[c] = p->E_ext[0];
            s->E[N + c] = p->E_ext[1];
        }
    }
    chemical_potential(s);
    const int cc = p->charge_convection;
    for (int c = 0; c < N; ++c) {
        double ux = s->u[c], uy = s->u[N + c];
        for (int i = 0; i < 3; ++i) {
            double ph = s->phi[i * N + c], mui = s->mu[i * N + c];
            for (int j = 0; j < 9; ++j)
                s->f[(9 * i + j) * N + c] = (j == 0) ? ph - (1.0 - W[0]) * mui
                                                     : W[j] * mui + W[j] * (CX[j] * ph * ux + CY[j] * ph * uy) / CS2;
        }
        for (int j = 0; j < 9; ++j) {
            /* g_eq with p = 0 (Eq. 39) */
            s->g[j * N + c] = s->rho[c] * s_j(j, ux, uy);
            double cu = CX[j] * ux + CY[j] * uy;
            s->l[j * N + c] = cc ? W[j] * s->q[c] * (1.0 + cu / CS2) : W[j] * s->q[c];
        }
    }
    if (noise) {
        for (size_t k = 0; k < 9 * (size_t)N; ++k) s->g[k] += noise[k];
        for (size_t k = 0; k < 27 * (size_t)N; ++k) s->f[k] += noise[9 * (size_t)N + k];
        for (size_t k = 0; k < 9 * (size_t)N; ++k) s->l[k] += noise[36 * (size_t)N + k];
    }
    s->step = 0;
    *status = 0;
    return s;
}

/* Start the ion species from the concentrations n_init[2N] (species-major): the
 * charge they carry is set, the potential solved for it (as at creation) and each
 * ion set put at its equilibrium with the stored u and that field.  Returns -1
 * when the state has no ion transport, -2 after the first step. */
int orc_set_ions(orc_state* s, const double* n_init) {
    const int N = s->N;
    if (!s->p.ions) return -1;
    if (s->step != 0) return -2;
    memcpy(s->nion, n_init, 2 * (size_t)N * sizeof(double));
    for (int c = 0; c < N; ++c)
        s->q[c] = s->p.ion_charge * (s->p.ion_z[0] * s->nion[c] + s->p.ion_z[1] * s->nion[N + c]);
    if (s->p.electric && s->p.potential_solver == 1) {
        s->last_iters = fd_solve(s, &s->last_res);
        s->last_converged = 1;
        fd_fields(s);
    } else if (s->p.electric) {
        int conv;
        s->last_iters = poisson_solve(s, s->p.poisson_tol, s->p.poisson_max_iter, s->p.poisson_fixed_iter,
                                      s->p.poisson_check_every, &s->last_res, &conv);
        s->last_converged = conv;
        potential_fields(s);
    }
    for (int i = 0; i < 2; ++i)
        for (int c = 0; c < N; ++c) {
            double n = s->nion[i * N + c], vx, vy;
            ion_velocity(s, i, c, &vx, &vy);
            for (int j = 0; j < 9; ++j)
                s->ion[(9 * i + j) * N + c] = W[j] * n * (1.0 + (CX[j] * vx + CY[j] * vy) / CS2);
        }
    return 0;
}

int orc_step(orc_state* s, int nsteps) {
    for (int k = 0; k < nsteps; ++k) one_step(s);
    return 0;
}

/* Solve the potential for the stored eps and a given charge field (or the stored
 * q), updating h, psi and E.  Returns the iteration count. */
int orc_solve_potential(orc_state* s, const double* q, double tol, int max_iter, int fixed, int check,
                        double* res, int* converged) {
    if (q) memcpy(s->q, q, (size_t)s->N * sizeof(double));
    if (s->p.potential_solver == 1) {
        int it = fd_solve(s, res);
        *converged = 1;
        fd_fields(s);
        return it;
    }
    int it = poisson_solve(s, tol, max_iter, fixed, check, res, converged);
    potential_fields(s);
    return it;
}

int orc_get_field(const orc_state* s, int id, double* out) {
    const int N = s->N;
    const double* src = NULL;
    switch (id) {
        case F_PHI1: case F_PHI2: case F_PHI3: src = s->phi + (id - F_PHI1) * N; break;
        case F_UX: src = s->u; break;
        case F_UY: src = s->u + N; break;
        case F_P: src = s->pr; break;
        case F_Q: src = s->q; break;
        case F_PSI:
            if (s->p.potential_solver == 1) { src = s->psi; break; }
            for (int c = 0; c < N; ++c) out[c] = psi_moment(s, s->h, c);
            return 0;
        case F_EX: src = s->E; break;
        case F_EY: src = s->E + N; break;
        case F_MU1: case F_MU2: case F_MU3: src = s->mu + (id - F_MU1) * N; break;
        case F_PHINOW1: case F_PHINOW2: case F_PHINOW3: {
            int i = id - F_PHINOW1;
            for (int c = 0; c < N; ++c) {
                double a = 0.0;
                for (int j = 0; j < 9; ++j) a += s->f[(9 * i + j) * N + c];
                out[c] = a;
            }
            return 0;
        }
        case F_N1: case F_N2: {
            int i = id - F_N1;
            for (int c = 0; c < N; ++c) {
                double a = 0.0;
                for (int j = 0; j < 9; ++j) a += s->ion[(9 * i + j) * N + c];
                out[c] = a;
            }
            return 0;
        }
        case F_QTILDE:
            for (int c = 0; c < N; ++c) {
                double a = 0.0;
                for (int j = 0; j < 9; ++j) a += s->l[j * N + c];
                out[c] = a;
            }
            return 0;
        default: break;
    }
    if (!src && id >= POP_BASE && id < POP_BASE + 72) {
        int set = (id - POP_BASE) / 9, j = (id - POP_BASE) % 9;
        const double* base = set == 0 ? s->g : set <= 3 ? s->f + 9 * (set - 1) * (size_t)N : set == 4 ? s->l
                           : set == 5 ? s->h : s->ion + 9 * (set - 6) * (size_t)N;
        src = base + j * N;
    }
    if (!src) return -1;
    memcpy(out, src, (size_t)N * sizeof(double));
    return 0;
}

/* Observables of the last completed step (Eq. 18 energy parts, per-phase mass,
 * deformation factors).  out[0..2] mass, [3] charge, [4..7] F_phi F_E F_u F_q,
 * [8] max|sum phi - 1|, [9] D_inner, [10] D_outer, [11] nonfinite count,
 * [12] step, [13] last potential iterations, [14] last residual. */
int orc_observables(const orc_state* s, double* out) {
    const int nx = s->p.nx, ny = s->p.ny, N = s->N;
    const double D = s->p.width_D;
    double mass[3] = {0, 0, 0}, charge = 0, Fphi = 0, FE = 0, Fu = 0, Fq = 0, dev = 0, nonfin = 0;
    double m[2][5] = {{0}}; /* sum chi, chi x, chi y, chi x^2, chi y^2 */
    int ii = s->p.inner_phase - 1, im = s->p.matrix_phase - 1;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            double ph[3], sum = 0.0;
            phis(s, c, ph);
            for (int i = 0; i < 3; ++i) {
                double gx, gy;
                mass[i] += ph[i];
                sum += ph[i];
                grad_at(s, s->phi + i * N, x, y, &gx, &gy);
                Fphi += 6.0 / D * s->lam[i] * ph[i] * ph[i] * (1.0 - ph[i]) * (1.0 - ph[i])
                      + 0.375 * D * s->lam[i] * (gx * gx + gy * gy);
            }
            dev = fmax(dev, fabs(sum - 1.0));
            double eps = perm(&s->p, ph);
            double Ex = s->E[c], Ey = s->E[N + c];
            FE += 0.5 * eps * (Ex * Ex + Ey * Ey);                 /* |D|^2 / (2 eps) */
            double rho = ph[0] * s->p.rho[0] + ph[1] * s->p.rho[1] + ph[2] * s->p.rho[2];
            double ux = s->u[c], uy = s->u[N + c];
            Fu += 0.5 * rho * (ux * ux + uy * uy);
            double sg = ph[0] * s->p.sigma[0] + ph[1] * s->p.sigma[1] + ph[2] * s->p.sigma[2];
            if (sg > 0) Fq += 0.5 * (s->p.alpha / sg) * s->q[c] * s->q[c];
            charge += s->q[c];
            double chis[2] = {ph[ii], 1.0 - ph[im]};
            for (int k = 0; k < 2; ++k) {
                m[k][0] += chis[k];
                m[k][1] += chis[k] * x;
                m[k][2] += chis[k] * y;
                m[k][3] += chis[k] * x * x;
                m[k][4] += chis[k] * y * y;
            }
            double vals[6] = {ph[0], ph[1], ph[2], ux, uy, s->q[c]};
            for (int k = 0; k < 6; ++k)
                if (!isfinite(vals[k])) nonfin += 1;
        }
    double Dk[2];
    for (int k = 0; k < 2; ++k) {
        double A = m[k][0];
        if (!(A > 0)) { Dk[k] = 0.0; continue; }
        double xc = m[k][1] / A, yc = m[k][2] / A;
        double Ixx = m[k][3] / A - xc * xc, Iyy = m[k][4] / A - yc * yc;
        double a = 2.0 * sqrt(fmax(Iyy, 0.0)), b = 2.0 * sqrt(fmax(Ixx, 0.0));
        Dk[k] = (a + b) > 0 ? (a - b) / (a + b) : 0.0;   /* D = (r_par - r_perp)/(r_par + r_perp) */
    }
    out[0] = mass[0]; out[1] = mass[1]; out[2] = mass[2]; out[3] = charge;
    out[4] = Fphi; out[5] = FE; out[6] = Fu; out[7] = Fq; out[8] = dev;
    out[9] = Dk[0]; out[10] = Dk[1]; out[11] = nonfin; out[12] = (double)s->step;
    out[13] = s->last_iters; out[14] = s->last_res;
    return 0;
}

/* lattice constants (for the pins that check Eq. 31) */
void orc_lattice(int* cx, int* cy, double* w, int* opp) {
    for (int j = 0; j < 9; ++j) { cx[j] = CX[j]; cy[j] = CY[j]; w[j] = W[j]; opp[j] = OPP[j]; }
}

/* Eq. 33 stencils of a field on an nx*ny grid with the oracle's ghost rule */
int orc_stencil(int nx, int ny, int bc_y, const double* chi, double* gx, double* gy, double* lap) {
    orc_state t;
    memset(&t, 0, sizeof t);
    t.p.nx = nx; t.p.ny = ny; t.p.bc_y = bc_y; t.N = nx * ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int c = y * nx + x;
            grad_at(&t, chi, x, y, &gx[c], &gy[c]);
            lap[c] = lap_at(&t, chi, x, y);
        }
    return 0;
}

int orc_last_poisson(const orc_state* s, int* iters, double* res, int* converged) {
    *iters = s->last_iters; *res = s->last_res; *converged = s->last_converged;
    return 0;
}

int64_t orc_step_count(const orc_state* s) { return s->step; }

/* ---------------- test facility: storage-rounding perturbations ----------------
 * Not part of the method.  Perturbs every population of the sets g, f^1..f^3 and l
 * as storing it in a narrower floating-point format would: by u * max(rel |v|, floor)
 * with u uniform in [-1, 1) from a counter-based hash (splitmix64 of the seed and
 * the population's index), v the stored value.  The rest population of each phase
 * set is taken as stored by its deviation from phi_i of the last step, as the GPU's
 * narrow storage keeps it, and phi_i itself (held in a field of relative precision
 * field_rel) as rounded once more: the anchor phi_i is a running quantity, rounded
 * every step.  Used to measure how much the scheme itself amplifies perturbations
 * of FP32, BF16 or FP16 size (floor: the format's smallest spacing near zero, 0
 * where it plays no part). */
static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
static double unit_pm1(uint64_t seed, uint64_t i) {
    uint64_t r = splitmix64(seed * 0x100000001B3ull ^ splitmix64(i));
    return (double)(r >> 11) * (2.0 / 9007199254740992.0) - 1.0; /* [-1, 1) */
}
static double perturbed(double v, double rel, double floor_abs, uint64_t seed, uint64_t i) {
    double a = fabs(v) * rel;
    if (a < floor_abs) a = floor_abs;
    return v + unit_pm1(seed, i) * a;
}
int orc_perturb(orc_state* s, double rel, double floor_abs, double field_rel, uint64_t seed) {
    const int N = s->N;
    uint64_t k = 0;
    for (int i = 0; i < 9 * N; ++i, ++k) s->g[i] = perturbed(s->g[i], rel, floor_abs, seed, k);
    for (int set = 0; set < 3; ++set)
        for (int j = 0; j < 9; ++j)
            for (int c = 0; c < N; ++c, ++k) {
                double* f = &s->f[(size_t)(9 * set + j) * N + c];
                if (j == 0) {
                    const double anchor = s->phi[(size_t)set * N + c];
                    const double dev = perturbed(*f - anchor, rel, floor_abs, seed, k);
                    *f = perturbed(anchor, field_rel, 0.0, seed ^ 0x5bd1e995ull, k) + dev;
                } else {
                    *f = perturbed(*f, rel, floor_abs, seed, k);
                }
            }
    for (int i = 0; i < 9 * N; ++i, ++k) s->l[i] = perturbed(s->l[i], rel, floor_abs, seed, k);
    return 0;
}

/* Round-to-nearest-even of v to a binary format with `bits` significant bits whose
 * smallest spacing (subnormal range) is 2^min_exp. */
static double round_to_format(double v, int bits, int min_exp) {
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    frexp(fabs(v), &e);                  /* |v| = m 2^e, m in [0.5, 1) */
    int ex = e - bits;                   /* spacing of the format at |v| */
    if (ex < min_exp) ex = min_exp;
    const double q = ldexp(1.0, ex);
    return copysign(nearbyint(fabs(v) / q) * q, v);   /* default rounding mode: ties to even */
}
/* Test facility (not part of the method): replace the stored populations by their
 * values rounded to a storage format, as the GPU's builds store them:
 * fmt 1 FP32, 2 FP16 (11 bits, subnormal spacing 2^-24), 3 BF16 (8 bits).  The phase
 * rest populations are stored by their deviation from phi_i, and phi_i itself is an
 * FP32 field.  Deterministic: this emulates the storage rounding exactly (with FP64
 * arithmetic everywhere else). */
int orc_round_storage(orc_state* s, int fmt) {
    const int bits = fmt == 2 ? 11 : (fmt == 3 ? 8 : 24);
    const int min_exp = fmt == 2 ? -24 : -149;
    const int N = s->N;
    for (int i = 0; i < 9 * N; ++i) s->g[i] = round_to_format(s->g[i], bits, min_exp);
    for (int i = 0; i < 9 * N; ++i) s->l[i] = round_to_format(s->l[i], bits, min_exp);
    for (int set = 0; set < 3; ++set)
        for (int j = 0; j < 9; ++j)
            for (int c = 0; c < N; ++c) {
                double* f = &s->f[(size_t)(9 * set + j) * N + c];
                if (j == 0) {
                    const double anchor = round_to_format(s->phi[(size_t)set * N + c], 24, -149);
                    *f = anchor + round_to_format(*f - anchor, bits, min_exp);
                } else {
                    *f = round_to_format(*f, bits, min_exp);
                }
            }
    return 0;
}
