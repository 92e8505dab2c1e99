/*
 * lb3e_oracle3d.c -- plain FP64 CPU oracle of the three-dimensional (D3Q15) form of
 * the three-phase EHD lattice Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY, like the two-dimensional oracle beside it: the test
 * suite, the smoke check and the benchmark's CPU leg load it; it shares no code with
 * the CUDA library.  Double precision, one cell at a time, in the order of the
 * paper's Section 3 with the D3Q15 lattice of Eq. 32 in place of D2Q9: moments,
 * properties (Eq. 29-30), isotropic stencils (Eq. 33 with the D3Q15 weights), the
 * potential solve (Eq. 42-45), the chemical potential (Eq. 20), the force (Eq.
 * 26/27b), flow moments (Eq. 41), collisions of the phase (Eq. 34-36), flow (Eq.
 * 37-40) and charge (Eq. 46-50) populations, streaming.  Build with
 * -ffp-contract=off.
 *
 * Readings beyond the two-dimensional ones: the potential source weights are
 * spread evenly over the 14 moving directions (varpi_0 = 0, varpi_j = 1/14, which
 * the paper states only for D2Q9 as 1/8); x and y are periodic and the walls (and
 * electrodes) sit at z = -1/2 and nz - 1/2, mirrored for the stencils; the
 * external field's second component lies along z (the wall normal); moving walls
 * slide along x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- D3Q15 lattice, Eq. 32 ---------------- */
#define Q 15
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1};
static const double W[Q] = {2.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
                            1.0 / 72.0, 1.0 / 72.0};
static const int OPP[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13};
#define CS2 (1.0 / 3.0)

/* parameters: the two-dimensional set plus nz; bc applies to the z walls */
typedef struct orc3_params {
    int32_t nx, ny, nz;
    int32_t bc;                /* 0 periodic, 1 walls, 2 walls + electrodes (normal to z) */
    int32_t electric;
    double rho[3], visc[3], tau_g;
    double gamma12, gamma13, gamma23, width_D, tau_f;
    double eps[3], sigma[3], eps_ref, alpha;
    double V_bottom, V_top;    /* electrode potentials at z = -1/2 and nz - 1/2 */
    double E_ext[2];           /* external field: [0] along x, [1] along z */
    double u_wall_bottom, u_wall_top; /* wall speeds along x */
    int32_t charge_convection, inner_phase, matrix_phase;
    double poisson_tol;
    int32_t poisson_max_iter, poisson_check_every, poisson_fixed_iter;
} orc3_params;

enum { G_PHI1 = 0, G_PHI2, G_PHI3, G_UX, G_UY, G_UZ, G_P, G_Q, G_PSI, G_EX, G_EY, G_EZ, G_MU1, G_MU2, G_MU3,
       G_PHINOW1, G_PHINOW2, G_PHINOW3, G_QTILDE };
enum { POP3_BASE = 100 }; /* POP3_BASE + 15*set + j, sets: g, f1, f2, f3, l, h */

typedef struct orc3_state {
    orc3_params p;
    int N;
    double lam[3], m0, tau_h, tau_l;
    double *g, *f, *l, *h, *gs, *fs, *ls, *hs;
    double *phi, *qt, *q, *rho, *sig, *eps, *lap, *geps, *gsig, *grho;
    double *E, *psi, *mu, *gmu, *F, *u, *pr, *R;
    double *prev_phiu, *prev_qu, *psi_prev, *J_prev;
    int64_t step;
    int last_iters;
    double last_res;
    int last_converged;
} orc3_state;

static double* alloc0(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }
static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* stencil ghost planes: periodic in z, or mirrored about the half-way wall */
static int ghost_z(const orc3_state* s, int z) {
    int nz = s->p.nz;
    if (s->p.bc == 0) return wrap(z, nz);
    if (z < 0) return -z - 1;
    if (z >= nz) return 2 * nz - z - 1;
    return z;
}
static double at(const orc3_state* s, const double* fld, int x, int y, int z) {
    return fld[(ghost_z(s, z) * s->p.ny + wrap(y, s->p.ny)) * s->p.nx + wrap(x, s->p.nx)];
}
/* Eq. 33 with the D3Q15 weights */
static void grad_at(const orc3_state* s, const double* fld, int x, int y, int z, double* g) {
    double a[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < Q; ++j) {
        double v = W[j] * at(s, fld, x + CX[j], y + CY[j], z + CZ[j]);
        a[0] += CX[j] * v;
        a[1] += CY[j] * v;
        a[2] += CZ[j] * v;
    }
    for (int k = 0; k < 3; ++k) g[k] = a[k] / CS2;
}
static double lap_at(const orc3_state* s, const double* fld, int x, int y, int z) {
    double c0 = at(s, fld, x, y, z), a = 0.0;
    for (int j = 0; j < Q; ++j) a += 2.0 * W[j] * (at(s, fld, x + CX[j], y + CY[j], z + CZ[j]) - c0);
    return a / CS2;
}

static double perm(const orc3_params* p, const double* ph) {   /* Eq. 30 */
    double e = 0.0;
    for (int i = 0; i < 3; ++i) e += p->eps[i] * ph[i] * ph[i] * (3.0 - 2.0 * ph[i]);
    return e;
}
static int use_visc(const orc3_params* p) { return p->visc[0] > 0 && p->visc[1] > 0 && p->visc[2] > 0; }
static void phis(const orc3_state* s, int c, double* ph) {
    for (int i = 0; i < 3; ++i) ph[i] = s->phi[i * s->N + c];
}

/* Eq. 45 moments of the potential populations */
static double psi_moment(const orc3_state* s, const double* h, int c) {
    double a = 0.0;
    for (int j = 1; j < Q; ++j) a += h[j * s->N + c];
    return a / (1.0 - W[0]);
}
static void first_moment(const orc3_state* s, const double* h, int c, double* J) {
    J[0] = J[1] = J[2] = 0.0;
    for (int j = 0; j < Q; ++j) {
        double v = h[j * s->N + c];
        J[0] += CX[j] * v;
        J[1] += CY[j] * v;
        J[2] += CZ[j] * v;
    }
}

/* Streaming: periodic in x and y; in z periodic or half-way bounce-back.  kind 0
 * plain bounce-back, 1 flow (moving wall along x), 2 potential (anti-bounce-back
 * to the electrode potential when bc == 2). */
static void stream(const orc3_state* s, const double* src, double* dst, int kind) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz, N = s->N;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c = (z * ny + y) * nx + x;
                for (int j = 0; j < Q; ++j) {
                    double v = src[j * N + c];
                    int zt = z + CZ[j];
                    if (s->p.bc != 0 && (zt < 0 || zt >= nz)) {
                        int top = zt >= nz;
                        double out = v;
                        if (kind == 1) {
                            double uw = top ? s->p.u_wall_top : s->p.u_wall_bottom;
                            out = v - 2.0 * W[j] * s->rho[c] * (CX[j] * uw) / CS2;
                        } else if (kind == 2 && s->p.bc == 2) {
                            double vw = top ? s->p.V_top : s->p.V_bottom;
                            out = -v + 2.0 * W[j] * vw;
                        }
                        dst[OPP[j] * N + c] = out;
                    } else {
                        int t = (wrap(zt, nz) * ny + wrap(y + CY[j], ny)) * nx + wrap(x + CX[j], nx);
                        dst[j * N + t] = v;
                    }
                }
            }
}

/* one pseudo-time iteration of Eq. 43 */
static void poisson_iteration(orc3_state* s) {
    const int N = s->N;
    const double th = s->tau_h;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; ++c) {
        double epshat = s->eps[c] - s->p.eps_ref;
        double psi = psi_moment(s, s->h, c), J[3], gpsi[3];
        first_moment(s, s->h, c, J);
        for (int k = 0; k < 3; ++k) gpsi[k] = -J[k] / (epshat + CS2 * th);
        for (int j = 0; j < Q; ++j) {
            double heq = (j == 0) ? (W[0] - 1.0) * psi : W[j] * psi;      /* Eq. 44 */
            double varpi = (j == 0) ? 0.0 : 1.0 / 14.0;
            double hj = s->h[j * N + c];
            double cg = CX[j] * gpsi[0] + CY[j] * gpsi[1] + CZ[j] * gpsi[2];
            s->hs[j * N + c] = hj - (hj - heq) / th - (epshat / CS2) * W[j] * cg / th + varpi * s->q[c];
        }
    }
    stream(s, s->hs, s->h, 2);
}

/* iterate until the relative increments of psi and J are <= tol (checked every
 * check iterations, before that iteration's collision), or a fixed count */
static int poisson_solve(orc3_state* s, double tol, int max_iter, int fixed, int check, double* res,
                         int* converged) {
    const int N = s->N;
    int n = fixed > 0 ? fixed : max_iter;
    if (check < 1) check = 1;
    *res = -1.0;
    *converged = fixed > 0;
    for (int k = 1; k <= n; ++k) {
        if (fixed <= 0 && k >= 2 && k % check == 0) {
            double dp = 0.0, pp = 0.0, dj = 0.0, jj = 0.0;
            for (int c = 0; c < N; ++c) {
                double pk = psi_moment(s, s->h, c), J[3];
                first_moment(s, s->h, c, J);
                double d = pk - s->psi_prev[c];
                dp += d * d;
                pp += pk * pk;
                for (int a = 0; a < 3; ++a) {
                    double e = J[a] - s->J_prev[a * N + c];
                    dj += e * e;
                    jj += J[a] * J[a];
                }
            }
            double r1 = pp > 0.0 ? sqrt(dp) / sqrt(pp) : (dp > 0.0 ? INFINITY : 0.0);
            double r2 = jj > 0.0 ? sqrt(dj) / sqrt(jj) : (dj > 0.0 ? INFINITY : 0.0);
            double r = r1 > r2 ? r1 : r2;
            *res = r;
            if (r <= tol) { *converged = 1; return k - 1; }
        }
        if (fixed <= 0 && (k + 1) % check == 0)
            for (int c = 0; c < N; ++c) {
                double J[3];
                s->psi_prev[c] = psi_moment(s, s->h, c);
                first_moment(s, s->h, c, J);
                for (int a = 0; a < 3; ++a) s->J_prev[a * N + c] = J[a];
            }
        poisson_iteration(s);
    }
    return n;
}

/* psi and E = -grad psi (+ external field: x and z components) */
static void potential_fields(orc3_state* s) {
    const int N = s->N;
    for (int c = 0; c < N; ++c) {
        double J[3], den = (s->eps[c] - s->p.eps_ref) + CS2 * s->tau_h;
        s->psi[c] = psi_moment(s, s->h, c);
        first_moment(s, s->h, c, J);
        s->E[c] = -(-J[0] / den) + s->p.E_ext[0];
        s->E[N + c] = -(-J[1] / den);
        s->E[2 * N + c] = -(-J[2] / den) + s->p.E_ext[1];
    }
}

/* S2 + S3 */
static void properties_and_stencils(orc3_state* s) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz, N = s->N;
    for (int c = 0; c < N; ++c) {
        double ph[3];
        phis(s, c, ph);
        s->rho[c] = ph[0] * s->p.rho[0] + ph[1] * s->p.rho[1] + ph[2] * s->p.rho[2];   /* Eq. 29 */
        s->sig[c] = ph[0] * s->p.sigma[0] + ph[1] * s->p.sigma[1] + ph[2] * s->p.sigma[2];
        s->eps[c] = perm(&s->p, ph);
    }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c = (z * ny + y) * nx + x;
                double g[3];
                for (int i = 0; i < 3; ++i) s->lap[i * N + c] = lap_at(s, s->phi + i * N, x, y, z);
                grad_at(s, s->eps, x, y, z, g);
                for (int a = 0; a < 3; ++a) s->geps[a * N + c] = g[a];
                grad_at(s, s->sig, x, y, z, g);
                for (int a = 0; a < 3; ++a) s->gsig[a * N + c] = g[a];
                grad_at(s, s->rho, x, y, z, g);
                for (int a = 0; a < 3; ++a) s->grho[a * N + c] = g[a];
            }
}

/* S6: Eq. 20 */
static void chemical_potential(orc3_state* s) {
    const int N = s->N;
    const double D = s->p.width_D;
    for (int c = 0; c < N; ++c) {
        double e2 = s->E[c] * s->E[c] + s->E[N + c] * s->E[N + c] + s->E[2 * N + c] * s->E[2 * N + c];
        for (int i = 0; i < 3; ++i) {
            double ph = s->phi[i * N + c];
            double bulk = 24.0 / D * s->lam[i] * ph * (ph - 0.5) * (ph - 1.0);
            double grad = 0.75 * D * s->lam[i] * s->lap[i * N + c];
            double deps = 6.0 * s->p.eps[i] * ph * (1.0 - ph);
            s->mu[i * N + c] = bulk - grad - 0.5 * deps * e2;
        }
    }
}

/* s_j(u), Eq. 40 */
static double s_j(int j, const double* u) {
    double cu = CX[j] * u[0] + CY[j] * u[1] + CZ[j] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[j] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}
static double tau_g_at(const orc3_state* s, int c) {
    if (!use_visc(&s->p)) return s->p.tau_g;
    double eta = 0.0;
    for (int i = 0; i < 3; ++i) eta += s->phi[i * s->N + c] * s->p.visc[i];
    return 0.5 + eta / (s->rho[c] * CS2);
}

/* S9: Eq. 41 */
static void flow_moments(orc3_state* s) {
    const int N = s->N;
    for (int c = 0; c < N; ++c) {
        double m[3] = {0.0, 0.0, 0.0}, g1 = 0.0, u[3];
        for (int j = 0; j < Q; ++j) {
            double gj = s->g[j * N + c];
            m[0] += CX[j] * gj;
            m[1] += CY[j] * gj;
            m[2] += CZ[j] * gj;
            if (j) g1 += gj;
        }
        for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * s->F[a * N + c]) / s->rho[c];
        double ugr = u[0] * s->grho[c] + u[1] * s->grho[N + c] + u[2] * s->grho[2 * N + c];
        for (int a = 0; a < 3; ++a) s->u[a * N + c] = u[a];
        s->pr[c] = CS2 / (1.0 - W[0]) * (g1 + 0.5 * ugr + s->rho[c] * s_j(0, u));
    }
}

/* S10-S13 collisions, then streaming */
static void collide_and_stream(orc3_state* s, int first) {
    const int N = s->N;
    const double tf = s->p.tau_f, tl = s->tau_l, m0 = s->m0;
    const int cc = s->p.charge_convection;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; ++c) {
        double ph[3], u[3], qc = s->q[c];
        phis(s, c, ph);
        for (int a = 0; a < 3; ++a) u[a] = s->u[a * N + c];
        double dpu[3][3], dqu[3];
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 3; ++a) dpu[i][a] = first ? 0.0 : ph[i] * u[a] - s->prev_phiu[(3 * i + a) * N + c];
        for (int a = 0; a < 3; ++a) dqu[a] = first ? 0.0 : qc * u[a] - s->prev_qu[a * N + c];

        /* phase populations, Eq. 34-36 with the mobility of Eq. 28 */
        for (int i = 0; i < 3; ++i) {
            double Y[3] = {0.0, 0.0, 0.0}, Mii = 0.0, A[3];
            for (int k = 0; k < 3; ++k)
                if (k != i) Mii += m0 * ph[i] * ph[k];
            for (int k = 0; k < 3; ++k) {
                double Mik = (k == i) ? (Mii - m0) : -m0 * ph[i] * ph[k];
                for (int a = 0; a < 3; ++a) Y[a] += Mik * s->gmu[(3 * k + a) * N + c];
            }
            for (int a = 0; a < 3; ++a) A[a] = dpu[i][a] / CS2 - Y[a] / m0;
            double mui = s->mu[i * N + c];
            for (int j = 0; j < Q; ++j) {
                double cpu = CX[j] * ph[i] * u[0] + CY[j] * ph[i] * u[1] + CZ[j] * ph[i] * u[2];
                double feq = (j == 0) ? ph[i] - (1.0 - W[0]) * mui : W[j] * mui + W[j] * cpu / CS2;
                double Fj = W[j] * (CX[j] * A[0] + CY[j] * A[1] + CZ[j] * A[2]);
                double fj = s->f[(Q * i + j) * N + c];
                s->fs[(Q * i + j) * N + c] = fj - (fj - feq) / tf + (1.0 - 1.0 / (2.0 * tf)) * Fj;
            }
        }
        /* flow populations, Eq. 37-40 */
        {
            double tg = tau_g_at(s, c), rho = s->rho[c], p = s->pr[c];
            double gr[3] = {s->grho[c], s->grho[N + c], s->grho[2 * N + c]};
            double Fv[3] = {s->F[c], s->F[N + c], s->F[2 * N + c]};
            double ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
            for (int j = 0; j < Q; ++j) {
                double geq = (j == 0) ? (W[0] - 1.0) * p / CS2 + rho * s_j(0, u) : W[j] * p / CS2 + rho * s_j(j, u);
                double cu = CX[j] * u[0] + CY[j] * u[1] + CZ[j] * u[2];
                double cgr = CX[j] * gr[0] + CY[j] * gr[1] + CZ[j] * gr[2];
                double cF = CX[j] * Fv[0] + CY[j] * Fv[1] + CZ[j] * Fv[2];
                double G = W[j] * (ugr + cF / CS2 + (cu * cgr - CS2 * ugr) / CS2);
                double gj = s->g[j * N + c];
                s->gs[j * N + c] = gj - (gj - geq) / tg + (1.0 - 1.0 / (2.0 * tg)) * G;
            }
        }
        /* charge populations, Eq. 48-50 */
        for (int j = 0; j < Q; ++j) {
            double cu = CX[j] * u[0] + CY[j] * u[1] + CZ[j] * u[2];
            double leq = cc ? W[j] * qc * (1.0 + cu / CS2) : W[j] * qc;
            double Sj = (1.0 - 1.0 / (2.0 * tl)) * W[j] * s->R[c];
            double Tj = cc ? (1.0 - 1.0 / (2.0 * tl)) * W[j] * (CX[j] * dqu[0] + CY[j] * dqu[1] + CZ[j] * dqu[2]) / CS2
                           : 0.0;
            double lj = s->l[j * N + c];
            s->ls[j * N + c] = lj - (lj - leq) / tl + Sj + Tj;
        }
    }
    for (int i = 0; i < 3; ++i) stream(s, s->fs + (size_t)Q * i * N, s->f + (size_t)Q * i * N, 0);
    stream(s, s->gs, s->g, 1);
    stream(s, s->ls, s->l, 0);
}

static void solve_now(orc3_state* s) {
    if (s->p.electric) {
        int conv;
        s->last_iters = poisson_solve(s, s->p.poisson_tol, s->p.poisson_max_iter, s->p.poisson_fixed_iter,
                                      s->p.poisson_check_every, &s->last_res, &conv);
        s->last_converged = conv;
        potential_fields(s);
    } else {
        for (int c = 0; c < s->N; ++c) {
            s->E[c] = s->p.E_ext[0];
            s->E[s->N + c] = 0.0;
            s->E[2 * s->N + c] = s->p.E_ext[1];
            s->psi[c] = 0.0;
        }
    }
}

static void one_step(orc3_state* s) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz, N = s->N;
    const int first = s->step == 0;
    /* S1 */
    for (int c = 0; c < N; ++c) {
        for (int i = 0; i < 3; ++i) {
            double a = 0.0;
            for (int j = 0; j < Q; ++j) a += s->f[(Q * i + j) * N + c];
            s->phi[i * N + c] = a;
        }
        double a = 0.0;
        for (int j = 0; j < Q; ++j) a += s->l[j * N + c];
        s->qt[c] = a;
    }
    properties_and_stencils(s);
    /* S4: closure with the previous step's field */
    for (int c = 0; c < N; ++c) {
        double r = s->sig[c] / s->eps[c], ge = 0.0, gs = 0.0;
        for (int a = 0; a < 3; ++a) {
            ge += s->geps[a * N + c] * s->E[a * N + c];
            gs += s->gsig[a * N + c] * s->E[a * N + c];
        }
        s->q[c] = (s->qt[c] + 0.5 * (r * ge - gs)) / (1.0 + 0.5 * r);
    }
    solve_now(s);   /* S5 */
    /* R^n of Eq. 47 */
    for (int c = 0; c < N; ++c) {
        double r = s->sig[c] / s->eps[c], ge = 0.0, gs = 0.0;
        for (int a = 0; a < 3; ++a) {
            ge += s->geps[a * N + c] * s->E[a * N + c];
            gs += s->gsig[a * N + c] * s->E[a * N + c];
        }
        s->R[c] = -r * s->q[c] + r * ge - gs;
    }
    chemical_potential(s);   /* S6 */
    for (int z = 0; z < nz; ++z)   /* S7 */
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c = (z * ny + y) * nx + x;
                for (int i = 0; i < 3; ++i) {
                    double g[3];
                    grad_at(s, s->mu + i * N, x, y, z, g);
                    for (int a = 0; a < 3; ++a) s->gmu[(3 * i + a) * N + c] = g[a];
                }
            }
    /* S8: F = -sum phi_i grad mu_i + q E */
    for (int c = 0; c < N; ++c)
        for (int a = 0; a < 3; ++a) {
            double Fa = 0.0;
            for (int i = 0; i < 3; ++i) Fa -= s->phi[i * N + c] * s->gmu[(3 * i + a) * N + c];
            s->F[a * N + c] = Fa + s->q[c] * s->E[a * N + c];
        }
    flow_moments(s);   /* S9 */
    collide_and_stream(s, first);
    for (int c = 0; c < N; ++c) {
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 3; ++a) s->prev_phiu[(3 * i + a) * N + c] = s->phi[i * N + c] * s->u[a * N + c];
        for (int a = 0; a < 3; ++a) s->prev_qu[a * N + c] = s->q[c] * s->u[a * N + c];
    }
    s->step += 1;
}

/* ---------------- public (test-only) API ---------------- */
void orc3_destroy(orc3_state* s) {
    if (!s) return;
    double* bufs[] = {s->g, s->f, s->l, s->h, s->gs, s->fs, s->ls, s->hs, s->phi, s->qt, s->q, s->rho, s->sig,
                      s->eps, s->lap, s->geps, s->gsig, s->grho, s->E, s->psi, s->mu, s->gmu, s->F, s->u, s->pr,
                      s->R, s->prev_phiu, s->prev_qu, s->psi_prev, s->J_prev};
    for (size_t k = 0; k < sizeof(bufs) / sizeof(bufs[0]); ++k) free(bufs[k]);
    free(s);
}

/* phi_init [3][nz][ny][nx]; u_init [3][..] or NULL; q_init [..] or NULL.
 * status: 0 ok, -1 bad parameters, -2 out of memory */
orc3_state* orc3_create(const orc3_params* p, const double* phi_init, const double* u_init, const double* q_init,
                        int* status) {
    *status = -1;
    if (p->nx < 2 || p->ny < 2 || p->nz < 2 || p->bc < 0 || p->bc > 2) return NULL;
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5) || !(p->width_D > 0) || !(p->eps_ref > 0) || !(p->alpha > 0))
        return NULL;
    for (int i = 0; i < 3; ++i)
        if (!(p->rho[i] > 0) || !(p->eps[i] > 0) || p->sigma[i] < 0) return NULL;
    double lam[3] = {p->gamma12 + p->gamma13 - p->gamma23, p->gamma12 + p->gamma23 - p->gamma13,
                     p->gamma13 + p->gamma23 - p->gamma12};   /* Eq. 9 */
    for (int i = 0; i < 3; ++i)
        if (!(lam[i] > 0)) return NULL;
    orc3_state* s = (orc3_state*)calloc(1, sizeof(orc3_state));
    *status = -2;
    if (!s) return NULL;
    s->p = *p;
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    s->N = (int)N;
    for (int i = 0; i < 3; ++i) s->lam[i] = lam[i];
    s->m0 = CS2 * (p->tau_f - 0.5);
    s->tau_h = 0.5 + p->eps_ref / CS2;
    s->tau_l = 0.5 + p->alpha / CS2;
    s->g = alloc0(Q * N); s->f = alloc0(3 * Q * N); s->l = alloc0(Q * N); s->h = alloc0(Q * N);
    s->gs = alloc0(Q * N); s->fs = alloc0(3 * Q * N); s->ls = alloc0(Q * N); s->hs = alloc0(Q * N);
    s->phi = alloc0(3 * N); s->qt = alloc0(N); s->q = alloc0(N); s->rho = alloc0(N); s->sig = alloc0(N);
    s->eps = alloc0(N); s->lap = alloc0(3 * N); s->geps = alloc0(3 * N); s->gsig = alloc0(3 * N);
    s->grho = alloc0(3 * N); s->E = alloc0(3 * N); s->psi = alloc0(N); s->mu = alloc0(3 * N);
    s->gmu = alloc0(9 * N); s->F = alloc0(3 * N); s->u = alloc0(3 * N); s->pr = alloc0(N); s->R = alloc0(N);
    s->prev_phiu = alloc0(9 * N); s->prev_qu = alloc0(3 * N); s->psi_prev = alloc0(N); s->J_prev = alloc0(3 * N);
    if (!s->J_prev) { orc3_destroy(s); return NULL; }
    memcpy(s->phi, phi_init, 3 * N * sizeof(double));
    if (u_init) memcpy(s->u, u_init, 3 * N * sizeof(double));
    if (q_init) memcpy(s->q, q_init, N * sizeof(double));
    properties_and_stencils(s);
    /* potential populations at equilibrium with the linear electrode profile */
    for (int z = 0; z < p->nz; ++z)
        for (int c2 = 0; c2 < p->nx * p->ny; ++c2) {
            int c = z * p->nx * p->ny + c2;
            double psi0 = p->bc == 2 ? p->V_bottom + (p->V_top - p->V_bottom) * (z + 0.5) / p->nz : 0.0;
            for (int j = 0; j < Q; ++j) s->h[j * N + c] = (j == 0) ? (W[0] - 1.0) * psi0 : W[j] * psi0;
        }
    solve_now(s);
    chemical_potential(s);
    const int cc = p->charge_convection;
    for (size_t c = 0; c < N; ++c) {
        double u[3] = {s->u[c], s->u[N + c], s->u[2 * N + c]};
        for (int i = 0; i < 3; ++i) {
            double ph = s->phi[i * N + c], mui = s->mu[i * N + c];
            for (int j = 0; j < Q; ++j) {
                double cpu = CX[j] * ph * u[0] + CY[j] * ph * u[1] + CZ[j] * ph * u[2];
                s->f[(Q * i + j) * N + c] = (j == 0) ? ph - (1.0 - W[0]) * mui : W[j] * mui + W[j] * cpu / CS2;
            }
        }
        for (int j = 0; j < Q; ++j) {
            s->g[j * N + c] = s->rho[c] * s_j(j, u);   /* g_eq with p = 0 */
            double cu = CX[j] * u[0] + CY[j] * u[1] + CZ[j] * u[2];
            s->l[j * N + c] = cc ? W[j] * s->q[c] * (1.0 + cu / CS2) : W[j] * s->q[c];
        }
    }
    s->step = 0;
    *status = 0;
    return s;
}

int orc3_step(orc3_state* s, int nsteps) {
    for (int k = 0; k < nsteps; ++k) one_step(s);
    return 0;
}

int orc3_get_field(const orc3_state* s, int id, double* out) {
    const int N = s->N;
    const double* src = NULL;
    switch (id) {
        case G_PHI1: case G_PHI2: case G_PHI3: src = s->phi + (id - G_PHI1) * N; break;
        case G_UX: case G_UY: case G_UZ: src = s->u + (id - G_UX) * N; break;
        case G_P: src = s->pr; break;
        case G_Q: src = s->q; break;
        case G_PSI:
            for (int c = 0; c < N; ++c) out[c] = psi_moment(s, s->h, c);
            return 0;
        case G_EX: case G_EY: case G_EZ: src = s->E + (id - G_EX) * N; break;
        case G_MU1: case G_MU2: case G_MU3: src = s->mu + (id - G_MU1) * N; break;
        case G_PHINOW1: case G_PHINOW2: case G_PHINOW3: {
            int i = id - G_PHINOW1;
            for (int c = 0; c < N; ++c) {
                double a = 0.0;
                for (int j = 0; j < Q; ++j) a += s->f[(Q * i + j) * N + c];
                out[c] = a;
            }
            return 0;
        }
        case G_QTILDE:
            for (int c = 0; c < N; ++c) {
                double a = 0.0;
                for (int j = 0; j < Q; ++j) a += s->l[j * N + c];
                out[c] = a;
            }
            return 0;
        default: break;
    }
    if (!src && id >= POP3_BASE && id < POP3_BASE + 6 * Q) {
        int set = (id - POP3_BASE) / Q, j = (id - POP3_BASE) % Q;
        const double* base = set == 0 ? s->g : set <= 3 ? s->f + (size_t)Q * (set - 1) * N : set == 4 ? s->l : s->h;
        src = base + (size_t)j * N;
    }
    if (!src) return -1;
    memcpy(out, src, (size_t)N * sizeof(double));
    return 0;
}

/* out[0..2] mass, [3] charge, [4] max|sum phi - 1|, [5] D_inner, [6] D_outer,
 * [7] nonfinite, [8] step, [9] last potential iterations, [10] last residual.
 * D = (a - b)/(a + b) with a along z (the wall normal, the field of the
 * electrodes) and b along x, from second moments of the phase indicators. */
int orc3_observables(const orc3_state* s, double* out) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz, N = s->N;
    double mass[3] = {0, 0, 0}, charge = 0, dev = 0, nonfin = 0, m[2][5] = {{0}};
    int ii = s->p.inner_phase - 1, im = s->p.matrix_phase - 1;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c = (z * ny + y) * nx + x;
                double ph[3], sum = 0.0;
                phis(s, c, ph);
                for (int i = 0; i < 3; ++i) { mass[i] += ph[i]; sum += ph[i]; }
                dev = fmax(dev, fabs(sum - 1.0));
                charge += s->q[c];
                double chis[2] = {ph[ii], 1.0 - ph[im]};
                for (int k = 0; k < 2; ++k) {
                    m[k][0] += chis[k];
                    m[k][1] += chis[k] * x;
                    m[k][2] += chis[k] * z;
                    m[k][3] += chis[k] * x * x;
                    m[k][4] += chis[k] * z * z;
                }
                double vals[7] = {ph[0], ph[1], ph[2], s->u[c], s->u[N + c], s->u[2 * N + c], s->q[c]};
                for (int k = 0; k < 7; ++k)
                    if (!isfinite(vals[k])) nonfin += 1;
            }
    for (int k = 0; k < 2; ++k) {
        double A = m[k][0], Dk = 0.0;
        if (A > 0) {
            double xc = m[k][1] / A, zc = m[k][2] / A;
            double Ixx = m[k][3] / A - xc * xc, Izz = m[k][4] / A - zc * zc;
            double a = 2.0 * sqrt(fmax(Izz, 0.0)), b = 2.0 * sqrt(fmax(Ixx, 0.0));
            Dk = (a + b) > 0 ? (a - b) / (a + b) : 0.0;
        }
        out[5 + k] = Dk;
    }
    out[0] = mass[0]; out[1] = mass[1]; out[2] = mass[2]; out[3] = charge; out[4] = dev;
    out[7] = nonfin; out[8] = (double)s->step; out[9] = s->last_iters; out[10] = s->last_res;
    return 0;
}

void orc3_lattice(int* cx, int* cy, int* cz, double* w, int* opp) {
    for (int j = 0; j < Q; ++j) { cx[j] = CX[j]; cy[j] = CY[j]; cz[j] = CZ[j]; w[j] = W[j]; opp[j] = OPP[j]; }
}

/* Eq. 33 stencils (D3Q15) of a field on an nx*ny*nz grid with the oracle's ghost rule */
int orc3_stencil(int nx, int ny, int nz, int bc, const double* chi, double* g, double* lap) {
    orc3_state t;
    memset(&t, 0, sizeof t);
    t.p.nx = nx; t.p.ny = ny; t.p.nz = nz; t.p.bc = bc; t.N = nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c = (z * ny + y) * nx + x;
                double gg[3];
                grad_at(&t, chi, x, y, z, gg);
                for (int a = 0; a < 3; ++a) g[a * t.N + c] = gg[a];
                lap[c] = lap_at(&t, chi, x, y, z);
            }
    return 0;
}

int64_t orc3_step_count(const orc3_state* s) { return s->step; }
