// lb3e_adjoint.cuh -- reverse mode (adjoint) of the two-dimensional step.
//
// The step maps the state X^n = (g, f, l, h, E, (phi_i u)^{n-1}, (q u)^{n-1}) and the
// parameters theta to X^{n+1}.  Given a^{n+1} = dJ/dX^{n+1} these kernels return
// a^n = (dX^{n+1}/dX^n)^T a^{n+1} and the parameter part (dX^{n+1}/dtheta)^T a^{n+1}
// (slots V_bottom, V_top, eps_1..3, sigma_1..3, gamma_12, gamma_13, gamma_23; the
// lambda_i of Eq. 9 map back to the gamma_jk).  The potential is differentiated
// through its fixed count of pseudo-time iterations (Eq. 43): a residual-controlled
// solve stops on a decision that has no derivative.
//
// Two groups of plain one-cell-per-thread kernels:
//  * the tape: the step's intermediates re-computed from X^n (moments, properties,
//    stencils, the charge closure, every potential iterate, E, R, mu, grad mu, F, u,
//    p), in the order of the step's statements;
//  * the transpose, statement by statement in reverse order.  A statement y = f(x)
//    of a cell becomes xbar += (df/dx)^T ybar; the stencils of Eq. 33 and the
//    streaming step are gathers forward, so their transposes are gathers from the
//    cells that read this one (the same links in the opposite direction, plus the
//    mirrored ghosts at walls).  Every kernel writes only its own cell.
// Parameter sums are FP64 block partials reduced in a fixed order, so repeated runs
// give the same bits.
//
// State-vector planes (N cells each, the layout of a^n and a^{n+1}): g 0-8, f 9-35
// (phase-major), l 36-44, h 45-53, E 54-55, (phi_i u)^{n-1} 56-61 (x, y per phase),
// (q u)^{n-1} 62-63.
#pragma once

#include "lb3e_kernels.cuh"

namespace lb3e {

enum { AV_G = 0, AV_F = 9, AV_L = 36, AV_H = 45, AV_E = 54, AV_PREV = 56, AV_N = 64 };
enum { AJ_VB = 0, AJ_VT = 1, AJ_EPS = 2, AJ_SIG = 5, AJ_GAM = 8, AJ_N = 11 };
constexpr int ADJ_THREADS = 256;

template <class R>
__device__ __forceinline__ R acs2() { return R(1.0 / 3.0); }
template <class R>
__device__ __forceinline__ R aw(int j) { return j == 0 ? R(4.0 / 9.0) : (j <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0)); }

// a / b in FP64 (the tape re-runs the FP64 step in its own rounding), a * (1/b) in
// FP32 (a division is a long instruction sequence there)
template <class R>
__device__ __forceinline__ R adiv(R a, R b, R ib) {
    if constexpr (std::is_same<R, double>::value) return a / b;
    else return a * ib;
}

// stencil ghost row: periodic, or mirrored about a half-way wall (Eq. 33 at walls)
__device__ __forceinline__ int adj_ghost_y(const DevParams& P, int y) {
    if (P.bc_y == 0) return y < 0 ? y + P.ny : (y >= P.ny ? y - P.ny : y);
    if (y < 0) return -1 - y;
    if (y >= P.ny) return 2 * P.ny - 1 - y;
    return y;
}
__device__ __forceinline__ int adj_wx(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

// s_j(u) of Eq. 40 and its gradient in u
template <class R>
__device__ __forceinline__ R adj_sj(int j, R ux, R uy) {
    const R cu = R(cx(j)) * ux + R(cy(j)) * uy, uu = ux * ux + uy * uy;
    return aw<R>(j) * (cu / acs2<R>() + cu * cu / (R(2) * acs2<R>() * acs2<R>()) - uu / (R(2) * acs2<R>()));
}

// the transposed gradient of Eq. 33 at cell (x, y): sum over the cells c and links j
// with ghost(c + c_j) = (x, y) of w_j c_j . gbar(c) / cs2
template <class R>
__device__ __forceinline__ R grad_T_at(const DevParams& P, const R* __restrict__ gx, const R* __restrict__ gy,
                                       int x, int y) {
    R acc = R(0);
    const int nx = P.nx, ny = P.ny;
#pragma unroll
    for (int j = 1; j < 9; ++j) {
        const R wc = aw<R>(j) / acs2<R>();
        const int sx = adj_wx(x - cx(j), nx);
        int sy = y - cy(j);
        bool in = true;
        if (P.bc_y == 0) sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        else in = sy >= 0 && sy < ny;
        if (in) {
            const int s = sy * nx + sx;
            acc += wc * (R(cx(j)) * gx[s] + R(cy(j)) * gy[s]);
        }
        if (P.bc_y != 0 && ((y == 0 && cy(j) == -1) || (y == ny - 1 && cy(j) == 1))) {
            const int s = y * nx + sx;  // a wall cell whose link j leaves the lattice reads its mirror, this cell
            acc += wc * (R(cx(j)) * gx[s] + R(cy(j)) * gy[s]);
        }
    }
    return acc;
}
// the transposed Laplacian of Eq. 33
template <class R>
__device__ __forceinline__ R lap_T_at(const DevParams& P, const R* __restrict__ lb, int x, int y) {
    R acc = R(0);
    const int nx = P.nx, ny = P.ny, c = y * nx + x;
#pragma unroll
    for (int j = 1; j < 9; ++j) {
        const R w2 = R(2) * aw<R>(j) / acs2<R>();
        const int sx = adj_wx(x - cx(j), nx);
        int sy = y - cy(j);
        bool in = true;
        if (P.bc_y == 0) sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        else in = sy >= 0 && sy < ny;
        if (in) acc += w2 * lb[sy * nx + sx];
        if (P.bc_y != 0 && ((y == 0 && cy(j) == -1) || (y == ny - 1 && cy(j) == 1))) acc += w2 * lb[y * nx + sx];
        acc -= w2 * lb[c];
    }
    return acc;
}

// the post-collision adjoint of link j of a plain bounce-back set (phase or charge
// populations): the streaming transposed, gathered from where the population went
template <class R>
__device__ __forceinline__ R post_T(const DevParams& P, const R* __restrict__ ain, int base, int j, int x, int y,
                                    int c) {
    const int yt = y + cy(j);
    if (P.bc_y != 0 && (yt < 0 || yt >= P.ny)) return ain[(size_t)(base + opp(j)) * P.N + c];
    const int t = (yt < 0 ? yt + P.ny : (yt >= P.ny ? yt - P.ny : yt)) * P.nx + adj_wx(x + cx(j), P.nx);
    return ain[(size_t)(base + j) * P.N + t];
}

// ============================================================ tape (forward re-run)

// the state vector of the current populations: the rest populations of the phase
// sets rebuilt from their anchor where the storage keeps deviations
template <class R, class S>
__global__ void k_adj_export(DevParams P, const S* __restrict__ pop, const R* __restrict__ phi_anchor,
                             const R* __restrict__ h, const R* __restrict__ E, const R* __restrict__ prev,
                             R* __restrict__ X) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    for (int k = 0; k < 45; ++k) {
        R v = R(Store<S>::ld(pop, (size_t)k * N + c));
        if (anchored<S>() && (k == 9 || k == 18 || k == 27)) v = phi_anchor[(size_t)((k - 9) / 9) * N + c] + v;
        X[(size_t)k * N + c] = v;
    }
    for (int j = 0; j < 9; ++j) X[(size_t)(AV_H + j) * N + c] = h[(size_t)j * N + c];
    for (int k = 0; k < 2; ++k) X[(size_t)(AV_E + k) * N + c] = E[(size_t)k * N + c];
    for (int k = 0; k < 8; ++k) X[(size_t)(AV_PREV + k) * N + c] = prev[(size_t)k * N + c];
}

// S1, S2: zeroth moments (or the given phi) and the properties of Eq. 29-30
template <class R>
__global__ void k_adj_props(DevParams P, const R* __restrict__ X, const R* __restrict__ phi_in,
                            R* __restrict__ phi, R* __restrict__ qt, R* __restrict__ rho, R* __restrict__ sig,
                            R* __restrict__ eps) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    R ph[3];
    for (int i = 0; i < 3; ++i) {
        if (phi_in) {
            ph[i] = phi_in[(size_t)i * N + c];
        } else {
            R a = R(0);
            for (int j = 0; j < 9; ++j) a += X[(size_t)(AV_F + 9 * i + j) * N + c];
            ph[i] = a;
        }
        phi[(size_t)i * N + c] = ph[i];
    }
    if (!phi_in) {
        R a = R(0);
        for (int j = 0; j < 9; ++j) a += X[(size_t)(AV_L + j) * N + c];
        qt[c] = a;
    }
    rho[c] = ph[0] * pv<R>(P.rho[0], P.frho[0]) + ph[1] * pv<R>(P.rho[1], P.frho[1]) + ph[2] * pv<R>(P.rho[2], P.frho[2]);
    sig[c] = ph[0] * pv<R>(P.sigma[0], P.fsig[0]) + ph[1] * pv<R>(P.sigma[1], P.fsig[1]) + ph[2] * pv<R>(P.sigma[2], P.fsig[2]);
    R e = R(0);
    for (int i = 0; i < 3; ++i) e += pv<R>(P.eps[i], P.feps[i]) * ph[i] * ph[i] * (R(3) - R(2) * ph[i]);
    eps[c] = e;
}

// S3 and S4: Laplacians of phi_i, gradients of eps, sigma, rho (Eq. 33); with
// `closure`, the charge q = (q~ + src/2) / (1 + r/2) with the previous field
template <class R>
__global__ void k_adj_stencils(DevParams P, const R* __restrict__ phi, const R* __restrict__ eps,
                               const R* __restrict__ sig, const R* __restrict__ rho, const R* __restrict__ Eprev,
                               const R* __restrict__ qt, int closure, R* __restrict__ lap, R* __restrict__ geps,
                               R* __restrict__ gsig, R* __restrict__ grho, R* __restrict__ q) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N, nx = P.nx;
    if (c >= N) return;
    const int x = c % nx, y = c / nx;
    int nb[9];
    for (int j = 0; j < 9; ++j) nb[j] = adj_ghost_y(P, y + cy(j)) * nx + adj_wx(x + cx(j), nx);
    for (int i = 0; i < 3; ++i) {
        const R* f = phi + (size_t)i * N;
        R a = R(0);
        for (int j = 0; j < 9; ++j) a += R(2) * aw<R>(j) * (f[nb[j]] - f[c]);
        lap[(size_t)i * N + c] = a / acs2<R>();
    }
    const R* fl[3] = {eps, sig, rho};
    R* gout[3] = {geps, gsig, grho};
    R g[3][2];
    for (int k = 0; k < 3; ++k) {
        R ax = R(0), ay = R(0);
        for (int j = 0; j < 9; ++j) {
            ax += aw<R>(j) * R(cx(j)) * fl[k][nb[j]];
            ay += aw<R>(j) * R(cy(j)) * fl[k][nb[j]];
        }
        g[k][0] = ax / acs2<R>();
        g[k][1] = ay / acs2<R>();
        gout[k][c] = g[k][0];
        gout[k][N + c] = g[k][1];
    }
    if (closure) {
        const R r = sig[c] / eps[c];
        const R Ex = Eprev[c], Ey = Eprev[N + c];
        const R src = r * (g[0][0] * Ex + g[0][1] * Ey) - (g[1][0] * Ex + g[1][1] * Ey);
        q[c] = (qt[c] + R(0.5) * src) / (R(1) + R(0.5) * r);
    }
}

// the potential populations at equilibrium with the linear electrode profile
// (the state's creation)
template <class R>
__global__ void k_adj_h_linear(DevParams P, R* __restrict__ h) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    const int y = c / P.nx;
    const R psi0 = P.bc_y == 2 ? pv<R>(P.V_bottom, P.fVb) + (pv<R>(P.V_top, P.fVt) - pv<R>(P.V_bottom, P.fVb)) * (R(y) + R(0.5)) / R(P.ny) : R(0);
    for (int j = 0; j < 9; ++j) h[(size_t)j * N + c] = j == 0 ? (aw<R>(0) - R(1)) * psi0 : aw<R>(j) * psi0;
}

// E = J(h) / (eps - eps_ref + cs2 tau_h) + E_ext (Eq. 45), or E_ext without a
// potential; J of the last iterate goes to Jout
template <class R>
__global__ void k_adj_field(DevParams P, const R* __restrict__ h, const R* __restrict__ eps, R* __restrict__ E,
                            R* __restrict__ Jout) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    if (!P.electric) {
        E[c] = R(P.E_ext[0]);
        E[N + c] = R(P.E_ext[1]);
        return;
    }
    R ax = R(0), ay = R(0);
    for (int j = 0; j < 9; ++j) {
        ax += R(cx(j)) * h[(size_t)j * N + c];
        ay += R(cy(j)) * h[(size_t)j * N + c];
    }
    Jout[c] = ax;
    Jout[N + c] = ay;
    const R den = eps[c] - pv<R>(P.eps_ref, P.feps_ref) + acs2<R>() * pv<R>(P.tau_h, P.ftau_h);
    const R gx = -ax / den, gy = -ay / den;
    E[c] = -gx + R(P.E_ext[0]);
    E[N + c] = -gy + R(P.E_ext[1]);
}

// R^n of Eq. 47 and the chemical potential of Eq. 20
template <class R>
__global__ void k_adj_source_mu(DevParams P, const R* __restrict__ phi, const R* __restrict__ lap,
                                const R* __restrict__ E, const R* __restrict__ q, const R* __restrict__ sig,
                                const R* __restrict__ eps, const R* __restrict__ geps, const R* __restrict__ gsig,
                                R* __restrict__ Rq, R* __restrict__ mu) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    const R Ex = E[c], Ey = E[N + c];
    const R r = sig[c] / eps[c];
    Rq[c] = -r * q[c] + r * (geps[c] * Ex + geps[N + c] * Ey) - (gsig[c] * Ex + gsig[N + c] * Ey);
    const R e2 = Ex * Ex + Ey * Ey;
    const R D = pv<R>(P.D, P.fD);
    for (int i = 0; i < 3; ++i) {
        const R ph = phi[(size_t)i * N + c], lam = pv<R>(P.lam[i], P.flam[i]);
        const R bulk = R(24) / D * lam * ph * (ph - R(0.5)) * (ph - R(1));
        const R grad = R(0.75) * D * lam * lap[(size_t)i * N + c];
        const R deps = R(6) * pv<R>(P.eps[i], P.feps[i]) * ph * (R(1) - ph);
        mu[(size_t)i * N + c] = bulk - grad - R(0.5) * deps * e2;
    }
}

// S7-S9: grad mu_i (Eq. 33), F = -sum phi_i grad mu_i + q E (Eq. 27b), u and p (Eq. 41)
template <class R>
__global__ void k_adj_force_flow(DevParams P, const R* __restrict__ phi, const R* __restrict__ mu,
                                 const R* __restrict__ q, const R* __restrict__ E, const R* __restrict__ X,
                                 const R* __restrict__ rho, const R* __restrict__ grho, R* __restrict__ gmu,
                                 R* __restrict__ F, R* __restrict__ u, R* __restrict__ pr) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N, nx = P.nx;
    if (c >= N) return;
    const int x = c % nx, y = c / nx;
    int nb[9];
    for (int j = 0; j < 9; ++j) nb[j] = adj_ghost_y(P, y + cy(j)) * nx + adj_wx(x + cx(j), nx);
    R Fx = R(0), Fy = R(0);
    for (int i = 0; i < 3; ++i) {
        const R* m = mu + (size_t)i * N;
        R ax = R(0), ay = R(0);
        for (int j = 0; j < 9; ++j) {
            ax += aw<R>(j) * R(cx(j)) * m[nb[j]];
            ay += aw<R>(j) * R(cy(j)) * m[nb[j]];
        }
        const R gx = ax / acs2<R>(), gy = ay / acs2<R>();
        gmu[(size_t)(2 * i) * N + c] = gx;
        gmu[(size_t)(2 * i + 1) * N + c] = gy;
        Fx -= phi[(size_t)i * N + c] * gx;
        Fy -= phi[(size_t)i * N + c] * gy;
    }
    Fx = Fx + q[c] * E[c];
    Fy = Fy + q[c] * E[N + c];
    F[c] = Fx;
    F[N + c] = Fy;
    R mx = R(0), my = R(0), g1 = R(0);
    for (int j = 0; j < 9; ++j) {
        const R gj = X[(size_t)(AV_G + j) * N + c];
        mx += R(cx(j)) * gj;
        my += R(cy(j)) * gj;
        if (j) g1 += gj;
    }
    const R rh = rho[c];
    const R ux = (mx + R(0.5) * Fx) / rh, uy = (my + R(0.5) * Fy) / rh;
    const R ugr = ux * grho[c] + uy * grho[N + c];
    u[c] = ux;
    u[N + c] = uy;
    pr[c] = acs2<R>() / (R(1) - aw<R>(0)) * (g1 + R(0.5) * ugr + rh * adj_sj<R>(0, ux, uy));
}

// ============================================================ transpose

// The transposed collisions and streaming (S10-S14), the d/dt state (S10), the flow
// moments (S9), the force (S8) and R^n, for one cell.  The post-collision adjoint
// of link j is gathered from where that population streamed (bounce-back at walls,
// with the moving-wall term's density dependence).
template <class R>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_collide_T(
    DevParams P, int first, const R* __restrict__ X, const R* __restrict__ ain, const R* __restrict__ phi,
    const R* __restrict__ q, const R* __restrict__ rho, const R* __restrict__ sig, const R* __restrict__ eps,
    const R* __restrict__ geps, const R* __restrict__ gsig, const R* __restrict__ grho, const R* __restrict__ E,
    const R* __restrict__ gmu, const R* __restrict__ F, const R* __restrict__ u, const R* __restrict__ pr,
    R* __restrict__ aout, R* __restrict__ a_phi, R* __restrict__ a_mu, R* __restrict__ a_gmu, R* __restrict__ a_q,
    R* __restrict__ a_E, R* __restrict__ a_rho, R* __restrict__ a_grho, R* __restrict__ a_geps,
    R* __restrict__ a_gsig, R* __restrict__ a_sig, R* __restrict__ a_eps) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N, nx = P.nx, ny = P.ny;
    if (c >= N) return;
    const int x = c % nx, y = c / nx;
    const R cs = acs2<R>(), ics = R(3), ics2 = R(9);
    // post-collision adjoint of (plane base, link j): S14 transposed
    R arho = R(0);
    auto post = [&](int base, int j, int kind) -> R {
        const int yt = y + cy(j);
        if (P.bc_y != 0 && (yt < 0 || yt >= ny)) {
            const R b = ain[(size_t)(base + opp(j)) * N + c];
            if (kind == 1) {
                const R uw = yt >= ny ? pv<R>(P.u_wall_top, P.fuwt) : pv<R>(P.u_wall_bottom, P.fuwb);
                arho += -R(2) * aw<R>(j) * (R(cx(j)) * uw) * ics * b;
            }
            return b;
        }
        const int t = (yt < 0 ? yt + ny : (yt >= ny ? yt - ny : yt)) * nx + adj_wx(x + cx(j), nx);
        return ain[(size_t)(base + j) * N + t];
    };
    R ph[3];
    for (int i = 0; i < 3; ++i) ph[i] = phi[(size_t)i * N + c];
    const R ux = u[c], uy = u[N + c], qc = q[c];
    R aph[3] = {R(0), R(0), R(0)}, amu[3] = {R(0), R(0), R(0)};
    R agm[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R aux = R(0), auy = R(0), aqc = R(0);
    // the d/dt state written at the end of the step
    for (int i = 0; i < 3; ++i) {
        const R bx = ain[(size_t)(AV_PREV + 2 * i) * N + c], by = ain[(size_t)(AV_PREV + 2 * i + 1) * N + c];
        aph[i] += ux * bx + uy * by;
        aux += ph[i] * bx;
        auy += ph[i] * by;
    }
    {
        const R bx = ain[(size_t)(AV_PREV + 6) * N + c], by = ain[(size_t)(AV_PREV + 7) * N + c];
        aqc += ux * bx + uy * by;
        aux += qc * bx;
        auy += qc * by;
    }
    // phase populations, Eq. 34-36, with the mobility of Eq. 28
    const R m0 = pv<R>(P.m0, P.fm0), itf = pv<R>(1.0 / P.tau_f, P.fitau_f), im0 = pv<R>(1.0 / P.m0, P.fim0);
    R aprev[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int i = 0; i < 3; ++i) {
        R aAx = R(0), aAy = R(0);
        for (int j = 0; j < 9; ++j) {
            const R fb = post(AV_F + 9 * i, j, 0);  // its direct part (1 - 1/tau_f) fb is added by k_adj_props_T
            const R feqb = fb * itf, Fjb = (R(1) - R(0.5) * itf) * fb;
            aAx += aw<R>(j) * R(cx(j)) * Fjb;
            aAy += aw<R>(j) * R(cy(j)) * Fjb;
            if (j == 0) {
                aph[i] += feqb;
                amu[i] += -(R(1) - aw<R>(0)) * feqb;
            } else {
                amu[i] += aw<R>(j) * feqb;
                const R tq = aw<R>(j) * feqb * ics;
                aph[i] += tq * (R(cx(j)) * ux + R(cy(j)) * uy);
                aux += tq * R(cx(j)) * ph[i];
                auy += tq * R(cy(j)) * ph[i];
            }
        }
        const R aYx = -aAx * im0, aYy = -aAy * im0;
        for (int k = 0; k < 3; ++k) {
            R Mii = R(0);
            for (int kk = 0; kk < 3; ++kk)
                if (kk != i) Mii += m0 * ph[i] * ph[kk];
            const R Mik = k == i ? Mii - m0 : -m0 * ph[i] * ph[k];
            agm[2 * k] += Mik * aYx;
            agm[2 * k + 1] += Mik * aYy;
            const R aM = aYx * gmu[(size_t)(2 * k) * N + c] + aYy * gmu[(size_t)(2 * k + 1) * N + c];
            if (k != i) {
                aph[i] += -m0 * ph[k] * aM;
                aph[k] += -m0 * ph[i] * aM;
            } else {
                for (int kk = 0; kk < 3; ++kk)
                    if (kk != i) {
                        aph[i] += m0 * ph[kk] * aM;
                        aph[kk] += m0 * ph[i] * aM;
                    }
            }
        }
        if (!first) {
            const R adx = aAx * ics, ady = aAy * ics;
            aph[i] += ux * adx + uy * ady;
            aux += ph[i] * adx;
            auy += ph[i] * ady;
            aprev[2 * i] -= adx;
            aprev[2 * i + 1] -= ady;
        }
    }
    // flow populations, Eq. 37-40
    const R rh = rho[c], p = pr[c];
    const R Fx = F[c], Fy = F[N + c], grx = grho[c], gry = grho[N + c];
    R tg = pv<R>(P.tau_g, P.ftau_g), eta = R(0);
    if (P.use_visc) {
        for (int i = 0; i < 3; ++i) eta += ph[i] * pv<R>(P.visc[i], P.fvisc[i]);
        tg = R(0.5) + eta / (rh * cs);
    }
    const R itg = R(1) / tg, irh = R(1) / rh;
    R ag[9], ap = R(0), agrx = R(0), agry = R(0), aFx = R(0), aFy = R(0), atg = R(0);
    {
        const R ugr = ux * grx + uy * gry;
        for (int j = 0; j < 9; ++j) {
            const R gb = post(AV_G, j, 1);
            ag[j] = (R(1) - itg) * gb;
            const R geqb = gb * itg, Gb = (R(1) - R(0.5) * itg) * gb;
            const R sj = adj_sj<R>(j, ux, uy);
            const R cu = R(cx(j)) * ux + R(cy(j)) * uy;
            const R cgr = R(cx(j)) * grx + R(cy(j)) * gry;
            if (P.use_visc) {
                const R geq = j == 0 ? (aw<R>(0) - R(1)) * p * ics + rh * sj : aw<R>(j) * p * ics + rh * sj;
                const R cF = R(cx(j)) * Fx + R(cy(j)) * Fy;
                const R G = aw<R>(j) * (ugr + cF * ics + (cu * cgr - cs * ugr) * ics);
                atg += gb * ((X[(size_t)(AV_G + j) * N + c] - geq) + R(0.5) * G) * (itg * itg);
            }
            ap += (j == 0 ? aw<R>(0) - R(1) : aw<R>(j)) * ics * geqb;
            arho += sj * geqb;
            aux += rh * geqb * aw<R>(j) * (R(cx(j)) * ics + cu * R(cx(j)) * ics2 - ux * ics);
            auy += rh * geqb * aw<R>(j) * (R(cy(j)) * ics + cu * R(cy(j)) * ics2 - uy * ics);
            // G_j: the u.grad rho terms cancel (their coefficient is w_j (1 - cs2/cs2) = 0)
            aFx += aw<R>(j) * R(cx(j)) * Gb * ics;
            aFy += aw<R>(j) * R(cy(j)) * Gb * ics;
            aux += aw<R>(j) * R(cx(j)) * cgr * Gb * ics;
            auy += aw<R>(j) * R(cy(j)) * cgr * Gb * ics;
            agrx += aw<R>(j) * R(cx(j)) * cu * Gb * ics;
            agry += aw<R>(j) * R(cy(j)) * cu * Gb * ics;
        }
        if (P.use_visc) {
            const R aeta = atg * irh * ics;
            arho += -atg * eta * irh * irh * ics;
            for (int i = 0; i < 3; ++i) aph[i] += pv<R>(P.visc[i], P.fvisc[i]) * aeta;
        }
    }
    // charge populations, Eq. 48-50
    R aR = R(0);
    {
        const R itl = pv<R>(1.0 / P.tau_l, P.fitau_l), pl = R(1) - R(0.5) * itl;
        R adqx = R(0), adqy = R(0);
        for (int j = 0; j < 9; ++j) {
            const R lb = post(AV_L, j, 0);
            aout[(size_t)(AV_L + j) * N + c] = (R(1) - itl) * lb;
            const R leqb = lb * itl;
            aR += pl * aw<R>(j) * lb;
            if (P.charge_convection) {
                const R cu = R(cx(j)) * ux + R(cy(j)) * uy;
                aqc += aw<R>(j) * (R(1) + cu * ics) * leqb;
                aux += aw<R>(j) * qc * R(cx(j)) * ics * leqb;
                auy += aw<R>(j) * qc * R(cy(j)) * ics * leqb;
                adqx += pl * aw<R>(j) * R(cx(j)) * lb * ics;
                adqy += pl * aw<R>(j) * R(cy(j)) * lb * ics;
            } else {
                aqc += aw<R>(j) * leqb;
            }
        }
        if (P.charge_convection && !first) {
            aqc += ux * adqx + uy * adqy;
            aux += qc * adqx;
            auy += qc * adqy;
            aprev[6] -= adqx;
            aprev[7] -= adqy;
        }
    }
    for (int k = 0; k < 8; ++k) aout[(size_t)(AV_PREV + k) * N + c] = aprev[k];
    // S9: u = (m + F/2) / rho, p = cs2/(1 - w0) (g1 + ugr/2 + rho s_0(u))
    {
        const R kp = cs * (R(1) / (R(1) - aw<R>(0)));
        const R ag1 = kp * ap, augr = R(0.5) * kp * ap;
        arho += kp * adj_sj<R>(0, ux, uy) * ap;
        aux += kp * rh * ap * aw<R>(0) * (-ux * ics);
        auy += kp * rh * ap * aw<R>(0) * (-uy * ics);
        aux += grx * augr;
        auy += gry * augr;
        agrx += ux * augr;
        agry += uy * augr;
        const R amx = aux * irh, amy = auy * irh;
        aFx += R(0.5) * amx;
        aFy += R(0.5) * amy;
        arho += -(ux * aux + uy * auy) * irh;
        for (int j = 0; j < 9; ++j)
            aout[(size_t)(AV_G + j) * N + c] = ag[j] + R(cx(j)) * amx + R(cy(j)) * amy + (j ? ag1 : R(0));
    }
    // S8: F = -sum phi_i grad mu_i + q E;  R^n = -r q + r geps.E - gsig.E, r = sig/eps
    const R Ex = E[c], Ey = E[N + c];
    R aEx = ain[(size_t)AV_E * N + c], aEy = ain[(size_t)(AV_E + 1) * N + c];
    for (int i = 0; i < 3; ++i) {
        aph[i] += -(gmu[(size_t)(2 * i) * N + c] * aFx + gmu[(size_t)(2 * i + 1) * N + c] * aFy);
        agm[2 * i] += -ph[i] * aFx;
        agm[2 * i + 1] += -ph[i] * aFy;
    }
    aqc += Ex * aFx + Ey * aFy;
    aEx += qc * aFx;
    aEy += qc * aFy;
    const R ieps = R(1) / eps[c], r = sig[c] * ieps;
    const R gex = geps[c], gey = geps[N + c], gsx = gsig[c], gsy = gsig[N + c];
    aqc += -r * aR;
    const R ar = (-qc + gex * Ex + gey * Ey) * aR;
    aEx += (r * gex - gsx) * aR;
    aEy += (r * gey - gsy) * aR;
    a_geps[c] = r * Ex * aR;
    a_geps[N + c] = r * Ey * aR;
    a_gsig[c] = -Ex * aR;
    a_gsig[N + c] = -Ey * aR;
    a_sig[c] = ar * ieps;
    a_eps[c] = -ar * r * ieps;
    for (int i = 0; i < 3; ++i) {
        a_phi[(size_t)i * N + c] = aph[i];
        a_mu[(size_t)i * N + c] = amu[i];
    }
    for (int k = 0; k < 6; ++k) a_gmu[(size_t)k * N + c] = agm[k];
    a_q[c] = aqc;
    a_E[c] = aEx;
    a_E[N + c] = aEy;
    a_rho[c] = arho;
    a_grho[c] = agrx;
    a_grho[N + c] = agry;
}

// S7 transposed (grad mu_i), then the chemical potential of Eq. 20 transposed; the
// density's gradient transposed.  Block partials: eps_1..3, lambda_1..3.
template <class R>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_mu_T(
    DevParams P, const R* __restrict__ phi, const R* __restrict__ lap, const R* __restrict__ E,
    const R* __restrict__ a_gmu, const R* __restrict__ a_grho, const R* __restrict__ a_mu_in,
    R* __restrict__ a_phi, R* __restrict__ a_lap, R* __restrict__ a_E, R* __restrict__ a_rho,
    double* __restrict__ partial) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N, nx = P.nx;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (c < N) {
        const int x = c % nx, y = c / nx;
        const R Ex = E[c], Ey = E[N + c];
        const R e2 = Ex * Ex + Ey * Ey, D = pv<R>(P.D, P.fD);
        R aEx = R(0), aEy = R(0);
        for (int i = 0; i < 3; ++i) {
            const R mb = (a_mu_in ? a_mu_in[(size_t)i * N + c] : R(0)) +
                         (a_gmu ? grad_T_at<R>(P, a_gmu + (size_t)(2 * i) * N, a_gmu + (size_t)(2 * i + 1) * N, x, y)
                                : R(0));
            const R ph = phi[(size_t)i * N + c], lam = pv<R>(P.lam[i], P.flam[i]), ei = pv<R>(P.eps[i], P.feps[i]);
            const R deps = R(6) * ei * ph * (R(1) - ph);
            a_phi[(size_t)i * N + c] += mb * (R(24) / D * lam * (R(3) * ph * ph - R(3) * ph + R(0.5)) -
                                              R(3) * ei * (R(1) - R(2) * ph) * e2);
            a_lap[(size_t)i * N + c] = -R(0.75) * D * lam * mb;
            aEx += -deps * Ex * mb;
            aEy += -deps * Ey * mb;
            v[3 + i] = (double)(mb * (R(24) / D * ph * (ph - R(0.5)) * (ph - R(1)) -
                                      R(0.75) * D * lap[(size_t)i * N + c]));
            v[i] = (double)(-R(3) * ph * (R(1) - ph) * e2 * mb);
        }
        a_E[c] += aEx;
        a_E[N + c] += aEy;
        if (a_grho) a_rho[c] += grad_T_at<R>(P, a_grho, a_grho + N, x, y);
    }
    block_reduce_store<6>(v, partial + (size_t)6 * blockIdx.x);
}

// E = J(h_K)/den + E_ext transposed into the last iterate's adjoint (hbar = the
// state's h adjoint plus this) and eps; J_K = sum_j c_j h_j of that iterate
template <class R>
__global__ void k_adj_field_T(DevParams P, const R* __restrict__ J, const R* __restrict__ eps,
                              const R* __restrict__ a_E, const R* __restrict__ ah_in, R* __restrict__ ah,
                              R* __restrict__ a_eps) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    const R iden = R(1) / (eps[c] - pv<R>(P.eps_ref, P.feps_ref) + acs2<R>() * pv<R>(P.tau_h, P.ftau_h));
    const R ax = J[c], ay = J[N + c];
    const R bx = a_E[c] * iden, by = a_E[N + c] * iden;
    for (int j = 0; j < 9; ++j) ah[(size_t)j * N + c] = ah_in[(size_t)j * N + c] + (R(cx(j)) * bx + R(cy(j)) * by);
    a_eps[c] += -(ax * bx + ay * by) * iden;
}

// S4 transposed: q = (q~ + src/2) / (1 + r/2), src = r geps.E' - gsig.E' with the
// previous field E' (a state plane): q~ = sum l adds to every l plane
template <class R>
__global__ void k_adj_closure_T(DevParams P, const R* __restrict__ X, const R* __restrict__ q,
                                const R* __restrict__ sig, const R* __restrict__ eps, const R* __restrict__ geps,
                                const R* __restrict__ gsig, const R* __restrict__ a_q, R* __restrict__ aout,
                                R* __restrict__ a_geps, R* __restrict__ a_gsig, R* __restrict__ a_sig,
                                R* __restrict__ a_eps) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    const R r = sig[c] / eps[c], d = R(1) + R(0.5) * r, aq = a_q[c];
    const R Ex = X[(size_t)AV_E * N + c], Ey = X[(size_t)(AV_E + 1) * N + c];
    const R gex = geps[c], gey = geps[N + c], gsx = gsig[c], gsy = gsig[N + c];
    const R aqt = aq / d, asrc = R(0.5) * aq / d;
    const R ar = R(0.5) * (-q[c] * aq / d) + (gex * Ex + gey * Ey) * asrc;
    a_geps[c] += r * Ex * asrc;
    a_geps[N + c] += r * Ey * asrc;
    a_gsig[c] += -Ex * asrc;
    a_gsig[N + c] += -Ey * asrc;
    aout[(size_t)AV_E * N + c] = (r * gex - gsx) * asrc;
    aout[(size_t)(AV_E + 1) * N + c] = (r * gey - gsy) * asrc;
    a_sig[c] += ar / eps[c];
    a_eps[c] += -ar * sig[c] / (eps[c] * eps[c]);
    for (int j = 0; j < 9; ++j) aout[(size_t)(AV_L + j) * N + c] += aqt;
}

// Fixed-order sum of the partials into the FP64 parameter adjoint (added), by one
// block: the mu-part (eps, lambda) and props-part (eps, sigma) partials of nb blocks
// each, the electrode columns (2 nx values of R) or nbv V partials, lambda mapped to
// gamma by Eq. 9.  Partials of the running kernel's other blocks are read past L1.
template <class R>
__device__ void params_reduce_block(const double* __restrict__ pmu, const double* pprops, int nb,
                                    const R* __restrict__ vbar, int nx, const double* __restrict__ pv, int nbv,
                                    double* __restrict__ dpar) {
    double v[14];
    for (int k = 0; k < 14; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        for (int k = 0; k < 6; ++k) v[k] += __ldcg(pmu + (size_t)6 * b + k);
        for (int k = 0; k < 6; ++k) v[6 + k] += __ldcg(pprops + (size_t)6 * b + k);
    }
    if (vbar)
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            v[12] += (double)vbar[x];
            v[13] += (double)vbar[nx + x];
        }
    if (pv)
        for (int b = threadIdx.x; b < nbv; b += blockDim.x) {
            v[12] += __ldcg(pv + (size_t)2 * b);
            v[13] += __ldcg(pv + (size_t)2 * b + 1);
        }
    __shared__ double out[14];
    block_reduce_store<14>(v, out);
    __syncthreads();
    if (threadIdx.x == 0) {
        // v: eps(mu) 0-2, lambda 3-5, eps(props) 6-8, sigma 9-11, V_bottom 12, V_top 13
        dpar[AJ_VB] += out[12];
        dpar[AJ_VT] += out[13];
        for (int i = 0; i < 3; ++i) {
            dpar[AJ_EPS + i] += out[i] + out[6 + i];
            dpar[AJ_SIG + i] += out[9 + i];
        }
        dpar[AJ_GAM + 0] += out[3] + out[4] - out[5];
        dpar[AJ_GAM + 1] += out[3] - out[4] + out[5];
        dpar[AJ_GAM + 2] += -out[3] + out[4] + out[5];
    }
}

// S3 and S2 transposed (Laplacians, gradients of eps and sigma, the properties of
// Eq. 29-30), then S1: phi_i = sum_j f^i_j adds phibar to every f^i plane, which here
// also gets its collision's direct part (1 - 1/tau_f) times the post-collision
// adjoint gathered from ain.  The h adjoint of the state is copied out here.  With
// dphi (the creation), phibar goes there in FP64 instead.  Block partials: eps_1..3,
// sigma_1..3; the last block to finish sums every partial of the step into dpar
// (the mu-part, these, the electrode columns or vpart's partials) and re-arms the
// counter.
template <class R>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_props_T(
    DevParams P, const R* __restrict__ phi, const R* __restrict__ a_lap, const R* __restrict__ a_geps,
    const R* __restrict__ a_gsig, const R* __restrict__ a_rho, const R* __restrict__ a_sig,
    const R* __restrict__ a_eps, const R* __restrict__ a_phi, const R* __restrict__ ah, const R* __restrict__ ain,
    R* __restrict__ aout, double* __restrict__ dphi, double* partial, const double* __restrict__ pmu,
    const R* __restrict__ vbar, const double* __restrict__ vpart, unsigned* __restrict__ count,
    double* __restrict__ dpar) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N, nx = P.nx;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (c < N) {
        const int x = c % nx, y = c / nx;
        const R ae = a_eps[c] + (a_geps ? grad_T_at<R>(P, a_geps, a_geps + N, x, y) : R(0));
        const R as = (a_sig ? a_sig[c] : R(0)) + (a_gsig ? grad_T_at<R>(P, a_gsig, a_gsig + N, x, y) : R(0));
        const R ar = a_rho ? a_rho[c] : R(0);
        const R dk = R(1) - R(1) / pv<R>(P.tau_f, P.ftau_f);
        for (int i = 0; i < 3; ++i) {
            const R ph = phi[(size_t)i * N + c];
            const R tot = a_phi[(size_t)i * N + c] + lap_T_at<R>(P, a_lap + (size_t)i * N, x, y) +
                          pv<R>(P.rho[i], P.frho[i]) * ar + pv<R>(P.sigma[i], P.fsig[i]) * as + pv<R>(P.eps[i], P.feps[i]) * R(6) * ph * (R(1) - ph) * ae;
            v[i] = (double)(ph * ph * (R(3) - R(2) * ph) * ae);
            v[3 + i] = (double)(ph * as);
            if (dphi) {
                dphi[(size_t)i * N + c] += (double)tot;
            } else {
                for (int j = 0; j < 9; ++j)
                    aout[(size_t)(AV_F + 9 * i + j) * N + c] = dk * post_T<R>(P, ain, AV_F + 9 * i, j, x, y, c) + tot;
            }
        }
        if (ah)
            for (int j = 0; j < 9; ++j) aout[(size_t)(AV_H + j) * N + c] = ah[(size_t)j * N + c];
    }
    block_reduce_store<6>(v, partial + (size_t)6 * blockIdx.x);
    __shared__ int is_last;
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        params_reduce_block<R>(pmu, partial, (int)gridDim.x, vbar, nx, vpart, vpart ? (int)gridDim.x : 0, dpar);
        if (threadIdx.x == 0) *count = 0u;
    }
}

// The creation's state transposed into its inputs: f = f_eq(phi, mu) with u held at
// its initial value, g = rho s_j(u), and the state's field; then Eq. 20 transposed
// (as k_adj_mu_T with no grad mu part).  Writes a_phi, a_mu, a_rho, a_E.
template <class R>
__global__ void k_adj_init_seed_T(DevParams P, const R* __restrict__ u, const R* __restrict__ ain,
                                  R* __restrict__ a_phi, R* __restrict__ a_mu, R* __restrict__ a_rho,
                                  R* __restrict__ a_E) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    const R ux = u ? u[c] : R(0), uy = u ? u[N + c] : R(0);
    for (int i = 0; i < 3; ++i) {
        R ap = R(0), am = R(0);
        for (int j = 0; j < 9; ++j) {
            const R fb = ain[(size_t)(AV_F + 9 * i + j) * N + c];
            if (j == 0) {
                ap += fb;
                am += -(R(1) - aw<R>(0)) * fb;
            } else {
                am += aw<R>(j) * fb;
                ap += aw<R>(j) * (R(cx(j)) * ux + R(cy(j)) * uy) / acs2<R>() * fb;
            }
        }
        a_phi[(size_t)i * N + c] = ap;
        a_mu[(size_t)i * N + c] = am;
    }
    R ar = R(0);
    for (int j = 0; j < 9; ++j) ar += adj_sj<R>(j, ux, uy) * ain[(size_t)(AV_G + j) * N + c];
    a_rho[c] = ar;
    a_E[c] = ain[(size_t)AV_E * N + c];
    a_E[N + c] = ain[(size_t)(AV_E + 1) * N + c];
}

// the linear electrode profile of the creation transposed: per-block partials of
// V_bottom, V_top
template <class R>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_h_linear_T(DevParams P, const R* __restrict__ ah,
                                                                double* __restrict__ partial) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0, 0};
    if (c < P.N && P.bc_y == 2) {
        const int y = c / P.nx;
        R apsi = R(0);
        for (int j = 0; j < 9; ++j) apsi += (j == 0 ? aw<R>(0) - R(1) : aw<R>(j)) * ah[(size_t)j * P.N + c];
        const R s = (R(y) + R(0.5)) / R(P.ny);
        v[1] = (double)(apsi * s);
        v[0] = (double)(apsi * (R(1) - s));
    }
    block_reduce_store<2>(v, partial + (size_t)2 * blockIdx.x);
}

// dst += src (FP64)
static __global__ void k_add_f64(double* __restrict__ dst, const double* __restrict__ src, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] += src[i];
}

// objective seeds: the state-vector adjoint of an objective of phi_i = sum_j f^i_j is
// dJ/dphi_i on every f^i plane (zero elsewhere).  Deformation factor: dD/dchi =
// sum_k dD/dm_k dm_k/dchi with m = (1, x, y, x^2, y^2) sums, chi = phi_inner or
// 1 - phi_matrix.  Shape objective: 2 (phi_i - target_i).
template <class R>
__global__ void k_adj_seed_deformation(DevParams P, int phase, double sign, double g0, double g1, double g2,
                                       double g3, double g4, R* __restrict__ aout) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    const double x = c % P.nx, y = c / P.nx;
    const R v = R(sign * (g0 + g1 * x + g2 * y + g3 * x * x + g4 * y * y));
    for (int k = 0; k < AV_N; ++k) aout[(size_t)k * N + c] = R(0);
    for (int j = 0; j < 9; ++j) aout[(size_t)(AV_F + 9 * phase + j) * N + c] = v;
}
template <class R>
__global__ void k_adj_seed_shape(DevParams P, const R* __restrict__ phi, const double* __restrict__ target,
                                 R* __restrict__ aout) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = P.N;
    if (c >= N) return;
    for (int k = 0; k < AV_N; ++k) aout[(size_t)k * N + c] = R(0);
    for (int i = 0; i < 3; ++i) {
        const R v = R(2.0 * ((double)phi[(size_t)i * N + c] - target[(size_t)i * N + c]));
        for (int j = 0; j < 9; ++j) aout[(size_t)(AV_F + 9 * i + j) * N + c] = v;
    }
}

// ============================================================ potential iterations in tiles
// (the tile geometry PT_* and tile_cell / tile_nb are those of k_poisson_tile)

// nit (<= PT_H) pseudo-time iterations of Eq. 43 from hin to hout, the first moment
// J of each input iterate to J + 2 N t (t = 0 .. nit - 1)
template <class R>
__global__ void __launch_bounds__(PT_NT) k_adj_pot_tape(DevParams P, const R* __restrict__ eps,
                                                        const R* __restrict__ q, const R* __restrict__ hin,
                                                        R* __restrict__ hout, R* __restrict__ J, int nit) {
    extern __shared__ __align__(16) unsigned char pt_raw[];
    R* cur = reinterpret_cast<R*>(pt_raw);
    R* post = cur + 9 * PT_NT;
    const TileCell tc = tile_cell(P);
    const int N = P.N, ny = P.ny;
    const R th = pv<R>(P.tau_h, P.ftau_h), ith = R(1) / th;
    R epshat = R(0), qc = R(0), den = R(1), iden = R(1);
    if (tc.present) {
        epshat = eps[tc.c] - pv<R>(P.eps_ref, P.feps_ref);
        qc = q[tc.c];
        den = epshat + acs2<R>() * th;
        iden = R(1) / den;
#pragma unroll
        for (int j = 0; j < 9; ++j) cur[j * PT_NT + tc.t] = hin[(size_t)j * N + tc.c];
    }
    const R ehc = adiv(epshat, acs2<R>(), R(3));
    for (int it = 0; it < nit; ++it) {
        __syncthreads();
        if (tc.present) {
            R hv[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) hv[j] = cur[j * PT_NT + tc.t];
            R a = R(0);
#pragma unroll
            for (int j = 1; j < 9; ++j) a += hv[j];
            const R psi = adiv(a, R(1) - aw<R>(0), R(9.0 / 5.0));
            R ax = R(0), ay = R(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                ax += R(cx(j)) * hv[j];
                ay += R(cy(j)) * hv[j];
            }
            if (tc.interior) {
                J[(size_t)(2 * it) * N + tc.c] = ax;
                J[(size_t)(2 * it + 1) * N + tc.c] = ay;
            }
            const R gx = -adiv(ax, den, iden), gy = -adiv(ay, den, iden);
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const R heq = j == 0 ? (aw<R>(0) - R(1)) * psi : aw<R>(j) * psi;
                const R varpi = j == 0 ? R(0) : R(1.0 / 8.0);
                const R cg = R(cx(j)) * gx + R(cy(j)) * gy;
                post[j * PT_NT + tc.t] =
                    hv[j] - adiv(hv[j] - heq, th, ith) - adiv(ehc * aw<R>(j) * cg, th, ith) + varpi * qc;
            }
        }
        __syncthreads();
        if (tc.present) {
            // pull: link j arrives from the cell at -c_j, or, where that is beyond a
            // wall, is this cell's own opp(j) population reflected there
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int ys = tc.gy - cy(j);
                R v;
                if (P.bc_y != 0 && (ys < 0 || ys >= ny)) {
                    const R o = post[opp(j) * PT_NT + tc.t];
                    const R vw = ys >= ny ? pv<R>(P.V_top, P.fVt) : pv<R>(P.V_bottom, P.fVb);
                    v = P.bc_y == 2 ? -o + R(2) * aw<R>(j) * vw : o;
                } else {
                    v = post[j * PT_NT + tile_nb(-cx(j), -cy(j))];
                }
                cur[j * PT_NT + tc.t] = v;
            }
        }
    }
    if (tc.interior)
#pragma unroll
        for (int j = 0; j < 9; ++j) hout[(size_t)j * N + tc.c] = cur[j * PT_NT + tc.t];
}

// nit (<= PT_H) transposed iterations, k = k0, k0 - 1, ..: J_k at J + 2 N k; the
// adjoint from ah_in to ah_out; eps, q and electrode adjoints accumulated by the
// interior cells
template <class R>
__global__ void __launch_bounds__(PT_NT) k_adj_pot_T(DevParams P, const R* __restrict__ J,
                                                     const R* __restrict__ eps, const R* __restrict__ ah_in,
                                                     R* __restrict__ ah_out, R* __restrict__ a_eps,
                                                     R* __restrict__ a_q, R* __restrict__ vbar, int k0, int nit) {
    extern __shared__ __align__(16) unsigned char pt_raw[];
    R* buf[2] = {reinterpret_cast<R*>(pt_raw), reinterpret_cast<R*>(pt_raw) + 9 * PT_NT};
    const TileCell tc = tile_cell(P);
    const int N = P.N, ny = P.ny;
    const R ith = pv<R>(1.0 / P.tau_h, P.fitau_h), ics = R(3);
    R epshat = R(0), iden = R(1);
    if (tc.present) {
        epshat = eps[tc.c] - pv<R>(P.eps_ref, P.feps_ref);
        iden = R(1) / (epshat + acs2<R>() * pv<R>(P.tau_h, P.ftau_h));
#pragma unroll
        for (int j = 0; j < 9; ++j) buf[0][j * PT_NT + tc.t] = ah_in[(size_t)j * N + tc.c];
    }
    const R kg = -(epshat * ics) * ith;
    const R apsi_c = ith * (R(1) / (R(1) - aw<R>(0)));
    R s_eh = R(0), s_q = R(0), s_v = R(0);
    for (int it = 0; it < nit; ++it) {
        const R* cur = buf[it & 1];
        R* nxt = buf[(it + 1) & 1];
        __syncthreads();
        if (tc.present) {
            const int k = k0 - it;
            R b[9], av = R(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int yt = tc.gy + cy(j);
                if (P.bc_y != 0 && (yt < 0 || yt >= ny)) {
                    const R t = cur[opp(j) * PT_NT + tc.t];
                    if (P.bc_y == 2) {
                        b[j] = -t;
                        av += R(2) * aw<R>(j) * t;
                    } else {
                        b[j] = t;
                    }
                } else {
                    b[j] = cur[j * PT_NT + tile_nb(cx(j), cy(j))];
                }
            }
            const R ax = J[(size_t)(2 * k) * N + tc.c], ay = J[(size_t)(2 * k + 1) * N + tc.c];
            const R gx = -ax * iden, gy = -ay * iden;
            R spsi = R(0), sgx = R(0), sgy = R(0), scg = R(0), sq = R(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                spsi += (j == 0 ? aw<R>(0) - R(1) : aw<R>(j)) * b[j];
                sgx += aw<R>(j) * R(cx(j)) * b[j];
                sgy += aw<R>(j) * R(cy(j)) * b[j];
                scg += aw<R>(j) * (R(cx(j)) * gx + R(cy(j)) * gy) * b[j];
                if (j) sq += b[j];
            }
            const R agx = kg * sgx, agy = kg * sgy;
            const R aax = -agx * iden, aay = -agy * iden;
            const R apsi_j = spsi * apsi_c;
#pragma unroll
            for (int j = 0; j < 9; ++j)
                nxt[j * PT_NT + tc.t] = (R(1) - ith) * b[j] + R(cx(j)) * aax + R(cy(j)) * aay + (j ? apsi_j : R(0));
            s_eh += -ics * ith * scg + (agx * ax + agy * ay) * iden * iden;
            s_q += sq * R(0.125);
            s_v += av;
        }
    }
    __syncthreads();
    if (tc.interior) {
        const R* fin = buf[nit & 1];
#pragma unroll
        for (int j = 0; j < 9; ++j) ah_out[(size_t)j * N + tc.c] = fin[j * PT_NT + tc.t];
        a_eps[tc.c] += s_eh;
        a_q[tc.c] += s_q;
        if (P.bc_y == 2 && (tc.gy == 0 || tc.gy == ny - 1)) vbar[(tc.gy == 0 ? 0 : P.nx) + tc.c % P.nx] += s_v;
    }
}

// ============================================================ host sequencing

// The adjoint workspace (caller-owned device memory): the tape of one step (the
// first moment of every potential iterate) and the adjoint scratch planes.
template <class R>
struct AdjointWS {
    R *X, *phi, *qt, *rho, *sig, *eps, *lap, *geps, *gsig, *grho, *q, *hb[2], *Jk, *E, *Rq, *mu, *gmu, *F, *u, *pr;
    R *a_phi, *a_mu, *a_gmu, *a_q, *a_E, *a_rho, *a_grho, *a_geps, *a_gsig, *a_sig, *a_eps, *a_lap, *a_h[2];
    R* vbar;
    double *pmu, *pprops, *pv, *dpar;
    unsigned* count;
    size_t total;

    static size_t align(size_t b) { return (b + 255) & ~(size_t)255; }
    // carve the layout from base (nullptr: sizes only)
    static AdjointWS make(const DevParams& P, int K, char* base) {
        AdjointWS w{};
        const size_t N = (size_t)P.N;
        const size_t nb = (N + ADJ_THREADS - 1) / ADJ_THREADS;
        size_t o = 0;
        auto R_ = [&](size_t planes) {
            R* p = base ? reinterpret_cast<R*>(base + o) : nullptr;
            o += align(planes * N * sizeof(R));
            return p;
        };
        auto D_ = [&](size_t n) {
            double* p = base ? reinterpret_cast<double*>(base + o) : nullptr;
            o += align(n * sizeof(double));
            return p;
        };
        w.X = R_(AV_N);
        w.phi = R_(3); w.qt = R_(1); w.rho = R_(1); w.sig = R_(1); w.eps = R_(1); w.lap = R_(3);
        w.geps = R_(2); w.gsig = R_(2); w.grho = R_(2); w.q = R_(1);
        w.hb[0] = R_(9); w.hb[1] = R_(9); w.Jk = R_((size_t)2 * (K + 1));
        w.E = R_(2); w.Rq = R_(1); w.mu = R_(3); w.gmu = R_(6); w.F = R_(2); w.u = R_(2); w.pr = R_(1);
        w.a_phi = R_(3); w.a_mu = R_(3); w.a_gmu = R_(6); w.a_q = R_(1); w.a_E = R_(2); w.a_rho = R_(1);
        w.a_grho = R_(2); w.a_geps = R_(2); w.a_gsig = R_(2); w.a_sig = R_(1); w.a_eps = R_(1); w.a_lap = R_(3);
        w.a_h[0] = R_(9); w.a_h[1] = R_(9);
        w.vbar = base ? reinterpret_cast<R*>(base + o) : nullptr;
        o += align(2 * (size_t)P.nx * sizeof(R));
        w.pmu = D_(6 * nb); w.pprops = D_(6 * nb); w.pv = D_(2 * nb); w.dpar = D_(AJ_N);
        w.count = reinterpret_cast<unsigned*>(D_(1));
        w.total = o;
        return w;
    }
};

// Runs the tape and the transposed kernels of one step (or of the state's creation)
// on a stream.  K is the fixed count of potential iterations (0 without a potential).
template <class R>
struct AdjointRunner {
    DevParams P;
    int K;
    cudaStream_t s;
    AdjointWS<R> w;
    int64_t launches = 0;
    unsigned nb() const { return (unsigned)((P.N + ADJ_THREADS - 1) / ADJ_THREADS); }
    dim3 pt_grid() const { return dim3((P.nx + PT_TX - 1) / PT_TX, (P.ny + PT_TY - 1) / PT_TY); }
    // the tiled potential kernels take more than the default 48 KB of shared memory
    // in FP64: set on the current device (before any launch, outside a stream capture)
    static int prepare() {
        if (cudaFuncSetAttribute(k_adj_pot_tape<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pt_smem_bytes<R>()) != cudaSuccess ||
            cudaFuncSetAttribute(k_adj_pot_T<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pt_smem_bytes<R>()) != cudaSuccess)
            return LB3E_ERR_CUDA;
        return LB3E_OK;
    }

    int ok() {
        ++launches;
        return cudaGetLastError() == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }
    // the tape from phi (phi_in, the creation) or from the state X (a step)
    int tape(const R* phi_in, int closure) {
        const unsigned g = nb(), t = ADJ_THREADS;
        const size_t N = (size_t)P.N;
        k_adj_props<R><<<g, t, 0, s>>>(P, w.X, phi_in, w.phi, w.qt, w.rho, w.sig, w.eps);
        TRY(ok());
        k_adj_stencils<R><<<g, t, 0, s>>>(P, w.phi, w.eps, w.sig, w.rho, w.X + (size_t)AV_E * N, w.qt, closure,
                                          w.lap, w.geps, w.gsig, w.grho, w.q);
        TRY(ok());
        int hc = 0;
        if (P.electric) {
            for (int k = 0; k < K; k += PT_H) {
                const int nit = K - k < PT_H ? K - k : PT_H;
                k_adj_pot_tape<R><<<pt_grid(), dim3(PT_W, PT_HT), pt_smem_bytes<R>(), s>>>(
                    P, w.eps, w.q, w.hb[hc], w.hb[hc ^ 1], w.Jk + (size_t)2 * k * N, nit);
                TRY(ok());
                hc ^= 1;
            }
        }
        k_adj_field<R><<<g, t, 0, s>>>(P, w.hb[hc], w.eps, w.E, w.Jk + (size_t)2 * K * N);
        TRY(ok());
        k_adj_source_mu<R><<<g, t, 0, s>>>(P, w.phi, w.lap, w.E, w.q, w.sig, w.eps, w.geps, w.gsig, w.Rq, w.mu);
        return ok();
    }
    // the potential part of the transpose: E, then the iterations in reverse; the
    // last adjoint of h ends in a_h[result]
    int potential_T(const R* ah_state, int* result) {
        const unsigned g = nb(), t = ADJ_THREADS;
        const size_t N = (size_t)P.N;
        if (!P.electric) {
            if (cudaMemcpyAsync(w.a_h[0], ah_state, 9 * N * sizeof(R), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return LB3E_ERR_CUDA;
            *result = 0;
            return LB3E_OK;
        }
        k_adj_field_T<R><<<g, t, 0, s>>>(P, w.Jk + (size_t)2 * K * N, w.eps, w.a_E, ah_state, w.a_h[0], w.a_eps);
        TRY(ok());
        int cur = 0;
        for (int k = K - 1; k >= 0; k -= PT_H) {
            const int nit = k + 1 < PT_H ? k + 1 : PT_H;
            k_adj_pot_T<R><<<pt_grid(), dim3(PT_W, PT_HT), pt_smem_bytes<R>(), s>>>(
                P, w.Jk, w.eps, w.a_h[cur], w.a_h[cur ^ 1], w.a_eps, w.a_q, w.vbar, k, nit);
            TRY(ok());
            cur ^= 1;
        }
        *result = cur;
        return LB3E_OK;
    }
    // the transpose of one step from the state X (already in w.X)
    int step_T(int first, const R* ain, R* aout) {
        const unsigned g = nb(), t = ADJ_THREADS;
        const size_t N = (size_t)P.N;
        if (cudaMemcpyAsync(w.hb[0], w.X + (size_t)AV_H * N, 9 * N * sizeof(R), cudaMemcpyDeviceToDevice, s) !=
                cudaSuccess ||
            cudaMemsetAsync(w.vbar, 0, 2 * (size_t)P.nx * sizeof(R), s) != cudaSuccess ||
            cudaMemsetAsync(w.count, 0, sizeof(unsigned), s) != cudaSuccess)
            return LB3E_ERR_CUDA;
        TRY(tape(nullptr, 1));
        k_adj_force_flow<R><<<g, t, 0, s>>>(P, w.phi, w.mu, w.q, w.E, w.X, w.rho, w.grho, w.gmu, w.F, w.u, w.pr);
        TRY(ok());
        k_adj_collide_T<R><<<g, t, 0, s>>>(P, first, w.X, ain, w.phi, w.q, w.rho, w.sig, w.eps, w.geps, w.gsig,
                                           w.grho, w.E, w.gmu, w.F, w.u, w.pr, aout, w.a_phi, w.a_mu, w.a_gmu,
                                           w.a_q, w.a_E, w.a_rho, w.a_grho, w.a_geps, w.a_gsig, w.a_sig, w.a_eps);
        TRY(ok());
        k_adj_mu_T<R><<<g, t, 0, s>>>(P, w.phi, w.lap, w.E, w.a_gmu, w.a_grho, w.a_mu, w.a_phi, w.a_lap, w.a_E,
                                      w.a_rho, w.pmu);
        TRY(ok());
        int hres = 0;
        TRY(potential_T(ain + (size_t)AV_H * N, &hres));
        k_adj_closure_T<R><<<g, t, 0, s>>>(P, w.X, w.q, w.sig, w.eps, w.geps, w.gsig, w.a_q, aout, w.a_geps,
                                           w.a_gsig, w.a_sig, w.a_eps);
        TRY(ok());
        k_adj_props_T<R><<<g, t, 0, s>>>(P, w.phi, w.a_lap, w.a_geps, w.a_gsig, w.a_rho, w.a_sig, w.a_eps, w.a_phi,
                                         w.a_h[hres], ain, aout, nullptr, w.pprops, w.pmu, w.vbar, nullptr, w.count,
                                         w.dpar);
        return ok();
    }
    // the transpose of the creation from phi_init (R planes, u held at zero)
    int init_T(const R* phi_init, const R* ain, double* dphi) {
        const unsigned g = nb(), t = ADJ_THREADS;
        const size_t N = (size_t)P.N;
        if (cudaMemsetAsync(w.q, 0, N * sizeof(R), s) != cudaSuccess ||
            cudaMemsetAsync(w.vbar, 0, 2 * (size_t)P.nx * sizeof(R), s) != cudaSuccess ||
            cudaMemsetAsync(w.a_eps, 0, N * sizeof(R), s) != cudaSuccess ||
            cudaMemsetAsync(w.a_q, 0, N * sizeof(R), s) != cudaSuccess ||
            cudaMemsetAsync(w.count, 0, sizeof(unsigned), s) != cudaSuccess)
            return LB3E_ERR_CUDA;
        k_adj_h_linear<R><<<g, t, 0, s>>>(P, w.hb[0]);
        TRY(ok());
        TRY(tape(phi_init, 0));
        k_adj_init_seed_T<R><<<g, t, 0, s>>>(P, nullptr, ain, w.a_phi, w.a_mu, w.a_rho, w.a_E);
        TRY(ok());
        k_adj_mu_T<R><<<g, t, 0, s>>>(P, w.phi, w.lap, w.E, nullptr, nullptr, w.a_mu, w.a_phi, w.a_lap, w.a_E,
                                      w.a_rho, w.pmu);
        TRY(ok());
        int hres = 0;
        TRY(potential_T(ain + (size_t)AV_H * N, &hres));
        k_adj_h_linear_T<R><<<g, t, 0, s>>>(P, w.a_h[hres], w.pv);
        TRY(ok());
        k_adj_props_T<R><<<g, t, 0, s>>>(P, w.phi, w.a_lap, nullptr, nullptr, w.a_rho, nullptr, w.a_eps, w.a_phi,
                                         nullptr, nullptr, nullptr, dphi, w.pprops, w.pmu, w.vbar, w.pv, w.count,
                                         w.dpar);
        return ok();
    }
};

}  // namespace lb3e
