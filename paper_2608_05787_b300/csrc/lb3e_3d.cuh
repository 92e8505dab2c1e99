// lb3e_3d.cuh -- the three-dimensional step on the D3Q15 lattice (Eq. 32): the
// schemes of Section 3 with 15 directions, the isotropic stencils of Eq. 33 with
// the D3Q15 weights, x and y periodic, walls (and electrodes) normal to z.
//
// Blocks of 32 x 8 cells in an x-y plane: one thread a cell and one grid layer a z
// plane, except the TMA-staged potential iteration (a block walks two planes) and
// the observables (a thread sums 16 planes).  Populations are structure-of-arrays
// planes (15 set + j) * N + cell, cell = (z ny + y) nx + x, sets g, f1, f2, f3, l;
// the potential populations h have their own 15 planes.  Push streaming between two
// buffers.
//
// Readings beyond the two-dimensional ones: the potential source is split evenly
// over the 14 moving directions (varpi_j = 1/14; the paper gives 1/8 on D2Q9's 8);
// the external field is (E_ext[0], 0, E_ext[1]) -- its second component along the
// wall normal; moving walls slide along x.
//
// The FP64 build evaluates each formula in the order a plain C evaluation takes
// it (compiled without FMA contraction), so it reproduces a plain FP64 CPU
// evaluation to rounding of reductions; the FP32 build uses the same expressions.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "lb3e_internal.h"
#include "lb3e_kernels.cuh"

namespace lb3e {

// ---------------------------------------------------------------- D3Q15 (Eq. 32)
__host__ __device__ constexpr int c3x(int j) {
    return (j == 1 || j == 7 || j == 9 || j == 11 || j == 14) ? 1 : (j == 2 || j == 8 || j == 10 || j == 12 || j == 13) ? -1 : 0;
}
__host__ __device__ constexpr int c3y(int j) {
    return (j == 3 || j == 7 || j == 9 || j == 12 || j == 13) ? 1 : (j == 4 || j == 8 || j == 10 || j == 11 || j == 14) ? -1 : 0;
}
__host__ __device__ constexpr int c3z(int j) {
    return (j == 5 || j == 7 || j == 10 || j == 11 || j == 13) ? 1 : (j == 6 || j == 8 || j == 9 || j == 12 || j == 14) ? -1 : 0;
}
__host__ __device__ constexpr int opp3(int j) { return j == 0 ? 0 : ((j & 1) ? j + 1 : j - 1); }
template <class R>
__host__ __device__ constexpr R w3(int j) { return j == 0 ? R(2.0 / 9.0) : (j <= 6 ? R(1.0 / 9.0) : R(1.0 / 72.0)); }
constexpr int Q3 = 15;

// c_j . (a, b, c) in the order x, y, z, zero components left out (the same value as
// cx*a + cy*b + cz*c: a product with a zero component only adds a signed zero)
template <class R>
__device__ __forceinline__ R cdot3(int j, R a, R b, R c) {
    R s = R(0);
    bool any = false;
    if (c3x(j) != 0) { s = c3x(j) > 0 ? a : -a; any = true; }
    if (c3y(j) != 0) { s = any ? (c3y(j) > 0 ? s + b : s - b) : (c3y(j) > 0 ? b : -b); any = true; }
    if (c3z(j) != 0) { s = any ? (c3z(j) > 0 ? s + c : s - c) : (c3z(j) > 0 ? c : -c); }
    return s;
}
template <class R>
__device__ __forceinline__ R ocs2(R a) { return exact_arith<R>() ? a / (R(1) / R(3)) : a * R(3); }

// launch-wide parameters (formed on the host in double precision)
struct P3 {
    int nx, ny, nz, bc, cc, use_visc;
    size_t N;
    double rho[3], visc[3], tau_g, lam[3], D, tau_f, m0, eps[3], sigma[3], eps_ref, tau_h, tau_l;
    double V_bottom, V_top, E0, E1, uwb, uwt;
    int inner, matrix;
    // FP32 roundings of the above and of the reciprocals the collisions take, formed on
    // the host (a double parameter converted or divided in device code costs FP64
    // instructions, a small fraction of the FP32 rate on this part)
    float frho[3], fvisc[3], flam[3], feps[3], fsig[3];
    float fD, ftau_f, fitau_f, fm0, fim0, ftau_g, ftau_l, fitau_l, feps_ref, ftau_h, fitau_h;
    float fVb, fVt, fE0, fE1, fuwb, fuwt;
};

inline P3 make_p3(const lb3e_params& p) {
    P3 q{};
    q.nx = p.nx; q.ny = p.ny; q.nz = p.nz; q.bc = p.bc_y; q.cc = p.charge_convection;
    q.use_visc = p.visc[0] > 0 && p.visc[1] > 0 && p.visc[2] > 0;
    q.N = (size_t)p.nx * p.ny * p.nz;
    for (int i = 0; i < 3; ++i) {
        q.rho[i] = p.rho[i]; q.visc[i] = p.visc[i]; q.eps[i] = p.eps[i]; q.sigma[i] = p.sigma[i];
    }
    q.lam[0] = p.gamma12 + p.gamma13 - p.gamma23;   // Eq. 9
    q.lam[1] = p.gamma12 + p.gamma23 - p.gamma13;
    q.lam[2] = p.gamma13 + p.gamma23 - p.gamma12;
    const double c2 = 1.0 / 3.0;
    q.tau_g = p.tau_g; q.D = p.width_D; q.tau_f = p.tau_f; q.m0 = c2 * (p.tau_f - 0.5);
    q.eps_ref = p.eps_ref; q.tau_h = 0.5 + p.eps_ref / c2; q.tau_l = 0.5 + p.alpha / c2;
    q.V_bottom = p.V_bottom; q.V_top = p.V_top; q.E0 = p.E_ext[0]; q.E1 = p.E_ext[1];
    q.uwb = p.u_wall_bottom; q.uwt = p.u_wall_top;
    q.inner = p.inner_phase; q.matrix = p.matrix_phase;
    for (int i = 0; i < 3; ++i) {
        q.frho[i] = (float)q.rho[i]; q.fvisc[i] = (float)q.visc[i]; q.flam[i] = (float)q.lam[i];
        q.feps[i] = (float)q.eps[i]; q.fsig[i] = (float)q.sigma[i];
    }
    q.fD = (float)q.D; q.ftau_f = (float)q.tau_f; q.fitau_f = (float)(1.0 / q.tau_f);
    q.fm0 = (float)q.m0; q.fim0 = (float)(1.0 / q.m0); q.ftau_g = (float)q.tau_g;
    q.ftau_l = (float)q.tau_l; q.fitau_l = (float)(1.0 / q.tau_l); q.feps_ref = (float)q.eps_ref;
    q.ftau_h = (float)q.tau_h; q.fitau_h = (float)(1.0 / q.tau_h);
    q.fVb = (float)q.V_bottom; q.fVt = (float)q.V_top; q.fE0 = (float)q.E0; q.fE1 = (float)q.E1;
    q.fuwb = (float)q.uwb; q.fuwt = (float)q.uwt;
    return q;
}

// cell coordinates of this thread; false outside the lattice
__device__ __forceinline__ bool cell3(const P3& P, int& x, int& y, int& z, size_t& c) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = blockIdx.z;
    c = ((size_t)z * P.ny + y) * P.nx + x;
    return x < P.nx && y < P.ny;
}
// A block's stencil tile: its 32 x 8 cells with a one-cell ring, on the planes z - 1,
// z, z + 1 (x and y periodic; z periodic or mirrored at the walls, the stencil
// ghosts), one 34 x 10 x 3 array a field in shared memory
constexpr int K3X = 34, K3Y = 10, K3P = K3X * K3Y, K3F = 3 * K3P;
// stage M fields' tiles (all threads of the 32 x 8 block, also those outside the
// lattice; 32-bit indices: at most LB3E_MAX_CELLS cells)
template <class R, int M>
__device__ __forceinline__ void stage_tile3(const P3& P, const R* const (&fl)[M], R* __restrict__ st) {
    const int x0 = blockIdx.x * 32 - 1, y0 = blockIdx.y * 8 - 1, zc = blockIdx.z;
    const unsigned nx = (unsigned)P.nx, nxy = nx * (unsigned)P.ny;
    unsigned zo[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int zz = zc + d - 1;
        if (P.bc == 0) zz = zz < 0 ? zz + P.nz : (zz >= P.nz ? zz - P.nz : zz);
        else zz = zz < 0 ? -zz - 1 : (zz >= P.nz ? 2 * P.nz - zz - 1 : zz);
        zo[d] = (unsigned)zz * nxy;
    }
    // every load of the thread issued before the first store: IT x M loads in flight
    constexpr int IT = (K3F + 255) / 256;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    R v[IT][M];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int k = tid + 256 * it;
        if (k < K3F) {
            const int pz = k / K3P, r = k - pz * K3P, ly = r / K3X, lx = r - ly * K3X;
            const unsigned n = zo[pz] + (unsigned)wrapi(y0 + ly, P.ny) * nx + (unsigned)wrapi(x0 + lx, P.nx);
#pragma unroll
            for (int m = 0; m < M; ++m) v[it][m] = fl[m][n];
        }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int k = tid + 256 * it;
        if (k < K3F) {
#pragma unroll
            for (int m = 0; m < M; ++m) st[m * K3F + k] = v[it][m];
        }
    }
}
// Eq. 33 gradient of a staged field at tile position sc
template <class R>
__device__ __forceinline__ void grad3_tile(const R* __restrict__ t, int sc, R g[3]) {
    R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
    for (int j = 0; j < Q3; ++j) {
        const R v = w3<R>(j) * t[sc + c3z(j) * K3P + c3y(j) * K3X + c3x(j)];
        cacc(a0, c3x(j), v);
        cacc(a1, c3y(j), v);
        cacc(a2, c3z(j), v);
    }
    g[0] = ocs2(a0); g[1] = ocs2(a1); g[2] = ocs2(a2);
}
// The stencil neighbours of a cell in 32-bit indices (at most LB3E_MAX_CELLS cells):
// the columns, rows and planes of the offsets -1, 0, +1 formed once a cell; x and y
// periodic, z periodic or mirrored at the walls (the stencil ghosts)
struct Nb3 {
    unsigned col[3], row[3], pln[3];
    __device__ __forceinline__ unsigned at(int j) const { return pln[c3z(j) + 1] + row[c3y(j) + 1] + col[c3x(j) + 1]; }
};
__device__ __forceinline__ Nb3 stencil3(const P3& P, int x, int y, int z) {
    Nb3 s;
    const unsigned nx = (unsigned)P.nx, ny = (unsigned)P.ny, nz = (unsigned)P.nz, nxy = nx * ny;
    const unsigned ux = (unsigned)x, uy = (unsigned)y, uz = (unsigned)z;
    s.col[0] = x == 0 ? nx - 1 : ux - 1;
    s.col[1] = ux;
    s.col[2] = ux + 1 == nx ? 0u : ux + 1;
    s.row[0] = (y == 0 ? ny - 1 : uy - 1) * nx;
    s.row[1] = uy * nx;
    s.row[2] = (uy + 1 == ny ? 0u : uy + 1) * nx;
    s.pln[0] = (z == 0 ? (P.bc ? 0u : nz - 1) : uz - 1) * nxy;
    s.pln[1] = uz * nxy;
    s.pln[2] = (uz + 1 == nz ? (P.bc ? nz - 1 : 0u) : uz + 1) * nxy;
    return s;
}
// Eq. 33 gradient of a field at a cell, its neighbours read through L1 (the closure
// has two fields: too little work a block to repay staging them behind a barrier)
template <class R>
__device__ __forceinline__ void grad3(const Nb3& nb, const R* __restrict__ f, R g[3]) {
    R a0 = R(0), a1 = R(0), a2 = R(0);
#pragma unroll
    for (int j = 0; j < Q3; ++j) {
        const R v = w3<R>(j) * f[nb.at(j)];
        cacc(a0, c3x(j), v);
        cacc(a1, c3y(j), v);
        cacc(a2, c3z(j), v);
    }
    g[0] = ocs2(a0); g[1] = ocs2(a1); g[2] = ocs2(a2);
}
// Eq. 33 Laplacian of a staged field at tile position sc
template <class R>
__device__ __forceinline__ R lap3_tile(const R* __restrict__ t, int sc) {
    const R c0 = t[sc];
    R a = R(0);
#pragma unroll
    for (int j = 0; j < Q3; ++j) a += R(2) * w3<R>(j) * (t[sc + c3z(j) * K3P + c3y(j) * K3X + c3x(j)] - c0);
    return ocs2(a);
}

template <class R>
__device__ __forceinline__ R s3(int j, R u0, R u1, R u2) {   // s_j(u), Eq. 40
    const R cu = cdot3<R>(j, u0, u1, u2);
    const R uu = u0 * u0 + u1 * u1 + u2 * u2;
    const R c2 = R(1) / R(3);
    if constexpr (exact_arith<R>()) return w3<R>(j) * (cu / c2 + cu * cu / (R(2) * c2 * c2) - uu / (R(2) * c2));
    else return w3<R>(j) * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
}

// ---------------------------------------------------------------- S1, S2
// phi_i, q~ of the current populations; rho, sigma, eps of those phi
template <class R>
__global__ void __launch_bounds__(256) k3_moments(P3 P, const R* __restrict__ pop, R* __restrict__ phi,
                                                  R* __restrict__ qt, R* __restrict__ rho, R* __restrict__ sig,
                                                  R* __restrict__ eps) {
    int x, y, z;
    size_t c;
    if (!cell3(P, x, y, z, c)) return;
    const size_t N = P.N;
    R ph[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R a = R(0);
#pragma unroll
        for (int j = 0; j < Q3; ++j) a += pop[(Q3 * (i + 1) + j) * N + c];
        ph[i] = a;
        phi[i * N + c] = a;
    }
    R a = R(0);
#pragma unroll
    for (int j = 0; j < Q3; ++j) a += pop[(Q3 * 4 + j) * N + c];
    qt[c] = a;
    rho[c] = ph[0] * pv<R>(P.rho[0], P.frho[0]) + ph[1] * pv<R>(P.rho[1], P.frho[1]) + ph[2] * pv<R>(P.rho[2], P.frho[2]);   // Eq. 29
    sig[c] = ph[0] * pv<R>(P.sigma[0], P.fsig[0]) + ph[1] * pv<R>(P.sigma[1], P.fsig[1]) + ph[2] * pv<R>(P.sigma[2], P.fsig[2]);
    R e = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) e += pv<R>(P.eps[i], P.feps[i]) * ph[i] * ph[i] * (R(3) - R(2) * ph[i]);   // Eq. 30
    eps[c] = e;
}
// properties only (initial state)
template <class R>
__global__ void __launch_bounds__(256) k3_props(P3 P, const R* __restrict__ phi, R* __restrict__ rho,
                                                R* __restrict__ sig, R* __restrict__ eps) {
    int x, y, z;
    size_t c;
    if (!cell3(P, x, y, z, c)) return;
    const size_t N = P.N;
    const R ph[3] = {phi[c], phi[N + c], phi[2 * N + c]};
    rho[c] = ph[0] * pv<R>(P.rho[0], P.frho[0]) + ph[1] * pv<R>(P.rho[1], P.frho[1]) + ph[2] * pv<R>(P.rho[2], P.frho[2]);
    sig[c] = ph[0] * pv<R>(P.sigma[0], P.fsig[0]) + ph[1] * pv<R>(P.sigma[1], P.fsig[1]) + ph[2] * pv<R>(P.sigma[2], P.fsig[2]);
    R e = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) e += pv<R>(P.eps[i], P.feps[i]) * ph[i] * ph[i] * (R(3) - R(2) * ph[i]);
    eps[c] = e;
}

// ---------------------------------------------------------------- S4
// q = (q~ + (r grad eps . E - grad sigma . E)/2) / (1 + r/2), r = sigma/eps, with the
// previous step's field
template <class R>
__global__ void __launch_bounds__(256) k3_closure(P3 P, const R* __restrict__ qt, const R* __restrict__ sig,
                                                  const R* __restrict__ eps, const R* __restrict__ E,
                                                  R* __restrict__ q) {
    int x, y, z;
    size_t cz;
    if (!cell3(P, x, y, z, cz)) return;
    const unsigned N = (unsigned)P.N, c = (unsigned)cz;
    const Nb3 nb = stencil3(P, x, y, z);
    R ge3[3], gs3[3];
    grad3<R>(nb, eps, ge3);
    grad3<R>(nb, sig, gs3);
    const R r = sig[c] / eps[c];
    R ge = R(0), gs = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ge += ge3[a] * E[a * N + c];
        gs += gs3[a] * E[a * N + c];
    }
    q[c] = (qt[c] + R(0.5) * (r * ge - gs)) / (R(1) + R(0.5) * r);
}

// ---------------------------------------------------------------- S5: Eq. 43-45
template <class R>
__device__ __forceinline__ void hmoments3(const R* __restrict__ h, size_t N, size_t c, R& psi, R J[3]) {
    R a = R(0);
#pragma unroll
    for (int j = 1; j < Q3; ++j) a += h[j * N + c];
    psi = a / (R(1) - w3<R>(0));
    R j0 = R(0), j1 = R(0), j2 = R(0);
#pragma unroll
    for (int j = 0; j < Q3; ++j) {
        const R v = h[j * N + c];
        cacc(j0, c3x(j), v);
        cacc(j1, c3y(j), v);
        cacc(j2, c3z(j), v);
    }
    J[0] = j0; J[1] = j1; J[2] = j2;
}

// psi and J of a cell's potential populations (Eq. 45)
template <class R>
__device__ __forceinline__ void pot3_moments(const R (&hv)[Q3], R& psi, R J[3]) {
    R a = R(0);
#pragma unroll
    for (int j = 1; j < Q3; ++j) a += hv[j];
    psi = a / (R(1) - w3<R>(0));
    J[0] = J[1] = J[2] = R(0);
#pragma unroll
    for (int j = 0; j < Q3; ++j) {
        cacc(J[0], c3x(j), hv[j]);
        cacc(J[1], c3y(j), hv[j]);
        cacc(J[2], c3z(j), hv[j]);
    }
}
// Collision of a cell's potential populations (Eq. 43, equilibrium Eq. 44) and
// push-streaming to its neighbours: columns, rows and planes formed once, 32-bit
// indices (at most LB3E_MAX_CELLS cells, so 15 N fits); across a z wall the
// population returns to this cell (electrodes: the Dirichlet rule)
template <class R>
__device__ __forceinline__ void pot3_collide_push(const P3& P, const R (&hv)[Q3], R psi, const R J[3], R epsc, R qc,
                                                  int x, int y, int z, unsigned c, unsigned N, R* __restrict__ hout) {
    // divisions: exact in the FP64 build, by a reciprocal formed once in FP32
    const R th = pv<R>(P.tau_h, P.ftau_h), ith = pv<R>(1.0 / P.tau_h, P.fitau_h),
            epshat = epsc - pv<R>(P.eps_ref, P.feps_ref);
    const R den = epshat + (R(1) / R(3)) * th, iden = rcp(den);
    const R g0 = dv(-J[0], den, iden), g1 = dv(-J[1], den, iden), g2 = dv(-J[2], den, iden);
    const R e3 = ocs2(epshat);
    const unsigned nx = (unsigned)P.nx, ny = (unsigned)P.ny, nz = (unsigned)P.nz, nxy = nx * ny;
    const unsigned col[3] = {x == 0 ? nx - 1 : (unsigned)x - 1, (unsigned)x, x == P.nx - 1 ? 0u : (unsigned)x + 1};
    const unsigned row[3] = {(y == 0 ? ny - 1 : (unsigned)y - 1) * nx, (unsigned)y * nx,
                             (y == P.ny - 1 ? 0u : (unsigned)y + 1) * nx};
    const unsigned pln[3] = {(z == 0 ? nz - 1 : (unsigned)z - 1) * nxy, (unsigned)z * nxy,
                             (z == P.nz - 1 ? 0u : (unsigned)z + 1) * nxy};
    const bool wall_lo = P.bc != 0 && z == 0, wall_hi = P.bc != 0 && z == P.nz - 1;
#pragma unroll
    for (int j = 0; j < Q3; ++j) {
        const R heq = j == 0 ? (w3<R>(0) - R(1)) * psi : w3<R>(j) * psi;     // Eq. 44
        const R varpi = j == 0 ? R(0) : R(1.0 / 14.0);
        const R hj = hv[j];
        const R cg = cdot3<R>(j, g0, g1, g2);
        const R v = hj - dv(hj - heq, th, ith) - dv(e3 * w3<R>(j) * cg, th, ith) + varpi * qc;
        if ((c3z(j) < 0 && wall_lo) || (c3z(j) > 0 && wall_hi)) {  // across a z wall: back to this cell
            R out = v;
            if (P.bc == 2) out = -v + R(2) * w3<R>(j) * pv<R>(c3z(j) > 0 ? P.V_top : P.V_bottom, c3z(j) > 0 ? P.fVt : P.fVb);
            hout[opp3(j) * N + c] = out;
        } else {
            hout[j * N + pln[c3z(j) + 1] + row[c3y(j) + 1] + col[c3x(j) + 1]] = v;
        }
    }
}

// One pseudo-iteration: collide and push-stream h.  save: store psi, J (the state
// a later check compares with); check: accumulate |d psi|^2, |psi|^2, |dJ|^2, |J|^2
// per block (FP64 partials).  FP32: held to 64 registers (four blocks an SM); the
// scheduler otherwise keeps all 15 populations live across the moments (79
// registers, three blocks an SM, measured 10% slower).
template <class R>
__global__ void __launch_bounds__(256, std::is_same<R, float>::value ? 4 : 1)
    k3_poisson(P3 P, const R* __restrict__ hin, R* __restrict__ hout, const R* __restrict__ eps,
               const R* __restrict__ q, R* __restrict__ prev, double* __restrict__ partial, int save, int check) {
    int x, y, z;
    size_t cz;
    const bool in = cell3(P, x, y, z, cz);
    const unsigned N = (unsigned)P.N, c = (unsigned)cz;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (in) {
        R hv[Q3];
#pragma unroll
        for (int j = 0; j < Q3; ++j) hv[j] = hin[j * N + c];
        R psi, J[3];
        pot3_moments(hv, psi, J);
        if (check) {
            const double d = (double)psi - (double)prev[c];
            acc[0] = d * d;
            acc[1] = (double)psi * (double)psi;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double e = (double)J[k] - (double)prev[(1 + k) * N + c];
                acc[2] += e * e;
                acc[3] += (double)J[k] * (double)J[k];
            }
        }
        if (save) {
            prev[c] = psi;
#pragma unroll
            for (int k = 0; k < 3; ++k) prev[(1 + k) * N + c] = J[k];
        }
        pot3_collide_push(P, hv, psi, J, eps[c], q[c], x, y, z, c, N, hout);
    }
    if (check) {
        const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        block_reduce_store<4>(acc, partial + 4 * (size_t)b);
    }
}

// The same iteration (no check, no save) with its inputs staged by the tensor memory
// accelerator: a block walks up to `walk` consecutive planes of its 32 x 8 tile, and
// one thread copies each plane's 15 population boxes, eps and q (17 boxes of 32 x 8
// cells) into one of P3ST shared-memory stages, so that the loads of the next
// planes are in flight while a plane is collided.  Boxes beyond the lattice arrive
// as zeros and are not used.  A wait that runs out sets the error flag; the block
// then waits, bounded, for its copies still in flight and returns.
constexpr int P3ST = 3, P3BOX = 17;
template <class R>
constexpr size_t k3_poisson_tma_smem() { return (size_t)P3ST * P3BOX * 256 * sizeof(R); }
template <class R>
__global__ void __launch_bounds__(256, 4)
    k3_poisson_tma(P3 P, const __grid_constant__ CUtensorMap tm_h, const __grid_constant__ CUtensorMap tm_eps,
                   const __grid_constant__ CUtensorMap tm_q, R* __restrict__ hout, int walk, int* err) {
    extern __shared__ __align__(128) unsigned char p3_raw[];
    R* st = reinterpret_cast<R*>(p3_raw);  // [stage][17 boxes][8 rows][32]
    __shared__ __align__(8) uint64_t bar[P3ST];
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8, z0 = blockIdx.z * walk;
    const int nzb = P.nz - z0 < walk ? P.nz - z0 : walk;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const unsigned N = (unsigned)P.N;
    auto issue = [&](int i) {  // plane z0 + i into stage i % P3ST (one thread)
        R* d = st + (size_t)(i % P3ST) * P3BOX * 256;
        uint64_t* b = &bar[i % P3ST];
        mbar_arrive_expect_tx(b, P3BOX * 256 * (unsigned)sizeof(R));
#pragma unroll 1
        for (int j = 0; j < Q3; ++j) tma_load_3d(d + j * 256, &tm_h, x0, y0, j * P.nz + z0 + i, b);
        tma_load_3d(d + 15 * 256, &tm_eps, x0, y0, z0 + i, b);
        tma_load_3d(d + 16 * 256, &tm_q, x0, y0, z0 + i, b);
    };
    if (tid == 0) {
        for (int s = 0; s < P3ST; ++s) mbar_init(&bar[s], 1);
        for (int i = 0; i < P3ST && i < nzb; ++i) issue(i);
    }
    __syncthreads();
    int i = 0;
    for (; i < nzb; ++i) {
        const int s = i % P3ST;
        const bool ok = mbar_wait(&bar[s], (unsigned)((i / P3ST) & 1), TMA_WAIT_LIMIT);
        if (ok && x < P.nx && y < P.ny) {
            const R* d = st + (size_t)s * P3BOX * 256 + tid;
            R hv[Q3];
#pragma unroll
            for (int j = 0; j < Q3; ++j) hv[j] = d[j * 256];
            R psi, J[3];
            pot3_moments(hv, psi, J);
            const int z = z0 + i;
            const unsigned c = ((unsigned)z * (unsigned)P.ny + (unsigned)y) * (unsigned)P.nx + (unsigned)x;
            pot3_collide_push(P, hv, psi, J, d[15 * 256], d[16 * 256], x, y, z, c, N, hout);
        }
        // stage s read by every thread; a failed wait anywhere seen by all
        if (__syncthreads_or(ok ? 0 : 1)) break;
        if (tid == 0 && i + P3ST < nzb) issue(i + P3ST);
    }
    if (i < nzb && tid == 0) {  // gave up: let the copies in flight land first
        const int e = i + P3ST < nzb ? i + P3ST : nzb;
        for (int k = i; k < e; ++k) mbar_wait(&bar[k % P3ST], (unsigned)((k / P3ST) & 1), TMA_WAIT_LIMIT);
        if (err) atomicExch(err, 1);
    }
}

// psi and E = -grad psi (+ the external field) from the potential populations (Eq. 45)
template <class R>
__global__ void __launch_bounds__(256) k3_fields(P3 P, const R* __restrict__ h, const R* __restrict__ eps,
                                                 R* __restrict__ E, R* __restrict__ psi_out) {
    int x, y, z;
    size_t c;
    if (!cell3(P, x, y, z, c)) return;
    const size_t N = P.N;
    R psi, J[3];
    hmoments3<R>(h, N, c, psi, J);
    const R den = (eps[c] - pv<R>(P.eps_ref, P.feps_ref)) + (R(1) / R(3)) * pv<R>(P.tau_h, P.ftau_h);
    E[c] = -(-J[0] / den) + pv<R>(P.E0, P.fE0);
    E[N + c] = -(-J[1] / den);
    E[2 * N + c] = -(-J[2] / den) + pv<R>(P.E1, P.fE1);
    if (psi_out) psi_out[c] = psi;
}
template <class R>
__global__ void k3_fill_E(P3 P, R* __restrict__ E) {
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= P.N) return;
    E[c] = pv<R>(P.E0, P.fE0);
    E[P.N + c] = R(0);
    E[2 * P.N + c] = pv<R>(P.E1, P.fE1);
}
// potential populations at equilibrium with the linear electrode profile
template <class R>
__global__ void __launch_bounds__(256) k3_init_h(P3 P, R* __restrict__ h) {
    int x, y, z;
    size_t c;
    if (!cell3(P, x, y, z, c)) return;
    const R psi0 = P.bc == 2 ? R(P.V_bottom + (P.V_top - P.V_bottom) * (z + 0.5) / P.nz) : R(0);
#pragma unroll
    for (int j = 0; j < Q3; ++j) h[j * P.N + c] = j == 0 ? (w3<R>(0) - R(1)) * psi0 : w3<R>(j) * psi0;
}

// ---------------------------------------------------------------- S6: Eq. 20
template <class R>
__global__ void __launch_bounds__(256) k3_chem(P3 P, const R* __restrict__ phi, const R* __restrict__ E,
                                               R* __restrict__ mu) {
    __shared__ R st[3 * K3F];  // phi_1..3 on the staged three-plane tile
    const R* const fl[3] = {phi, phi + P.N, phi + 2 * P.N};
    stage_tile3<R, 3>(P, fl, st);
    __syncthreads();
    int x, y, z;
    size_t cz;
    if (!cell3(P, x, y, z, cz)) return;
    const unsigned N = (unsigned)P.N, c = (unsigned)cz;
    const int sc = K3P + (threadIdx.y + 1) * K3X + threadIdx.x + 1;
    const R e2 = E[c] * E[c] + E[N + c] * E[N + c] + E[2 * N + c] * E[2 * N + c];
    const R D = pv<R>(P.D, P.fD);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const R ph = st[i * K3F + sc], lam = pv<R>(P.lam[i], P.flam[i]);
        const R lap = lap3_tile<R>(st + i * K3F, sc);
        const R bulk = R(24) / D * lam * ph * (ph - R(0.5)) * (ph - R(1));
        const R grad = R(0.75) * D * lam * lap;
        const R deps = R(6) * pv<R>(P.eps[i], P.feps[i]) * ph * (R(1) - ph);
        mu[i * N + c] = bulk - grad - R(0.5) * deps * e2;
    }
}

// ---------------------------------------------------------------- S7-S14
// Force, flow moments, d/dt terms, collision of the phase (Eq. 34-36), flow (Eq.
// 37-40) and charge (Eq. 46-50) populations, push-streaming with bounce-back at the
// z walls (moving walls along x for the flow set).
//
// The six stencilled fields (mu_1..3, eps, sigma, rho) of the block's 32 x 8 tile,
// with a one-cell halo, on the planes z - 1, z, z + 1 (periodic or mirrored at the
// walls, as the stencil ghosts), are staged in shared memory first: each thread
// then forms the six gradients from shared memory, in the neighbour order of
// grad3_tile (the same sums), instead of 90 global loads with their index
// arithmetic.  Blocks of consecutive planes run close together in time, so the
// neighbour planes come from L2.
// Shared memory: the six staged stencil fields, then the cell's 75 populations and
// 12 d/dt history planes, requested as cp.async copies at entry so that all of them
// are in flight together (the kernel was bound by the latency of these loads).
constexpr int K3T = 256;  // cells (threads) a block
template <class R>
constexpr size_t k3_collide_smem() { return (size_t)(6 * K3F + (5 * Q3 + 12) * K3T) * sizeof(R); }
// blocks per SM: FP32 two (its shared memory), so up to 128 registers a thread;
// FP64 one
template <class R>
constexpr int k3_collide_min_blocks() { return std::is_same<R, float>::value ? 2 : 1; }
template <class R>
__global__ void __launch_bounds__(256, k3_collide_min_blocks<R>()) k3_collide(P3 P, const R* __restrict__ pin, R* __restrict__ pout,
                                                  const R* __restrict__ phi, const R* __restrict__ q,
                                                  const R* __restrict__ E, const R* __restrict__ mu,
                                                  const R* __restrict__ rho_f, const R* __restrict__ sig_f,
                                                  const R* __restrict__ eps_f, R* __restrict__ prev,
                                                  R* __restrict__ diag, int first, int write_diag) {
    extern __shared__ __align__(16) unsigned char k3_raw[];
    R* st = reinterpret_cast<R*>(k3_raw);  // [6 fields][3 planes][10][34]
    R* sp = st + 6 * K3F;                  // [75 population planes][256 cells], then [12 history planes][256]
    const size_t N = P.N;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    {
        // this cell's populations and history: 4- or 8-byte copies (one per plane), or
        // 16-byte copies of row segments when the tile's rows are whole and aligned
        const int xa = blockIdx.x * 32, ya = blockIdx.y * 8, za = blockIdx.z;
        constexpr int V = 16 / (int)sizeof(R), SEG = 32 / V;  // cells per 16 bytes, segments per row
        const bool whole = xa + 32 <= P.nx && ya + 8 <= P.ny && (P.nx % V) == 0 && (N % V) == 0;
        auto plane = [&](int k) -> const R* { return k < 5 * Q3 ? pin + (size_t)k * N : prev + (size_t)(k - 5 * Q3) * N; };
        if (whole) {
            for (int t = tid; t < (5 * Q3 + 12) * 8 * SEG; t += K3T) {
                const int k = t / (8 * SEG), r = (t / SEG) % 8, m = t % SEG;
                const size_t g = ((size_t)za * P.ny + ya + r) * P.nx + xa + m * V;
                cp_async16(sp + k * K3T + r * 32 + m * V, plane(k) + g);
            }
        } else if (xa + (int)threadIdx.x < P.nx && ya + (int)threadIdx.y < P.ny) {
            const size_t g = ((size_t)za * P.ny + ya + threadIdx.y) * P.nx + xa + threadIdx.x;
            for (int k = 0; k < 5 * Q3 + 12; ++k) cp_async(sp + k * K3T + tid, plane(k) + g);
        }
        cp_async_commit();
    }
    {
        const R* const fl[6] = {mu, mu + N, mu + 2 * N, eps_f, sig_f, rho_f};
        stage_tile3<R, 6>(P, fl, st);
    }
    cp_async_wait_all();  // the copies are published by the barrier
    __syncthreads();
    int x, y, z;
    size_t c;
    if (!cell3(P, x, y, z, c)) return;
    const R c2 = R(1) / R(3);
    R ph[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ph[i] = phi[i * N + c];
    const int sc = K3P + (threadIdx.y + 1) * K3X + threadIdx.x + 1;  // this cell in the staged tile
    const R qc = q[c], rho = st[5 * K3F + sc], irho = rcp(rho);
    const R Ev[3] = {E[c], E[N + c], E[2 * N + c]};
    // S7, S8: grad mu_i (and, in the same neighbour pass, grad eps, grad sigma,
    // grad rho), F = -sum phi_i grad mu_i + q E
    R gg[6][3];
    {
        R a[6][3];
#pragma unroll
        for (int m = 0; m < 6; ++m) a[m][0] = a[m][1] = a[m][2] = R(0);
#pragma unroll
        for (int j = 0; j < Q3; ++j) {
            const int sn = sc + c3z(j) * K3P + c3y(j) * K3X + c3x(j);
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const R v = w3<R>(j) * st[m * K3F + sn];
                cacc(a[m][0], c3x(j), v);
                cacc(a[m][1], c3y(j), v);
                cacc(a[m][2], c3z(j), v);
            }
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            gg[m][0] = ocs2(a[m][0]);
            gg[m][1] = ocs2(a[m][1]);
            gg[m][2] = ocs2(a[m][2]);
        }
    }
    R (&gmu)[6][3] = gg;
    R F[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R Fa = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) Fa -= ph[i] * gmu[i][a];
        F[a] = Fa + qc * Ev[a];
    }
    // R^n of Eq. 47
    const R* ge3 = gg[3];
    const R* gs3 = gg[4];
    const R* gr = gg[5];
    R Rc;
    {
        const R r = st[4 * K3F + sc] / st[3 * K3F + sc];
        R ge = R(0), gs = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ge += ge3[a] * Ev[a];
            gs += gs3[a] * Ev[a];
        }
        Rc = -r * qc + r * ge - gs;
    }
    // S9: Eq. 41
    R g[Q3];
#pragma unroll
    for (int j = 0; j < Q3; ++j) g[j] = sp[j * K3T + tid];
    R u[3], p;
    {
        R m0 = R(0), m1 = R(0), m2 = R(0), g1 = R(0);
#pragma unroll
        for (int j = 0; j < Q3; ++j) {
            cacc(m0, c3x(j), g[j]);
            cacc(m1, c3y(j), g[j]);
            cacc(m2, c3z(j), g[j]);
            if (j) g1 += g[j];
        }
        u[0] = dv(m0 + R(0.5) * F[0], rho, irho);
        u[1] = dv(m1 + R(0.5) * F[1], rho, irho);
        u[2] = dv(m2 + R(0.5) * F[2], rho, irho);
        const R ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
        p = c2 / (R(1) - w3<R>(0)) * (g1 + R(0.5) * ugr + rho * s3<R>(0, u[0], u[1], u[2]));
    }
    // S10
    R dpu[3][3], dqu[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) dpu[i][a] = first ? R(0) : ph[i] * u[a] - sp[(5 * Q3 + 3 * i + a) * K3T + tid];
#pragma unroll
    for (int a = 0; a < 3; ++a) dqu[a] = first ? R(0) : qc * u[a] - sp[(5 * Q3 + 9 + a) * K3T + tid];

    // streaming targets, the same for the five sets: the neighbour's index within a
    // plane (from its column, row and plane formed once, 32-bit: at most
    // LB3E_MAX_CELLS cells, so 75 N fits), or this cell (bit j of wall set) when link j
    // leaves through a z wall
    unsigned tgt[Q3];
    unsigned wall = 0u;
    {
        const unsigned nx = (unsigned)P.nx, ny = (unsigned)P.ny, nz = (unsigned)P.nz, nxy = nx * ny;
        const unsigned col[3] = {x == 0 ? nx - 1 : (unsigned)x - 1, (unsigned)x,
                                 x == P.nx - 1 ? 0u : (unsigned)x + 1};
        const unsigned row[3] = {(y == 0 ? ny - 1 : (unsigned)y - 1) * nx, (unsigned)y * nx,
                                 (y == P.ny - 1 ? 0u : (unsigned)y + 1) * nx};
        const unsigned pln[3] = {(z == 0 ? nz - 1 : (unsigned)z - 1) * nxy, (unsigned)z * nxy,
                                 (z == P.nz - 1 ? 0u : (unsigned)z + 1) * nxy};
        const bool wall_lo = P.bc != 0 && z == 0, wall_hi = P.bc != 0 && z == P.nz - 1;
#pragma unroll
        for (int j = 0; j < Q3; ++j) {
            if ((c3z(j) < 0 && wall_lo) || (c3z(j) > 0 && wall_hi)) {
                tgt[j] = (unsigned)c;
                wall |= 1u << j;
            } else {
                tgt[j] = pln[c3z(j) + 1] + row[c3y(j) + 1] + col[c3x(j) + 1];
            }
        }
    }
    // post-collision value v of population j of `set`: to the neighbour, or back to
    // this cell in the opposite direction at a wall
    const unsigned N32 = (unsigned)N;
    auto push = [&](int set, int j, R v) {
        const int jj = ((wall >> j) & 1u) ? opp3(j) : j;
        pout[(unsigned)(Q3 * set + jj) * N32 + tgt[j]] = v;
    };

    // S11: phase populations with the mobility of Eq. 28
    const R tf = pv<R>(P.tau_f, P.ftau_f), itf = pv<R>(1.0 / P.tau_f, P.fitau_f), m0 = pv<R>(P.m0, P.fm0), im0 = pv<R>(1.0 / P.m0, P.fim0);
    const R pf = R(1) - R(1) / (R(2) * tf);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R Mii = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (k != i) Mii += m0 * ph[i] * ph[k];
        R Y[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const R Mik = (k == i) ? (Mii - m0) : -m0 * ph[i] * ph[k];
#pragma unroll
            for (int a = 0; a < 3; ++a) Y[a] += Mik * gmu[k][a];
        }
        R A[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) A[a] = ocs2(dpu[i][a]) - dv(Y[a], m0, im0);
        const R mui = st[i * K3F + sc];
        const R pu0 = ph[i] * u[0], pu1 = ph[i] * u[1], pu2 = ph[i] * u[2];
#pragma unroll
        for (int j = 0; j < Q3; ++j) {
            const R feq = (j == 0) ? ph[i] - (R(1) - w3<R>(0)) * mui
                                   : w3<R>(j) * mui + ocs2(w3<R>(j) * cdot3<R>(j, pu0, pu1, pu2));
            const R Fj = w3<R>(j) * cdot3<R>(j, A[0], A[1], A[2]);
            const R fj = sp[(Q3 * (i + 1) + j) * K3T + tid];
            push(i + 1, j, fj - dv(fj - feq, tf, itf) + pf * Fj);
        }
    }
    // S12: flow populations
    {
        R tg = pv<R>(P.tau_g, P.ftau_g);
        if (P.use_visc) {
            R eta = R(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) eta += ph[i] * pv<R>(P.visc[i], P.fvisc[i]);
            tg = R(0.5) + dv(eta, rho * c2, irho * R(3));
        }
        const R itg = rcp(tg), pg = R(1) - R(1) / (R(2) * tg);
        const R ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
#pragma unroll
        for (int j = 0; j < Q3; ++j) {
            const R geq = (j == 0) ? ocs2((w3<R>(0) - R(1)) * p) + rho * s3<R>(0, u[0], u[1], u[2])
                                   : ocs2(w3<R>(j) * p) + rho * s3<R>(j, u[0], u[1], u[2]);
            const R cu = cdot3<R>(j, u[0], u[1], u[2]);
            const R cgr = cdot3<R>(j, gr[0], gr[1], gr[2]);
            const R cF = cdot3<R>(j, F[0], F[1], F[2]);
            const R G = w3<R>(j) * (ugr + ocs2(cF) + ocs2(cu * cgr - c2 * ugr));
            const R v = g[j] - dv(g[j] - geq, tg, itg) + pg * G;
            if ((wall >> j) & 1u) {
                const R uw = pv<R>(c3z(j) > 0 ? P.uwt : P.uwb, c3z(j) > 0 ? P.fuwt : P.fuwb);
                push(0, j, v - ocs2(R(2) * w3<R>(j) * rho * (R(c3x(j)) * uw)));
            } else {
                push(0, j, v);
            }
        }
    }
    // S13: charge populations
    {
        const R tl = pv<R>(P.tau_l, P.ftau_l), itl = pv<R>(1.0 / P.tau_l, P.fitau_l), pl = R(1) - R(1) / (R(2) * tl);
#pragma unroll
        for (int j = 0; j < Q3; ++j) {
            const R cu = cdot3<R>(j, u[0], u[1], u[2]);
            const R leq = P.cc ? w3<R>(j) * qc * (R(1) + ocs2(cu)) : w3<R>(j) * qc;
            const R Sj = pl * w3<R>(j) * Rc;
            const R Tj = P.cc ? ocs2(pl * w3<R>(j) * cdot3<R>(j, dqu[0], dqu[1], dqu[2])) : R(0);
            const R lj = sp[(Q3 * 4 + j) * K3T + tid];
            push(4, j, lj - dv(lj - leq, tl, itl) + Sj + Tj);
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int a = 0; a < 3; ++a) prev[(3 * i + a) * N + c] = ph[i] * u[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) prev[(9 + a) * N + c] = qc * u[a];
    if (write_diag) {
#pragma unroll
        for (int a = 0; a < 3; ++a) diag[a * N + c] = u[a];
        diag[3 * N + c] = p;
    }
}

// initial populations: phases at equilibrium with mu (Eq. 20), flow at g_eq(p = 0, u),
// charge at l_eq(q, u)
template <class R>
__global__ void __launch_bounds__(256) k3_init_pops(P3 P, R* __restrict__ pop, const R* __restrict__ phi,
                                                    const R* __restrict__ q, const R* __restrict__ uin,
                                                    const R* __restrict__ mu, const R* __restrict__ rho_f) {
    int x, y, z;
    size_t c;
    if (!cell3(P, x, y, z, c)) return;
    const size_t N = P.N;
    const R c2 = R(1) / R(3);
    const R u0 = uin[c], u1 = uin[N + c], u2 = uin[2 * N + c];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const R ph = phi[i * N + c], mui = mu[i * N + c];
        const R pu0 = ph * u0, pu1 = ph * u1, pu2 = ph * u2;
#pragma unroll
        for (int j = 0; j < Q3; ++j)
            pop[(Q3 * (i + 1) + j) * N + c] = (j == 0) ? ph - (R(1) - w3<R>(0)) * mui
                                                       : w3<R>(j) * mui + w3<R>(j) * cdot3<R>(j, pu0, pu1, pu2) / c2;
    }
    const R rho = rho_f[c], qc = q[c];
#pragma unroll
    for (int j = 0; j < Q3; ++j) {
        pop[j * N + c] = rho * s3<R>(j, u0, u1, u2);
        const R cu = cdot3<R>(j, u0, u1, u2);
        pop[(Q3 * 4 + j) * N + c] = P.cc ? w3<R>(j) * qc * (R(1) + cu / c2) : w3<R>(j) * qc;
    }
}

// observables: per-block FP64 sums of mass (3), charge, nonfinite count and the
// second moments of the two indicators (x and z), plus a block max of |sum phi - 1|
constexpr int NOBS3 = 15;
// OBS3_Z planes a thread: a block of 32 x 8 threads covers 32 x 8 x OBS3_Z cells, so
// the FP64 block reduction is shared by OBS3_Z cells a thread and the final
// single-block reduction sees nz / OBS3_Z times fewer partials.  The per-cell terms
// are evaluated in FP32 in the FP32 build and summed as FP32 sum-and-error pairs
// (ObsAcc), FP64 otherwise.
constexpr int OBS3_Z = 16;
inline dim3 obs3_grid(const lb3e_params& p) { return dim3((p.nx + 31) / 32, (p.ny + 7) / 8, (p.nz + OBS3_Z - 1) / OBS3_Z); }
template <class R>
__global__ void __launch_bounds__(256) k3_observables(P3 P, const R* __restrict__ phi, const R* __restrict__ q,
                                                      const R* __restrict__ u, double* __restrict__ partial,
                                                      double* __restrict__ maxpart) {
    using T = typename std::conditional<std::is_same<R, float>::value, float, double>::type;
    ObsAcc<T, NOBS3> acc;
    T mdev = T(0);
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x < P.nx && y < P.ny) {
        const unsigned N = (unsigned)P.N;
        const int z1 = (int)(blockIdx.z + 1) * OBS3_Z < P.nz ? (int)(blockIdx.z + 1) * OBS3_Z : P.nz;
        for (int z = blockIdx.z * OBS3_Z; z < z1; ++z) {
            const unsigned c = ((unsigned)z * (unsigned)P.ny + (unsigned)y) * (unsigned)P.nx + (unsigned)x;
            T ph[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ph[i] = (T)phi[i * N + c];
                acc.add(i, ph[i]);
            }
            const T qc = (T)q[c];
            acc.add(3, qc);
            const T vals[7] = {ph[0], ph[1], ph[2], (T)u[c], (T)u[N + c], (T)u[2 * N + c], qc};
#pragma unroll
            for (int k = 0; k < 7; ++k)
                if (!isfinite(vals[k])) acc.add(4, T(1));
            const T chis[2] = {ph[P.inner - 1], T(1) - ph[P.matrix - 1]};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                acc.add(5 + 5 * k, chis[k]);
                acc.add(6 + 5 * k, chis[k] * T(x));
                acc.add(7 + 5 * k, chis[k] * T(z));
                acc.add(8 + 5 * k, chis[k] * T(x) * T(x));
                acc.add(9 + 5 * k, chis[k] * T(z) * T(z));
            }
            const T dv = sum_dev3(ph[0], ph[1], ph[2]);
            mdev = dv > mdev ? dv : mdev;  // as fmax: a NaN is left to the nonfinite count
        }
    }
    const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    double v[NOBS3];
    acc.out(v);
    block_reduce_store<NOBS3>(v, partial + (size_t)NOBS3 * b);
    // block max of the deviation
    __shared__ double red[8];
    double m = (double)mdev;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a = fmax(a, red[k]);
        maxpart[b] = a;
    }
}

template <class R>
__global__ void k3_pop_to_f64(double* __restrict__ dst, const R* __restrict__ src, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// ---------------------------------------------------------------- host sequencing
template <class R>
class Sim3 final : public SimBase {
  public:
    struct Layout {
        size_t pop[2], h[2], phi, qt, q, rho, sig, eps, E, mu, prev, diag, psi_prev, partial, result, stage, total;
    };
    static size_t nblocks(const lb3e_params& p) { return (size_t)((p.nx + 31) / 32) * ((p.ny + 7) / 8) * p.nz; }
    static Layout layout(const lb3e_params& p) {
        const size_t N = (size_t)p.nx * p.ny * p.nz;
        Layout L{};
        size_t o = 0;
        auto take = [&](size_t b) { size_t a = o; o += (b + 255) & ~size_t(255); return a; };
        L.pop[0] = take(5 * Q3 * N * sizeof(R));
        L.pop[1] = take(5 * Q3 * N * sizeof(R));
        L.h[0] = take(Q3 * N * sizeof(R));
        L.h[1] = take(Q3 * N * sizeof(R));
        L.phi = take(3 * N * sizeof(R));
        L.qt = take(N * sizeof(R));
        L.q = take(N * sizeof(R));
        L.rho = take(N * sizeof(R));
        L.sig = take(N * sizeof(R));
        L.eps = take(N * sizeof(R));
        L.E = take(3 * N * sizeof(R));
        L.mu = take(3 * N * sizeof(R));
        L.prev = take(12 * N * sizeof(R));
        L.diag = take(4 * N * sizeof(R));
        L.psi_prev = take(4 * N * sizeof(R));
        L.partial = take(nblocks(p) * (NOBS3 + 1) * sizeof(double));
        L.result = take(64 * sizeof(double));
        L.stage = take(N * sizeof(double) + 4 * N * sizeof(R));
        L.total = o;
        return L;
    }

    Sim3(const lb3e_params& prm, void* ws, cudaStream_t st) : p_(prm), stream_(st) {
        L_ = layout(prm);
        char* b = static_cast<char*>(ws);
        auto at = [&](size_t off) { return reinterpret_cast<R*>(b + off); };
        pop_[0] = at(L_.pop[0]); pop_[1] = at(L_.pop[1]); h_[0] = at(L_.h[0]); h_[1] = at(L_.h[1]);
        phi_ = at(L_.phi); qt_ = at(L_.qt); q_ = at(L_.q); rho_ = at(L_.rho); sig_ = at(L_.sig); eps_ = at(L_.eps);
        E_ = at(L_.E); mu_ = at(L_.mu); prev_ = at(L_.prev); diag_ = at(L_.diag); psi_prev_ = at(L_.psi_prev);
        partial_ = reinterpret_cast<double*>(b + L_.partial);
        result_ = reinterpret_cast<double*>(b + L_.result);
        stage_ = reinterpret_cast<double*>(b + L_.stage);
        P_ = make_p3(prm);
        N_ = P_.N;
        grid_ = dim3((prm.nx + 31) / 32, (prm.ny + 7) / 8, prm.nz);
        nblk_ = (int)nblocks(prm);
    }
    ~Sim3() override {
        if (pinned_) cudaFreeHost(pinned_);
    }

    int init(const double* phi, const double* u, const double* q, const double* noise) override {
        if (noise) return LB3E_ERR_PARAM;  // the 3-D path takes no population noise
        // the staged stencil tile exceeds the default 48 KB of dynamic shared memory in FP64
        if (cudaFuncSetAttribute(k3_collide<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)k3_collide_smem<R>()) != cudaSuccess)
            return LB3E_ERR_CUDA;
        if (cudaHostAlloc(reinterpret_cast<void**>(&pinned_), 64 * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
            return LB3E_ERR_CUDA;
        TRY(zero(err_flag(), sizeof(int)));
        tma_ready_ = tma_prepare();
        TRY(upload(phi, 3 * N_, phi_));
        if (u) TRY(upload(u, 3 * N_, diag_));
        else TRY(zero(diag_, 3 * N_ * sizeof(R)));
        if (q) TRY(upload(q, N_, q_));
        else TRY(zero(q_, N_ * sizeof(R)));
        TRY(zero(prev_, 12 * N_ * sizeof(R)));
        TRY(zero(psi_prev_, 4 * N_ * sizeof(R)));
        cur_ = hcur_ = 0;
        k3_props<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, phi_, rho_, sig_, eps_);
        TRY(launched());
        k3_init_h<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, h_[0]);
        TRY(launched());
        TRY(solve_now());
        k3_chem<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, phi_, E_, mu_);
        TRY(launched());
        k3_init_pops<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, pop_[0], phi_, q_, diag_, mu_, rho_);
        TRY(launched());
        step_ = 0;
        return sync();
    }

    int step(int nsteps) override {
        for (int s = 0; s < nsteps; ++s) {
            const int last = s == nsteps - 1;
            timer.begin(stream_, KC_MOMENTS);
            k3_moments<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, pop_[cur_], phi_, qt_, rho_, sig_, eps_);
            TRY(launched());
            timer.begin(stream_, KC_PROLOGUE);
            k3_closure<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, qt_, sig_, eps_, E_, q_);
            TRY(launched());
            TRY(solve_now());
            timer.begin(stream_, KC_OTHER);
            k3_chem<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, phi_, E_, mu_);
            TRY(launched());
            timer.begin(stream_, KC_FUSED);
            k3_collide<R><<<grid_, dim3(32, 8), k3_collide_smem<R>(), stream_>>>(P_, pop_[cur_], pop_[cur_ ^ 1], phi_, q_, E_, mu_, rho_,
                                                              sig_, eps_, prev_, diag_, step_ == 0 ? 1 : 0, last);
            TRY(launched());
            cur_ ^= 1;
            ++step_;
        }
        return LB3E_OK;
    }

    int solve_potential(const double* q, double tol, int max_iter, int check, int* iters, double* res) override {
        if (q) TRY(upload(q, N_, q_));
        TRY(poisson(tol, max_iter, 0, check));
        if (iters) *iters = last_iters_;
        if (res) *res = last_res_;
        TRY(sync());
        return last_conv_ ? LB3E_OK : LB3E_ERR_NOT_CONVERGED;
    }

    int observables(lb3e_observables_t* o) override {
        timer.begin(stream_, KC_REDUCE);
        const dim3 og = obs3_grid(p_);
        const int nob = (int)(og.x * og.y * og.z);
        k3_observables<R><<<og, dim3(32, 8), 0, stream_>>>(P_, phi_, q_, diag_, partial_,
                                                           partial_ + (size_t)nob * NOBS3);
        TRY(launched());
        k_reduce_partials<NOBS3><<<1, 256, 0, stream_>>>(partial_, nob, result_);
        TRY(launched());
        k_max_partials<<<1, 256, 0, stream_>>>(partial_ + (size_t)nob * NOBS3, nob, result_ + NOBS3);
        TRY(launched());
        if (cudaMemcpyAsync(pinned_, result_, (NOBS3 + 1) * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
            cudaSuccess)
            return LB3E_ERR_CUDA;
        TRY(sync());
        const double* v = pinned_;
        std::memset(o, 0, sizeof(*o));
        for (int i = 0; i < 3; ++i) o->mass[i] = v[i];
        o->charge = v[3];
        o->nonfinite = (int64_t)v[4];
        double Dk[2];
        for (int k = 0; k < 2; ++k) {
            const double* m = v + 5 + 5 * k;
            const double A = m[0];
            if (!(A > 0)) { Dk[k] = 0.0; continue; }
            const double xc = m[1] / A, zc = m[2] / A;
            const double Ixx = m[3] / A - xc * xc, Izz = m[4] / A - zc * zc;
            const double a = 2.0 * std::sqrt(Izz > 0 ? Izz : 0.0), bb = 2.0 * std::sqrt(Ixx > 0 ? Ixx : 0.0);
            Dk[k] = (a + bb) > 0 ? (a - bb) / (a + bb) : 0.0;
        }
        o->D_inner = Dk[0];
        o->D_outer = Dk[1];
        o->max_sum_dev = v[NOBS3];
        o->poisson_residual = last_res_;
        o->poisson_iters = last_iters_;
        o->poisson_converged = last_conv_;
        o->step = step_;
        return LB3E_OK;
    }

    int get_field(int id, double* dst) override {
        const R* src = nullptr;
        switch (id) {
            case LB3E_FIELD_PHI1: case LB3E_FIELD_PHI2: case LB3E_FIELD_PHI3: src = phi_ + (id - LB3E_FIELD_PHI1) * N_; break;
            case LB3E_FIELD_UX: src = diag_; break;
            case LB3E_FIELD_UY: src = diag_ + N_; break;
            case LB3E_FIELD_UZ: src = diag_ + 2 * N_; break;
            case LB3E_FIELD_P: src = diag_ + 3 * N_; break;
            case LB3E_FIELD_Q: src = q_; break;
            case LB3E_FIELD_EX: src = E_; break;
            case LB3E_FIELD_EY: src = E_ + N_; break;
            case LB3E_FIELD_EZ: src = E_ + 2 * N_; break;
            case LB3E_FIELD_MU1: case LB3E_FIELD_MU2: case LB3E_FIELD_MU3: src = mu_ + (id - LB3E_FIELD_MU1) * N_; break;
            case LB3E_FIELD_PSI: {
                R* tmp = reinterpret_cast<R*>(stage_ + N_);
                R* Etmp = tmp + N_;
                k3_fields<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, h_[hcur_], eps_, Etmp, tmp);
                TRY(launched());
                src = tmp;
                break;
            }
            case LB3E_FIELD_PHINOW1: case LB3E_FIELD_PHINOW2: case LB3E_FIELD_PHINOW3: case LB3E_FIELD_QTILDE: {
                R* tmp = reinterpret_cast<R*>(stage_ + N_);   // 4 planes: phi (3), q~
                R* scratch = reinterpret_cast<R*>(base_scratch());
                k3_moments<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, pop_[cur_], tmp, tmp + 3 * N_, scratch,
                                                                  scratch + N_, scratch + 2 * N_);
                TRY(launched());
                src = id == LB3E_FIELD_QTILDE ? tmp + 3 * N_ : tmp + (id - LB3E_FIELD_PHINOW1) * N_;
                break;
            }
            default: break;
        }
        if (!src && id >= LB3E_FIELD_POP && id < LB3E_FIELD_POP + 6 * Q3) {
            const int set = (id - LB3E_FIELD_POP) / Q3, j = (id - LB3E_FIELD_POP) % Q3;
            src = set < 5 ? pop_[cur_] + (size_t)(Q3 * set + j) * N_ : h_[hcur_] + (size_t)j * N_;
        }
        if (!src) return LB3E_ERR_FIELD;
        k3_pop_to_f64<R><<<(unsigned)((N_ + 255) / 256), 256, 0, stream_>>>(stage_, src, N_);
        TRY(launched());
        if (cudaMemcpyAsync(dst, stage_, N_ * sizeof(double), cudaMemcpyDefault, stream_) != cudaSuccess)
            return LB3E_ERR_CUDA;
        return sync();
    }

    size_t state_bytes() const override { return 0; }
    int save(void*) override { return LB3E_ERR_PARAM; }
    int load(const void*) override { return LB3E_ERR_PARAM; }
    int kernel_times(double* ms, int64_t* counts) override {
        TRY(sync());
        timer.collect();
        for (int k = 0; k < KC_COUNT; ++k) {
            if (ms) ms[k] = timer.ms[k];
            if (counts) counts[k] = timer.n[k];
            timer.ms[k] = 0.0;
            timer.n[k] = 0;
        }
        return LB3E_OK;
    }
    int64_t potential_iterations() const override { return iters_run_; }
    int set_chunk(int k) override { return k == 1 ? LB3E_OK : LB3E_ERR_PARAM; }
    int set_ions(const double*) override { return LB3E_ERR_PARAM; }
    int fd_residual(double*) override { return LB3E_ERR_PARAM; }
    int deformation(double*, double*) override { return LB3E_ERR_PARAM; }
    int shape_objective(const double*, double*, double*) override { return LB3E_ERR_PARAM; }
    int set_fused_tile(int) override { return LB3E_ERR_PARAM; }
    int set_staging(int planes) override {
        if (planes < 0 || planes > 1024) return LB3E_ERR_PARAM;
        staging_ = planes;
        return LB3E_OK;
    }

  private:
    // Scratch for the rho, sigma, eps outputs of a field-readback moments pass: the
    // residual-check planes.  Field readback happens between steps, and every solve
    // saves those planes before its first check reads them.
    R* base_scratch() { return psi_prev_; }
    int launched() {
        ++launches;
        timer.end(stream_);
        return cudaGetLastError() == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }
    // a kernel's error flag (a timed-out wait), read back by sync()
    int* err_flag() { return reinterpret_cast<int*>(result_ + 63); }
    int sync() {
        if (!pinned_) return cudaStreamSynchronize(stream_) == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
        int* fl = reinterpret_cast<int*>(pinned_ + 63);
        if (cudaMemcpyAsync(fl, err_flag(), sizeof(int), cudaMemcpyDeviceToHost, stream_) != cudaSuccess)
            return LB3E_ERR_CUDA;
        if (cudaStreamSynchronize(stream_) != cudaSuccess) return LB3E_ERR_CUDA;
        if (*fl) {
            *fl = 0;
            cudaMemsetAsync(err_flag(), 0, sizeof(int), stream_);
            return LB3E_ERR_CUDA;
        }
        return LB3E_OK;
    }
    // Tensor maps of the staged potential iteration: the two h buffers as (nx, ny,
    // 15 nz) arrays, eps and q as (nx, ny, nz), boxes of 32 x 8 x 1 (FP32 only; the
    // row pitch must be a multiple of 16 bytes)
    bool tma_prepare() {
        if constexpr (!std::is_same<R, float>::value) {
            return false;
        } else {
            if (p_.nx % 4 != 0) return false;
            using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                        const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                        CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
            static Encode encode = [] {
                void* f = nullptr;
                cudaDriverEntryPointQueryResult q{};
                if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                        cudaSuccess ||
                    q != cudaDriverEntryPointSuccess)
                    f = nullptr;
                return reinterpret_cast<Encode>(f);
            }();
            if (!encode) return false;
            const cuuint64_t nx = (cuuint64_t)p_.nx, ny = (cuuint64_t)p_.ny, nz = (cuuint64_t)p_.nz;
            const cuuint32_t one[3] = {1, 1, 1}, box[3] = {32, 8, 1};
            auto make = [&](CUtensorMap* m, void* base, cuuint64_t planes) {
                const cuuint64_t dims[3] = {nx, ny, planes};
                const cuuint64_t strides[2] = {nx * sizeof(float), nx * ny * sizeof(float)};
                return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, one,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
            };
            if (!make(&tm_h_[0], h_[0], Q3 * nz) || !make(&tm_h_[1], h_[1], Q3 * nz) || !make(&tm_eps_, eps_, nz) ||
                !make(&tm_q_, q_, nz))
                return false;
            return cudaFuncSetAttribute(k3_poisson_tma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)k3_poisson_tma_smem<float>()) == cudaSuccess;
        }
    }
    int zero(void* p, size_t b) { return cudaMemsetAsync(p, 0, b, stream_) == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA; }
    int upload(const double* src, size_t n, R* dst) {
        for (size_t off = 0; off < n; off += N_) {
            const size_t m = (n - off) < N_ ? (n - off) : N_;
            if (cudaMemcpyAsync(stage_, src + off, m * sizeof(double), cudaMemcpyDefault, stream_) != cudaSuccess)
                return LB3E_ERR_CUDA;
            k_from_f64<R><<<(unsigned)((m + 255) / 256), 256, 0, stream_>>>(dst + off, stage_, m);
            TRY(launched());
        }
        return LB3E_OK;
    }
    int solve_now() {
        if (p_.electric) return poisson(p_.poisson_tol, p_.poisson_max_iter, p_.poisson_fixed_iter, p_.poisson_check_every);
        k3_fill_E<R><<<(unsigned)((N_ + 255) / 256), 256, 0, stream_>>>(P_, E_);
        return launched();
    }
    // Iterate Eq. 43 until the relative increments of psi and J are <= tol (checked
    // every `check` iterations before that iteration's collision, against the state
    // saved one iteration earlier), or exactly `fixed` iterations.
    int poisson(double tol, int max_iter, int fixed, int check) {
        const int n = fixed > 0 ? fixed : max_iter;
        if (check < 1) check = 1;
        last_res_ = -1.0;
        last_conv_ = fixed > 0;
        last_iters_ = n;
        for (int k = 1; k <= n; ++k) {
            const int do_check = fixed <= 0 && k >= 2 && k % check == 0;
            const int save = fixed <= 0 && (k + 1) % check == 0;
            timer.begin(stream_, KC_POISSON);
            if (tma_ready_ && staging_ && !save && !do_check) {
                if constexpr (std::is_same<R, float>::value) {
                    const dim3 g((p_.nx + 31) / 32, (p_.ny + 7) / 8, (p_.nz + staging_ - 1) / staging_);
                    k3_poisson_tma<float><<<g, dim3(32, 8), k3_poisson_tma_smem<float>(), stream_>>>(
                        P_, tm_h_[hcur_], tm_eps_, tm_q_, h_[hcur_ ^ 1], staging_, err_flag());
                }
            } else {
                k3_poisson<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, h_[hcur_], h_[hcur_ ^ 1], eps_, q_, psi_prev_,
                                                                  partial_, save, do_check);
            }
            TRY(launched());
            if (do_check) {
                // the residual of the state before this launch's collision
                k_reduce_partials<4><<<1, 256, 0, stream_>>>(partial_, nblk_, result_);
                TRY(launched());
                if (cudaMemcpyAsync(pinned_, result_, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream_) != cudaSuccess)
                    return LB3E_ERR_CUDA;
                TRY(sync());
                const double dp = pinned_[0], pp = pinned_[1], dj = pinned_[2], jj = pinned_[3];
                const double r1 = pp > 0.0 ? std::sqrt(dp) / std::sqrt(pp) : (dp > 0.0 ? INFINITY : 0.0);
                const double r2 = jj > 0.0 ? std::sqrt(dj) / std::sqrt(jj) : (dj > 0.0 ? INFINITY : 0.0);
                last_res_ = r1 > r2 ? r1 : r2;
                if (last_res_ <= tol) {
                    // the launch also collided and streamed: its output is discarded
                    last_conv_ = 1;
                    last_iters_ = k - 1;
                    ++iters_run_;
                    break;
                }
            }
            hcur_ ^= 1;
            ++iters_run_;
        }
        timer.begin(stream_, KC_FIELDS);
        k3_fields<R><<<grid_, dim3(32, 8), 0, stream_>>>(P_, h_[hcur_], eps_, E_, nullptr);
        return launched();
    }

    lb3e_params p_;
    cudaStream_t stream_;
    Layout L_;
    P3 P_{};
    size_t N_ = 0;
    dim3 grid_;
    int nblk_ = 0;
    R *pop_[2]{}, *h_[2]{}, *phi_{}, *qt_{}, *q_{}, *rho_{}, *sig_{}, *eps_{}, *E_{}, *mu_{}, *prev_{}, *diag_{},
        *psi_prev_{};
    double *partial_{}, *result_{}, *stage_{};
    double* pinned_ = nullptr;
    CUtensorMap tm_h_[2]{}, tm_eps_{}, tm_q_{};  // the staged potential iteration's tensor maps (tma_prepare)
    bool tma_ready_ = false;
    int staging_ = 2;  // planes a block walks in the staged potential iteration (0: per-thread loads)
    int cur_ = 0, hcur_ = 0;
    int64_t step_ = 0;
    int last_iters_ = 0, last_conv_ = 0;
    double last_res_ = -1.0;
    int64_t iters_run_ = 0;
};

}  // namespace lb3e
