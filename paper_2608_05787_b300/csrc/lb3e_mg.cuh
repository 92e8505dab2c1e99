// lb3e_mg.cuh -- geometric multigrid for the finite-difference form of the
// potential equation div(eps grad psi) + q = 0 (Eq. 27d), an alternative to the
// paper's pseudo-time LB solve for lattices where the latter needs far too many
// iterations per step.
//
// Discretisation (cell-centred, lattice units): 5-point stencil, face
// permittivity = harmonic mean of the two cells, electrodes as Dirichlet faces at
// distance 1/2 (flux 2 eps_C (V - psi_C)), x periodic.  Only walls carrying
// electrodes are supported (bc_y = 2).  The operator is applied unscaled
// (A psi = sum of face fluxes), so a coarse level, with cells 2x larger, takes
// the sum of its four children's residuals as right-hand side.  Red-black
// Gauss-Seidel smoothing, bilinear prolongation, FP64 throughout; the V-cycle is
// repeated until ||b - A psi|| / ||b|| <= tol on the fine level.  Face
// coefficients and inverse diagonals are formed once per solve, so the sweeps are
// multiply-adds only (FP64 division is expensive on this part).
#pragma once

#include "lb3e_kernels.cuh"

namespace lb3e {

struct MGLevel {
    int nx, ny;
    double *psi, *rhs, *res, *eps;
    double *ae, *an, *dg, *idg;  // east / north face coefficients, diagonal and its inverse
};

__device__ __forceinline__ double mg_hmean(double a, double b) { return 2.0 * a * b / (a + b); }

// Face coefficients of level L (harmonic means; no face across an electrode wall,
// which instead adds 2 eps_C to the diagonal).  The only FP64 divisions of a solve
// happen here, once per level.
static __global__ void __launch_bounds__(256) k_mg_coeffs(MGLevel L) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int c = y * L.nx + x;
    const double ec = L.eps[c];
    const int xe = x + 1 == L.nx ? 0 : x + 1, xw = x == 0 ? L.nx - 1 : x - 1;
    const double ae = mg_hmean(ec, L.eps[y * L.nx + xe]);
    const double aw = mg_hmean(ec, L.eps[y * L.nx + xw]);
    const double an = y + 1 < L.ny ? mg_hmean(ec, L.eps[c + L.nx]) : 0.0;
    const double as = y > 0 ? mg_hmean(ec, L.eps[c - L.nx]) : 0.0;
    const double d = ae + aw + (y + 1 < L.ny ? an : 2.0 * ec) + (y > 0 ? as : 2.0 * ec);
    L.ae[c] = ae;
    L.an[c] = an;
    L.dg[c] = d;
    L.idg[c] = 1.0 / d;
}

// sum_{faces} a_f psi_neighbour at cell (x, y)
__device__ __forceinline__ double mg_offdiag(const MGLevel& L, int x, int y, int c) {
    const int xe = x + 1 == L.nx ? 0 : x + 1, xw = x == 0 ? L.nx - 1 : x - 1;
    double off = L.ae[c] * L.psi[y * L.nx + xe] + L.ae[y * L.nx + xw] * L.psi[y * L.nx + xw];
    if (y + 1 < L.ny) off += L.an[c] * L.psi[c + L.nx];
    if (y > 0) off += L.an[c - L.nx] * L.psi[c - L.nx];
    return off;
}

// one colour of red-black Gauss-Seidel on level L
static __global__ void __launch_bounds__(256) k_mg_smooth(MGLevel L, int color) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny || ((x + y) & 1) != color) return;
    const int c = y * L.nx + x;
    L.psi[c] = (L.rhs[c] + mg_offdiag(L, x, y, c)) * L.idg[c];
}

// res = rhs - A psi; optionally FP64 partial sums of res^2 and rhs^2 per block
static __global__ void __launch_bounds__(256) k_mg_residual(MGLevel L, double* __restrict__ partial) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    double acc[2] = {0.0, 0.0};
    if (x < L.nx && y < L.ny) {
        const int c = y * L.nx + x;
        const double b = L.rhs[c];
        const double r = b - (L.dg[c] * L.psi[c] - mg_offdiag(L, x, y, c));
        L.res[c] = r;
        acc[0] = r * r;
        acc[1] = b * b;
    }
    if (partial) block_reduce_store<2>(acc, partial + 2 * (size_t)(blockIdx.x + gridDim.x * blockIdx.y));
}

// coarse right-hand side = sum of the four children's residuals; coarse guess 0
static __global__ void __launch_bounds__(256) k_mg_restrict(MGLevel F, MGLevel C) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= C.nx || y >= C.ny) return;
    const int f = 2 * y * F.nx + 2 * x;
    C.rhs[y * C.nx + x] = F.res[f] + F.res[f + 1] + F.res[f + F.nx] + F.res[f + F.nx + 1];
    C.psi[y * C.nx + x] = 0.0;
}

// coarse permittivity = mean of the four children (re-discretised coarse operator)
static __global__ void __launch_bounds__(256) k_mg_coarsen_eps(MGLevel F, MGLevel C) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= C.nx || y >= C.ny) return;
    const int f = 2 * y * F.nx + 2 * x;
    C.eps[y * C.nx + x] = 0.25 * (F.eps[f] + F.eps[f + 1] + F.eps[f + F.nx] + F.eps[f + F.nx + 1]);
}

// psi_fine += bilinear interpolation of the coarse correction (x periodic; the
// coarse error vanishes on the electrode faces, so its ghost is -value)
__device__ __forceinline__ double mg_coarse_at(const MGLevel& C, int x, int y) {
    x = x < 0 ? x + C.nx : (x >= C.nx ? x - C.nx : x);
    if (y < 0) return -C.psi[x];
    if (y >= C.ny) return -C.psi[(C.ny - 1) * C.nx + x];
    return C.psi[y * C.nx + x];
}
static __global__ void __launch_bounds__(256) k_mg_prolong(MGLevel F, MGLevel C) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= F.nx || y >= F.ny) return;
    const int cx0 = x >> 1, cy0 = y >> 1;
    const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1;
    const double v = 0.5625 * mg_coarse_at(C, cx0, cy0) + 0.1875 * mg_coarse_at(C, cx0 + sx, cy0) +
                     0.1875 * mg_coarse_at(C, cx0, cy0 + sy) + 0.0625 * mg_coarse_at(C, cx0 + sx, cy0 + sy);
    F.psi[y * F.nx + x] += v;
}

// the coarsest level, solved by many red-black sweeps inside one block
static __global__ void __launch_bounds__(256) k_mg_coarse_solve(MGLevel L, int sweeps) {
    const int n = L.nx * L.ny;
    for (int s = 0; s < sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                const int x = c % L.nx, y = c / L.nx;
                if (((x + y) & 1) != color) continue;
                L.psi[c] = (L.rhs[c] + mg_offdiag(L, x, y, c)) * L.idg[c];
            }
            __syncthreads();
        }
}

// level-0 inputs: eps (R) -> FP64; rhs = q plus the electrode terms 2 eps_C V of
// the wall rows (the coarse error equations are homogeneous)
template <class R>
static __global__ void __launch_bounds__(256) k_mg_load(MGLevel L, const R* __restrict__ eps, const R* __restrict__ q,
                                                        double vb, double vt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int c = y * L.nx + x;
    const double e = (double)eps[c];
    double b = (double)q[c];
    if (y + 1 == L.ny) b += 2.0 * e * vt;
    if (y == 0) b += 2.0 * e * vb;
    L.eps[c] = e;
    L.rhs[c] = b;
}

// E = -grad psi with the isotropic stencil of Eq. 33; ghosts 2V - psi at electrodes
__device__ __forceinline__ double mg_psi_ghost(const MGLevel& L, int x, int y, double vb, double vt) {
    x = x < 0 ? x + L.nx : (x >= L.nx ? x - L.nx : x);
    if (y < 0) return 2.0 * vb - L.psi[x];
    if (y >= L.ny) return 2.0 * vt - L.psi[(L.ny - 1) * L.nx + x];
    return L.psi[y * L.nx + x];
}
template <class R>
static __global__ void __launch_bounds__(256) k_mg_fields(MGLevel L, double vb, double vt, double ex, double ey,
                                                          R* __restrict__ E) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const double v = mg_psi_ghost(L, x + cx(j), y + cy(j), vb, vt);
        ax += wgt<double>(j) * cx(j) * v;
        ay += wgt<double>(j) * cy(j) * v;
    }
    const int c = y * L.nx + x;
    const size_t N = (size_t)L.nx * L.ny;
    E[c] = R(-(ax * 3.0) + ex);  // / cs^2 (a multiply: FP64 division is slow here)
    E[N + c] = R(-(ay * 3.0) + ey);
}

// initial guess: the linear electrode profile
static __global__ void __launch_bounds__(256) k_mg_init(MGLevel L, double vb, double vt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    L.psi[y * L.nx + x] = vb + (vt - vb) * (y + 0.5) / L.ny;
}

// levels for an nx x ny lattice: halve while both sides stay even and >= 8
inline int mg_levels(int nx, int ny) {
    int L = 1;
    while ((nx % 2) == 0 && (ny % 2) == 0 && nx / 2 >= 4 && ny / 2 >= 4 && L < 16) {
        nx /= 2;
        ny /= 2;
        ++L;
    }
    return L;
}

}  // namespace lb3e
