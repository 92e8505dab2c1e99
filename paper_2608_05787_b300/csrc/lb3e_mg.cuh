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
// Gauss-Seidel smoothing, bilinear prolongation.
//
// Precision: defect correction.  The fine-level potential, right-hand side and
// coefficients are FP64, and so is each residual r = b - A psi (formed in FP64,
// its norm summed in FP64 across warps).  The V-cycle then solves A e = r in FP32
// on a parallel FP32 hierarchy, and psi += e in FP64.  Each cycle cuts the FP64
// residual by the V-cycle's factor as long as that factor is well above FP32
// rounding, so the loop reaches FP64-level tolerances; the V-cycle itself runs on
// the FP32 pipe (FP64 runs at a small fraction of its rate on this part) and moves
// half the bytes.  Repeated until ||b - A psi|| / ||b|| <= tol.  Face coefficients
// and inverse diagonals are formed once per solve (FP64, then rounded to FP32), so
// the sweeps are multiply-adds only.
#pragma once

#include "lb3e_kernels.cuh"

namespace lb3e {

template <class T>
struct MGLevelT {
    int nx, ny;
    T *psi, *rhs, *res, *eps;  // eps: FP64 levels only
    T *ae, *an, *dg, *idg;     // east / north face coefficients, diagonal and its inverse
};
using MGLevel = MGLevelT<double>;   // the equation itself (coefficients on every level)
using MGLevelF = MGLevelT<float>;   // the FP32 error equation of the V-cycle

__device__ __forceinline__ double mg_hmean(double a, double b) { return 2.0 * a * b / (a + b); }

// Face coefficients of level L (harmonic means; no face across an electrode wall,
// which instead adds 2 eps_C to the diagonal).  Fine level, FP64 (the FP64 residual
// uses them), in two passes so that each face's division happens once: the east and
// north faces of every cell, then the diagonal from a cell's own faces and its west
// and south neighbours' (the harmonic mean is symmetric, so these equal the faces
// seen from this cell bit for bit).  Copies rounded to FP32 feed the V-cycle.
static __global__ void __launch_bounds__(256) k_mg_faces(MGLevel L) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int c = y * L.nx + x;
    const double ec = L.eps[c];
    const int xe = x + 1 == L.nx ? 0 : x + 1;
    L.ae[c] = mg_hmean(ec, L.eps[y * L.nx + xe]);
    L.an[c] = y + 1 < L.ny ? mg_hmean(ec, L.eps[c + L.nx]) : 0.0;
}
static __global__ void __launch_bounds__(256) k_mg_diag(MGLevel L, MGLevelF F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int c = y * L.nx + x;
    const double ec = L.eps[c];
    const int xw = x == 0 ? L.nx - 1 : x - 1;
    const double ae = L.ae[c], an = L.an[c];
    const double aw = L.ae[y * L.nx + xw];
    const double as = y > 0 ? L.an[c - L.nx] : 0.0;
    const double d = ae + aw + (y + 1 < L.ny ? an : 2.0 * ec) + (y > 0 ? as : 2.0 * ec);
    L.dg[c] = d;
    L.idg[c] = 1.0 / d;
    F.ae[c] = (float)ae;
    F.an[c] = (float)an;
    F.dg[c] = (float)d;
    F.idg[c] = (float)(1.0 / d);
}
// Coarse levels: coefficients only set the V-cycle's rate of convergence, not the
// answer (the FP64 fine residual does), so they are formed in FP32 from the
// coarsened permittivity, directly into the FP32 level.
static __global__ void __launch_bounds__(256) k_mg_coeffs_f(MGLevel L, MGLevelF F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int c = y * L.nx + x;
    auto hm = [](float a, float b) { return 2.0f * a * b / (a + b); };
    const float ec = (float)L.eps[c];
    const int xe = x + 1 == L.nx ? 0 : x + 1, xw = x == 0 ? L.nx - 1 : x - 1;
    const float ae = hm(ec, (float)L.eps[y * L.nx + xe]);
    const float aw = hm(ec, (float)L.eps[y * L.nx + xw]);
    const float an = y + 1 < L.ny ? hm(ec, (float)L.eps[c + L.nx]) : 0.0f;
    const float as = y > 0 ? hm(ec, (float)L.eps[c - L.nx]) : 0.0f;
    const float d = ae + aw + (y + 1 < L.ny ? an : 2.0f * ec) + (y > 0 ? as : 2.0f * ec);
    F.ae[c] = ae;
    F.an[c] = an;
    F.dg[c] = d;
    F.idg[c] = 1.0f / d;
}

// sum_{faces} a_f psi_neighbour at cell (x, y)
template <class T>
__device__ __forceinline__ T mg_offdiag(const MGLevelT<T>& L, int x, int y, int c) {
    const int xe = x + 1 == L.nx ? 0 : x + 1, xw = x == 0 ? L.nx - 1 : x - 1;
    T off = L.ae[c] * L.psi[y * L.nx + xe] + L.ae[y * L.nx + xw] * L.psi[y * L.nx + xw];
    if (y + 1 < L.ny) off += L.an[c] * L.psi[c + L.nx];
    if (y > 0) off += L.an[c - L.nx] * L.psi[c - L.nx];
    return off;
}

// one colour of red-black Gauss-Seidel on level L
template <class T>
__global__ void __launch_bounds__(256) k_mg_smooth(MGLevelT<T> L, int color) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny || ((x + y) & 1) != color) return;
    const int c = y * L.nx + x;
    L.psi[c] = (L.rhs[c] + mg_offdiag(L, x, y, c)) * L.idg[c];
}

// res = rhs - A psi (in the level's precision); optionally per-block sums of res^2
// and rhs^2 (squares in FP32, summed in FP32 within a warp and in FP64 across
// warps: a norm needs a few digits, the residual itself is formed in full)
template <class T>
__global__ void __launch_bounds__(256) k_mg_residual(MGLevelT<T> L, double* __restrict__ partial) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    float acc[2] = {0.f, 0.f};
    if (x < L.nx && y < L.ny) {
        const int c = y * L.nx + x;
        const T b = L.rhs[c];
        const T r = b - (L.dg[c] * L.psi[c] - mg_offdiag(L, x, y, c));
        L.res[c] = r;
        acc[0] = (float)r * (float)r;
        acc[1] = (float)b * (float)b;
    }
    if (partial) block_reduce_store_r<2>(acc, partial + 2 * (size_t)(blockIdx.x + gridDim.x * blockIdx.y));
}

// start of a V-cycle on the error equation: F.rhs = the fine FP64 residual, F.psi = 0
static __global__ void __launch_bounds__(256) k_mg_defect(MGLevel D, MGLevelF F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= D.nx || y >= D.ny) return;
    const int c = y * D.nx + x;
    F.rhs[c] = (float)D.res[c];
    F.psi[c] = 0.f;
}
// end of a V-cycle: psi += e (FP64)
static __global__ void __launch_bounds__(256) k_mg_correct(MGLevel D, MGLevelF F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= D.nx || y >= D.ny) return;
    const int c = y * D.nx + x;
    D.psi[c] += (double)F.psi[c];
}

// coarse right-hand side = sum of the four children's residuals; coarse guess 0
template <class T>
__global__ void __launch_bounds__(256) k_mg_restrict(MGLevelT<T> F, MGLevelT<T> C) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= C.nx || y >= C.ny) return;
    const int f = 2 * y * F.nx + 2 * x;
    C.rhs[y * C.nx + x] = F.res[f] + F.res[f + 1] + F.res[f + F.nx] + F.res[f + F.nx + 1];
    C.psi[y * C.nx + x] = T(0);
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
template <class T>
__device__ __forceinline__ T mg_coarse_at(const MGLevelT<T>& C, int x, int y) {
    x = x < 0 ? x + C.nx : (x >= C.nx ? x - C.nx : x);
    if (y < 0) return -C.psi[x];
    if (y >= C.ny) return -C.psi[(C.ny - 1) * C.nx + x];
    return C.psi[y * C.nx + x];
}
template <class T>
__global__ void __launch_bounds__(256) k_mg_prolong(MGLevelT<T> F, MGLevelT<T> C) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= F.nx || y >= F.ny) return;
    const int cx0 = x >> 1, cy0 = y >> 1;
    const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1;
    const T v = T(0.5625) * mg_coarse_at(C, cx0, cy0) + T(0.1875) * mg_coarse_at(C, cx0 + sx, cy0) +
                T(0.1875) * mg_coarse_at(C, cx0, cy0 + sy) + T(0.0625) * mg_coarse_at(C, cx0 + sx, cy0 + sy);
    F.psi[y * F.nx + x] += v;
}

// the coarsest level, solved by many red-black sweeps inside one block
template <class T>
__global__ void __launch_bounds__(256) k_mg_coarse_solve(MGLevelT<T> L, int sweeps) {
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

// The small levels of a V-cycle in one block: from level lv[0] (its rhs restricted,
// psi = 0) down to the coarsest and back, each pass a block-strided loop closed by a
// barrier, with the per-cell arithmetic of k_mg_smooth, k_mg_residual,
// k_mg_restrict, k_mg_coarse_solve and k_mg_prolong.  These levels hold a few
// thousand cells or fewer, so one block does them in less time than their ~10
// launches a level take to issue.
constexpr int MG_SMALL_MAX = 12, MG_SMALL_CELLS = 4096, MG_SMALL_THREADS = 1024;
template <class T>
struct MGSmall {
    MGLevelT<T> lv[MG_SMALL_MAX];
    int n;  // levels lv[0 .. n-1], lv[n-1] the coarsest
};
template <class T>
__device__ __forceinline__ void mgb_smooth(const MGLevelT<T>& L, int sweeps) {
    const int n = L.nx * L.ny;
    for (int s = 0; s < sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                const int y = c / L.nx, x = c - y * L.nx;
                if (((x + y) & 1) != color) continue;
                L.psi[c] = (L.rhs[c] + mg_offdiag(L, x, y, c)) * L.idg[c];
            }
            __syncthreads();
        }
}
template <class T>
__global__ void __launch_bounds__(MG_SMALL_THREADS) k_mg_small_cycle(MGSmall<T> S) {
    for (int l = 0; l + 1 < S.n; ++l) {
        const MGLevelT<T>& F = S.lv[l];
        const MGLevelT<T>& C = S.lv[l + 1];
        mgb_smooth(F, 2);
        const int nf = F.nx * F.ny;
        for (int c = threadIdx.x; c < nf; c += blockDim.x) {
            const int y = c / F.nx, x = c - y * F.nx;
            F.res[c] = F.rhs[c] - (F.dg[c] * F.psi[c] - mg_offdiag(F, x, y, c));
        }
        __syncthreads();
        const int nc = C.nx * C.ny;
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const int y = c / C.nx, x = c - y * C.nx;
            const int f = 2 * y * F.nx + 2 * x;
            C.rhs[c] = F.res[f] + F.res[f + 1] + F.res[f + F.nx] + F.res[f + F.nx + 1];
            C.psi[c] = T(0);
        }
        __syncthreads();
    }
    mgb_smooth(S.lv[S.n - 1], 50);  // the coarsest level (the sweeps of k_mg_coarse_solve)
    for (int l = S.n - 2; l >= 0; --l) {
        const MGLevelT<T>& F = S.lv[l];
        const MGLevelT<T>& C = S.lv[l + 1];
        const int nf = F.nx * F.ny;
        for (int c = threadIdx.x; c < nf; c += blockDim.x) {
            const int y = c / F.nx, x = c - y * F.nx;
            const int cx0 = x >> 1, cy0 = y >> 1;
            const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1;
            F.psi[c] += T(0.5625) * mg_coarse_at(C, cx0, cy0) + T(0.1875) * mg_coarse_at(C, cx0 + sx, cy0) +
                        T(0.1875) * mg_coarse_at(C, cx0, cy0 + sy) + T(0.0625) * mg_coarse_at(C, cx0 + sx, cy0 + sy);
        }
        __syncthreads();
        mgb_smooth(F, 2);
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
// (FP64 output: all in FP64)
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
    const int c = y * L.nx + x;
    const size_t N = (size_t)L.nx * L.ny;
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const double v = mg_psi_ghost(L, x + cx(j), y + cy(j), vb, vt);
        ax += wgt<double>(j) * cx(j) * v;
        ay += wgt<double>(j) * cy(j) * v;
    }
    E[c] = R(-(ax * 3.0) + ex);  // / cs^2 (a multiply: FP64 division is slow here)
    E[N + c] = R(-(ay * 3.0) + ey);
}
// FP32 output.  The electrode profile makes psi large against its neighbour
// differences, so the differences need more than FP32: the block stages psi (ghosts
// included) of its tile and one-cell ring as hi + lo FP32 pairs, one FP64 split a
// cell (FP64 runs at a small fraction of the FP32 rate), and forms each difference
// as (hi_n - hi_c) + (lo_n - lo_c) in FP32; weighted sums in FP32
template <class R>
static __global__ void __launch_bounds__(256) k_mg_fields_f32(MGLevel L, double vb, double vt, double ex, double ey,
                                                              R* __restrict__ E) {
    constexpr int SX = 34, SY = 10;  // blockDim (32, 8) and a one-cell ring
    __shared__ float shi[SY * SX], slo[SY * SX];
    const int x0 = blockIdx.x * blockDim.x, y0 = blockIdx.y * blockDim.y;
    for (int k = threadIdx.x + blockDim.x * threadIdx.y; k < SX * SY; k += blockDim.x * blockDim.y) {
        const int ly = k / SX, lx = k - ly * SX;
        const int gy = y0 + ly - 1, gx = x0 + lx - 1;
        double v = 0.0;
        if (gy >= -1 && gy <= L.ny) v = mg_psi_ghost(L, gx, gy, vb, vt);  // rows beyond the ring row: unused
        const float hi = (float)v;
        shi[k] = hi;
        slo[k] = (float)(v - (double)hi);
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int c = y * L.nx + x;
    const size_t N = (size_t)L.nx * L.ny;
    const int sc = (threadIdx.y + 1) * SX + threadIdx.x + 1;
    const float hc = shi[sc], lc = slo[sc];
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int j = 1; j < 9; ++j) {
        const int sn = sc + cy(j) * SX + cx(j);
        const float d = (shi[sn] - hc) + (slo[sn] - lc);
        cacc(ax, cx(j), wgt<float>(j), d);
        cacc(ay, cy(j), wgt<float>(j), d);
    }
    E[c] = R(-(ax * 3.0f) + (float)ex);  // / cs^2
    E[N + c] = R(-(ay * 3.0f) + (float)ey);
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
