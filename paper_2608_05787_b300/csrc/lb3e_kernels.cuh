// lb3e_kernels.cuh -- sm_103a kernels of the three-phase EHD lattice Boltzmann step.
//
// Templated on the arithmetic type R (double or float) and the population storage
// type S (double, float or __half).  lb3e_f64.cu instantiates <double,double> with
// --fmad=false so its arithmetic rounds exactly like a plain C evaluation of the
// same formulas; lb3e_f32.cu instantiates <float,float> and <float,__half>.
//
// Layout in HBM (structure of arrays, x fastest): population plane (set, j) of a
// buffer is the contiguous [ny][nx] array at offset (9*set + j) * N, sets 0 = g
// (flow), 1..3 = f^1..f^3 (phase), 4 = l (charge).  The potential populations h
// live in their own 9-plane buffers.  Populations are stored post-streaming (the
// state at the start of a step); collision kernels read their own cell and push
// each post-collision value to the neighbour it streams to (x periodic, half-way
// bounce-back at y walls).
#pragma once

#include <cuda.h>  // CUtensorMap (the tensor-map descriptor type of the TMA copies)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lb3e_dual.cuh"

namespace lb3e {

// ---------------------------------------------------------------- parameters
struct DevParams {
    int nx, ny, N, bc_y, electric, charge_convection, use_visc;
    int inner, matrix;  // 0-based phase indices for the deformation moments
    double rho[3], visc[3], tau_g, lam[3], D, tau_f, m0, eps[3], sigma[3];
    double eps_ref, tau_h, alpha, tau_l;
    double V_bottom, V_top, E_ext[2], u_wall_bottom, u_wall_top;
    // tangent seeds (dual-number builds only): d(param)/d(theta_k), k < 4
    double t_eps[3][4], t_lam[3][4], t_Vb[4], t_Vt[4];
    // single-precision copies used by the FP32 kernels (FP64 arithmetic, including
    // conversions, is slow on this part)
    float frho[3], fvisc[3], feps[3], fsig[3], flam[3];
    float fD, ftau_f, fm0, ftau_g, ftau_l, ftau_h, feps_ref, fVb, fVt, fuwb, fuwt, fE[2];
    // launch-wide constants of the FP32 collisions, formed once on the host:
    // 1/tau, the source prefactor 1 - 1/(2 tau), 1/m0 and 24/D
    float fitau_f, fpf, fim0, fitau_g, fpg, fitau_l, fpl, fitau_h, fc24;
};

// Device-side buffers of one simulation (pointers into the caller's workspace).
template <class R, class S>
struct DevState {
    S* pop[2];       // 45 planes each; pop[cur] holds the current state
    R* h[2];         // 9 planes each
    R* phi;          // 3 planes: phi_i of the last step
    R* qt;           // sum l of the last step
    R* q;            // corrected charge of the last step
    R* eps;          // permittivity of the last step
    R* E;            // 2 planes: field used in the last step
    R* prev;         // 8 planes: (phi_i u)_x, (phi_i u)_y for i = 1..3, then (q u)_x, (q u)_y
    R* diag;         // 6 planes: u_x, u_y, p, mu_1, mu_2, mu_3 of the last output step
    R* psi_prev;     // 3 planes: psi, J_x, J_y at the previous pseudo-iteration
    double* partial; // FP64 per-block partial sums
    double* result;  // FP64 reduction results
    double* stage;   // FP64 staging (9 planes)
};

// ---------------------------------------------------------------- lattice (Eq. 31)
__host__ __device__ constexpr int cx(int j) { return (j == 1 || j == 5 || j == 8) ? 1 : (j == 3 || j == 6 || j == 7) ? -1 : 0; }
__host__ __device__ constexpr int cy(int j) { return (j == 2 || j == 5 || j == 6) ? 1 : (j == 4 || j == 7 || j == 8) ? -1 : 0; }
__host__ __device__ constexpr int opp(int j) { return j == 0 ? 0 : (j <= 4 ? ((j + 1) & 3) + 1 : ((j - 3) & 3) + 5); }
template <class R>
__host__ __device__ constexpr R wgt(int j) { return j == 0 ? R(4.0 / 9.0) : (j <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0)); }
template <class R>
__host__ __device__ constexpr R cs2() { return R(1.0 / 3.0); }
// c_j . (ax, ay) with the zero components left out and the unit ones as adds: the
// same value as cx*ax + cy*ay (x * 0 is not folded away without fast-math, so the
// literal form costs a multiply per zero component)
template <class R>
__device__ __forceinline__ R cdot(int j, R ax, R ay) {
    if (cx(j) == 0 && cy(j) == 0) return R(0);
    if (cy(j) == 0) return cx(j) > 0 ? ax : -ax;
    if (cx(j) == 0) return cy(j) > 0 ? ay : -ay;
    const R a = cx(j) > 0 ? ax : -ax;
    return cy(j) > 0 ? a + ay : a - ay;
}
// acc += c_j,x * v (or c_j,y * v) in j order, skipping zero components
template <class R>
__device__ __forceinline__ void cacc(R& acc, int c, R v) {
    if (c > 0) acc += v;
    else if (c < 0) acc -= v;
}
// a * b + c rounded once.  The factored FP32 collisions spell out every FMA, so
// their rounding does not depend on how the compiler contracts one kernel or
// another (a batched and a single-lattice kernel then give the same bits).
__device__ __forceinline__ float fmaf_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// the same for FP32 dual numbers: (a b + c)' = a' b + a b' + c', each part rounded once
template <int M>
__device__ __forceinline__ Dual<float, M> fmaf_(const Dual<float, M>& a, const Dual<float, M>& b,
                                                const Dual<float, M>& c) {
    Dual<float, M> r;
    r.v = __fmaf_rn(a.v, b.v, c.v);
#pragma unroll
    for (int k = 0; k < M; ++k) r.d[k] = __fmaf_rn(a.v, b.d[k], __fmaf_rn(a.d[k], b.v, c.d[k]));
    return r;
}
// FP32 arithmetic, plain or with FP32 tangents: the builds that take the factored
// collision forms (the FP64 builds evaluate the paper's equations as written)
template <class R> struct f32_family { static constexpr bool value = std::is_same<R, float>::value; };
template <int M> struct f32_family<Dual<float, M>> { static constexpr bool value = true; };
// acc += c * w * v for a lattice component c in {-1, 0, 1} (one FMA, or nothing)
template <class R>
__device__ __forceinline__ void cacc(R& acc, int c, R w, R v) {
    if (c > 0) acc += w * v;
    else if (c < 0) acc -= w * v;
}

template <class R>
__host__ __device__ constexpr bool exact_arith() { return std::is_same<R, double>::value; }
// blocks per SM the register budget is sized for: FP32 80 registers a thread, FP32
// duals 128 (at 255 they held one block, 8 warps, per SM), FP64 unconstrained
template <class R, int BY = 8>
__host__ __device__ constexpr int fused_min_blocks() {
    // tiles of other heights (batches only): the same ~80 registers a thread for 32 x 4
    // (six blocks); 32 x 16 holds one block by its shared memory
    if constexpr (std::is_same<R, float>::value) return BY == 4 ? 7 : (BY == 16 ? 1 : 3);
    return f32_family<R>::value ? 2 : 1;
}

// A parameter as an R: the FP32 build reads its single-precision copy.
template <class R>
__device__ __forceinline__ R pv(double v, float vf) {
    if constexpr (std::is_same<R, float>::value) return vf;
    else return R(v);
}

// A model parameter as an R: plain builds take the value; dual builds also carry
// its seeded tangents (one per differentiated parameter direction).
template <class R>
__device__ __forceinline__ R prm(double v, const double* t, float vf = 0.f) {
    if constexpr (std::is_same<R, float>::value) {
        return vf;
    } else if constexpr (is_dual<R>::value) {
        R r(v);
#pragma unroll
        for (int k = 0; k < (int)(sizeof(r.d) / sizeof(r.d[0])); ++k) r.d[k] = decltype(r.v)(t[k]);
        return r;
    } else {
        return R(v);
    }
}

// Divisions.  The FP64 build divides exactly where a plain C evaluation of the
// same formula divides (it is compared with the oracle to 1e-12 after thousands of
// steps); the FP32 builds multiply by a reciprocal formed once per thread, which
// removes most of their instruction count.
template <class R>
__device__ __forceinline__ R dv(R a, R b, R inv_b) {
    if constexpr (exact_arith<R>()) return a / b;
    else return a * inv_b;
}
template <class R>
__device__ __forceinline__ R rcp(R b) {
    if constexpr (std::is_same<R, float>::value) return __fdividef(1.0f, b);  // approximate, ~2 ulp
    else return R(1) / b;
}
// A launch-wide constant: the FP32 build reads the host-formed copy, the others
// evaluate the expression (exactly, in the FP64 build)
template <class R, class F>
__device__ __forceinline__ R kconst(float host_value, F expr) {
    if constexpr (std::is_same<R, float>::value) return host_value;
    else return expr();
}
template <class R>
__device__ __forceinline__ R oc2(R a) {  // a / cs^2
    if constexpr (exact_arith<R>()) return a / cs2<R>();
    else return a * R(3);
}

// ---------------------------------------------------------------- storage conversion
// Storage types.  With fp32 or fp16 storage the rest population f^i_0 of each
// phase set (close to phi_i, an O(1) number) is stored as its deviation from the
// phi_i of the step that wrote it -- the "anchor", held in the phi field until the
// next moments pass reads it -- and its collision is carried out in deviation form,
// so no O(1) terms cancel: f_0 - f_0^eq = (1 - w_0) mu - sum_{j>0} f_j.  The
// deviation is O(mu), resolved to ~1e-10 (fp32) or ~1e-6 (fp16) absolute; every
// other plane is small already and stored as is.  The fp64 build stores plainly.
template <class S> struct Store;
template <> struct Store<double> {
    static __device__ __forceinline__ double ld(const double* p, size_t i) { return p[i]; }
    static __device__ __forceinline__ void st(double* p, size_t i, double v) { p[i] = v; }
};
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p, size_t i) { return p[i]; }
    static __device__ __forceinline__ void st(float* p, size_t i, float v) { p[i] = v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p, size_t i) { return __half2float(p[i]); }
    static __device__ __forceinline__ void st(__half* p, size_t i, float v) { p[i] = __float2half_rn(v); }
};
// BF16: the FP32 exponent range (no subnormals at the small magnitudes of the flow
// and charge populations), 8 significant bits
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, size_t i, float v) { p[i] = __float2bfloat16_rn(v); }
};
template <class T, int M> struct Store<Dual<T, M>> {
    static __device__ __forceinline__ Dual<T, M> ld(const Dual<T, M>* p, size_t i) { return p[i]; }
    static __device__ __forceinline__ void st(Dual<T, M>* p, size_t i, Dual<T, M> v) { p[i] = v; }
};
template <class S>
__host__ __device__ constexpr bool anchored() {
    return std::is_same<S, float>::value || std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
}

// ---------------------------------------------------------------- grid helpers
// periodic index for a in [-n, 2n) (one lattice link from a cell), without branches
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
__device__ __forceinline__ int wrapi(int a, int n) {
    if (a < 0) a += n;
    else if (a >= n) a -= n;
    if ((unsigned)a >= (unsigned)n) {  // only on grids smaller than the offset
        a %= n;
        if (a < 0) a += n;
    }
    return a;
}
// stencil ghost rows: periodic, or mirror about the half-way wall
__device__ __forceinline__ int ghost_row(int y, int ny, int bc_y) {
    if (bc_y == 0) return wrapi(y, ny);
    if (y < 0) return -1 - y;
    if (y >= ny) return 2 * ny - 1 - y;
    return y;
}
// the same, clamped into the grid: tile loaders may touch rows beyond the ghost
// ring on small or ragged grids, whose values are never used
__device__ __forceinline__ int tile_row(int y, int ny, int bc_y) {
    const int r = ghost_row(y, ny, bc_y);
    return r < 0 ? 0 : (r >= ny ? ny - 1 : r);
}

// Eq. 30
template <class R>
__device__ __forceinline__ R perm(const DevParams& P, R p0, R p1, R p2) {
    R e = R(0);
    e += prm<R>(P.eps[0], P.t_eps[0], P.feps[0]) * p0 * p0 * (R(3) - R(2) * p0);
    e += prm<R>(P.eps[1], P.t_eps[1], P.feps[1]) * p1 * p1 * (R(3) - R(2) * p1);
    e += prm<R>(P.eps[2], P.t_eps[2], P.feps[2]) * p2 * p2 * (R(3) - R(2) * p2);
    return e;
}
template <class R>
__device__ __forceinline__ R cond(const DevParams& P, R p0, R p1, R p2) {
    return p0 * pv<R>(P.sigma[0], P.fsig[0]) + p1 * pv<R>(P.sigma[1], P.fsig[1]) + p2 * pv<R>(P.sigma[2], P.fsig[2]);
}
template <class R>
__device__ __forceinline__ R dens(const DevParams& P, R p0, R p1, R p2) {
    return p0 * pv<R>(P.rho[0], P.frho[0]) + p1 * pv<R>(P.rho[1], P.frho[1]) + p2 * pv<R>(P.rho[2], P.frho[2]);
}
// Eq. 40
template <class R>
__device__ __forceinline__ R s_eq(int j, R ux, R uy) {
    R cu = R(cx(j)) * ux + R(cy(j)) * uy;
    R uu = ux * ux + uy * uy;
    if constexpr (exact_arith<R>())
        return wgt<R>(j) * (cu / cs2<R>() + cu * cu / (R(2) * cs2<R>() * cs2<R>()) - uu / (R(2) * cs2<R>()));
    else
        return wgt<R>(j) * (cu * R(3) + cu * cu * R(4.5) - uu * R(1.5));
}

// ---------------------------------------------------------------- block reduction (FP64)
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* out) {
    __shared__ double red[32][NV];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = lane < nwarps ? red[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) out[k] = a;
        }
    }
}

// The same for values of type R: FP32 values are summed within a warp in FP32
// (a residual needs a few digits; FP64 shuffles and adds cost far more on this
// part), the warp sums across the block and the grid in FP64.  Other types are
// converted to FP64 first.
template <int NV, class R>
__device__ __forceinline__ void block_reduce_store_r(R (&v)[NV], double* out) {
    if constexpr (std::is_same<R, float>::value) {
        __shared__ double red[32][NV];
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        const int lane = tid & 31, warp = tid >> 5;
        const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k)
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[warp][k] = (double)v[k];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double a = lane < nwarps ? red[lane][k] : 0.0;
                for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
                if (lane == 0) out[k] = a;
            }
        }
    } else {
        double d[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) d[k] = (double)v[k];
        block_reduce_store<NV>(d, out);
    }
}

// ---------------------------------------------------------------- S1: moments
template <class R, class S>
__device__ __forceinline__ void body_moments(const DevParams P, const S* __restrict__ pop, const R* phi_anchor,
                                                 R* phi, R* __restrict__ qt, int bx, int by, int gdx) {
    const int x = bx * blockDim.x + threadIdx.x, y = by * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R a = R(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) a += Store<S>::ld(pop, (9 * (i + 1) + j) * N + c);
        if (anchored<S>()) a = phi_anchor[i * N + c] + a;  // anchor + (deviation + moving populations)
        phi[i * N + c] = a;  // may alias phi_anchor: read above, written here
    }
    R a = R(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) a += Store<S>::ld(pop, (36 + j) * N + c);
    qt[c] = a;
}
template <class R, class S>
__global__ void __launch_bounds__(256) k_moments(DevParams P, const S* __restrict__ pop, const R* phi_anchor,
                                                 R* phi, R* __restrict__ qt) {
    body_moments<R, S>(P, pop, phi_anchor, phi, qt, blockIdx.x, blockIdx.y, gridDim.x);
}

// ---------------------------------------------------------------- S2-S4: properties, stencils, charge
// the Eq. 33 gradients of eps and sigma at this thread's cell from a staged tile of
// pitch SX (the cell at row srow, column threadIdx.x + 1 of the tile), then eps and,
// with use_qt, the closed-form charge from q~ = qt and E of the previous step
template <class R, int SX>
__device__ __forceinline__ void prologue_cell(const DevParams& P, const R* se_, const R* ss_, R qt,
                                              const R* __restrict__ E, R* __restrict__ q, R* __restrict__ eps_out,
                                              int use_qt, unsigned c, int srow) {
    const unsigned N = P.N;
    const int sc = srow * SX + threadIdx.x + 1;
    R gex = R(0), gey = R(0), gsx = R(0), gsy = R(0), e0 = R(0), s0 = R(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const R e = se_[sc + cy(j) * SX + cx(j)], s = ss_[sc + cy(j) * SX + cx(j)];
        gex += wgt<R>(j) * R(cx(j)) * e;
        gey += wgt<R>(j) * R(cy(j)) * e;
        gsx += wgt<R>(j) * R(cx(j)) * s;
        gsy += wgt<R>(j) * R(cy(j)) * s;
        if (j == 0) { e0 = e; s0 = s; }
    }
    gex = oc2(gex); gey = oc2(gey); gsx = oc2(gsx); gsy = oc2(gsy);
    eps_out[c] = e0;
    if (!use_qt) return;
    const R r = dv(s0, e0, rcp(e0));
    const R Ex = E[c], Ey = E[N + c];
    const R src = r * (gex * Ex + gey * Ey) - (gsx * Ex + gsy * Ey);
    const R den = R(1) + R(0.5) * r;
    q[c] = dv(qt + R(0.5) * src, den, rcp(den));
}
// eps and sigma (Eq. 29-30) of the block's 32 x 8 tile and its one-cell ring are
// formed once per cell into shared memory (ghost rows mirrored at walls, as the
// stencil expects); each thread then takes the Eq. 33 gradients from there (the
// same sums, in the same order, as a per-neighbour evaluation) and writes eps and
// the closed-form charge q = [q~ + (sigma/eps grad eps . E - grad sigma . E)/2] /
// (1 + sigma/(2 eps)), with E of the previous step.
template <class R>
__device__ __forceinline__ void body_prologue(const DevParams P, const R* __restrict__ phi, const R* __restrict__ qt,
                                                  const R* __restrict__ E, R* __restrict__ q, R* __restrict__ eps_out,
                                                  int use_qt, int bx, int by, int gdx) {
    constexpr int SX = 34, SY = 10;  // blockDim (32, 8) and a one-cell ring
    __shared__ R se_[SY * SX], ss_[SY * SX];
    const int x0 = bx * blockDim.x, y0 = by * blockDim.y;
    const unsigned N = P.N;
    for (int k = threadIdx.x + blockDim.x * threadIdx.y; k < SX * SY; k += blockDim.x * blockDim.y) {
        const int ly = k / SX, lx = k - ly * SX;
        const unsigned n = (unsigned)tile_row(y0 + ly - 1, P.ny, P.bc_y) * P.nx + wrapi(x0 + lx - 1, P.nx);
        const R p0 = phi[n], p1 = phi[N + n], p2 = phi[2 * N + n];
        se_[k] = perm<R>(P, p0, p1, p2);
        ss_[k] = cond<R>(P, p0, p1, p2);
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned c = (unsigned)y * P.nx + x;
    prologue_cell<R, SX>(P, se_, ss_, use_qt ? qt[c] : R(0), E, q, eps_out, use_qt, c, threadIdx.y + 1);
}
template <class R>
__global__ void __launch_bounds__(256) k_prologue(DevParams P, const R* __restrict__ phi, const R* __restrict__ qt,
                                                  const R* __restrict__ E, R* __restrict__ q, R* __restrict__ eps_out,
                                                  int use_qt) {
    body_prologue<R>(P, phi, qt, E, q, eps_out, use_qt, blockIdx.x, blockIdx.y, gridDim.x);
}

// S1-S4 in one pass: the block forms phi of its 32 x 8 tile and one-cell ring from
// the phase populations (ring rows mirrored at walls, as the stencil expects; the
// ring's moments are formed again by the neighbouring blocks), writes phi of its own
// cells, stages eps and sigma, sums q~ from the charge populations and closes the
// charge as the prologue does.  With the rest population stored as a deviation
// (anchored storage) phi = the previous phi (phi_old) + the sum; phi_old and phi
// are different sets of planes, since neighbouring blocks read phi_old on their
// rings.  The sums run in the order of the separate passes, so the results are the
// same bit for bit; what is saved is the q~ plane and the prologue's re-read of phi.
template <class R, class S>
__device__ __forceinline__ void body_moments_closure(const DevParams P, const S* __restrict__ pop,
                                                     const R* __restrict__ phi_old, R* __restrict__ phi,
                                                     const R* __restrict__ E, R* __restrict__ q,
                                                     R* __restrict__ eps_out, int use_qt, int bx, int by) {
    constexpr int MC_Y = 8, SX = 34, SY = MC_Y + 2;  // blockDim (32, 8), one-cell ring
    __shared__ R se_[SY * SX], ss_[SY * SX];
    const int x0 = bx * blockDim.x, y0 = by * MC_Y;
    const int nx = P.nx, ny = P.ny;
    const unsigned N = P.N;
    for (int k = threadIdx.x + blockDim.x * threadIdx.y; k < SX * SY; k += blockDim.x * blockDim.y) {
        const int ly = k / SX, lx = k - ly * SX;
        const unsigned n = (unsigned)tile_row(y0 + ly - 1, ny, P.bc_y) * nx + wrapi(x0 + lx - 1, nx);
        R p[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R a = R(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) a += Store<S>::ld(pop, (9 * (i + 1) + j) * N + n);
            if (anchored<S>()) a = phi_old[i * N + n] + a;  // anchor + (deviation + moving populations)
            p[i] = a;
        }
        se_[k] = perm<R>(P, p[0], p[1], p[2]);
        ss_[k] = cond<R>(P, p[0], p[1], p[2]);
        if (lx >= 1 && lx <= 32 && ly >= 1 && ly <= MC_Y && x0 + lx - 1 < nx && y0 + ly - 1 < ny) {
#pragma unroll
            for (int i = 0; i < 3; ++i) phi[i * N + n] = p[i];  // an own cell (row in the domain)
        }
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= nx) return;
#pragma unroll
    for (int r = 0; r < MC_Y; r += 8) {
        const int y = y0 + threadIdx.y + r;
        if (y >= ny) return;
        const unsigned c = (unsigned)y * nx + x;
        R qt = R(0);
        if (use_qt) {
#pragma unroll
            for (int j = 0; j < 9; ++j) qt += Store<S>::ld(pop, (36 + j) * N + c);
        }
        prologue_cell<R, SX>(P, se_, ss_, qt, E, q, eps_out, use_qt, c, threadIdx.y + r + 1);
    }
}
// the merged pass covers 32 x 8 cells a block (32 x 16 measured no faster)
__host__ __device__ constexpr int moments_closure_rows() { return 8; }
template <class R, class S>
__global__ void __launch_bounds__(256) k_moments_closure(DevParams P, const S* __restrict__ pop,
                                                         const R* __restrict__ phi_old, R* __restrict__ phi,
                                                         const R* __restrict__ E, R* __restrict__ q,
                                                         R* __restrict__ eps_out, int use_qt) {
    body_moments_closure<R, S>(P, pop, phi_old, phi, E, q, eps_out, use_qt, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- S5: potential iteration (Eq. 43-45)
// Post-collision h_j of one cell (Eq. 43) with heq_0 = (w_0 - 1) psi, heq_j = w_j psi,
// source varpi_j q (varpi_0 = 0, varpi_j = 1/8) and grad psi = -J / den,
// den = eps_hat + cs2 tau_h.  The FP64 and dual builds evaluate Eq. 43 as written;
// the FP32 builds (plain and dual) use the equal factored form
//   h_j* = (1 - 1/tau_h) h_j + w_j (psi/tau_h + Kc c_j.J) + q/8,
//   h_0* = (1 - 1/tau_h) h_0 + (w_0 - 1) psi/tau_h,   Kc = 3 eps_hat / (tau_h den),
// which takes a third of the instructions.
template <class R>
__device__ __forceinline__ R h_collide(int j, R hj, R ps, R gx, R gy, R jx, R jy, R th, R ith, R epshat, R Kc, R qc,
                                       R q8) {
    if constexpr (f32_family<R>::value) {
        const R A = ith * ps, om = R(1) - ith;
        if (j == 0) return fmaf_(om, hj, (wgt<R>(0) - R(1)) * A);
        return fmaf_(om, hj, fmaf_(wgt<R>(j), fmaf_(Kc, cdot<R>(j, jx, jy), A), q8));
    } else {
        const R heq = (j == 0) ? (wgt<R>(0) - R(1)) * ps : wgt<R>(j) * ps;
        const R varpi = (j == 0) ? R(0) : R(1.0 / 8.0);
        const R cg = cdot<R>(j, gx, gy);
        return hj - dv(hj - heq, th, ith) - dv(oc2(epshat) * wgt<R>(j) * cg, th, ith) + varpi * qc;
    }
}

// The FP32 build's collision of Eq. 43, one sequence of explicitly rounded
// operations shared by the per-iteration and blocked kernels, so that the two
// produce bitwise-equal iterates.  The factored form
//   h_j* = (1 - 1/tau_h) h_j + w_j (psi/tau_h + Kc c_j.J) + q/8
// (h_0* without the source and Kc term) is evaluated from S = sum_{j>0} h_j (psi =
// 1.8 S) as  h_j* = om h_j + (cw_j S + q/8) + (w_j Kc) c_j.J, with the direction
// sums paired so that J costs 8 operations and each population 2.
template <class V> struct F32Ops;
template <> struct F32Ops<float> {
    static __device__ __forceinline__ float splat(float a) { return a; }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
};
// launch-wide constants of the FP32 collision: 1 - 1/tau_h and the equilibrium
// weights times 1.8/tau_h (w_0 - 1, w_1, w_5)
struct PoissonF32 {
    float om, cw0, cw1, cw5;
};
__device__ __forceinline__ PoissonF32 poisson_f32(const DevParams& P) {
    const float a = P.fitau_h * 1.8f;
    return {1.0f - P.fitau_h, (wgt<float>(0) - 1.0f) * a, wgt<float>(1) * a, wgt<float>(5) * a};
}
// w_1 Kc = w_1 3 eps_hat / (tau_h den) of a cell (w_5 Kc = w_1 Kc / 4 exactly)
__device__ __forceinline__ float poisson_k1(const DevParams& P, float eps_c) {
    const float eh = eps_c - P.feps_ref;
    return wgt<float>(1) * (3.0f * P.fitau_h * eh * rcp(eh + cs2<float>() * P.ftau_h));
}
// S = sum_{j>0} h_j and J = sum_j c_j h_j
template <class V>
__device__ __forceinline__ void moments_f32(const V (&h)[9], V& S, V& jx, V& jy) {
    using O = F32Ops<V>;
    const V a = O::sub(h[1], h[3]), b = O::sub(h[5], h[7]), c = O::sub(h[8], h[6]), d = O::sub(h[2], h[4]);
    S = O::add(O::add(O::add(h[1], h[3]), O::add(h[2], h[4])), O::add(O::add(h[5], h[7]), O::add(h[6], h[8])));
    jx = O::add(O::add(a, b), c);
    jy = O::sub(O::add(d, b), c);
}
// post-collision values v[0..8] from h, S, J, w_1 Kc and (with Q) q/8
template <class V, bool Q>
__device__ __forceinline__ void collide_f32(const V (&h)[9], V S, V jx, V jy, V K1, V q8, const PoissonF32& C,
                                            V (&v)[9]) {
    using O = F32Ops<V>;
    const V om = O::splat(C.om);
    const V W0 = O::mul(O::splat(C.cw0), S);
    const V W1 = Q ? O::fma(O::splat(C.cw1), S, q8) : O::mul(O::splat(C.cw1), S);
    const V W5 = Q ? O::fma(O::splat(C.cw5), S, q8) : O::mul(O::splat(C.cw5), S);
    const V K5 = O::mul(K1, O::splat(0.25f));
    const V sp = O::add(jx, jy), sm = O::sub(jx, jy);  // c.J of directions 5 (+) and 8 (-)
    v[0] = O::fma(om, h[0], W0);
    v[1] = O::fma(om, h[1], O::fma(K1, jx, W1));
    v[3] = O::fma(om, h[3], O::fma(O::neg(K1), jx, W1));
    v[2] = O::fma(om, h[2], O::fma(K1, jy, W1));
    v[4] = O::fma(om, h[4], O::fma(O::neg(K1), jy, W1));
    v[5] = O::fma(om, h[5], O::fma(K5, sp, W5));
    v[7] = O::fma(om, h[7], O::fma(O::neg(K5), sp, W5));
    v[8] = O::fma(om, h[8], O::fma(K5, sm, W5));
    v[6] = O::fma(om, h[6], O::fma(O::neg(K5), sm, W5));
}

// One pseudo-time collide + push-stream of h.  On iterations before a check it
// saves psi and J = sum c_j h_j; on a check it accumulates (FP64, per block)
// |d psi|^2, |psi|^2, |d J|^2, |J|^2.
// RS (the correction to an FP64 anchor, lb3e_anchor.cuh): no charge source,
// electrodes at zero, and the anchor's increment rres (post-streaming layout)
// added where each population arrives.
template <class R, bool RS = false>
__device__ __forceinline__ void body_poisson(const DevParams P, const R* __restrict__ hin, R* __restrict__ hout,
                                                 const R* __restrict__ eps, const R* __restrict__ q,
                                                 R* __restrict__ prev, double* __restrict__ partial,
                                                 int save_prev, int check, int bx, int by, int gdx,
                                                 const R* __restrict__ rres = nullptr) {
    const int x = bx * blockDim.x + threadIdx.x, y = by * blockDim.y + threadIdx.y;
    const bool in = x < P.nx && y < P.ny;
    const unsigned N = P.N, c = in ? (unsigned)y * P.nx + x : 0;
    R acc[4] = {R(0), R(0), R(0), R(0)};
    if constexpr (std::is_same<R, float>::value) {
        if (in) {
            float hj[9], S, jx, jy, v[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) hj[j] = hin[j * N + c];
            moments_f32<float>(hj, S, jx, jy);
            const float ps = S * 1.8f;
            if (check) {
                const float d = ps - prev[c], ex = jx - prev[N + c], ey = jy - prev[2 * N + c];
                acc[0] = d * d;
                acc[1] = ps * ps;
                acc[2] = ex * ex + ey * ey;
                acc[3] = jx * jx + jy * jy;
            }
            if (save_prev) { prev[c] = ps; prev[N + c] = jx; prev[2 * N + c] = jy; }
            const PoissonF32 C = poisson_f32(P);
            collide_f32<float, !RS>(hj, S, jx, jy, poisson_k1(P, eps[c]), RS ? 0.f : 0.125f * q[c], C, v);
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int yt = y + cy(j);
                if (P.bc_y != 0 && (yt < 0 || yt >= P.ny)) {
                    float out = v[j];
                    if (P.bc_y == 2) out = RS ? -v[j] : __fmaf_rn(2.0f * wgt<float>(j), yt >= P.ny ? P.fVt : P.fVb, -v[j]);
                    const unsigned to = opp(j) * N + c;
                    hout[to] = RS ? __fadd_rn(out, rres[to]) : out;
                } else {
                    const unsigned to = j * N + (unsigned)wrapi(yt, P.ny) * P.nx + wrapi(x + cx(j), P.nx);
                    hout[to] = RS ? __fadd_rn(v[j], rres[to]) : v[j];
                }
            }
        }
    } else if (in) {
        R hj[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) hj[j] = hin[j * N + c];
        R ps = R(0), jx = R(0), jy = R(0);
#pragma unroll
        for (int j = 1; j < 9; ++j) ps += hj[j];
        ps = dv(ps, R(1) - wgt<R>(0), R(1.8));
#pragma unroll
        for (int j = 0; j < 9; ++j) { cacc(jx, cx(j), hj[j]); cacc(jy, cy(j), hj[j]); }
        if (check) {
            const R d = ps - prev[c], ex = jx - prev[N + c], ey = jy - prev[2 * N + c];
            acc[0] = d * d;
            acc[1] = ps * ps;
            acc[2] = ex * ex + ey * ey;
            acc[3] = jx * jx + jy * jy;
        }
        if (save_prev) { prev[c] = ps; prev[N + c] = jx; prev[2 * N + c] = jy; }
        const R th = pv<R>(P.tau_h, P.ftau_h), ith = kconst<R>(P.fitau_h, [&] { return rcp(th); });
        const R epshat = eps[c] - pv<R>(P.eps_ref, P.feps_ref);
        const R den = epshat + cs2<R>() * th, iden = rcp(den);
        const R gx = dv(-jx, den, iden), gy = dv(-jy, den, iden);
        const R qc = RS ? R(0) : q[c];
        const R Kc = R(3) * ith * epshat * iden;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const R v = h_collide<R>(j, hj[j], ps, gx, gy, jx, jy, th, ith, epshat, Kc, qc, R(0.125) * qc);
            const int yt = y + cy(j);
            if (P.bc_y != 0 && (yt < 0 || yt >= P.ny)) {
                R out = v;
                if (P.bc_y == 2) {
                    if constexpr (RS) out = -v;
                    else
                        out = -v + R(2) * wgt<R>(j) * (yt >= P.ny ? prm<R>(P.V_top, P.t_Vt, P.fVt)
                                                                  : prm<R>(P.V_bottom, P.t_Vb, P.fVb));
                }
                const unsigned to = opp(j) * N + c;
                if constexpr (RS) out = out + rres[to];
                hout[to] = out;
            } else {
                const unsigned to = j * N + (unsigned)wrapi(yt, P.ny) * P.nx + wrapi(x + cx(j), P.nx);
                if constexpr (RS) hout[to] = v + rres[to];
                else hout[to] = v;
            }
        }
    }
    if (check) {
        const int b = bx + gdx * by;
        block_reduce_store_r<4>(acc, partial + 4 * (size_t)b);
    }
}
template <class R>
__global__ void __launch_bounds__(256) k_poisson(DevParams P, const R* __restrict__ hin, R* __restrict__ hout,
                                                 const R* __restrict__ eps, const R* __restrict__ q,
                                                 R* __restrict__ prev, double* __restrict__ partial,
                                                 int save_prev, int check) {
    body_poisson<R>(P, hin, hout, eps, q, prev, partial, save_prev, check, blockIdx.x, blockIdx.y, gridDim.x);
}
// one iteration on the correction to an FP64 anchor (no residual sums; save_prev:
// psi and J before the collision into prev)
template <class R>
__global__ void __launch_bounds__(256) k_poisson_rs(DevParams P, const R* __restrict__ hin, R* __restrict__ hout,
                                                    const R* __restrict__ eps, const R* __restrict__ rres,
                                                    R* __restrict__ prev, int save_prev) {
    body_poisson<R, true>(P, hin, hout, eps, nullptr, prev, nullptr, save_prev, 0, blockIdx.x, blockIdx.y,
                          gridDim.x, rres);
}

// ---------------------------------------------------------------- S5 on tiles, one thread a cell
// Up to PT_H pseudo-iterations per launch on a tile of PT_TX x PT_TY cells held in
// shared memory with a halo of PT_H cells, one thread per tile cell: each iteration
// collides every cell into a post-collision buffer, then each cell pulls its
// incoming populations (at a wall, its own reflected ones).  After t iterations the
// values within t cells of the tile's edge are stale, so the interior is exact after
// PT_H.  Used where a value is too wide for the register tiles of k_poisson_tb (the
// dual numbers of the tangent builds) and by the reverse mode.
// The tile geometry: TY rows of PT_TX cells with an H-cell halo.
template <int TY, int H>
struct PTGeom {
    static constexpr int TX = 32, W = TX + 2 * H, HT = TY + 2 * H, NT = W * HT;
};
// the reverse mode's tiles: 32 x 8 with a 4-cell halo (640 threads)
constexpr int PT_TX = 32, PT_TY = 8, PT_H = 4, PT_W = PT_TX + 2 * PT_H, PT_HT = PT_TY + 2 * PT_H;
constexpr int PT_NT = PT_W * PT_HT;
template <class R>
constexpr size_t pt_smem_bytes() { return 2 * 9 * PT_NT * sizeof(R); }
// the tangent builds' tiles: the same 32 x 8 with a 4-cell halo (dual numbers take 16
// bytes a value: two sets of 9 planes fill 184 KB; a 2-cell halo on 32 x 16 tiles,
// 8 launches a step instead of 4, measured slower)
using PTTangent = PTGeom<8, 4>;

struct TileCell {
    int t, c;          // tile index, lattice index (0 where absent)
    bool present;      // the lattice has this cell (not beyond a wall)
    bool interior;     // this launch's tile owns it (writes it back)
    int gy;            // lattice row
};
template <class G>
__device__ __forceinline__ TileCell tile_cell_g(const DevParams& P, int H) {
    TileCell r;
    const int tx = threadIdx.x, ty = threadIdx.y;
    r.t = ty * G::W + tx;
    const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * (G::HT - 2 * H);
    int gx = x0 - H + tx, gy = y0 - H + ty;
    gx = ((gx % P.nx) + P.nx) % P.nx;
    r.present = true;
    if (P.bc_y == 0) gy = ((gy % P.ny) + P.ny) % P.ny;
    else r.present = gy >= 0 && gy < P.ny;
    r.gy = gy;
    r.c = r.present ? gy * P.nx + gx : 0;
    r.interior = r.present && tx >= H && tx < H + G::TX && ty >= H && ty < G::HT - H && x0 + tx - H < P.nx &&
                 y0 + ty - H < P.ny;
    return r;
}
__device__ __forceinline__ TileCell tile_cell(const DevParams& P) { return tile_cell_g<PTGeom<PT_TY, PT_H>>(P, PT_H); }
// tile index of the neighbour at (dx, dy), clamped into the tile (a clamped read only
// happens in the stale rim)
template <class G>
__device__ __forceinline__ int tile_nb_g(int dx, int dy) {
    const int tx = min(max((int)threadIdx.x + dx, 0), G::W - 1);
    const int ty = min(max((int)threadIdx.y + dy, 0), G::HT - 1);
    return ty * G::W + tx;
}
__device__ __forceinline__ int tile_nb(int dx, int dy) { return tile_nb_g<PTGeom<PT_TY, PT_H>>(dx, dy); }

// nit (<= 4) iterations of Eq. 43 with the arithmetic of body_poisson (fixed counts:
// no residual sums), on the tangent builds' tiles
template <class R>
__global__ void __launch_bounds__(PTTangent::NT) k_poisson_tile(DevParams P, const R* __restrict__ hin,
                                                                R* __restrict__ hout, const R* __restrict__ eps,
                                                                const R* __restrict__ q, int nit) {
    using G = PTTangent;
    extern __shared__ __align__(16) unsigned char ptl_raw[];
    R* cur = reinterpret_cast<R*>(ptl_raw);
    R* post = cur + 9 * G::NT;
    const TileCell tc = tile_cell_g<G>(P, 4);
    const int N = P.N, ny = P.ny;
    const R th = pv<R>(P.tau_h, P.ftau_h), ith = kconst<R>(P.fitau_h, [&] { return rcp(th); });
    R epshat = R(0), den = R(1), iden = R(1), qc = R(0);
    if (tc.present) {
        epshat = eps[tc.c] - pv<R>(P.eps_ref, P.feps_ref);
        den = epshat + cs2<R>() * th;
        iden = rcp(den);
        qc = q[tc.c];
#pragma unroll
        for (int j = 0; j < 9; ++j) cur[j * G::NT + tc.t] = hin[(size_t)j * N + tc.c];
    }
    const R Kc = R(3) * ith * epshat * iden;
    for (int it = 0; it < nit; ++it) {
        __syncthreads();
        if (tc.present) {
            R hj[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) hj[j] = cur[j * G::NT + tc.t];
            R ps = R(0), jx = R(0), jy = R(0);
#pragma unroll
            for (int j = 1; j < 9; ++j) ps += hj[j];
            ps = dv(ps, R(1) - wgt<R>(0), R(1.8));
#pragma unroll
            for (int j = 0; j < 9; ++j) { cacc(jx, cx(j), hj[j]); cacc(jy, cy(j), hj[j]); }
            const R gx = dv(-jx, den, iden), gy = dv(-jy, den, iden);
#pragma unroll
            for (int j = 0; j < 9; ++j)
                post[j * G::NT + tc.t] = h_collide<R>(j, hj[j], ps, gx, gy, jx, jy, th, ith, epshat, Kc, qc,
                                                      R(0.125) * qc);
        }
        __syncthreads();
        if (tc.present) {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int ys = tc.gy - cy(j);
                R v;
                if (P.bc_y != 0 && (ys < 0 || ys >= ny)) {
                    const R o = post[opp(j) * G::NT + tc.t];
                    if (P.bc_y == 2)
                        v = -o + R(2) * wgt<R>(j) * (ys >= ny ? prm<R>(P.V_top, P.t_Vt, P.fVt)
                                                              : prm<R>(P.V_bottom, P.t_Vb, P.fVb));
                    else
                        v = o;
                } else {
                    v = post[j * G::NT + tile_nb_g<G>(-cx(j), -cy(j))];
                }
                cur[j * G::NT + tc.t] = v;
            }
        }
    }
    if (tc.interior)
#pragma unroll
        for (int j = 0; j < 9; ++j) hout[(size_t)j * N + tc.c] = cur[j * G::NT + tc.t];
}

// ---------------------------------------------------------------- S5, temporally blocked
// K (<= H) pseudo-iterations of Eq. 43 per launch.  A block loads the h
// populations of its PB_TX x PB_TY tile plus an H-cell halo into registers (three
// cells per thread), and per-cell constants into shared memory.  Each iteration
// collides in registers, writes the post-collision values to shared memory, and
// pulls each cell's incoming populations back.  Cells at an electrode (or no-slip)
// wall also write their reflected populations into the ghost row beyond the wall,
// so the pull reads one slot per direction with no wall cases.  A cell at distance d
// outside the tile collides at iteration t only while d <= K - t and pulls while
// d <= K - 1 - t, so after K iterations the tile is exact and is written out.  The
// arithmetic per cell is that of body_poisson.  Residual partials (check) are taken
// before the first collision, the residual state (save_prev) before the last one.
constexpr int PB_TX = 32, PB_TY = 16, PB_HALO = 8;
// CPT cells per thread: 3 for the plain kernel, 2 on the correction to an FP64
// anchor (RS), whose anchor increments then fit in registers (9 per cell) at about
// the same number of resident threads.
template <int H, int CPT_>
struct PBGeom {
    static constexpr int RX = PB_TX + 2 * H, RY = PB_TY + 2 * H, CELLS = RX * RY;
    static constexpr int CPT = CPT_, THREADS = CELLS / CPT;
    static_assert(CELLS % CPT == 0, "region cells split evenly over the threads");
};
template <class R, bool RS = false>
__host__ __device__ constexpr int pb_cpt() { return RS ? 2 : 3; }
// FP32 post-collision plane sets (two: double-buffered, one barrier an iteration)
template <class R, bool RS = false>
__host__ __device__ constexpr int pb_sets() { return RS ? 2 : 1; }
template <class R, int H, bool RS = false>
__host__ __device__ constexpr int pb_threads() { return PBGeom<H, pb_cpt<R, RS>()>::THREADS; }
// blocks per SM the register budget is sized for (64 registers a thread in FP32)
template <class R, int H, bool RS = false>
__host__ __device__ constexpr int pb_min_blocks() {
    if constexpr (RS) return std::is_same<R, float>::value ? (H == 8 ? 1 : 2) : 1;
    return std::is_same<R, float>::value ? (H == 8 ? 2 : 3) : 1;
}
// shared planes.  FP32: one or two sets of 8 post-collision planes (directions
// 1-8), w_1 Kc and, unless RS, q/8.  FP64: 9 planes, eps and q
// (RS: no charge; the anchor's increments sit in registers).
template <class R, int H, bool RS = false>
constexpr size_t pb_smem_bytes() {
    constexpr int planes = std::is_same<R, float>::value ? 8 * pb_sets<R, RS>() + (RS ? 1 : 2) : (RS ? 10 : 11);
    return (size_t)planes * PBGeom<H, pb_cpt<R, RS>()>::CELLS * sizeof(R);
}
// halo depth of the region that serves a chunk of K iterations
__host__ __device__ constexpr int pb_halo_for(int K) { return K <= 2 ? 2 : (K <= 4 ? 4 : 8); }

// The FP32 blocked kernel.  Thread i owns the region cells i + m NT (m < CPT, NT =
// the region over CPT), so a warp's cells are consecutive in a region row and the
// thread's cells are independent instruction streams.  The collision is collide_f32, the
// per-iteration kernel's sequence of operations, so the two kernels produce
// bitwise-equal iterates.  Streaming moves only directions 1-8 through shared
// memory (the rest population stays in registers).  On the correction to the
// anchor (2 blocks an SM) two sets of planes alternate between iterations: an
// iteration's pulls read the set its collisions wrote, the next collisions write
// the other, so one barrier an iteration suffices.  The plain kernel (3 blocks an
// SM) keeps one set and two barriers: a second set would leave the SM's unified
// L1 too little room for the tile loads (measured slower).
// A cell collides while it is inside the dependency cone (d <= K - t) and pulls
// while its pull is still needed (d <= K - 1 - t); non-fluid rows (beyond a wall)
// neither collide nor store: their slots are the ghost slots the wall rows write.
template <int H, int KC, bool RS, bool INC = false>
__device__ __forceinline__ void body_poisson_tb_f32(const DevParams P, const float* __restrict__ hin,
                                                    float* __restrict__ hout, const float* __restrict__ eps,
                                                    const float* __restrict__ q, float* __restrict__ prev,
                                                    double* __restrict__ partial, int Kdyn, int save_prev,
                                                    int check, int bx, int by, int gdx,
                                                    const float* __restrict__ rres, float* __restrict__ rhs,
                                                    float* __restrict__ e0) {
    using G = PBGeom<H, pb_cpt<float, RS>()>;
    constexpr int RX = G::RX, CELLS = G::CELLS, CPT = G::CPT, NT = G::THREADS, SET = 8 * CELLS;
    constexpr int SETS = pb_sets<float, RS>();
    extern __shared__ __align__(16) unsigned char pb_raw[];
    float* hs = reinterpret_cast<float*>(pb_raw);  // [SETS][directions 1..8][CELLS]
    float* sk = hs + SETS * SET;                   // [CELLS] w_1 Kc
    float* sq = sk + CELLS;                        // [CELLS] q/8 (not RS)
    const int nx = P.nx, ny = P.ny;
    const unsigned N = P.N;
    const int x0 = bx * PB_TX - H, y0 = by * PB_TY - H;
    const int tid = threadIdx.x;
    const bool walls = P.bc_y != 0;

    // per owned cell k = tid + m NT, packed in one word: bits 0-7 the distance d
    // outside the tile (0 inside; 255: not a fluid cell), bit 8 bottom wall row, bit
    // 9 top wall row, bit 10 a tile cell inside the grid
    float h[CPT][9];
    float rr[RS ? CPT : 1][9];
    float pv[RS && INC ? CPT : 1][3];  // RS with INC: psi, J before the last collision
    int meta[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int k = tid + m * NT;
        const int ly = k / RX, lx = k % RX;
        const int gy = y0 + ly, gx = x0 + lx;
        const bool real = !walls || (gy >= 0 && gy < ny);
        const int dx = lx < H ? H - lx : (lx >= H + PB_TX ? lx - (H + PB_TX - 1) : 0);
        const int dy = ly < H ? H - ly : (ly >= H + PB_TY ? ly - (H + PB_TY - 1) : 0);
        const int d = dx > dy ? dx : dy;
        meta[m] = (real ? d : 255) | (walls && gy == 0 ? 256 : 0) | (walls && gy == ny - 1 ? 512 : 0) |
                  (real && d == 0 && gx < nx && gy < ny ? 1024 : 0);
        if (real) {
            const unsigned c = (unsigned)wrapi(gy, ny) * nx + wrapi(gx, nx);
#pragma unroll
            for (int j = 0; j < 9; ++j) h[m][j] = hin[j * N + c];
            sk[k] = poisson_k1(P, eps[c]);
            if constexpr (RS) {
#pragma unroll
                for (int j = 0; j < 9; ++j) rr[m][j] = rres[j * N + c];
            } else {
                sq[k] = 0.125f * q[c];
            }
        } else {
#pragma unroll
            for (int j = 0; j < 9; ++j) h[m][j] = 0.f;
            if constexpr (RS) {
#pragma unroll
                for (int j = 0; j < 9; ++j) rr[m][j] = 0.f;
            }
            sk[k] = 0.f;
            if constexpr (!RS) sq[k] = 0.f;
        }
    }
    auto cell = [&](int m) {
        const int k = tid + m * NT;
        return (unsigned)(y0 + k / RX) * nx + (unsigned)(x0 + k % RX);
    };
    const PoissonF32 C = poisson_f32(P);
    const bool electrodes = P.bc_y == 2;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int K = KC > 0 ? KC : Kdyn;
    constexpr int kUnroll = KC > 0 ? KC : 1;
    __syncthreads();  // sk, sq
#pragma unroll kUnroll
    for (int t = 0; t < K; ++t) {
        float* const hp = hs + (SETS == 2 ? (t & 1) * SET : 0) - CELLS;  // hp + j * CELLS: direction j
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            if ((meta[m] & 255) > K - t) continue;  // no longer feeds the tile (or not a fluid cell)
            const int k = tid + m * NT;
            float S, jx, jy, v[9];
            moments_f32<float>(h[m], S, jx, jy);
            if ((meta[m] & 1024) && ((check && t == 0) || (save_prev && t == K - 1))) {
                const unsigned c = cell(m);
                const float ps = S * 1.8f;
                if (check && t == 0) {
                    const float d = ps - prev[c], ex = jx - prev[N + c], ey = jy - prev[2 * N + c];
                    acc[0] += d * d;
                    acc[1] += ps * ps;
                    acc[2] += ex * ex + ey * ey;
                    acc[3] += jx * jx + jy * jy;
                }
                if (save_prev && t == K - 1) {
                    if constexpr (RS && INC) {  // kept for the check below
                        pv[m][0] = ps;
                        pv[m][1] = jx;
                        pv[m][2] = jy;
                    } else {
                        prev[c] = ps;
                        prev[N + c] = jx;
                        prev[2 * N + c] = jy;
                    }
                }
            }
            collide_f32<float, !RS>(h[m], S, jx, jy, sk[k], RS ? 0.f : sq[k], C, v);
            h[m][0] = RS ? __fadd_rn(v[0], rr[m][0]) : v[0];  // the rest population stays
#pragma unroll
            for (int j = 1; j < 9; ++j) hp[j * CELLS + k] = v[j];
            // a wall cell whose own pull is still needed (so it is not on the region
            // border, and its ghost slots lie inside the region): the populations
            // leaving toward the wall come back in the opposite direction, through
            // the ghost cell they would be pulled from (anti-bounce-back to the
            // electrode potential, or plain bounce-back)
            if ((meta[m] & 768) && (meta[m] & 255) <= K - 1 - t) {
                const bool top = meta[m] & 512;
                const float V = top ? P.fVt : P.fVb;
#pragma unroll
                for (int j = 1; j < 9; ++j) {
                    if (!((cy(j) < 0 && !top) || (cy(j) > 0 && top))) continue;
                    const int jo = opp(j);  // arriving direction
                    hp[jo * CELLS + k - cy(jo) * RX - cx(jo)] =
                        electrodes ? (RS ? -v[j] : __fmaf_rn(2.0f * wgt<float>(j), V, -v[j])) : v[j];
                }
            }
        }
        __syncthreads();
        // pull streaming inside the region (cells whose sources were all updated):
        // cell k takes direction j from k - cy RX - cx
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            if ((meta[m] & 255) > K - 1 - t) continue;
            const int k = tid + m * NT;
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                const float g = hp[j * CELLS + k - cy(j) * RX - cx(j)];
                h[m][j] = RS ? __fadd_rn(g, rr[m][j]) : g;
            }
        }
        if (SETS == 1 && t + 1 < K) __syncthreads();  // one set: the pulls end before the next stores
    }
    // write the tile
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        if (!(meta[m] & 1024)) continue;
        const unsigned c = cell(m);
#pragma unroll
        for (int j = 0; j < 9; ++j) hout[j * N + c] = h[m][j];
    }
    if (check) block_reduce_store_r<4>(acc, partial + 4 * (size_t)(bx + gdx * by));
    // RS, INC (with save_prev): the check of k_rs_increment on the tile, from
    // the final delta and psi, J before the last collision, all in registers (prev
    // is not written): per-block sums of |d psi|^2, |d J|^2, sum_j delta_j^2 and,
    // with rhs, the coarse correction's right-hand side and zero initial guess
    if constexpr (RS && INC) {
        {
            float ai[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int m = 0; m < CPT; ++m) {
                if (!(meta[m] & 1024)) continue;
                const unsigned c = cell(m);
                float S, jx, jy;
                moments_f32<float>(h[m], S, jx, jy);
#pragma unroll
                for (int j = 0; j < 9; ++j) ai[2] += h[m][j] * h[m][j];
                const float pp = pv[m][0];
                const float dp = S * 1.8f - pp, ex = jx - pv[m][1], ey = jy - pv[m][2];
                ai[0] += dp * dp;
                ai[1] += ex * ex + ey * ey;
                if (rhs) {
                    rhs[c] = S - (1.0f - wgt<float>(0)) * pp;
                    e0[c] = 0.f;
                }
            }
            block_reduce_store_r<3>(ai, partial + 3 * (size_t)(bx + gdx * by));
        }
    }
}

template <class R, int H, int KC = 0, bool RS = false, bool INC = false>
__device__ __forceinline__ void body_poisson_tb(const DevParams P, const R* __restrict__ hin,
                                                R* __restrict__ hout, const R* __restrict__ eps,
                                                const R* __restrict__ q, R* __restrict__ prev,
                                                double* __restrict__ partial, int Kdyn, int save_prev, int check,
                                                int bx, int by, int gdx, const R* __restrict__ rres = nullptr,
                                                float* __restrict__ rhs = nullptr, float* __restrict__ e0 = nullptr) {
    if constexpr (std::is_same<R, float>::value) {
        body_poisson_tb_f32<H, KC, RS, INC>(P, hin, hout, eps, q, prev, partial, Kdyn, save_prev, check, bx, by, gdx,
                                            rres, rhs, e0);
        return;
    }
    using G = PBGeom<H, pb_cpt<R, RS>()>;
    constexpr int RX = G::RX, CELLS = G::CELLS, CPT = G::CPT, NT = G::THREADS;
    extern __shared__ __align__(16) unsigned char pb_raw[];
    R* hs = reinterpret_cast<R*>(pb_raw);  // [9][CELLS] post-collision values
    // per cell, fixed over the iterations: eps and q, or, in the factored FP32
    // form, Kc = 3 eps_hat / (tau_h den) and q / 8
    constexpr bool kFact = std::is_same<R, float>::value;
    R* se = hs + 9 * CELLS;  // eps (Kc)
    R* sq = se + CELLS;      // q (q / 8); RS: not allocated
    const int nx = P.nx, ny = P.ny;
    const unsigned N = P.N;
    const int x0 = bx * PB_TX - H, y0 = by * PB_TY - H;
    const int tid = threadIdx.x;
    const bool walls = P.bc_y != 0;

    // per owned cell k = tid + m * NT, fixed over the iterations, packed in one word:
    // bits 0-7 the distance d outside the tile (0 inside; 255: not a fluid cell),
    // bit 8 bottom wall row, bit 9 top wall row, bit 10 a tile cell inside the grid
    R h[CPT][9];
    R rr[RS ? CPT : 1][9];  // RS: the anchor's increment at each owned cell, added after each pull
    int meta[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        const int k = tid + m * NT;
        const int ly = k / RX, lx = k % RX;
        const int gy = y0 + ly, gx = x0 + lx;
        const bool real = !walls || (gy >= 0 && gy < ny);
        const int dx = lx < H ? H - lx : (lx >= H + PB_TX ? lx - (H + PB_TX - 1) : 0);
        const int dy = ly < H ? H - ly : (ly >= H + PB_TY ? ly - (H + PB_TY - 1) : 0);
        const int d = dx > dy ? dx : dy;
        meta[m] = (real ? d : 255) | (walls && gy == 0 ? 256 : 0) | (walls && gy == ny - 1 ? 512 : 0) |
                  (real && d == 0 && gx < nx && gy < ny ? 1024 : 0);
        if (real) {
            const unsigned c = (unsigned)wrapi(gy, ny) * nx + wrapi(gx, nx);
#pragma unroll
            for (int j = 0; j < 9; ++j) h[m][j] = hin[j * N + c];
            if constexpr (kFact) {
                const R eh = eps[c] - P.feps_ref;
                se[k] = R(3) * P.fitau_h * eh * rcp(eh + cs2<R>() * P.ftau_h);
                if constexpr (!RS) sq[k] = R(0.125) * q[c];
            } else {
                se[k] = eps[c];
                if constexpr (!RS) sq[k] = q[c];
            }
            if constexpr (RS) {
#pragma unroll
                for (int j = 0; j < 9; ++j) rr[m][j] = rres[j * N + c];
            }
        } else {
#pragma unroll
            for (int j = 0; j < 9; ++j) h[m][j] = R(0);
            se[k] = kFact ? R(0) : pv<R>(P.eps_ref, P.feps_ref);
            if constexpr (RS) {
#pragma unroll
                for (int j = 0; j < 9; ++j) rr[m][j] = R(0);
            } else {
                sq[k] = R(0);
            }
        }
    }
    __syncthreads();

    // the global index of an owned tile cell
    auto cell = [&](int m) {
        const int k = tid + m * NT;
        return (unsigned)(y0 + k / RX) * nx + (unsigned)(x0 + k % RX);
    };
    const R th = pv<R>(P.tau_h, P.ftau_h), ith = kconst<R>(P.fitau_h, [&] { return rcp(th); });
    const R vb = prm<R>(P.V_bottom, P.t_Vb, P.fVb), vt = prm<R>(P.V_top, P.t_Vt, P.fVt);
    const R eref = pv<R>(P.eps_ref, P.feps_ref);
    const bool electrodes = P.bc_y == 2;
    // residual sums: a thread's own cells (three at most) in R, the block and grid
    // sums in FP64
    R acc[4] = {R(0), R(0), R(0), R(0)};
    // K = 4 (the default chunk) is a compile-time constant in its own instantiation:
    // the iteration loop unrolls and its cone and check conditions resolve per t
    const int K = KC > 0 ? KC : Kdyn;
    constexpr int kUnroll = KC > 0 ? KC : 1;
#pragma unroll kUnroll
    for (int t = 0; t < K; ++t) {
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            if ((meta[m] & 255) > K - t) continue;  // no longer feeds the tile (or not a fluid cell)
            const int k = tid + m * NT;
            R ps = R(0), jx = R(0), jy = R(0);
#pragma unroll
            for (int j = 1; j < 9; ++j) ps += h[m][j];
            ps = dv(ps, R(1) - wgt<R>(0), R(1.8));
#pragma unroll
            for (int j = 0; j < 9; ++j) { cacc(jx, cx(j), h[m][j]); cacc(jy, cy(j), h[m][j]); }
            if ((meta[m] & 1024) && (check && t == 0 || save_prev && t == K - 1)) {
                const unsigned c = cell(m);
                if (check && t == 0) {
                    const R d = ps - prev[c], ex = jx - prev[N + c], ey = jy - prev[2 * N + c];
                    acc[0] += d * d;
                    acc[1] += ps * ps;
                    acc[2] += ex * ex + ey * ey;
                    acc[3] += jx * jx + jy * jy;
                }
                if (save_prev && t == K - 1) { prev[c] = ps; prev[N + c] = jx; prev[2 * N + c] = jy; }
            }
            R hc[9];
            if constexpr (kFact) {
                const R Kc = se[k], q8 = RS ? R(0) : sq[k];
#pragma unroll
                for (int j = 0; j < 9; ++j) hc[j] = h_collide<R>(j, h[m][j], ps, R(0), R(0), jx, jy, th, ith, R(0), Kc, R(0), q8);
            } else {
                const R epshat = se[k] - eref;
                const R den = epshat + cs2<R>() * th, iden = rcp(den);
                const R gx = dv(-jx, den, iden), gy2 = dv(-jy, den, iden);
                const R qc = RS ? R(0) : sq[k];
#pragma unroll
                for (int j = 0; j < 9; ++j)
                    hc[j] = h_collide<R>(j, h[m][j], ps, gx, gy2, jx, jy, th, ith, epshat, R(0), qc, R(0));
            }
#pragma unroll
            for (int j = 0; j < 9; ++j) hs[j * CELLS + k] = hc[j];
            // a wall cell whose own pull is still needed (so it is not on the region
            // border, and its ghost slots lie inside the region): the populations
            // leaving toward the wall come back in the opposite direction, through
            // the ghost cell they would be pulled from (anti-bounce-back to the
            // electrode potential, or plain bounce-back)
            if ((meta[m] & 768) && (meta[m] & 255) <= K - 1 - t) {
#pragma unroll
                for (int j = 1; j < 9; ++j) {
                    const bool bottom = cy(j) < 0 && (meta[m] & 256), top = cy(j) > 0 && (meta[m] & 512);
                    if (!bottom && !top) continue;
                    const int jo = opp(j);  // arriving direction
                    const R v = electrodes ? (RS ? -hc[j] : -hc[j] + R(2) * wgt<R>(j) * (top ? vt : vb)) : hc[j];
                    hs[jo * CELLS + k - cy(jo) * RX - cx(jo)] = v;
                }
            }
        }
        __syncthreads();
        // pull streaming inside the region (cells whose sources were all updated)
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            if ((meta[m] & 255) > K - 1 - t) continue;
            const int k = tid + m * NT;
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                h[m][j] = hs[j * CELLS + k - cy(j) * RX - cx(j)];
                if constexpr (RS) h[m][j] += rr[m][j];
            }
        }
        __syncthreads();
    }
    // write the tile
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
        if (!(meta[m] & 1024)) continue;
        const unsigned c = cell(m);
#pragma unroll
        for (int j = 0; j < 9; ++j) hout[j * N + c] = h[m][j];
    }
    if (check) block_reduce_store_r<4>(acc, partial + 4 * (size_t)(bx + gdx * by));
}
// Asynchronous global->shared copies (cp.async) of 4, 8 or 16 bytes
template <class T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async of 4 or 8 bytes");
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
template <class T>
__device__ __forceinline__ void cp_async16(T* smem, const T* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Tensor-memory-accelerator (TMA) copies of boxes of a 2-D or 3-D array into shared
// memory, completing on an mbarrier with transaction counting (sm_90 and later)
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
                 "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                     (unsigned)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"((unsigned)__cvta_generic_to_shared(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"((unsigned)__cvta_generic_to_shared(bar)), "r"(x), "r"(y)
        : "memory");
}
// wait for phase `parity` of the barrier, at most `limit` polls; false on giving up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    for (int i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// polls of a TMA wait before a block gives up, sets the error flag and returns
constexpr int TMA_WAIT_LIMIT = 1 << 22;

template <class R, int H, int KC = 0>
__global__ void __launch_bounds__(pb_threads<R, H>(), pb_min_blocks<R, H>())
    k_poisson_tb(DevParams P, const R* __restrict__ hin, R* __restrict__ hout, const R* __restrict__ eps,
                 const R* __restrict__ q, R* __restrict__ prev, double* __restrict__ partial, int K, int save_prev,
                 int check) {
    body_poisson_tb<R, H, KC>(P, hin, hout, eps, q, prev, partial, K, save_prev, check, blockIdx.x, blockIdx.y,
                          gridDim.x);
}
// K iterations on the correction to the anchor (save_prev: psi and J before the
// last collision into prev; FP32 with INC, the last launch before a check: the
// check's block sums instead, see body_poisson_tb_f32)
template <class R, int H, int KC = 0, bool INC = false>
__global__ void __launch_bounds__(pb_threads<R, H, true>(), pb_min_blocks<R, H, true>())
    k_poisson_tb_rs(DevParams P, const R* __restrict__ hin, R* __restrict__ hout, const R* __restrict__ eps,
                    const R* __restrict__ rres, R* __restrict__ prev, int K, int save_prev,
                    double* __restrict__ partial, float* __restrict__ rhs, float* __restrict__ e0) {
    body_poisson_tb<R, H, KC, true, INC>(P, hin, hout, eps, nullptr, prev, partial, K, save_prev, 0, blockIdx.x,
                                         blockIdx.y, gridDim.x, rres, rhs, e0);
}

// final reduction of nblk x NV partials in a fixed order (one block of 256 threads)
template <int NV>
__global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ partial, int nblk,
                                                         double* __restrict__ out) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += partial[(size_t)b * NV + k];
    block_reduce_store<NV>(v, out);
}

// first stage of a two-stage reduction: block b sums partial rows
// [b*chunk, (b+1)*chunk) into out[b]; k_reduce_partials then sums the gridDim.x rows.
// Both stages run in a fixed order, so the result does not depend on timing.
template <int NV>
__global__ void __launch_bounds__(256) k_reduce_stage1(const double* __restrict__ partial, int nblk, int chunk,
                                                       double* __restrict__ out) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    const int b0 = blockIdx.x * chunk, b1 = min(nblk, b0 + chunk);
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += partial[(size_t)b * NV + k];
    block_reduce_store<NV>(v, out + (size_t)NV * blockIdx.x);
}

// psi and E = sum c_j h_j / (eps - eps_ref + cs2 tau_h) + E_ext from the current h
template <class R>
__device__ __forceinline__ void body_potential_fields(const DevParams P, const R* __restrict__ h,
                                                          const R* __restrict__ eps, R* __restrict__ E,
                                                          double* __restrict__ psi_out, int bx, int by, int gdx) {
    const int x = bx * blockDim.x + threadIdx.x, y = by * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    R ps = R(0), jx = R(0), jy = R(0);
#pragma unroll
    for (int j = 1; j < 9; ++j) ps += h[j * N + c];
#pragma unroll
    for (int j = 0; j < 9; ++j) { jx += R(cx(j)) * h[j * N + c]; jy += R(cy(j)) * h[j * N + c]; }
    if (psi_out) { psi_out[c] = (double)(ps / (R(1) - wgt<R>(0))); return; }
    const R den = (eps[c] - pv<R>(P.eps_ref, P.feps_ref)) + cs2<R>() * pv<R>(P.tau_h, P.ftau_h);
    const R gx = -jx / den, gy = -jy / den;
    E[c] = -gx + pv<R>(P.E_ext[0], P.fE[0]);
    E[N + c] = -gy + pv<R>(P.E_ext[1], P.fE[1]);
}
template <class R>
__global__ void __launch_bounds__(256) k_potential_fields(DevParams P, const R* __restrict__ h,
                                                          const R* __restrict__ eps, R* __restrict__ E,
                                                          double* __restrict__ psi_out) {
    body_potential_fields<R>(P, h, eps, E, psi_out, blockIdx.x, blockIdx.y, gridDim.x);
}

// h at equilibrium with the linear electrode profile (or zero)
template <class R>
__global__ void k_init_h(DevParams P, R* __restrict__ h) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    R ps;
    if constexpr (is_dual<R>::value) {
        const R vb = prm<R>(P.V_bottom, P.t_Vb), vt = prm<R>(P.V_top, P.t_Vt);
        ps = P.bc_y == 2 ? vb + (vt - vb) * R((y + 0.5) / P.ny) : R(0);
    } else {
        ps = R(P.bc_y == 2 ? P.V_bottom + (P.V_top - P.V_bottom) * (y + 0.5) / P.ny : 0.0);
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) h[j * N + c] = (j == 0) ? (wgt<R>(0) - R(1)) * ps : wgt<R>(j) * ps;
}

template <class R>
__global__ void k_fill_E(DevParams P, R* __restrict__ E) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)P.N) return;
    E[i] = R(P.E_ext[0]);
    E[P.N + i] = R(P.E_ext[1]);
}

// ---------------------------------------------------------------- Eq. 20 at one cell from a phi tile
template <class R>
__device__ __forceinline__ R lap_tile(const R* t, int pitch, int ty, int tx) {
    const R c = t[ty * pitch + tx];
    R a = R(0);  // the j = 0 term, 2 w_0 (c - c), is exactly zero
#pragma unroll
    for (int j = 1; j < 9; ++j) a += R(2) * wgt<R>(j) * (t[(ty + cy(j)) * pitch + tx + cx(j)] - c);
    return oc2(a);
}
template <class R>
__device__ __forceinline__ R chem_pot(const DevParams& P, int i, R ph, R lap, R e2, R c24) {
    // c24 = 24 / D, formed once by the caller
    const R D = pv<R>(P.D, P.fD), lam = prm<R>(P.lam[i], P.t_lam[i], P.flam[i]);
    const R bulk = c24 * lam * ph * (ph - R(0.5)) * (ph - R(1));
    const R grad = R(0.75) * D * lam * lap;
    const R deps = R(6) * prm<R>(P.eps[i], P.t_eps[i], P.feps[i]) * ph * (R(1) - ph);
    return bulk - grad - R(0.5) * deps * e2;
}

// ---------------------------------------------------------------- S6-S14: fused collide + stream
// One thread per cell of a TX x TY tile.  phi (2-ring halo) and E (1-ring) are
// staged in shared memory; mu is evaluated on the 1-ring there (mirrored at walls);
// then each thread forms grad mu, the force, u and p, and collides and pushes its
// 45 populations.  write_diag stores u, p, mu for field output.
constexpr int TX = 32, TY = 8;

// The fused pass stages through cp.async: a thread's populations, d/dt state and
// charge are requested at kernel entry and stream in while the phi/E tiles load
// and mu is evaluated, so many loads are in flight per warp without holding
// registers.
template <class S>
__host__ __device__ constexpr bool fused_prefetch() {
    return std::is_same<S, float>::value || std::is_same<S, double>::value || std::is_same<S, __half>::value ||
           std::is_same<S, __nv_bfloat16>::value;
}
// staging area: 45 population planes in the storage type, then the 8 d/dt planes
// and the charge in the arithmetic type, TX * TY cells each
template <class R, class S, int BY = 8>
__host__ __device__ constexpr size_t fused_dyn_smem() {
    return fused_prefetch<S>() ? (size_t)45 * TX * BY * sizeof(S) + (size_t)9 * TX * BY * sizeof(R) : 0;
}

template <class R, class S, int BY = 8>
__device__ __forceinline__ void body_fused(const DevParams P, const S* __restrict__ pin, S* __restrict__ pout,
                                                   const R* __restrict__ phi, const R* __restrict__ qf,
                                                   const R* __restrict__ E, R* __restrict__ prev,
                                                   R* __restrict__ diag, int first, int write_diag, int bx, int by, int gdx,
                                                   const CUtensorMap* tm_pop = nullptr,
                                                   const CUtensorMap* tm_prev = nullptr,
                                                   const CUtensorMap* tm_q = nullptr, int* err = nullptr) {
    constexpr int PX = TX + 4, PY = BY + 4;  // phi tile, 2-ring
    constexpr int MX = TX + 2, MY = BY + 2;  // mu / E tile, 1-ring
    __shared__ R sphi[3][PY * PX];
    __shared__ R sE[2][MY * MX];
    __shared__ R smu[3][MY * MX];
    // rho, eps, sigma of the 1-ring cells (formed once per tile; dual types, whose
    // tiles would exceed the static shared-memory limit, evaluate them per stencil)
    constexpr bool kProps = !is_dual<R>::value;
    // FP32 collisions (plain and dual) in factored form (same expressions up to
    // rounding, fewer instructions); the FP64 builds evaluate Eq. 34-50 as written
    constexpr bool kFact = f32_family<R>::value;
    __shared__ R sprop[kProps ? 3 : 1][kProps ? MY * MX : 1];
    const int nx = P.nx, ny = P.ny;
    const unsigned N = P.N;
    const int x0 = bx * TX, y0 = by * BY;
    const int tid = threadIdx.x + TX * threadIdx.y;

    // request the tile's populations, d/dt state and charge first: 16-byte copies
    // of row segments when rows are 16-byte aligned (nx a multiple of 16/sizeof for
    // both types), else one element per copy (4- or 8-byte types) or, for 2-byte
    // storage, plain loads later; slot layout [plane][ty * TX + tx]
    constexpr bool kStage = fused_prefetch<S>();
    extern __shared__ __align__(128) unsigned char fz_raw[];
    __shared__ __align__(8) uint64_t fz_bar;  // the TMA staging's barrier
    S* sp = reinterpret_cast<S*>(fz_raw);                                      // [45][TX * BY]
    R* sr = reinterpret_cast<R*>(fz_raw + (size_t)45 * TX * BY * sizeof(S));  // [9][TX * BY]
    bool staged = false;  // the same for the whole block (depends on nx only)
    const bool tma = kStage && tm_pop != nullptr;
    if (tma) {
        // one thread copies the tile of every needed population plane, of the 8 d/dt
        // planes and of the charge with the tensor memory accelerator (boxes of 32 x
        // BY cells; parts beyond the lattice arrive as zeros and are never used)
        staged = true;
        if (tid == 0) {
            constexpr unsigned PB = TX * BY * sizeof(S), RB = TX * BY * sizeof(R);
            constexpr int NP = anchored<S>() ? 42 : 45;
            mbar_init(&fz_bar, 1);
            mbar_arrive_expect_tx(&fz_bar, NP * PB + 9 * RB);
            for (int k = 0; k < 45; ++k) {
                if (anchored<S>() && (k == 9 || k == 18 || k == 27)) continue;  // rest populations rebuilt
                tma_load_3d(sp + k * (TX * BY), tm_pop, x0, y0, k, &fz_bar);
            }
            tma_load_3d(sr, tm_prev, x0, y0, 0, &fz_bar);
            tma_load_2d(sr + 8 * (TX * BY), tm_q, x0, y0, &fz_bar);
        }
    } else if constexpr (kStage) {
        constexpr int VS = 16 / (int)sizeof(S), VR = 16 / (int)sizeof(R);  // cells per 16-byte segment
        constexpr int SGS = TX / VS, SGR = TX / VR;                        // segments per tile row
        auto rplane = [&](int k) -> const R* { return k < 8 ? prev + (size_t)k * N : qf; };
        if (nx % (VS > VR ? VS : VR) == 0) {
            staged = true;
            for (int t = tid; t < 45 * BY * SGS; t += TX * BY) {
                const int k = t / (BY * SGS), r = (t / SGS) % BY, m = t % SGS;
                if (anchored<S>() && (k == 9 || k == 18 || k == 27)) continue;  // rest populations rebuilt
                const int ys = y0 + r, xs = x0 + m * VS;
                if (ys >= ny || xs >= nx) continue;  // nx % VS == 0: a segment is all in or all out
                cp_async16(sp + k * (TX * BY) + r * TX + m * VS, pin + (size_t)k * N + (unsigned)ys * nx + xs);
            }
            for (int t = tid; t < 9 * BY * SGR; t += TX * BY) {
                const int k = t / (BY * SGR), r = (t / SGR) % BY, m = t % SGR;
                const int ys = y0 + r, xs = x0 + m * VR;
                if (ys >= ny || xs >= nx) continue;
                cp_async16(sr + k * (TX * BY) + r * TX + m * VR, rplane(k) + (unsigned)ys * nx + xs);
            }
        } else if constexpr (sizeof(S) >= 4) {
            staged = true;
            const int xs = x0 + threadIdx.x, ys = y0 + threadIdx.y;
            if (xs < nx && ys < ny) {
                const unsigned cs = (unsigned)ys * nx + xs;
                for (int k = 0; k < 45; ++k) {
                    if (anchored<S>() && (k == 9 || k == 18 || k == 27)) continue;
                    cp_async(sp + k * (TX * BY) + tid, pin + (size_t)k * N + cs);
                }
                for (int k = 0; k < 9; ++k) cp_async(sr + k * (TX * BY) + tid, rplane(k) + cs);
            }
        }
    }
    if (kStage && !tma) cp_async_commit();
    // population k (plane k of the set-major layout) of this cell
    auto popk = [&](int k, unsigned cc) -> R {
        if (kStage && staged) return (R)sp[k * (TX * BY) + tid];
        return Store<S>::ld(pin, k * N + cc);
    };

    for (int k = tid; k < PY * PX; k += TX * BY) {
        const int ly = k / PX, lx = k % PX;
        const unsigned n = (unsigned)tile_row(y0 + ly - 2, ny, P.bc_y) * nx + wrapi(x0 + lx - 2, nx);
        sphi[0][k] = phi[n];
        sphi[1][k] = phi[N + n];
        sphi[2][k] = phi[2 * N + n];
    }
    for (int k = tid; k < MY * MX; k += TX * BY) {
        const int ly = k / MX, lx = k % MX;
        const unsigned n = (unsigned)tile_row(y0 + ly - 1, ny, P.bc_y) * nx + wrapi(x0 + lx - 1, nx);
        sE[0][k] = E[n];
        sE[1][k] = E[N + n];
    }
    __syncthreads();
    // mu on the 1-ring at in-domain rows
    const R c24 = kconst<R>(P.fc24, [&] { return R(24) / pv<R>(P.D, P.fD); });
    for (int k = tid; k < MY * MX; k += TX * BY) {
        const int ly = k / MX, lx = k % MX;
        const int gy = y0 + ly - 1;
        if constexpr (kProps) {
            // ghost rows hold the mirrored phi, as the stencil expects
            const int kp = (ly + 1) * PX + lx + 1;
            const R p0 = sphi[0][kp], p1 = sphi[1][kp], p2 = sphi[2][kp];
            sprop[0][k] = dens<R>(P, p0, p1, p2);
            sprop[1][k] = perm<R>(P, p0, p1, p2);
            sprop[2][k] = cond<R>(P, p0, p1, p2);
        }
        if (P.bc_y != 0 && (gy < 0 || gy >= ny)) continue;
        const R ex = sE[0][k], ey = sE[1][k];
        const R e2 = ex * ex + ey * ey;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const R ph = sphi[i][(ly + 1) * PX + lx + 1];
            smu[i][k] = chem_pot<R>(P, i, ph, lap_tile<R>(sphi[i], PX, ly + 1, lx + 1), e2, c24);
        }
    }
    if (tma) {
        // every thread sees the copies complete (the barrier's phase 0); a failed wait
        // anywhere makes the whole block give up, after a second bounded wait by the
        // issuing thread so that no copy still lands in this block's shared memory
        const bool ok = mbar_wait(&fz_bar, 0, TMA_WAIT_LIMIT);
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                if (!ok) mbar_wait(&fz_bar, 0, TMA_WAIT_LIMIT);
                if (err) atomicExch(err, 1);
            }
            return;
        }
    } else {
        if constexpr (kStage) cp_async_wait_all();  // slots are published by the barrier
        __syncthreads();
    }
    // ghost rows of mu mirror the in-domain row they face
    if (P.bc_y != 0) {
        for (int k = tid; k < MY * MX; k += TX * BY) {
            const int ly = k / MX, lx = k % MX;
            const int gy = y0 + ly - 1;
            if (gy >= 0 && gy < ny) continue;
            const int src = ghost_row(gy, ny, P.bc_y) - (y0 - 1);
            if (src >= 0 && src < MY)
#pragma unroll
                for (int i = 0; i < 3; ++i) smu[i][k] = smu[i][src * MX + lx];
        }
        __syncthreads();
    }

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const unsigned c = (unsigned)y * nx + x;
    const int py = threadIdx.y + 2, px = threadIdx.x + 2;
    const int my = threadIdx.y + 1, mx = threadIdx.x + 1;

    R ph[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ph[i] = sphi[i][py * PX + px];
    // stencils (Eq. 33) of mu_i, rho, eps, sigma
    R gmu[3][2], grx = R(0), gry = R(0), gex = R(0), gey = R(0), gsx = R(0), gsy = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R ax = R(0), ay = R(0);
#pragma unroll
        for (int j = 1; j < 9; ++j) {
            const R v = smu[i][(my + cy(j)) * MX + mx + cx(j)];
            cacc(ax, cx(j), wgt<R>(j), v);
            cacc(ay, cy(j), wgt<R>(j), v);
        }
        gmu[i][0] = oc2(ax);
        gmu[i][1] = oc2(ay);
    }
    R rho = R(0), sg = R(0), ep = R(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        R r, e, s;
        if constexpr (kProps) {
            const int k = (my + cy(j)) * MX + mx + cx(j);
            r = sprop[0][k];
            e = sprop[1][k];
            s = sprop[2][k];
        } else {
            const int k = (py + cy(j)) * PX + px + cx(j);
            const R p0 = sphi[0][k], p1 = sphi[1][k], p2 = sphi[2][k];
            r = dens<R>(P, p0, p1, p2);
            e = perm<R>(P, p0, p1, p2);
            s = cond<R>(P, p0, p1, p2);
        }
        if (j == 0) { rho = r; ep = e; sg = s; continue; }
        cacc(grx, cx(j), wgt<R>(j), r);
        cacc(gry, cy(j), wgt<R>(j), r);
        cacc(gex, cx(j), wgt<R>(j), e);
        cacc(gey, cy(j), wgt<R>(j), e);
        cacc(gsx, cx(j), wgt<R>(j), s);
        cacc(gsy, cy(j), wgt<R>(j), s);
    }
    grx = oc2(grx); gry = oc2(gry);
    gex = oc2(gex); gey = oc2(gey);
    gsx = oc2(gsx); gsy = oc2(gsy);

    const R Ex = sE[0][my * MX + mx], Ey = sE[1][my * MX + mx];
    const R qc = (kStage && staged) ? sr[8 * (TX * BY) + tid] : qf[c];
    // R of Eq. 47 with q^n and E^n
    const R rr = dv(sg, ep, rcp(ep));
    const R Rc = -rr * qc + rr * (gex * Ex + gey * Ey) - (gsx * Ex + gsy * Ey);
    // force, Eq. 27b
    R Fx = R(0), Fy = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) { Fx -= ph[i] * gmu[i][0]; Fy -= ph[i] * gmu[i][1]; }
    Fx = Fx + qc * Ex;
    Fy = Fy + qc * Ey;

    // flow moments, Eq. 41
    R g[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) g[j] = popk(j, c);
    R mxm = R(0), mym = R(0), g1 = R(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        cacc(mxm, cx(j), g[j]);
        cacc(mym, cy(j), g[j]);
        if (j) g1 += g[j];
    }
    const R irho = rcp(rho);
    const R ux = dv(mxm + R(0.5) * Fx, rho, irho);
    const R uy = dv(mym + R(0.5) * Fy, rho, irho);
    const R ugr = ux * grx + uy * gry;
    const R pr = cs2<R>() / (R(1) - wgt<R>(0)) * (g1 + R(0.5) * ugr + rho * s_eq<R>(0, ux, uy));

    // d/dt terms (first-order backward differences)
    auto prevk = [&](int k) -> R {
        if (kStage && staged) return sr[k * (TX * BY) + tid];
        return prev[k * N + c];
    };
    R dpu[3][2], dqu[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dpu[i][0] = first ? R(0) : ph[i] * ux - prevk(2 * i);
        dpu[i][1] = first ? R(0) : ph[i] * uy - prevk(2 * i + 1);
    }
    dqu[0] = first ? R(0) : qc * ux - prevk(6);
    dqu[1] = first ? R(0) : qc * uy - prevk(7);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        prev[(2 * i) * N + c] = ph[i] * ux;
        prev[(2 * i + 1) * N + c] = ph[i] * uy;
    }
    prev[6 * N + c] = qc * ux;
    prev[7 * N + c] = qc * uy;

    if (write_diag) {
        diag[c] = ux;
        diag[N + c] = uy;
        diag[2 * N + c] = pr;
#pragma unroll
        for (int i = 0; i < 3; ++i) diag[(3 + i) * N + c] = smu[i][my * MX + mx];
    }

    const bool walls = P.bc_y != 0;
    // link j of this cell crosses a wall (half-way bounce-back) instead of reaching a neighbour
    auto to_wall = [&](int j) { return cy(j) != 0 && walls && (y + cy(j) < 0 || y + cy(j) >= ny); };
    // push targets within a set, formed once for the five sets: post-collision value
    // v of plane (set, j) leaving cell (x, y) goes to the neighbour's plane j, or, on
    // a link into a wall, back to this cell in the opposite direction
    unsigned tgt[9];
    {
        const unsigned rows[3] = {(unsigned)wrap1(y - 1, ny) * nx, (unsigned)y * nx, (unsigned)wrap1(y + 1, ny) * nx};
        const unsigned cols[3] = {(unsigned)wrap1(x - 1, nx), (unsigned)x, (unsigned)wrap1(x + 1, nx)};
#pragma unroll
        for (int j = 0; j < 9; ++j)
            tgt[j] = to_wall(j) ? (unsigned)opp(j) * N + c : (unsigned)j * N + rows[cy(j) + 1] + cols[cx(j) + 1];
    }
    auto push = [&](int set, int j, R v) { Store<S>::st(pout, (size_t)(9 * set) * N + tgt[j], v); };

    // phase populations, Eq. 34-36 with the mobility of Eq. 28
    const R tf = pv<R>(P.tau_f, P.ftau_f), m0 = pv<R>(P.m0, P.fm0);
    const R itf = kconst<R>(P.fitau_f, [&] { return rcp(tf); });
    const R im0 = kconst<R>(P.fim0, [&] { return rcp(m0); });
    const R pf = kconst<R>(P.fpf, [&] { return R(1) - R(1) / (R(2) * tf); });
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        R Mii = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (k != i) Mii += m0 * ph[i] * ph[k];
        R Yx = R(0), Yy = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const R Mik = (k == i) ? (Mii - m0) : -m0 * ph[i] * ph[k];
            Yx += Mik * gmu[k][0];
            Yy += Mik * gmu[k][1];
        }
        const R Ax = oc2(dpu[i][0]) - dv(Yx, m0, im0);
        const R Ay = oc2(dpu[i][1]) - dv(Yy, m0, im0);
        const R mui = smu[i][my * MX + mx];
        R fv[9];
#pragma unroll
        for (int j = anchored<S>() ? 1 : 0; j < 9; ++j) fv[j] = popk(9 * (i + 1) + j, c);
        if constexpr (anchored<S>()) {
            // rest population in deviation form about phi_i: f_0 - phi_i = -sum_{j>0} f_j,
            // f_0 - f_0^eq = (1 - w_0) mu_i - sum_{j>0} f_j; the source term of j = 0 is zero
            R a = R(0);
#pragma unroll
            for (int j = 1; j < 9; ++j) a += fv[j];
            const R neq0 = (R(1) - wgt<R>(0)) * mui - a;
            push(i + 1, 0, -a - dv(neq0, tf, itf));
        }
        if constexpr (kFact) {
            // f_j* = (1 - 1/tau_f) f_j + w_j (mu/tau_f + c_j.Q), Q = 3 phi u / tau_f + pf A
            const R om = R(1) - itf, b = itf * mui, c3 = R(3) * itf;
            const R Qx = fmaf_(pf, Ax, c3 * (ph[i] * ux)), Qy = fmaf_(pf, Ay, c3 * (ph[i] * uy));
            if constexpr (!anchored<S>())  // plain rest population: f_0^eq = phi - (1 - w_0) mu, F_0 = 0
                push(i + 1, 0, fmaf_(om, fv[0], itf * (ph[i] - (R(1) - wgt<R>(0)) * mui)));
#pragma unroll
            for (int j = 1; j < 9; ++j) push(i + 1, j, fmaf_(om, fv[j], wgt<R>(j) * (b + cdot<R>(j, Qx, Qy))));
        } else {
#pragma unroll
            for (int j = anchored<S>() ? 1 : 0; j < 9; ++j) {
                const R feq = (j == 0) ? ph[i] - (R(1) - wgt<R>(0)) * mui
                                       : wgt<R>(j) * mui + oc2(wgt<R>(j) * cdot<R>(j, ph[i] * ux, ph[i] * uy));
                const R Fj = wgt<R>(j) * cdot<R>(j, Ax, Ay);
                push(i + 1, j, fv[j] - dv(fv[j] - feq, tf, itf) + pf * Fj);
            }
        }
    }

    // flow populations, Eq. 37-40
    {
        R tg = pv<R>(P.tau_g, P.ftau_g);
        R itg = kconst<R>(P.fitau_g, [&] { return rcp(tg); });
        R pg = kconst<R>(P.fpg, [&] { return R(1) - R(1) / (R(2) * tg); });
        if (P.use_visc) {
            R eta = R(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) eta += ph[i] * pv<R>(P.visc[i], P.fvisc[i]);
            tg = R(0.5) + dv(eta, rho * cs2<R>(), oc2(irho));
            itg = rcp(tg);
            pg = R(1) - dv(R(1), R(2) * tg, R(0.5) * itg);
        }
        const R uw = y == 0 ? pv<R>(P.u_wall_bottom, P.fuwb) : pv<R>(P.u_wall_top, P.fuwt);
        // into a moving wall: g_opp = g* - 2 w rho (c . u_w) / cs2
        auto wall_term = [&](int j) { return oc2(R(2) * wgt<R>(j) * rho * (R(cx(j)) * uw)); };
        if constexpr (kFact) {
            // g_j* = (1 - 1/tau_g) g_j + w_j [B + rho/tau_g c.u (3 + 4.5 c.u) + 3 pg (c.F + c.u c.grad rho)],
            // B = (3 pr - 1.5 rho |u|^2)/tau_g; j = 0: (1 - 1/tau_g) g_0 + w_0 B - 3 pr/tau_g
            // (G_0 = 0: the u.grad rho terms of Eq. 38 cancel for the rest direction)
            const R om = R(1) - itg, uu = fmaf_(ux, ux, uy * uy);
            const R B = itg * fmaf_(R(-1.5) * rho, uu, R(3) * pr);
            const R c3 = R(3) * itg * rho, c45 = R(4.5) * itg * rho, p3 = R(3) * pg;
            push(0, 0, fmaf_(om, g[0], fmaf_(wgt<R>(0), B, R(-3) * itg * pr)));
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                const R cu = cdot<R>(j, ux, uy);
                const R t = fmaf_(p3, fmaf_(cu, cdot<R>(j, grx, gry), cdot<R>(j, Fx, Fy)), fmaf_(cu, fmaf_(c45, cu, c3), B));
                const R v = fmaf_(om, g[j], wgt<R>(j) * t);
                push(0, j, to_wall(j) ? v - wall_term(j) : v);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const R geq = (j == 0) ? oc2((wgt<R>(0) - R(1)) * pr) + rho * s_eq<R>(0, ux, uy)
                                       : oc2(wgt<R>(j) * pr) + rho * s_eq<R>(j, ux, uy);
                const R cu = cdot<R>(j, ux, uy);
                const R cgr = cdot<R>(j, grx, gry);
                const R cF = cdot<R>(j, Fx, Fy);
                const R G = wgt<R>(j) * (ugr + oc2(cF) + oc2(cu * cgr - cs2<R>() * ugr));
                const R v = g[j] - dv(g[j] - geq, tg, itg) + pg * G;
                push(0, j, to_wall(j) ? v - wall_term(j) : v);
            }
        }
    }

    // charge populations, Eq. 48-50
    {
        const R tl = pv<R>(P.tau_l, P.ftau_l);
        const R itl = kconst<R>(P.fitau_l, [&] { return rcp(tl); });
        const R pl = kconst<R>(P.fpl, [&] { return R(1) - R(1) / (R(2) * tl); });
        const bool cc = P.charge_convection != 0;
        if constexpr (kFact) {
            // l_j* = (1 - 1/tau_l) l_j + w_j (q/tau_l + pl R + c_j.K),
            // K = 3 (q u / tau_l + pl d(qu)/dt) with convection, else 0
            const R om = R(1) - itl, iq = itl * qc, a0 = fmaf_(pl, Rc, iq);
            const R Kx = cc ? R(3) * fmaf_(pl, dqu[0], iq * ux) : R(0);
            const R Ky = cc ? R(3) * fmaf_(pl, dqu[1], iq * uy) : R(0);
            push(4, 0, fmaf_(om, popk(36, c), wgt<R>(0) * a0));
#pragma unroll
            for (int j = 1; j < 9; ++j) push(4, j, fmaf_(om, popk(36 + j, c), wgt<R>(j) * (a0 + cdot<R>(j, Kx, Ky))));
        } else {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const R cu = cdot<R>(j, ux, uy);
                const R leq = cc ? wgt<R>(j) * qc * (R(1) + oc2(cu)) : wgt<R>(j) * qc;
                const R Sj = pl * wgt<R>(j) * Rc;
                const R Tj = cc ? oc2(pl * wgt<R>(j) * cdot<R>(j, dqu[0], dqu[1])) : R(0);
                const R lj = popk(36 + j, c);
                push(4, j, lj - dv(lj - leq, tl, itl) + Sj + Tj);
            }
        }
    }
}
// the fused pass on one lattice, tiles of 32 x BY cells (lb3e_set_fused_tile)
template <class R, class S, int BY = 8>
__global__ void __launch_bounds__(TX * BY, fused_min_blocks<R, BY>()) k_fused(DevParams P, const S* __restrict__ pin, S* __restrict__ pout,
                                                   const R* __restrict__ phi, const R* __restrict__ qf,
                                                   const R* __restrict__ E, R* __restrict__ prev,
                                                   R* __restrict__ diag, int first, int write_diag,
                                                   const __grid_constant__ CUtensorMap tm_pop,
                                                   const __grid_constant__ CUtensorMap tm_prev,
                                                   const __grid_constant__ CUtensorMap tm_q, int use_tma, int* err) {
    body_fused<R, S, BY>(P, pin, pout, phi, qf, E, prev, diag, first, write_diag, blockIdx.x, blockIdx.y, gridDim.x,
                         use_tma ? &tm_pop : nullptr, &tm_prev, &tm_q, err);
}

// ---------------------------------------------------------------- initial populations
// f^i = f^eq(phi, mu, u), g = g_eq(p = 0, u), l = l_eq(q, u); mu from Eq. 20 with
// the initial field (global-memory stencil; init only).
template <class R, class S>
__global__ void k_init_pops(DevParams P, S* __restrict__ pop, const R* __restrict__ phi, const R* __restrict__ q,
                            const R* __restrict__ E, R* __restrict__ diag) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    const R ux = diag[c], uy = diag[N + c];
    const R Ex = E[c], Ey = E[N + c];
    const R e2 = Ex * Ex + Ey * Ey;
    R ph[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const R* f = phi + i * N;
        const R cc = f[c];
        R a = R(0);
#pragma unroll
        for (int j = 0; j < 9; ++j)
            a += R(2) * wgt<R>(j) * (f[(size_t)ghost_row(y + cy(j), P.ny, P.bc_y) * P.nx + wrapi(x + cx(j), P.nx)] - cc);
        const R lap = a / cs2<R>();
        ph[i] = cc;
        const R mui = chem_pot<R>(P, i, cc, lap, e2, R(24) / R(P.D));
        diag[(3 + i) * N + c] = mui;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const R feq = (j == 0) ? cc - (R(1) - wgt<R>(0)) * mui
                                   : wgt<R>(j) * mui + wgt<R>(j) * (R(cx(j)) * cc * ux + R(cy(j)) * cc * uy) / cs2<R>();
            // anchored storage keeps f_0 - phi = -(1 - w_0) mu without forming phi - ... - phi
            Store<S>::st(pop, (9 * (i + 1) + j) * N + c,
                         (anchored<S>() && j == 0) ? -((R(1) - wgt<R>(0)) * mui) : feq);
        }
    }
    const R rho = dens<R>(P, ph[0], ph[1], ph[2]);
    const R qc = q[c];
    const bool cc = P.charge_convection != 0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        Store<S>::st(pop, j * N + c, rho * s_eq<R>(j, ux, uy));
        const R cu = R(cx(j)) * ux + R(cy(j)) * uy;
        Store<S>::st(pop, (36 + j) * N + c, cc ? wgt<R>(j) * qc * (R(1) + cu / cs2<R>()) : wgt<R>(j) * qc);
    }
    diag[2 * N + c] = R(0);
}

// add caller noise (FP64 staging, 9 planes of one set) to set `set`; an anchored
// rest population is a deviation, so the noise adds to it unchanged
template <class R, class S>
__global__ void k_add_noise(DevParams P, S* __restrict__ pop, const double* __restrict__ nz, int set) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x, N = P.N;
    if (i >= 9 * N) return;
    const size_t idx = (size_t)(9 * set) * N + i;
    Store<S>::st(pop, idx, Store<S>::ld(pop, idx) + R(nz[i]));
}

// ---------------------------------------------------------------- conversions
template <class R>
__global__ void k_from_f64(R* __restrict__ dst, const double* __restrict__ src, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = R(src[i]);
}
template <class T>
__global__ void k_to_f64(double* __restrict__ dst, const T* __restrict__ src, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}
// component `comp` of a dual field (0 value, k >= 1 tangent k-1) as doubles
template <class R>
__global__ void k_comp_to_f64(double* __restrict__ dst, const R* __restrict__ src, size_t n, int comp) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (is_dual<R>::value)
        dst[i] = comp == 0 ? (double)src[i].v : (double)src[i].d[comp - 1];
    else
        dst[i] = (double)src[i];
}
template <class R, class S>
__global__ void k_pop_to_f64(double* __restrict__ dst, const S* __restrict__ pop, const R* __restrict__ phi,
                             int set, int j, size_t N) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double v = (double)Store<S>::ld(pop, (size_t)(9 * set + j) * N + i);
    if (anchored<S>() && set >= 1 && set <= 3 && j == 0) v += (double)phi[(size_t)(set - 1) * N + i];
    dst[i] = v;
}

// ---------------------------------------------------------------- observables (FP64 reductions)
// Per block: mass[3], charge, F_phi, F_E, F_u, F_q, nonfinite, then the indicator
// moments (sum chi, chi x, chi y, chi x^2, chi y^2) for inner and outer; the max
// deviation |sum phi - 1| is a separate per-block max.
constexpr int NOBS = 19;
// OBS_Y cells per thread along y: a 32 x 8 block covers 32 x 256 cells, so the
// FP64 conversions and block reduction of the NOBS sums (FP64 runs at a small
// fraction of the FP32 rate) are shared by 32 cells per thread.
constexpr int OBS_Y = 32;
inline dim3 obs_grid(int nx, int ny) { return dim3((nx + TX - 1) / TX, (ny + TY * OBS_Y - 1) / (TY * OBS_Y)); }
// A thread's sums of its OBS_Y cells.  FP64: plain FP64 sums.  FP32 terms: an FP32
// sum and the exact rounding error of each of its additions (Knuth's TwoSum),
// accumulated beside it, so that s + c carries the sum to about the square of the
// FP32 precision; converted to FP64 once per thread, where the block and grid
// reductions continue.  (FP64 adds and conversions run at a small fraction of the
// FP32 rate on this part, and the per-cell FP64 accumulation was most of the
// kernel's time.)
template <class T, int NV>
struct ObsAcc {
    double v[NV];
    __device__ __forceinline__ ObsAcc() {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = 0.0;
    }
    __device__ __forceinline__ void add(int k, T x) { v[k] += (double)x; }
    __device__ __forceinline__ void out(double (&o)[NV]) const {
#pragma unroll
        for (int k = 0; k < NV; ++k) o[k] = v[k];
    }
};
template <int NV>
struct ObsAcc<float, NV> {
    float s[NV], c[NV];
    __device__ __forceinline__ ObsAcc() {
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] = c[k] = 0.f;
    }
    __device__ __forceinline__ void add(int k, float x) {
        const float t = __fadd_rn(s[k], x);
        const float bp = __fsub_rn(t, s[k]);
        const float e = __fadd_rn(__fsub_rn(s[k], __fsub_rn(t, bp)), __fsub_rn(x, bp));
        s[k] = t;
        c[k] = __fadd_rn(c[k], e);
    }
    __device__ __forceinline__ void out(double (&o)[NV]) const {
#pragma unroll
        for (int k = 0; k < NV; ++k) o[k] = (double)s[k] + (double)c[k];
    }
};
// |a + b + c - 1| for phase fractions near 1: FP64 in the FP64 build; in FP32 the two
// additions are error-free transformed and 1 is subtracted exactly (Sterbenz)
__device__ __forceinline__ double sum_dev3(double a, double b, double c) { return fabs(a + b + c - 1.0); }
__device__ __forceinline__ float sum_dev3(float a, float b, float c) {
    float s1 = __fadd_rn(a, b), bp = __fsub_rn(s1, a);
    const float e1 = __fadd_rn(__fsub_rn(a, __fsub_rn(s1, bp)), __fsub_rn(b, bp));
    const float s2 = __fadd_rn(s1, c);
    bp = __fsub_rn(s2, s1);
    const float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, bp)), __fsub_rn(c, bp));
    return fabsf(__fadd_rn(__fsub_rn(s2, 1.0f), __fadd_rn(e1, e2)));
}

// Per-block FP64 sums of the NOBS observables (partial[b * NOBS + k]) and the
// per-block max |sum phi - 1| (maxpart[b]).  The per-cell terms are evaluated in
// FP32 in the FP32 builds and in FP64 otherwise (FP64 arithmetic runs at a small
// fraction of the FP32 rate on this part); a thread's sums are ObsAcc pairs, the
// block and grid sums and the max FP64.
template <class R>
__global__ void __launch_bounds__(256) k_observables(DevParams P, const R* __restrict__ phi, const R* __restrict__ q,
                                                     const R* __restrict__ E, const R* __restrict__ diag,
                                                     double* __restrict__ partial, double* __restrict__ maxpart) {
    using T = typename std::conditional<std::is_same<R, float>::value, float, double>::type;
    ObsAcc<T, NOBS> acc;
    T mdev = T(0);
    const int x = blockIdx.x * TX + threadIdx.x;
    // the stencil's columns, formed once a thread (32-bit: at most LB3E_MAX_CELLS cells)
    const unsigned col[3] = {(unsigned)wrapi(x - 1, P.nx), (unsigned)x, (unsigned)wrapi(x + 1, P.nx)};
    for (int r = 0; r < OBS_Y; ++r) {
        const int y = blockIdx.y * (TY * OBS_Y) + r * TY + threadIdx.y;
        if (x >= P.nx || y >= P.ny) continue;
        const unsigned N = P.N, c = (unsigned)y * P.nx + x;
        const unsigned row[3] = {(unsigned)ghost_row(y - 1, P.ny, P.bc_y) * (unsigned)P.nx, (unsigned)y * (unsigned)P.nx,
                                 (unsigned)ghost_row(y + 1, P.ny, P.bc_y) * (unsigned)P.nx};
        const T D = pv<T>(P.D, P.fD);
        T ph[3];
        T fphi = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const R* f = phi + i * N;
            T ax = T(0), ay = T(0);
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                const T w = (T)f[row[cy(j) + 1] + col[cx(j) + 1]];
                cacc(ax, cx(j), wgt<T>(j), w);
                cacc(ay, cy(j), wgt<T>(j), w);
            }
            ax = oc2(ax);
            ay = oc2(ay);
            ph[i] = (T)f[c];
            acc.add(i, ph[i]);
            const T lam = pv<T>(P.lam[i], P.flam[i]);
            fphi += T(6) / D * lam * ph[i] * ph[i] * (T(1) - ph[i]) * (T(1) - ph[i]) +
                    T(0.375) * D * lam * (ax * ax + ay * ay);
        }
        acc.add(4, fphi);
        T eps = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) eps += pv<T>(P.eps[i], P.feps[i]) * ph[i] * ph[i] * (T(3) - T(2) * ph[i]);
        const T Ex = (T)E[c], Ey = (T)E[N + c];
        acc.add(5, T(0.5) * eps * (Ex * Ex + Ey * Ey));
        const T rho = ph[0] * pv<T>(P.rho[0], P.frho[0]) + ph[1] * pv<T>(P.rho[1], P.frho[1]) +
                      ph[2] * pv<T>(P.rho[2], P.frho[2]);
        const T ux = (T)diag[c], uy = (T)diag[N + c];
        acc.add(6, T(0.5) * rho * (ux * ux + uy * uy));
        const T sg = ph[0] * pv<T>(P.sigma[0], P.fsig[0]) + ph[1] * pv<T>(P.sigma[1], P.fsig[1]) +
                     ph[2] * pv<T>(P.sigma[2], P.fsig[2]);
        const T qc = (T)q[c];
        if (sg > T(0)) acc.add(7, T(0.5) * (T(P.alpha) / sg) * qc * qc);
        acc.add(3, qc);
        const T vals[6] = {ph[0], ph[1], ph[2], ux, uy, qc};
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (!isfinite(vals[k])) acc.add(8, T(1));
        const T chis[2] = {ph[P.inner], T(1) - ph[P.matrix]};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            acc.add(9 + 5 * k, chis[k]);
            acc.add(10 + 5 * k, chis[k] * T(x));
            acc.add(11 + 5 * k, chis[k] * T(y));
            acc.add(12 + 5 * k, chis[k] * T(x) * T(x));
            acc.add(13 + 5 * k, chis[k] * T(y) * T(y));
        }
        const T dv = sum_dev3(ph[0], ph[1], ph[2]);
        mdev = dv > mdev ? dv : mdev;  // as fmax: a NaN is left to the nonfinite count
    }
    const int b = blockIdx.x + gridDim.x * blockIdx.y;
    double v[NOBS];
    acc.out(v);
    block_reduce_store<NOBS>(v, partial + (size_t)NOBS * b);
    // block max of the sum deviation (the reduction above ends with a barrier-free
    // warp-0 stage, so this uses its own shared array)
    double md = (double)mdev;
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_down_sync(0xffffffffu, md, o));
    __shared__ double mred[8];
    const int tid = threadIdx.x + TX * threadIdx.y;
    if ((tid & 31) == 0) mred[tid >> 5] = md;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < (TX * TY) / 32; ++k) a = fmax(a, mred[k]);
        maxpart[b] = a;
    }
}

// component m of a value: 0 its value, m >= 1 its tangent m - 1 (dual builds)
template <class R>
__device__ __forceinline__ double comp_of(const R& v, int m) {
    if constexpr (is_dual<R>::value) return m == 0 ? (double)v.v : (double)v.d[m - 1];
    else return m == 0 ? (double)v : 0.0;
}
template <class R> struct n_comp { static constexpr int value = 1; };
template <class T, int M> struct n_comp<Dual<T, M>> { static constexpr int value = 1 + M; };

// Per-block FP64 sums for the deformation factors and their tangents: for the
// indicators chi_inner = phi_inner and chi_outer = 1 - phi_matrix, and for each
// component m (value, tangents), sum chi, chi x, chi y, chi x^2, chi y^2 -- at
// partial[b * 10 M + (5 M) k + 5 m + i], k = 0 inner, 1 outer.
template <class R>
__global__ void __launch_bounds__(256) k_deform_moments(DevParams P, const R* __restrict__ phi,
                                                        double* __restrict__ partial) {
    constexpr int M = n_comp<R>::value, NV = 10 * M;
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    const int x = blockIdx.x * TX + threadIdx.x;
    for (int r = 0; r < OBS_Y; ++r) {
        const int y = blockIdx.y * (TY * OBS_Y) + r * TY + threadIdx.y;
        if (x >= P.nx || y >= P.ny) continue;
        const unsigned N = P.N, c = (unsigned)y * P.nx + x;
        const R pin = phi[P.inner * N + c], pmx = phi[P.matrix * N + c];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const double chis[2] = {comp_of(pin, m), (m == 0 ? 1.0 : 0.0) - comp_of(pmx, m)};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                double* o = v + 5 * M * k + 5 * m;
                o[0] += chis[k];
                o[1] += chis[k] * x;
                o[2] += chis[k] * y;
                o[3] += chis[k] * x * x;
                o[4] += chis[k] * y * y;
            }
        }
    }
    block_reduce_store<NV>(v, partial + (size_t)NV * (blockIdx.x + gridDim.x * blockIdx.y));
}

// Per-block FP64 sums for the shape objective of one phase: sum (phi - target)^2 and,
// per tangent direction t, sum 2 (phi - target) dphi/dtheta_t, at partial[b * M + m]
template <class R>
__global__ void __launch_bounds__(256) k_shape_objective(DevParams P, const R* __restrict__ phi,
                                                         const double* __restrict__ target,
                                                         double* __restrict__ partial) {
    constexpr int M = n_comp<R>::value;
    double v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = 0.0;
    const int x = blockIdx.x * TX + threadIdx.x;
    for (int r = 0; r < OBS_Y; ++r) {
        const int y = blockIdx.y * (TY * OBS_Y) + r * TY + threadIdx.y;
        if (x >= P.nx || y >= P.ny) continue;
        const unsigned c = (unsigned)y * P.nx + x;
        const R f = phi[c];
        const double d = comp_of(f, 0) - target[c];
        v[0] += d * d;
#pragma unroll
        for (int m = 1; m < M; ++m) v[m] += 2.0 * d * comp_of(f, m);
    }
    block_reduce_store<M>(v, partial + (size_t)M * (blockIdx.x + gridDim.x * blockIdx.y));
}

// fixed-order max of n per-block maxima
static __global__ void k_max_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
    double m = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) m = fmax(m, partial[b]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) a = fmax(a, red[k]);
        *out = a;
    }
}

}  // namespace lb3e

namespace lb3e {

// ---------------------------------------------------------------- batched launches
// Many lattices of different sizes stepped together: each block takes one tile
// from a work list (instance, tile x, tile y) and runs the same tile body as the
// single-lattice kernels on that instance's parameters and buffers.
template <class R, class S>
struct InstState {
    DevParams P;
    S* pop[2];
    R* h[2];
    R *phi, *qt, *q, *eps, *E, *prev, *diag;
};

template <class R, class S>
__global__ void __launch_bounds__(256) kb_moments(const InstState<R, S>* __restrict__ st, const int4* __restrict__ tiles,
                                                  int cur) {
    const int4 t = tiles[blockIdx.x];
    const InstState<R, S>& e = st[t.x];
    body_moments<R, S>(e.P, e.pop[cur], e.phi, e.phi, e.qt, t.y, t.z, 0);
}
template <class R, class S>
__global__ void __launch_bounds__(256) kb_prologue(const InstState<R, S>* __restrict__ st, const int4* __restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const InstState<R, S>& e = st[t.x];
    body_prologue<R>(e.P, e.phi, e.qt, e.E, e.q, e.eps, 1, t.y, t.z, 0);
}
template <class R, class S>
__global__ void __launch_bounds__(256) kb_poisson(const InstState<R, S>* __restrict__ st, const int4* __restrict__ tiles,
                                                  int hcur) {
    const int4 t = tiles[blockIdx.x];
    const InstState<R, S>& e = st[t.x];
    if (!e.P.electric) return;
    body_poisson<R>(e.P, e.h[hcur], e.h[hcur ^ 1], e.eps, e.q, nullptr, nullptr, 0, 0, t.y, t.z, 0);
}
// K pseudo-iterations per launch over the 32 x 16 tiles of all instances
template <class R, class S, int H, int KC = 0>
__global__ void __launch_bounds__(pb_threads<R, H>(), pb_min_blocks<R, H>())
    kb_poisson_tb(const InstState<R, S>* __restrict__ st, const int4* __restrict__ tiles, int hcur, int K) {
    const int4 t = tiles[blockIdx.x];
    const InstState<R, S>& e = st[t.x];
    if (!e.P.electric) return;
    body_poisson_tb<R, H, KC>(e.P, e.h[hcur], e.h[hcur ^ 1], e.eps, e.q, nullptr, nullptr, K, 0, 0, t.y, t.z, 0);
}
template <class R, class S>
__global__ void __launch_bounds__(256) kb_potential_fields(const InstState<R, S>* __restrict__ st,
                                                           const int4* __restrict__ tiles, int hcur) {
    const int4 t = tiles[blockIdx.x];
    const InstState<R, S>& e = st[t.x];
    if (!e.P.electric) return;
    body_potential_fields<R>(e.P, e.h[hcur], e.eps, e.E, nullptr, t.y, t.z, 0);
}
// the fused pass over tiles of 32 x BY cells (BY 4, 8 or 16, picked by the autotuner)
template <class R, class S, int BY = 8>
__global__ void __launch_bounds__(TX * BY, fused_min_blocks<R, BY>())
    kb_fused(const InstState<R, S>* __restrict__ st, const int4* __restrict__ tiles, int cur, int first, int write_diag) {
    const int4 t = tiles[blockIdx.x];
    const InstState<R, S>& e = st[t.x];
    body_fused<R, S, BY>(e.P, e.pop[cur], e.pop[cur ^ 1], e.phi, e.q, e.E, e.prev, e.diag, first, write_diag, t.y, t.z,
                         0);
}

}  // namespace lb3e
