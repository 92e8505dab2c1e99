// lb3e_anchor.cuh -- the LB potential solve (Eq. 42-45) on an FP64 anchor, with an
// optional finite-difference coarse correction.
//
// The pseudo-time iteration of Eq. 43 is affine in h: h <- T h + s, with s the
// charge source and the electrode terms of the anti-bounce-back walls.  Here the
// state is split as h = a + delta: the anchor a is FP64, the correction delta is
// in the build's precision.  Each refresh folds delta into a and forms, in FP64,
// the anchor's own increment r = T a + s - a (one pseudo-iteration applied to a,
// minus a).  The iterations in between run on delta with the homogeneous operator
// (no charge, electrodes at zero) plus r after streaming:
//     delta <- T0 delta + r,
// which in exact arithmetic gives the same iterates as the plain iteration of h
// (T0 (h - a) + T a + s - a = T h + s - a).  FP32 rounding then acts on delta, not
// on h, so the relative increment can be driven far below the FP32 resolution of
// h itself (the plain FP32 iteration stalls near 2e-5 on a 4096^2 drop under a
// field: the electrode profile makes psi large against its increments).
//
// The relative increments of psi and J = sum_j c_j h_j that stop the solve are
// those of r at the refresh, summed in FP64.
//
// Coarse correction.  The slowest modes of the pseudo-time iteration decay at a
// rate of order eps k^2 per iteration, so a plain iteration needs O(n^2)
// iterations on an n^2 lattice.  At a refresh, the zeroth moment of the anchor's
// increment, sum_{j>0} r_j = (1 - w_0) (psi' - psi), is the residual of the
// macroscopic equation div(eps grad psi) + q = 0 that the iteration relaxes (the
// moving populations carry psi with weight 1 - w_0).  One FP32 V-cycle of the
// finite-difference multigrid (lb3e_mg.cuh) on A e = sum_{j>0} r_j gives a potential
// correction e, which enters delta as its local equilibrium, w_j e (j > 0) and
// (w_0 - 1) e, plus the first-order flux part -w_j c_j . grad e (eps_hat + cs^2
// tau_h)/cs^2 that the collision would otherwise relax to.  The correction only
// moves the iterate: the fixed point is the one of Eq. 43 (the stopping test reads
// the LB increment), while the finite-difference operator stands in for the LB's
// effective operator on the modes the iteration is slow on.
#pragma once

#include "lb3e_kernels.cuh"
#include "lb3e_mg.cuh"

namespace lb3e {

// ---------------------------------------------------------------- double-float numbers
// The FP32 builds hold the anchor as an unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)/2, about 48 significant bits) and do the refresh's state
// arithmetic on them with error-free transformations: Knuth's TwoSum and Dekker's
// FastTwoSum for sums, the FMA-based exact product for products.  That keeps the
// refresh on the FP32 pipe (FP64 runs at about 1/64 of its rate on this part) at
// far more precision than the tolerance needs.  The __f*_rn intrinsics keep the
// compiler from contracting or reordering these steps.
struct df32 {
    float hi, lo;
};
// a + b exactly as hi + lo (Knuth)
__device__ __forceinline__ df32 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// a + b exactly as hi + lo when |a| >= |b| (Dekker)
__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.hi, -a.lo}; }
// a + b with an error of a few units of 2^-48 of the larger operand (Dekker's add:
// one TwoSum on the leading parts, the trailing parts added plainly).  The refresh
// needs its results to that accuracy in absolute terms, relative to the anchor's
// size, not relative to a cancelled difference; the full TwoSum add costs twice the
// instructions on a pass bound by them.
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    df32 s = df_two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df32 df_add_f(df32 a, float b) {
    df32 s = df_two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return df_fast_two_sum(s.hi, s.lo);
}
// products: hi*hi exactly through one FMA, the cross terms added to its error
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_fast_two_sum(p, e);
}
__host__ __device__ inline df32 df_of(double x) {
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double df_value(df32 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float df_round(df32 a) { return __fadd_rn(a.hi, a.lo); }

// the anchor's number type: FP64 in the FP64 build, double-float in the FP32 builds
template <class R> struct AnchorOf { using type = double; };
template <> struct AnchorOf<float> { using type = df32; };
template <class A> __device__ __forceinline__ double anchor_value(const A& a);
template <> __device__ __forceinline__ double anchor_value<double>(const double& a) { return a; }
template <> __device__ __forceinline__ double anchor_value<df32>(const df32& a) { return df_value(a); }

// the refresh's coefficients as double-float numbers (formed on the host from FP64):
// 1 - 1/tau_h, 1/tau_h, w_0 - 1, w_1..4, w_5..8, 1/(1 - w_0), and 2 w V at the two
// electrodes for the two classes of moving directions
struct AnchorCoef {
    df32 om, ith, w0m1, w1, w5, c18, wv[2][2];  // wv[top][class 0: |c| = 1, 1: diagonal]
};

// a and delta at the start of a solve: the equilibrium of the linear electrode
// profile (or zero) in the anchor, delta = 0
template <class R>
__global__ void __launch_bounds__(256) k_anchor_init(DevParams P, typename AnchorOf<R>::type* __restrict__ a,
                                                     R* __restrict__ d) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    const double ps = P.bc_y == 2 ? P.V_bottom + (P.V_top - P.V_bottom) * (y + 0.5) / P.ny : 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const double v = (j == 0) ? (wgt<double>(0) - 1.0) * ps : wgt<double>(j) * ps;
        if constexpr (std::is_same<R, float>::value) a[j * N + c] = df_of(v);
        else a[j * N + c] = v;
        d[j * N + c] = R(0);
    }
}

// The refresh and the anchor's increment in one pass (FP32 builds): a block of
// 32 x 8 cells folds delta into the anchor and collides (Eq. 43, double-float, the
// factored form of k_anchor_refresh) on its tile and one-cell ring, keeps the
// post-collision values in shared memory, and each of its cells pulls what streams
// into it (across a wall: the reflected value of its own opposite direction, as the
// push form writes it) and forms r = pulled - a, with the per-block sums of
// k_anchor_residual over the same 32 x 8 blocks.  The folded anchor goes to a_out
// and, with d_out, delta = 0 to d_out: neighbouring blocks read a_in and d on their
// rings.  d = nullptr: delta is zero (already folded).
static __global__ void __launch_bounds__(256) k_anchor_refresh_pull_df(DevParams P, const df32* __restrict__ a_in,
                                                                       df32* __restrict__ a_out,
                                                                       const float* __restrict__ d,
                                                                       float* __restrict__ d_out,
                                                                       const float* __restrict__ eps,
                                                                       const float* __restrict__ q,
                                                                       float* __restrict__ r, float* __restrict__ ja,
                                                                       double* __restrict__ partial, AnchorCoef K) {
    constexpr int SX = 34, SY = 10, NC = SX * SY, TC = 32 * 8;
    __shared__ df32 sv[9 * NC];  // post-collision values of the tile and its ring
    __shared__ df32 sh[9 * TC];  // the folded anchor of the tile's cells
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8, tid = threadIdx.x + 32 * threadIdx.y;
    const int nx = P.nx, ny = P.ny;
    const unsigned N = P.N;
    const bool walls = P.bc_y != 0;
    for (int k = tid; k < NC; k += TC) {
        const int ly = k / SX, lx = k - ly * SX;
        const int gy = y0 + ly - 1, gx = x0 + lx - 1;
        if (walls && (gy < 0 || gy >= ny)) continue;  // beyond a wall: no cell, never a source
        const unsigned c = (unsigned)wrapi(gy, ny) * nx + wrapi(gx, nx);
        const bool own = lx >= 1 && lx <= 32 && ly >= 1 && ly <= 8 && gx < nx && gy < ny;
        df32 h[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) h[j] = d ? df_add_f(a_in[j * N + c], d[j * N + c]) : a_in[j * N + c];
        df32 sum = h[1], jx = {0.f, 0.f}, jy = {0.f, 0.f};
#pragma unroll
        for (int j = 2; j < 9; ++j) sum = df_add(sum, h[j]);
        const df32 ps = df_mul(sum, K.c18);
#pragma unroll
        for (int j = 1; j < 9; ++j) {
            if (cx(j)) jx = df_add(jx, cx(j) > 0 ? h[j] : df_neg(h[j]));
            if (cy(j)) jy = df_add(jy, cy(j) > 0 ? h[j] : df_neg(h[j]));
        }
        if (own) {
            const int t = (ly - 1) * 32 + lx - 1;
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                a_out[j * N + c] = h[j];
                sh[j * TC + t] = h[j];
                if (d_out) d_out[j * N + c] = 0.f;
            }
            ja[c] = df_round(jx);
            ja[N + c] = df_round(jy);
        }
        const float eh = eps[c] - P.feps_ref;
        const float Kc = 3.0f * P.fitau_h * eh * rcp(eh + cs2<float>() * P.ftau_h);
        const df32 A = df_mul(K.ith, ps);
        const float q8 = 0.125f * q[c];
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            df32 v;
            if (j == 0) {
                v = df_add(df_mul(K.om, h[0]), df_mul(K.w0m1, A));
            } else {
                df32 cj = cx(j) > 0 ? jx : (cx(j) < 0 ? df_neg(jx) : df32{0.f, 0.f});
                if (cy(j) > 0) cj = df_add(cj, jy);
                else if (cy(j) < 0) cj = df_add(cj, df_neg(jy));
                const df32 t = df_add(A, df_mul_f(cj, Kc));
                v = df_add_f(df_add(df_mul(K.om, h[j]), df_mul(j <= 4 ? K.w1 : K.w5, t)), q8);
            }
            sv[j * NC + k] = v;
        }
    }
    __syncthreads();
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x < nx && y < ny) {
        const unsigned c = (unsigned)y * nx + x;
        const int k = (threadIdx.y + 1) * SX + threadIdx.x + 1;
        float dps = 0.f, ps = 0.f, djx = 0.f, djy = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int ys = y - cy(j);  // the source row
            df32 g;
            if (walls && (ys < 0 || ys >= ny)) {
                const int jl = opp(j);  // the direction that left this cell toward the wall
                g = sv[jl * NC + k];
                if (P.bc_y == 2) g = df_add(df_neg(g), K.wv[ys >= ny ? 1 : 0][jl <= 4 ? 0 : 1]);
            } else {
                g = sv[j * NC + k - cy(j) * SX - cx(j)];
            }
            const df32 aj = sh[j * TC + tid];
            const float rj = df_round(df_add(g, df_neg(aj))), ar = df_round(aj);
            r[j * N + c] = rj;
            if (j) { dps += rj; ps += ar; }
            cacc(djx, cx(j), rj);
            cacc(djy, cy(j), rj);
            cacc(jx, cx(j), ar);
            cacc(jy, cy(j), ar);
        }
        dps *= 1.8f;
        ps *= 1.8f;
        acc[0] = dps * dps;
        acc[1] = ps * ps;
        acc[2] = djx * djx + djy * djy;
        acc[3] = jx * jx + jy * jy;
    }
    block_reduce_store_r<4>(acc, partial + 4 * (size_t)(blockIdx.x + gridDim.x * blockIdx.y));
}


// Fold delta into the anchor (a += delta, delta = 0) and push the FP64 collision
// of the folded anchor (Eq. 43 with the charge source and the electrode walls) to
// the FP64 staging planes: stage = T a + s after the launch.  The collision is the
// factored form h_j* = (1 - 1/tau_h) h_j + w_j (psi/tau_h + Kc c_j . J) + q/8,
// h_0* = (1 - 1/tau_h) h_0 + (w_0 - 1) psi/tau_h, Kc = 3 eps_hat / (tau_h den).
// Arithmetic and coefficients are FP64 here, whatever the build: this operator
// defines the fixed point.  (The D2Q9 weights and 1/(1 - w_0) are not exact in
// binary.  With FP32 coefficients the collision does not conserve sum_{j>0} h_j
// exactly, which acts as a spurious source proportional to psi; its effect on the
// solution grows as the lattice side squared: about 3e-5 of E at 128^2 with FP32
// arithmetic, 3e-6 with FP64 arithmetic but FP32-rounded coefficients.  The
// correction kernels keep FP32 coefficients: their bias scales with delta, not
// with h.)
template <class R>
__global__ void __launch_bounds__(256) k_anchor_refresh(DevParams P, double* __restrict__ a, R* __restrict__ d,
                                                        const R* __restrict__ eps, const R* __restrict__ q,
                                                        double* __restrict__ stage, R* __restrict__ ja,
                                                        double ith, double Kn) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    double h[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        h[j] = a[j * N + c] + (double)d[j * N + c];
        a[j * N + c] = h[j];
        d[j * N + c] = R(0);
    }
    double ps = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int j = 1; j < 9; ++j) ps += h[j];
    ps *= 1.8;  // / (1 - w_0), to within an FP64 rounding
#pragma unroll
    for (int j = 0; j < 9; ++j) { cacc(jx, cx(j), h[j]); cacc(jy, cy(j), h[j]); }
    // ith = 1/tau_h and Kn = cs^2 tau_h are formed on the host.  Kc scales the
    // first moment only (sum_j w_j c_j = 0 in any precision), so the FP32 builds
    // take the FP32 value of their correction kernels (no FP64 division)
    const double om = 1.0 - ith;
    double Kc;
    if constexpr (std::is_same<R, float>::value) {
        const float eh = eps[c] - P.feps_ref;
        Kc = (double)(3.0f * P.fitau_h * eh * rcp(eh + cs2<float>() * P.ftau_h));
    } else {
        const double eh = (double)eps[c] - P.eps_ref;
        Kc = 3.0 * ith * eh / (eh + Kn);
    }
    // the anchor's flux, for the fields kernel
    ja[c] = R(jx);
    ja[N + c] = R(jy);
    const double A = ith * ps, q8 = 0.125 * (double)q[c];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const double v = j == 0 ? om * h[0] + (wgt<double>(0) - 1.0) * A
                                : om * h[j] + wgt<double>(j) * (A + Kc * cdot<double>(j, jx, jy)) + q8;
        const int yt = y + cy(j);
        if (P.bc_y != 0 && (yt < 0 || yt >= P.ny)) {
            double out = v;
            if (P.bc_y == 2) out = -v + 2.0 * wgt<double>(j) * (yt >= P.ny ? P.V_top : P.V_bottom);
            stage[opp(j) * N + c] = out;
        } else {
            stage[j * N + (unsigned)wrapi(yt, P.ny) * P.nx + wrapi(x + cx(j), P.nx)] = v;
        }
    }
}

// r = stage - a (the anchor's increment over one pseudo-iteration), stored in R,
// and per-block sums of |d psi|^2, |psi|^2, |d J|^2, |J|^2 (psi = sum_{j>0} h_j /
// (1 - w_0), J = sum_j c_j h_j).  Only the subtraction needs FP64 (it cancels O(psi)
// values down to the increment); the increments are then small and the anchor's
// psi and J serve only as denominators, so the sums are taken in R within a thread
// and a warp, and in FP64 across warps.
template <class R>
__global__ void __launch_bounds__(256) k_anchor_residual(DevParams P, const double* __restrict__ a,
                                                         const double* __restrict__ stage, R* __restrict__ r,
                                                         double* __restrict__ partial) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    R acc[4] = {R(0), R(0), R(0), R(0)};
    if (x < P.nx && y < P.ny) {
        const unsigned N = P.N, c = (unsigned)y * P.nx + x;
        R dps = R(0), ps = R(0), djx = R(0), djy = R(0), jx = R(0), jy = R(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const double aj = a[j * N + c];
            const R rj = R(stage[j * N + c] - aj), ar = R(aj);
            r[j * N + c] = rj;
            if (j) { dps += rj; ps += ar; }
            cacc(djx, cx(j), rj);
            cacc(djy, cy(j), rj);
            cacc(jx, cx(j), ar);
            cacc(jy, cy(j), ar);
        }
        dps = dps * R(1.8);
        ps = ps * R(1.8);
        acc[0] = dps * dps;
        acc[1] = ps * ps;
        acc[2] = djx * djx + djy * djy;
        acc[3] = jx * jx + jy * jy;
    }
    block_reduce_store_r<4>(acc, partial + 4 * (size_t)(blockIdx.x + gridDim.x * blockIdx.y));
}

// psi and E = sum c_j h_j / (eps - eps_ref + cs2 tau_h) + E_ext of h = a + delta
// (moments of a in FP64, of delta in R, added in FP64); psi_out != nullptr: write
// psi (FP64) instead of E
template <class R>
__global__ void __launch_bounds__(256) k_anchor_fields(DevParams P, const typename AnchorOf<R>::type* __restrict__ a,
                                                       const R* __restrict__ d, const R* __restrict__ eps,
                                                       R* __restrict__ E, double* __restrict__ psi_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    double ps = 0.0, jx = 0.0, jy = 0.0;
    R dps = R(0), djx = R(0), djy = R(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const double aj = anchor_value(a[j * N + c]);
        const R dj = d[j * N + c];
        if (j) { ps += aj; dps += dj; }
        cacc(jx, cx(j), aj);
        cacc(jy, cy(j), aj);
        cacc(djx, cx(j), dj);
        cacc(djy, cy(j), dj);
    }
    if (psi_out) {
        psi_out[c] = (ps + (double)dps) * 1.8;
        return;
    }
    // the flux in FP64, then the division in R (E is stored in R)
    const R den = (eps[c] - pv<R>(P.eps_ref, P.feps_ref)) + cs2<R>() * pv<R>(P.tau_h, P.ftau_h);
    const R iden = rcp(den);
    E[c] = dv(R(jx + (double)djx), den, iden) + pv<R>(P.E_ext[0], (float)P.E_ext[0]);
    E[N + c] = dv(R(jy + (double)djy), den, iden) + pv<R>(P.E_ext[1], (float)P.E_ext[1]);
}

// E = (J_a + J(delta)) / (eps - eps_ref + cs2 tau_h) + E_ext with J_a the anchor's
// flux stored by the last refresh: no FP64 traffic
template <class R>
__global__ void __launch_bounds__(256) k_anchor_efield(DevParams P, const R* __restrict__ ja, const R* __restrict__ d,
                                                       const R* __restrict__ eps, R* __restrict__ E) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    R jx = ja[c], jy = ja[N + c];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const R dj = d[j * N + c];
        cacc(jx, cx(j), dj);
        cacc(jy, cy(j), dj);
    }
    const R den = (eps[c] - pv<R>(P.eps_ref, P.feps_ref)) + cs2<R>() * pv<R>(P.tau_h, P.ftau_h);
    const R iden = rcp(den);
    E[c] = dv(jx, den, iden) + pv<R>(P.E_ext[0], (float)P.E_ext[0]);
    E[N + c] = dv(jy, den, iden) + pv<R>(P.E_ext[1], (float)P.E_ext[1]);
}

// population j of h = a + delta as FP64
// The starting state of a time step's solve, extrapolated linearly in time: with h =
// a + delta the state the last step's solve ended at and hs the one the step before
// ended at, delta += h - hs (the solve starts from 2h - hs); then hs = h.  With
// extrap = 0 only hs = h (the first step after initialisation).  h and hs in R: the
// extrapolation is a starting guess, so its rounding does not matter.
template <class R>
__global__ void k_anchor_extrapolate(const typename AnchorOf<R>::type* __restrict__ a, R* __restrict__ d,
                                     R* __restrict__ hs, size_t n, int extrap) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    R h;
    if constexpr (std::is_same<R, float>::value) h = __fadd_rn(a[i].hi, __fadd_rn(a[i].lo, d[i]));
    else h = R(anchor_value(a[i]) + (double)d[i]);
    if (extrap) d[i] += h - hs[i];
    hs[i] = h;
}

template <class R>
__global__ void k_anchor_pop(double* __restrict__ dst, const typename AnchorOf<R>::type* __restrict__ a,
                             const R* __restrict__ d, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = anchor_value(a[i]) + (double)d[i];
}

// coarse correction, level-0 input: rhs = sum_{j>0} r_j (the macroscopic residual
// at the anchor), e = 0
template <class R>
__global__ void __launch_bounds__(256) k_lbmg_rhs(DevParams P, const R* __restrict__ r, MGLevelF F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    float s = 0.f;
#pragma unroll
    for (int j = 1; j < 9; ++j) s += (float)r[j * N + c];
    F.rhs[c] = s;
    F.psi[c] = 0.f;
}

// level-0 permittivity (FP64 copy for the coarsening) from the step's eps
template <class R>
__global__ void __launch_bounds__(256) k_lbmg_eps(MGLevel L, const R* __restrict__ eps) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    const int c = y * L.nx + x;
    L.eps[c] = (double)eps[c];
}

// delta = the local equilibrium of the potential correction e plus its first-order
// flux part: delta_0 = (w_0 - 1) e, delta_j = w_j e - w_j (c_j . grad e) den / cs^2,
// den = eps_hat + cs^2 tau_h; grad e by central differences (x periodic; e vanishes
// on the electrode faces, so its ghost beyond a wall is -e)
template <class R>
__global__ void __launch_bounds__(256) k_lbmg_correct(DevParams P, MGLevelF F, const R* __restrict__ eps,
                                                      R* __restrict__ d, int add) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const unsigned N = P.N, c = (unsigned)y * P.nx + x;
    const int nx = P.nx, ny = P.ny;
    const float e = F.psi[c];
    const float ee = F.psi[y * nx + (x + 1 == nx ? 0 : x + 1)], ew = F.psi[y * nx + (x == 0 ? nx - 1 : x - 1)];
    const float en = y + 1 < ny ? F.psi[c + nx] : -e, es = y > 0 ? F.psi[c - nx] : -e;
    const float gx = 0.5f * (ee - ew), gy = 0.5f * (en - es);
    const float den = ((float)eps[c] - P.feps_ref) + P.ftau_h * (1.0f / 3.0f);
    const float k = 3.0f * den;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const float v = j == 0 ? (wgt<float>(0) - 1.f) * e : wgt<float>(j) * (e - k * cdot<float>(j, gx, gy));
        d[j * N + c] = add ? R(d[j * N + c] + R(v)) : R(v);
    }
}

// The increment of the last pseudo-iteration of delta (the same as that of h = a +
// delta): psi and J of the current delta against the values saved before its last
// collision; per-block sums of |d psi|^2, |d J|^2 and of sum_j delta_j^2 (the size of
// delta, which bounds the rounding noise of these increments: FP32 per thread, FP64
// across warps).  With rhs != nullptr also the coarse correction's right-hand
// side, the macroscopic residual sum_{j>0} (delta_j - delta_j^prev) = (1 - w_0) d psi,
// and a zero initial guess.
template <class R>
__global__ void __launch_bounds__(256) k_rs_increment(DevParams P, const R* __restrict__ d,
                                                      const R* __restrict__ prev, double* __restrict__ partial,
                                                      float* __restrict__ rhs, float* __restrict__ e0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    R acc[3] = {R(0), R(0), R(0)};
    if (x < P.nx && y < P.ny) {
        const unsigned N = P.N, c = (unsigned)y * P.nx + x;
        R ps = R(0), jx = R(0), jy = R(0);
        if constexpr (std::is_same<R, float>::value) {  // the moments as the FP32 iteration forms them
            float v[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                v[j] = d[j * N + c];
                acc[2] += v[j] * v[j];
            }
            moments_f32<float>(v, ps, jx, jy);
        } else {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const R v = d[j * N + c];
                if (j) ps += v;
                cacc(jx, cx(j), v);
                cacc(jy, cy(j), v);
                acc[2] += v * v;
            }
        }
        const R s = ps;  // (1 - w_0) psi
        ps = dv(ps, R(1) - wgt<R>(0), R(1.8));
        const R dp = ps - prev[c], ex = jx - prev[N + c], ey = jy - prev[2 * N + c];
        acc[0] = dp * dp;
        acc[1] = ex * ex + ey * ey;
        if (rhs) {
            rhs[c] = (float)(s - (R(1) - wgt<R>(0)) * prev[c]);
            e0[c] = 0.f;
        }
    }
    block_reduce_store_r<3>(acc, partial + 3 * (size_t)(blockIdx.x + gridDim.x * blockIdx.y));
}

// Diagnostic: per-block FP64 sums of r^2 and b^2 for r = b - A psi, the residual of
// psi in the finite-difference form of div(eps grad psi) + q = 0 (5-point stencil,
// harmonic-mean face permittivity; electrode walls as Dirichlet faces at half a cell,
// flux 2 eps_C (V - psi_C), b = q + 2 eps_C V on the wall rows; plain walls carry no
// flux; y periodic when there are no walls)
template <class R>
__global__ void __launch_bounds__(256) k_fd_residual(DevParams P, const double* __restrict__ psi,
                                                     const R* __restrict__ eps, const R* __restrict__ q,
                                                     double* __restrict__ partial) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    double acc[2] = {0.0, 0.0};
    if (x < P.nx && y < P.ny) {
        const int nx = P.nx, ny = P.ny;
        const int c = y * nx + x;
        const double ec = (double)eps[c], pc = psi[c];
        double b = (double)q[c], ap = 0.0;
        auto face = [&](int n) {
            const double en = (double)eps[n];
            ap += 2.0 * ec * en / (ec + en) * (pc - psi[n]);
        };
        face(y * nx + (x + 1 == nx ? 0 : x + 1));
        face(y * nx + (x == 0 ? nx - 1 : x - 1));
        if (y + 1 < ny) face(c + nx);
        else if (P.bc_y == 0) face(x);
        else if (P.bc_y == 2) { ap += 2.0 * ec * pc; b += 2.0 * ec * P.V_top; }
        if (y > 0) face(c - nx);
        else if (P.bc_y == 0) face((ny - 1) * nx + x);
        else if (P.bc_y == 2) { ap += 2.0 * ec * pc; b += 2.0 * ec * P.V_bottom; }
        const double r = b - ap;
        acc[0] = r * r;
        acc[1] = b * b;
    }
    block_reduce_store<2>(acc, partial + 2 * (size_t)(blockIdx.x + gridDim.x * blockIdx.y));
}

}  // namespace lb3e
