// lb3e_ions.cuh -- Nernst-Planck ion transport (Eq. 52) for the electro-osmotic
// validation of Section 5.1: two ion species with concentrations n_i, each carried
// by its own D2Q9 population set in the form of the charge scheme of Eq. 48-50.
//
//   n^i_j(x + c_j, t + 1) = n^i_j - (n^i_j - n^{i,eq}_j) / tau_i + T^i_j
//   n^{i,eq}_j = w_j n_i (1 + c_j . v_i / cs2),   v_i = u + z_i beta D_i E
//   T^i_j = (1 - 1/(2 tau_i)) w_j c_j . d/dt(n_i v_i) / cs2   (backward difference)
//   tau_i = 1/2 + D_i / cs2,   q = e_q sum_i z_i n_i
//
// v_i is the advection velocity plus the migration velocity along E (beta = e/k_BT,
// the inverse thermal voltage).  Walls bounce the populations back (no flux).
// The charge the ions carry replaces the closure charge of the transported-charge
// scheme.  Layout: 18 planes, species-major (9 i + j) * N + cell, double-buffered;
// the step's n_i (2 planes) and (n_i v_i)^{n-1} (4 planes: x, y per species).
#pragma once

#include "lb3e_kernels.cuh"

namespace lb3e {

// Per-species constants formed on the host in double precision, in the order a
// plain C evaluation takes them (the FP64 build then matches it bit for bit).
struct IonParams {
    double tau[2];   // 1/2 + D_i / cs2
    double itau[2];  // 1 / tau_i (FP32 builds)
    double pre[2];   // 1 - 1 / (2 tau_i)
    double mig[2];   // z_i beta D_i
    double z[2];
    double e;        // charge per unit concentration
    // their FP32 roundings (an FP64 conversion in device code costs FP64 instructions)
    float ftau[2], fitau[2], fpre[2], fmig[2], fz[2], fe;
};

inline IonParams make_ion_params(const lb3e_params& p) {
    IonParams ip{};
    const double c2 = 1.0 / 3.0;
    for (int i = 0; i < 2; ++i) {
        ip.tau[i] = 0.5 + p.ion_D[i] / c2;
        ip.itau[i] = 1.0 / ip.tau[i];
        ip.pre[i] = 1.0 - 1.0 / (2.0 * ip.tau[i]);
        ip.mig[i] = p.ion_z[i] * p.ion_beta * p.ion_D[i];
        ip.z[i] = p.ion_z[i];
    }
    ip.e = p.ion_charge;
    for (int i = 0; i < 2; ++i) {
        ip.ftau[i] = (float)ip.tau[i];
        ip.fitau[i] = (float)ip.itau[i];
        ip.fpre[i] = (float)ip.pre[i];
        ip.fmig[i] = (float)ip.mig[i];
        ip.fz[i] = (float)ip.z[i];
    }
    ip.fe = (float)ip.e;
    return ip;
}

// q = e_q (z_1 n_1 + z_2 n_2) at one cell
template <class R>
__device__ __forceinline__ R ion_charge_of(const IonParams& ip, R n0, R n1) {
    R a = R(0);
    a += pv<R>(ip.z[0], ip.fz[0]) * n0;
    a += pv<R>(ip.z[1], ip.fz[1]) * n1;
    return pv<R>(ip.e, ip.fe) * a;
}

// Moments n_i = sum_j n^i_j of the current ion populations and the charge they carry.
template <class R>
__global__ void __launch_bounds__(256) k_ion_moments(int nx, int ny, const R* __restrict__ ion, R* __restrict__ nion,
                                                     R* __restrict__ q, IonParams ip) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const size_t N = (size_t)nx * ny, c = (size_t)y * nx + x;
    R n[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        R a = R(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) a += ion[(9 * i + j) * N + c];
        n[i] = a;
        nion[i * N + c] = a;
    }
    q[c] = ion_charge_of<R>(ip, n[0], n[1]);
}

// Charge of given concentrations (initial state).
template <class R>
__global__ void k_ion_charge(size_t N, const R* __restrict__ nion, R* __restrict__ q, IonParams ip) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    q[c] = ion_charge_of<R>(ip, nion[c], nion[N + c]);
}

// drift velocity v_i = u + z_i beta D_i E
template <class R>
__device__ __forceinline__ void ion_velocity(const IonParams& ip, int i, size_t N, size_t c, const R* __restrict__ u,
                                             const R* __restrict__ E, R& vx, R& vy) {
    const R m = pv<R>(ip.mig[i], ip.fmig[i]);
    vx = u[c] + m * E[c];
    vy = u[N + c] + m * E[N + c];
}

// Populations at equilibrium with the stored concentrations, u and E.
template <class R>
__global__ void __launch_bounds__(256) k_init_ions(int nx, int ny, R* __restrict__ ion, const R* __restrict__ nion,
                                                   const R* __restrict__ u, const R* __restrict__ E, IonParams ip) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const size_t N = (size_t)nx * ny, c = (size_t)y * nx + x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        R vx, vy;
        ion_velocity<R>(ip, i, N, c, u, E, vx, vy);
        const R n = nion[i * N + c];
#pragma unroll
        for (int j = 0; j < 9; ++j) ion[(9 * i + j) * N + c] = wgt<R>(j) * n * (R(1) + oc2(cdot<R>(j, vx, vy)));
    }
}

// Collision with the u^n and E^n of the step, then push-streaming with bounce-back
// at walls (the step's n_i come from k_ion_moments at its start).
template <class R>
__global__ void __launch_bounds__(256) k_ions(int nx, int ny, int bc_y, const R* __restrict__ in, R* __restrict__ out,
                                              const R* __restrict__ nion, const R* __restrict__ u,
                                              const R* __restrict__ E, R* __restrict__ prev, IonParams ip, int first) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const size_t N = (size_t)nx * ny, c = (size_t)y * nx + x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const R n = nion[i * N + c];
        R vx, vy;
        ion_velocity<R>(ip, i, N, c, u, E, vx, vy);
        const R nvx = n * vx, nvy = n * vy;
        const R dx = first ? R(0) : nvx - prev[(2 * i) * N + c];
        const R dy = first ? R(0) : nvy - prev[(2 * i + 1) * N + c];
        const R tau = pv<R>(ip.tau[i], ip.ftau[i]), itau = pv<R>(ip.itau[i], ip.fitau[i]),
                pre = pv<R>(ip.pre[i], ip.fpre[i]);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const R neq = wgt<R>(j) * n * (R(1) + oc2(cdot<R>(j, vx, vy)));
            const R Tj = oc2(pre * wgt<R>(j) * cdot<R>(j, dx, dy));
            const R nj = in[(9 * i + j) * N + c];
            const R v = nj - dv(nj - neq, tau, itau) + Tj;
            const int yt = y + cy(j);
            if (bc_y != 0 && (yt < 0 || yt >= ny))
                out[(9 * i + opp(j)) * N + c] = v;
            else
                out[(9 * i + j) * N + (size_t)wrapi(yt, ny) * nx + wrapi(x + cx(j), nx)] = v;
        }
        prev[(2 * i) * N + c] = nvx;
        prev[(2 * i + 1) * N + c] = nvy;
    }
}

}  // namespace lb3e
