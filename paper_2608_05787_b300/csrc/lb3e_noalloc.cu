// lb3e_noalloc.cu -- lb3e_observables_noalloc: the observables reductions for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need these
// numbers: code running inside a memory pool that must not grow, a process whose
// allocator is owned by another framework, or a monitoring hook that must not
// disturb the caller's memory.  For them this file keeps the reduction scratch
// (per-block FP64 partial sums and the final sums) in a fixed file-scope device
// array instead of the caller's workspace.  Every GPU that loads the library holds
// that array until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "lb3e_internal.h"
#include "lb3e_kernels.cuh"
#include "lb3e_params.cuh"

namespace lb3e {

// Blocks of 32 x 8 threads: at most 16384 of them for 4 194 304 cells (2048 x 2048).
// The observables grid (32 x 64 cells a block) needs about an eighth of that; the
// size check in the entry point makes sure its NOBS sums and block maxima fit.
constexpr int kNoallocMaxBlocks = LB3E_NOALLOC_MAX_CELLS / (TX * TY);
constexpr int kNoallocSlots = kNoallocMaxBlocks * NOBS + 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocSlots];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (set up once per device)
int scratch_for_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LB3E_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LB3E_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return LB3E_OK;
}
// the host-side finish of the reductions (deformation factors from the moments)
void finish_observables(const double* v, lb3e_observables_t* o) {
    *o = lb3e_observables_t{};
    for (int i = 0; i < 3; ++i) o->mass[i] = v[i];
    o->charge = v[3];
    for (int k = 0; k < 4; ++k) o->free_energy[k] = v[4 + k];
    o->nonfinite = (int64_t)v[8];
    double Dk[2];
    for (int k = 0; k < 2; ++k) {
        const double* m = v + 9 + 5 * k;
        const double A = m[0];
        if (!(A > 0)) { Dk[k] = 0.0; continue; }
        const double xc = m[1] / A, yc = m[2] / A;
        const double Ixx = m[3] / A - xc * xc, Iyy = m[4] / A - yc * yc;
        const double a = 2.0 * std::sqrt(Iyy > 0 ? Iyy : 0.0), b = 2.0 * std::sqrt(Ixx > 0 ? Ixx : 0.0);
        Dk[k] = (a + b) > 0 ? (a - b) / (a + b) : 0.0;
    }
    o->D_inner = Dk[0];
    o->D_outer = Dk[1];
    o->max_sum_dev = v[NOBS];
}
}  // namespace

}  // namespace lb3e

extern "C" int lb3e_observables_noalloc(const lb3e_params* params, const double* phi, const double* q,
                                        const double* E, const double* u, void* stream,
                                        lb3e_observables_t* out) {
    using namespace lb3e;
    if (!params || !phi || !q || !E || !u || !out) return LB3E_ERR_NULL;
    // the same checks as lb3e_init (ranges, positivity, finiteness), then the
    // limits of this entry point: two-dimensional lattices within the fixed scratch
    if (params->nx < 2 || params->ny < 2) return LB3E_ERR_PARAM;
    if ((int64_t)params->nx * params->ny > LB3E_NOALLOC_MAX_CELLS) return LB3E_ERR_TOO_LARGE;
    TRY(validate_params(params));
    if (params->nz >= 2) return LB3E_ERR_PARAM;
    const dim3 grid = obs_grid(params->nx, params->ny);
    const int64_t nblk64 = (int64_t)grid.x * grid.y;
    // NOBS sums and one max per block must fit before the result slots
    if (nblk64 * (NOBS + 1) > (int64_t)kNoallocMaxBlocks * NOBS) return LB3E_ERR_TOO_LARGE;
    const int nblk = (int)nblk64;

    double* scratch = nullptr;
    TRY(scratch_for_current_device(&scratch));
    double* partial = scratch;  // nblk * NOBS sums, then nblk maxima, each written by its block
    double* result = scratch + (size_t)kNoallocMaxBlocks * NOBS;  // NOBS + 1 slots, written by the final kernels
    const DevParams dp = make_dev_params(*params);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Every slot read below is written earlier in this same call, so nothing
    // needs clearing; the array keeps the last call's values afterwards.
    k_observables<double><<<grid, dim3(TX, TY), 0, st>>>(dp, phi, q, E, u, partial, partial + (size_t)nblk * NOBS);
    k_reduce_partials<NOBS><<<1, 256, 0, st>>>(partial, nblk, result);
    k_max_partials<<<1, 256, 0, st>>>(partial + (size_t)nblk * NOBS, nblk, result + NOBS);
    if (cudaGetLastError() != cudaSuccess) return LB3E_ERR_CUDA;
    double v[NOBS + 1];
    if (cudaMemcpyAsync(v, result, sizeof v, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LB3E_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LB3E_ERR_CUDA;
    finish_observables(v, out);
    out->poisson_residual = -1.0;
    return LB3E_OK;
}
