// lb3e_internal.h -- pieces shared by the precision-specific translation units
// and the C ABI layer (host side only).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/lb3e.h"

#define TRY(expr)                         \
    do {                                  \
        int _rc = (expr);                 \
        if (_rc != LB3E_OK) return _rc;   \
    } while (0)

namespace lb3e {

struct DevParams;

// range and finiteness checks of every lb3e_params field (LB3E_OK or LB3E_ERR_*)
int validate_params(const lb3e_params* p);

// kernel classes for the timing facility (lb3e_kernel_times)
enum KernelClass { KC_MOMENTS = 0, KC_PROLOGUE, KC_POISSON, KC_REDUCE, KC_FIELDS, KC_FUSED, KC_OTHER, KC_IONS,
                   KC_ANCHOR, KC_COARSE, KC_COUNT };

// CUDA-event timing of kernel launches on the simulation's stream (off by default)
struct LaunchTimer {
    bool enabled = false;
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[KC_COUNT] = {0};
    int64_t n[KC_COUNT] = {0};
    cudaEvent_t take() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void begin(cudaStream_t s, int cls) {
        if (!enabled) return;
        Rec r{cls, take(), take()};
        cudaEventRecord(r.a, s);
        recs.push_back(r);
    }
    void end(cudaStream_t s) {
        if (!enabled || recs.empty()) return;
        cudaEventRecord(recs.back().b, s);
    }
    // fold recorded pairs into the totals (the stream must be synchronised)
    void collect() {
        for (auto& r : recs) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) { ms[r.cls] += t; n[r.cls] += 1; }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
    ~LaunchTimer() {
        for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// one simulation, whatever its precision
struct SimBase {
    virtual ~SimBase() = default;
    virtual int init(const double* phi, const double* u, const double* q, const double* noise) = 0;
    virtual int step(int nsteps) = 0;
    virtual int solve_potential(const double* q, double tol, int max_iter, int check, int* iters, double* res) = 0;
    virtual int observables(lb3e_observables_t* out) = 0;
    virtual int get_field(int id, double* dst) = 0;
    virtual size_t state_bytes() const = 0;
    virtual int save(void* dst) = 0;
    virtual int load(const void* src) = 0;
    virtual int kernel_times(double* ms, int64_t* counts) = 0;
    virtual int64_t potential_iterations() const = 0;
    virtual int set_chunk(int k) = 0;
    virtual int set_ions(const double* n) = 0;
    virtual int fd_residual(double* out) = 0;
    virtual int deformation(double* D, double* dD) = 0;
    virtual int shape_objective(const double* target, double* J, double* dJ) = 0;
    virtual int set_fused_tile(int rows) = 0;
    // TMA staging of the D3Q15 potential iteration's inputs (three-dimensional only)
    virtual int set_staging(int planes) { (void)planes; return LB3E_ERR_UNSUPPORTED; }
    // reverse mode (two-dimensional plain builds with a fixed potential count)
    virtual int adjoint_workspace_bytes(size_t* bytes) { (void)bytes; return LB3E_ERR_UNSUPPORTED; }
    virtual int state_vector(void* dst) { (void)dst; return LB3E_ERR_UNSUPPORTED; }
    virtual int adjoint_step(const void* state, const void* a_in, void* a_out, double* dparams, void* ws,
                             size_t bytes) {
        (void)state; (void)a_in; (void)a_out; (void)dparams; (void)ws; (void)bytes;
        return LB3E_ERR_UNSUPPORTED;
    }
    virtual int adjoint_init(const double* phi, const void* a_in, double* dparams, double* dphi, void* ws,
                             size_t bytes) {
        (void)phi; (void)a_in; (void)dparams; (void)dphi; (void)ws; (void)bytes;
        return LB3E_ERR_UNSUPPORTED;
    }
    virtual int first_step() const { return 0; }
    virtual int adjoint_step_x(const void* X, int first, const void* a_in, void* a_out, double* dparams, void* ws,
                               size_t bytes) {
        (void)X; (void)first; (void)a_in; (void)a_out; (void)dparams; (void)ws; (void)bytes;
        return LB3E_ERR_UNSUPPORTED;
    }
    virtual int deformation_seed(int which, double* D, void* a_out) {
        (void)which; (void)D; (void)a_out;
        return LB3E_ERR_UNSUPPORTED;
    }
    virtual int shape_seed(const double* target, double* J, void* a_out) {
        (void)target; (void)J; (void)a_out;
        return LB3E_ERR_UNSUPPORTED;
    }
    int64_t launches = 0;
    LaunchTimer timer;
    // potential solves since the last lb3e_potential_stats call: count, how many
    // ended above the tolerance (cap or stall), the largest final residual
    int64_t solves = 0, unconverged = 0;
    double max_residual = -1.0;
    void record_solve(int conv, double res) {
        ++solves;
        if (conv != 1) ++unconverged;
        if (res > max_residual) max_residual = res;
    }
};

// a batch of lattices of one precision, stepped together
struct BatchBase {
    virtual ~BatchBase() = default;
    virtual int run(int nsteps) = 0;
    virtual int observables(lb3e_observables_t* out) = 0;
    virtual int get_field(int inst, int id, double* dst) = 0;
    virtual int count() const = 0;
    virtual int64_t total_launches() const = 0;
    virtual int set_chunk(int k) = 0;
    virtual int set_fused_tile(int rows) = 0;
    int64_t launches = 0;
};

// factories, one per translation unit (precision)
size_t workspace_bytes_f64(const lb3e_params& p);
SimBase* make_sim_f64(const lb3e_params& p, void* ws, void* stream);
size_t workspace_bytes_f32(const lb3e_params& p);
SimBase* make_sim_f32(const lb3e_params& p, void* ws, void* stream);
size_t workspace_bytes_f16s(const lb3e_params& p);
SimBase* make_sim_f16s(const lb3e_params& p, void* ws, void* stream);
size_t workspace_bytes_t32(const lb3e_params& p);
SimBase* make_sim_t32(const lb3e_params& p, void* ws, void* stream);
size_t workspace_bytes_t64(const lb3e_params& p);
SimBase* make_sim_t64(const lb3e_params& p, void* ws, void* stream);
size_t workspace_bytes_3d_f64(const lb3e_params& p);
SimBase* make_sim_3d_f64(const lb3e_params& p, void* ws, void* stream);
size_t workspace_bytes_3d_f32(const lb3e_params& p);
SimBase* make_sim_3d_f32(const lb3e_params& p, void* ws, void* stream);
size_t batch_bytes_f64(const lb3e_params* ps, int n);
BatchBase* new_batch_f64(const lb3e_params* ps, int n, void* ws, void* stream);
int init_batch_f64(BatchBase* b, const double* const* phis);
size_t batch_bytes_f32(const lb3e_params* ps, int n);
BatchBase* new_batch_f32(const lb3e_params* ps, int n, void* ws, void* stream);
int init_batch_f32(BatchBase* b, const double* const* phis);
size_t batch_bytes_f16s(const lb3e_params* ps, int n);
BatchBase* new_batch_f16s(const lb3e_params* ps, int n, void* ws, void* stream);
int init_batch_f16s(BatchBase* b, const double* const* phis);
size_t workspace_bytes_bf16s(const lb3e_params& p);
SimBase* make_sim_bf16s(const lb3e_params& p, void* ws, void* stream);
size_t batch_bytes_bf16s(const lb3e_params* ps, int n);
BatchBase* new_batch_bf16s(const lb3e_params* ps, int n, void* ws, void* stream);
int init_batch_bf16s(BatchBase* b, const double* const* phis);

// Deformation factor (a - b)/(a + b) of an indicator from its moments m = (sum chi,
// chi x, chi y, chi x^2, chi y^2), with a = 2 sqrt(Iyy), b = 2 sqrt(Ixx) the radii
// along and across the field (y); and its derivative along a tangent dm of those
// moments (0 where the radii vanish).
inline double deformation_of(const double* m, const double* dm, double* dD) {
    if (dD) *dD = 0.0;
    const double A = m[0];
    if (!(A > 0)) return 0.0;
    const double xc = m[1] / A, yc = m[2] / A;
    const double Ixx = m[3] / A - xc * xc, Iyy = m[4] / A - yc * yc;
    if (!(Ixx > 0) || !(Iyy > 0)) return 0.0;
    const double a = 2.0 * std::sqrt(Iyy), b = 2.0 * std::sqrt(Ixx);
    if (dD && dm) {
        const double dxc = (dm[1] - xc * dm[0]) / A, dyc = (dm[2] - yc * dm[0]) / A;
        const double dIxx = (dm[3] - (m[3] / A) * dm[0]) / A - 2.0 * xc * dxc;
        const double dIyy = (dm[4] - (m[4] / A) * dm[0]) / A - 2.0 * yc * dyc;
        const double da = dIyy / std::sqrt(Iyy), db = dIxx / std::sqrt(Ixx);  // d(2 sqrt(I)) = dI / sqrt(I)
        *dD = 2.0 * (b * da - a * db) / ((a + b) * (a + b));
    }
    return (a - b) / (a + b);
}

// precision codes: the plain builds (one arithmetic type, populations stored in it
// or in a narrower type) and the dual-number tangent builds
inline bool plain_precision(int prec) { return prec == 0 || prec == 1 || prec == 2 || prec == 5; }

}  // namespace lb3e
