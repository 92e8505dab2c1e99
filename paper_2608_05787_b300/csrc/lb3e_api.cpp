// lb3e_api.cpp -- the extern "C" entry points declared in include/lb3e.h.
// Parameter validation, precision dispatch and status mapping; no kernels here.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>

#include "lb3e_internal.h"

struct lb3e_handle {
    lb3e::SimBase* sim;
    lb3e_params params;
};

namespace lb3e {

// every parameter of the model and the run checked for range and finiteness
int validate_params(const lb3e_params* p) {
    if (!p) return LB3E_ERR_NULL;
    if (p->nx < 2 || p->ny < 2) return LB3E_ERR_PARAM;
    if ((int64_t)p->nx * p->ny > LB3E_MAX_CELLS) return LB3E_ERR_PARAM;  // 32-bit plane offsets
    if (p->ny > LB3E_MAX_NY) return LB3E_ERR_PARAM;  // grid y extent of the 32 x 8 tile launches
    if (p->bc_y < 0 || p->bc_y > 2 || p->precision < 0 || p->precision > 5) return LB3E_ERR_PARAM;
    const bool plain = lb3e::plain_precision(p->precision);
    for (int k = 0; k < 3; ++k)
        if (p->tangent_param[k] < -1 || p->tangent_param[k] > 6) return LB3E_ERR_PARAM;
    if (p->potential_solver < 0 || p->potential_solver > 3) return LB3E_ERR_PARAM;
    // multigrid (solver 1, and the coarse correction of solver 2): electrodes, plain
    // precisions, even nx (red-black across the seam); the FP64 anchor (2, 3): plain precisions
    if ((p->potential_solver == 1 || p->potential_solver == 2) && p->electric &&
        (p->bc_y != 2 || !plain || (p->nx & 1)))
        return LB3E_ERR_PARAM;
    if (p->potential_solver == 3 && !plain) return LB3E_ERR_PARAM;
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5) || !(p->width_D > 0) || !(p->eps_ref > 0) || !(p->alpha > 0))
        return LB3E_ERR_PARAM;
    for (int i = 0; i < 3; ++i)
        if (!(p->rho[i] > 0) || !(p->eps[i] > 0) || !(p->sigma[i] >= 0) || !std::isfinite(p->visc[i]))
            return LB3E_ERR_PARAM;
    const double lam[3] = {p->gamma12 + p->gamma13 - p->gamma23, p->gamma12 + p->gamma23 - p->gamma13,
                           p->gamma13 + p->gamma23 - p->gamma12};
    for (double l : lam)
        if (!(l > 0)) return LB3E_ERR_PARAM;
    if (p->inner_phase < 1 || p->inner_phase > 3 || p->matrix_phase < 1 || p->matrix_phase > 3) return LB3E_ERR_PARAM;
    if (p->poisson_max_iter < 0 || p->poisson_fixed_iter < 0) return LB3E_ERR_PARAM;
    const double vals[] = {p->V_bottom, p->V_top, p->E_ext[0], p->E_ext[1], p->u_wall_bottom, p->u_wall_top,
                           p->poisson_tol};
    for (double v : vals)
        if (!std::isfinite(v)) return LB3E_ERR_PARAM;
    if (p->ions < 0 || p->ions > 1) return LB3E_ERR_PARAM;
    if (p->nz < 0 || p->nz > 65535) return LB3E_ERR_PARAM;
    if (p->nz >= 2) {  // the three-dimensional D3Q15 step
        if ((int64_t)p->nx * p->ny * p->nz > LB3E_MAX_CELLS || p->ny > LB3E_MAX_NY) return LB3E_ERR_PARAM;
        if (p->precision > 1 || p->potential_solver != 0 || p->ions) return LB3E_ERR_PARAM;
    }
    if (p->ions) {  // Nernst-Planck ions: plain precisions, positive diffusivities
        if (!plain || !(p->ion_D[0] > 0) || !(p->ion_D[1] > 0)) return LB3E_ERR_PARAM;
        const double iv[] = {p->ion_z[0], p->ion_z[1], p->ion_beta, p->ion_charge};
        for (double v : iv)
            if (!std::isfinite(v)) return LB3E_ERR_PARAM;
    }
    return LB3E_OK;
}

}  // namespace lb3e

namespace {

int validate(const lb3e_params* p) { return lb3e::validate_params(p); }

size_t ws_bytes(const lb3e_params& p) {
    if (p.nz >= 2) return p.precision == 0 ? lb3e::workspace_bytes_3d_f64(p) : lb3e::workspace_bytes_3d_f32(p);
    switch (p.precision) {
        case 0: return lb3e::workspace_bytes_f64(p);
        case 1: return lb3e::workspace_bytes_f32(p);
        case 2: return lb3e::workspace_bytes_f16s(p);
        case 5: return lb3e::workspace_bytes_bf16s(p);
        case 3: return lb3e::workspace_bytes_t32(p);
        default: return lb3e::workspace_bytes_t64(p);
    }
}

// every instance valid, one precision, the same fixed potential iteration count
int validate_batch(const lb3e_params* ps, int32_t n) {
    if (!ps) return LB3E_ERR_NULL;
    if (n < 1) return LB3E_ERR_PARAM;
    int iters = -1;
    for (int i = 0; i < n; ++i) {
        TRY(validate(ps + i));
        if (ps[i].precision != ps[0].precision || !lb3e::plain_precision(ps[i].precision) ||
            ps[i].potential_solver != 0 || ps[i].ions ||
            ps[i].nz >= 2)
            return LB3E_ERR_PARAM;
        if (ps[i].electric) {
            if (ps[i].poisson_fixed_iter <= 0) return LB3E_ERR_PARAM;
            if (iters >= 0 && ps[i].poisson_fixed_iter != iters) return LB3E_ERR_PARAM;
            iters = ps[i].poisson_fixed_iter;
        }
    }
    return LB3E_OK;
}

size_t batch_ws_bytes(const lb3e_params* ps, int n) {
    switch (ps[0].precision) {
        case 0: return lb3e::batch_bytes_f64(ps, n);
        case 1: return lb3e::batch_bytes_f32(ps, n);
        case 5: return lb3e::batch_bytes_bf16s(ps, n);
        default: return lb3e::batch_bytes_f16s(ps, n);
    }
}

}  // namespace

struct lb3e_batch {
    lb3e::BatchBase* b;
};

extern "C" {

int lb3e_workspace_bytes(const lb3e_params* params, size_t* bytes) {
    if (!bytes) return LB3E_ERR_NULL;
    TRY(validate(params));
    *bytes = ws_bytes(*params);
    return LB3E_OK;
}

int lb3e_init(const lb3e_params* params, void* workspace, size_t workspace_bytes, const double* phi_init,
              const double* u_init, const double* q_init, const double* pop_noise, void* stream,
              lb3e_handle** out) {
    if (!out || !phi_init) return LB3E_ERR_NULL;
    *out = nullptr;
    TRY(validate(params));
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 || workspace_bytes < ws_bytes(*params))
        return LB3E_ERR_WORKSPACE;
    lb3e::SimBase* sim = nullptr;
    if (params->nz >= 2) {
        sim = params->precision == 0 ? lb3e::make_sim_3d_f64(*params, workspace, stream)
                                     : lb3e::make_sim_3d_f32(*params, workspace, stream);
    } else switch (params->precision) {
        case 0: sim = lb3e::make_sim_f64(*params, workspace, stream); break;
        case 1: sim = lb3e::make_sim_f32(*params, workspace, stream); break;
        case 2: sim = lb3e::make_sim_f16s(*params, workspace, stream); break;
        case 5: sim = lb3e::make_sim_bf16s(*params, workspace, stream); break;
        case 3: sim = lb3e::make_sim_t32(*params, workspace, stream); break;
        default: sim = lb3e::make_sim_t64(*params, workspace, stream); break;
    }
    if (!sim) return LB3E_ERR_CUDA;
    const int rc = sim->init(phi_init, u_init, q_init, pop_noise);
    if (rc != LB3E_OK) {
        delete sim;
        return rc;
    }
    lb3e_handle* h = new (std::nothrow) lb3e_handle{sim, *params};
    if (!h) {
        delete sim;
        return LB3E_ERR_CUDA;
    }
    *out = h;
    return LB3E_OK;
}

int lb3e_step(lb3e_handle* h, int32_t nsteps) {
    if (!h) return LB3E_ERR_NULL;
    if (nsteps < 0) return LB3E_ERR_PARAM;
    return h->sim->step(nsteps);
}

int lb3e_solve_potential(lb3e_handle* h, const double* q, double tol, int32_t max_iter, int32_t check_every,
                         int32_t* iters, double* residual) {
    if (!h) return LB3E_ERR_NULL;
    if (max_iter < 0 || !std::isfinite(tol)) return LB3E_ERR_PARAM;
    int it = 0;
    double res = -1.0;
    const int rc = h->sim->solve_potential(q, tol, max_iter, check_every, &it, &res);
    if (iters) *iters = it;
    if (residual) *residual = res;
    return rc;
}

int lb3e_observables(lb3e_handle* h, lb3e_observables_t* out) {
    if (!h || !out) return LB3E_ERR_NULL;
    return h->sim->observables(out);
}

int lb3e_get_field(lb3e_handle* h, int32_t field_id, double* dst) {
    if (!h || !dst) return LB3E_ERR_NULL;
    return h->sim->get_field(field_id, dst);
}

int lb3e_state_bytes(const lb3e_handle* h, size_t* bytes) {
    if (!h || !bytes) return LB3E_ERR_NULL;
    *bytes = h->sim->state_bytes();
    return LB3E_OK;
}

int lb3e_save_state(lb3e_handle* h, void* dst) {
    if (!h || !dst) return LB3E_ERR_NULL;
    return h->sim->save(dst);
}

int lb3e_load_state(lb3e_handle* h, const void* src) {
    if (!h || !src) return LB3E_ERR_NULL;
    return h->sim->load(src);
}

int64_t lb3e_launch_count(const lb3e_handle* h) { return h ? h->sim->launches : 0; }

int64_t lb3e_potential_iterations(const lb3e_handle* h) { return h ? h->sim->potential_iterations() : 0; }

int lb3e_set_potential_chunk(lb3e_handle* h, int32_t iterations_per_launch) {
    if (!h) return LB3E_ERR_NULL;
    return h->sim->set_chunk(iterations_per_launch);
}

int lb3e_potential_stats(lb3e_handle* h, int64_t* solves, int64_t* not_converged, double* max_residual) {
    if (!h) return LB3E_ERR_NULL;
    lb3e::SimBase* s = h->sim;
    if (solves) *solves = s->solves;
    if (not_converged) *not_converged = s->unconverged;
    if (max_residual) *max_residual = s->max_residual;
    s->solves = 0;
    s->unconverged = 0;
    s->max_residual = -1.0;
    return LB3E_OK;
}

int lb3e_set_fused_tile(lb3e_handle* h, int32_t rows) {
    if (!h) return LB3E_ERR_NULL;
    return h->sim->set_fused_tile(rows);
}

int lb3e_set_staging(lb3e_handle* h, int32_t planes) {
    if (!h) return LB3E_ERR_NULL;
    if (planes < 0 || planes > 1024) return LB3E_ERR_PARAM;
    return h->sim->set_staging(planes);
}

int lb3e_deformation(lb3e_handle* h, double* D, double* dD) {
    if (!h || !D) return LB3E_ERR_NULL;
    return h->sim->deformation(D, dD);
}

int lb3e_shape_objective(lb3e_handle* h, const double* phi_target, double* J, double* dJ) {
    if (!h || !phi_target || !J) return LB3E_ERR_NULL;
    return h->sim->shape_objective(phi_target, J, dJ);
}

int lb3e_adjoint_workspace_bytes(const lb3e_handle* h, size_t* bytes) {
    if (!h || !bytes) return LB3E_ERR_NULL;
    return h->sim->adjoint_workspace_bytes(bytes);
}

int lb3e_state_vector(lb3e_handle* h, void* dst) {
    if (!h || !dst) return LB3E_ERR_NULL;
    return h->sim->state_vector(dst);
}

int lb3e_adjoint_step(lb3e_handle* h, const void* saved_state, const void* adj_in, void* adj_out,
                      double* dparams, void* adj_workspace, size_t adj_bytes) {
    if (!h || !adj_in || !adj_out || !dparams) return LB3E_ERR_NULL;
    return h->sim->adjoint_step(saved_state, adj_in, adj_out, dparams, adj_workspace, adj_bytes);
}

int lb3e_adjoint_step_x(lb3e_handle* h, const void* X, int32_t first, const void* adj_in, void* adj_out,
                        double* dparams, void* adj_workspace, size_t adj_bytes) {
    if (!h || !X || !adj_in || !adj_out || !dparams) return LB3E_ERR_NULL;
    return h->sim->adjoint_step_x(X, first, adj_in, adj_out, dparams, adj_workspace, adj_bytes);
}

int lb3e_is_first_step(const lb3e_handle* h, int32_t* first) {
    if (!h || !first) return LB3E_ERR_NULL;
    *first = h->sim->first_step();
    return LB3E_OK;
}

int lb3e_adjoint_init(lb3e_handle* h, const double* phi_init, const void* adj_in, double* dparams,
                      double* dphi_init, void* adj_workspace, size_t adj_bytes) {
    if (!h || !phi_init || !adj_in || !dparams) return LB3E_ERR_NULL;
    return h->sim->adjoint_init(phi_init, adj_in, dparams, dphi_init, adj_workspace, adj_bytes);
}

int lb3e_deformation_seed(lb3e_handle* h, int32_t which, double* D, void* adj_out) {
    if (!h || !D || !adj_out) return LB3E_ERR_NULL;
    if (which != 0 && which != 1) return LB3E_ERR_PARAM;
    return h->sim->deformation_seed(which, D, adj_out);
}

int lb3e_shape_seed(lb3e_handle* h, const double* phi_target, double* J, void* adj_out) {
    if (!h || !phi_target || !J || !adj_out) return LB3E_ERR_NULL;
    return h->sim->shape_seed(phi_target, J, adj_out);
}

int lb3e_potential_fd_residual(lb3e_handle* h, double* residual) {
    if (!h || !residual) return LB3E_ERR_NULL;
    return h->sim->fd_residual(residual);
}

int lb3e_set_ions(lb3e_handle* h, const double* n_init) {
    if (!h || !n_init) return LB3E_ERR_NULL;
    return h->sim->set_ions(n_init);
}

int lb3e_set_timing(lb3e_handle* h, int32_t enable) {
    if (!h) return LB3E_ERR_NULL;
    TRY(h->sim->kernel_times(nullptr, nullptr));
    h->sim->timer.enabled = enable != 0;
    return LB3E_OK;
}

int lb3e_kernel_times(lb3e_handle* h, double* ms, int64_t* launches) {
    if (!h || !ms || !launches) return LB3E_ERR_NULL;
    return h->sim->kernel_times(ms, launches);
}

void lb3e_destroy(lb3e_handle* h) {
    if (!h) return;
    delete h->sim;
    delete h;
}

int lb3e_batch_workspace_bytes(const lb3e_params* params, int32_t n, size_t* bytes) {
    if (!bytes) return LB3E_ERR_NULL;
    TRY(validate_batch(params, n));
    *bytes = batch_ws_bytes(params, n);
    return LB3E_OK;
}

int lb3e_batch_create(const lb3e_params* params, int32_t n, const double* const* phi_init, void* workspace,
                      size_t workspace_bytes, void* stream, lb3e_batch** out) {
    if (!out || !phi_init) return LB3E_ERR_NULL;
    *out = nullptr;
    TRY(validate_batch(params, n));
    for (int i = 0; i < n; ++i)
        if (!phi_init[i]) return LB3E_ERR_NULL;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
        workspace_bytes < batch_ws_bytes(params, n))
        return LB3E_ERR_WORKSPACE;
    lb3e::BatchBase* b = nullptr;
    int rc = LB3E_OK;
    switch (params[0].precision) {
        case 0: b = lb3e::new_batch_f64(params, n, workspace, stream); rc = b ? lb3e::init_batch_f64(b, phi_init) : LB3E_ERR_CUDA; break;
        case 1: b = lb3e::new_batch_f32(params, n, workspace, stream); rc = b ? lb3e::init_batch_f32(b, phi_init) : LB3E_ERR_CUDA; break;
        case 5: b = lb3e::new_batch_bf16s(params, n, workspace, stream); rc = b ? lb3e::init_batch_bf16s(b, phi_init) : LB3E_ERR_CUDA; break;
        default: b = lb3e::new_batch_f16s(params, n, workspace, stream); rc = b ? lb3e::init_batch_f16s(b, phi_init) : LB3E_ERR_CUDA; break;
    }
    if (rc != LB3E_OK) {
        delete b;
        return rc;
    }
    lb3e_batch* h = new (std::nothrow) lb3e_batch{b};
    if (!h) {
        delete b;
        return LB3E_ERR_CUDA;
    }
    *out = h;
    return LB3E_OK;
}

int lb3e_batch_set_fused_tile(lb3e_batch* b, int32_t rows) {
    if (!b) return LB3E_ERR_NULL;
    return b->b->set_fused_tile(rows);
}

int lb3e_batch_run(lb3e_batch* b, int32_t nsteps) {
    if (!b) return LB3E_ERR_NULL;
    if (nsteps < 0) return LB3E_ERR_PARAM;
    return b->b->run(nsteps);
}

int lb3e_batch_observables(lb3e_batch* b, lb3e_observables_t* out) {
    if (!b || !out) return LB3E_ERR_NULL;
    return b->b->observables(out);
}

int lb3e_batch_get_field(lb3e_batch* b, int32_t instance, int32_t field_id, double* dst) {
    if (!b || !dst) return LB3E_ERR_NULL;
    return b->b->get_field(instance, field_id, dst);
}

int64_t lb3e_batch_launch_count(const lb3e_batch* b) { return b ? b->b->total_launches() : 0; }

int lb3e_batch_set_potential_chunk(lb3e_batch* b, int32_t iterations_per_launch) {
    if (!b) return LB3E_ERR_NULL;
    return b->b->set_chunk(iterations_per_launch);
}

void lb3e_batch_destroy(lb3e_batch* b) {
    if (!b) return;
    delete b->b;
    delete b;
}

const char* lb3e_status_string(int status) {
    switch (status) {
        case LB3E_OK: return "ok";
        case LB3E_ERR_PARAM: return "invalid parameter";
        case LB3E_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case LB3E_ERR_CUDA: return "CUDA error";
        case LB3E_ERR_NOT_CONVERGED: return "potential solve did not reach the tolerance";
        case LB3E_ERR_FIELD: return "unknown field id";
        case LB3E_ERR_NULL: return "NULL handle or pointer";
        case LB3E_ERR_TOO_LARGE: return "lattice larger than the fixed scratch of lb3e_observables_noalloc";
        case LB3E_ERR_UNSUPPORTED: return "no reverse mode for this configuration";
        default: return "unknown status";
    }
}

}  // extern "C"
