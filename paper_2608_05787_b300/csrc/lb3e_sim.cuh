// lb3e_sim.cuh -- host-side sequencing of the kernels for one precision.
//
// Sim<R,S> owns no device memory: it carves the caller's workspace into the
// buffers listed in DevState and issues every kernel on the caller's stream.
// The potential solve is a host loop of pseudo-iterations; every
// poisson_check_every iterations one FP64 residual is read back to pinned host
// memory (the only device->host traffic of a time step).
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <utility>
#include <vector>

#include "lb3e_adjoint.cuh"
#include "lb3e_anchor.cuh"
#include "lb3e_internal.h"
#include "lb3e_ions.cuh"
#include "lb3e_kernels.cuh"
#include "lb3e_mg.cuh"

namespace lb3e {

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <class R, class S>
class Sim final : public SimBase {
  public:
    // workspace layout (byte offsets), computed identically by bytes() and the constructor
    struct Layout {
        size_t pop[2], h[2], phi, qt, q, eps, E, prev, diag, psi_prev, partial, result, stage, mg, ion[2], ionst,
            anchor, rres, ja, phi2, anchor2, hprev, total;
    };
    static Layout layout(const lb3e_params& p) {
        const size_t N = (size_t)p.nx * p.ny;
        const size_t nblk = (size_t)((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
        Layout L{};
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t a = o; o += align256(bytes); return a; };
        L.pop[0] = take(45 * N * sizeof(S));
        L.pop[1] = take(45 * N * sizeof(S));
        L.h[0] = take(9 * N * sizeof(R));
        L.h[1] = take(9 * N * sizeof(R));
        L.phi = take(3 * N * sizeof(R));
        L.qt = take(N * sizeof(R));
        L.q = take(N * sizeof(R));
        L.eps = take(N * sizeof(R));
        L.E = take(2 * N * sizeof(R));
        L.prev = take(8 * N * sizeof(R));
        L.diag = take(6 * N * sizeof(R));
        L.psi_prev = take(3 * N * sizeof(R));
        // the other set of phi planes: the moments pass reads the previous step's phi
        // (the rest populations' anchor) from one set and writes the new phi to the other
        L.phi2 = take(3 * N * sizeof(R));
        // per-block partials: NOBS per 32 x 8 tile, or the observables' NOBS sums
        // and one max per 32 x 64 block, whichever is larger
        const dim3 og = obs_grid(p.nx, p.ny);
        const size_t nobs = (size_t)og.x * og.y * (NOBS + 1);
        L.partial = take((nblk * NOBS > nobs ? nblk * NOBS : nobs) * sizeof(double));
        L.result = take(64 * sizeof(double));
        // FP64 staging: 9 planes, or room for 4 planes of R after the first plane
        L.stage = take(9 * N * sizeof(double) > N * sizeof(double) + 4 * N * sizeof(R)
                           ? 9 * N * sizeof(double)
                           : N * sizeof(double) + 4 * N * sizeof(R));
        // multigrid levels (finite-difference potential only): FP64 psi, rhs, res, eps
        // and coefficients; FP32 error-equation psi, rhs, res and coefficients
        size_t mg = 0;
        if ((p.potential_solver == 1 || p.potential_solver == 2) && p.electric) {
            const int nl = mg_levels(p.nx, p.ny);
            for (int l = 0; l < nl; ++l) {
                const size_t n = (size_t)(p.nx >> l) * (p.ny >> l);
                mg += 8 * align256(n * sizeof(double)) + 7 * align256(n * sizeof(float));
            }
        }
        L.mg = take(mg);
        // Nernst-Planck ions: 2 x 18 population planes, then n_i (2 planes) and
        // (n_i v_i)^{n-1} (4 planes) in one block
        const size_t ni = p.ions ? N : 0;
        L.ion[0] = take(18 * ni * sizeof(R));
        L.ion[1] = take(18 * ni * sizeof(R));
        L.ionst = take(6 * ni * sizeof(R));
        // LB potential on an FP64 anchor (solvers 2, 3): the anchor's 9 FP64 planes
        // and its increment's 9 planes in R
        const size_t na = (p.potential_solver >= 2 && p.electric) ? N : 0;
        L.anchor = take(9 * na * sizeof(double));
        L.rres = take(9 * na * sizeof(R));
        L.ja = take(2 * na * sizeof(R));
        // FP32 builds: a second set of anchor planes (the one-pass refresh writes the
        // folded anchor there while neighbouring blocks read the current one)
        L.anchor2 = take(9 * (std::is_same<R, float>::value ? na : 0) * sizeof(double));
        // the state the step before last ended at (the time extrapolation of the
        // solve's starting state)
        L.hprev = take(9 * na * sizeof(R));
        L.total = o;
        return L;
    }

    Sim(const lb3e_params& prm, void* ws, cudaStream_t st) : p_(prm), stream_(st) {
        L_ = layout(prm);
        char* b = static_cast<char*>(ws);
        d_.pop[0] = reinterpret_cast<S*>(b + L_.pop[0]);
        d_.pop[1] = reinterpret_cast<S*>(b + L_.pop[1]);
        d_.h[0] = reinterpret_cast<R*>(b + L_.h[0]);
        d_.h[1] = reinterpret_cast<R*>(b + L_.h[1]);
        d_.phi = reinterpret_cast<R*>(b + L_.phi);
        phi_alt_ = reinterpret_cast<R*>(b + L_.phi2);
        d_.qt = reinterpret_cast<R*>(b + L_.qt);
        d_.q = reinterpret_cast<R*>(b + L_.q);
        d_.eps = reinterpret_cast<R*>(b + L_.eps);
        d_.E = reinterpret_cast<R*>(b + L_.E);
        d_.prev = reinterpret_cast<R*>(b + L_.prev);
        d_.diag = reinterpret_cast<R*>(b + L_.diag);
        d_.psi_prev = reinterpret_cast<R*>(b + L_.psi_prev);
        d_.partial = reinterpret_cast<double*>(b + L_.partial);
        d_.result = reinterpret_cast<double*>(b + L_.result);
        d_.stage = reinterpret_cast<double*>(b + L_.stage);
        base_ = b;
        N_ = (size_t)prm.nx * prm.ny;
        if (prm.ions) {
            ion_[0] = reinterpret_cast<R*>(b + L_.ion[0]);
            ion_[1] = reinterpret_cast<R*>(b + L_.ion[1]);
            nion_ = reinterpret_cast<R*>(b + L_.ionst);
            ionprev_ = nion_ + 2 * N_;
            ip_ = make_ion_params(prm);
        }
        dp_ = make_dev_params(prm);
        grid2_ = dim3((prm.nx + TX - 1) / TX, (prm.ny + TY - 1) / TY);
        nblk_ = (int)(grid2_.x * grid2_.y);
        if (prm.electric && prm.potential_solver >= 2) {
            anchor_ = reinterpret_cast<AT*>(b + L_.anchor);
            if (std::is_same<R, float>::value) anchor_alt_ = reinterpret_cast<AT*>(b + L_.anchor2);
            hprev_ = reinterpret_cast<R*>(b + L_.hprev);
            rres_ = reinterpret_cast<R*>(b + L_.rres);
            ja_ = reinterpret_cast<R*>(b + L_.ja);
            const double ith = 1.0 / dp_.tau_h, w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w5 = 1.0 / 36.0;
            acoef_ = {df_of(1.0 - ith), df_of(ith), df_of(w0 - 1.0), df_of(w1), df_of(w5), df_of(1.0 / (1.0 - w0)),
                      {{df_of(2 * w1 * dp_.V_bottom), df_of(2 * w5 * dp_.V_bottom)},
                       {df_of(2 * w1 * dp_.V_top), df_of(2 * w5 * dp_.V_top)}}};
        }
        if ((prm.potential_solver == 1 || prm.potential_solver == 2) && prm.electric) {
            const int nl = mg_levels(prm.nx, prm.ny);
            char* m = b + L_.mg;
            for (int l = 0; l < nl; ++l) {
                MGLevel v;
                v.nx = prm.nx >> l;
                v.ny = prm.ny >> l;
                const size_t sz = align256((size_t)v.nx * v.ny * sizeof(double));
                v.psi = reinterpret_cast<double*>(m);
                v.rhs = reinterpret_cast<double*>(m + sz);
                v.res = reinterpret_cast<double*>(m + 2 * sz);
                v.eps = reinterpret_cast<double*>(m + 3 * sz);
                v.ae = reinterpret_cast<double*>(m + 4 * sz);
                v.an = reinterpret_cast<double*>(m + 5 * sz);
                v.dg = reinterpret_cast<double*>(m + 6 * sz);
                v.idg = reinterpret_cast<double*>(m + 7 * sz);
                m += 8 * sz;
                mg_.push_back(v);
                MGLevelF f;
                f.nx = v.nx;
                f.ny = v.ny;
                const size_t fz = align256((size_t)v.nx * v.ny * sizeof(float));
                f.psi = reinterpret_cast<float*>(m);
                f.rhs = reinterpret_cast<float*>(m + fz);
                f.res = reinterpret_cast<float*>(m + 2 * fz);
                f.eps = nullptr;
                f.ae = reinterpret_cast<float*>(m + 3 * fz);
                f.an = reinterpret_cast<float*>(m + 4 * fz);
                f.dg = reinterpret_cast<float*>(m + 5 * fz);
                f.idg = reinterpret_cast<float*>(m + 6 * fz);
                m += 7 * fz;
                mgf_.push_back(f);
            }
        }
    }
    ~Sim() override {
        if (pinned_) cudaFreeHost(pinned_);
        if (vgraph_) cudaGraphExecDestroy(vgraph_);
        for (auto& g : adj_graphs_) cudaGraphExecDestroy(g.exec);
    }

    int init(const double* phi, const double* u, const double* q, const double* noise) override {
        if constexpr (fused_dyn_smem<R, S>() > 0) {
            if (cudaFuncSetAttribute(k_fused<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)fused_dyn_smem<R, S>()) != cudaSuccess)
                return LB3E_ERR_CUDA;
            if constexpr (!is_dual<R>::value) {
                if (cudaFuncSetAttribute(k_fused<R, S, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_dyn_smem<R, S, 4>()) != cudaSuccess)
                    return LB3E_ERR_CUDA;
            }
            if constexpr (std::is_same<R, float>::value) {
                if (cudaFuncSetAttribute(k_fused<R, S, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_dyn_smem<R, S, 16>()) != cudaSuccess)
                    return LB3E_ERR_CUDA;
            }
        }
        if (cudaHostAlloc(reinterpret_cast<void**>(&pinned_), 64 * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
            return LB3E_ERR_CUDA;
        pinned_[63] = 0.0;
        TRY(memset_async(err_flag(), sizeof(int)));
        hprev_valid_ = 0;  // the first step's solve starts from the initial solution
        // phi, u, q -> device fields (through the FP64 staging area)
        TRY(upload(phi, 3 * N_, d_.phi));
        if (u) {
            TRY(upload(u, 2 * N_, d_.diag));
        } else {
            TRY(memset_async(d_.diag, 2 * N_ * sizeof(R)));
        }
        if (q) {
            TRY(upload(q, N_, d_.q));
        } else {
            TRY(memset_async(d_.q, N_ * sizeof(R)));
        }
        TRY(memset_async(d_.prev, 8 * N_ * sizeof(R)));
        TRY(memset_async(d_.psi_prev, 3 * N_ * sizeof(R)));
        cur_ = 0;
        hcur_ = 0;
        // permittivity of the initial phase field
        timer.begin(stream_, KC_PROLOGUE);
        k_prologue<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.phi, d_.qt, d_.E, d_.q, d_.eps, 0);
        TRY(launched());
        timer.begin(stream_, KC_OTHER);
        k_init_h<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.h[0]);
        TRY(launched());
        if constexpr (!is_dual<R>::value) {
            if (anchor_) {
                timer.begin(stream_, KC_OTHER);
                k_anchor_init<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, anchor_, d_.h[0]);
                TRY(launched());
            }
        }
        if (p_.electric && p_.potential_solver == 1) {
            timer.begin(stream_, KC_OTHER);
            k_mg_init<<<mg_grid(0), dim3(TX, TY), 0, stream_>>>(mg_[0], p_.V_bottom, p_.V_top);
            TRY(launched());
            TRY(potential());
        } else if (p_.electric) {
            TRY(potential());
        } else {
            timer.begin(stream_, KC_OTHER);
            k_fill_E<R><<<blocks1(N_), 256, 0, stream_>>>(dp_, d_.E);
            TRY(launched());
        }
        timer.begin(stream_, KC_OTHER);
        k_init_pops<R, S><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.pop[0], d_.phi, d_.q, d_.E, d_.diag);
        TRY(launched());
        if (noise) {
            for (int set = 0; set < 5; ++set) {
                if (cudaMemcpyAsync(d_.stage, noise + (size_t)set * 9 * N_, 9 * N_ * sizeof(double),
                                    cudaMemcpyDefault, stream_) != cudaSuccess)
                    return LB3E_ERR_CUDA;
                timer.begin(stream_, KC_OTHER);
                k_add_noise<R, S><<<blocks1(9 * N_), 256, 0, stream_>>>(dp_, d_.pop[0], d_.stage, set);
                TRY(launched());
            }
        }
        step_ = 0;
        return sync();
    }

    int step(int nsteps) override {
        for (int s = 0; s < nsteps; ++s) {
            const int last = (s == nsteps - 1);
            // moments, properties and the closed-form charge in one pass: the new phi
            // goes to the other set of planes (the current set is the anchor of the
            // rest populations, read by the neighbouring blocks for their rings)
            timer.begin(stream_, KC_MOMENTS);
            k_moments_closure<R, S><<<mc_grid(), dim3(TX, TY), 0, stream_>>>(dp_, d_.pop[cur_], d_.phi, phi_alt_, d_.E,
                                                                           d_.q, d_.eps, p_.ions ? 0 : 1);
            TRY(launched());
            std::swap(d_.phi, phi_alt_);
            if constexpr (!is_dual<R>::value) {
                if (p_.ions) {  // the charge the ions carry replaces the closure charge
                    timer.begin(stream_, KC_IONS);
                    k_ion_moments<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(p_.nx, p_.ny, ion_[icur_], nion_, d_.q, ip_);
                    TRY(launched());
                }
            }
            if (p_.electric) {
                in_step_ = true;
                const int rc = potential();
                in_step_ = false;
                TRY(rc);
            }
            timer.begin(stream_, KC_FUSED);
            fused_launch(step_ == 0 ? 1 : 0, (last || p_.ions) ? 1 : 0);
            TRY(launched());
            if constexpr (!is_dual<R>::value) {
                if (p_.ions) {  // with the u^n (diag) and E^n of this step
                    timer.begin(stream_, KC_IONS);
                    k_ions<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(p_.nx, p_.ny, p_.bc_y, ion_[icur_], ion_[icur_ ^ 1],
                                                                    nion_, d_.diag, d_.E, ionprev_, ip_,
                                                                    step_ == 0 ? 1 : 0);
                    TRY(launched());
                    icur_ ^= 1;
                }
            }
            cur_ ^= 1;
            ++step_;
        }
        return LB3E_OK;
    }

    int solve_potential(const double* q, double tol, int max_iter, int check, int* iters, double* res) override {
        if (q) TRY(upload(q, N_, d_.q));
        TRY(potential(tol, max_iter, 0, check));
        if (iters) *iters = last_iters_;
        if (res) *res = last_res_;
        TRY(sync());
        return last_conv_ == 1 ? LB3E_OK : LB3E_ERR_NOT_CONVERGED;
    }

    int set_ions(const double* n) override {
        if constexpr (is_dual<R>::value) {
            return LB3E_ERR_PARAM;
        } else {
            if (!p_.ions || step_ != 0) return LB3E_ERR_PARAM;
            TRY(upload(n, 2 * N_, nion_));
            timer.begin(stream_, KC_OTHER);
            k_ion_charge<R><<<blocks1(N_), 256, 0, stream_>>>(N_, nion_, d_.q, ip_);
            TRY(launched());
            if (p_.electric) TRY(potential());
            icur_ = 0;
            timer.begin(stream_, KC_OTHER);
            k_init_ions<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(p_.nx, p_.ny, ion_[0], nion_, d_.diag, d_.E, ip_);
            TRY(launched());
            TRY(memset_async(ionprev_, 4 * N_ * sizeof(R)));
            return sync();
        }
    }

    int observables(lb3e_observables_t* o) override {
        timer.begin(stream_, KC_REDUCE);
        // sums in partial[0, nb * NOBS), block maxima after them (the layout sizes
        // the partial area for both)
        const dim3 og = obs_grid(p_.nx, p_.ny);
        const int nb = (int)(og.x * og.y);
        k_observables<R><<<og, dim3(TX, TY), 0, stream_>>>(dp_, d_.phi, d_.q, d_.E, d_.diag, d_.partial,
                                                          d_.partial + (size_t)nb * NOBS);
        TRY(launched());
        timer.begin(stream_, KC_REDUCE);
        k_reduce_partials<NOBS><<<1, 256, 0, stream_>>>(d_.partial, nb, d_.result);
        TRY(launched());
        timer.begin(stream_, KC_REDUCE);
        k_max_partials<<<1, 256, 0, stream_>>>(d_.partial + (size_t)nb * NOBS, nb, d_.result + NOBS);
        TRY(launched());
        if (cudaMemcpyAsync(pinned_, d_.result, (NOBS + 1) * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
            cudaSuccess)
            return LB3E_ERR_CUDA;
        TRY(sync());
        const double* v = pinned_;
        std::memset(o, 0, sizeof(*o));
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
        o->poisson_residual = last_res_;
        o->poisson_iters = last_iters_;
        o->poisson_converged = last_conv_;
        o->step = step_;
        return LB3E_OK;
    }

    int get_field(int id, double* dst) override {
        const R* src = nullptr;
        int comp = 0;  // tangent builds: component 0 value, k >= 1 tangent k-1
        if (id >= LB3E_TANGENT) {
            comp = id / LB3E_TANGENT;
            id %= LB3E_TANGENT;
            if constexpr (is_dual<R>::value) {
                if (comp > (int)(sizeof(R().d) / sizeof(R().d[0]))) return LB3E_ERR_FIELD;
            } else {
                return LB3E_ERR_FIELD;
            }
        }
        switch (id) {
            case LB3E_FIELD_PHI1: case LB3E_FIELD_PHI2: case LB3E_FIELD_PHI3: src = d_.phi + (id - LB3E_FIELD_PHI1) * N_; break;
            case LB3E_FIELD_UX: src = d_.diag; break;
            case LB3E_FIELD_UY: src = d_.diag + N_; break;
            case LB3E_FIELD_P: src = d_.diag + 2 * N_; break;
            case LB3E_FIELD_Q: src = d_.q; break;
            case LB3E_FIELD_EX: src = d_.E; break;
            case LB3E_FIELD_EY: src = d_.E + N_; break;
            case LB3E_FIELD_MU1: case LB3E_FIELD_MU2: case LB3E_FIELD_MU3: src = d_.diag + (3 + id - LB3E_FIELD_MU1) * N_; break;
            case LB3E_FIELD_PSI:
                if (comp) return LB3E_ERR_FIELD;
                if (p_.potential_solver == 1 && !mg_.empty()) return copy_out(dst, mg_[0].psi);
                TRY(psi_to_stage());
                return copy_out(dst, d_.stage);
            case LB3E_FIELD_PHINOW1: case LB3E_FIELD_PHINOW2: case LB3E_FIELD_PHINOW3: case LB3E_FIELD_QTILDE: {
                // moments of the current populations into scratch planes of the other buffer's view
                R* tmp = reinterpret_cast<R*>(d_.stage + N_);  // 4 N R-values after the output plane
                timer.begin(stream_, KC_MOMENTS);
                k_moments<R, S><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.pop[cur_], d_.phi, tmp, tmp + 3 * N_);
                TRY(launched());
                const R* t = id == LB3E_FIELD_QTILDE ? tmp + 3 * N_ : tmp + (id - LB3E_FIELD_PHINOW1) * N_;
                timer.begin(stream_, KC_OTHER);
                k_comp_to_f64<R><<<blocks1(N_), 256, 0, stream_>>>(d_.stage, t, N_, comp);
                TRY(launched());
                return copy_out(dst, d_.stage);
            }
            case LB3E_FIELD_N1: case LB3E_FIELD_N2:
                if constexpr (is_dual<R>::value) {
                    return LB3E_ERR_FIELD;
                } else {
                    if (!p_.ions || comp) return LB3E_ERR_FIELD;
                    // moments of the current ion populations into scratch after the output plane
                    R* tmp = reinterpret_cast<R*>(d_.stage + N_);
                    timer.begin(stream_, KC_MOMENTS);
                    k_ion_moments<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(p_.nx, p_.ny, ion_[icur_], tmp, tmp + 2 * N_, ip_);
                    TRY(launched());
                    timer.begin(stream_, KC_OTHER);
                    k_to_f64<R><<<blocks1(N_), 256, 0, stream_>>>(d_.stage, tmp + (id - LB3E_FIELD_N1) * N_, N_);
                    TRY(launched());
                    return copy_out(dst, d_.stage);
                }
            default: break;
        }
        if (!src && id >= LB3E_FIELD_POP + 54 && id < LB3E_FIELD_POP + 72) {
            if (!p_.ions || comp) return LB3E_ERR_FIELD;
            timer.begin(stream_, KC_OTHER);
            k_to_f64<R><<<blocks1(N_), 256, 0, stream_>>>(d_.stage, ion_[icur_] + (size_t)(id - LB3E_FIELD_POP - 54) * N_, N_);
            TRY(launched());
            return copy_out(dst, d_.stage);
        }
        if (!src && id >= LB3E_FIELD_POP && id < LB3E_FIELD_POP + 54) {
            if (comp) return LB3E_ERR_FIELD;
            const int set = (id - LB3E_FIELD_POP) / 9, j = (id - LB3E_FIELD_POP) % 9;
            if (set < 5) {
                timer.begin(stream_, KC_OTHER);
                k_pop_to_f64<R, S><<<blocks1(N_), 256, 0, stream_>>>(d_.stage, d_.pop[cur_], d_.phi, set, j, N_);
            } else if (anchor_) {  // h = a + delta
                if constexpr (!is_dual<R>::value) {
                    timer.begin(stream_, KC_OTHER);
                    k_anchor_pop<R><<<blocks1(N_), 256, 0, stream_>>>(d_.stage, anchor_ + j * N_, d_.h[hcur_] + j * N_, N_);
                }
            } else {
                timer.begin(stream_, KC_OTHER);
                k_to_f64<R><<<blocks1(N_), 256, 0, stream_>>>(d_.stage, d_.h[hcur_] + j * N_, N_);
            }
            TRY(launched());
            return copy_out(dst, d_.stage);
        }
        if (!src) return LB3E_ERR_FIELD;
        timer.begin(stream_, KC_OTHER);
        k_comp_to_f64<R><<<blocks1(N_), 256, 0, stream_>>>(d_.stage, src, N_, comp);
        TRY(launched());
        return copy_out(dst, d_.stage);
    }

    // snapshot: current pops, current h, then phi..psi_prev fields, then a trailer
    size_t state_bytes() const override {
        return 45 * N_ * sizeof(S) + 9 * N_ * sizeof(R) + fields_bytes() + ion_bytes() + anchor_bytes() +
               hprev_bytes() + 5 * sizeof(int64_t);
    }
    int save(void* dst) override {
        char* o = static_cast<char*>(dst);
        TRY(copy(o, d_.pop[cur_], 45 * N_ * sizeof(S)));
        o += 45 * N_ * sizeof(S);
        TRY(copy(o, d_.h[hcur_], 9 * N_ * sizeof(R)));
        o += 9 * N_ * sizeof(R);
        TRY(copy(o, d_.phi, phi_bytes()));  // the current of the two phi sets
        TRY(copy(o + phi_bytes(), base_ + L_.phi + phi_bytes(), fields_bytes() - phi_bytes()));
        o += fields_bytes();
        if (p_.ions) {  // current ion populations, then n_i and (n_i v_i)^{n-1}
            TRY(copy(o, ion_[icur_], 18 * N_ * sizeof(R)));
            o += 18 * N_ * sizeof(R);
            TRY(copy(o, nion_, 6 * N_ * sizeof(R)));
            o += 6 * N_ * sizeof(R);
        }
        if (anchor_) {  // the anchor of the potential populations (h = anchor + the planes above)
            TRY(copy(o, anchor_, anchor_bytes()));
            o += anchor_bytes();
            TRY(copy(o, hprev_, hprev_bytes()));  // the time extrapolation's previous state
            o += hprev_bytes();
        }
        int64_t trailer[5] = {step_, last_iters_, last_conv_, 0, hprev_valid_};
        std::memcpy(&trailer[3], &last_res_, sizeof(double));
        TRY(copy(o, trailer, sizeof trailer));
        return sync();
    }
    int load(const void* src) override {
        const char* s = static_cast<const char*>(src);
        cur_ = 0;
        hcur_ = 0;
        TRY(copy(d_.pop[0], s, 45 * N_ * sizeof(S)));
        s += 45 * N_ * sizeof(S);
        TRY(copy(d_.h[0], s, 9 * N_ * sizeof(R)));
        s += 9 * N_ * sizeof(R);
        TRY(copy(d_.phi, s, phi_bytes()));
        TRY(copy(base_ + L_.phi + phi_bytes(), s + phi_bytes(), fields_bytes() - phi_bytes()));
        s += fields_bytes();
        if (p_.ions) {
            icur_ = 0;
            TRY(copy(ion_[0], s, 18 * N_ * sizeof(R)));
            s += 18 * N_ * sizeof(R);
            TRY(copy(nion_, s, 6 * N_ * sizeof(R)));
            s += 6 * N_ * sizeof(R);
        }
        if (anchor_) {
            TRY(copy(anchor_, s, anchor_bytes()));
            s += anchor_bytes();
            TRY(copy(hprev_, s, hprev_bytes()));
            s += hprev_bytes();
        }
        int64_t trailer[5];
        TRY(copy(trailer, s, sizeof trailer));
        TRY(sync());
        step_ = trailer[0];
        last_iters_ = (int)trailer[1];
        last_conv_ = (int)trailer[2];
        std::memcpy(&last_res_, &trailer[3], sizeof(double));
        hprev_valid_ = (int)trailer[4];
        return LB3E_OK;
    }

    int64_t potential_iterations() const override { return poisson_iters_run_; }

    // tile height of the fused pass (4, 8 or 16 rows of 32 cells; 16 in the FP32
    // compute builds, 8 only in the tangent builds)
    int set_fused_tile(int rows) override {
        if (rows == 8) { ftile_ = 8; return LB3E_OK; }
        if constexpr (is_dual<R>::value) return LB3E_ERR_PARAM;
        if (rows == 4 || (rows == 16 && std::is_same<R, float>::value)) { ftile_ = rows; return LB3E_OK; }
        return LB3E_ERR_PARAM;
    }
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

    void fused_launch(int first, int write_diag) {
        auto grid = [&](int rows) { return dim3((p_.nx + TX - 1) / TX, (p_.ny + rows - 1) / rows); };
        const int by = ftile_ == 4 && !is_dual<R>::value ? 4 : (ftile_ == 16 && std::is_same<R, float>::value ? 16 : 8);
        const int tma = tma_prepare(by) ? 1 : 0;
        if constexpr (!is_dual<R>::value) {
            if (by == 4) {
                k_fused<R, S, 4><<<grid(4), dim3(TX, 4), fused_dyn_smem<R, S, 4>(), stream_>>>(
                    dp_, d_.pop[cur_], d_.pop[cur_ ^ 1], d_.phi, d_.q, d_.E, d_.prev, d_.diag, first, write_diag,
                    tm_pop_[cur_], tm_prev_, tm_q_, tma, err_flag());
                return;
            }
        }
        if constexpr (std::is_same<R, float>::value) {
            if (by == 16) {
                k_fused<R, S, 16><<<grid(16), dim3(TX, 16), fused_dyn_smem<R, S, 16>(), stream_>>>(
                    dp_, d_.pop[cur_], d_.pop[cur_ ^ 1], d_.phi, d_.q, d_.E, d_.prev, d_.diag, first, write_diag,
                    tm_pop_[cur_], tm_prev_, tm_q_, tma, err_flag());
                return;
            }
        }
        k_fused<R, S><<<grid2_, dim3(TX, TY), fused_dyn_smem<R, S>(), stream_>>>(
            dp_, d_.pop[cur_], d_.pop[cur_ ^ 1], d_.phi, d_.q, d_.E, d_.prev, d_.diag, first, write_diag,
            tm_pop_[cur_], tm_prev_, tm_q_, tma, err_flag());
    }

    // TMA descriptors of the fused pass's staging, made once for the tile height in
    // use: the two population buffers ([45][ny][nx] in the storage type), the 8 d/dt
    // planes and the charge, in boxes of 32 x BY cells.  Needs rows of a multiple of
    // 16 bytes (tensor-map strides); otherwise, or if the driver offers no encoder,
    // the pass stages with per-thread cp.async copies.  True when the descriptors for
    // BY are ready.
    bool tma_prepare(int BY) {
        if constexpr (is_dual<R>::value || !fused_prefetch<S>()) {
            return false;
        } else {
            if (tma_by_ == BY) return true;
            tma_by_ = 0;
            if (p_.nx % (16 / (int)sizeof(S)) != 0 || p_.nx % (16 / (int)sizeof(R)) != 0) return false;
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
            auto type_of = [](size_t bytes, bool bf16) {
                return bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                  : (bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                : (bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16));
            };
            const cuuint64_t nx = (cuuint64_t)p_.nx, ny = (cuuint64_t)p_.ny;
            const cuuint32_t one[3] = {1, 1, 1};
            auto make = [&](CUtensorMap* m, void* base, size_t es, bool bf16, cuuint32_t rank, cuuint64_t planes,
                            cuuint32_t zbox) {
                const cuuint64_t dims[3] = {nx, ny, planes};
                const cuuint64_t strides[2] = {nx * es, nx * ny * es};
                const cuuint32_t box[3] = {(cuuint32_t)TX, (cuuint32_t)BY, zbox};
                return encode(m, type_of(es, bf16), rank, base, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
            };
            constexpr bool bf = std::is_same<S, __nv_bfloat16>::value;
            if (!make(&tm_pop_[0], d_.pop[0], sizeof(S), bf, 3, 45, 1) ||
                !make(&tm_pop_[1], d_.pop[1], sizeof(S), bf, 3, 45, 1) ||
                !make(&tm_prev_, d_.prev, sizeof(R), false, 3, 8, 8) || !make(&tm_q_, d_.q, sizeof(R), false, 2, 1, 1))
                return false;
            tma_by_ = BY;
            return true;
        }
    }
    // a kernel's error flag (a timed-out wait), read back by sync()
    int* err_flag() { return reinterpret_cast<int*>(d_.result + 63); }

    // --- used by Batch: device buffers, and bookkeeping after steps run elsewhere
    const DevState<R, S>& dev() const { return d_; }
    const DevParams& dev_params() const { return dp_; }
    int cur() const { return cur_; }
    int hcur() const { return hcur_; }
    int64_t steps_done() const { return step_; }
    void stepped_externally(int nsteps, int iters_per_step, int swaps_per_step) {
        if (p_.electric) {
            hcur_ ^= (int)(((int64_t)nsteps * swaps_per_step) & 1);
            poisson_iters_run_ += (int64_t)nsteps * iters_per_step;
            last_iters_ = iters_per_step;
            last_conv_ = 1;
            last_res_ = -1.0;
        }
        cur_ ^= nsteps & 1;
        step_ += nsteps;
    }

  private:
    size_t fields_bytes() const { return L_.psi_prev + align256(3 * N_ * sizeof(R)) - L_.phi; }
    size_t phi_bytes() const { return align256(3 * N_ * sizeof(R)); }
    dim3 mc_grid() const {
        return dim3((p_.nx + TX - 1) / TX, (p_.ny + moments_closure_rows() - 1) / moments_closure_rows());
    }
    size_t ion_bytes() const { return p_.ions ? 24 * N_ * sizeof(R) : 0; }
    size_t anchor_bytes() const { return anchor_ ? 9 * N_ * sizeof(AT) : 0; }
    size_t hprev_bytes() const { return anchor_ ? 9 * N_ * sizeof(R) : 0; }
    static unsigned blocks1(size_t n) { return (unsigned)((n + 255) / 256); }
    int launched() {
        ++launches;
        timer.end(stream_);
        return cudaGetLastError() == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }
    // wait for the stream; a kernel that gave up a bounded wait (error flag) fails it
    int sync() {
        if (pinned_) {
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
        return cudaStreamSynchronize(stream_) == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }
    int memset_async(void* p, size_t b) { return cudaMemsetAsync(p, 0, b, stream_) == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA; }
    int copy(void* d, const void* s, size_t b) {
        return cudaMemcpyAsync(d, s, b, cudaMemcpyDefault, stream_) == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }
    // host-or-device doubles -> R field, through the staging area (chunks of 9 N)
    int upload(const double* src, size_t n, R* dst) {
        for (size_t off = 0; off < n; off += 9 * N_) {
            const size_t m = (n - off) < 9 * N_ ? (n - off) : 9 * N_;
            TRY(copy(d_.stage, src + off, m * sizeof(double)));
            timer.begin(stream_, KC_OTHER);
            k_from_f64<R><<<blocks1(m), 256, 0, stream_>>>(dst + off, d_.stage, m);
            TRY(launched());
        }
        return LB3E_OK;
    }
    // sum nb x 4 block partials into result[0..3]: 148 first-stage blocks write
    // their sums after the partial rows (the partial area holds nblk x NOBS
    // doubles, and 4 * nb + 4 * 148 fits for every grid), then one block adds those
    int reduce4(int nb) { return reduce_nv<4>(nb); }
    template <int NV>
    int reduce_nv(int nb) {
        const int s1 = nb < 148 ? 1 : 148;
        const int chunk = (nb + s1 - 1) / s1;
        double* mid = d_.partial + NV * (size_t)nb;
        timer.begin(stream_, KC_REDUCE);
        k_reduce_stage1<NV><<<s1, 256, 0, stream_>>>(d_.partial, nb, chunk, mid);
        TRY(launched());
        timer.begin(stream_, KC_REDUCE);
        k_reduce_partials<NV><<<1, 256, 0, stream_>>>(mid, s1, d_.result);
        return launched();
    }
    int copy_out(double* dst, const double* dsrc) {
        TRY(copy(dst, dsrc, N_ * sizeof(double)));
        return sync();
    }

    dim3 mg_grid(int l) const { return dim3((mg_[l].nx + TX - 1) / TX, (mg_[l].ny + TY - 1) / TY); }
    // FD potential by multigrid V-cycles (warm-started from the last psi)
    int mg_solve(double tol, int max_cycles) {
        const int nl = (int)mg_.size();
        const dim3 blk(TX, TY);
        const double vb = p_.V_bottom, vt = p_.V_top;
        timer.begin(stream_, KC_POISSON);
        k_mg_load<R><<<mg_grid(0), blk, 0, stream_>>>(mg_[0], d_.eps, d_.q, vb, vt);
        TRY(launched());
        for (int l = 0; l < nl; ++l) {
            if (l > 0) {
                timer.begin(stream_, KC_POISSON);
                k_mg_coarsen_eps<<<mg_grid(l), blk, 0, stream_>>>(mg_[l - 1], mg_[l]);
                TRY(launched());
            }
            timer.begin(stream_, KC_POISSON);
            if (l == 0) {
                k_mg_faces<<<mg_grid(0), blk, 0, stream_>>>(mg_[0]);
                TRY(launched());
                timer.begin(stream_, KC_POISSON);
                k_mg_diag<<<mg_grid(0), blk, 0, stream_>>>(mg_[0], mgf_[0]);
            } else {
                k_mg_coeffs_f<<<mg_grid(l), blk, 0, stream_>>>(mg_[l], mgf_[l]);
            }
            TRY(launched());
        }
        last_res_ = -1.0;
        last_conv_ = 0;
        int cycles = 0;
        for (;;) {
            timer.begin(stream_, KC_REDUCE);
            k_mg_residual<double><<<mg_grid(0), blk, 0, stream_>>>(mg_[0], d_.partial);
            TRY(launched());
            TRY(reduce_nv<2>((int)(mg_grid(0).x * mg_grid(0).y)));
            if (cudaMemcpyAsync(pinned_, d_.result, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
                cudaSuccess)
                return LB3E_ERR_CUDA;
            TRY(sync());
            last_res_ = pinned_[1] > 0 ? std::sqrt(pinned_[0] / pinned_[1]) : 0.0;
            if (last_res_ <= tol) { last_conv_ = 1; break; }
            if (cycles >= max_cycles) break;
            // V-cycle on the FP32 error equation A e = r (r: the fine residual in
            // mg_[0].res), then psi += e in FP64
            timer.begin(stream_, KC_POISSON);
            k_mg_defect<<<mg_grid(0), blk, 0, stream_>>>(mg_[0], mgf_[0]);
            TRY(launched());
            TRY(vcycle(KC_POISSON));
            timer.begin(stream_, KC_POISSON);
            k_mg_correct<<<mg_grid(0), blk, 0, stream_>>>(mg_[0], mgf_[0]);
            TRY(launched());
            ++cycles;
            poisson_iters_run_ += 1;
        }
        last_iters_ = cycles;
        timer.begin(stream_, KC_FIELDS);
        if constexpr (std::is_same<R, double>::value)
            k_mg_fields<R><<<mg_grid(0), blk, 0, stream_>>>(mg_[0], vb, vt, p_.E_ext[0], p_.E_ext[1], d_.E);
        else
            k_mg_fields_f32<R><<<mg_grid(0), blk, 0, stream_>>>(mg_[0], vb, vt, p_.E_ext[0], p_.E_ext[1], d_.E);
        return launched();
    }

    // One FP32 V-cycle on level 0's A e = rhs (rhs and e = 0 set by the caller):
    // 2 red-black pre- and post-sweeps per level, residual restriction by sums of the
    // four children, bilinear prolongation, 50 sweeps on the coarsest level.  With
    // first > 0 the cycle starts on level `first` from the level-0 rhs restricted down
    // to it and ends with the prolongations of its solution back to level 0: no sweeps
    // on the levels above it (the coarse correction of the LB solve, whose own
    // iterations smooth the fine scales).  About 10 launches a level, most of them small: on a created stream
    // the sequence is captured once as a CUDA graph and replayed (the level pointers
    // are fixed for the simulation's lifetime; a simulation uses one first level),
    // timed as one interval of class kc.
    int vcycle(int kc, int first = 0) {
        if (stream_ == nullptr) return vcycle_launches(kc, true, first);  // the legacy stream cannot be captured
        if (!vgraph_) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return LB3E_ERR_CUDA;
            const int64_t l0 = launches;
            const int rc = vcycle_launches(kc, false, first);
            vgraph_nodes_ = launches - l0;
            launches = l0;
            if (cudaStreamEndCapture(stream_, &graph) != cudaSuccess || rc != LB3E_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc != LB3E_OK ? rc : LB3E_ERR_CUDA;
            }
            const cudaError_t e = cudaGraphInstantiate(&vgraph_, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                vgraph_ = nullptr;
                return LB3E_ERR_CUDA;
            }
        }
        timer.begin(stream_, kc);
        if (cudaGraphLaunch(vgraph_, stream_) != cudaSuccess) return LB3E_ERR_CUDA;
        timer.end(stream_);
        launches += vgraph_nodes_;
        return cudaGetLastError() == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }
    int vcycle_launches(int kc, bool timed, int first = 0) {
        const int nl = (int)mgf_.size();
        if (first > nl - 1) first = nl - 1;  // a small lattice: start on its coarsest level
        const dim3 blk(TX, TY);
        auto begin = [&]() { if (timed) timer.begin(stream_, kc); };
        auto done = [&]() -> int {
            if (timed) return launched();
            ++launches;
            return cudaGetLastError() == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
        };
        auto smooth = [&](int l, int sweeps) -> int {
            for (int s = 0; s < sweeps; ++s)
                for (int color = 0; color < 2; ++color) {
                    begin();
                    k_mg_smooth<float><<<mg_grid(l), blk, 0, stream_>>>(mgf_[l], color);
                    TRY(done());
                }
            return LB3E_OK;
        };
        if (first > 0) {  // with e = 0 each level's residual is its rhs: restricted down to level first
            for (int l = 0; l < first; ++l) {
                MGLevelF fl = mgf_[l];
                fl.res = fl.rhs;
                begin();
                k_mg_restrict<float><<<mg_grid(l + 1), blk, 0, stream_>>>(fl, mgf_[l + 1]);
                TRY(done());
            }
        }
        if (nl == 1) {
            begin();
            k_mg_coarse_solve<float><<<1, 256, 0, stream_>>>(mgf_[0], 2);
            return done();
        }
        // the small levels (from ls on, at most MG_SMALL_CELLS cells) in one block
        int ls = first;
        while (ls + 1 < nl && (size_t)mgf_[ls].nx * mgf_[ls].ny > (size_t)MG_SMALL_CELLS) ++ls;
        for (int l = first; l < ls; ++l) {
            TRY(smooth(l, 2));
            begin();
            k_mg_residual<float><<<mg_grid(l), blk, 0, stream_>>>(mgf_[l], nullptr);
            TRY(done());
            begin();
            k_mg_restrict<float><<<mg_grid(l + 1), blk, 0, stream_>>>(mgf_[l], mgf_[l + 1]);
            TRY(done());
        }
        MGSmall<float> small{};
        small.n = nl - ls;
        for (int l = ls; l < nl; ++l) small.lv[l - ls] = mgf_[l];
        begin();
        k_mg_small_cycle<float><<<1, MG_SMALL_THREADS, 0, stream_>>>(small);
        TRY(done());
        for (int l = ls - 1; l >= 0; --l) {
            begin();
            k_mg_prolong<float><<<mg_grid(l), blk, 0, stream_>>>(mgf_[l], mgf_[l + 1]);
            TRY(done());
            if (l >= first) TRY(smooth(l, 2));
        }
        return LB3E_OK;
    }

    // the potential solve of this simulation's solver with the run parameters
    int potential() {
        return potential(p_.poisson_tol, p_.poisson_max_iter, p_.poisson_fixed_iter, p_.poisson_check_every);
    }
    int potential(double tol, int max_iter, int fixed, int check) {
        int rc;
        if (p_.potential_solver == 1) {
            rc = mg_solve(tol, max_iter);
        } else {
            rc = LB3E_ERR_PARAM;
            if constexpr (!is_dual<R>::value) {
                if (anchor_) rc = poisson_anchored(tol, max_iter, fixed, check);
            }
            if (!anchor_) rc = poisson(tol, max_iter, fixed, check);
        }
        if (rc == LB3E_OK) record_solve(last_conv_, last_res_);
        return rc;
    }
    // psi of the current potential state into the FP64 staging plane
    int psi_to_stage() {
        timer.begin(stream_, KC_FIELDS);
        if constexpr (!is_dual<R>::value) {
            if (anchor_) {
                k_anchor_fields<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, anchor_, d_.h[hcur_], d_.eps, d_.E,
                                                                         d_.stage);
                return launched();
            }
        }
        if (p_.potential_solver == 1 && !mg_.empty()) {
            if (cudaMemcpyAsync(d_.stage, mg_[0].psi, N_ * sizeof(double), cudaMemcpyDeviceToDevice, stream_) !=
                cudaSuccess)
                return LB3E_ERR_CUDA;
            return launched();
        }
        k_potential_fields<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.h[hcur_], d_.eps, d_.E, d_.stage);
        return launched();
    }

  public:
    // ||b - A psi|| / ||b|| of the current psi for the finite-difference form of the
    // potential equation (5-point, harmonic-mean faces, half-cell electrodes), FP64:
    // a diagnostic of how close the LB fixed point is to that discretisation
    int fd_residual(double* out) {
        if (!p_.electric) return LB3E_ERR_PARAM;
        if constexpr (is_dual<R>::value) {
            return LB3E_ERR_PARAM;
        } else {
            TRY(psi_to_stage());
            timer.begin(stream_, KC_REDUCE);
            k_fd_residual<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.stage, d_.eps, d_.q, d_.partial);
            TRY(launched());
            TRY(reduce_nv<2>(nblk_));
            if (cudaMemcpyAsync(pinned_, d_.result, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
                cudaSuccess)
                return LB3E_ERR_CUDA;
            TRY(sync());
            *out = pinned_[1] > 0 ? std::sqrt(pinned_[0] / pinned_[1]) : 0.0;
            return LB3E_OK;
        }
    }

    // D_inner, D_outer of the current populations' phi (sum_j f^i_j) and, in the
    // tangent builds, their derivatives along each tangent direction (dD[3 k + t],
    // k = 0 inner, 1 outer; zero where a build has no such direction)
    int deformation(double* D, double* dD) override {
        constexpr int M = n_comp<R>::value, NV = 10 * M;
        R* tmp = reinterpret_cast<R*>(d_.stage + N_);  // phi (3 planes) and q~ after the first plane
        timer.begin(stream_, KC_MOMENTS);
        k_moments<R, S><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.pop[cur_], d_.phi, tmp, tmp + 3 * N_);
        TRY(launched());
        const dim3 og = obs_grid(p_.nx, p_.ny);
        const int nb = (int)(og.x * og.y);
        timer.begin(stream_, KC_REDUCE);
        k_deform_moments<R><<<og, dim3(TX, TY), 0, stream_>>>(dp_, tmp, d_.partial);
        TRY(launched());
        timer.begin(stream_, KC_REDUCE);
        k_reduce_partials<NV><<<1, 256, 0, stream_>>>(d_.partial, nb, d_.result);
        TRY(launched());
        if (cudaMemcpyAsync(pinned_, d_.result, NV * sizeof(double), cudaMemcpyDeviceToHost, stream_) != cudaSuccess)
            return LB3E_ERR_CUDA;
        TRY(sync());
        for (int k = 0; k < 2; ++k) {
            const double* m = pinned_ + 5 * M * k;
            D[k] = deformation_of(m, nullptr, nullptr);
            for (int t = 0; t < 3; ++t) {
                double g = 0.0;
                if (t + 1 < M) deformation_of(m, m + 5 * (t + 1), &g);
                if (dD) dD[3 * k + t] = g;
            }
        }
        return LB3E_OK;
    }

    // J = sum_i sum_cells (phi_i - target_i)^2 of the current populations' phi and,
    // in the tangent builds, dJ[t] = sum 2 (phi_i - target_i) dphi_i/dtheta_t
    int shape_objective(const double* target, double* J, double* dJ) override {
        constexpr int M = n_comp<R>::value;
        R* tmp = reinterpret_cast<R*>(d_.stage + N_);  // phi (3 planes) and q~ after the first plane
        timer.begin(stream_, KC_MOMENTS);
        k_moments<R, S><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.pop[cur_], d_.phi, tmp, tmp + 3 * N_);
        TRY(launched());
        const dim3 og = obs_grid(p_.nx, p_.ny);
        const int nb = (int)(og.x * og.y);
        double sum[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < 3; ++i) {
            // the target plane goes to the first staging plane (host or device source)
            if (cudaMemcpyAsync(d_.stage, target + (size_t)i * N_, N_ * sizeof(double), cudaMemcpyDefault,
                                stream_) != cudaSuccess)
                return LB3E_ERR_CUDA;
            timer.begin(stream_, KC_REDUCE);
            k_shape_objective<R><<<og, dim3(TX, TY), 0, stream_>>>(dp_, tmp + (size_t)i * N_, d_.stage, d_.partial);
            TRY(launched());
            timer.begin(stream_, KC_REDUCE);
            k_reduce_partials<M><<<1, 256, 0, stream_>>>(d_.partial, nb, d_.result);
            TRY(launched());
            if (cudaMemcpyAsync(pinned_, d_.result, M * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
                cudaSuccess)
                return LB3E_ERR_CUDA;
            TRY(sync());
            for (int m = 0; m < M; ++m) sum[m] += pinned_[m];
        }
        *J = sum[0];
        if (dJ)
            for (int t = 0; t < 3; ++t) dJ[t] = t + 1 < M ? sum[t + 1] : 0.0;
        return LB3E_OK;
    }

    // ---------------------------------------------------------------- reverse mode
    // (lb3e_adjoint.cuh): plain builds, no ions, the LB potential at a fixed count
    int adjoint_K() const { return p_.electric ? p_.poisson_fixed_iter : 0; }
    int adjoint_supported() const {
        if constexpr (is_dual<R>::value) {
            return LB3E_ERR_UNSUPPORTED;
        } else {
            if (p_.ions) return LB3E_ERR_UNSUPPORTED;
            if (p_.electric && (p_.potential_solver != 0 || p_.poisson_fixed_iter <= 0)) return LB3E_ERR_UNSUPPORTED;
            return LB3E_OK;
        }
    }
    int adjoint_workspace_bytes(size_t* bytes) override {
        TRY(adjoint_supported());
        if constexpr (!is_dual<R>::value) *bytes = AdjointWS<R>::make(dp_, adjoint_K(), nullptr).total;
        return LB3E_OK;
    }
    int state_vector(void* dst) override {
        TRY(adjoint_supported());
        if constexpr (!is_dual<R>::value) {
            timer.begin(stream_, KC_OTHER);
            k_adj_export<R, S><<<blocks1(N_), 256, 0, stream_>>>(dp_, d_.pop[cur_], d_.phi, d_.h[hcur_], d_.E,
                                                                 d_.prev, static_cast<R*>(dst));
            return launched();
        }
        return LB3E_OK;
    }
    int first_step() const override { return step_ == 0; }
    // one step backwards from a state vector: no snapshot, and with device dparams no
    // host round trip; on a created stream the step's launches replay as a graph
    int adjoint_step_x(const void* X, int first, const void* a_in, void* a_out, double* dparams, void* ws,
                       size_t bytes) override {
        TRY(adjoint_supported());
        if constexpr (!is_dual<R>::value) {
            if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LB3E_ERR_WORKSPACE;
            AdjointWS<R> w = AdjointWS<R>::make(dp_, adjoint_K(), static_cast<char*>(ws));
            if (bytes < w.total) return LB3E_ERR_WORKSPACE;
            cudaPointerAttributes at{};
            const bool dev = cudaPointerGetAttributes(&at, dparams) == cudaSuccess &&
                             (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
            cudaGetLastError();  // a host pointer may leave an error code behind on older drivers
            if (dev) w.dpar = dparams;
            else if (cudaMemsetAsync(w.dpar, 0, AJ_N * sizeof(double), stream_) != cudaSuccess) return LB3E_ERR_CUDA;
            if (cudaMemcpyAsync(w.X, X, (size_t)AV_N * N_ * sizeof(R), cudaMemcpyDeviceToDevice, stream_) !=
                cudaSuccess)
                return LB3E_ERR_CUDA;
            if (!adj_ready_) {
                TRY(AdjointRunner<R>::prepare());
                adj_ready_ = true;
            }
            AdjointRunner<R> run{dp_, adjoint_K(), stream_, w};
            const R* ain = static_cast<const R*>(a_in);
            R* aout = static_cast<R*>(a_out);
            if (stream_ == nullptr) {  // the legacy stream cannot be captured
                TRY(run.step_T(first != 0, ain, aout));
                launches += run.launches;
            } else {
                cudaGraphExec_t exec = nullptr;
                for (auto& g : adj_graphs_)
                    if (g.ws == ws && g.ain == a_in && g.aout == a_out && g.first == (first != 0) && g.dpar == w.dpar)
                        exec = g.exec;
                if (!exec) {
                    if (adj_graphs_.size() >= 8) {
                        cudaGraphExecDestroy(adj_graphs_.front().exec);
                        adj_graphs_.erase(adj_graphs_.begin());
                    }
                    cudaGraph_t graph = nullptr;
                    if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                        return LB3E_ERR_CUDA;
                    const int rc = run.step_T(first != 0, ain, aout);
                    if (cudaStreamEndCapture(stream_, &graph) != cudaSuccess || rc != LB3E_OK) {
                        if (graph) cudaGraphDestroy(graph);
                        return rc != LB3E_OK ? rc : LB3E_ERR_CUDA;
                    }
                    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
                    cudaGraphDestroy(graph);
                    if (e != cudaSuccess) return LB3E_ERR_CUDA;
                    adj_graphs_.push_back({ws, a_in, a_out, first != 0, w.dpar, exec, run.launches});
                }
                if (cudaGraphLaunch(exec, stream_) != cudaSuccess) return LB3E_ERR_CUDA;
                for (auto& g : adj_graphs_)
                    if (g.exec == exec) launches += g.nodes;
            }
            if (!dev) return adjoint_params_out(w, dparams);
            return cudaGetLastError() == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
        }
        return LB3E_OK;
    }
    int adjoint_step(const void* state, const void* a_in, void* a_out, double* dparams, void* ws,
                     size_t bytes) override {
        TRY(adjoint_supported());
        if constexpr (!is_dual<R>::value) {
            AdjointWS<R> w;
            TRY(adjoint_ws(ws, bytes, &w));
            if (state) TRY(load(state));
            k_adj_export<R, S><<<blocks1(N_), 256, 0, stream_>>>(dp_, d_.pop[cur_], d_.phi, d_.h[hcur_], d_.E,
                                                                 d_.prev, w.X);
            TRY(launched());
            if (!adj_ready_) {
                TRY(AdjointRunner<R>::prepare());
                adj_ready_ = true;
            }
            AdjointRunner<R> run{dp_, adjoint_K(), stream_, w};
            TRY(run.step_T(step_ == 0, static_cast<const R*>(a_in), static_cast<R*>(a_out)));
            launches += run.launches;
            return adjoint_params_out(w, dparams);
        }
        return LB3E_OK;
    }
    int adjoint_init(const double* phi, const void* a_in, double* dparams, double* dphi, void* ws,
                     size_t bytes) override {
        TRY(adjoint_supported());
        if constexpr (!is_dual<R>::value) {
            AdjointWS<R> w;
            TRY(adjoint_ws(ws, bytes, &w));
            TRY(upload(phi, 3 * N_, w.X));  // phi_init in the first state-vector planes
            if (cudaMemsetAsync(d_.stage, 0, 3 * N_ * sizeof(double), stream_) != cudaSuccess) return LB3E_ERR_CUDA;
            if (!adj_ready_) {
                TRY(AdjointRunner<R>::prepare());
                adj_ready_ = true;
            }
            AdjointRunner<R> run{dp_, adjoint_K(), stream_, w};
            TRY(run.init_T(w.X, static_cast<const R*>(a_in), d_.stage));
            launches += run.launches;
            if (dphi) {
                // add the FP64 planes to the caller's (host or device) dphi through the staging area
                TRY(copy(d_.stage + 3 * N_, dphi, 3 * N_ * sizeof(double)));
                timer.begin(stream_, KC_OTHER);
                k_add_f64<<<blocks1(3 * N_), 256, 0, stream_>>>(d_.stage + 3 * N_, d_.stage, 3 * N_);
                TRY(launched());
                TRY(copy(dphi, d_.stage + 3 * N_, 3 * N_ * sizeof(double)));
            }
            return adjoint_params_out(w, dparams);
        }
        return LB3E_OK;
    }
    int deformation_seed(int which, double* D, void* a_out) override {
        TRY(adjoint_supported());
        if constexpr (!is_dual<R>::value) {
            double Ds[2];
            TRY(deformation(Ds, nullptr));  // leaves the moment sums in pinned_
            const double* m = pinned_ + 5 * which;
            double g[5];
            for (int k = 0; k < 5; ++k) {
                double e[5] = {0, 0, 0, 0, 0};
                e[k] = 1.0;
                deformation_of(m, e, &g[k]);
            }
            *D = Ds[which];
            timer.begin(stream_, KC_OTHER);
            k_adj_seed_deformation<R><<<blocks1(N_), 256, 0, stream_>>>(
                dp_, which == 0 ? dp_.inner : dp_.matrix, which == 0 ? 1.0 : -1.0, g[0], g[1], g[2], g[3], g[4],
                static_cast<R*>(a_out));
            TRY(launched());
            return sync();
        }
        return LB3E_OK;
    }
    int shape_seed(const double* target, double* J, void* a_out) override {
        TRY(adjoint_supported());
        if constexpr (!is_dual<R>::value) {
            TRY(shape_objective(target, J, nullptr));  // leaves phi of the current populations after the first plane
            const R* tmp = reinterpret_cast<const R*>(d_.stage + N_);
            TRY(copy(d_.stage + 5 * N_, target, 3 * N_ * sizeof(double)));
            timer.begin(stream_, KC_OTHER);
            k_adj_seed_shape<R><<<blocks1(N_), 256, 0, stream_>>>(dp_, tmp, d_.stage + 5 * N_,
                                                                  static_cast<R*>(a_out));
            TRY(launched());
            return sync();
        }
        return LB3E_OK;
    }

  private:
    struct AdjGraph {
        const void* ws;
        const void* ain;
        const void* aout;
        bool first;
        const double* dpar;
        cudaGraphExec_t exec;
        int64_t nodes;
    };
    std::vector<AdjGraph> adj_graphs_;  // captured backward steps (at most 8)
    bool adj_ready_ = false;             // the reverse mode's kernel attributes are set
    template <class W>
    int adjoint_ws(void* ws, size_t bytes, W* w) {
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LB3E_ERR_WORKSPACE;
        *w = W::make(dp_, adjoint_K(), static_cast<char*>(ws));
        if (bytes < w->total) return LB3E_ERR_WORKSPACE;
        if (cudaMemsetAsync(w->dpar, 0, AJ_N * sizeof(double), stream_) != cudaSuccess) return LB3E_ERR_CUDA;
        return LB3E_OK;
    }
    template <class W>
    int adjoint_params_out(const W& w, double* dparams) {
        if (cudaMemcpyAsync(pinned_, w.dpar, AJ_N * sizeof(double), cudaMemcpyDeviceToHost, stream_) != cudaSuccess)
            return LB3E_ERR_CUDA;
        TRY(sync());
        for (int k = 0; k < AJ_N; ++k) dparams[k] += pinned_[k];
        return LB3E_OK;
    }

    // relative residual from the 4 FP64 sums |d psi|^2, |psi|^2, |d J|^2, |J|^2
    static double rel_residual(const double* v) {
        const double dp = v[0], pp = v[1], dj = v[2], jj = v[3];
        const double r1 = pp > 0.0 ? std::sqrt(dp) / std::sqrt(pp) : (dp > 0.0 ? INFINITY : 0.0);
        const double r2 = jj > 0.0 ? std::sqrt(dj) / std::sqrt(jj) : (dj > 0.0 ? INFINITY : 0.0);
        return r1 > r2 ? r1 : r2;
    }
    // the plateau rule: a residual-controlled solve stops, not converged, once the
    // best residual has not fallen by 1% over `window` consecutive checks (a
    // rounding floor, or a rate too slow to reach the tolerance in bounded work)
    struct Plateau {
        double best = INFINITY;
        int since = 0;
        bool stalled(double r, int window) {
            if (r < 0.99 * best) {
                best = r;
                since = 0;
                return false;
            }
            return ++since >= window;
        }
    };

    // Fold delta into the FP64 anchor and form the anchor's increment r = T a + s - a
    // (rres), delta = 0.  With `residual`: the relative increments of psi and J in
    // *res, and the anchor's |psi|^2, |J|^2 (the denominators of later checks) in norms.
    // zero_delta = false (a coarse correction that overwrites delta follows): the FP32
    // builds leave delta as it is and mark it stale (cleared if the solve ends first)
    int anchor_refresh(bool residual, double* res, double* norms, bool zero_delta = true) {
        if constexpr (is_dual<R>::value) {
            return LB3E_ERR_PARAM;
        } else {
            timer.begin(stream_, KC_ANCHOR);
            if constexpr (std::is_same<R, float>::value) {  // double-float anchor, one pass
                k_anchor_refresh_pull_df<<<grid2_, dim3(TX, TY), 0, stream_>>>(
                    dp_, anchor_, anchor_alt_, delta_stale_ ? nullptr : d_.h[hcur_], zero_delta ? d_.h[hcur_ ^ 1] : nullptr,
                    d_.eps, d_.q,
                    rres_, ja_, d_.partial, acoef_);
                std::swap(anchor_, anchor_alt_);
                if (zero_delta) hcur_ ^= 1;
                delta_stale_ = !zero_delta;
            } else {
                k_anchor_refresh<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, anchor_, d_.h[hcur_], d_.eps, d_.q,
                                                                          d_.stage, ja_, 1.0 / dp_.tau_h,
                                                                          dp_.tau_h / 3.0);
                TRY(launched());
                timer.begin(stream_, KC_ANCHOR);
                k_anchor_residual<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, anchor_, d_.stage, rres_, d_.partial);
            }
            TRY(launched());
            if (!residual) return LB3E_OK;
            TRY(reduce4(nblk_));
            if (cudaMemcpyAsync(pinned_, d_.result, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
                cudaSuccess)
                return LB3E_ERR_CUDA;
            TRY(sync());
            *res = rel_residual(pinned_);
            norms[0] = pinned_[1];
            norms[1] = pinned_[3];
            return LB3E_OK;
        }
    }
    // the increment of the last pseudo-iteration of delta, relative to the anchor's
    // norms; with `rhs`, also the coarse correction's right-hand side.  *noisy: the
    // rounding floor of these increments (the precision's epsilon times the size of
    // delta) is above a tenth of tol -- time to fold delta into the anchor.
    int rs_check(const double* norms, bool rhs, double tol, double* res, bool* noisy, int inc_blocks = 0) {
        if constexpr (!is_dual<R>::value) {
            if (inc_blocks > 0) {  // the last iteration launch formed the block sums
                TRY(reduce_nv<3>(inc_blocks));
            } else {
                timer.begin(stream_, KC_REDUCE);
                k_rs_increment<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(
                    dp_, d_.h[hcur_], d_.psi_prev, d_.partial, rhs ? mgf_[0].rhs : nullptr, rhs ? mgf_[0].psi : nullptr);
                TRY(launched());
                TRY(reduce_nv<3>(nblk_));
            }
            if (cudaMemcpyAsync(pinned_, d_.result, 3 * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
                cudaSuccess)
                return LB3E_ERR_CUDA;
            TRY(sync());
            const double v[4] = {pinned_[0], norms[0], pinned_[1], norms[1]};
            *res = rel_residual(v);
            const double eps = std::is_same<R, float>::value ? 6e-8 : 1.2e-16;
            const double floor_abs = 2.0 * eps * std::sqrt(pinned_[2]);
            const double nmin = std::sqrt(norms[0] < norms[1] ? norms[0] : norms[1]);
            *noisy = floor_abs > 0.1 * tol * nmin;
        }
        return LB3E_OK;
    }
    // permittivity of every multigrid level and the FP32 coefficients (once per solve:
    // eps is fixed within it)
    int lbmg_setup() {
        if constexpr (!is_dual<R>::value) {
            const int nl = (int)mg_.size();
            const dim3 blk(TX, TY);
            timer.begin(stream_, KC_COARSE);
            k_lbmg_eps<R><<<mg_grid(0), blk, 0, stream_>>>(mg_[0], d_.eps);
            TRY(launched());
            for (int l = 0; l < nl; ++l) {
                if (l > 0) {
                    timer.begin(stream_, KC_COARSE);
                    k_mg_coarsen_eps<<<mg_grid(l), blk, 0, stream_>>>(mg_[l - 1], mg_[l]);
                    TRY(launched());
                }
                timer.begin(stream_, KC_COARSE);
                k_mg_coeffs_f<<<mg_grid(l), blk, 0, stream_>>>(mg_[l], mgf_[l]);
                TRY(launched());
            }
        }
        return LB3E_OK;
    }
    // One V-cycle on A e = (the macroscopic residual), its solution e entering delta
    // as its local equilibrium and first-order flux.  Right after a refresh the
    // residual is sum_{j>0} r_j of the anchor and delta = e; otherwise rs_check left
    // it in level 0's rhs and delta += e.
    int lbmg_correct(bool after_refresh) {
        if constexpr (!is_dual<R>::value) {
            const dim3 blk(TX, TY);
            if (after_refresh) {
                timer.begin(stream_, KC_COARSE);
                k_lbmg_rhs<R><<<grid2_, blk, 0, stream_>>>(dp_, rres_, mgf_[0]);
                TRY(launched());
            }
            TRY(vcycle(KC_COARSE, lbmg_first_));
            timer.begin(stream_, KC_COARSE);
            k_lbmg_correct<R><<<grid2_, blk, 0, stream_>>>(dp_, mgf_[0], d_.eps, d_.h[hcur_], after_refresh ? 0 : 1);
            TRY(launched());
            if (after_refresh) delta_stale_ = false;  // delta = the correction
        }
        return LB3E_OK;
    }
    // iterations per launch on delta: the chunk, within the shared memory the
    // blocked kernel needs (the 8-cell halo does not fit for FP64)
    int rs_chunk() const {
        if (pb_smem_bytes<R, 8, true>() > 227 * 1024 && chunk_ > 4) return 4;
        return chunk_;
    }
    // m pseudo-iterations on delta (blocked, rs_chunk() per launch); with save,
    // psi and J before the last collision go to psi_prev for rs_check.  FP32 builds:
    // a blocked last launch also forms the check's block sums (and, with rhs, the
    // coarse right-hand side); *inc_blocks is their number (0: rs_check forms them)
    int rs_iterations(int m, bool save, bool rhs = false, int* inc_blocks = nullptr) {
        if (inc_blocks) *inc_blocks = 0;
        if constexpr (!is_dual<R>::value) {
            TRY(pb_prepare());
            const dim3 pgrid((p_.nx + PB_TX - 1) / PB_TX, (p_.ny + PB_TY - 1) / PB_TY);
            const int kmax = rs_chunk();
            for (int k = 0; k < m;) {
                const int c = m - k < kmax ? m - k : kmax;
                const int sv = save && k + c == m;
                const bool inc = sv && c > 1 && std::is_same<R, float>::value && inc_blocks;
                float* rp = inc && rhs ? mgf_[0].rhs : nullptr;
                float* ep = inc && rhs ? mgf_[0].psi : nullptr;
                auto launch = [&](auto kern, int threads, size_t smem) {
                    kern<<<pgrid, threads, smem, stream_>>>(dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps, rres_,
                                                            d_.psi_prev, c, sv, d_.partial, rp, ep);
                };
                timer.begin(stream_, KC_POISSON);
                if (c == 1)
                    k_poisson_rs<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps,
                                                                          rres_, d_.psi_prev, sv);
                else if (pb_halo_for(c) == 2)
                    launch(inc ? k_poisson_tb_rs<R, 2, 0, true> : k_poisson_tb_rs<R, 2>, pb_threads<R, 2, true>(),
                           pb_smem_bytes<R, 2, true>());
                else if (c == 4)
                    launch(inc ? k_poisson_tb_rs<R, 4, 4, true> : k_poisson_tb_rs<R, 4, 4>, pb_threads<R, 4, true>(),
                           pb_smem_bytes<R, 4, true>());
                else if (pb_halo_for(c) == 4)
                    launch(inc ? k_poisson_tb_rs<R, 4, 0, true> : k_poisson_tb_rs<R, 4>, pb_threads<R, 4, true>(),
                           pb_smem_bytes<R, 4, true>());
                else if constexpr (pb_smem_bytes<R, 8, true>() <= 227 * 1024)
                    launch(inc ? k_poisson_tb_rs<R, 8, 0, true> : k_poisson_tb_rs<R, 8>, pb_threads<R, 8, true>(),
                           pb_smem_bytes<R, 8, true>());
                TRY(launched());
                if (inc) *inc_blocks = (int)(pgrid.x * pgrid.y);
                poisson_iters_run_ += c;
                hcur_ ^= 1;
                k += c;
            }
        }
        return LB3E_OK;
    }
    // The LB potential solve on an FP64 anchor (solver 3), with a multigrid coarse
    // correction before every run of check_every iterations (solver 2).  One refresh
    // at the start gives the exact FP64 increment of the warm start; later checks
    // take the increment of the last iteration of delta.  A stalled residual leads to
    // one more refresh (delta folded into the anchor); a stall right after a refresh
    // ends the solve (-1).  With fixed > 0: exactly that many plain pseudo-iterations.
    int poisson_anchored(double tol, int max_iter, int fixed, int check) {
        if (check < 1) check = 1;
        last_res_ = -1.0;
        last_conv_ = fixed > 0;
        last_iters_ = 0;
        const bool coarse = p_.potential_solver == 2 && fixed <= 0;
        if (coarse) TRY(lbmg_setup());
        double norms[2] = {0.0, 0.0}, res = -1.0;
        if constexpr (!is_dual<R>::value) {
            if (fixed <= 0 && in_step_) {  // start from 2 h_n - h_{n-1} (fixed point and test unchanged)
                timer.begin(stream_, KC_OTHER);
                k_anchor_extrapolate<R><<<blocks1(9 * N_), 256, 0, stream_>>>(anchor_, d_.h[hcur_], hprev_, 9 * N_,
                                                                                hprev_valid_);
                TRY(launched());
                hprev_valid_ = 1;
            }
        }
        TRY(anchor_refresh(fixed <= 0, &res, norms, !coarse));
        int it = 0;
        if (fixed > 0) {
            // the plain iterates, delta folded into the anchor every check iterations so
            // that it stays small against h
            while (it < fixed) {
                if (it > 0) TRY(anchor_refresh(false, &res, norms));
                const int m = fixed - it < check ? fixed - it : check;
                TRY(rs_iterations(m, false));
                it += m;
            }
        } else {
            Plateau pl;
            bool after_refresh = true, stall_refreshed = false;
            for (;;) {
                last_res_ = res;
                if (res <= tol) { last_conv_ = 1; break; }
                if (pl.stalled(res, coarse ? 4 : 32)) {
                    // a stall again after a stall refresh, with no progress between: a floor
                    if (stall_refreshed) { last_conv_ = -1; break; }
                    TRY(anchor_refresh(true, &res, norms, !coarse));
                    after_refresh = true;
                    stall_refreshed = true;
                    pl = Plateau();
                    continue;
                }
                if (pl.since == 0) stall_refreshed = false;  // progress since the last stall
                if (it >= max_iter) break;
                if (coarse) TRY(lbmg_correct(after_refresh));
                after_refresh = false;
                // with the coarse correction, the increment is checked max(2, check/16)
                // times a cycle (a check costs a fraction of a correction)
                const int nsub = coarse && check >= 16 ? (check / 16 > 2 ? check / 16 : 2) : 1;
                for (int sub = 0; sub < nsub && it < max_iter; ++sub) {
                    const int want = check / nsub + (sub < check % nsub ? 1 : 0);
                    const int m = max_iter - it < want ? max_iter - it : want;
                    // the coarse right-hand side only from the cycle's last check
                    const bool rhs = coarse && (sub == nsub - 1 || it + m >= max_iter);
                    int inc_blocks = 0;
                    TRY(rs_iterations(m, true, rhs, &inc_blocks));
                    it += m;
                    bool noisy = false;
                    TRY(rs_check(norms, rhs, tol, &res, &noisy, inc_blocks));
                    if (noisy && res > tol) {  // the exact increment at a fresh anchor instead
                        TRY(anchor_refresh(true, &res, norms, !coarse));
                        after_refresh = true;
                        break;
                    }
                    if (res <= tol) break;
                }
            }
        }
        last_iters_ = it;
        if (delta_stale_) {  // the solve ended at a refresh: h = the anchor
            if (cudaMemsetAsync(d_.h[hcur_], 0, 9 * N_ * sizeof(R), stream_) != cudaSuccess) return LB3E_ERR_CUDA;
            delta_stale_ = false;
        }
        if constexpr (!is_dual<R>::value) {
            timer.begin(stream_, KC_FIELDS);
            k_anchor_efield<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, ja_, d_.h[hcur_], d_.eps, d_.E);
            TRY(launched());
        }
        return LB3E_OK;
    }

    // blocked-iteration kernels need more than the default dynamic shared memory
    int pb_prepare() {
        if constexpr (is_dual<R>::value) {
            if (!pb_ready_) {
                if (cudaFuncSetAttribute(k_poisson_tile<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * 9 * PTTangent::NT * sizeof(R))) != cudaSuccess)
                    return LB3E_ERR_CUDA;
                pb_ready_ = true;
            }
        }
        if constexpr (!is_dual<R>::value) {
            if (!pb_ready_) {
                if (cudaFuncSetAttribute(k_poisson_tb<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pb_smem_bytes<R, 2>()) != cudaSuccess ||
                    cudaFuncSetAttribute(k_poisson_tb<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pb_smem_bytes<R, 4>()) != cudaSuccess ||
                    cudaFuncSetAttribute(k_poisson_tb<R, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pb_smem_bytes<R, 4>()) != cudaSuccess ||
                    cudaFuncSetAttribute(k_poisson_tb<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pb_smem_bytes<R, 8>()) != cudaSuccess)
                    return LB3E_ERR_CUDA;
                if (anchor_) {
                    auto attr = [](auto kern, size_t bytes) {
                        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
                               cudaSuccess;
                    };
                    if (!attr(k_poisson_tb_rs<R, 2>, pb_smem_bytes<R, 2, true>()) ||
                        !attr(k_poisson_tb_rs<R, 2, 0, true>, pb_smem_bytes<R, 2, true>()) ||
                        !attr(k_poisson_tb_rs<R, 4>, pb_smem_bytes<R, 4, true>()) ||
                        !attr(k_poisson_tb_rs<R, 4, 0, true>, pb_smem_bytes<R, 4, true>()) ||
                        !attr(k_poisson_tb_rs<R, 4, 4>, pb_smem_bytes<R, 4, true>()) ||
                        !attr(k_poisson_tb_rs<R, 4, 4, true>, pb_smem_bytes<R, 4, true>()))
                        return LB3E_ERR_CUDA;
                }
                if constexpr (pb_smem_bytes<R, 8, true>() <= 227 * 1024) {
                    if (anchor_ &&
                        (cudaFuncSetAttribute(k_poisson_tb_rs<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)pb_smem_bytes<R, 8, true>()) != cudaSuccess ||
                         cudaFuncSetAttribute(k_poisson_tb_rs<R, 8, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)pb_smem_bytes<R, 8, true>()) != cudaSuccess))
                        return LB3E_ERR_CUDA;
                }
                pb_ready_ = true;
            }
        }
        return LB3E_OK;
    }
    // one blocked launch of c iterations, on the region sized for c; returns the
    // number of blocks (residual partial sums) it launched
    int pb_launch(dim3 pgrid, int c, int save, int check) {
        if constexpr (!is_dual<R>::value) {
            if (pb_halo_for(c) == 2)
                k_poisson_tb<R, 2><<<pgrid, pb_threads<R, 2>(), pb_smem_bytes<R, 2>(), stream_>>>(
                    dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps, d_.q, d_.psi_prev, d_.partial, c, save, check);
            else if (c == 4)
                k_poisson_tb<R, 4, 4><<<pgrid, pb_threads<R, 4>(), pb_smem_bytes<R, 4>(), stream_>>>(
                    dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps, d_.q, d_.psi_prev, d_.partial, c, save, check);
            else if (pb_halo_for(c) == 4)
                k_poisson_tb<R, 4><<<pgrid, pb_threads<R, 4>(), pb_smem_bytes<R, 4>(), stream_>>>(
                    dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps, d_.q, d_.psi_prev, d_.partial, c, save, check);
            else
                k_poisson_tb<R, 8><<<pgrid, pb_threads<R, 8>(), pb_smem_bytes<R, 8>(), stream_>>>(
                    dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps, d_.q, d_.psi_prev, d_.partial, c, save, check);
        }
        return (int)(pgrid.x * pgrid.y);
    }

  public:
    // pseudo-iterations per potential launch: 1 (one per launch), 2 (blocked,
    // 2-cell halo), 3..4 (4-cell halo) or 5..8 (8-cell halo)
    int set_chunk(int k) override {
        if (k < 1 || k > PB_HALO) return LB3E_ERR_PARAM;
        if constexpr (is_dual<R>::value) {
            if (k > 4) return LB3E_ERR_PARAM;
        }
        chunk_ = k;
        return LB3E_OK;
    }

  private:
    // the pseudo-time potential solve (Eq. 43) from the current h.  Iterations
    // run in chunks of up to chunk_ per launch (k_poisson_tb); a chunk never
    // straddles a residual check, which is taken before the first collision of a
    // chunk, and the state for the next check is saved before the last one.
    int poisson(double tol, int max_iter, int fixed, int check) {
        const int n = fixed > 0 ? fixed : max_iter;
        if (check < 1) check = 1;
        last_res_ = -1.0;
        last_conv_ = fixed > 0;
        last_iters_ = n;
        TRY(pb_prepare());
        const dim3 pgrid((p_.nx + PB_TX - 1) / PB_TX, (p_.ny + PB_TY - 1) / PB_TY);
        int pblk = (int)(pgrid.x * pgrid.y);
        Plateau pl;
        int k = 1;
        while (k <= n) {
            int c = n - k + 1 < chunk_ ? n - k + 1 : chunk_;
            if (fixed <= 0) {
                int next = (k / check + 1) * check;  // next check iteration after k
                if (next < 2) next = 2;
                if (next - k < c) c = next - k;
            }
            const int do_check = fixed <= 0 && k >= 2 && k % check == 0;
            const int save = fixed <= 0 && (k + c) % check == 0;
            bool blocked = false;
            if constexpr (is_dual<R>::value) {  // dual numbers: tiles of one cell a thread
                if (fixed > 0 && c >= 2) {
                    using G = PTTangent;
                    c = c < 4 ? c : 4;
                    timer.begin(stream_, KC_POISSON);
                    k_poisson_tile<R><<<dim3((p_.nx + G::TX - 1) / G::TX, (p_.ny + G::HT - 9) / (G::HT - 8)),
                                        dim3(G::W, G::HT), 2 * 9 * G::NT * sizeof(R), stream_>>>(
                        dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps, d_.q, c);
                    TRY(launched());
                    poisson_iters_run_ += c;
                    blocked = true;
                }
            } else {
                if (c >= 2) {
                    timer.begin(stream_, KC_POISSON);
                    pblk = pb_launch(pgrid, c, save, do_check);
                    TRY(launched());
                    poisson_iters_run_ += c;
                    blocked = true;
                }
            }
            if (!blocked) {
                c = 1;
                timer.begin(stream_, KC_POISSON);
                k_poisson<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.h[hcur_], d_.h[hcur_ ^ 1], d_.eps, d_.q,
                                                                   d_.psi_prev, d_.partial, (k + 1) % check == 0 && fixed <= 0,
                                                                   do_check);
                TRY(launched());
                poisson_iters_run_ += 1;
            }
            if (do_check) {
                TRY(reduce4(blocked ? pblk : nblk_));
                if (cudaMemcpyAsync(pinned_, d_.result, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream_) !=
                    cudaSuccess)
                    return LB3E_ERR_CUDA;
                TRY(sync());
                last_res_ = rel_residual(pinned_);
                if (last_res_ <= tol) {  // the state before this chunk's first collision is the answer
                    last_conv_ = 1;
                    last_iters_ = k - 1;
                    break;
                }
                if (pl.stalled(last_res_, 32)) {  // the state before this chunk, as above
                    last_conv_ = -1;
                    last_iters_ = k - 1;
                    break;
                }
            }
            hcur_ ^= 1;
            k += c;
        }
        timer.begin(stream_, KC_FIELDS);
        k_potential_fields<R><<<grid2_, dim3(TX, TY), 0, stream_>>>(dp_, d_.h[hcur_], d_.eps, d_.E, nullptr);
        return launched();
    }

    lb3e_params p_;
    cudaStream_t stream_;
    Layout L_;
    DevState<R, S> d_{};
    DevParams dp_{};
    char* base_ = nullptr;
    size_t N_ = 0;
    dim3 grid2_;
    int nblk_ = 0;
    int cur_ = 0, hcur_ = 0;
    int64_t step_ = 0;
    int last_iters_ = 0, last_conv_ = 0;
    double last_res_ = -1.0;
    double* pinned_ = nullptr;
    bool pb_ready_ = false;
    int chunk_ = 4;  // pseudo-iterations per potential launch (4: fastest measured on a 4096^2 lattice)
    // rows of the fused pass's 32-wide tiles: 4 in FP32 compute (3% faster than 8 on a
    // 4096^2 lattice, six blocks a SM), 8 otherwise
    int ftile_ = std::is_same<R, float>::value ? 4 : 8;
    std::vector<MGLevel> mg_;
    std::vector<MGLevelF> mgf_;
    cudaGraphExec_t vgraph_ = nullptr;  // the captured V-cycle (multigrid solvers, created streams)
    int lbmg_first_ = 3;                // first V-cycle level of the LB solve's coarse correction
    int64_t vgraph_nodes_ = 0;
    // the anchor of the potential populations (solvers 2, 3): FP64 in the FP64 build,
    // double-float in the FP32 builds, with the refresh's coefficients in that form
    using AT = typename AnchorOf<R>::type;
    AT* anchor_ = nullptr;
    CUtensorMap tm_pop_[2]{}, tm_prev_{}, tm_q_{};  // TMA descriptors of the fused pass (tma_prepare)
    int tma_by_ = 0;                                // the tile height they were made for (0: none)
    AT* anchor_alt_ = nullptr;   // FP32 builds: the anchor planes the next refresh writes
    bool delta_stale_ = false;   // delta was folded into the anchor but not yet cleared
    R* hprev_ = nullptr;         // the state the last step's solve started from (see k_anchor_extrapolate)
    int hprev_valid_ = 0;        // hprev_ holds the state after the previous step's solve
    bool in_step_ = false;       // a time step's solve (extrapolated from the two before)
    R* phi_alt_ = nullptr;  // the set of phi planes the next moments pass writes
    AnchorCoef acoef_{};
    R* rres_ = nullptr;         // the anchor's increment over one pseudo-iteration
    R* ja_ = nullptr;           // the anchor's flux J = sum_j c_j a_j (2 planes), for E
    R* ion_[2] = {nullptr, nullptr};  // Nernst-Planck populations (ions = 1)
    R* nion_ = nullptr;               // n_i of the step (2 planes), then (n_i v_i)^{n-1} (4 planes)
    R* ionprev_ = nullptr;
    int icur_ = 0;
    IonParams ip_{};

  public:
    int64_t poisson_iters_run_ = 0;  // pseudo-iterations executed (all solves)
};

// ---------------------------------------------------------------- batches
// Instances of one precision stepped together.  Each instance is a Sim laid out
// in its own slice of the caller's workspace; the batch adds a device table of
// instance parameters/pointers and the tile work list, and replays each pair of
// steps as one CUDA graph (potential iterations per step are fixed, so the
// ping-pong parities return to where they started after two steps).
template <class R, class S>
class Batch final : public BatchBase {
  public:
    static size_t tiles_of(const lb3e_params& p) {
        return (size_t)((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
    }
    static size_t ptiles_of(const lb3e_params& p) {
        return (size_t)((p.nx + PB_TX - 1) / PB_TX) * ((p.ny + PB_TY - 1) / PB_TY);
    }
    // tiles of 32 x rows cells for the fused pass
    static size_t ftiles_of(const lb3e_params& p, int rows) {
        return (size_t)((p.nx + TX - 1) / TX) * ((p.ny + rows - 1) / rows);
    }
    static size_t bytes(const lb3e_params* ps, int n) {
        size_t ntiles = 0, nptiles = 0, nft = 0, b = 0;
        for (int i = 0; i < n; ++i) {
            ntiles += tiles_of(ps[i]);
            nptiles += ptiles_of(ps[i]);
            nft += ftiles_of(ps[i], 4);  // the smallest tile height needs the longest list
            b += align256(Sim<R, S>::layout(ps[i]).total);
        }
        return b + align256(n * sizeof(InstState<R, S>)) + align256(ntiles * sizeof(int4)) +
               align256(nptiles * sizeof(int4)) + align256(nft * sizeof(int4));
    }

    Batch(const lb3e_params* ps, int n, void* ws, cudaStream_t st) : stream_(st), n_(n) {
        char* b = static_cast<char*>(ws);
        size_t ntiles = 0, nptiles = 0;
        for (int i = 0; i < n; ++i) {
            ntiles += tiles_of(ps[i]);
            nptiles += ptiles_of(ps[i]);
        }
        table_ = reinterpret_cast<InstState<R, S>*>(b);
        b += align256(n * sizeof(InstState<R, S>));
        tiles_ = reinterpret_cast<int4*>(b);
        b += align256(ntiles * sizeof(int4));
        ptiles_ = reinterpret_cast<int4*>(b);
        b += align256(nptiles * sizeof(int4));
        size_t nft = 0;
        for (int i = 0; i < n; ++i) nft += ftiles_of(ps[i], 4);
        ftiles_ = reinterpret_cast<int4*>(b);
        b += align256(nft * sizeof(int4));
        ntiles_ = (int)ntiles;
        nptiles_ = (int)nptiles;
        iters_ = 0;
        for (int i = 0; i < n; ++i) {
            sims_.push_back(new Sim<R, S>(ps[i], b, st));
            b += align256(Sim<R, S>::layout(ps[i]).total);
            if (ps[i].electric) iters_ = ps[i].poisson_fixed_iter;
        }
    }
    ~Batch() override {
        for (auto& g : graphs_)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        for (auto* s : sims_) delete s;
    }

    int init(const double* const* phis) {
        if constexpr (fused_dyn_smem<R, S>() > 0) {
            if (cudaFuncSetAttribute(kb_fused<R, S, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)fused_dyn_smem<R, S, 4>()) != cudaSuccess ||
                cudaFuncSetAttribute(kb_fused<R, S, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)fused_dyn_smem<R, S, 8>()) != cudaSuccess)
                return LB3E_ERR_CUDA;
            if constexpr (std::is_same<R, float>::value) {
                if (cudaFuncSetAttribute(kb_fused<R, S, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_dyn_smem<R, S, 16>()) != cudaSuccess)
                    return LB3E_ERR_CUDA;
            }
        }
        for (int i = 0; i < n_; ++i) TRY(sims_[i]->init(phis[i], nullptr, nullptr, nullptr));
        std::vector<InstState<R, S>> tab(n_);
        std::vector<int4> tl, ptl;
        tl.reserve(ntiles_);
        ptl.reserve(nptiles_);
        for (int i = 0; i < n_; ++i) {
            const auto& d = sims_[i]->dev();
            InstState<R, S>& e = tab[i];
            e.P = sims_[i]->dev_params();
            e.pop[0] = d.pop[0];
            e.pop[1] = d.pop[1];
            e.h[0] = d.h[0];
            e.h[1] = d.h[1];
            e.phi = d.phi;
            e.qt = d.qt;
            e.q = d.q;
            e.eps = d.eps;
            e.E = d.E;
            e.prev = d.prev;
            e.diag = d.diag;
            const int gx = (e.P.nx + TX - 1) / TX, gy = (e.P.ny + TY - 1) / TY;
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) tl.push_back(make_int4(i, bx, by, 0));
            const int px = (e.P.nx + PB_TX - 1) / PB_TX, py = (e.P.ny + PB_TY - 1) / PB_TY;
            for (int by = 0; by < py; ++by)
                for (int bx = 0; bx < px; ++bx) ptl.push_back(make_int4(i, bx, by, 0));
        }
        // ping-pong parities shared by all instances (every electric instance ran
        // the same fixed number of initial potential iterations)
        cur_ = 0;
        hcur_ = 0;
        for (auto* s : sims_)
            if (s->dev_params().electric) { hcur_ = s->hcur(); break; }
        steps_ = 0;
        if (cudaMemcpyAsync(table_, tab.data(), n_ * sizeof(InstState<R, S>), cudaMemcpyHostToDevice, stream_) !=
                cudaSuccess ||
            cudaMemcpyAsync(tiles_, tl.data(), tl.size() * sizeof(int4), cudaMemcpyHostToDevice, stream_) !=
                cudaSuccess ||
            cudaMemcpyAsync(ptiles_, ptl.data(), ptl.size() * sizeof(int4), cudaMemcpyHostToDevice, stream_) !=
                cudaSuccess ||
            cudaStreamSynchronize(stream_) != cudaSuccess)
            return LB3E_ERR_CUDA;
        return set_fused_tile(8);
    }

    // tile height of the fused pass (32 x rows cells a block): 4, 8, or 16 in the FP32
    // compute builds; the result does not depend on it, the speed does
    int set_fused_tile(int rows) override {
        if (rows != 4 && rows != 8 && !(rows == 16 && std::is_same<R, float>::value)) return LB3E_ERR_PARAM;
        std::vector<int4> ft;
        for (int i = 0; i < n_; ++i) {
            const DevParams& P = sims_[i]->dev_params();
            const int gx = (P.nx + TX - 1) / TX, gy = (P.ny + rows - 1) / rows;
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) ft.push_back(make_int4(i, bx, by, 0));
        }
        if (cudaMemcpyAsync(ftiles_, ft.data(), ft.size() * sizeof(int4), cudaMemcpyHostToDevice, stream_) !=
                cudaSuccess ||
            cudaStreamSynchronize(stream_) != cudaSuccess)
            return LB3E_ERR_CUDA;
        nftiles_ = (int)ft.size();
        ftile_ = rows;
        return LB3E_OK;
    }

    int run(int nsteps) override {
        int done = 0;
        while (done < nsteps) {
            const int left = nsteps - done;
            int k = 1;
            // pairs of steps by graph (not on the legacy default stream, which cannot be
            // captured); the last step stays a plain launch
            if (stream_ != nullptr && steps_ > 0 && left > 2) {
                cudaGraphExec_t g = nullptr;
                TRY(graph_for(cur_, hcur_, &g));
                if (cudaGraphLaunch(g, stream_) != cudaSuccess) return LB3E_ERR_CUDA;
                launches += 2 * (3 + swaps() + (iters_ > 0));
                k = 2;
            } else {
                TRY(issue_step(cur_, hcur_, steps_ == 0, left == 1));
            }
            for (auto* s : sims_) s->stepped_externally(k, iters_, swaps());
            cur_ ^= k & 1;
            hcur_ ^= (k * swaps()) & 1;
            steps_ += k;
            done += k;
        }
        return cudaStreamSynchronize(stream_) == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }

    int observables(lb3e_observables_t* out) override {
        for (int i = 0; i < n_; ++i) TRY(sims_[i]->observables(out + i));
        return LB3E_OK;
    }
    int get_field(int inst, int id, double* dst) override {
        if (inst < 0 || inst >= n_) return LB3E_ERR_PARAM;
        return sims_[inst]->get_field(id, dst);
    }
    int count() const override { return n_; }
    int64_t total_launches() const override {
        int64_t l = launches;
        for (auto* s : sims_) l += s->launches;
        return l;
    }

    // pseudo-iterations per potential launch (1: one iteration per launch; 2
    // blocked on a 2-cell halo, 3..4 on a 4-cell halo, 5..8 on an 8-cell halo);
    // chosen by the caller's autotuner
    int set_chunk(int k) override {
        if (k < 1 || k > PB_HALO) return LB3E_ERR_PARAM;
        if constexpr (is_dual<R>::value) return k == 1 ? LB3E_OK : LB3E_ERR_PARAM;
        if (k > 1 && !pb_ready_) {
            if (cudaFuncSetAttribute(kb_poisson_tb<R, S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pb_smem_bytes<R, 2>()) != cudaSuccess ||
                cudaFuncSetAttribute(kb_poisson_tb<R, S, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pb_smem_bytes<R, 4>()) != cudaSuccess ||
                cudaFuncSetAttribute(kb_poisson_tb<R, S, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pb_smem_bytes<R, 4>()) != cudaSuccess ||
                cudaFuncSetAttribute(kb_poisson_tb<R, S, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pb_smem_bytes<R, 8>()) != cudaSuccess)
                return LB3E_ERR_CUDA;
            pb_ready_ = true;
        }
        chunk_ = k;
        return LB3E_OK;
    }

  private:
    struct Graph {
        int cur, hcur, chunk, ftile;
        cudaGraphExec_t exec;
    };
    // potential launches per step (each swaps the h buffers once)
    int swaps() const { return iters_ == 0 ? 0 : (chunk_ <= 1 ? iters_ : (iters_ + chunk_ - 1) / chunk_); }
    int issue_step(int cur, int hcur, bool first, bool diag) {
        const dim3 blk(TX, TY);
        kb_moments<R, S><<<ntiles_, blk, 0, stream_>>>(table_, tiles_, cur);
        kb_prologue<R, S><<<ntiles_, blk, 0, stream_>>>(table_, tiles_);
        int h = hcur;
        if (chunk_ <= 1) {
            for (int k = 0; k < iters_; ++k, h ^= 1) kb_poisson<R, S><<<ntiles_, blk, 0, stream_>>>(table_, tiles_, h);
        } else {
            for (int k = 0; k < iters_; k += chunk_, h ^= 1) {
                const int c = iters_ - k < chunk_ ? iters_ - k : chunk_;
                if (pb_halo_for(c) == 2)
                    kb_poisson_tb<R, S, 2><<<nptiles_, pb_threads<R, 2>(), pb_smem_bytes<R, 2>(), stream_>>>(
                        table_, ptiles_, h, c);
                else if (c == 4)
                    kb_poisson_tb<R, S, 4, 4><<<nptiles_, pb_threads<R, 4>(), pb_smem_bytes<R, 4>(), stream_>>>(
                        table_, ptiles_, h, c);
                else if (pb_halo_for(c) == 4)
                    kb_poisson_tb<R, S, 4><<<nptiles_, pb_threads<R, 4>(), pb_smem_bytes<R, 4>(), stream_>>>(
                        table_, ptiles_, h, c);
                else
                    kb_poisson_tb<R, S, 8><<<nptiles_, pb_threads<R, 8>(), pb_smem_bytes<R, 8>(), stream_>>>(
                        table_, ptiles_, h, c);
            }
        }
        if (iters_ > 0) kb_potential_fields<R, S><<<ntiles_, blk, 0, stream_>>>(table_, tiles_, h);
        if (ftile_ == 4)
            kb_fused<R, S, 4><<<nftiles_, dim3(TX, 4), fused_dyn_smem<R, S, 4>(), stream_>>>(table_, ftiles_, cur,
                                                                                           first ? 1 : 0, diag ? 1 : 0);
        else if (ftile_ == 8)
            kb_fused<R, S, 8><<<nftiles_, dim3(TX, 8), fused_dyn_smem<R, S, 8>(), stream_>>>(table_, ftiles_, cur,
                                                                                           first ? 1 : 0, diag ? 1 : 0);
        else if constexpr (std::is_same<R, float>::value)
            kb_fused<R, S, 16><<<nftiles_, dim3(TX, 16), fused_dyn_smem<R, S, 16>(), stream_>>>(
                table_, ftiles_, cur, first ? 1 : 0, diag ? 1 : 0);
        launches += 3 + swaps() + (iters_ > 0);
        return cudaGetLastError() == cudaSuccess ? LB3E_OK : LB3E_ERR_CUDA;
    }
    int graph_for(int cur, int hcur, cudaGraphExec_t* out) {
        for (auto& g : graphs_)
            if (g.cur == cur && g.hcur == hcur && g.chunk == chunk_ && g.ftile == ftile_) { *out = g.exec; return LB3E_OK; }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LB3E_ERR_CUDA;
        const int64_t l0 = launches;
        int rc = issue_step(cur, hcur, false, false);
        if (rc == LB3E_OK) rc = issue_step(cur ^ 1, hcur ^ (swaps() & 1), false, false);
        launches = l0;  // counted when the graph is launched
        if (cudaStreamEndCapture(stream_, &graph) != cudaSuccess || rc != LB3E_OK) {
            if (graph) cudaGraphDestroy(graph);
            return LB3E_ERR_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return LB3E_ERR_CUDA;
        graphs_.push_back({cur, hcur, chunk_, ftile_, exec});
        *out = exec;
        return LB3E_OK;
    }

    cudaStream_t stream_;
    int n_ = 0, ntiles_ = 0, nptiles_ = 0, nftiles_ = 0, ftile_ = 8, iters_ = 0, chunk_ = 1;
    bool pb_ready_ = false;
    int cur_ = 0, hcur_ = 0;
    int64_t steps_ = 0;
    InstState<R, S>* table_ = nullptr;
    int4* tiles_ = nullptr;
    int4* ptiles_ = nullptr;
    int4* ftiles_ = nullptr;  // the fused pass's tiles of 32 x ftile_ cells
    std::vector<Sim<R, S>*> sims_;
    std::vector<Graph> graphs_;
};

}  // namespace lb3e
