// lb3e_params.cuh -- derived constants of the model (host side).
#pragma once

#include "lb3e_internal.h"
#include "lb3e_kernels.cuh"

namespace lb3e {

// lambda_i of Eq. 9, m0 = cs^2 (tau_f - 1/2), tau_h = 1/2 + eps_ref/cs^2 (Eq. 43),
// tau_l = 1/2 + alpha/cs^2 (Eq. 49)
inline DevParams make_dev_params(const lb3e_params& p) {
    DevParams d{};
    d.nx = p.nx;
    d.ny = p.ny;
    d.N = p.nx * p.ny;
    d.bc_y = p.bc_y;
    d.electric = p.electric;
    d.charge_convection = p.charge_convection;
    d.use_visc = p.visc[0] > 0 && p.visc[1] > 0 && p.visc[2] > 0;
    d.inner = p.inner_phase - 1;
    d.matrix = p.matrix_phase - 1;
    for (int i = 0; i < 3; ++i) {
        d.rho[i] = p.rho[i];
        d.visc[i] = p.visc[i];
        d.eps[i] = p.eps[i];
        d.sigma[i] = p.sigma[i];
    }
    d.lam[0] = p.gamma12 + p.gamma13 - p.gamma23;
    d.lam[1] = p.gamma12 + p.gamma23 - p.gamma13;
    d.lam[2] = p.gamma13 + p.gamma23 - p.gamma12;
    d.tau_g = p.tau_g;
    d.D = p.width_D;
    d.tau_f = p.tau_f;
    d.m0 = (1.0 / 3.0) * (p.tau_f - 0.5);
    d.eps_ref = p.eps_ref;
    d.tau_h = 0.5 + p.eps_ref / (1.0 / 3.0);
    d.alpha = p.alpha;
    d.tau_l = 0.5 + p.alpha / (1.0 / 3.0);
    d.V_bottom = p.V_bottom;
    d.V_top = p.V_top;
    d.E_ext[0] = p.E_ext[0];
    d.E_ext[1] = p.E_ext[1];
    d.u_wall_bottom = p.u_wall_bottom;
    d.u_wall_top = p.u_wall_top;
    for (int i = 0; i < 3; ++i) {
        d.frho[i] = (float)d.rho[i];
        d.fvisc[i] = (float)d.visc[i];
        d.feps[i] = (float)d.eps[i];
        d.fsig[i] = (float)d.sigma[i];
        d.flam[i] = (float)d.lam[i];
    }
    d.fD = (float)d.D;
    d.ftau_f = (float)d.tau_f;
    d.fm0 = (float)d.m0;
    d.ftau_g = (float)d.tau_g;
    d.ftau_l = (float)d.tau_l;
    d.ftau_h = (float)d.tau_h;
    d.feps_ref = (float)d.eps_ref;
    d.fVb = (float)d.V_bottom;
    d.fVt = (float)d.V_top;
    d.fuwb = (float)d.u_wall_bottom;
    d.fuwt = (float)d.u_wall_top;
    d.fE[0] = (float)d.E_ext[0];
    d.fE[1] = (float)d.E_ext[1];
    d.fitau_f = (float)(1.0 / d.tau_f);
    d.fpf = (float)(1.0 - 1.0 / (2.0 * d.tau_f));
    d.fim0 = (float)(1.0 / d.m0);
    d.fitau_g = (float)(1.0 / d.tau_g);
    d.fpg = (float)(1.0 - 1.0 / (2.0 * d.tau_g));
    d.fitau_l = (float)(1.0 / d.tau_l);
    d.fpl = (float)(1.0 - 1.0 / (2.0 * d.tau_l));
    d.fitau_h = (float)(1.0 / d.tau_h);
    d.fc24 = (float)(24.0 / d.D);
    // tangent seeds: d lambda_i / d gamma_jk from Eq. 9
    static const double dlam[3][3] = {{1, 1, -1}, {1, -1, 1}, {-1, 1, 1}};
    for (int k = 0; k < 3; ++k) {
        const int id = p.tangent_param[k];
        if (id == 0) d.t_Vt[k] = 1.0;
        if (id >= 1 && id <= 3) d.t_eps[id - 1][k] = 1.0;
        if (id >= 4 && id <= 6)
            for (int i = 0; i < 3; ++i) d.t_lam[i][k] = dlam[i][id - 4];
    }
    return d;
}

}  // namespace lb3e
