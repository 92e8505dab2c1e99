"""Parameter derivatives of the deformation factor (tangent builds) against
central finite differences in FP64, on the GPU and in the oracle.

Workload: compound drop under a field between electrodes, walls sliding at -/+1e-3
(the adjoint workload's setting) on a 64 x 64 lattice for 40 steps, the potential
iterated 20 times per step.  Finite differences use a relative step of 1e-4.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

WRT = ("V_top", "eps3", "gamma23")


def _setup(n=64, steps=40):
    E0 = W.field_for_capillary(0.5, 1e-3, 1.0, 16.0)
    p = W.params(nx=n, ny=n, bc_y=2, electric=1, eps=(1.0, 2.0, 4.0), sigma=(1.0, 0.5, 0.25), eps_ref=4.0,
                 V_top=E0 * n, u_wall_bottom=-1e-3, u_wall_top=1e-3, poisson_fixed_iter=20, precision=0)
    phi = W.compound_droplet(n, n, 8.0, 16.0, 4.0)
    return p, phi, steps


def _perturb(p, name, h):
    q = dict(p)
    if name == "V_top":
        q["V_top"] = p["V_top"] + h
    elif name == "eps3":
        q["eps"] = (p["eps"][0], p["eps"][1], p["eps"][2] + h)
    elif name == "gamma23":
        q["gamma23"] = p["gamma23"] + h
    return q


def _base(p, name):
    return {"V_top": p["V_top"], "eps3": p["eps"][2], "gamma23": p["gamma23"]}[name]


def _D_outer(field_fn, p):
    from paper_2608_05787_b300.gradients import deformation_from_moments
    chi = 1.0 - field_fn(f"phinow{p['matrix_phase']}")
    return deformation_from_moments(chi, [])[0]


def _fd_gpu(p, phi, steps, name):
    import paper_2608_05787_b300 as L
    h = 1e-4 * _base(p, name)
    vals = []
    for s in (+1, -1):
        sim = L.Sim(_perturb(p, name, s * h), phi)
        sim.step(steps)
        vals.append(_D_outer(sim.field, p))
    return (vals[0] - vals[1]) / (2 * h)


def _fd_oracle(p, phi, steps, name):
    h = 1e-4 * _base(p, name)
    vals = []
    for s in (+1, -1):
        o = oracle.Oracle(_perturb(p, name, s * h), phi)
        o.step(steps)
        vals.append(_D_outer(o.field, p))
    return (vals[0] - vals[1]) / (2 * h)


def test_fp64_tangent_matches_gpu_and_oracle_central_differences():
    from paper_2608_05787_b300.gradients import deformation_tangents
    p, phi, steps = _setup()
    D, g = deformation_tangents(p, phi, steps, wrt=WRT, precision=4)
    for name in WRT:
        fd_g = _fd_gpu(p, phi, steps, name)
        fd_o = _fd_oracle(p, phi, steps, name)
        print(f"{name}: tangent {g[name]:.9e}  fd(gpu) {fd_g:.9e}  fd(oracle) {fd_o:.9e}")
        assert abs(g[name] - fd_g) <= 1e-4 * abs(fd_g), name
        assert abs(g[name] - fd_o) <= 1e-4 * abs(fd_o), name


# FP32 tangent accuracy per parameter (relative to the FP64 tangent).  The
# tension derivative is the weakest: its effect on phi is a small difference
# between the tangents of the rest and the moving populations, which FP32 resolves
# to a few 1e-3 (measured 4.8e-3); the field and permittivity derivatives agree to
# a few 1e-6.
FP32_TOL = {"V_top": 1e-4, "eps3": 1e-4, "gamma23": 1e-2}


def test_fp32_tangent_matches_fp64_tangent():
    from paper_2608_05787_b300.gradients import deformation_tangents
    p, phi, steps = _setup()
    D64, g64 = deformation_tangents(p, phi, steps, wrt=WRT, precision=4)
    D32, g32 = deformation_tangents(p, phi, steps, wrt=WRT, precision=3)
    for name in WRT:
        print(f"{name}: fp32 {g32[name]:.6e} fp64 {g64[name]:.6e}")
        assert abs(g32[name] - g64[name]) <= FP32_TOL[name] * abs(g64[name]), name
    # D ~ 2e-4 is the small difference of two second-moment radii: FP32 fields give
    # it to a few 1e-3 (measured 2.0e-3)
    assert abs(D32 - D64) <= 5e-3 * abs(D64)


def test_tangent_value_is_the_plain_step():
    import paper_2608_05787_b300 as L
    p, phi, steps = _setup(steps=15)
    t = L.Sim(dict(p, precision=4, tangent_param=(0, -1, -1)), phi)
    s = L.Sim(p, phi)
    t.step(steps)
    s.step(steps)
    for f in ("phinow1", "phinow2", "phinow3", "ux", "q", "ex"):
        a, b = t.field(f), s.field(f)
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max(), f


def test_autograd_function_returns_the_tangent_derivatives():
    import torch

    from paper_2608_05787_b300.gradients import deformation, deformation_tangents
    p, phi, steps = _setup(steps=20)
    E0 = torch.tensor(p["V_top"] / p["ny"], dtype=torch.float64, requires_grad=True)
    er = torch.tensor(4.0, dtype=torch.float64, requires_grad=True)
    g23 = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    D = deformation(E0, er, g23, p, phi, steps)
    D.backward()
    _, g = deformation_tangents(p, phi, steps)
    assert abs(E0.grad.item() - g["V_top"] * p["ny"]) <= 1e-12 * abs(g["V_top"] * p["ny"])
    assert abs(er.grad.item() - g["eps3"]) <= 1e-12 * abs(g["eps3"])
    assert abs(g23.grad.item() - g["gamma23"]) <= 1e-12 * abs(g["gamma23"])
