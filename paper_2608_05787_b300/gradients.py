"""Derivatives of droplet deformation with respect to model parameters.

The step kernels are instantiated on dual numbers (the tangent builds, precision 3
and 4), so one run carries the exact derivative of the discrete state with respect
to up to three parameters alongside the state itself.  The library's
lb3e_deformation reduces the phase indicator's moments and their tangents on the GPU
and forms the deformation factor D = (r_par - r_perp) / (r_par + r_perp) of the
paper's Section 5.3 (radii from second moments) and its derivatives; this module
sequences the runs and wraps them in a torch.autograd.Function.
"""
from __future__ import annotations

from . import TANGENT_PARAMS, Sim


def deformation_tangents(params: dict, phi, steps: int, wrt=("V_top", "eps3", "gamma23"),
                         precision: int = 3, which: str = "outer") -> tuple[float, dict]:
    """Run `steps` steps in a tangent build and return D and {parameter: dD/dparameter}.
    Precision 3 (FP32) carries three directions in one run; precision 4 (FP64) one."""
    wrt = list(wrt)
    per_run = 3 if precision == 3 else 1
    out, D = {}, None
    for start in range(0, len(wrt), per_run):
        names = wrt[start:start + per_run]
        seeds = [TANGENT_PARAMS[nm] for nm in names] + [-1] * (3 - len(names))
        p = dict(params, precision=precision, tangent_param=tuple(seeds))
        sim = Sim(p, phi)
        sim.step(steps)
        Ds, dDs = sim.deformation()
        k = 1 if which == "outer" else 0
        D, g = Ds[k], list(dDs[k][:len(names)])
        out.update(dict(zip(names, g)))
        sim.close()
    return D, out


def shape_objective_tangents(params: dict, phi, steps: int, target, wrt=("V_top", "eps3", "gamma23"),
                             precision: int = 3) -> tuple[float, dict]:
    """Run `steps` steps in a tangent build and return the target-shape objective J =
    sum (phi_i - target_i)^2 (lb3e_shape_objective) and {parameter: dJ/dparameter}."""
    wrt = list(wrt)
    per_run = 3 if precision == 3 else 1
    out, J = {}, None
    for start in range(0, len(wrt), per_run):
        names = wrt[start:start + per_run]
        seeds = [TANGENT_PARAMS[nm] for nm in names] + [-1] * (3 - len(names))
        sim = Sim(dict(params, precision=precision, tangent_param=tuple(seeds)), phi)
        sim.step(steps)
        J, dJ = sim.shape_objective(target)
        out.update(dict(zip(names, dJ[:len(names)])))
        sim.close()
    return J, out


def _scaled_inputs(params: dict, E0, eps_ratio, gamma23) -> tuple[dict, float]:
    """The parameters with E0 (through the electrode potential), eps3 = eps_ratio eps1
    and gamma23 set; returns them and eps1."""
    p = dict(params)
    e1 = float(p["eps"][0])
    p["V_top"] = float(E0) * p["ny"] + p["V_bottom"]
    p["eps"] = (e1, p["eps"][1], float(eps_ratio) * e1)
    p["gamma23"] = float(gamma23)
    return p, e1


def _shape_fn():
    import torch

    class ShapeObjectiveFn(torch.autograd.Function):
        """The target-shape objective after `steps` steps as a differentiable function
        of E0, eps3/eps1 and gamma23 (forward: one FP32 tangent run; backward: the
        stored derivatives)."""

        @staticmethod
        def forward(ctx, E0, eps_ratio, gamma23, params, phi, steps, target):
            p, e1 = _scaled_inputs(params, E0, eps_ratio, gamma23)
            J, g = shape_objective_tangents(p, phi, steps, target)
            ctx.save_for_backward(torch.tensor([g["V_top"] * p["ny"], g["eps3"] * e1, g["gamma23"]],
                                               dtype=torch.float64))
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            (d,) = ctx.saved_tensors
            return grad * d[0], grad * d[1], grad * d[2], None, None, None, None

    return ShapeObjectiveFn


def shape_objective(E0, eps_ratio, gamma23, params: dict, phi, steps: int, target):
    """Differentiable target-shape objective (see ShapeObjectiveFn)."""
    return _shape_fn().apply(E0, eps_ratio, gamma23, params, phi, steps, target)


def _deformation_fn():
    import torch

    class DeformationFn(torch.autograd.Function):
        """D_outer after `steps` steps as a differentiable function of the field
        strength E0, the permittivity ratio eps3/eps1 and the tension gamma23
        (forward: one FP32 tangent run; backward: the stored derivatives)."""

        @staticmethod
        def forward(ctx, E0, eps_ratio, gamma23, params, phi, steps):
            p, e1 = _scaled_inputs(params, E0, eps_ratio, gamma23)
            D, g = deformation_tangents(p, phi, steps)
            ctx.save_for_backward(torch.tensor([g["V_top"] * p["ny"], g["eps3"] * e1, g["gamma23"]],
                                               dtype=torch.float64))
            return torch.tensor(D, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            (d,) = ctx.saved_tensors
            return grad * d[0], grad * d[1], grad * d[2], None, None, None

    return DeformationFn


def deformation(E0, eps_ratio, gamma23, params: dict, phi, steps: int):
    """Differentiable D_outer (see DeformationFn)."""
    return _deformation_fn().apply(E0, eps_ratio, gamma23, params, phi, steps)
