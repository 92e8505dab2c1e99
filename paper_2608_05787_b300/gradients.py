"""Derivatives of droplet deformation with respect to model parameters.

Two modes, both exact derivatives of the discrete step:
* tangent (forward) mode: the step kernels instantiated on dual numbers (precision 3
  and 4) carry d(state)/d(theta) for up to three parameters alongside the state;
* reverse mode: the library's adjoint of the step (lb3e_adjoint_step), run backwards
  from the objective's seed with checkpoint-and-recompute, gives dJ/dtheta for all
  eleven parameter slots and dJ/dphi_init in one backward sweep.
The library reduces the phase indicator's moments on the GPU and forms the
deformation factor D = (r_par - r_perp) / (r_par + r_perp) of the paper's Section
5.3 (radii from second moments) and its seeds; this module sequences the runs and
wraps them in torch.autograd.Functions.
"""
from __future__ import annotations

import numpy as np

from . import ADJ_PARAMS, TANGENT_PARAMS, Sim


def reverse_gradient(params: dict, phi, steps: int, objective: str = "deformation", which: str = "outer",
                     target=None, checkpoint_every: int = 200, want_dphi: bool = False):
    """J after `steps` steps and its gradient by reverse mode: returns (J, {slot:
    dJ/dslot} over ADJ_PARAMS, dJ/dphi_init or None).  The forward run keeps a
    snapshot every `checkpoint_every` steps (device memory); the backward sweep
    re-runs each segment from its snapshot, keeping each step's state vector
    (lb3e_state_vector), and steps back through them with lb3e_adjoint_step_x on a
    stream of its own (each backward step a replayed CUDA graph, the parameter
    gradient accumulated on the device).  `objective`: "deformation" (D of
    lb3e_deformation, `which` inner or outer) or "shape" (lb3e_shape_objective
    against `target`).  The parameters must give a fixed potential count
    (poisson_fixed_iter > 0, potential_solver 0)."""
    import torch
    stream = torch.cuda.Stream()
    C = max(1, int(checkpoint_every))
    with torch.cuda.stream(stream):
        sim = Sim(params, phi, stream=stream)
        ckpt = {}
        for n in range(steps):
            if n % C == 0:
                ckpt[n] = sim.save_state()
            sim.step(1)
        J, a = sim.deformation_seed(which) if objective == "deformation" else sim.shape_seed(target)
        b = torch.empty_like(a)
        dpar = torch.zeros(len(ADJ_PARAMS), dtype=torch.float64, device=a.device)
        for start in sorted(ckpt, reverse=True):
            sim.load_state(ckpt[start])
            n_seg = min(start + C, steps) - start
            X = torch.empty((n_seg,) + tuple(a.shape), dtype=a.dtype, device=a.device)
            first = []
            for k in range(n_seg):
                first.append(sim.is_first_step)
                sim.state_vector(out=X[k])
                if k + 1 < n_seg:
                    sim.step(1)
            for k in reversed(range(n_seg)):
                sim.adjoint_step_x(X[k], first[k], a, b, dpar)
                a, b = b, a
            del X
        dp0, dphi0 = sim.adjoint_init(phi, a, want_dphi=want_dphi)
        stream.synchronize()
        total = dpar.cpu().numpy() + dp0
    sim.close()
    return J, dict(zip(ADJ_PARAMS, total.tolist())), dphi0


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


def _deformation_reverse_fn():
    import torch

    class DeformationReverseFn(torch.autograd.Function):
        """D_outer after `steps` steps as a differentiable function of E0, eps3/eps1
        and gamma23 (forward: the run and one reverse sweep with checkpoints every
        `checkpoint_every` steps; backward: the stored gradient)."""

        @staticmethod
        def forward(ctx, E0, eps_ratio, gamma23, params, phi, steps, checkpoint_every):
            p, e1 = _scaled_inputs(params, E0, eps_ratio, gamma23)
            D, g, _ = reverse_gradient(p, phi, steps, checkpoint_every=checkpoint_every)
            ctx.save_for_backward(torch.tensor([g["V_top"] * p["ny"], g["eps3"] * e1, g["gamma23"]],
                                               dtype=torch.float64))
            return torch.tensor(D, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            (d,) = ctx.saved_tensors
            return grad * d[0], grad * d[1], grad * d[2], None, None, None, None

    return DeformationReverseFn


def deformation_reverse(E0, eps_ratio, gamma23, params: dict, phi, steps: int, checkpoint_every: int = 200):
    """Differentiable D_outer by reverse mode (see DeformationReverseFn)."""
    return _deformation_reverse_fn().apply(E0, eps_ratio, gamma23, params, phi, steps, checkpoint_every)


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
