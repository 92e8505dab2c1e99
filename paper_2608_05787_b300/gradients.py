"""Derivatives of droplet deformation with respect to model parameters.

The step kernels are instantiated on dual numbers (the tangent builds, precision 3
and 4), so one run carries the exact derivative of the discrete state with respect
to up to three parameters alongside the state itself.  This module turns the phase
fields and their tangents into the deformation factor D = (r_par - r_perp) /
(r_par + r_perp) of the paper's Section 4.4 (radii from second moments of the
phase indicator) and its derivatives, and wraps that in a torch.autograd.Function.
"""
from __future__ import annotations

import numpy as np

from . import TANGENT_PARAMS, Sim


def deformation_from_moments(chi: np.ndarray, dchi: list[np.ndarray]) -> tuple[float, list[float]]:
    """D from the second moments of the indicator chi (radius along y: 2 sqrt(Iyy),
    along x: 2 sqrt(Ixx)), and its derivative along each tangent field dchi[k]."""
    ny, nx = chi.shape
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    basis = (np.ones_like(x), x, y, x * x, y * y)
    m = [float((chi * b).sum()) for b in basis]
    A = m[0]
    xc, yc = m[1] / A, m[2] / A
    Ixx, Iyy = m[3] / A - xc * xc, m[4] / A - yc * yc
    a, b = 2 * np.sqrt(Iyy), 2 * np.sqrt(Ixx)
    D = (a - b) / (a + b)
    grads = []
    for dc in dchi:
        dm = [float((dc * bb).sum()) for bb in basis]
        dxc = (dm[1] - xc * dm[0]) / A
        dyc = (dm[2] - yc * dm[0]) / A
        dIxx = (dm[3] - (m[3] / A) * dm[0]) / A - 2 * xc * dxc
        dIyy = (dm[4] - (m[4] / A) * dm[0]) / A - 2 * yc * dyc
        da, db = dIyy / np.sqrt(Iyy), dIxx / np.sqrt(Ixx)
        grads.append(float(2 * (b * da - a * db) / (a + b) ** 2))
    return float(D), grads


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
        if which == "outer":
            k = int(params["matrix_phase"])
            chi = 1.0 - sim.field(f"phinow{k}")
            dchi = [-sim.field(f"phinow{k}", tangent=t + 1) for t in range(len(names))]
        else:
            k = int(params["inner_phase"])
            chi = sim.field(f"phinow{k}")
            dchi = [sim.field(f"phinow{k}", tangent=t + 1) for t in range(len(names))]
        D, g = deformation_from_moments(chi, dchi)
        out.update(dict(zip(names, g)))
        sim.close()
    return D, out


def _deformation_fn():
    import torch

    class DeformationFn(torch.autograd.Function):
        """D_outer after `steps` steps as a differentiable function of the field
        strength E0, the permittivity ratio eps3/eps1 and the tension gamma23
        (forward: one FP32 tangent run; backward: the stored derivatives)."""

        @staticmethod
        def forward(ctx, E0, eps_ratio, gamma23, params, phi, steps):
            p = dict(params)
            e1 = float(p["eps"][0])
            p["V_top"] = float(E0) * p["ny"] + p["V_bottom"]
            p["eps"] = (e1, p["eps"][1], float(eps_ratio) * e1)
            p["gamma23"] = float(gamma23)
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
