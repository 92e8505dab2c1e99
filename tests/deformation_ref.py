"""Test-side reference of the deformation factor (plain NumPy): D = (a - b)/(a + b)
from the second moments of an indicator field, a = 2 sqrt(Iyy) along y and b =
2 sqrt(Ixx) along x, and its derivative along a tangent of the field.  Used to
check the library's GPU reduction (lb3e_deformation) and to take finite
differences of D from fields."""
from __future__ import annotations

import numpy as np


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
