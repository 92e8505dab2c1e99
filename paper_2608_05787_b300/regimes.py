"""Outcome measures for the two-drop and confined-shear studies (host-side, on
fields read back from the GPU): connected drop regions with x periodic, the
centroid distance of a drop pair and the matrix film between them, and the
deformation and inclination of a drop from second moments.

A drop region is where the matrix fraction is below one half (phases 2 and 3
together, the compound drop); regions smaller than `min_cells` are ignored.
"""
from __future__ import annotations

import math

import numpy as np


def drop_regions(phi_matrix: np.ndarray, min_cells: int = 20):
    """Labels of the drop regions (4-connected, periodic in x): (labels, sizes)
    with labels 1..k in order of decreasing size; 0 marks the matrix."""
    from scipy import ndimage
    mask = phi_matrix < 0.5
    lab, n = ndimage.label(mask)
    if n == 0:
        return lab, []
    # merge regions that meet across the periodic x boundary
    parent = list(range(n + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    left, right = lab[:, 0], lab[:, -1]
    for a, b in zip(left, right):
        if a and b:
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[rb] = ra
    roots = np.array([find(i) for i in range(n + 1)])
    merged = roots[lab]
    sizes = {r: int((merged == r).sum()) for r in set(roots[1:].tolist())}
    keep = sorted((r for r, s in sizes.items() if s >= min_cells), key=lambda r: -sizes[r])
    out = np.zeros_like(lab)
    for k, r in enumerate(keep, start=1):
        out[merged == r] = k
    return out, [sizes[r] for r in keep]


def count_drops(phi_matrix: np.ndarray, min_cells: int = 20) -> int:
    return len(drop_regions(phi_matrix, min_cells)[1])


def pair_measures(phi_matrix: np.ndarray) -> dict:
    """For two drops stacked along y about the lattice centre: the distance of the
    centroids of the drop fractions (1 - phi_matrix) in the lower and upper halves,
    and the largest matrix fraction on the line x = nx/2 between the two centroids
    (1: a full film of matrix separates them; ~0: they have merged)."""
    ny, nx = phi_matrix.shape
    chi = 1.0 - phi_matrix
    y = np.arange(ny, dtype=float)[:, None]
    lo, hi = chi[: ny // 2], chi[ny // 2:]
    c_lo = float((lo * y[: ny // 2]).sum() / lo.sum())
    c_hi = float((hi * y[ny // 2:]).sum() / hi.sum())
    a, b = int(math.ceil(c_lo)), int(math.floor(c_hi))
    film = float(phi_matrix[a:b + 1, nx // 2].max()) if b >= a else 0.0
    return {"distance": c_hi - c_lo, "film": film}


def shape_measures(phi_matrix: np.ndarray) -> dict:
    """Deformation D = (a - b)/(a + b) of the drop fraction chi = 1 - phi_matrix from
    the eigenvalues of its second-moment tensor (a, b: the semi-axes of the
    equivalent ellipse), and the inclination of the major axis to the x axis in
    degrees (0..180).  x is periodic: moments are taken about the circular centroid."""
    ny, nx = phi_matrix.shape
    chi = 1.0 - phi_matrix
    m = chi.sum()
    x = np.arange(nx, dtype=float)[None, :]
    y = np.arange(ny, dtype=float)[:, None]
    ang = 2 * np.pi * x / nx
    cx = (math.atan2((chi * np.sin(ang)).sum(), (chi * np.cos(ang)).sum()) % (2 * np.pi)) * nx / (2 * np.pi)
    cy = float((chi * y).sum() / m)
    dx = (x - cx + nx / 2) % nx - nx / 2
    dy = y - cy
    ixx = float((chi * dx * dx).sum() / m)
    iyy = float((chi * dy * dy).sum() / m)
    ixy = float((chi * dx * dy).sum() / m)
    tr, det = ixx + iyy, ixx * iyy - ixy * ixy
    l1 = tr / 2 + math.sqrt(max(tr * tr / 4 - det, 0.0))
    l2 = tr / 2 - math.sqrt(max(tr * tr / 4 - det, 0.0))
    a, b = math.sqrt(max(l1, 0.0)), math.sqrt(max(l2, 0.0))
    theta = 0.5 * math.degrees(math.atan2(2 * ixy, ixx - iyy)) % 180.0
    return {"D": (a - b) / (a + b) if a + b > 0 else 0.0, "angle": theta}
