"""Outcome measures of the two-drop and confined-shear studies, on synthetic
shapes with known answers (host-side code, no GPU)."""
import math

import numpy as np

import workloads as W
from paper_2608_05787_b300 import regimes


def _disk_matrix(nx, ny, centres, r, W_=4.0):
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    drop = np.zeros((ny, nx))
    for cx, cy in centres:
        dx = (x - cx + nx / 2) % nx - nx / 2  # periodic in x
        drop = np.maximum(drop, 0.5 + 0.5 * np.tanh(2 * (r - np.hypot(dx, y - cy)) / W_))
    return 1.0 - drop


def test_counts_separate_drops_and_merges_across_the_periodic_edge():
    assert regimes.count_drops(_disk_matrix(128, 64, [(40, 32), (90, 32)], 10)) == 2
    # one drop centred on the x seam is one region, not two halves
    assert regimes.count_drops(_disk_matrix(128, 64, [(0, 32)], 10)) == 1
    assert regimes.count_drops(_disk_matrix(128, 64, [], 10)) == 0


def test_pair_measures_of_the_initial_two_drops():
    n, r_in, r_out, gap = 256, 12.0, 24.0, 8.0
    phi = W.two_compound_drops(n, n, r_in, r_out, 4.0, gap)
    m = regimes.pair_measures(phi[0])
    assert abs(m["distance"] - 2 * (r_out + gap / 2)) < 0.5
    assert m["film"] > 0.95                       # a full matrix film between them
    assert regimes.count_drops(phi[0]) == 2


def test_shape_measures_of_a_tilted_ellipse():
    nx, ny, a, b, th = 256, 200, 40.0, 20.0, math.radians(30)
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    dx, dy = x - 128, y - 100
    u = dx * math.cos(th) + dy * math.sin(th)
    v = -dx * math.sin(th) + dy * math.cos(th)
    inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    m = regimes.shape_measures(np.where(inside, 0.0, 1.0))
    assert abs(m["D"] - (a - b) / (a + b)) < 0.01
    assert abs(m["angle"] - 30.0) < 0.5
