"""Lens geometry for the spreading-lens checks: the Neumann-triangle closed form
(Eq. 57-58) and the measurement of cap angles and chord from phase fields."""
import math

import numpy as np


def neumann(g12, g13, g23, area):
    """Eq. 57-58: cap angles and the chord d enclosing the lens area."""
    th_up = math.acos((g12 ** 2 + g13 ** 2 - g23 ** 2) / (2 * g12 * g13))
    th_lo = math.acos((g12 ** 2 + g23 ** 2 - g13 ** 2) / (2 * g12 * g23))
    s = sum((t / math.sin(t) - math.cos(t)) / math.sin(t) for t in (th_up, th_lo))
    d = 2 * math.sqrt(area / s)
    return math.degrees(th_up), math.degrees(th_lo), d


def _crossing(a, b, profile=None):
    """First linear-interpolated index where profile (a - b) changes sign."""
    f = a - b
    idx = np.where(np.sign(f[:-1]) != np.sign(f[1:]))[0]
    if len(idx) == 0:
        return None
    k = idx[0]
    return k + f[k] / (f[k] - f[k + 1])


def measure_lens(phi1, phi2, phi3):
    """Cap heights on the centre column, chord on the flat-interface level, and
    circular-cap angles theta = 2 atan(2 h / d)."""
    ny, nx = phi1.shape
    # flat interface level far from the lens (left and right edges)
    levels = []
    for x in (2, nx - 3):
        c = _crossing(phi2[:, x], phi1[:, x], None)
        levels.append(c)
    y0 = float(np.mean(levels))
    xc = int(np.argmax(phi3.sum(axis=0)))
    col3, col1, col2 = phi3[:, xc], phi1[:, xc], phi2[:, xc]
    yi = int(np.argmax(col3))
    up = _crossing(col3[yi:], col1[yi:], None)
    lo = _crossing(col3[:yi + 1][::-1], col2[:yi + 1][::-1], None)
    y_top, y_bot = yi + up, yi - lo
    # chord: lens extent (phi3 = 1/2) on the row of the flat interface
    j = int(math.floor(y0))
    w = y0 - j
    row = (1 - w) * phi3[j] + w * phi3[j + 1]
    inside = np.where(row >= 0.5)[0]
    left, right = inside[0], inside[-1]
    xl = left - 1 + (0.5 - row[left - 1]) / (row[left] - row[left - 1])
    xr = right + (row[right] - 0.5) / (row[right] - row[right + 1])
    d = xr - xl
    h_up, h_lo = y_top - y0, y0 - y_bot
    th_up = math.degrees(2 * math.atan(2 * h_up / d))
    th_lo = math.degrees(2 * math.atan(2 * h_lo / d))
    return th_up, th_lo, d


