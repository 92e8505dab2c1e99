"""The test-side deformation factor and its tangent (no GPU): the reference the
library's lb3e_deformation is checked against."""
import numpy as np

from deformation_ref import deformation_from_moments  # tests/ is on sys.path (pytest rootdir conftest)


def _ellipse(n, a, b, w=3.0):
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    r = np.sqrt(((x - n / 2) / b) ** 2 + ((y - n / 2) / a) ** 2)
    return 0.5 + 0.5 * np.tanh(2 * (1 - r) * min(a, b) / w)


def test_circle_has_zero_deformation_and_ellipse_the_moment_ratio():
    D0, _ = deformation_from_moments(_ellipse(96, 20, 20), [])
    assert abs(D0) < 1e-12
    D, _ = deformation_from_moments(_ellipse(128, 30, 20, w=1e-3), [])
    assert abs(D - (30 - 20) / (30 + 20)) < 0.01       # sharp ellipse: second-moment radii are the semi-axes


def test_tangent_matches_finite_difference():
    rng = np.random.default_rng(0)
    chi = _ellipse(64, 18, 14)
    dchi = rng.standard_normal(chi.shape) * chi * (1 - chi)
    _, (g,) = deformation_from_moments(chi, [dchi])
    h = 1e-6
    fd = (deformation_from_moments(chi + h * dchi, [])[0] - deformation_from_moments(chi - h * dchi, [])[0]) / (2 * h)
    assert abs(g - fd) <= 1e-6 * abs(fd)
