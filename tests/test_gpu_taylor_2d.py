"""Two-phase limit of the method against 2-D small-deformation theory of a
leaky-dielectric drop (derived in oracle/THEORY.md, the paper giving only its 3-D
compound form): D = (Ca_E / 3) (R^2 + R + 1 - 3S) / (R + 1)^2, R = sigma_in /
sigma_out, S = eps_in / eps_out.

A drop of phase 3 (radius 20, interface width 4) in phase 1, phase 2 absent (it
stays absent: reduction consistency), 256 x 256 between electrodes, equal
viscosities, FP32 batch, 40k steps (about 20 capillary times; D changes by < 1%
after 30k).  Checks: the sign, the magnitude within 10%, linearity in Ca_E within
10%."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N, A = 256, 20.0


def _two_phase_drop():
    x, y = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float))
    p3 = 0.5 + 0.5 * np.tanh(2.0 * (A - np.hypot(x - N / 2, y - N / 2)) / 4.0)
    return np.ascontiguousarray(np.stack([1.0 - p3, np.zeros_like(p3), p3]))


def _theory(R, S, ca):
    return ca / 3.0 * (R * R + R + 1.0 - 3.0 * S) / (R + 1.0) ** 2


def test_two_phase_drop_deformation_matches_small_deformation_theory():
    import paper_2608_05787_b300 as L
    cases = [(R, S, ca) for (R, S) in ((2.0, 1.0), (0.5, 2.0)) for ca in (0.05, 0.1)]
    params = []
    for R, S, ca in cases:
        eps, sig = (1.0, 1.0, S), (0.05, 0.05, 0.05 * R)
        E0 = W.field_for_capillary(ca, 1e-3, 1.0, A)
        params.append(W.params(nx=N, ny=N, bc_y=2, electric=1, precision=1, eps=eps, sigma=sig, eps_ref=max(eps),
                               V_top=E0 * N, poisson_fixed_iter=16, inner_phase=3, matrix_phase=1))
    phi = _two_phase_drop()
    b = L.Batch(params, [phi] * len(params)).set_chunk(4)
    b.run(40000)
    D = [o["D_inner"] for o in b.observables()]
    for (R, S, ca), d in zip(cases, D):
        th = _theory(R, S, ca)
        assert np.sign(d) == np.sign(th), (R, S, ca, d, th)
        assert abs(d - th) <= 0.10 * abs(th), (R, S, ca, d, th)
    for k in (0, 2):  # Ca_E 0.05 -> 0.1 doubles D
        assert abs(D[k + 1] / D[k] - 2.0) <= 0.2, (D[k], D[k + 1])
    assert np.abs(b.field(0, "phinow2")).max() < 1e-12
