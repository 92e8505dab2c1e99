"""Compound-drop deformation regimes under a field (the paper's Section 5.3, its
Figs. 7-9): for (R12, R23, S12, S23) = (10, 8, 0.1, 5), (10, 0.1, 2, 0.5) and
(0.1, 10, 2, 0.5) the paper reports (D12, D23) = (+, +), (+, -), (-, +), D12 the
inner (core-shell) and D23 the outer (shell-matrix) deformation, positive when
elongated along the field.  These signs come from the leaky-dielectric charge
balance at each interface and test the whole coupling: charge transport, potential,
Maxwell stresses through mu and qE, and the flow.

Set-up: 256 x 256, core radius 20, shell radius 40, Ca_E = 0.2 (Eq. 51 with the
matrix permittivity), FP32, one batch.  The paper's ratios (its phase 1 core, 3 bulk)
fix eps and sigma up to a scale; conductivities are scaled so that sigma / eps <= 0.5
in every phase (charge relaxation resolved by the time step).  After 120k steps the
signs are settled; the (-, +) core passes through zero near 70k steps and keeps
falling."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

CASES = {(+1, +1): (10.0, 8.0, 0.1, 5.0), (+1, -1): (10.0, 0.1, 2.0, 0.5), (-1, +1): (0.1, 10.0, 2.0, 0.5)}


def _instance(R12, R23, S12, S23, n=256, r_out=40.0, r_in=20.0):
    eps, sig = W._ratios_to_props(S12=S12, S23=S23, R12=R12, R23=R23, sigma_matrix=0.05)
    scale = max(s / e for s, e in zip(sig, eps))
    if scale > 0.5:
        sig = tuple(s * 0.5 / scale for s in sig)
    E0 = W.field_for_capillary(0.2, 1e-3, eps[0], r_out)
    p = W.params(nx=n, ny=n, bc_y=2, electric=1, precision=1, eps=eps, sigma=sig, eps_ref=max(eps), V_top=E0 * n,
                 poisson_fixed_iter=16)
    return p, W.compound_droplet(n, n, r_in, r_out, 4.0)


def test_deformation_signs_of_the_three_regimes():
    import paper_2608_05787_b300 as L
    inst = [_instance(*v) for v in CASES.values()]
    b = L.Batch([p for p, _ in inst], [phi for _, phi in inst]).set_chunk(4)
    b.run(120000)
    obs = b.observables()
    for (s_in, s_out), o in zip(CASES, obs):
        assert o["nonfinite"] == 0
        # measured (1.2e5 steps): (+,+) 0.0073, 0.069; (+,-) 0.084, -0.082; (-,+) -0.0040, 0.072
        assert s_in * o["D_inner"] > 0.002, (s_in, s_out, o["D_inner"], o["D_outer"])
        assert s_out * o["D_outer"] > 0.03, (s_in, s_out, o["D_inner"], o["D_outer"])
