"""Spreading liquid lens (512 x 256, walls, no field): Neumann-triangle angles and
chord (Eq. 57-58), FP32 against FP64 after the stated 20 000 steps, and FP64
parity with the oracle at full size over a shorter horizon.

At the stated 20 000 steps the lens is still spreading (67 degrees on its way to
60 for equal tensions); the angles settle after about 4e5 steps, so the
equilibrium check runs 400 000 steps (10 s in FP32).

Labels: phase 1 upper layer, phase 2 lower layer, phase 3 lens (radius 40).
Angles are measured from the flat upper|lower interface: the upper cap meets it
at theta_up, with cos theta_up = (g12^2 + g13^2 - g23^2) / (2 g12 g13), and the
lower cap at theta_low likewise with 13 <-> 23.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from lens_geometry import measure_lens, neumann

pytestmark = pytest.mark.gpu

TRIPLES = [(1e-3, 1e-3, 1e-3), (1e-3, 8e-4, 6e-4)]


def _run(precision, tens, steps):
    import paper_2608_05787_b300 as L
    cfg = W.config_lens(tensions=tens, precision=precision)
    sim = L.Sim(cfg["params"], cfg["phi"])
    sim.step(steps)
    return sim


@pytest.mark.slow
@pytest.mark.parametrize("tens", TRIPLES)
def test_lens_neumann_angles_and_chord(tens):
    """Equilibrium cap angles within 9% and chord within 6% of Eq. 57-58 (the paper
    reports 0.5-6% for its own runs, Table 2)."""
    sim = _run(1, tens, 400000)
    p1, p2, p3 = (sim.field(f"phinow{i}") for i in (1, 2, 3))
    th_up, th_lo, d = measure_lens(p1, p2, p3)
    a_up, a_lo, a_d = neumann(*tens, area=float(p3.sum()))
    print(f"lens {tens}: theta_up {th_up:.2f} (Neumann {a_up:.2f}), theta_low {th_lo:.2f} "
          f"({a_lo:.2f}), d {d:.2f} ({a_d:.2f})")
    assert abs(th_up / a_up - 1) < 0.09
    assert abs(th_lo / a_lo - 1) < 0.09
    assert abs(d / a_d - 1) < 0.06


@pytest.mark.slow
def test_lens_fp32_against_fp64_after_20000_steps():
    """FP32 phase fields against the FP64 GPU run over the stated 20 000 steps of a
    spreading (moving-contact-line) lens, gated at each step count of
    tests/golden/lens_sensitivity.json by the FP64 oracle's own response to
    FP32-size perturbations that push every stored value the same way every step
    (the "correlated" model; written from the oracle alone by
    make_lens_sensitivity.py).  The deviation grows about linearly with the steps
    (1.2e-6 after 100, 1.4e-5 after 2000, 1.4e-4 after 20 000): the rounding of a
    slowly changing state by the same FP32 arithmetic is correlated in time, and the
    lens's motion is a small residual of cancelling forces.  It lies between the
    oracle's uncorrelated and correlated responses.  FP32 copies of the parameters
    (1.8e-7 after 20 000 steps in an FP64 run) and of the initial phases (2e-8)
    account for none of it, nor does storage rounding (2e-9 after 2000 steps)."""
    import json
    from pathlib import Path
    ref = json.loads((Path(__file__).parent / "golden" / "lens_sensitivity.json").read_text())["after"]
    tens = TRIPLES[1]
    import paper_2608_05787_b300 as L
    sims = {}
    for prec in (0, 1):
        cfg = W.config_lens(tensions=tens, precision=prec)
        sims[prec] = L.Sim(cfg["params"], cfg["phi"])
    done = 0
    for n in sorted(int(k) for k in ref):
        for s in sims.values():
            s.step(n - done)
        done = n
        err = max(float(np.abs(sims[1].field(f) - sims[0].field(f)).max() / np.abs(sims[0].field(f)).max())
                  for f in ("phinow1", "phinow2", "phinow3"))
        bound = ref[str(n)]["correlated"]
        print(f"lens fp32 vs fp64 after {n} steps: {err:.3e} (oracle: uncorrelated "
              f"{ref[str(n)]['uncorrelated']:.2e}, correlated {bound:.2e})")
        assert err <= bound, (n, err, bound)


@pytest.mark.slow
def test_lens_fp64_full_size_parity_with_oracle():
    tens = TRIPLES[1]
    cfg = W.config_lens(tensions=tens, precision=0)
    import paper_2608_05787_b300 as L
    sim = L.Sim(cfg["params"], cfg["phi"])
    orc = oracle.Oracle(cfg["params"], cfg["phi"])
    sim.step(150)
    orc.step(150)
    for f in ("phinow1", "phinow2", "phinow3", "ux", "uy", "p", "mu1", "mu3"):
        ref = orc.field(f)
        assert np.abs(sim.field(f) - ref).max() <= 1e-12 * np.abs(ref).max(), f
