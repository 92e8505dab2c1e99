"""Consistency of the stored precision-sensitivity records (written from the oracle
alone by tests/golden/make_*_sensitivity.py), which the reduced-precision GPU tests
use as bounds."""
import json
from pathlib import Path

GOLDEN = Path(__file__).parent / "golden"


def test_lens_sensitivity_brackets_are_ordered_and_grow():
    """Correlated perturbations move the lens more than uncorrelated ones of the same
    size, and both responses grow with the number of steps."""
    d = json.loads((GOLDEN / "lens_sensitivity.json").read_text())["after"]
    steps = sorted(int(k) for k in d)
    assert steps and steps[0] == 2000
    for n in steps:
        u, c = d[str(n)]["uncorrelated"], d[str(n)]["correlated"]
        assert 0 < u < c < 1e-2, (n, u, c)
    for a, b in zip(steps, steps[1:]):
        assert d[str(b)]["correlated"] > d[str(a)]["correlated"]
        assert d[str(b)]["uncorrelated"] >= 0.5 * d[str(a)]["uncorrelated"]


def test_static_compound_sensitivity_covers_every_gated_field():
    """Every field the 2000-step reduced-precision test gates has a model value for
    each storage format, FP16 storage moves every field at least as far as FP32
    rounding does, and the velocity is the most sensitive field under FP32."""
    d = json.loads((GOLDEN / "precision_sensitivity.json").read_text())["formats"]
    fields = ("phi1", "phi2", "phi3", "phinow1", "phinow2", "phinow3", "qtilde", "ux", "uy", "p", "q", "psi",
              "ex", "ey", "mu1", "mu2", "mu3")
    for fmt in ("fp32", "fp16", "bf16"):
        for model in ("rounding", "perturbation"):
            assert all(d[fmt][model][f] >= 0 for f in fields), (fmt, model)
    assert all(d["fp16"]["rounding"][f] >= d["fp32"]["rounding"][f] for f in fields)
    fp32 = d["fp32"]["perturbation"]
    assert fp32["ux"] == max(fp32[f] for f in fields)
