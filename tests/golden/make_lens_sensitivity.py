"""Writes lens_sensitivity.json: how far the FP64 oracle's own phase fields move under
perturbations of the FP32 size on the stated spreading lens (512 x 256, walls, no
field, tensions 1e-3 / 8e-4 / 6e-4, 20 000 steps).

Three oracle runs in lock step from the same state; before every step the second
and third have every stored population (and the FP32 anchor phi_i) perturbed by
u * 2^-24 * |v|, u uniform in [-1, 1) from a seeded hash (oracle.Oracle.perturb):
* "uncorrelated": a fresh seed every step, so the perturbations are a random walk;
* "correlated": the same seed every step, so each value is pushed the same way
  step after step, as the rounding of a slowly changing state by the same
  arithmetic is.
The FP32 build's deviation lies between the two if it is FP32 rounding that the
scheme amplifies.  (Rounding only the stored populations to FP32 every step moves the
fields by 2e-9 after 2000 steps: storage is not what the FP32 build's deviation is
made of.)  For each of phinow1..3: max |perturbed - plain| / max |plain| after 2000,
5000, 10 000 and 20 000 steps; the file is rewritten at each of them.  Only the
oracle runs here (about two hours on 8 cores).
Usage: python tests/golden/make_lens_sensitivity.py
"""
from __future__ import annotations

import json
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

TENSIONS = (1e-3, 8e-4, 6e-4)
FIELDS = ("phinow1", "phinow2", "phinow3")
STEPS = 20000
REPORT = (2000, 5000, 10000, 20000)
U = 2.0 ** -24


def _diff(a, b) -> float:
    return max(float(np.abs(a.field(f) - b.field(f)).max() / np.abs(a.field(f)).max()) for f in FIELDS)


def main():
    cfg = W.config_lens(tensions=TENSIONS, precision=0)
    a, b, c = (oracle.Oracle(cfg["params"], cfg["phi"]) for _ in range(3))
    out = {"workload": "spreading lens 512x256, walls, no field, tensions %s" % (TENSIONS,),
           "models": {"uncorrelated": "stored values perturbed at the FP32 unit roundoff, a fresh seed every step",
                      "correlated": "stored values perturbed at the FP32 unit roundoff, the same seed every step"},
           "after": {}}
    for k in range(STEPS):
        b.perturb(U, 0.0, U, seed=k + 1)
        c.perturb(U, 0.0, U, seed=1)
        a.step(1)
        b.step(1)
        c.step(1)
        if k + 1 in REPORT:
            out["after"][str(k + 1)] = {"uncorrelated": _diff(a, b), "correlated": _diff(a, c)}
            print(k + 1, out["after"][str(k + 1)], flush=True)
            (Path(__file__).parent / "lens_sensitivity.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
