"""Writes lens_sensitivity.json: how far the FP64 oracle's own phase fields move under
rounding of the FP32 size on the stated spreading lens (512 x 256, walls, no field,
tensions 1e-3 / 8e-4 / 6e-4, 20 000 steps).

Three oracle runs in lock step from the same state:
* plain;
* "perturbation": before every step every stored population (and the FP32 anchor
  phi_i) is perturbed by u * 2^-24 * |v|, u uniform in [-1, 1) from a seeded hash
  (oracle.Oracle.perturb), fresh every step: rounding as a random walk;
* "rounding": after every step the stored populations are rounded to FP32 exactly
  as the FP32 build stores them (oracle.Oracle.round_storage): deterministic, so a
  cell whose values change slowly is rounded the same way step after step.
For each of phinow1..3: max |modified - plain| / max |plain| after 2000, 5000, 10 000
and 20 000 steps.  Only the oracle runs here (about 1.5 hours on 8 cores).
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


def _diff(a, b) -> dict:
    return {f: float(np.abs(a.field(f) - b.field(f)).max() / np.abs(a.field(f)).max()) for f in FIELDS}


def main():
    cfg = W.config_lens(tensions=TENSIONS, precision=0)
    a, b, c = (oracle.Oracle(cfg["params"], cfg["phi"]) for _ in range(3))
    c.round_storage("fp32")
    out = {"workload": "spreading lens 512x256, walls, no field, tensions %s" % (TENSIONS,),
           "models": {"perturbation": "every stored value perturbed at the FP32 unit roundoff before every step",
                      "rounding": "the stored populations rounded to FP32 after every step"},
           "after": {}}
    for k in range(STEPS):
        b.perturb(2.0 ** -24, 0.0, 2.0 ** -24, seed=k + 1)
        a.step(1)
        b.step(1)
        c.step(1)
        c.round_storage("fp32")
        if k + 1 in REPORT:
            out["after"][str(k + 1)] = {"perturbation": _diff(a, b), "rounding": _diff(a, c)}
            print(k + 1, out["after"][str(k + 1)], flush=True)
    (Path(__file__).parent / "lens_sensitivity.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
