"""Writes lens_sensitivity.json: how far the FP64 oracle's own phase fields move under
rounding of the FP32 size on the stated spreading lens (512 x 256, walls, no field,
tensions 1e-3 / 8e-4 / 6e-4, 20 000 steps).

Two oracle runs from the same state; before every step the second has every stored
population (and the FP32 anchor phi_i) perturbed by u * 2^-24 * |v|, u uniform in
[-1, 1) from a seeded hash (oracle.Oracle.perturb), the model of the FP32 build's
rounding that the static-compound gates use.  For each of phinow1..3:
max |perturbed - plain| / max |plain| after the last step.  The lens is still
spreading at 20 000 steps (its contact lines move), so rounding of this size shifts
the interfaces by a small fraction of a lattice spacing, and the relative field
difference is that shift times the interface gradient.  Only the oracle runs here
(about an hour on 8 cores).
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


def main():
    cfg = W.config_lens(tensions=TENSIONS, precision=0)
    a = oracle.Oracle(cfg["params"], cfg["phi"])
    b = oracle.Oracle(cfg["params"], cfg["phi"])
    out = {"workload": "spreading lens 512x256, walls, no field, tensions %s" % (TENSIONS,),
           "model": "every stored value perturbed at the FP32 unit roundoff before every step", "after": {}}
    for k in range(STEPS):
        b.perturb(2.0 ** -24, 0.0, 2.0 ** -24, seed=k + 1)
        a.step(1)
        b.step(1)
        if k + 1 in REPORT:
            d = {f: float(np.abs(a.field(f) - b.field(f)).max() / np.abs(a.field(f)).max()) for f in FIELDS}
            out["after"][str(k + 1)] = d
            print(k + 1, d, flush=True)
    (Path(__file__).parent / "lens_sensitivity.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
