"""Writes precision_sensitivity.json: what the FP64 oracle's own fields do under the
rounding that each reduced-precision build adds, on the stated 64 x 64 static
compound drop (2000 steps, seeded noise 1e-8, electrodes, the potential iterated a
fixed 40 times a step so that every run does the same work).  For each field:
max |modified - plain oracle| / max |plain oracle| after the last step.  Two models:

* "rounding": every step, the stored populations are rounded to the storage format
  exactly as the GPU stores them (oracle.Oracle.round_storage: round to nearest
  even; FP16 with its subnormal range; the phase rest populations by their
  deviation from phi_i, phi_i itself an FP32 field); arithmetic stays FP64.  For the
  FP16- and BF16-stored builds the storage rounding dominates, and this reproduces
  their measured errors on every field within a factor 1.3.
* "perturbation": every step, every stored population (and the FP32 anchor phi_i)
  is perturbed by u * (unit roundoff) * |v|, u uniform in [-1, 1) from a seeded hash
  (oracle.Oracle.perturb).  For the FP32 build the rounding of its arithmetic (every
  intermediate of the step, not only the stored values) dominates; this random
  model stands for it, and the FP32 errors on every field are 0.4-0.8 of it.

The numbers say how much the scheme itself amplifies rounding of each size: the
velocity of this near-static drop is a small residual of balanced forces, so it
moves most (u_x by 2e-3 of its maximum under FP32-sized, 0.4 under FP16-sized
rounding).  Only the oracle runs here.
Usage: python tests/golden/make_precision_sensitivity.py
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

FIELDS = ("phi1", "phi2", "phi3", "phinow1", "phinow2", "phinow3", "qtilde", "ux", "uy", "p", "q", "psi",
          "ex", "ey", "mu1", "mu2", "mu3")
# unit roundoff of each format (half the spacing at 1) and, for FP16, the spacing of
# its subnormals (its normal range ends at 6.1e-5, inside the range of the flow and
# charge populations)
UNIT = {"fp32": (2.0 ** -24, 0.0), "fp16": (2.0 ** -12, 2.0 ** -25), "bf16": (2.0 ** -9, 0.0)}
FIELD_REL = 2.0 ** -24   # the FP32 fields (phi among them) of every reduced build
STEPS = 2000


def _pair():
    cfg = W.config_static_compound(precision=0)
    p = dict(cfg["params"], poisson_fixed_iter=40)
    return (oracle.Oracle(p, cfg["phi"], noise=cfg["noise"]), oracle.Oracle(p, cfg["phi"], noise=cfg["noise"]))


def _diff(a, b) -> dict:
    return {f: float(np.abs(a.field(f) - b.field(f)).max() / np.abs(a.field(f)).max()) for f in FIELDS}


def rounding(fmt: str) -> dict:
    a, b = _pair()
    b.round_storage(fmt)
    for _ in range(STEPS):
        a.step(1)
        b.step(1)
        b.round_storage(fmt)
    return _diff(a, b)


def perturbation(fmt: str) -> dict:
    rel, floor_abs = UNIT[fmt]
    a, b = _pair()
    for k in range(STEPS):
        b.perturb(rel, floor_abs, FIELD_REL, seed=k + 1)
        a.step(1)
        b.step(1)
    return _diff(a, b)


def main():
    out = {"workload": "static compound drop 64x64, 2000 steps, 40 potential iterations a step", "formats": {}}
    for fmt in UNIT:
        out["formats"][fmt] = {"rounding": rounding(fmt), "perturbation": perturbation(fmt)}
        print(fmt, out["formats"][fmt], flush=True)
    (Path(__file__).parent / "precision_sensitivity.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
