"""Autotuner for batched runs: the temporal blocking depth of the potential solve.

A batch iterates the potential a fixed number of times per step.  Those
iterations can run one per launch (each streams the 9 h planes through HBM) or
several per launch on a tile held in shared memory (fewer HBM passes, more
redundant halo work and synchronisation).  The best depth depends on the lattice
sizes, the iteration count and the precision, so it is measured: a probe batch
with one instance of each distinct size is timed for each candidate depth, and
the fastest is cached in a JSON file keyed by (precision, sizes, iterations).
"""
from __future__ import annotations

import hashlib
import json
import os
from pathlib import Path

CANDIDATES = (1, 2, 4, 8)


def cache_path() -> Path:
    return Path(os.environ.get("LB3E_AUTOTUNE_CACHE", Path(__file__).resolve().parent / "autotune_cache.json"))


def _key(params_list) -> str:
    sizes = sorted({(int(p["nx"]), int(p["ny"])) for p in params_list})
    iters = sorted({int(p["poisson_fixed_iter"]) for p in params_list if p["electric"]})
    prec = int(params_list[0]["precision"])
    raw = json.dumps([prec, sizes, iters])
    return hashlib.sha1(raw.encode()).hexdigest()[:16]


def tune_batch_chunk(params_list, candidates=CANDIDATES, steps: int = 6, use_cache: bool = True) -> int:
    """Potential iterations per launch that minimise the time per cell-step."""
    import torch

    from . import Batch
    import workloads as W

    key = _key(params_list)
    path = cache_path()
    cache = json.loads(path.read_text()) if path.exists() else {}
    if use_cache and key in cache:
        return int(cache[key]["chunk"])
    # one probe instance per distinct size (the first instance seen of that size)
    probe, seen = [], set()
    for p in params_list:
        sz = (int(p["nx"]), int(p["ny"]))
        if sz not in seen:
            seen.add(sz)
            probe.append(p)
    phis = [W.compound_droplet(int(p["nx"]), int(p["ny"]), 0.125 * min(p["nx"], p["ny"]),
                               0.25 * min(p["nx"], p["ny"]), 4.0) for p in probe]
    cells = sum(int(p["nx"]) * int(p["ny"]) for p in probe)
    times = {}
    for k in candidates:
        b = Batch(probe, phis).set_chunk(k)
        b.run(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.run(steps)
        e1.record(b.stream)
        torch.cuda.synchronize()
        times[k] = e0.elapsed_time(e1) / (steps * cells)
        b.close()
    best = min(times, key=times.get)
    cache[key] = {"chunk": best, "ms_per_cell_step": times}
    try:
        path.write_text(json.dumps(cache, indent=1))
    except OSError:
        pass
    return best
