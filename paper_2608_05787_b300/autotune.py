"""Autotuner for batched runs: the launch shapes of the two dominant kernels.

* The temporal blocking depth of the potential solve.  A batch iterates the
  potential a fixed number of times per step; the iterations can run one per
  launch (each streams the 9 h planes through HBM) or several per launch on a tile
  held on chip (fewer HBM passes, more redundant halo work and synchronisation).
* The tile of the fused collide/stream pass: 32 x 4, 32 x 8 or 32 x 16 cells a block
  (the last only in FP32 compute).  Taller tiles re-read less of the phi/E halo and
  take more shared memory a block (fewer blocks per SM); shorter ones give more
  blocks on the many small tiles of a batch of small lattices.

The best pair depends on the lattice sizes, the iteration count and the precision,
so it is measured: a probe batch with one instance of each distinct size is timed
for every pair, and the fastest is cached in a JSON file keyed by (precision,
sizes, iterations).  The choice changes launches, not results (the per-cell
arithmetic is the same for every shape).
"""
from __future__ import annotations

import hashlib
import json
import os
from pathlib import Path

CHUNKS = (1, 2, 4, 8)
TILES = (4, 8, 16)


def cache_path() -> Path:
    return Path(os.environ.get("LB3E_AUTOTUNE_CACHE", Path(__file__).resolve().parent / "autotune_cache.json"))


def _key(params_list) -> str:
    sizes = sorted({(int(p["nx"]), int(p["ny"])) for p in params_list})
    iters = sorted({int(p["poisson_fixed_iter"]) for p in params_list if p["electric"]})
    prec = int(params_list[0]["precision"])
    raw = json.dumps(["chunk+tile", prec, sizes, iters])
    return hashlib.sha1(raw.encode()).hexdigest()[:16]


def tune_batch(params_list, chunks=CHUNKS, tiles=TILES, steps: int = 6, use_cache: bool = True) -> dict:
    """{"chunk": potential iterations per launch, "tile": fused tile rows} that
    minimise the time per cell-step of a probe batch."""
    import torch

    from . import Batch
    import workloads as W

    key = _key(params_list)
    path = cache_path()
    cache = json.loads(path.read_text()) if path.exists() else {}
    if use_cache and key in cache:
        return {"chunk": int(cache[key]["chunk"]), "tile": int(cache[key]["tile"])}
    if int(params_list[0]["precision"]) == 0:
        tiles = tuple(t for t in tiles if t != 16)   # FP64 tiles of 16 rows exceed the shared-memory limit
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
    b = Batch(probe, phis)
    times = {}
    for k in chunks:
        for t in tiles:
            b.set_chunk(k).set_tile(t)
            b.run(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            b.run(steps)
            e1.record(b.stream)
            torch.cuda.synchronize()
            times[f"{k},{t}"] = e0.elapsed_time(e1) / (steps * cells)
    b.close()
    best = min(times, key=times.get)
    k, t = (int(v) for v in best.split(","))
    cache[key] = {"chunk": k, "tile": t, "ms_per_cell_step": times}
    try:
        path.write_text(json.dumps(cache, indent=1))
    except OSError:
        pass
    return {"chunk": k, "tile": t}
