"""Parameter sweeps: many compound-drop lattices, sharded over ranks.

Instances are independent, so a sweep shards without any data exchange: each rank
steps its share as one lb3e batch (one launch per kernel over the tiles of all its
instances, pairs of steps replayed as a CUDA graph), and only the per-instance
results (deformation factors) are gathered at the end.  Shares are balanced by
cell count: largest instance first, to the least-loaded rank.
"""
from __future__ import annotations

from typing import Callable, Sequence


def shard(cells: Sequence[int], world: int) -> list[list[int]]:
    """Greedy longest-first assignment of instances (by cell count) to ranks.
    Returns, per rank, the instance indices in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(cells)), key=lambda k: (-cells[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += cells[i]
    return [sorted(p) for p in parts]


def run_shard(instances: Sequence[dict], indices: Sequence[int], steps: int,
              run: Callable[[list, int], list] | None = None) -> dict[int, dict]:
    """Step this rank's instances; returns {instance index: observables}.
    ``run(list_of_instances, steps)`` defaults to one lb3e batch on the GPU."""
    mine = [instances[i] for i in indices]
    if not mine:
        return {}
    if run is None:
        run = _run_batch
    obs = run(mine, steps)
    return {i: o for i, o in zip(indices, obs)}


def _run_batch(mine: list, steps: int) -> list:
    from . import Batch
    from .autotune import tune_batch
    params = [m["params"] for m in mine]
    tuned = tune_batch(params)
    b = Batch(params, [m["phi"] for m in mine]).set_chunk(tuned["chunk"]).set_tile(tuned["tile"])
    b.run(steps)
    return b.observables()


def sweep(instances: Sequence[dict], steps: int, run=None, group=None) -> list[dict]:
    """Run all instances over the ranks of ``group`` (torch.distributed, any
    backend) or locally when it is not initialised; every rank gets the full,
    ordered list of observables."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    else:
        world, rank = 1, 0
    cells = [int(m["params"]["nx"]) * int(m["params"]["ny"]) for m in instances]
    parts = shard(cells, world)
    local = run_shard(instances, parts[rank], steps, run)
    if world == 1:
        merged = local
    else:
        gathered: list = [None] * world
        dist.all_gather_object(gathered, local, group=group)
        merged = {}
        for g in gathered:
            merged.update(g)
    return [merged[i] for i in range(len(instances))]
