"""Sharding of a parameter sweep over ranks (host logic, CPU, gloo)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2608_05787_b300.sweep import shard, sweep


def test_shard_covers_every_instance_once_and_balances():
    cells = [128 ** 2, 512 ** 2, 192 ** 2, 384 ** 2, 256 ** 2] * 20
    for world in (1, 2, 3, 8):
        parts = shard(cells, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(cells)   # greedy longest-first bound


def test_shard_is_deterministic():
    cells = [3, 1, 4, 1, 5, 9, 2, 6]
    assert shard(cells, 3) == shard(list(cells), 3)
    assert shard(cells, 1) == [list(range(8))]


def _fake_run(instances, steps):
    # stands in for the GPU batch: a deterministic function of the instance
    return [{"D_outer": inst["params"]["nx"] * 1e-3 + steps, "id": inst["id"]} for inst in instances]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = [{"params": {"nx": n, "ny": n}, "id": k} for k, n in enumerate([128, 512, 192, 384, 256, 128, 512])]
    out = sweep(inst, 10, run=_fake_run)
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_rank_gloo_sweep_gathers_in_instance_order():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1]
    assert [r["id"] for r in res[0]] == list(range(7))
    assert res[0][1]["D_outer"] == pytest.approx(512e-3 + 10)
