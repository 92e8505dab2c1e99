"""Batched stepping (many lattices of uneven sizes in one set of launches, pairs
of steps replayed as a CUDA graph) against single-lattice runs and the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _instances(precision, iters=6):
    specs = [(48, 40, 1.0, 2.0), (64, 64, 4.0, 0.5), (37, 29, 0.7, 1.3), (32, 24, 2.0, 2.0)]
    out = []
    for k, (nx, ny, s_ratio, r_ratio) in enumerate(specs):
        r_out = 0.25 * min(nx, ny)
        p = W.params(nx=nx, ny=ny, bc_y=2, electric=1, precision=precision, eps=(1.0, (s_ratio) ** 0.5, s_ratio),
                     sigma=(1.0, r_ratio ** 0.5, r_ratio), eps_ref=max(1.0, s_ratio), V_top=0.02 * (k + 1),
                     poisson_fixed_iter=iters)
        out.append((p, W.compound_droplet(nx, ny, 0.5 * r_out, r_out, 4.0)))
    return out


@pytest.mark.parametrize("precision,tol", [(0, 0.0), (1, 1e-5), (2, 1e-4)])
def test_batch_equals_single_lattice_runs(precision, tol):
    """Every instance of a batch matches the lattice stepped alone over 9 steps
    (plain, graph pairs, plain): bitwise in FP64 (no contraction), to 1e-5 in FP32
    (the batched and single kernels are compiled separately and may fuse different
    multiply-adds), to 1e-4 with FP16 storage (an ulp of FP32 may flip an FP16
    rounding)."""
    import paper_2608_05787_b300 as L
    import torch
    inst = _instances(precision)
    b = L.Batch([p for p, _ in inst], [phi for _, phi in inst], stream=torch.cuda.Stream())
    b.run(4)
    b.run(5)
    obs = b.observables()
    for i, (p, phi) in enumerate(inst):
        s = L.Sim(p, phi)
        s.step(4)
        s.step(5)
        for f in ("phinow1", "phinow2", "phinow3", "psi", "ex", "ey", "ux", "p", "q"):
            a, r = b.field(i, f), s.field(f)
            assert np.abs(a - r).max() <= tol * np.abs(r).max(), (i, f, np.abs(a - r).max())
        so = s.observables()
        assert abs(obs[i]["D_outer"] - so["D_outer"]) <= max(tol, 1e-12) and obs[i]["step"] == 9


def test_batch_fp64_matches_oracle():
    import paper_2608_05787_b300 as L
    inst = _instances(0, iters=5)
    b = L.Batch([p for p, _ in inst], [phi for _, phi in inst])
    b.run(12)
    for i in (0, 2):
        p, phi = inst[i]
        o = oracle.Oracle(p, phi)
        o.step(12)
        for f in ("phinow1", "phinow2", "phinow3", "psi", "ex", "ey", "q", "ux"):
            ref = o.field(f)
            err = np.abs(b.field(i, f) - ref).max() / max(np.abs(ref).max(), 1e-300)
            assert err <= 1e-12, (i, f, err)


@pytest.mark.parametrize("chunk", [2, 3, 4, 5, 8])
def test_blocked_potential_chunks_give_the_same_state(chunk):
    """Temporal blocking depth changes the launches, not the result: FP64 batches
    with 1 and `chunk` iterations per launch agree bitwise."""
    import paper_2608_05787_b300 as L
    inst = _instances(0, iters=7)
    a = L.Batch([p for p, _ in inst], [phi for _, phi in inst])
    b = L.Batch([p for p, _ in inst], [phi for _, phi in inst]).set_chunk(chunk)
    a.run(6)
    b.run(6)
    for i in range(len(inst)):
        for f in ("phinow1", "phinow3", "psi", "ex", "ux"):
            assert np.array_equal(a.field(i, f), b.field(i, f)), (chunk, i, f)


def test_autotuner_picks_a_candidate_and_caches(tmp_path, monkeypatch):
    from paper_2608_05787_b300 import autotune
    monkeypatch.setenv("LB3E_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    inst = _instances(1, iters=8)
    t = autotune.tune_batch([p for p, _ in inst], steps=2)
    assert t["chunk"] in autotune.CHUNKS and t["tile"] in autotune.TILES
    assert autotune.tune_batch([p for p, _ in inst]) == t     # served from the cache
    assert (tmp_path / "tune.json").exists()


@pytest.mark.parametrize("precision,rows,tol", [(0, 4, 0.0), (1, 4, 1e-5), (1, 16, 1e-5), (2, 16, 1e-4),
                                               (5, 4, 1e-4)])
def test_fused_tile_shapes_give_the_same_state(precision, rows, tol):
    """The fused pass over tiles of 32 x 4 or 32 x 16 cells against the default 32 x 8:
    bitwise in FP64 (no contraction; the per-cell arithmetic does not depend on the
    tile), within the batch-vs-single bounds otherwise (each instantiation may fuse
    different multiply-adds)."""
    import paper_2608_05787_b300 as L
    inst = _instances(precision, iters=5)
    a = L.Batch([p for p, _ in inst], [phi for _, phi in inst])
    b = L.Batch([p for p, _ in inst], [phi for _, phi in inst]).set_tile(rows)
    a.run(6)
    b.run(6)
    for i in range(len(inst)):
        for f in ("phinow1", "phinow3", "psi", "ex", "ux", "p", "q"):
            x, r = b.field(i, f), a.field(i, f)
            assert np.abs(x - r).max() <= tol * np.abs(r).max(), (rows, i, f, np.abs(x - r).max())


def test_fused_tile_of_16_rows_is_refused_in_fp64():
    import paper_2608_05787_b300 as L
    inst = _instances(0, iters=5)
    b = L.Batch([p for p, _ in inst], [phi for _, phi in inst])
    with pytest.raises(L.LB3EError):
        b.set_tile(16)


def test_batch_rejects_mixed_iteration_counts():
    import paper_2608_05787_b300 as L
    inst = _instances(1)
    inst[1][0]["poisson_fixed_iter"] = 7
    with pytest.raises(L.LB3EError):
        L.Batch([p for p, _ in inst], [phi for _, phi in inst])


@pytest.mark.slow
def test_sweep_instances_at_full_size_match_the_oracle():
    """Eight seeded instances of the 256-instance sweep at their stated sizes (the
    first instance of each side 128, 192, 256, 384, 512 and the next three), stepped
    together as one FP64 batch for 50 steps with the sweep's 16 warm-started
    potential iterations a step, against the oracle run on each: every field to
    1e-12 and the deformation factors to 1e-12."""
    import paper_2608_05787_b300 as L
    insts = W.config_batched_sweep(precision=0)
    picks = []
    for side in (128, 192, 256, 384, 512):
        picks.append(next(i for i, s in enumerate(insts) if s["shape"][0] == side))
    picks += [i for i in range(len(insts)) if i not in picks][:3]
    assert len(picks) == 8 and {insts[i]["shape"][0] for i in picks} == {128, 192, 256, 384, 512}
    b = L.Batch([insts[i]["params"] for i in picks], [W.sweep_phi(insts[i]) for i in picks]).set_chunk(4)
    b.run(50)
    obs = b.observables()
    for k, i in enumerate(picks):
        o = oracle.Oracle(insts[i]["params"], W.sweep_phi(insts[i]))
        o.step(50)
        for f in ("phi1", "phi2", "phi3", "phinow1", "phinow3", "psi", "ex", "ey", "q", "ux", "uy", "p"):
            ref = o.field(f)
            err = np.abs(b.field(k, f) - ref).max() / max(np.abs(ref).max(), 1e-300)
            assert err <= 1e-12, (i, insts[i]["shape"], f, err)
        oo = o.observables()
        for key in ("D_inner", "D_outer"):
            assert abs(obs[k][key] - oo[key]) <= 1e-12, (i, key, obs[k][key], oo[key])
