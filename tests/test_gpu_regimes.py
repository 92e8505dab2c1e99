"""Second workload: two compound drops under a field, and a compound drop in a
confined shear flow under a field, run through the batched path.

Parity: FP64 batches of small instances of both set-ups (electrodes, moving walls,
the paper's property ratios) against the oracle.  Outcomes: the paper gives no
numbers for these studies, so the checks are the qualitative ones it states.
* Drop pairs: with S23 > R23 the pair drains the matrix film and merges, shells
  first and cores after; with R23 > S23 the pair is pushed apart and stays two drops.
* Confined shear: the steady deformation grows with Ca_E and with confinement W_c.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2608_05787_b300 import regimes as G

pytestmark = pytest.mark.gpu


def _small_instances():
    out = []
    for regime in ("coalescence", "separation"):
        c = W.config_two_drops(regime, n=64, r_in=5.0, r_out=10.0, gap=6.0, iters=6, precision=0)
        out.append((c["params"], c["phi"]))
    s = W.config_shear_regimes(ca_e=(1.0,), wc=(0.75,), r_in=6.0, r_out=12.0, nx=64, iters=6, precision=0)[0]
    out.append((s["params"], s["phi"]))
    return out


def test_fp64_batch_matches_oracle_on_the_second_workload():
    import paper_2608_05787_b300 as L
    inst = _small_instances()
    b = L.Batch([p for p, _ in inst], [phi for _, phi in inst])
    b.run(30)
    for i, (p, phi) in enumerate(inst):
        o = oracle.Oracle(p, phi)
        o.step(30)
        for f in ("phinow1", "phinow2", "phinow3", "psi", "ux", "uy", "q"):
            ref = o.field(f)
            err = np.abs(b.field(i, f) - ref).max() / max(np.abs(ref).max(), 1e-300)
            assert err <= 1e-12, (i, f, err)


def test_drop_pairs_coalesce_or_separate():
    import paper_2608_05787_b300 as L
    cfgs = [W.config_two_drops(r) for r in ("coalescence", "separation")]
    b = L.Batch([c["params"] for c in cfgs], [c["phi"] for c in cfgs]).set_chunk(4)
    d0 = [G.pair_measures(c["phi"][0])["distance"] for c in cfgs]
    b.run(50000)
    mid = [G.pair_measures(b.field(i, "phinow1")) for i in range(2)]
    b.run(150000)
    shells = [G.count_drops(b.field(i, "phinow1")) for i in range(2)]
    cores = [G.count_drops(1.0 - b.field(i, "phinow3")) for i in range(2)]
    end = [G.pair_measures(b.field(i, "phinow1")) for i in range(2)]
    # attraction: the pair approaches, its shells and then its cores merge
    assert mid[0]["distance"] < d0[0] - 1.0
    assert shells[0] == 1 and cores[0] == 1 and end[0]["film"] < 0.05
    # repulsion: pushed apart, a matrix film remains, still two drops
    assert mid[1]["distance"] > d0[1] + 1.0
    assert shells[1] == 2 and end[1]["film"] > 0.8


def test_confined_shear_deformation_grows_with_field_and_confinement():
    import paper_2608_05787_b300 as L
    ca_e, wc = (0.2, 0.6, 1.0), (0.3, 0.5, 0.75)
    inst = W.config_shear_regimes(ca_e=ca_e, wc=wc)
    b = L.Batch([c["params"] for c in inst], [c["phi"] for c in inst]).set_chunk(4)
    b.run(50000)
    D = {(c["wc"], c["ca_e"]): G.shape_measures(b.field(i, "phinow1"))["D"] for i, c in enumerate(inst)}
    for w in wc:
        assert D[(w, 0.2)] < D[(w, 0.6)] < D[(w, 1.0)], w
    for c in ca_e:
        assert D[(0.3, c)] < D[(0.5, c)] < D[(0.75, c)], c
    assert all(G.count_drops(b.field(i, "phinow1")) == 1 for i in range(len(inst)))
