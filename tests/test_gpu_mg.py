"""Multigrid solve of the finite-difference potential (the alternative to the
LB pseudo-time solve) against the oracle's conjugate-gradient solve of the same
FD system, and a full step with it.

Both solve A psi = b to a relative residual (oracle 1e-13, GPU 1e-12 here); the
fields then agree to the solve tolerance times the conditioning, asserted at 1e-9.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _params(n=64, **kw):
    E0 = W.field_for_capillary(0.5, 1e-3, 1.0, 16.0)
    return W.params(nx=n, ny=n, bc_y=2, electric=1, eps=(1.0, 2.0, 4.0), sigma=(1.0, 0.5, 0.25), eps_ref=4.0,
                    V_top=E0 * n, potential_solver=1, poisson_tol=1e-12, poisson_max_iter=200, **kw)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n", [64, 96])
def test_mg_initial_potential_matches_oracle_cg(n):
    import paper_2608_05787_b300 as L
    p = _params(n, precision=0)
    phi = W.compound_droplet(n, n, n / 8, n / 4, 4.0)
    rng = np.random.default_rng(n)
    q = rng.uniform(-1e-4, 1e-4, size=(n, n))
    sim = L.Sim(p, phi, q=q)
    orc = oracle.Oracle(p, phi, q=q)
    for f in ("psi", "ex", "ey"):
        assert _rel(sim.field(f), orc.field(f)) <= 1e-9, f
    it = sim.observables()["poisson_iters"]
    assert 1 <= it <= 25          # multigrid: a handful of V-cycles to 1e-12
    print("V-cycles to 1e-12:", it)


def test_mg_full_step_parity_fp64():
    import paper_2608_05787_b300 as L
    p = _params(64, precision=0)
    phi = W.compound_droplet(64, 64, 8.0, 16.0, 4.0)
    sim = L.Sim(p, phi)
    orc = oracle.Oracle(p, phi)
    sim.step(20)
    orc.step(20)
    for f in ("phinow1", "phinow2", "phinow3", "ux", "uy", "p", "q", "psi", "ex", "ey", "mu1"):
        assert _rel(sim.field(f), orc.field(f)) <= 1e-9, f


def test_mg_fp32_step_close_to_oracle():
    import paper_2608_05787_b300 as L
    p = _params(64, precision=1, )
    p["poisson_tol"] = 1e-10
    phi = W.compound_droplet(64, 64, 8.0, 16.0, 4.0)
    sim = L.Sim(p, phi)
    orc = oracle.Oracle(dict(p, precision=0), phi)
    sim.step(50)
    orc.step(50)
    for f in ("phinow1", "phinow2", "phinow3", "psi", "ex", "ey"):
        assert _rel(sim.field(f), orc.field(f)) <= 1e-5, f


def test_mg_rejects_unsupported_setups():
    import paper_2608_05787_b300 as L
    with pytest.raises(L.LB3EError):
        L.workspace_bytes(dict(_params(64, precision=0), bc_y=1))
    with pytest.raises(L.LB3EError):
        L.workspace_bytes(dict(_params(64, precision=0), nx=63))
