"""lb3e_observables_noalloc, the entry point for callers that cannot allocate.

Callers running under a memory pool that must not grow, inside an allocator owned
by another framework, or in a monitoring hook cannot call cudaMalloc when they want
these numbers.  lb3e_observables_noalloc takes their FP64 device fields and keeps its
reduction scratch in a fixed array inside the library.  Through the C ABI, it must
agree with the handle-based lb3e_observables on the same fields, call after call
(the shared array keeps the previous call's contents: a small lattice after a larger
one must not see the larger call's block sums).  This file is collected last.
"""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu

KEYS_REL = ("mass1", "mass2", "mass3", "charge", "F_phi", "F_E", "F_u", "F_q", "max_sum_dev")


def _device(sim, names):
    import torch
    return torch.stack([torch.from_numpy(sim.field(n)) for n in names]).cuda().contiguous()


def _compare(L, p, sim):
    import torch
    ref = sim.observables()
    phi = _device(sim, ["phi1", "phi2", "phi3"])
    q = torch.from_numpy(sim.field("q")).cuda().contiguous()
    E = _device(sim, ["ex", "ey"])
    u = _device(sim, ["ux", "uy"])
    got = L.observables_noalloc(p, phi, q, E, u)
    for k in KEYS_REL:
        assert abs(got[k] - ref[k]) <= 1e-11 * max(abs(ref[k]), 1e-30), (k, got[k], ref[k])
    for k in ("D_inner", "D_outer"):
        assert abs(got[k] - ref[k]) <= 1e-12, (k, got[k], ref[k])
    assert got["nonfinite"] == ref["nonfinite"] == 0


def test_noalloc_matches_observables_on_consecutive_calls():
    import paper_2608_05787_b300 as L
    import workloads as W

    cfg = W.config_static_compound(precision=0, n=48)
    p = dict(cfg["params"], poisson_fixed_iter=20)
    sim = L.Sim(p, cfg["phi"], noise=cfg["noise"])
    for _ in range(2):
        sim.step(7)
        _compare(L, p, sim)


@pytest.mark.parametrize("bc_y", [0, 1, 2])
def test_noalloc_small_lattice_after_a_larger_one(bc_y):
    """A 256^2 lattice (32 observables blocks) then a 48^2 one (2 blocks), each against
    lb3e_observables; the second call's reduction must read only its own blocks."""
    import paper_2608_05787_b300 as L
    import workloads as W

    for n in (256, 48):
        cfg = W.config_static_compound(precision=0, n=n)
        p = dict(cfg["params"], bc_y=bc_y, electric=1 if bc_y == 2 else 0, poisson_fixed_iter=8,
                 V_top=0.01 if bc_y == 2 else 0.0)
        sim = L.Sim(p, cfg["phi"], noise=cfg["noise"])
        sim.step(5)
        _compare(L, p, sim)


def test_noalloc_rejects_lattices_beyond_its_scratch_and_bad_fields():
    import torch

    import paper_2608_05787_b300 as L
    import workloads as W

    p = L.Params.from_dict(W.params(nx=4096, ny=4096))
    out = L.Observables()
    dummy = C.c_void_p(256)  # never dereferenced: the size check comes first
    rc = L.lib().lb3e_observables_noalloc(C.byref(p), dummy, dummy, dummy, dummy, None, C.byref(out))
    assert rc == -7
    assert "fixed scratch" in L.status_string(rc)
    # parameters lb3e_init rejects are rejected before any launch
    bad = L.Params.from_dict(W.params(nx=64, ny=64, bc_y=3))
    rc = L.lib().lb3e_observables_noalloc(C.byref(bad), dummy, dummy, dummy, dummy, None, C.byref(out))
    assert rc == -1
    # the binding checks the field shapes against nx, ny before the call
    f = lambda *s: torch.zeros(*s, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        L.observables_noalloc(W.params(nx=64, ny=64), f(3, 64, 64), f(64, 64), f(2, 64, 64), f(2, 32, 64))
