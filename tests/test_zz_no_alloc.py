"""lb3e_observables_noalloc, the entry point for callers that cannot allocate.

Callers running under a memory pool that must not grow, inside an allocator owned
by another framework, or in a monitoring hook cannot call cudaMalloc when they want
these numbers.  lb3e_observables_noalloc takes their FP64 device fields and keeps its
reduction scratch in a fixed array inside the library.  Through the C ABI, it must
agree with the handle-based lb3e_observables on the same fields, call after call
(the shared array keeps the previous call's contents).  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _device(sim, names):
    import torch
    return torch.stack([torch.from_numpy(sim.field(n)) for n in names]).cuda().contiguous()


def test_noalloc_matches_observables_on_consecutive_calls():
    import torch

    import paper_2608_05787_b300 as L
    import workloads as W

    cfg = W.config_static_compound(precision=0, n=48)
    p = dict(cfg["params"], poisson_fixed_iter=20)
    sim = L.Sim(p, cfg["phi"], noise=cfg["noise"])
    for _ in range(2):
        sim.step(7)
        ref = sim.observables()
        phi = _device(sim, ["phi1", "phi2", "phi3"])
        q = torch.from_numpy(sim.field("q")).cuda().contiguous()
        E = _device(sim, ["ex", "ey"])
        u = _device(sim, ["ux", "uy"])
        got = L.observables_noalloc(p, phi, q, E, u)
        for k in ("mass1", "mass2", "mass3", "charge", "F_phi", "F_E", "F_u", "F_q", "max_sum_dev"):
            assert abs(got[k] - ref[k]) <= 1e-11 * max(abs(ref[k]), 1e-30), (k, got[k], ref[k])
        for k in ("D_inner", "D_outer"):
            assert abs(got[k] - ref[k]) <= 1e-12, (k, got[k], ref[k])
        assert got["nonfinite"] == ref["nonfinite"] == 0


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import paper_2608_05787_b300 as L
    import workloads as W

    p = L.Params.from_dict(W.params(nx=4096, ny=4096))
    out = L.Observables()
    dummy = C.c_void_p(256)  # never dereferenced: the size check comes first
    rc = L.lib().lb3e_observables_noalloc(C.byref(p), dummy, dummy, dummy, dummy, None, C.byref(out))
    assert rc == -7
    assert "fixed scratch" in L.status_string(rc)
