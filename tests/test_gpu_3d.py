"""The three-dimensional (D3Q15) step on the GPU through the C ABI against the FP64
D3Q15 oracle on the same seeded inputs: FP64 <= 1e-12 relative L-infinity per
field, FP32 <= 1e-5; and the 256^3 compound drop in the bench's launch
configuration, checked by properties that hold at any size."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ["phi1", "phi2", "phi3", "ux", "uy", "uz", "p", "q", "psi", "ex", "ey", "ez", "mu1", "mu2", "mu3",
          "phinow1", "phinow2", "phinow3", "qtilde"]


def _lb():
    import paper_2608_05787_b300 as L
    return L


def rel_linf(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 1e-300 else np.abs(a - b).max()


def _case(bc, precision=0, shape=(37, 11, 10)):
    """37 x 11 x 10 cells (ragged against the 32 x 8 tiles), a compound sphere,
    unequal densities and viscosities, permittivity and conductivity contrasts, an
    external field, moving walls and electrodes (bc >= 1), an initial flow and
    charge (seeded).  Without electrodes the net charge leaves the potential
    undetermined, so those cases run a fixed number of potential iterations."""
    nx, ny, nz = shape
    rng = np.random.default_rng(17)
    p = W.params(nx=nx, ny=ny, bc_y=bc, electric=1, precision=precision, rho=(1.0, 1.3, 0.8),
                 visc=(0.1, 0.05, 0.2), gamma12=1e-3, gamma13=8e-4, gamma23=6e-4, eps=(1.0, 3.0, 2.0),
                 sigma=(0.5, 0.1, 1.0), eps_ref=3.0, V_bottom=0.02, V_top=-0.01, E_ext=(1e-3, 5e-4),
                 u_wall_bottom=-2e-4 if bc else 0.0, u_wall_top=3e-4 if bc else 0.0, poisson_tol=1e-10,
                 poisson_check_every=3, poisson_fixed_iter=0 if bc == 2 else 30, inner_phase=3, matrix_phase=1)
    p["nz"] = nz
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float), np.arange(nx, dtype=float),
                          indexing="ij")
    r = np.sqrt((x - 17.3) ** 2 + (y - 5.2) ** 2 + (z - 4.6) ** 2)
    core = 0.5 - 0.5 * np.tanh(2 * (r - 2.0) / 4.0)
    drop = 0.5 - 0.5 * np.tanh(2 * (r - 4.5) / 4.0)
    phi = np.stack([1 - drop, drop - core, core])
    u = rng.uniform(-1e-4, 1e-4, size=(3, nz, ny, nx))
    q = rng.uniform(-1e-4, 1e-4, size=(nz, ny, nx))
    return p, phi, u, q


def _pair(p, phi, u, q, steps):
    L = _lb()
    sim = L.Sim(p, phi, u=u, q=q)
    orc = oracle.Oracle3D(p, phi, u=u, q=q)
    sim.step(steps)
    orc.step(steps)
    return sim, orc


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_fp64_3d_matches_oracle(bc):
    p, phi, u, q = _case(bc)
    sim, orc = _pair(p, phi, u, q, 12)
    errs = {f: rel_linf(sim.field(f), orc.field(f)) for f in FIELDS}
    assert all(v <= 1e-12 for v in errs.values()), errs
    for set_name in ("g", "f1", "f3", "l", "h"):
        for j in (0, 1, 6, 7, 14):
            assert rel_linf(sim.pop(set_name, j), orc.pop(set_name, j)) <= 1e-12, (set_name, j)
    a, b = sim.observables(), orc.observables()
    assert a["poisson_iters"] == b["poisson_iters"]
    for k in ("mass1", "mass2", "mass3", "D_inner", "D_outer", "max_sum_dev"):
        assert abs(a[k] - b[k]) <= 1e-12 * max(1.0, abs(b[k])), (k, a[k], b[k])


def test_fp32_3d_matches_oracle():
    p, phi, u, q = _case(2, precision=1)
    sim, orc = _pair(p, phi, u, q, 12)
    errs = {f: rel_linf(sim.field(f), orc.field(f)) for f in ("phinow1", "phinow2", "phinow3", "psi", "ex", "ez", "q")}
    assert all(v <= 1e-5 for v in errs.values()), errs


@pytest.mark.parametrize("bc", [0, 2])
def test_fp32_3d_staged_potential(bc):
    """The potential iteration with its inputs staged by TMA (FP32, nx a multiple of
    4) on 40 x 12 x 20 cells, ragged against the 32 x 8 tiles and the 16-plane walks:
    bitwise the states of the per-thread loads (fixed iterations all staged; with the
    residual test the checking and saving iterations take the per-thread kernel), and
    the oracle's fields to 1e-5."""
    L = _lb()
    p, phi, u, q = _case(bc, precision=1, shape=(40, 12, 20))
    a = L.Sim(p, phi, u=u, q=q)
    b = L.Sim(p, phi, u=u, q=q).set_staging(0)
    c = L.Sim(p, phi, u=u, q=q).set_staging(7)   # walks of 7, 7 and 6 planes
    for s in (a, b, c):
        s.step(12)
    for f in FIELDS:
        assert np.array_equal(a.field(f), b.field(f)), f
        assert np.array_equal(c.field(f), b.field(f)), f
    assert a.observables()["poisson_iters"] == b.observables()["poisson_iters"]
    orc = oracle.Oracle3D(p, phi, u=u, q=q)
    orc.step(12)
    errs = {f: rel_linf(a.field(f), orc.field(f)) for f in ("phinow1", "phinow2", "phinow3", "psi", "ex", "ez", "q")}
    assert all(v <= 1e-5 for v in errs.values()), errs


def test_3d_rejects_unsupported_options():
    L = _lb()
    p, phi, u, q = _case(2)
    for bad in (dict(precision=2), dict(potential_solver=1), dict(ions=1, ion_D=(0.1, 0.1))):
        with pytest.raises(L.LB3EError):
            L.workspace_bytes(dict(p, **bad))
    s = L.Sim(p, phi)
    with pytest.raises(L.LB3EError):
        s.save_state()
    with pytest.raises(L.LB3EError):
        s.set_staging(-1)
    with pytest.raises(L.LB3EError):
        L.Sim(p, phi, noise=np.zeros((5, 15, 10, 11, 37)))


def test_full_size_3d_drop_properties():
    """The 256^3 compound drop under field (FP32, 16 warm-started potential
    iterations a step, as the bench runs it): finite, each phase conserved to FP32
    rounding, and symmetric under exchanging x and y (the drop is centred and the
    field is along z)."""
    cfg = W.config_deformation_3d()
    L = _lb()
    s = L.Sim(cfg["params"], cfg["phi"])
    o0 = s.observables()
    s.step(5)
    o1 = s.observables()
    assert o1["nonfinite"] == 0
    for k in ("mass1", "mass2", "mass3"):
        assert abs(o1[k] - o0[k]) <= 1e-5 * abs(o0[k]), k
    for f in ("phinow1", "phinow3", "psi"):
        a = s.field(f)
        assert np.abs(a - a.transpose(0, 2, 1)).max() <= 1e-5 * np.abs(a).max(), f
