"""Nernst-Planck ion transport (Eq. 52) on the GPU through the C ABI against the
FP64 oracle on the same seeded inputs: FP64 <= 1e-12 relative L-infinity per field,
FP32 <= 1e-5, FP16-stored populations <= 1e-3 (the ion populations themselves are
held in the compute precision).  Plus the full-size channel in the bench's launch
configuration, checked by properties that hold at any size."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ["n1", "n2", "q", "psi", "ex", "ey", "ux", "uy", "p", "phinow1", "phinow2", "phinow3"]


def _lb():
    import paper_2608_05787_b300 as L
    return L


def rel_linf(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 1e-300 else np.abs(a - b).max()


def _errors(sim, orc, fields=FIELDS):
    return {f: rel_linf(sim.field(f), orc.field(f)) for f in fields}


def _ragged_case(bc_y, precision=0):
    """53 x 37 lattice (ragged against the 32 x 8 tiles), a two-phase drop with
    unequal permittivities, electrodes (bc_y = 2) or plain walls, an axial field,
    an initial flow, and ion concentrations 1 and 1/2 (valences 1 and -2) +- 20%
    (seeded).  Without electrodes a net charge leaves the potential undetermined, so
    those cases run a fixed number of potential iterations."""
    nx, ny = 53, 37
    rng = np.random.default_rng(11)
    p = W.params(nx=nx, ny=ny, bc_y=bc_y, electric=1, precision=precision, eps=(1.0, 3.0, 2.0),
                 sigma=(0.0, 0.0, 0.0), eps_ref=3.0, V_bottom=0.02, V_top=-0.01, E_ext=(2e-3, 0.0),
                 poisson_tol=1e-10, poisson_check_every=3, poisson_fixed_iter=0 if bc_y == 2 else 30, ions=1, ion_D=(0.05, 0.12), ion_z=(1.0, -2.0),
                 ion_beta=4.0, ion_charge=1e-3, inner_phase=3, matrix_phase=1)
    phi = W.compound_droplet(nx, ny, 0.0, 10.0, 4.0, xc=25.3, yc=17.6)
    phi[1] += phi[2]
    phi[2] = 0.0
    u = rng.uniform(-1e-4, 1e-4, size=(2, ny, nx))
    ions = W.ion_concentrations(nx, ny, 1.0, 0.2, seed=5)
    ions[1] *= 0.5
    return p, phi, u, ions


def _pair(p, phi, u, ions, steps):
    L = _lb()
    sim = L.Sim(p, phi, u=u, ions=ions)
    orc = oracle.Oracle(p, phi, u=u, ions=ions)
    sim.step(steps)
    orc.step(steps)
    return sim, orc


@pytest.mark.parametrize("bc_y", [0, 1, 2])
def test_fp64_ions_match_oracle(bc_y):
    p, phi, u, ions = _ragged_case(bc_y)
    sim, orc = _pair(p, phi, u, ions, 20)
    errs = _errors(sim, orc)
    assert all(v <= 1e-12 for v in errs.values()), errs
    for set_name in ("n1", "n2"):          # the ion population sets
        for j in range(9):
            assert rel_linf(sim.pop(set_name, j), orc.pop(set_name, j)) <= 1e-12, (set_name, j)
    assert sim.observables()["poisson_iters"] == orc.observables()["poisson_iters"]


@pytest.mark.parametrize("precision,tol", [(1, 1e-5), (2, 1e-3)])
def test_reduced_precision_ions_match_oracle(precision, tol):
    p, phi, u, ions = _ragged_case(2, precision)
    sim, orc = _pair(p, phi, u, ions, 20)
    errs = _errors(sim, orc, ["n1", "n2", "q", "psi", "ex", "ey", "phinow1", "phinow2"])
    assert all(v <= tol for v in errs.values()), errs


def test_fp64_passive_drift_periodic():
    """Periodic box, no potential solve, passive ions (no charge): the ions drift
    at u + z beta D E; GPU and oracle agree step for step."""
    n = 48
    p = W.params(nx=n, ny=n, bc_y=0, electric=0, sigma=(0, 0, 0), E_ext=(0.05, -0.02), ions=1,
                 ion_D=(0.05, 0.1), ion_beta=2.0, ion_charge=0.0)
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    blob = np.exp(-((x - 20.0) ** 2 + (y - 27.0) ** 2) / 18.0)
    u = np.zeros((2, n, n))
    u[0] = 0.01
    sim, orc = _pair(p, W.single_phase(n, n, 1), u, np.stack([blob, 2 * blob]), 60)
    for f in ("n1", "n2"):
        assert rel_linf(sim.field(f), orc.field(f)) <= 1e-12, f


def test_multigrid_potential_with_ions():
    """The finite-difference (multigrid) potential with the charge the ions carry,
    against the oracle's direct solve of the same equations (both to 1e-12)."""
    cfg = W.config_eof_channel(nx=64, ny=40, kappa_h=5.0, precision=0, poisson_tol=1e-12, poisson_max_iter=200)
    p = cfg["params"]
    sim, orc = _pair(p, cfg["phi"], None, cfg["ions"], 40)
    errs = _errors(sim, orc, ["n1", "n2", "q", "psi", "ux", "uy"])
    assert all(v <= 1e-9 for v in errs.values()), errs


def test_ion_snapshot_roundtrip():
    """save_state / load_state carry the ion populations and their history."""
    p, phi, u, ions = _ragged_case(2)
    L = _lb()
    a = L.Sim(p, phi, u=u, ions=ions).step(5)
    snap = a.save_state()
    a.step(7)
    b = L.Sim(p, phi, u=u, ions=ions)
    b.load_state(snap)
    b.step(7)
    for f in ("n1", "n2", "ux", "psi"):
        assert np.array_equal(a.field(f), b.field(f)), f


def test_set_ions_refused_after_a_step_and_without_ions():
    L = _lb()
    p, phi, u, ions = _ragged_case(2)
    s = L.Sim(p, phi, u=u).step(1)
    assert L.lib().lb3e_set_ions(s._h, ions.ctypes.data) == -1
    with pytest.raises(L.LB3EError):
        L.Sim(dict(p, ions=0), phi, ions=ions)


def test_full_size_channel_properties():
    """The 10240 x 2048 channel in the bench's configuration (FP32, multigrid
    potential): no non-finite value, each species conserved to FP32 rounding, the
    flow symmetric about the mid-plane and, inside the double layers where the
    Coulomb force acts (the bulk has not moved yet), against E as Eq. 53 has it for
    positive zeta and E."""
    cfg = W.config_eof_channel()
    L = _lb()
    s = L.Sim(cfg["params"], cfg["phi"], ions=cfg["ions"])
    m0 = [s.field(k).sum() for k in ("n1", "n2")]
    s.step(20)
    o = s.observables()
    assert o["nonfinite"] == 0
    for k, a in zip(("n1", "n2"), m0):
        b = s.field(k).sum()
        assert abs(b - a) <= 1e-5 * a, (k, a, b)
    ux = s.field("ux")
    assert np.all(np.isfinite(ux))
    prof = ux.mean(axis=1)
    assert np.abs(prof - prof[::-1]).max() <= 1e-3 * np.abs(prof).max()
    assert prof[5:50].mean() < 0 and prof[-50:-5].mean() < 0
