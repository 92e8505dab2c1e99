"""The 4096 x 4096 compound-drop workload at its full size, in the launch
configuration the bench times (FP32, potential blocked 4 iterations per launch).

The FP64 oracle cannot step a lattice this size in reasonable time, and its potential
solve couples the whole lattice, so no window of it can be computed alone.  These
checks use properties that hold at any size instead:

* no non-finite value;
* per-phase mass conserved (the LB phase update conserves Σ_x φ_i up to FP32 rounding);
* the drop is centred, so every step keeps the x-mirror symmetry φ(x) = φ(nx − x),
  u_x(x) = −u_x(nx − x), up to the rounding of sums taken in mirrored order;
* the blocked potential kernel matches the one-iteration-per-launch kernel at this
  size (the per-cell arithmetic is the same; FP32 rounding of a per-cell constant
  differs).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N = 4096
STEPS = 3


def _config():
    cfg = W.config_deformation(n=N, r_out=600.0, r_in=300.0, precision=1)
    # the bench runs the solve to its tolerance (20000 iterations a step); a fixed
    # count keeps this check short and both runs below doing the same work
    return dict(cfg["params"], poisson_fixed_iter=16), cfg["phi"]


def _mirror_x(a):
    return np.roll(a[:, ::-1], 1, axis=1)  # a[y, (nx - x) mod nx]


@pytest.fixture(scope="module")
def runs():
    import paper_2608_05787_b300 as L
    p, phi = _config()
    out = {}
    for chunk in (4, 1):
        s = L.Sim(p, phi).set_chunk(chunk)
        o0 = s.observables()
        s.step(STEPS)
        out[chunk] = dict(o0=o0, o1=s.observables(),
                          f={f: s.field(f) for f in ("phinow1", "phinow2", "phinow3", "psi", "ux", "uy", "q")})
        s.close()
    return out


def test_full_size_finite_and_mass_conserved(runs):
    r = runs[4]
    assert r["o1"]["nonfinite"] == 0 and r["o1"]["step"] == STEPS
    for k in ("mass1", "mass2", "mass3"):
        m0, m1 = r["o0"][k], r["o1"][k]
        assert abs(m1 - m0) <= 1e-6 * abs(m0), (k, m0, m1)


def test_full_size_mirror_symmetry(runs):
    """Bounds relative to each field's maximum: 1e-5 for phases and potential; the
    charge and velocity are formed from differences of larger terms (interface
    jumps of eps and sigma; balanced capillary, Coulomb and pressure forces), so
    rounding in mirrored summation order shows more there (measured 2.4e-5 for q).
    An indexing mistake would break the symmetry at order one."""
    f = runs[4]["f"]
    for name, tol in (("phinow1", 1e-5), ("phinow2", 1e-5), ("phinow3", 1e-5), ("psi", 1e-5), ("q", 1e-4),
                      ("uy", 1e-3)):
        a = f[name]
        assert np.abs(a - _mirror_x(a)).max() <= tol * np.abs(a).max(), name
    ux = f["ux"]
    assert np.abs(ux + _mirror_x(ux)).max() <= 1e-3 * np.abs(f["uy"]).max()


def test_full_size_blocked_potential_matches_per_iteration(runs):
    a, b = runs[4]["f"], runs[1]["f"]
    for name in ("phinow1", "phinow3", "psi", "q"):
        assert np.abs(a[name] - b[name]).max() <= 1e-6 * np.abs(b[name]).max(), name
