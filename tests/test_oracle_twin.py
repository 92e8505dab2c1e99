"""Transcription check of the C oracle: an independent vectorised NumPy
implementation of the same step (tests/numpy_twin.py, written from the equations
and readings, not from the C code's structure) against the oracle on 8 x 8
lattices, all population sets and fields, after initialisation and after 5 steps.
Every term is active: unequal densities and viscosities (local tau_g), distinct
tensions, conductivities and permittivities, charge convection, moving walls,
electrodes and an external field, noise on the populations.  The two differ only
by rounding order: <= 1e-13 of each field's magnitude."""
import numpy as np
import pytest

import oracle
import workloads as W
from numpy_twin import Twin  # tests/ is on sys.path (pytest rootdir conftest)

SETS = ("g", "f1", "f2", "f3", "l", "h")
FIELDS = ("phi1", "phi2", "phi3", "ux", "uy", "p", "q", "psi", "ex", "ey", "mu1", "mu2", "mu3")


def _case(bc_y):
    n = 8
    p = W.params(nx=n, ny=n, bc_y=bc_y, electric=1, rho=(1.0, 1.3, 0.8), visc=(0.1, 0.15, 0.12),
                 gamma12=1e-3, gamma13=1.4e-3, gamma23=0.8e-3, width_D=2.0, tau_f=0.9,
                 eps=(1.0, 2.5, 4.0), sigma=(0.3, 0.2, 0.1), eps_ref=4.0, alpha=0.15,
                 V_bottom=0.01 if bc_y == 2 else 0.0, V_top=0.03 if bc_y == 2 else 0.0, E_ext=(1e-3, 2e-3),
                 u_wall_bottom=-1e-3 if bc_y else 0.0, u_wall_top=2e-3 if bc_y else 0.0,
                 charge_convection=1, poisson_fixed_iter=7)
    phi = W.compound_droplet(n, n, 1.5, 3.0, 2.0, xc=3.7, yc=4.2)
    rng = np.random.default_rng(7)
    u = 1e-3 * rng.standard_normal((2, n, n))
    q = 1e-3 * rng.standard_normal((n, n))
    noise = W.noise(n, n, 1e-3, seed=11)
    return p, phi, u, q, noise


def _compare(o, t, tol=1e-13):
    pops = {"g": t.g, "f1": t.f[0], "f2": t.f[1], "f3": t.f[2], "l": t.l, "h": t.h}
    for name in SETS:
        ref = np.array([o.pop(name, j) for j in range(9)])
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(pops[name] - ref).max() <= tol * scale, (name, np.abs(pops[name] - ref).max(), scale)


@pytest.mark.parametrize("bc_y", [0, 1, 2])
def test_oracle_and_numpy_twin_agree(bc_y):
    p, phi, u, q, noise = _case(bc_y)
    o = oracle.Oracle(p, phi, u=u, q=q, noise=noise)
    t = Twin(p, phi, u=u, q=q, noise=noise)
    _compare(o, t)
    o.step(5)
    t.step(5)
    _compare(o, t)
    fields = {"phi1": t.phi[0], "phi2": t.phi[1], "phi3": t.phi[2], "ux": t.u[0], "uy": t.u[1], "p": t.pr,
              "q": t.q, "psi": t.psi, "ex": t.E[0], "ey": t.E[1], "mu1": t.mu[0], "mu2": t.mu[1], "mu3": t.mu[2]}
    for f in FIELDS:
        ref = o.field(f)
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(fields[f] - ref).max() <= 1e-13 * scale, (f, np.abs(fields[f] - ref).max(), scale)


OBS = ("mass1", "mass2", "mass3", "charge", "F_phi", "F_E", "F_u", "F_q", "max_sum_dev", "D_inner", "D_outer")


@pytest.mark.parametrize("bc_y", [0, 1, 2])
def test_oracle_and_numpy_twin_observables_agree(bc_y):
    """The reductions of the oracle (masses, charge, the Eq. 18 energy parts, the sum
    deviation, the deformation factors) against the twin's own, after init and after
    5 steps of the all-terms case on a 16 x 12 lattice (off-centre compound drop)."""
    p, _, _, _, _ = _case(bc_y)
    nx, ny = 16, 12
    p = dict(p, nx=nx, ny=ny)
    phi = W.compound_droplet(nx, ny, 2.5, 4.5, 2.0, xc=7.3, yc=5.6)
    rng = np.random.default_rng(9)
    u = 1e-3 * rng.standard_normal((2, ny, nx))
    q = 1e-3 * rng.standard_normal((ny, nx))
    o = oracle.Oracle(p, phi, u=u, q=q)
    t = Twin(p, phi, u=u, q=q)
    for n in (0, 5):
        if n:
            o.step(n)
            t.step(n)
        ref, got = o.observables(), t.observables()
        for k in OBS:
            # D is a small difference of two radii: compared on its own O(1) scale
            scale = 1.0 if k.startswith("D_") else max(abs(ref[k]), 1e-300)
            assert abs(got[k] - ref[k]) <= 1e-12 * scale, (n, k, got[k], ref[k])
        assert got["D_inner"] != 0.0 and got["F_E"] > 0 and got["F_q"] > 0


@pytest.mark.parametrize("bc_y", [0, 2])
def test_oracle_and_numpy_twin_agree_with_ion_transport(bc_y):
    """The same check with the Nernst-Planck species on (valences +1 and -2, unequal
    D, concentrations 1 and 1/2 +- 20%): ion populations and every field."""
    p, phi, u, q, noise = _case(bc_y)
    p = dict(p, ions=1, ion_D=(0.05, 0.12), ion_z=(1.0, -2.0), ion_beta=4.0, ion_charge=1e-3)
    n = W.ion_concentrations(8, 8, 1.0, 0.2, seed=5)
    n[1] *= 0.5
    o = oracle.Oracle(p, phi, u=u, q=q, noise=noise, ions=n)
    t = Twin(p, phi, u=u, q=q, noise=noise, ions=n)
    for step in (0, 5):
        if step:
            o.step(step)
            t.step(step)
        for k, name in enumerate(("n1", "n2")):
            ref = np.array([o.pop(name, j) for j in range(9)])
            assert np.abs(t.ion[k] - ref).max() <= 1e-13 * np.abs(ref).max(), (step, name)
        _compare(o, t)
    fields = {"q": t.q, "psi": t.psi, "ex": t.E[0], "ey": t.E[1], "ux": t.u[0], "uy": t.u[1]}
    for f, a in fields.items():
        ref = o.field(f)
        assert np.abs(a - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300), f
