"""Pins of the oracle's Nernst-Planck ion transport (Eq. 52, the electro-osmotic
validation of Section 5.1) against closed forms: drift and diffusion of passive
ions, the Boltzmann distribution of ions in equilibrium with their own potential,
and the electro-osmotic channel of Eq. 53.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _ion_params(**kw):
    base = dict(sigma=(0.0, 0.0, 0.0), eps=(1.0, 1.0, 1.0), eps_ref=1.0, ions=1)
    base.update(kw)
    return W.params(**base)


def test_passive_ions_drift_at_u_plus_z_beta_D_E_and_spread_at_2D():
    """Eq. 52 for a constant velocity u and field E: n_i is advected at the drift
    velocity v_i = u + z_i beta D_i E and diffuses with D_i, so a Gaussian's
    centroid moves at v_i and its variance grows by 2 D_i t along and across the
    drift.  Passive ions (zero charge per concentration) keep the flow uniform.
    The two species have opposite valences and different D, so a sign slip in z,
    a missing D in the migration term or a wrong relaxation time each fail."""
    n, D, u0, E, beta, s0 = 96, 0.05, 0.02, 0.2, 2.0, 4.0
    p = _ion_params(nx=n, ny=n, bc_y=0, electric=0, E_ext=(E, 0.0), ion_D=(D, 2 * D), ion_z=(1.0, -1.0),
                    ion_beta=beta, ion_charge=0.0)
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    blob = np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (2 * s0 * s0))
    u = np.zeros((2, n, n))
    u[0] = u0
    o = oracle.Oracle(p, W.single_phase(n, n, 1), u=u, ions=np.stack([blob, blob]))

    def moments(f):
        ang = 2 * np.pi * x / n
        cx = (math.atan2((f * np.sin(ang)).sum(), (f * np.cos(ang)).sum()) % (2 * np.pi)) * n / (2 * np.pi)
        dx = (x - cx + n / 2) % n - n / 2
        dy = y - n / 2
        return cx, (f * dx * dx).sum() / f.sum(), (f * dy * dy).sum() / f.sum()

    T = 200
    o.step(20)
    m0 = [moments(o.field(k)) for k in ("n1", "n2")]
    o.step(T)
    for i, key in enumerate(("n1", "n2")):
        f = o.field(key)
        c1, vx1, vy1 = moments(f)
        c0, vx0, vy0 = m0[i]
        z, Di = p["ion_z"][i], p["ion_D"][i]
        v = u0 + z * beta * Di * E
        assert abs(f.sum() - blob.sum()) < 1e-11 * blob.sum()
        assert abs(((c1 - c0 + n / 2) % n - n / 2) - v * T) < 1e-2       # circular-mean centroid
        assert abs((vx1 - vx0) / (2 * T) - Di) < 1e-6 * Di
        assert abs((vy1 - vy0) / (2 * T) - Di) < 1e-6 * Di
    assert np.abs(o.field("ux") - u0).max() < 1e-15


def _boltzmann_run(ny):
    """Ions between electrodes at +-V, started uniform: at rest the flux vanishes,
    so n_i exp(z_i beta psi) is uniform.  kappa ny = 4 at every resolution."""
    nx, beta, D, V = 2, 20.0, 0.3, 0.05
    kappa = 4.0 / ny
    p = _ion_params(nx=nx, ny=ny, bc_y=2, electric=1, V_bottom=V, V_top=-V, ion_D=(D, D), ion_z=(1.0, -1.0),
                    ion_beta=beta, ion_charge=kappa * kappa / (2 * beta), potential_solver=1)
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1), ions=np.ones((2, ny, nx)))
    o.step(int(6 * ny * ny / D))
    psi = o.field("psi")
    n1, n2 = o.field("n1"), o.field("n2")
    dev = max(float(np.ptp(np.log(n) + z * beta * psi)) for n, z in ((n1, 1.0), (n2, -1.0)))
    return dev, n1, n2


def test_ions_relax_to_the_boltzmann_distribution_at_second_order():
    """Zero-flux equilibrium of Eq. 52 with the potential they carry (the nonlinear
    Poisson-Boltzmann state; beta V = 1, ion concentrations vary 0.35 to 2.3):
    ln n_i + z_i beta psi is constant.  The lattice reaches it to O(dx^2): the
    spread of ln n_i + z_i beta psi falls by ~4 when the resolution doubles
    (measured 0.031 and 0.0085).  The walls conserve each species, and the
    antisymmetric electrodes make n_2 the mirror image of n_1."""
    d16, _, _ = _boltzmann_run(16)
    d32, n1, n2 = _boltzmann_run(32)
    assert d32 < 1.2e-2
    assert 3.4 < d16 / d32 < 4.4
    assert abs(n1.sum() - n1.size) < 1e-11 * n1.size and abs(n2.sum() - n2.size) < 1e-11 * n2.size
    assert np.abs(n2 - n1[::-1]).max() < 1e-12
    assert n1[0, 0] < 1.0 < n1[-1, 0]          # cations leave the positive electrode


def test_nernst_planck_electro_osmotic_channel_matches_eq53():
    """The channel of Section 5.1 with both ion species transported (Eq. 52): walls at
    the zeta potential with beta zeta << 1 (Debye-Hueckel regime), the bulk at
    concentration n0 and the double layers at their Boltzmann profile from the
    start, a uniform axial field E.  Eq. 53 fixes psi(y) = zeta cosh(kappa y) /
    cosh(kappa h) with kappa^2 = e_q beta sum_i z_i^2 n0 / eps, and the flow
    u(y) = -(eps zeta E / mu)(1 - cosh(kappa y)/cosh(kappa h)).  The ions stay in
    their double layers while the charge they carry drives the flow; errors are
    O((kappa dx)^2) (measured 0.47% for psi, 0.14% for u).  The wall-normal force
    q E_y leaves the scheme's staggered momentum oscillation in u_y (1.2e-5 of u)."""
    nx, ny = 2, 50
    h = ny / 2
    kappa, zeta, E, beta, D = 5.0 / h, 1e-3, 1e-3, 1.0, 0.1
    tau_g = 0.5 + math.sqrt(3.0 / 16.0)
    mu = (tau_g - 0.5) / 3.0
    p = _ion_params(nx=nx, ny=ny, bc_y=2, electric=1, V_bottom=zeta, V_top=zeta, E_ext=(E, 0.0), tau_g=tau_g,
                    ion_D=(D, D), ion_z=(1.0, -1.0), ion_beta=beta, ion_charge=kappa * kappa / (2 * beta),
                    potential_solver=1)
    yc = np.arange(ny) + 0.5 - h
    prof = np.cosh(kappa * yc) / np.cosh(kappa * h)
    n_init = np.stack([np.repeat(np.exp(-z * beta * zeta * prof)[:, None], nx, axis=1) for z in (1.0, -1.0)])
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1), ions=n_init)
    o.step(22000)
    psi = o.field("psi")[:, 0]
    ux = o.field("ux")[:, 0]
    u_ref = -(zeta * E / mu) * (1.0 - prof)
    assert np.abs(psi - zeta * prof).max() <= 1e-2 * zeta
    assert np.abs(ux - u_ref).max() <= 1e-2 * np.abs(u_ref).max()
    assert np.abs(o.field("uy")).max() <= 1e-4 * np.abs(u_ref).max()


@pytest.mark.parametrize("bad", [dict(ion_D=(0.0, 0.1)), dict(ion_D=(0.1, -1.0)), dict(debye_kappa2=0.01),
                                 dict(ions=2)])
def test_ion_parameters_are_validated(bad):
    p = _ion_params(nx=8, ny=8, **bad)
    with pytest.raises(ValueError):
        oracle.Oracle(p, W.single_phase(8, 8, 1))


def test_ion_concentrations_need_ion_transport():
    p = W.params(nx=8, ny=8)
    with pytest.raises(ValueError):
        oracle.Oracle(p, W.single_phase(8, 8, 1), ions=np.ones((2, 8, 8)))
