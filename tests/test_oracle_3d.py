"""Pins of the three-dimensional (D3Q15, Eq. 32) oracle: lattice identities, the
Eq. 33 stencils on polynomials, closed forms (linear potential, layered
dielectric, bounce-back Poiseuille flow with walls normal to z), reductions to the
independently pinned two-dimensional oracle (fields invariant along one axis:
D3Q15 projected on a plane has exactly the D2Q9 weights), and exact symmetries.
CPU only."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

CS2 = 1.0 / 3.0


def params3(nz, **kw):
    p = W.params(**kw)
    p["nz"] = nz
    return p


def test_d3q15_lattice_identities():
    """Eq. 32: weights sum to 1, odd moments vanish, second moments cs2 delta, fourth
    moments cs2^2 (delta delta + delta delta + delta delta); opposite directions."""
    cx, cy, cz, w, opp = oracle.lattice3()
    c = np.stack([cx, cy, cz], axis=1).astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs((w[:, None] * c).sum(0)).max() < 1e-15
    assert np.allclose(np.einsum("j,ja,jb->ab", w, c, c), CS2 * np.eye(3), atol=1e-15)
    d = np.eye(3)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("j,ja,jb,jc,jd->abcd", w, c, c, c, c), iso4, atol=1e-15)
    assert np.all(c[opp] == -c)
    assert abs(w[0] - 2 / 9) < 1e-16 and np.allclose(w[1:7], 1 / 9) and np.allclose(w[7:], 1 / 72)


def test_d3q15_stencils_exact_on_polynomials_and_mirror_ghosts():
    """Eq. 33: the gradient is exact on quadratics and the Laplacian on cubics (at
    cells whose stencil does not wrap); with walls the ghost planes mirror the
    field, so a field even about the wall plane has zero normal gradient there."""
    n = 9
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float),) * 3, indexing="ij")
    quad = 0.3 * x * x - 0.2 * y * z + 0.1 * z * z + 0.5 * x - y
    g, _ = oracle.stencil3(quad, 0)
    cubic = x ** 3 - 2 * x * y * z + 0.5 * y * y * z + z ** 3
    _, lap = oracle.stencil3(cubic, 0)
    s = (slice(1, -1),) * 3
    assert np.allclose(g[0][s], (0.6 * x + 0.5)[s], atol=1e-12)
    assert np.allclose(g[1][s], (-0.2 * z - 1)[s], atol=1e-12)
    assert np.allclose(g[2][s], (-0.2 * y + 0.2 * z)[s], atol=1e-12)
    assert np.allclose(lap[s], (6 * x + 7 * z)[s], atol=1e-10)
    ev = np.cos(2 * np.pi * x / n) * (z - (n - 1) / 2) ** 2
    g, _ = oracle.stencil3(ev, 1)
    # the half-way wall mirrors plane 0 onto plane -1: the z-gradient at the walls is
    # the one-sided difference against the mirror, equal in size and opposite in sign
    assert np.allclose(g[2][0], -g[2][-1], atol=1e-12)


def _potential3(nz, eps_lo, eps_hi, q=None, nx=4, ny=4):
    p = params3(nz, nx=nx, ny=ny, bc_y=2, electric=1, eps=(eps_lo, eps_hi, 1.0), sigma=(0, 0, 0),
                eps_ref=max(eps_lo, eps_hi), V_bottom=0.0, V_top=1.0, poisson_tol=1e-13, poisson_max_iter=400000,
                poisson_check_every=10)
    phi = np.zeros((3, nz, ny, nx))
    phi[0, : nz // 2] = 1
    phi[1, nz // 2:] = 1
    return oracle.Oracle3D(p, phi, q=q)


def test_potential_linear_and_layered_dielectric_closed_forms():
    """Eq. 42-45 on D3Q15 with electrodes normal to z: uniform permittivity gives the
    exact linear potential; two layers 1:4 give fields in the ratio 4:1 with the
    series-capacitor drop (closed forms of the discrete problem)."""
    nz = 16
    o = _potential3(nz, 1.0, 1.0)
    z = np.arange(nz) + 0.5
    assert np.abs(o.field("psi")[:, 0, 0] - z / nz).max() < 1e-10
    assert np.abs(o.field("ez") + 1.0 / nz).max() < 1e-10
    o = _potential3(nz, 1.0, 4.0)
    ez = o.field("ez")[:, 0, 0]
    # V = E_lo h + E_hi h with eps_lo E_lo = eps_hi E_hi, h = nz/2
    e_lo = 1.0 / (nz / 2 * (1 + 1 / 4.0))
    assert np.abs(ez[: nz // 2] + e_lo).max() < 1e-9 and np.abs(ez[nz // 2:] + e_lo / 4).max() < 1e-9


def _y_invariant_pair(nx, nz, q2=None, **kw):
    phi2 = W.compound_droplet(nx, nz, 5.0 * nx / 40, 10.0 * nx / 40, 4.0, xc=0.48 * nx, yc=0.49 * nz)
    base = dict(bc_y=2, electric=1, poisson_tol=1e-13, poisson_max_iter=2000000, poisson_check_every=10)
    base.update(kw)
    o2 = oracle.Oracle(W.params(nx=nx, ny=nz, **base), phi2, q=q2)
    o3 = oracle.Oracle3D(params3(nz, nx=nx, ny=2, **base), np.repeat(phi2[:, :, None, :], 2, axis=2),
                         q=None if q2 is None else np.repeat(q2[:, None, :], 2, axis=1))
    return o2, o3


def test_y_invariant_state_reduces_to_the_two_dimensional_oracle():
    """A field invariant along y with walls normal to z is the two-dimensional problem
    in the x-z plane (D3Q15 projected on that plane has the D2Q9 weights).  With a
    compound drop, permittivity contrast 1:3:2, electrodes, an external field and
    moving walls, the initial potential solve and the first step's phases,
    velocity and field agree with the two-dimensional oracle (written separately)
    to rounding; the out-of-plane velocity is zero."""
    o2, o3 = _y_invariant_pair(40, 32, eps=(1.0, 3.0, 2.0), sigma=(0.0, 0.0, 0.0), eps_ref=3.0,
                               V_bottom=0.02, V_top=-0.01, E_ext=(1e-3, 0.0), u_wall_bottom=-2e-4,
                               u_wall_top=3e-4)
    for a, b in (("psi", "psi"), ("ex", "ex"), ("ey", "ez")):
        x2, x3 = o2.field(a), o3.field(b)[:, 0]
        assert np.abs(x2 - x3).max() <= 1e-9 * np.abs(x2).max(), a
    o2.step(1)
    o3.step(1)
    for a, b, tol in (("phinow1", "phinow1", 1e-13), ("phinow3", "phinow3", 1e-13), ("ux", "ux", 1e-11),
                      ("uy", "uz", 1e-11), ("psi", "psi", 1e-9), ("mu2", "mu2", 1e-11)):
        x2, x3 = o2.field(a), o3.field(b)[:, 0]
        assert np.abs(x2 - x3).max() <= tol * np.abs(x2).max(), a
    assert np.abs(o3.field("uy")).max() < 1e-18


def test_charge_source_agrees_with_two_dimensions_at_second_order():
    """The potential's source weights differ between the lattices (1/14 on the 14
    moving D3Q15 directions, two of which project on the D2Q9 rest; 1/8 on the 8
    moving D2Q9 ones): the two discrete solutions of the same Poisson problem differ
    at O(dx^2) -- by ~5x less when the resolution doubles (measured 0.016, 0.0033)."""
    diffs = []
    for s in (1, 2):
        nx, nz = 40 * s, 32 * s
        q2 = 1e-4 / s ** 2 * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :] * np.ones((nz, 1))
        o2, o3 = _y_invariant_pair(nx, nz, q2=q2, eps=(1.0, 1.0, 1.0), sigma=(0, 0, 0), eps_ref=1.0,
                                   V_bottom=0.02, V_top=-0.01)
        lin = 0.02 - 0.03 * (np.arange(nz) + 0.5)[:, None] / nz
        a, b = o2.field("psi"), o3.field("psi")[:, 0]
        diffs.append(np.abs(a - b).max() / np.abs(a - lin).max())
    assert diffs[0] < 0.03
    assert 3.5 < diffs[0] / diffs[1] < 6.0


@pytest.mark.parametrize("tau_g", [0.5 + math.sqrt(3.0 / 16.0), 1.2])
def test_poiseuille_between_walls_normal_to_z(tau_g):
    """Eq. 37-41 on D3Q15 with the Coulomb force qE_x between resting electrodes at
    z = -1/2, nz - 1/2: the bounce-back parabola with its wall slip
    (4/3)((tau - 1/2)^2 - 3/16), as for D2Q9."""
    nx, ny, nz, q0, Ex = 4, 4, 16, 1e-5, 1e-2
    mu = CS2 * (tau_g - 0.5)
    p = params3(nz, nx=nx, ny=ny, bc_y=2, electric=1, eps=(1.0, 1.0, 1.0), sigma=(0, 0, 0), eps_ref=1.0,
                V_bottom=0.0, V_top=0.0, E_ext=(Ex, 0.0), tau_g=tau_g, poisson_tol=1e-13,
                poisson_max_iter=100000, poisson_check_every=10)
    phi = np.zeros((3, nz, ny, nx))
    phi[0] = 1
    o = oracle.Oracle3D(p, phi, q=np.full((nz, ny, nx), q0))
    o.step(3500)
    z = np.arange(nz, dtype=float)
    s = 4.0 / 3.0 * ((tau_g - 0.5) ** 2 - 3.0 / 16.0)
    exact = q0 * Ex / (2 * mu) * ((z + 0.5) * (nz - z - 0.5) + s)
    assert np.abs(o.field("ux") - exact[:, None, None]).max() < 1e-6 * exact.max()
    assert np.abs(o.field("uy")).max() < 1e-15


def test_cylinder_laplace_jump_matches_two_dimensions():
    """A drop invariant along z (a cylinder, periodic) on D3Q15 reaches the same
    equilibrium as the two-dimensional oracle's disc: pressure jump (Eq. 27b through
    Eq. 41) within 1%, phases within 1e-4, out-of-plane velocity zero."""
    L, R = 24, 8.0
    p = W.params(nx=L, ny=L, bc_y=0, electric=0, tau_g=1.0)
    phi2 = W.compound_droplet(L, L, 0.0, R, 4.0)
    phi2[1] += phi2[2]
    phi2[2] = 0.0
    o2 = oracle.Oracle(p, phi2).step(2500)
    o3 = oracle.Oracle3D(dict(p, nz=2), np.repeat(phi2[:, None], 2, axis=1)).step(2500)
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    r = np.hypot(x - L / 2, y - L / 2)
    jump = lambda pr: pr[r < R - 3].mean() - pr[r > R + 4].mean()
    d2, d3 = jump(o2.field("p")), jump(o3.field("p")[0])
    assert abs(d3 / d2 - 1) < 0.01, (d2, d3)
    assert np.abs(o2.field("phinow2") - o3.field("phinow2")[0]).max() < 1e-4
    assert np.abs(o3.field("uz")).max() < 1e-18


def test_sphere_conserves_mass_and_keeps_the_xy_exchange_symmetry():
    """A compound sphere between electrodes (field along z), charge on: each phase's
    mass is conserved to rounding, and since D3Q15 and the set-up are symmetric
    under exchanging x and y, every field is too (to rounding of sums taken in
    another order)."""
    n = 14
    p = params3(n, nx=n, ny=n, bc_y=2, electric=1, V_top=0.05, poisson_tol=1e-11, poisson_check_every=5)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float),) * 3, indexing="ij")
    r = np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2 + (z - n / 2 + 0.3) ** 2)
    core = 0.5 - 0.5 * np.tanh(2 * (r - 2.5) / 4.0)
    drop = 0.5 - 0.5 * np.tanh(2 * (r - 5.0) / 4.0)
    phi = np.stack([1 - drop, drop - core, core])
    o = oracle.Oracle3D(p, phi)
    m0 = o.observables()
    o.step(30)
    m1 = o.observables()
    for k in ("mass1", "mass2", "mass3"):
        assert abs(m1[k] - m0[k]) < 1e-11 * n ** 3
    for f in ("phinow1", "phinow3", "psi", "q", "uz", "p"):
        a = o.field(f)
        assert np.abs(a - a.transpose(0, 2, 1)).max() <= 1e-12 * max(np.abs(a).max(), 1e-300), f
    ux, uy = o.field("ux"), o.field("uy")
    assert np.abs(ux - uy.transpose(0, 2, 1)).max() <= 1e-12 * np.abs(ux).max()
    assert m1["nonfinite"] == 0


def test_couette_between_moving_walls_normal_to_z():
    """Eq. 37-41 on D3Q15 with the walls at z = -1/2, nz - 1/2 sliding along x: the
    steady plane Couette flow u_x = U_b + (U_t - U_b)(z + 1/2)/nz, exact up to the
    O(Ma^2) error of the quadratic equilibrium."""
    nx, ny, nz = 4, 4, 12
    Ub, Ut = -1e-4, 2e-4
    p = params3(nz, nx=nx, ny=ny, bc_y=1, electric=0, u_wall_bottom=Ub, u_wall_top=Ut)
    phi = np.zeros((3, nz, ny, nx))
    phi[0] = 1
    o = oracle.Oracle3D(p, phi).step(6000)
    z = np.arange(nz)
    exact = Ub + (Ut - Ub) * (z + 0.5) / nz
    assert np.abs(o.field("ux") - exact[:, None, None]).max() < 1e-7 * Ut
    assert np.abs(o.field("uz")).max() < 1e-9 * Ut and np.abs(o.field("uy")).max() < 1e-18


def test_charge_transport_with_walls_reduces_exactly_to_two_dimensions():
    """With the flow exactly at rest (one phase, no field: mu = 0 and qE = 0), the
    charge populations (Eq. 46-50) of a y-invariant state between walls normal to z
    evolve as the D2Q9 ones: the D3Q15 equilibrium, source and bounce-back project
    exactly onto the x-z plane.  A charge blob diffusing and relaxing (sigma/eps)
    beside a wall agrees with the two-dimensional oracle to rounding over 200 steps."""
    nx, nz = 24, 16
    base = dict(bc_y=1, electric=0, sigma=(0.02, 0.02, 0.02), eps=(1.0, 1.0, 1.0), alpha=0.1, E_ext=(0.0, 0.0))
    x = np.arange(nx)[None, :]
    z = np.arange(nz)[:, None]
    q2 = 1e-3 * np.exp(-((x - 9.3) ** 2 + (z - 2.2) ** 2) / 8.0)
    phi2 = W.single_phase(nx, nz, 1)
    o2 = oracle.Oracle(W.params(nx=nx, ny=nz, **base), phi2, q=q2).step(200)
    o3 = oracle.Oracle3D(params3(nz, nx=nx, ny=2, **base), np.repeat(phi2[:, :, None, :], 2, axis=2),
                         q=np.repeat(q2[:, None, :], 2, axis=1)).step(200)
    a, b = o2.field("q"), o3.field("q")[:, 0]
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(a).max() < 0.5 * 1e-3          # it did relax
    assert np.abs(o3.field("ux")).max() == 0.0 and np.abs(o3.field("uz")).max() == 0.0
