"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a lattice
identity, a closed-form solution, an exact discrete invariant, or a value the paper
prints.  They are chosen so that a plausible slip anywhere in the oracle (a dropped
term, a flipped sign, a wrong index or coefficient) fails at least one of them; the
docstrings say which part of the scheme each one pins.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

CS2 = 1.0 / 3.0


# --------------------------------------------------------------------------- lattice
def test_d2q9_lattice_identities():
    """Eq. 31: weights sum to 1, first moment vanishes, second moment is cs^2 I,
    fourth moment is isotropic, opposite directions are exact negatives."""
    cx, cy, w, opp = oracle.lattice()
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert abs((w * cx).sum()) < 1e-16 and abs((w * cy).sum()) < 1e-16
    assert np.isclose((w * cx * cx).sum(), CS2, atol=1e-15)
    assert np.isclose((w * cy * cy).sum(), CS2, atol=1e-15)
    assert abs((w * cx * cy).sum()) < 1e-16
    assert np.isclose((w * cx ** 4).sum(), 3 * CS2 ** 2, atol=1e-15)
    assert np.isclose((w * cx ** 2 * cy ** 2).sum(), CS2 ** 2, atol=1e-15)
    assert (cx[opp] == -cx).all() and (cy[opp] == -cy).all()
    assert list(cx) == [0, 1, 0, -1, 0, 1, -1, -1, 1] and list(cy) == [0, 0, 1, 0, -1, 1, 1, -1, -1]


# --------------------------------------------------------------------------- stencils
def test_isotropic_stencils_exact_on_polynomials():
    """Eq. 33: the gradient is exact for quadratics and the Laplacian for cubics
    (interior cells, away from the periodic seam)."""
    ny, nx = 24, 20
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    a = [0.3, -1.1, 0.7, 0.05, -0.02, 0.03, 0.004, -0.003, 0.002, 0.001]
    quad = a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y
    gx, gy, lap = oracle.stencil(quad, bc_y=0)
    sl = (slice(2, -2), slice(2, -2))
    assert np.allclose(gx[sl], (a[1] + 2 * a[3] * x + a[4] * y)[sl], rtol=0, atol=1e-12)
    assert np.allclose(gy[sl], (a[2] + a[4] * x + 2 * a[5] * y)[sl], rtol=0, atol=1e-12)
    cub = quad + a[6] * x ** 3 + a[7] * x * x * y + a[8] * x * y * y + a[9] * y ** 3
    _, _, lap = oracle.stencil(cub, bc_y=0)
    exact = 2 * a[3] + 2 * a[5] + 6 * a[6] * x + 2 * a[7] * y + 2 * a[8] * x + 6 * a[9] * y
    assert np.allclose(lap[sl], exact[sl], rtol=0, atol=1e-11)


def test_wall_ghosts_are_mirror_images():
    """Half-way walls: a field mirrored about y = -1/2 has zero normal gradient
    at the wall, so a field that is even about the wall reproduces the periodic
    stencil of its even extension."""
    ny, nx = 8, 6
    rng = np.random.default_rng(1)
    f = rng.standard_normal((ny, nx))
    ext = np.concatenate([f[::-1], f], axis=0)          # rows -ny..ny-1, mirror about -1/2
    ext = np.concatenate([ext, ext[::-1]], axis=0)      # periodic even extension, period 4 ny
    gx_e, gy_e, lap_e = oracle.stencil(ext, bc_y=0)
    gx, gy, lap = oracle.stencil(f, bc_y=1)
    assert np.allclose(gx, gx_e[ny:2 * ny], atol=1e-14)
    assert np.allclose(gy, gy_e[ny:2 * ny], atol=1e-14)
    assert np.allclose(lap, lap_e[ny:2 * ny], atol=1e-14)


# --------------------------------------------------------------------------- free energy
TENS = {(1, 2): 1e-3, (1, 3): 8e-4, (2, 3): 6e-4}


@pytest.mark.parametrize("pair", list(TENS))
def test_flat_interface_energy_equals_surface_tension(pair):
    """Eq. 7-9, 18: a flat i|j tanh interface of width D stores (lambda_i +
    lambda_j)/2 = gamma_ij per unit length; the discrete value converges to it at
    second order in 1/D.  Distinct tensions make a swapped lambda visible."""
    i, j = pair
    errs = []
    for D in (4.0, 8.0):
        p = W.params(nx=4, ny=96, bc_y=1, electric=0, gamma12=1e-3, gamma13=8e-4, gamma23=6e-4, width_D=D)
        o = oracle.Oracle(p, W.flat_interface(4, 96, D, i, j))
        errs.append(o.observables()["F_phi"] / 4 / TENS[pair] - 1.0)
    assert abs(errs[0]) < 0.035 and abs(errs[1]) < 0.01
    assert 3.0 < errs[0] / errs[1] < 5.0          # second-order convergence


@pytest.mark.parametrize("pair", list(TENS))
def test_chemical_potential_vanishes_on_equilibrium_profile(pair):
    """Eq. 20: for the tanh profile (the 1-D minimiser) the bulk term
    24/D lambda phi(phi-1/2)(phi-1) and -3/4 D lambda lap(phi) cancel; the
    residual is the O(1/D^2) stencil error.  The absent phase has mu = 0."""
    i, j = pair
    lam = {1: 1.2e-3, 2: 8e-4, 3: 4e-4}
    rel = []
    for D in (4.0, 8.0):
        p = W.params(nx=4, ny=96, bc_y=1, electric=0, gamma12=1e-3, gamma13=8e-4, gamma23=6e-4, width_D=D)
        o = oracle.Oracle(p, W.flat_interface(4, 96, D, i, j))
        scale = {k: lam[k] * 24.0 / D * (math.sqrt(3) / 18) for k in (1, 2, 3)}   # max |phi(phi-1/2)(phi-1)|
        r = [np.abs(o.field(f"mu{k}")).max() / scale[k] for k in (1, 2, 3)]
        k_absent = ({1, 2, 3} - {i, j}).pop()
        assert r[k_absent - 1] == 0.0
        rel.append(max(r))
    assert rel[0] < 0.05 and rel[1] < 0.017
    assert rel[0] / rel[1] > 2.5


# --------------------------------------------------------------------------- phase field
def test_reduction_consistency_absent_phase_stays_zero():
    """Eq. 28 + the source of Eq. 36: with phase 3 absent, M_3k = 0 and mu_3 = 0,
    so f^3 stays identically zero, with the field on."""
    n = 32
    p = W.params(nx=n, ny=n, bc_y=2, electric=1, V_top=0.01, poisson_check_every=5)
    phi = W.compound_droplet(n, n, 0.0, 8.0, 4.0)  # r_in = 0: core absent
    phi[1] += phi[2]
    phi[2] = 0.0
    o = oracle.Oracle(p, phi)
    o.step(40)
    assert np.abs(o.field("phinow3")).max() == 0.0
    assert np.abs(o.field("phinow2")).max() > 0.9


def test_wide_interface_relaxes_toward_equilibrium_profile():
    """Eq. 27c-28 through Eq. 34-36: a flat binary interface started twice as wide
    as D relaxes, by mobility-driven diffusion, toward the tanh(2 y/D) profile that
    minimises Eq. 18: the central slope rises monotonically from 1/(2D) toward the
    discrete equilibrium slope and never overshoots it.  With lambda_1 = lambda_2
    the off-diagonal M_12 carries half the flux, so a sign slip in it (the two
    fluxes cancelling) leaves the profile wide."""
    nx, ny, D = 4, 48, 4.0
    p = W.params(nx=nx, ny=ny, bc_y=1, electric=0, gamma12=1e-2, gamma13=1e-2, gamma23=1e-2,
                 width_D=D, tau_f=1.0)
    o = oracle.Oracle(p, W.flat_interface(nx, ny, 2 * D, 1, 2))
    eq = np.diff(W.flat_interface(nx, ny, D, 1, 2)[1][:, 0]).max()
    slopes = []
    for T in (0, 500, 1000, 2000):
        o.step(T - o.steps_done)
        slopes.append(np.diff(o.field("phinow2")[:, 0]).max())
    assert abs(slopes[0] * D - 0.5) < 0.01
    assert all(b > a for a, b in zip(slopes, slopes[1:]))
    assert 0.72 * eq < slopes[-1] < eq


def test_drop_carried_by_uniformly_accelerating_fluid():
    """Coulomb force qE of Eq. 27b and the d/dt(phi u) source of Eq. 36: a uniform
    charge in a uniform field accelerates the whole (equal-density) fluid at
    a = qE/rho, and a drop is carried along: its centroid moves by the time
    integral of u (the trapezoid rule is exact for u linear in t), to 1e-3."""
    n, q0, E, T = 64, 1e-3, 1e-3, 300
    p = W.params(nx=n, ny=n, bc_y=0, electric=0, sigma=(0, 0, 0), E_ext=(E, 0.0), alpha=0.02)
    phi = W.compound_droplet(n, n, 0.0, 10.0, 4.0)
    phi[1] += phi[2]
    phi[2] = 0.0
    o = oracle.Oracle(p, phi, q=np.full((n, n), q0))
    x = np.arange(n, dtype=float)[None, :]
    cen = lambda f: (f * x).sum() / f.sum()
    c0 = cen(o.field("phinow2"))
    us = []
    for _ in range(T):
        o.step(1)
        us.append(o.field("ux").mean())
    assert abs(us[-1] - us[-2] - q0 * E) < 1e-3 * q0 * E          # uniform acceleration a = qE/rho
    us.append(2 * us[-1] - us[-2])
    travel = sum(0.5 * (us[k] + us[k + 1]) for k in range(T))
    assert abs((cen(o.field("phinow2")) - c0) / travel - 1) < 1e-3


@pytest.mark.parametrize("bc_y", [0, 1, 2])
def test_per_phase_mass_conserved_to_roundoff(bc_y):
    """Sum_j F_j^i = 0, sum_j f^eq = phi_i, and bounce-back/periodic streaming move
    populations without loss: every phase's total is conserved to round-off."""
    cfg = W.config_static_compound(n=32)
    p = dict(cfg["params"], bc_y=bc_y, electric=1 if bc_y == 2 else 0)
    o = oracle.Oracle(p, cfg["phi"], noise=W.noise(32, 32, 1e-8))
    o.step(1)
    m0 = o.observables()
    o.step(60)
    m1 = o.observables()
    for k in ("mass1", "mass2", "mass3"):
        assert abs(m1[k] - m0[k]) < 1e-11 * 32 * 32


# --------------------------------------------------------------------------- flow
def test_couette_profile_exact():
    """Eq. 37-41 with moving half-way walls: steady plane Couette flow is linear,
    u(y) = U_b + (U_t - U_b)(y + 1/2)/ny.  The linear scheme reproduces it exactly;
    the only deviation is the O(Ma^2) relative error of the quadratic equilibrium
    (it falls 100x when the wall speeds fall 10x)."""
    nx, ny = 4, 12
    errs = []
    for s in (1.0, 0.1):
        Ub, Ut = -1e-3 * s, 2e-3 * s
        p = W.params(nx=nx, ny=ny, bc_y=1, electric=0, u_wall_bottom=Ub, u_wall_top=Ut)
        o = oracle.Oracle(p, W.single_phase(nx, ny, 1))
        o.step(6000)
        u = o.field("ux")[:, 0]
        y = np.arange(ny)
        exact = Ub + (Ut - Ub) * (y + 0.5) / ny
        errs.append(np.abs(u - exact).max() / Ut)
        assert np.abs(o.field("uy")).max() < 1e-8 * Ut
    assert errs[0] < 1e-6
    assert 90 < errs[0] / errs[1] < 110


@pytest.mark.parametrize("tau_g", [0.5 + math.sqrt(3.0 / 16.0), 1.2])
def test_poiseuille_profile_matches_bounce_back_closed_form(tau_g):
    """Eq. 37-41 driven by the Coulomb force qE of Eq. 27b between resting half-way
    walls (electrodes at zero potential, sigma = 0 so q stays uniform): the steady
    flow is the parabola u(y) = F/(2 mu) [(y + 1/2)(ny - y - 1/2) + s] with F = q E_x.
    For BGK with half-way bounce-back and a second-order force term the discrete
    solution is known in closed form (He, Zou, Luo & Dembo 1997; Ginzburg &
    d'Humieres 2003): the wall slip is s = (4/3)((tau - 1/2)^2 - 3/16), which vanishes
    at tau = 1/2 + sqrt(3/16).  A missing half-force in u, a wrong force weight or
    a wall off by half a cell each change s or the amplitude at order one.
    E_y from the charge's own potential gives a wall-normal force F_y = (q^2/eps)
    (y - (ny-1)/2), balanced by the pressure; it perturbs u_x at order q^2, kept below
    the checked bound by q << E_x.  It also drives the scheme's staggered momentum
    invariant: streaming and half-way bounce-back carry (-1)^(y+t) c_y f unchanged and
    collision conserves momentum, so sum_y (-1)^(y+t) j_y moves only by the force's
    alternating row sum each step.  With u = (j + F/2)/rho that leaves the two-cell
    oscillation u_y = +-q^2/(4 eps), flipping sign every step, independent of tau."""
    nx, ny, q0, Ex = 4, 16, 1e-5, 1e-2
    mu = CS2 * (tau_g - 0.5)
    p = W.params(nx=nx, ny=ny, bc_y=2, electric=1, eps=(1.0, 1.0, 1.0), sigma=(0.0, 0.0, 0.0), eps_ref=1.0,
                 V_bottom=0.0, V_top=0.0, E_ext=(Ex, 0.0), tau_g=tau_g, poisson_tol=1e-13,
                 poisson_max_iter=100000, poisson_check_every=10)
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1), q=np.full((ny, nx), q0))
    o.step(3500)
    y = np.arange(ny, dtype=float)
    s = 4.0 / 3.0 * ((tau_g - 0.5) ** 2 - 3.0 / 16.0)
    exact = q0 * Ex / (2 * mu) * ((y + 0.5) * (ny - y - 0.5) + s)
    ux = o.field("ux")
    assert np.abs(ux - exact[:, None]).max() < 1e-6 * exact.max()
    uy = o.field("uy")
    stag = q0 * q0 / 4.0 * (-1.0) ** (y + o.steps_done)
    assert np.abs(uy * stag[:, None] / abs(stag[0]) ** 2 - 1.0).max() < 1e-3


@pytest.mark.parametrize("visc", [None, 0.05])
def test_shear_wave_decays_at_viscous_rate(visc):
    """Eq. 37-41: a shear wave u_x = U sin(k y) decays as exp(-nu k^2 t) with
    nu = cs^2 (tau_g - 1/2), or nu = mu/rho with the viscosity of Eq. 29."""
    nx, ny, U = 4, 64, 1e-4
    kw = dict(visc=(visc, visc, visc)) if visc else dict(tau_g=0.9)
    nu = visc if visc else CS2 * (0.9 - 0.5)
    p = W.params(nx=nx, ny=ny, bc_y=0, electric=0, **kw)
    k = 2 * math.pi / ny
    y = np.arange(ny, dtype=float)
    u = np.zeros((2, ny, nx))
    u[0] = (U * np.sin(k * y))[:, None]
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1), u=u)
    amp = []
    for t in (100, 600):
        o.step(t - o.steps_done)
        ux = o.field("ux")[:, 0]
        amp.append((ux * np.sin(k * y)).sum() * 2 / ny)
    rate = -math.log(amp[1] / amp[0]) / 500.0
    assert abs(rate / (nu * k * k) - 1.0) < 2e-3


# --------------------------------------------------------------------------- potential
def _potential(p, phi, q=None, tol=1e-13, max_iter=200000):
    o = oracle.Oracle(dict(p, poisson_tol=1e-30, poisson_max_iter=1, poisson_fixed_iter=1), phi)
    it, res, conv = o.solve_potential(q=q, tol=tol, max_iter=max_iter, check=10)
    assert conv
    return o


def test_potential_linear_between_electrodes():
    """Eq. 42-45 with uniform permittivity and no charge: the potential between
    electrodes at y = -1/2 (0) and ny - 1/2 (V) is linear, and E = -V/ny."""
    nx, ny, V = 4, 16, 1.0
    p = W.params(nx=nx, ny=ny, bc_y=2, electric=1, V_bottom=0.0, V_top=V, eps=(2.0, 2.0, 2.0), eps_ref=2.0)
    o = _potential(p, W.single_phase(nx, ny, 1))
    y = np.arange(ny)
    assert np.allclose(o.field("psi")[:, 0], V * (y + 0.5) / ny, atol=1e-9)
    assert np.allclose(o.field("ey"), -V / ny, atol=1e-9)


def test_potential_uniform_charge_slab():
    """Eq. 43 source term: a uniform charge q between grounded electrodes gives
    E_y = -q (ny - 1 - 2y) / (2 eps) exactly (sign and scale of varpi_j q and of
    Eq. 45), and psi = q (y + 1/2)(ny - 1/2 - y) / (2 eps) up to a uniform offset
    left by the anti-bounce-back walls, which is O(dx^2): it falls 4x per refinement."""
    rel = []
    for ny in (24, 48):
        nx, q0, e = 4, 1e-4, 2.0
        p = W.params(nx=nx, ny=ny, bc_y=2, electric=1, eps=(e, e, e), eps_ref=e)
        o = _potential(p, W.single_phase(nx, ny, 1), q=np.full((ny, nx), q0), tol=1e-12, max_iter=400000)
        y = np.arange(ny)
        exact = q0 * (y + 0.5) * (ny - 0.5 - y) / (2 * e)
        ey_exact = -q0 * (ny - 1 - 2 * y) / (2 * e)
        assert np.abs(o.field("ey")[:, 0] - ey_exact).max() < 1e-8 * np.abs(ey_exact).max()
        d = o.field("psi")[:, 0] - exact
        assert d.max() - d.min() < 1e-7 * exact.max()
        rel.append(d.mean() / exact.max())
    assert 3.9 < rel[0] / rel[1] < 4.1


@pytest.mark.parametrize("eps_ref", [1.0, 4.0])
def test_potential_layered_dielectric(eps_ref):
    """Eq. 42-45 with a permittivity contrast 1:4 across a flat interface: the
    steady flux eps dpsi/dy is uniform, so psi = V int dy/eps / int dy/eps.  Both
    choices of the split constant converge to the same solution."""
    nx, ny, D, V = 4, 64, 6.0, 1.0
    p = W.params(nx=nx, ny=ny, bc_y=2, electric=1, V_top=V, eps=(1.0, 2.0, 4.0), eps_ref=eps_ref, width_D=D)
    phi = W.flat_interface(nx, ny, D, 1, 3)
    o = _potential(p, phi)
    eps = (phi[0] ** 2 * (3 - 2 * phi[0]) * 1.0 + phi[2] ** 2 * (3 - 2 * phi[2]) * 4.0)[:, 0]
    # fine quadrature of 1/eps with eps linearly interpolated between cell centres
    yy = np.linspace(-0.5, ny - 0.5, 64 * ny + 1)
    ef = np.interp(yy, np.arange(ny), eps)
    inv = np.concatenate([[0.0], np.cumsum(0.5 * (1 / ef[1:] + 1 / ef[:-1]) * np.diff(yy))])
    exact = np.interp(np.arange(ny), yy, V * inv / inv[-1])
    psi = o.field("psi")[:, 0]
    assert np.abs(psi - exact).max() < 3e-3 * V
    flux = -o.field("ey")[:, 0] * eps
    assert np.abs(flux / flux.mean() - 1).max() < 1e-2


# --------------------------------------------------------------------------- charge
def test_uniform_charge_relaxation_factor():
    """Eq. 46-50 with the closed-form q = sum l + R/2: in a uniform medium
    q^{n+1} = q^n (1 - k/2)/(1 + k/2) with k = sigma/eps, exactly."""
    nx, ny = 4, 4
    s, e = 0.3, 2.0
    p = W.params(nx=nx, ny=ny, bc_y=0, electric=0, sigma=(s, s, s), eps=(e, e, e))
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1), q=np.full((ny, nx), 1e-3))
    qs = []
    for _ in range(6):
        o.step(1)
        qs.append(o.field("q")[0, 0])
    k = s / e
    ratio = np.array(qs[1:]) / np.array(qs[:-1])
    assert np.allclose(ratio, (1 - k / 2) / (1 + k / 2), rtol=1e-13, atol=0)
    assert np.isclose(qs[0], 1e-3 / (1 + k / 2), rtol=1e-14)


def test_charge_diffusion_gaussian():
    """Eq. 48 with R = 0 (no conductivity): a Gaussian charge blob keeps its total
    and its variance grows by exactly 2 alpha per step (closed form, tau_l =
    1/2 + alpha/cs^2)."""
    nx = ny = 64
    alpha, s0 = 0.1, 3.0
    p = W.params(nx=nx, ny=ny, bc_y=0, electric=0, sigma=(0, 0, 0), alpha=alpha)
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    r2 = (x - 32) ** 2 + (y - 32) ** 2
    q0 = 1e-3 * np.exp(-r2 / (2 * s0 * s0))
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1), q=q0)
    var = []
    for t in (20, 120):
        o.step(t - o.steps_done)
        q = o.field("q")
        var.append((q * r2).sum() / q.sum() / 2)
        assert abs(q.sum() - q0.sum()) < 1e-12
    assert abs((var[1] - var[0]) / (2 * alpha * 100) - 1) < 2e-3


def test_charge_blob_advected_by_uniform_flow():
    """Eq. 48-50 with convection (l^eq carries c.u, and T_j the backward difference
    of q u) and R = 0: a Gaussian charge blob in a uniform flow moves with the
    flow and spreads at the rate alpha in both directions (closed form of
    advection-diffusion: centroid x0 + u t, variance growth 2 alpha t per axis).
    Without the T_j source the lattice adds an O((tau_l - 1/2) u^2) diffusivity
    along the flow: here 1.2 of the 40 cells^2 (2.4 with T_j's sign reversed)."""
    n, alpha, u0, s0 = 96, 0.1, 0.1, 4.0
    p = W.params(nx=n, ny=n, bc_y=0, electric=0, sigma=(0, 0, 0), eps=(1.0, 1.0, 1.0), alpha=alpha,
                 charge_convection=1)
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    q0 = 1e-3 * np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (2 * s0 * s0))
    u = np.zeros((2, n, n))
    u[0] = u0
    o = oracle.Oracle(p, W.single_phase(n, n, 1), u=u, q=q0)

    def moments(q):
        # centroid along x on the periodic axis (circular mean), then variances
        ang = 2 * np.pi * x / n
        cx = (math.atan2((q * np.sin(ang)).sum(), (q * np.cos(ang)).sum()) % (2 * np.pi)) * n / (2 * np.pi)
        dx = (x - cx + n / 2) % n - n / 2
        dy = y - n / 2
        return cx, (q * dx * dx).sum() / q.sum(), (q * dy * dy).sum() / q.sum()

    o.step(20)
    c0, vx0, vy0 = moments(o.field("q"))
    o.step(200)
    q = o.field("q")
    c1, vx1, vy1 = moments(q)
    assert abs(q.sum() - q0.sum()) < 1e-12
    assert abs(((c1 - c0) % n) - u0 * 200) < 5e-3  # circular-mean estimate of the centroid
    assert abs((vx1 - vx0) - 2 * alpha * 200) < 0.01
    assert abs((vy1 - vy0) - 2 * alpha * 200) < 0.01


# --------------------------------------------------------------------------- coupled
def _laplace_jump(phi, p, steps, r_probe_in, r_probe_out):
    o = oracle.Oracle(p, phi)
    o.step(steps)
    pr = o.field("p")
    ny, nx = pr.shape
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r = np.hypot(x - nx / 2, y - ny / 2)
    return pr[r < r_probe_in].mean() - pr[r > r_probe_out].mean(), o


def test_laplace_pressure_two_phase_drop():
    """Capillary force of Eq. 27b through the pressure of Eq. 41: a 2-D drop of
    radius R at rest carries the jump p_in - p_out = gamma/R (within 10% at R = 16,
    D = 4)."""
    n, R = 64, 16.0
    p = W.params(nx=n, ny=n, bc_y=0, electric=0)
    phi = W.compound_droplet(n, n, 0.0, R, 4.0)
    phi[1] += phi[2]
    phi[2] = 0.0
    dp, o = _laplace_jump(phi, p, 3000, R - 6, R + 8)
    assert abs(dp / (1e-3 / R) - 1) < 0.10
    # parasitic currents stay far below the capillary velocity gamma / mu
    umax = np.hypot(o.field("ux"), o.field("uy")).max()
    assert umax < 1e-3 * 1e-3 / (1.0 * CS2 * 0.3)


def test_laplace_pressure_compound_drop():
    """Compound drop (core radius 8 in shell radius 16): the two jumps are
    gamma_23/R_in and gamma_12/R_out, here 1.6e-4 and 6.25e-5 with distinct
    tensions (within 12%)."""
    n = 64
    p = W.params(nx=n, ny=n, bc_y=0, electric=0, gamma12=1e-3, gamma13=1e-3, gamma23=1.28e-3)
    phi = W.compound_droplet(n, n, 8.0, 16.0, 4.0)
    o = oracle.Oracle(p, phi)
    o.step(3000)
    pr = o.field("p")
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r = np.hypot(x - n / 2, y - n / 2)
    p_in, p_shell, p_out = pr[r < 4].mean(), pr[(r > 11.5) & (r < 12.5)].mean(), pr[r > 24].mean()
    assert abs((p_in - p_shell) / (1.28e-3 / 8) - 1) < 0.12
    assert abs((p_shell - p_out) / (1e-3 / 16) - 1) < 0.12


def test_free_energy_non_increasing_without_field():
    """Eq. 18-25 (continuum dissipation): with no field, F_phi + F_u of a relaxing
    elliptical drop does not increase (sampled every 50 steps after 200)."""
    n = 48
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    r = np.sqrt(((x - 24) / 1.3) ** 2 + ((y - 24) / 0.8) ** 2)
    drop = 0.5 + 0.5 * np.tanh(2 * (10 - r) / 4)
    phi = np.stack([1 - drop, drop, 0 * drop])
    o = oracle.Oracle(W.params(nx=n, ny=n, bc_y=0, electric=0), phi)
    o.step(200)
    vals = []
    for _ in range(12):
        ob = o.observables()
        vals.append(ob["F_phi"] + ob["F_u"])
        o.step(50)
    d = np.diff(vals)
    assert (d <= 1e-12 * vals[0]).all()
    assert vals[-1] < vals[0]


@pytest.mark.parametrize("eps_in", [4.0, 0.25])
def test_perfect_dielectric_drop_elongates_along_field(eps_in):
    """The electric term -1/2 eps'(phi)|E|^2 of Eq. 20 (no conductivity, no
    charge): a perfect-dielectric drop stretches along the field whatever the
    permittivity ratio (classical electrostriction result), so D > 0."""
    n, R = 48, 10.0
    E0 = 0.02
    p = W.params(nx=n, ny=n, bc_y=2, electric=1, V_top=E0 * n, sigma=(0, 0, 0),
                 eps=(1.0, eps_in, 1.0), eps_ref=max(1.0, eps_in), inner_phase=2,
                 poisson_check_every=5, poisson_tol=1e-10)
    phi = W.compound_droplet(n, n, 0.0, R, 4.0)
    phi[1] += phi[2]
    phi[2] = 0.0
    o = oracle.Oracle(p, phi)
    o.step(400)
    D = o.observables()["D_inner"]
    assert D > 1e-4


# --------------------------------------------------------------------------- FD potential
def _fd(p, phi, q=None):
    o = oracle.Oracle(dict(p, potential_solver=1), phi)
    it, res, conv = o.solve_potential(q=q)
    assert conv and res < 1e-12
    return o


def test_fd_potential_linear_between_electrodes_exact():
    """Eq. 27d in 5-point form, uniform eps, no charge: psi = V (y + 1/2)/ny and
    E = -V/ny exactly (the half-cell Dirichlet face and the Eq. 33 gradient are
    exact on linear fields)."""
    nx, ny, V = 8, 20, 0.7
    p = W.params(nx=nx, ny=ny, bc_y=2, V_top=V, eps=(3.0, 3.0, 3.0))
    o = _fd(p, W.single_phase(nx, ny, 1))
    y = np.arange(ny)
    assert np.allclose(o.field("psi")[:, 0], V * (y + 0.5) / ny, atol=1e-12)
    assert np.allclose(o.field("ey"), -V / ny, atol=1e-12)
    assert np.abs(o.field("ex")).max() < 1e-13


def test_fd_potential_periodic_mode_is_the_discrete_eigenfunction():
    """Periodic, uniform eps, q = sin(2 pi k x / nx): the 5-point operator's
    eigenvalue is eps (2 - 2 cos(2 pi k / nx)), so psi = q / that, exactly."""
    nx, ny, e, k = 32, 6, 2.0, 3
    p = W.params(nx=nx, ny=ny, bc_y=0, eps=(e, e, e))
    x = np.arange(nx)
    q = np.tile(1e-3 * np.sin(2 * np.pi * k * x / nx), (ny, 1))
    o = _fd(p, W.single_phase(nx, ny, 1), q=q)
    lam = e * (2 - 2 * np.cos(2 * np.pi * k / nx))
    assert np.allclose(o.field("psi"), q / lam, rtol=0, atol=1e-12 * np.abs(q / lam).max())


def test_fd_potential_layered_dielectric_discrete_series():
    """eps varying in y only, no charge, electrodes: the discrete flux through
    every face is the same, so psi follows the series of face resistances
    (harmonic-mean faces, half-cell Dirichlet faces at the walls) exactly."""
    nx, ny, D, V = 4, 40, 6.0, 1.0
    p = W.params(nx=nx, ny=ny, bc_y=2, V_top=V, eps=(1.0, 2.0, 4.0), width_D=D)
    phi = W.flat_interface(nx, ny, D, 1, 3)
    o = _fd(p, phi)
    eps = (phi[0] ** 2 * (3 - 2 * phi[0]) * 1.0 + phi[2] ** 2 * (3 - 2 * phi[2]) * 4.0)[:, 0]
    r = [1 / (2 * eps[0])] + [1 / (2 * eps[i] * eps[i + 1] / (eps[i] + eps[i + 1])) for i in range(ny - 1)] \
        + [1 / (2 * eps[-1])]
    cum = np.cumsum(r)
    exact = V * cum[:-1] / cum[-1]
    assert np.allclose(o.field("psi")[:, 0], exact, atol=1e-12)


def test_fd_potential_charge_slab_second_order():
    """Uniform charge between grounded electrodes: the FD potential converges to
    q (y + 1/2)(ny - 1/2 - y) / (2 eps) at second order."""
    errs = []
    for ny in (16, 32, 64):
        nx, q0, e = 4, 1e-3, 2.0
        p = W.params(nx=nx, ny=ny, bc_y=2, eps=(e, e, e))
        o = _fd(p, W.single_phase(nx, ny, 1), q=np.full((ny, nx), q0))
        y = np.arange(ny)
        exact = q0 * (y + 0.5) * (ny - 0.5 - y) / (2 * e)
        errs.append(np.abs(o.field("psi")[:, 0] - exact).max() / exact.max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert errs[2] < 2e-3


def test_electroosmotic_channel_matches_debye_hueckel_profiles():
    """The electro-osmotic channel of the paper's Section 5.1 with its
    Debye-Hueckel closure (q = -eps kappa^2 psi, the linearised Boltzmann response
    of a symmetric electrolyte): walls at the zeta potential, a uniform axial field
    E, single phase.  Eq. 53 fixes the steady profiles
        psi(y) = zeta cosh(kappa y) / cosh(kappa h),
        u(y) = -(eps zeta E / mu) (1 - cosh(kappa y) / cosh(kappa h)),
    y from the mid-plane, h the half-height.  This pins the potential solve with
    electrodes and a charge source, the sign and size of the Coulomb force qE, and
    the flow's response with no-slip walls; errors are O((kappa dx)^2)."""
    nx, ny = 2, 100
    h = ny / 2
    kappa, zeta, E = 5.0 / h, 1e-3, 1e-3
    tau_g = 0.8
    mu = (tau_g - 0.5) / 3.0
    p = W.params(nx=nx, ny=ny, bc_y=2, electric=1, eps=(1.0, 1.0, 1.0), sigma=(0.0, 0.0, 0.0), eps_ref=1.0,
                 V_bottom=zeta, V_top=zeta, E_ext=(E, 0.0), tau_g=tau_g, debye_kappa2=kappa * kappa,
                 poisson_tol=1e-11, poisson_max_iter=200000, poisson_check_every=10)
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1))
    o.step(60000)
    yc = np.arange(ny) + 0.5 - h
    prof = np.cosh(kappa * yc) / np.cosh(kappa * h)
    psi = o.field("psi")[:, 0]
    ux = o.field("ux")[:, 0]
    u_ref = -(1.0 * zeta * E / mu) * (1.0 - prof)
    # measured 0.9% (psi) and 0.35% (u); psi also carries the O(dx^2) electrode
    # offset of anti-bounce-back with charge present
    assert np.abs(psi - zeta * prof).max() <= 2e-2 * zeta
    assert np.abs(ux - u_ref).max() <= 2e-2 * np.abs(u_ref).max()
    assert np.abs(o.field("uy")).max() <= 1e-6 * np.abs(u_ref).max()


def test_lb_potential_converges_to_the_fd_solution_with_variable_permittivity():
    """Eq. 42-45 split the permittivity into eps_ref (in tau_h) and eps_hat (in the
    source); the fixed point must solve div(eps grad psi) + q = 0 for a variable eps.
    Against the oracle's independent finite-difference solve of that equation
    (harmonic-mean faces, conjugate gradients), on a smooth low-contrast eps (1 to
    1.45) with charge and electrodes: the difference falls toward second order
    with the grid (measured 3.7e-3, 1.3e-3, 3.6e-4 on 32, 64, 128)."""
    diffs = []
    for n in (32, 64, 128):
        x, y = np.meshgrid((np.arange(n) + 0.5) / n, (np.arange(n) + 0.5) / n)
        p2 = 0.3 * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.05)
        phi = np.stack([1 - p2, p2, np.zeros_like(p2)])
        q = 64e-3 * np.sin(2 * np.pi * x) * np.sin(np.pi * y) / n ** 2
        psi = []
        for solver in (0, 1):
            p = W.params(nx=n, ny=n, bc_y=2, electric=1, eps=(1.0, 1.5, 1.0), sigma=(0.0, 0.0, 0.0), eps_ref=1.5,
                         V_bottom=0.0, V_top=0.02, potential_solver=solver, poisson_tol=1e-12,
                         poisson_max_iter=2000000, poisson_check_every=50)
            psi.append(oracle.Oracle(p, phi, q=q).field("psi"))
        diffs.append(np.abs(psi[0] - psi[1]).max() / np.abs(psi[1]).max())
    rates = [math.log2(diffs[k] / diffs[k + 1]) for k in range(2)]
    assert diffs[-1] < 5e-4 and min(rates) > 1.3, (diffs, rates)


# --------------------------------------------------------------------------- observables (Eq. 18, Section 5.3)
def _ellipse(nx, ny, a, b, xc, yc, W=4.0):
    """Smooth indicator of an ellipse with semi-axis a along y and b along x: a tanh
    of the elliptic radius, so its second moments scale exactly as a^2 and b^2."""
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    r = np.sqrt(((x - xc) / b) ** 2 + ((y - yc) / a) ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * (1.0 - r) * np.sqrt(a * b) / W)


def test_deformation_factors_of_ellipses():
    """Section 5.3's D = (a - b)/(a + b), a along the field (y), b across it, from the
    indicator's second moments: the inner indicator phi_inner and the outer one
    1 - phi_matrix, on two off-centre ellipses of different shape and orientation."""
    n = 256
    inner = _ellipse(n, n, 30.0, 20.0, 127.3, 129.6)          # elongated along y: D = +0.2
    outer = _ellipse(n, n, 50.0, 70.0, 127.3, 129.6)          # elongated along x: D = -1/6
    phi3 = inner
    phi2 = outer * (1.0 - inner)
    phi = np.stack([1.0 - phi2 - phi3, phi2, phi3])
    p = W.params(nx=n, ny=n, bc_y=1, electric=0, inner_phase=3, matrix_phase=1)
    obs = oracle.Oracle(p, phi).observables()
    assert abs(obs["D_inner"] - 0.2) < 1e-6, obs["D_inner"]
    assert abs(obs["D_outer"] - (-20.0 / 120.0)) < 1e-6, obs["D_outer"]
    # a sharp ellipse: the same value up to the lattice quadrature of its edge
    y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    sharp = ((((x - 120.4) / 40.0) ** 2 + ((y - 131.1) / 60.0) ** 2) <= 1.0).astype(float)
    phi = np.stack([1.0 - sharp, np.zeros_like(sharp), sharp])
    obs = oracle.Oracle(p, phi).observables()
    assert abs(obs["D_inner"] / 0.2 - 1.0) < 5e-3, obs["D_inner"]
    assert abs(obs["D_outer"] / 0.2 - 1.0) < 5e-3, obs["D_outer"]


def test_electric_energy_of_a_uniform_and_a_layered_dielectric():
    """Eq. 18's electric part |D|^2/(2 eps) = eps |E|^2 / 2 summed over cells.
    Uniform permittivity 2.5 between electrodes: E = dV/ny exactly, so F_E =
    eps (dV/ny)^2 N / 2.  Sharp layers of permittivity 1 and 4 (series
    capacitor): E_k = dV / (L_1/eps_1 + L_3/eps_3) / eps_k in each layer, F_E =
    sum_k eps_k E_k^2 L_k nx / 2 (the LB potential is exact on cell-wise layers)."""
    nx, ny, V = 8, 64, 0.3
    p = W.params(nx=nx, ny=ny, bc_y=2, electric=1, V_top=V, eps=(2.5, 2.5, 2.5), eps_ref=2.5,
                 poisson_tol=1e-13, poisson_max_iter=400000)
    o = oracle.Oracle(p, W.single_phase(nx, ny, 1))
    assert abs(o.observables()["F_E"] / (0.5 * 2.5 * (V / ny) ** 2 * nx * ny) - 1.0) < 1e-9
    phi = np.zeros((3, ny, nx))
    phi[0, : ny // 2] = 1.0
    phi[2, ny // 2:] = 1.0
    p = dict(p, eps=(1.0, 2.0, 4.0), eps_ref=4.0)
    o = oracle.Oracle(p, phi)
    L = ny / 2
    D = V / (L / 1.0 + L / 4.0)
    want = 0.5 * nx * L * (D ** 2 / 1.0 + D ** 2 / 4.0)
    assert abs(o.observables()["F_E"] / want - 1.0) < 1e-9, (o.observables()["F_E"], want)


def test_charge_and_kinetic_energy_of_uniform_states():
    """Eq. 18's charge part alpha q^2 / (2 sigma) and the kinetic part rho |u|^2 / 2,
    summed over cells, on the initial state: uniform q and u over two half-lattices
    of phases with different conductivity and density."""
    nx, ny = 16, 12
    q0, u0, v0, alpha = 2e-3, 3e-3, -1e-3, 0.1
    phi = np.zeros((3, ny, nx))
    phi[0, : ny // 2] = 1.0
    phi[1, ny // 2:] = 1.0
    p = W.params(nx=nx, ny=ny, bc_y=1, electric=0, alpha=alpha, sigma=(0.4, 0.1, 0.2), rho=(1.0, 3.0, 1.0))
    u = np.stack([np.full((ny, nx), u0), np.full((ny, nx), v0)])
    o = oracle.Oracle(p, phi, u=u, q=np.full((ny, nx), q0))
    obs = o.observables()
    half = nx * ny / 2
    want_q = 0.5 * alpha * q0 ** 2 * half * (1 / 0.4 + 1 / 0.1)
    want_u = 0.5 * (u0 ** 2 + v0 ** 2) * half * (1.0 + 3.0)
    assert abs(obs["F_q"] / want_q - 1.0) < 1e-12, (obs["F_q"], want_q)
    assert abs(obs["F_u"] / want_u - 1.0) < 1e-12, (obs["F_u"], want_u)
    assert abs(obs["charge"] / (q0 * nx * ny) - 1.0) < 1e-12
