"""Seeded synthetic workloads for the three-phase EHD lattice Boltzmann step.

This module holds the inputs both implementations are fed with: parameter sets,
initial phase fields and population noise.  It contains none of the method's
update arithmetic -- only the initial conditions the paper prescribes for its
benchmarks (the tanh profiles of Eq. 54 and Eq. 56) and seeded random numbers.

Phase labels follow the workload definitions, not the paper's figures:
  * compound droplet: phase 1 = matrix, phase 2 = shell, phase 3 = inner core;
  * liquid lens:      phase 1 = upper fluid, phase 2 = lower fluid, phase 3 = lens.
Arrays are C-ordered ``[..., ny, nx]`` float64, x fastest.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20261202

#: ordered parameter keys shared by both implementations (plain numbers only)
PARAM_DEFAULTS = dict(
    nx=64, ny=64,
    bc_y=2,                      # 0 periodic, 1 walls, 2 walls carrying electrodes
    electric=1,                  # 1: solve the potential every step; 0: E = E_ext
    precision=0,                 # GPU only: 0 fp64, 1 fp32, 2 fp32 compute + fp16 store
    rho=(1.0, 1.0, 1.0),
    visc=(0.0, 0.0, 0.0),        # dynamic viscosity per phase; all <= 0 -> constant tau_g
    tau_g=0.8,
    gamma12=1e-3, gamma13=1e-3, gamma23=1e-3,
    width_D=4.0,
    tau_f=0.8,
    eps=(1.0, 2.0, 4.0),
    sigma=(1.0, 0.5, 0.25),
    eps_ref=4.0,
    alpha=0.1,
    V_bottom=0.0, V_top=0.0,
    E_ext=(0.0, 0.0),
    u_wall_bottom=0.0, u_wall_top=0.0,
    charge_convection=1,
    inner_phase=3, matrix_phase=1,
    poisson_tol=1e-8,
    poisson_max_iter=20000,
    poisson_check_every=8,
    poisson_fixed_iter=0,
    potential_solver=0,          # 0 the LB pseudo-time solve of the paper; 1 multigrid on its FD form
    tangent_param=(-1, -1, -1),  # GPU tangent builds: parameter per tangent direction
    debye_kappa2=0.0,            # oracle only: > 0 replaces the charge by -eps kappa^2 psi (EOF check)
    ions=0,                      # 1: two Nernst-Planck ion species carry the charge (Eq. 52)
    ion_D=(0.05, 0.05),          # ion diffusivities (lattice units)
    ion_z=(1.0, -1.0),           # valences
    ion_beta=1.0,                # e / (k_B T): inverse thermal voltage
    ion_charge=1.0,              # charge per unit concentration
)


def params(**kw) -> dict:
    p = dict(PARAM_DEFAULTS)
    for k, v in kw.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def _grid(nx: int, ny: int):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    return x, y


def compound_droplet(nx: int, ny: int, r_in: float, r_out: float, W: float,
                     xc: float | None = None, yc: float | None = None) -> np.ndarray:
    """Concentric compound drop, Eq. 54 with the workload labels:
    phase 3 (core) radius r_in inside phase 2 (shell) radius r_out inside phase 1."""
    x, y = _grid(nx, ny)
    xc = nx / 2 if xc is None else xc
    yc = ny / 2 if yc is None else yc
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    p3 = 0.5 + 0.5 * np.tanh(2.0 * (r_in - r) / W)
    p2 = (1.0 - p3) * (0.5 + 0.5 * np.tanh(2.0 * (r_out - r) / W))
    p1 = 1.0 - p2 - p3
    return np.ascontiguousarray(np.stack([p1, p2, p3]))


def liquid_lens(nx: int, ny: int, R: float, D: float, xc: float, yc: float) -> np.ndarray:
    """Lens between two layers, Eq. 56 with the workload labels: phase 3 is the
    circular lens, phase 1 the upper layer (clipped at 0), phase 2 the rest."""
    x, y = _grid(nx, ny)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    p3 = 0.5 + 0.5 * np.tanh(2.0 * (R - r) / D)
    p1 = np.maximum(0.5 + 0.5 * np.tanh(2.0 * (y - yc) / D) - p3, 0.0)
    p2 = 1.0 - p1 - p3
    return np.ascontiguousarray(np.stack([p1, p2, p3]))


def single_phase(nx: int, ny: int, phase: int = 1) -> np.ndarray:
    phi = np.zeros((3, ny, nx))
    phi[phase - 1] = 1.0
    return phi


def flat_interface(nx: int, ny: int, D: float, i: int, j: int, y0: float | None = None) -> np.ndarray:
    """Phase i below, phase j above a flat tanh interface at height y0."""
    _, y = _grid(nx, ny)
    y0 = ny / 2 - 0.5 if y0 is None else y0
    top = 0.5 + 0.5 * np.tanh(2.0 * (y - y0) / D)
    phi = np.zeros((3, ny, nx))
    phi[j - 1] = top
    phi[i - 1] = 1.0 - top
    return phi


def noise(nx: int, ny: int, amp: float, seed: int = SEED) -> np.ndarray:
    """Uniform population noise U(-amp, amp) for the sets (g, f1, f2, f3, l),
    drawn in order set, direction, y, x; never added to the potential set."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=(5, 9, ny, nx))


def ion_concentrations(nx: int, ny: int, n0: float = 1.0, amp: float = 0.0, seed: int = SEED) -> np.ndarray:
    """Concentrations [2, ny, nx] of two ion species: n0 (1 + U(-amp, amp)), drawn in
    order species, y, x."""
    rng = np.random.default_rng(seed)
    return n0 * (1.0 + rng.uniform(-amp, amp, size=(2, ny, nx)))


def debye_layers(nx: int, ny: int, zeta: float, kappa: float, beta: float, n0: float = 1.0,
                 z=(1.0, -1.0)) -> np.ndarray:
    """Concentrations [2, ny, nx] of a symmetric electrolyte in the Debye-Hueckel double
    layers of a channel whose walls (y = -1/2, ny - 1/2) sit at the zeta potential:
    n_i = n0 exp(-z_i beta psi(y)) with psi = zeta cosh(kappa y') / cosh(kappa h), y'
    measured from the mid-plane, h = ny / 2 (Eq. 53)."""
    h = ny / 2
    yc = np.arange(ny) + 0.5 - h
    psi = zeta * np.cosh(kappa * yc) / np.cosh(kappa * h)
    return np.stack([np.repeat(n0 * np.exp(-zi * beta * psi)[:, None], nx, axis=1) for zi in z])


# ---------------------------------------------------------------------------
# The five workloads.  Sizes and parameters are the stated ones.  Where a value is
# left open: gamma = 1e-3, D = 4, rho = 1 and tau_g = 0.8 everywhere; permittivity
# and conductivity taken literally in lattice units; E0 from Eq. 51 with the
# matrix permittivity and the outer radius.
# ---------------------------------------------------------------------------

def config_static_compound(precision: int = 0, n: int = 64, field: bool = True, **kw):
    """64x64 static compound drop (core radius 8, shell radius 16), electrodes at
    the y walls with potential difference 0.01, noise 1e-8; 2000 steps."""
    r_out = 16.0 * n / 64
    r_in = 8.0 * n / 64
    p = params(nx=n, ny=n, bc_y=2 if field else 1, electric=1 if field else 0,
               precision=precision, V_bottom=0.0, V_top=0.01 if field else 0.0, **kw)
    phi = compound_droplet(n, n, r_in, r_out, 4.0)
    return dict(name=f"static_compound_{n}x{n}", params=p, phi=phi,
                noise=noise(n, n, 1e-8), steps=2000)


def config_lens(tensions=(1e-3, 1e-3, 1e-3), nx: int = 512, ny: int = 256, R: float = 40.0,
                precision: int = 1, **kw):
    """Liquid lens spreading on a flat interface between walls, no field; 20000 steps."""
    g12, g13, g23 = tensions
    p = params(nx=nx, ny=ny, bc_y=1, electric=0, precision=precision,
               gamma12=g12, gamma13=g13, gamma23=g23, V_top=0.0, **kw)
    phi = liquid_lens(nx, ny, R, 4.0, nx / 2, ny / 2)
    return dict(name=f"lens_{nx}x{ny}", params=p, phi=phi, noise=None, steps=20000)


def field_for_capillary(ca_e: float, gamma: float, eps_matrix: float, radius: float) -> float:
    """Field magnitude from the electric capillary number of Eq. 51."""
    return math.sqrt(ca_e * gamma / (eps_matrix * radius))


def config_deformation(n: int = 4096, r_out: float = 600.0, r_in: float = 300.0,
                       ca_e: float = 0.5, precision: int = 1, **kw):
    """Compound drop deforming in a uniform field between electrodes (4096^2)."""
    eps = (1.0, 2.0, 4.0)
    E0 = field_for_capillary(ca_e, 1e-3, eps[0], r_out)
    p = params(nx=n, ny=n, bc_y=2, electric=1, precision=precision, eps=eps,
               sigma=(1.0, 0.5, 0.25), eps_ref=eps[2], V_bottom=0.0, V_top=E0 * n,
               charge_convection=1, **kw)
    phi = compound_droplet(n, n, r_in, r_out, 4.0)
    return dict(name=f"deformation_{n}x{n}", params=p, phi=phi, noise=None, steps=5000, E0=E0)


def config_batched_sweep(count: int = 256, seed: int = SEED, iters: int = 16, precision: int = 1):
    """Parameter-sweep instances: side from {128,192,256,384,512}, Ca_E ~ U[0.1,1],
    permittivity ratio inner/outer ~ U[0.5,4], conductivity ratio ~ U[0.25,2].
    The sweep states no potential tolerance; every instance iterates the potential
    a fixed `iters` times per step (warm-started), so all do the same work.
    Initial fields come from `sweep_phi(instance)`."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.array([128, 192, 256, 384, 512]), size=count)
    ca = rng.uniform(0.1, 1.0, size=count)
    s_ratio = rng.uniform(0.5, 4.0, size=count)
    r_ratio = rng.uniform(0.25, 2.0, size=count)
    out = []
    for k in range(count):
        n = int(sides[k])
        e1, e3 = 1.0, float(s_ratio[k])
        s1, s3 = 1.0, float(r_ratio[k])
        e2, s2 = math.sqrt(e1 * e3), math.sqrt(s1 * s3)
        r_out = 0.25 * n
        E0 = field_for_capillary(float(ca[k]), 1e-3, e1, r_out)
        p = params(nx=n, ny=n, bc_y=2, electric=1, precision=precision, eps=(e1, e2, e3),
                   sigma=(s1, s2, s3), eps_ref=max(e1, e2, e3), V_top=E0 * n, poisson_fixed_iter=iters)
        out.append(dict(name=f"sweep_{k}", params=p, ca_e=float(ca[k]), eps_ratio=e3 / e1,
                        sigma_ratio=s3 / s1, shape=(n, n), r_out=r_out, r_in=0.5 * r_out, steps=3000))
    return out


def sweep_phi(inst: dict) -> np.ndarray:
    n = inst["shape"][0]
    return compound_droplet(n, n, inst["r_in"], inst["r_out"], 4.0)


def config_adjoint(n: int = 256, precision: int = 1, **kw):
    """Compound drop under field plus shear (walls at -/+1e-3)."""
    eps = (1.0, 2.0, 4.0)
    E0 = field_for_capillary(0.5, 1e-3, eps[0], 64.0)
    p = params(nx=n, ny=n, bc_y=2, electric=1, precision=precision, eps=eps,
               sigma=(1.0, 0.5, 0.25), eps_ref=eps[2], V_top=E0 * n,
               u_wall_bottom=-1e-3, u_wall_top=1e-3, **kw)
    phi = compound_droplet(n, n, 32.0, 64.0, 4.0)
    return dict(name=f"adjoint_{n}x{n}", params=p, phi=phi, noise=None, steps=4000, E0=E0)


# ---------------------------------------------------------------------------
# Second workload: two compound drops under a field, and a compound drop in a
# confined shear flow under a field (the paper's Section 5.4-5.5 studies).  Phase
# labels as above: 1 matrix, 2 shell, 3 core.  The paper writes its ratios
# S_ij = eps_i / eps_j, R_ij = sigma_i / sigma_j with 1 core, 2 shell, 3 bulk, so
# its S23, R23 are shell / matrix and S12, R12 core / shell.
# ---------------------------------------------------------------------------

def _ratios_to_props(S12: float, S23: float, R12: float, R23: float, sigma_matrix: float):
    """(eps, sigma) per workload phase (matrix, shell, core) from the paper's ratios,
    matrix permittivity 1."""
    e_shell = S23
    e_core = S12 * e_shell
    s_shell = R23 * sigma_matrix
    s_core = R12 * s_shell
    return (1.0, e_shell, e_core), (sigma_matrix, s_shell, s_core)


def two_compound_drops(nx: int, ny: int, r_in: float, r_out: float, W: float, gap: float) -> np.ndarray:
    """Two equal compound drops centred on the vertical line x = nx/2 (along the
    field), their shells `gap` cells apart; each profile as in Eq. 54."""
    x, y = _grid(nx, ny)
    d = r_out + gap / 2
    p3 = np.zeros((ny, nx))
    shell = np.zeros((ny, nx))
    for yc in (ny / 2 - d, ny / 2 + d):
        r = np.sqrt((x - nx / 2) ** 2 + (y - yc) ** 2)
        p3 += 0.5 + 0.5 * np.tanh(2.0 * (r_in - r) / W)
        shell += 0.5 + 0.5 * np.tanh(2.0 * (r_out - r) / W)
    p3 = np.minimum(p3, 1.0)
    p2 = (1.0 - p3) * np.minimum(shell, 1.0)
    p1 = 1.0 - p2 - p3
    return np.ascontiguousarray(np.stack([p1, p2, p3]))


# the paper's two regimes of drop pairs (its Figs. 10, 11)
TWO_DROP_REGIMES = {
    "coalescence": dict(S12=1.0 / 8.0, S23=8.0, R12=1.0 / 6.0, R23=6.0),
    "separation": dict(S12=5.0, S23=0.2, R12=1.0 / 1.04, R23=1.04),
}


def config_two_drops(regime: str, n: int = 256, r_in: float = 12.0, r_out: float = 24.0, gap: float = 8.0,
                     ca_e: float = 0.2, sigma_matrix: float = 0.1, iters: int = 16, precision: int = 1, **kw):
    """Two compound drops aligned with the field between electrodes (Ca_E = 0.2,
    equal densities and viscosities); the potential iterated `iters` times a step."""
    eps, sigma = _ratios_to_props(sigma_matrix=sigma_matrix, **TWO_DROP_REGIMES[regime])
    E0 = field_for_capillary(ca_e, 1e-3, eps[0], r_out)
    p = params(nx=n, ny=n, bc_y=2, electric=1, precision=precision, eps=eps, sigma=sigma,
               eps_ref=max(eps), V_bottom=0.0, V_top=E0 * n, poisson_fixed_iter=iters, **kw)
    return dict(name=f"two_drops_{regime}_{n}", params=p, phi=two_compound_drops(n, n, r_in, r_out, 4.0, gap),
                noise=None, regime=regime, gap=gap, r_out=r_out)


def config_shear_regimes(ca_e=(0.2, 0.4, 0.6, 0.8, 1.0), wc=(0.3, 0.5, 0.6, 0.75), r_in: float = 15.0,
                         r_out: float = 30.0, nx: int = 256, ca: float = 0.5, tau_g: float = 1.5,
                         re_e: float = 0.01, iters: int = 16, precision: int = 1):
    """Compound drop in a channel whose walls slide at -/+U and carry electrodes,
    one instance per (Ca_E, W_c): the paper's regime diagram (its Fig. 15) with its
    ratios S12 = 0.5, S23 = 2, R12 = 2, R23 = 0.5 and Ca = 0.5.  Readings: W_c =
    R_b / H with H the half-height (channel height 2 R_b / W_c); Ca = mu gamma_dot
    R_b / gamma with gamma_dot = 2 U / height; Re_E = eps gamma_dot / sigma fixes the
    matrix conductivity; tau_g = 1.5 gives Re = rho gamma_dot R_b^2 / mu ~ 0.14."""
    gamma = 1e-3
    mu = (tau_g - 0.5) / 3.0  # rho = 1
    gdot = ca * gamma / (mu * r_out)
    eps, sigma = _ratios_to_props(S12=0.5, S23=2.0, R12=2.0, R23=0.5, sigma_matrix=gdot / re_e)
    out = []
    for w in wc:
        ny = 2 * int(round(r_out / w))
        U = 0.5 * gdot * ny
        for c in ca_e:
            E0 = field_for_capillary(c, gamma, eps[0], r_out)
            p = params(nx=nx, ny=ny, bc_y=2, electric=1, precision=precision, eps=eps, sigma=sigma,
                       eps_ref=max(eps), tau_g=tau_g, V_bottom=0.0, V_top=E0 * ny,
                       u_wall_bottom=-U, u_wall_top=U, poisson_fixed_iter=iters)
            out.append(dict(params=p, phi=compound_droplet(nx, ny, r_in, r_out, 4.0), ca_e=c, wc=w,
                            shear_rate=gdot, capillary_time=mu * r_out / gamma))
    return out


def config_eof_channel(nx: int = 10240, ny: int = 2048, kappa_h: float = 20.0, zeta: float = 1e-3,
                       E: float = 1e-3, beta: float = 1.0, D: float = 0.1, precision: int = 1, **kw):
    """The electro-osmotic channel of Section 5.1 in lattice units (length 5 H, as in
    the paper's 5 um x 1 um channel): one phase between electrodes at the zeta
    potential, two Nernst-Planck species (z = +-1, n0 = 1) started in their Debye-
    Hueckel double layers, a uniform axial field E.  The charge per concentration
    gives kappa^2 = 2 beta e_q n0 / eps.  The potential is the multigrid solve of its
    finite-difference form."""
    kappa = kappa_h / (ny / 2)
    base = dict(nx=nx, ny=ny, bc_y=2, electric=1, precision=precision, eps=(1.0, 1.0, 1.0),
                sigma=(0.0, 0.0, 0.0), eps_ref=1.0, V_bottom=zeta, V_top=zeta, E_ext=(E, 0.0),
                tau_g=0.5 + math.sqrt(3.0 / 16.0), ions=1, ion_D=(D, D), ion_z=(1.0, -1.0), ion_beta=beta,
                ion_charge=kappa * kappa / (2.0 * beta), potential_solver=1, poisson_tol=1e-8,
                poisson_max_iter=50)
    base.update(kw)
    p = params(**base)
    return dict(name=f"eof_channel_{nx}x{ny}", params=p, phi=single_phase(nx, ny, 1),
                ions=debye_layers(nx, ny, zeta, kappa, beta), kappa=kappa, steps=1000)


def compound_sphere(n: int, r_in: float, r_out: float, W: float) -> np.ndarray:
    """[3, n, n, n] phases of a compound sphere centred in an n^3 box: core (phase 3)
    of radius r_in, shell (phase 2) out to r_out, matrix (phase 1); tanh profiles of
    width W (the three-dimensional counterpart of compound_droplet)."""
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float),) * 3, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    core = 0.5 - 0.5 * np.tanh(2.0 * (r - r_in) / W)
    drop = 0.5 - 0.5 * np.tanh(2.0 * (r - r_out) / W)
    return np.stack([1.0 - drop, drop - core, core])


def config_deformation_3d(n: int = 256, r_out: float = 40.0, r_in: float = 20.0, ca_e: float = 0.5,
                          precision: int = 1, iters: int = 16, **kw):
    """Compound drop deforming in a uniform field between electrodes on a D3Q15
    lattice (the paper's compound-drop deformation runs are three-dimensional):
    n^3 cells, walls and electrodes normal to z, permittivity 1:2:4, conductivity
    1:0.5:0.25, Ca_E from Eq. 51.  The potential is iterated a fixed `iters` times a
    step, warm-started."""
    eps = (1.0, 2.0, 4.0)
    E0 = field_for_capillary(ca_e, 1e-3, eps[0], r_out)
    p = params(nx=n, ny=n, bc_y=2, electric=1, precision=precision, eps=eps, sigma=(1.0, 0.5, 0.25),
               eps_ref=eps[2], V_bottom=0.0, V_top=E0 * n, charge_convection=1, poisson_fixed_iter=iters, **kw)
    p["nz"] = n
    return dict(name=f"deformation3d_{n}^3", params=p, phi=compound_sphere(n, r_in, r_out, 4.0), E0=E0)
