"""Pins of the oracle's reverse mode (the transposed step and creation) against
central differences of the oracle's own forward step.

The adjoint is the transpose of the derivative of the discrete step: for any
directions v (state) and w (next state), <(dX'/dX) v, w> = <v, (dX'/dX)^T w>, and for
the parameters dJ/dtheta of J = <w, X^M(theta)> must equal the derivative of the
forward runs.  The forward derivative is taken by central differences in FP64, so a
check is as tight as their truncation and rounding allow (1e-8 relative here); the
blocks of the map that are affine (the potential populations into themselves and
into the field) are checked to rounding.  The configurations cover electrodes with
moving walls, insulating walls, periodic y, per-phase viscosity, charge convection on
and off, unequal densities, and the first step (no d/dt terms).
"""
import numpy as np
import pytest

import oracle
import workloads as W

SP = oracle.STATE_PLANES


def _case(bc_y=2, visc=False, cc=1, K=6, nx=24, ny=20):
    kw = dict(nx=nx, ny=ny, bc_y=bc_y, electric=1, precision=0, eps=(1.0, 2.0, 4.0), sigma=(1.0, 0.5, 0.25),
              eps_ref=4.0, V_top=0.02 if bc_y == 2 else 0.0, V_bottom=0.0, charge_convection=cc,
              poisson_fixed_iter=K, rho=(1.0, 1.3, 0.8), gamma12=1e-3, gamma13=1.2e-3, gamma23=0.8e-3)
    if bc_y:
        kw.update(u_wall_bottom=-1e-3, u_wall_top=1e-3)
    if bc_y != 2:
        kw["E_ext"] = (1e-3, 2e-3)      # a field without electrodes
    if visc:
        kw["visc"] = (0.1, 0.2, 0.15)
    p = W.params(**kw)
    phi = W.compound_droplet(nx, ny, 3.0, 6.0, 4.0)
    return p, phi


CASES = [dict(), dict(visc=True), dict(bc_y=1), dict(bc_y=0), dict(cc=0)]


def _dirs(o, seed):
    X = o.state_vector()
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(X.shape) * np.maximum(np.abs(X).max(axis=(1, 2), keepdims=True), 1e-8)
    Y = o.clone().step(1).state_vector()
    w = rng.standard_normal(X.shape) / np.maximum(np.abs(Y).max(axis=(1, 2), keepdims=True), 1e-8)
    return X, v, w


def _jv(o, X, v, h, richardson=False):
    """Central difference of the step along v; with `richardson`, the h and h/2
    quotients combined to fourth order."""
    def cd(hh):
        Y = []
        for s in (+1, -1):
            t = o.clone().set_state_vector(X + s * hh * v)
            t.step(1)
            Y.append(t.state_vector())
        return (Y[0] - Y[1]) / (2 * hh)
    return (4.0 * cd(h / 2) - cd(h)) / 3.0 if richardson else cd(h)


@pytest.mark.parametrize("warm", [0, 3])
@pytest.mark.parametrize("kw", CASES)
def test_step_transpose_full_state(kw, warm):
    """<J v, w> = <v, J^T w> for random directions over all 64 state planes."""
    p, phi = _case(**kw)
    o = oracle.Oracle(p, phi).step(warm)
    X, v, w = _dirs(o, seed=warm)
    lhs = float((_jv(o, X, v, 1e-5) * w).sum())
    a, _ = o.adjoint_step(w)
    rhs = float((v * a).sum())
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("src,dst", [("l", "f"), ("E", "g"), ("E", "f"), ("f", "E"), ("g", "l"),
                                     ("prev_qu", "l"), ("prev_phiu", "f"), ("h", "prev_phiu")])
def test_step_transpose_blocks(src, dst):
    """Single blocks of the Jacobian, where a small block would hide in the full sum."""
    p, phi = _case()
    o = oracle.Oracle(p, phi).step(3)
    X, v, w = _dirs(o, seed=7)
    a0, a1 = SP[src]
    b0, b1 = SP[dst]
    vb = np.zeros_like(v)
    vb[a0:a1] = v[a0:a1]
    wb = np.zeros_like(w)
    wb[b0:b1] = w[b0:b1]
    lhs = float((_jv(o, X, vb, 1e-3, richardson=True) * wb).sum())
    a, _ = o.adjoint_step(wb)
    rhs = float((vb * a).sum())
    assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (lhs, rhs)


@pytest.mark.parametrize("dst", ["h", "E"])
def test_potential_blocks_are_exact(dst):
    """h' and E' are affine in h (the potential iterations and E = J/(eps^ + cs2 tau_h)
    at fixed eps and q), so the difference quotient is exact and the transpose agrees
    to rounding."""
    p, phi = _case()
    o = oracle.Oracle(p, phi).step(2)
    X, v, w = _dirs(o, seed=3)
    vb = np.zeros_like(v)
    vb[SP["h"][0]:SP["h"][1]] = v[SP["h"][0]:SP["h"][1]]
    wb = np.zeros_like(w)
    wb[SP[dst][0]:SP[dst][1]] = w[SP[dst][0]:SP[dst][1]]
    lhs = float((_jv(o, X, vb, 1.0) * wb).sum())
    a, _ = o.adjoint_step(wb)
    rhs = float((vb * a).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs), (lhs, rhs)


def _set(p, name, val):
    q = dict(p)
    if name.startswith("eps"):
        e = list(q["eps"])
        e[int(name[3]) - 1] = val
        q["eps"] = tuple(e)
    elif name.startswith("sigma"):
        e = list(q["sigma"])
        e[int(name[5]) - 1] = val
        q["sigma"] = tuple(e)
    else:
        q[name] = val
    return q


def _get(p, name):
    if name.startswith("eps"):
        return p["eps"][int(name[3]) - 1]
    if name.startswith("sigma"):
        return p["sigma"][int(name[5]) - 1]
    return p[name]


@pytest.mark.parametrize("kw", CASES)
def test_parameter_and_initial_field_gradients(kw):
    """dJ/dtheta for J = <w, X^3> through the creation and three steps, every slot
    against central differences (relative step 1e-4), and dJ/dphi_init along a random
    direction."""
    p, phi = _case(**kw)
    M = 3
    o = oracle.Oracle(p, phi)
    states = []
    for _ in range(M):
        states.append(o.clone())
        o.step(1)
    X = o.state_vector()
    rng = np.random.default_rng(11)
    w = rng.standard_normal(X.shape) / np.maximum(np.abs(X).max(axis=(1, 2), keepdims=True), 1e-8)
    a = w.copy()
    dpar = np.zeros(len(oracle.ADJ_PARAMS))
    for st in reversed(states):
        a, dp = st.adjoint_step(a)
        dpar += dp
    dp0, dphi0 = oracle.adjoint_init(p, phi, a)
    dpar += dp0

    def J(q, ph=phi):
        return float((oracle.Oracle(q, ph).step(M).state_vector() * w).sum())

    scale = np.abs(dpar).max()
    for k, name in enumerate(oracle.ADJ_PARAMS):
        base = _get(p, name)
        h = 1e-4 * abs(base) if base != 0 else 1e-6
        fd = (J(_set(p, name, base + h)) - J(_set(p, name, base - h))) / (2 * h)
        assert abs(dpar[k] - fd) <= 1e-7 * abs(fd) + 1e-12 * scale, (name, dpar[k], fd)
    v = rng.standard_normal(phi.shape) * 1e-3
    fd = (J(p, phi + 1e-3 * v) - J(p, phi - 1e-3 * v)) / 2e-3
    ad = float((dphi0 * v).sum())
    assert abs(ad - fd) <= 1e-8 * abs(fd), (ad, fd)


def test_deformation_gradient():
    """The chain used by the derivative workloads: D_outer of the final populations'
    phi after 6 steps, its dD/dV_top, dD/deps3 and dD/dgamma23 by reverse mode against
    central differences of the forward runs."""
    p, phi = _case(K=8, nx=32, ny=32)
    inner, matrix = p["inner_phase"] - 1, p["matrix_phase"] - 1

    def obj(ph):
        return oracle.deformation_seed(ph, inner, matrix, "outer")

    D, g, _ = oracle.gradient(p, phi, 6, obj)

    def Df(q):
        o = oracle.Oracle(q, phi).step(6)
        return obj(oracle.phi_of_state(o.state_vector()))[0]

    assert abs(Df(p) - D) <= 1e-15
    for name in ("V_top", "eps3", "gamma23"):
        # D is ~1e-7 after 6 steps and carries ~1e-15 of rounding: wide steps,
        # combined to fourth order
        base = _get(p, name)
        h = 3e-2 * abs(base)

        def cd(hh):
            return (Df(_set(p, name, base + hh)) - Df(_set(p, name, base - hh))) / (2 * hh)

        fd = (4.0 * cd(h / 2) - cd(h)) / 3.0
        assert abs(g[name] - fd) <= 1e-5 * abs(fd), (name, g[name], fd)


def test_deformation_seed_is_the_derivative_of_D():
    """dD/dphi of the moment-based D (the objective's seed) against central
    differences along a random field."""
    rng = np.random.default_rng(5)
    phi = W.compound_droplet(32, 28, 4.0, 9.0, 4.0)
    phi[:, 10:14, 12:20] += 0.05      # break the symmetry so D != 0
    for which in ("inner", "outer"):
        D, dphi = oracle.deformation_seed(phi, 2, 0, which)
        v = rng.standard_normal(phi.shape)
        h = 1e-6
        fd = (oracle.deformation_seed(phi + h * v, 2, 0, which)[0]
              - oracle.deformation_seed(phi - h * v, 2, 0, which)[0]) / (2 * h)
        assert abs((dphi * v).sum() - fd) <= 1e-6 * abs(fd), (which, (dphi * v).sum(), fd)


def test_unsupported_configurations_are_refused():
    p, phi = _case()
    o = oracle.Oracle(dict(p, poisson_fixed_iter=0), phi)
    with pytest.raises(ValueError):
        o.adjoint_step(np.zeros((oracle.N_STATE, p["ny"], p["nx"])))
