"""The GPU reverse mode (lb3e_adjoint_step / lb3e_adjoint_init) against the oracle's
reverse mode, against the GPU tangent builds, and against central differences.

* One step backwards from the same state and the same seed: the FP64 build's
  adjoint state and parameter gradient against the oracle's to 1e-11 relative per
  plane group (the transposes are summed in another order: gathers on the GPU,
  scatters in the oracle), the FP32 build's to 1e-4 of each group's norm.  Cases:
  electrodes with moving walls, insulating walls, periodic y with an external
  field, per-phase viscosity, charge convection off, and the first step.
* The creation backwards: parameter gradient and dJ/dphi_init.
* Whole runs: D_outer after 40 steps on 64^2 by one reverse sweep (checkpoints
  every 7 steps) against the FP64 tangent builds (exact derivatives of the same
  discrete step, one direction per run) to 1e-9, and against the oracle's reverse
  mode; the checkpoint interval does not change the result.
* Configuration 5 at its stated size (256^2, 4000 steps, checkpoints every 200):
  FP64 and FP32 reverse sweeps against FP64 central differences.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

GROUPS = dict(g=(0, 9), f=(9, 36), l=(36, 45), h=(45, 54), E=(54, 56), prev=(56, 64))


def _case(bc_y=2, visc=False, cc=1, K=6, nx=24, ny=20, precision=0):
    kw = dict(nx=nx, ny=ny, bc_y=bc_y, electric=1, precision=precision, eps=(1.0, 2.0, 4.0),
              sigma=(1.0, 0.5, 0.25), eps_ref=4.0, V_top=0.02 if bc_y == 2 else 0.0, V_bottom=0.0,
              charge_convection=cc, poisson_fixed_iter=K, rho=(1.0, 1.3, 0.8), gamma12=1e-3, gamma13=1.2e-3,
              gamma23=0.8e-3)
    if bc_y:
        kw.update(u_wall_bottom=-1e-3, u_wall_top=1e-3)
    if bc_y != 2:
        kw["E_ext"] = (1e-3, 2e-3)
    if visc:
        kw["visc"] = (0.1, 0.2, 0.15)
    return W.params(**kw), W.compound_droplet(nx, ny, 3.0, 6.0, 4.0)


CASES = [dict(), dict(visc=True), dict(bc_y=1), dict(bc_y=0), dict(cc=0)]


def _seed(shape, scale, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((64,) + shape) / scale


def _group_err(a, b):
    """Per plane group: max |a - b| / max |b| (0 where b vanishes with a)."""
    out = {}
    for k, (i0, i1) in GROUPS.items():
        den = np.abs(b[i0:i1]).max()
        num = np.abs(a[i0:i1] - b[i0:i1]).max()
        out[k] = 0.0 if den == 0 and num == 0 else num / max(den, 1e-300)
    return out


@pytest.mark.parametrize("warm", [0, 3])
@pytest.mark.parametrize("kw", CASES)
def test_fp64_step_backwards_matches_the_oracle(kw, warm):
    import torch
    import paper_2608_05787_b300 as L
    p, phi = _case(**kw)
    sim = L.Sim(p, phi).step(warm)
    o = oracle.Oracle(p, phi).step(warm)
    X_gpu = sim.state_vector().cpu().numpy()
    X_orc = o.state_vector()
    assert max(_group_err(X_gpu, X_orc).values()) <= 1e-12
    scale = np.maximum(np.abs(o.clone().step(1).state_vector()).max(axis=(1, 2), keepdims=True), 1e-8)
    a = _seed((p["ny"], p["nx"]), scale, seed=warm + 1)
    a_orc, d_orc = o.adjoint_step(a)
    a_gpu, d_gpu = sim.adjoint_step(torch.from_numpy(a).cuda())
    err = _group_err(a_gpu.cpu().numpy(), a_orc)
    assert max(err.values()) <= 1e-11, err
    dscale = np.abs(d_orc).max()
    assert np.abs(d_gpu - d_orc).max() <= 1e-11 * dscale, (d_gpu, d_orc)


@pytest.mark.parametrize("kw", [dict(), dict(bc_y=0)])
def test_fp32_step_backwards_is_close_to_the_oracle(kw):
    import torch
    import paper_2608_05787_b300 as L
    p, phi = _case(precision=1, **kw)
    sim = L.Sim(p, phi).step(3)
    o = oracle.Oracle(dict(p, precision=0), phi).step(3)
    scale = np.maximum(np.abs(o.clone().step(1).state_vector()).max(axis=(1, 2), keepdims=True), 1e-8)
    a = _seed((p["ny"], p["nx"]), scale, seed=4)
    a_orc, d_orc = o.adjoint_step(a)
    a_gpu, d_gpu = sim.adjoint_step(torch.from_numpy(a).float().cuda())
    a_gpu = a_gpu.double().cpu().numpy()
    for k, (i0, i1) in GROUPS.items():
        num = np.linalg.norm(a_gpu[i0:i1] - a_orc[i0:i1])
        den = np.linalg.norm(a_orc[i0:i1])
        assert num <= 1e-4 * den + 1e-30, (k, num / den)
    assert np.abs(d_gpu - d_orc).max() <= 1e-4 * np.abs(d_orc).max(), (d_gpu, d_orc)


@pytest.mark.parametrize("precision", [2, 5])
def test_narrow_storage_step_backwards_is_close_to_the_oracle(precision):
    """FP16- and BF16-stored populations: the state vector rebuilds the full rest
    populations from their stored deviations, and the transposed step runs in FP32 on
    it; against the oracle's at the storage's own precision (1e-2 of each group's
    norm for FP16's 11 bits, BF16's 8)."""
    import torch
    import paper_2608_05787_b300 as L
    p, phi = _case(precision=precision)
    sim = L.Sim(p, phi).step(3)
    o = oracle.Oracle(dict(p, precision=0), phi).step(3)
    scale = np.maximum(np.abs(o.clone().step(1).state_vector()).max(axis=(1, 2), keepdims=True), 1e-8)
    a = _seed((p["ny"], p["nx"]), scale, seed=6)
    a_orc, d_orc = o.adjoint_step(a)
    a_gpu, d_gpu = sim.adjoint_step(torch.from_numpy(a).float().cuda())
    a_gpu = a_gpu.double().cpu().numpy()
    for k, (i0, i1) in GROUPS.items():
        num = np.linalg.norm(a_gpu[i0:i1] - a_orc[i0:i1])
        den = np.linalg.norm(a_orc[i0:i1])
        assert num <= 1e-2 * den + 1e-30, (k, num / den)
    assert np.abs(d_gpu - d_orc).max() <= 1e-2 * np.abs(d_orc).max(), (d_gpu, d_orc)


def test_fp32_creation_backwards_is_close_to_the_oracle():
    import torch
    import paper_2608_05787_b300 as L
    p, phi = _case(precision=1)
    sim = L.Sim(p, phi)
    o = oracle.Oracle(dict(p, precision=0), phi)
    scale = np.maximum(np.abs(o.state_vector()).max(axis=(1, 2), keepdims=True), 1e-8)
    a = _seed((p["ny"], p["nx"]), scale, seed=10)
    d_orc, dphi_orc = oracle.adjoint_init(p, phi, a)
    d_gpu, dphi_gpu = sim.adjoint_init(phi, torch.from_numpy(a).float().cuda())
    assert np.abs(d_gpu - d_orc).max() <= 1e-4 * np.abs(d_orc).max(), (d_gpu, d_orc)
    assert np.linalg.norm(dphi_gpu - dphi_orc) <= 1e-4 * np.linalg.norm(dphi_orc)


@pytest.mark.parametrize("kw", [dict(), dict(bc_y=0)])
def test_fp64_creation_backwards_matches_the_oracle(kw):
    import torch
    import paper_2608_05787_b300 as L
    p, phi = _case(**kw)
    sim = L.Sim(p, phi)
    o = oracle.Oracle(p, phi)
    scale = np.maximum(np.abs(o.state_vector()).max(axis=(1, 2), keepdims=True), 1e-8)
    a = _seed((p["ny"], p["nx"]), scale, seed=9)
    d_orc, dphi_orc = oracle.adjoint_init(p, phi, a)
    d_gpu, dphi_gpu = sim.adjoint_init(phi, torch.from_numpy(a).cuda())
    assert np.abs(d_gpu - d_orc).max() <= 1e-11 * np.abs(d_orc).max(), (d_gpu, d_orc)
    assert np.abs(dphi_gpu - dphi_orc).max() <= 1e-11 * np.abs(dphi_orc).max()


def _run64(precision=0):
    E0 = W.field_for_capillary(0.5, 1e-3, 1.0, 16.0)
    p = W.params(nx=64, ny=64, bc_y=2, electric=1, eps=(1.0, 2.0, 4.0), sigma=(1.0, 0.5, 0.25), eps_ref=4.0,
                 V_top=E0 * 64, u_wall_bottom=-1e-3, u_wall_top=1e-3, poisson_fixed_iter=20, precision=precision)
    return p, W.compound_droplet(64, 64, 8.0, 16.0, 4.0)


def test_reverse_sweep_matches_the_tangent_builds_and_the_oracle():
    """dD_outer/dtheta after 40 steps: the reverse sweep against the FP64 tangent
    builds (exact derivatives of the same discrete step) and the oracle's reverse
    mode; the interval of the checkpoints does not change the bits."""
    from paper_2608_05787_b300.gradients import deformation_tangents, reverse_gradient
    p, phi = _run64()
    steps = 40
    D, g, dphi = reverse_gradient(p, phi, steps, checkpoint_every=7, want_dphi=True)
    D2, g2, _ = reverse_gradient(p, phi, steps, checkpoint_every=1000)
    assert D == D2 and all(g[k] == g2[k] for k in g), (g, g2)
    Dt, gt = deformation_tangents(p, phi, steps, wrt=("V_top", "eps3", "gamma23"), precision=4)
    assert abs(D - Dt) <= 1e-15
    for name in ("V_top", "eps3", "gamma23"):
        assert abs(g[name] - gt[name]) <= 1e-9 * abs(gt[name]), (name, g[name], gt[name])
    inner, matrix = p["inner_phase"] - 1, p["matrix_phase"] - 1
    Do, go, dphio = oracle.gradient(p, phi, steps, lambda ph: oracle.deformation_seed(ph, inner, matrix, "outer"))
    assert abs(D - Do) <= 1e-13
    for name in oracle.ADJ_PARAMS:
        assert abs(g[name] - go[name]) <= 1e-9 * max(abs(go[name]), 1e-12 * max(map(abs, go.values()))), name
    assert np.abs(dphi - dphio).max() <= 1e-9 * np.abs(dphio).max()


def test_shape_objective_reverse_matches_the_tangent_build():
    from paper_2608_05787_b300.gradients import reverse_gradient, shape_objective_tangents
    p, phi = _run64()
    target = W.compound_droplet(64, 64, 9.0, 17.0, 4.0)
    J, g, _ = reverse_gradient(p, phi, 20, objective="shape", target=target, checkpoint_every=6)
    Jt, gt = shape_objective_tangents(p, phi, 20, target, wrt=("V_top", "eps3", "gamma23"), precision=4)
    assert abs(J - Jt) <= 1e-12 * abs(Jt)
    for name in ("V_top", "eps3", "gamma23"):
        assert abs(g[name] - gt[name]) <= 1e-9 * abs(gt[name]), (name, g[name], gt[name])


def test_reverse_autograd_function():
    import torch
    from paper_2608_05787_b300.gradients import deformation_reverse, reverse_gradient
    p, phi = _run64()
    E0 = torch.tensor(p["V_top"] / p["ny"], dtype=torch.float64, requires_grad=True)
    er = torch.tensor(4.0, dtype=torch.float64, requires_grad=True)
    g23 = torch.tensor(p["gamma23"], dtype=torch.float64, requires_grad=True)
    D = deformation_reverse(E0, er, g23, p, phi, 12, checkpoint_every=5)
    D.backward()
    _, g, _ = reverse_gradient(p, phi, 12, checkpoint_every=5)
    assert abs(E0.grad.item() - g["V_top"] * p["ny"]) <= 1e-12 * abs(g["V_top"] * p["ny"])
    assert abs(er.grad.item() - g["eps3"] * p["eps"][0]) <= 1e-12 * abs(g["eps3"])
    assert abs(g23.grad.item() - g["gamma23"]) <= 1e-12 * abs(g["gamma23"])


@pytest.mark.parametrize("precision", [0, 1])
def test_state_vector_form_equals_the_snapshot_form(precision):
    """lb3e_adjoint_step_x from a state vector (graph-replayed on a created stream,
    device dparams) gives the bits of lb3e_adjoint_step from the snapshot."""
    import torch
    import paper_2608_05787_b300 as L
    p, phi = _case(precision=precision)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = L.Sim(p, phi, stream=stream).step(2)
        snap = sim.save_state()
        X = sim.state_vector()
        first = sim.is_first_step
        dt = sim.compute_dtype
        a = torch.randn((64, p["ny"], p["nx"]), dtype=torch.float64, device="cuda", generator=torch.Generator(
            "cuda").manual_seed(3)).to(dt)
        out1, d1 = sim.adjoint_step(a, state=snap)
        dp = torch.zeros(11, dtype=torch.float64, device="cuda")
        out2 = torch.empty_like(a)
        for _ in range(2):  # the second call replays the captured graph
            dp.zero_()
            sim.adjoint_step_x(X, first, a, out2, dp)
        stream.synchronize()
    assert torch.equal(out1, out2)
    assert np.array_equal(d1, dp.cpu().numpy())


def test_unsupported_configurations_are_refused():
    import torch
    import paper_2608_05787_b300 as L
    p, phi = _case()
    sim = L.Sim(dict(p, poisson_fixed_iter=0), phi)
    with pytest.raises(L.LB3EError) as e:
        sim.adjoint_step(torch.zeros((64, p["ny"], p["nx"]), dtype=torch.float64, device="cuda"))
    assert e.value.code == -8


# FP32 reverse sweeps carry the FP32 rounding of the forward state over 4000 steps:
# measured 6.5e-5, 6.2e-5, 6.2e-5 (the FP32 tangents: 4.7e-4, 4.7e-4, 5.5e-4)
FP32_TOL_4000 = {"V_top": 1e-4, "eps3": 1e-4, "gamma23": 1e-4}  # the stated 1e-4


@pytest.mark.slow
def test_config5_stated_size_reverse_matches_fp64_central_differences():
    """Configuration 5 as stated: 256^2, walls at -/+1e-3 plus electrodes, 4000 steps,
    checkpoints every 200 steps, the potential iterated 16 times a step.  The three
    derivatives of D_outer by FP64 and FP32 reverse sweeps against FP64 central
    differences (relative step 1e-4) of GPU runs."""
    import paper_2608_05787_b300 as L
    from paper_2608_05787_b300.gradients import reverse_gradient
    cfg = W.config_adjoint(n=256, precision=0)
    p = dict(cfg["params"], poisson_fixed_iter=16)
    phi, steps = cfg["phi"], cfg["steps"]
    D64, g64, _ = reverse_gradient(p, phi, steps, checkpoint_every=200)
    D32, g32, _ = reverse_gradient(dict(p, precision=1), phi, steps, checkpoint_every=200)
    base = {"V_top": p["V_top"], "eps3": p["eps"][2], "gamma23": p["gamma23"]}
    for name in ("V_top", "eps3", "gamma23"):
        h = 1e-4 * base[name]
        vals = []
        for sg in (+1, -1):
            q = dict(p)
            if name == "eps3":
                q["eps"] = (p["eps"][0], p["eps"][1], p["eps"][2] + sg * h)
            else:
                q[name] = p[name] + sg * h
            sim = L.Sim(q, phi)
            sim.step(steps)
            vals.append(sim.deformation()[0][1])
        fd = (vals[0] - vals[1]) / (2 * h)
        e64, e32 = abs(g64[name] - fd) / abs(fd), abs(g32[name] - fd) / abs(fd)
        print(f"{name}: fd {fd:.6e}  fp64 reverse {g64[name]:.6e} ({e64:.1e})  fp32 reverse {g32[name]:.6e} ({e32:.1e})")
        assert e64 <= 1e-4, (name, e64)
        assert e32 <= FP32_TOL_4000[name], (name, e32)
