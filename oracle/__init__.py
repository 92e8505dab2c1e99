"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path never does: it shares no code
with the oracle, and the oracle shares none with it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "lb3e_oracle.c"
_SRC3 = _HERE / "lb3e_oracle3d.c"
_LIB = _HERE / "liblb3e_oracle.so"

FIELDS = dict(phi1=0, phi2=1, phi3=2, ux=3, uy=4, p=5, q=6, psi=7, ex=8, ey=9,
              mu1=10, mu2=11, mu3=12, phinow1=13, phinow2=14, phinow3=15, qtilde=16, n1=17, n2=18)
SETS = dict(g=0, f1=1, f2=2, f3=3, l=4, h=5, n1=6, n2=7)
POP_BASE = 100
OBS_KEYS = ("mass1", "mass2", "mass3", "charge", "F_phi", "F_E", "F_u", "F_q",
            "max_sum_dev", "D_inner", "D_outer", "nonfinite", "step", "poisson_iters",
            "poisson_residual")


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc_y", C.c_int32), ("electric", C.c_int32),
        ("rho", C.c_double * 3), ("visc", C.c_double * 3), ("tau_g", C.c_double),
        ("gamma12", C.c_double), ("gamma13", C.c_double), ("gamma23", C.c_double),
        ("width_D", C.c_double), ("tau_f", C.c_double),
        ("eps", C.c_double * 3), ("sigma", C.c_double * 3), ("eps_ref", C.c_double),
        ("alpha", C.c_double), ("V_bottom", C.c_double), ("V_top", C.c_double),
        ("E_ext", C.c_double * 2), ("u_wall_bottom", C.c_double), ("u_wall_top", C.c_double),
        ("charge_convection", C.c_int32), ("inner_phase", C.c_int32), ("matrix_phase", C.c_int32),
        ("poisson_tol", C.c_double), ("poisson_max_iter", C.c_int32),
        ("poisson_check_every", C.c_int32), ("poisson_fixed_iter", C.c_int32),
        ("potential_solver", C.c_int32),
        ("debye_kappa2", C.c_double),
        ("ions", C.c_int32), ("ion_D", C.c_double * 2), ("ion_z", C.c_double * 2),
        ("ion_beta", C.c_double), ("ion_charge", C.c_double),
    ]


FIELDS3 = dict(phi1=0, phi2=1, phi3=2, ux=3, uy=4, uz=5, p=6, q=7, psi=8, ex=9, ey=10, ez=11,
               mu1=12, mu2=13, mu3=14, phinow1=15, phinow2=16, phinow3=17, qtilde=18)
OBS3_KEYS = ("mass1", "mass2", "mass3", "charge", "max_sum_dev", "D_inner", "D_outer", "nonfinite", "step",
             "poisson_iters", "poisson_residual")


class _Params3(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("bc", C.c_int32), ("electric", C.c_int32),
        ("rho", C.c_double * 3), ("visc", C.c_double * 3), ("tau_g", C.c_double),
        ("gamma12", C.c_double), ("gamma13", C.c_double), ("gamma23", C.c_double),
        ("width_D", C.c_double), ("tau_f", C.c_double),
        ("eps", C.c_double * 3), ("sigma", C.c_double * 3), ("eps_ref", C.c_double), ("alpha", C.c_double),
        ("V_bottom", C.c_double), ("V_top", C.c_double), ("E_ext", C.c_double * 2),
        ("u_wall_bottom", C.c_double), ("u_wall_top", C.c_double),
        ("charge_convection", C.c_int32), ("inner_phase", C.c_int32), ("matrix_phase", C.c_int32),
        ("poisson_tol", C.c_double), ("poisson_max_iter", C.c_int32),
        ("poisson_check_every", C.c_int32), ("poisson_fixed_iter", C.c_int32),
    ]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP over cells)."""
    newest = max(_SRC.stat().st_mtime, _SRC3.stat().st_mtime)
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= newest:
        return _LIB
    tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", str(tmp), str(_SRC), str(_SRC3), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(str(build()))
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Params), dp, dp, dp, dp, C.POINTER(C.c_int)]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_field.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_observables.argtypes = [C.c_void_p, dp]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_solve_potential.argtypes = [C.c_void_p, dp, C.c_double, C.c_int, C.c_int, C.c_int, dp,
                                          C.POINTER(C.c_int)]
        L.orc_last_poisson.argtypes = [C.c_void_p, C.POINTER(C.c_int), dp, C.POINTER(C.c_int)]
        L.orc_stencil.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
        L.orc_lattice.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), dp, C.POINTER(C.c_int)]
        L.orc_set_ions.argtypes = [C.c_void_p, dp]
        L.orc3_create.restype = C.c_void_p
        L.orc3_create.argtypes = [C.POINTER(_Params3), dp, dp, dp, C.POINTER(C.c_int)]
        L.orc3_step.argtypes = [C.c_void_p, C.c_int]
        L.orc3_get_field.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc3_observables.argtypes = [C.c_void_p, dp]
        L.orc3_destroy.argtypes = [C.c_void_p]
        L.orc3_stencil.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp]
        L.orc3_lattice.argtypes = [C.POINTER(C.c_int)] * 3 + [dp, C.POINTER(C.c_int)]
        L.orc3_step_count.restype = C.c_int64
        L.orc3_step_count.argtypes = [C.c_void_p]
        L.orc_step_count.restype = C.c_int64
        L.orc_step_count.argtypes = [C.c_void_p]
        L.orc_perturb.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_uint64]
        L.orc_round_storage.argtypes = [C.c_void_p, C.c_int]
        L.orc_clone.restype = C.c_void_p
        L.orc_clone.argtypes = [C.c_void_p]
        L.orc_get_state_vector.argtypes = [C.c_void_p, dp]
        L.orc_set_state_vector.argtypes = [C.c_void_p, dp]
        L.orc_adjoint_step.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_adjoint_init.argtypes = [C.POINTER(_Params), dp, dp, dp, dp, dp, dp]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# reverse mode: planes of the state vector X = (g, f, l, h, E, (phi_i u)^{n-1}, (q u)^{n-1})
# and the parameter slots of dJ/dtheta
STATE_PLANES = dict(g=(0, 9), f=(9, 36), l=(36, 45), h=(45, 54), E=(54, 56), prev_phiu=(56, 62),
                    prev_qu=(62, 64))
N_STATE = 64
ADJ_PARAMS = ("V_bottom", "V_top", "eps1", "eps2", "eps3", "sigma1", "sigma2", "sigma3",
              "gamma12", "gamma13", "gamma23")


def make_params(p: dict) -> _Params:
    s = _Params()
    for name, ctype in _Params._fields_:
        v = p[name if name != "width_D" else "width_D"]
        if hasattr(ctype, "_length_"):
            getattr(s, name)[:] = list(v)
        else:
            setattr(s, name, v)
    return s


class Oracle:
    """FP64 reference simulation (one state per instance)."""

    def __init__(self, params: dict, phi, u=None, q=None, noise=None, ions=None):
        """`ions`: initial concentrations (2, ny, nx) of the Nernst-Planck species, for
        parameters with `ions` = 1."""
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self._keep = [_c64(phi), _c64(u), _c64(q), _c64(noise)]
        st = C.c_int(0)
        self._p = make_params(params)
        h = lib().orc_create(C.byref(self._p), *(_ptr(a) for a in self._keep), C.byref(st))
        if not h:
            raise ValueError(f"oracle rejected parameters (status {st.value})")
        self._h = C.c_void_p(h)
        if ions is not None:
            n = _c64(ions)
            if lib().orc_set_ions(self._h, _ptr(n)) != 0:
                raise ValueError("ion concentrations need parameters with ions = 1")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))
        return self

    @property
    def steps_done(self) -> int:
        return int(lib().orc_step_count(self._h))

    def field(self, name: str) -> np.ndarray:
        out = np.empty((self.ny, self.nx))
        if lib().orc_get_field(self._h, FIELDS[name], _ptr(out)) != 0:
            raise KeyError(name)
        return out

    def pop(self, set_name: str, j: int) -> np.ndarray:
        out = np.empty((self.ny, self.nx))
        lib().orc_get_field(self._h, POP_BASE + 9 * SETS[set_name] + j, _ptr(out))
        return out

    def observables(self) -> dict:
        out = np.zeros(16)
        lib().orc_observables(self._h, _ptr(out))
        return dict(zip(OBS_KEYS, out.tolist()))

    def solve_potential(self, q=None, tol=1e-8, max_iter=100000, fixed=0, check=10):
        qa = _c64(q)
        res = C.c_double(0)
        conv = C.c_int(0)
        it = lib().orc_solve_potential(self._h, _ptr(qa), tol, max_iter, fixed, check, C.byref(res),
                                       C.byref(conv))
        return it, res.value, conv.value == 1

    def perturb(self, rel: float, floor_abs: float = 0.0, field_rel: float = 0.0, seed: int = 0):
        """Test facility: perturb the populations (g, f, l) as storing them in a format
        of relative precision `rel` (and spacing `floor_abs` near zero) would; the
        phase rest populations by their deviation from phi_i, and phi_i itself as a
        field of relative precision `field_rel`.  Deterministic in seed."""
        lib().orc_perturb(self._h, float(rel), float(floor_abs), float(field_rel), int(seed))
        return self

    def round_storage(self, fmt: str):
        """Test facility: round the stored populations to a storage format ('fp32',
        'fp16' or 'bf16') as the GPU's builds store them (phase rest populations by
        their deviation from phi_i, phi_i itself an FP32 field)."""
        lib().orc_round_storage(self._h, {"fp32": 1, "fp16": 2, "bf16": 3}[fmt])
        return self

    def clone(self) -> "Oracle":
        """An independent copy of the current state."""
        o = Oracle.__new__(Oracle)
        o.params, o.nx, o.ny, o._keep, o._p = dict(self.params), self.nx, self.ny, self._keep, self._p
        o._h = C.c_void_p(lib().orc_clone(self._h))
        return o

    def state_vector(self) -> np.ndarray:
        """The state X as (64, ny, nx) planes (STATE_PLANES)."""
        out = np.empty((N_STATE, self.ny, self.nx))
        lib().orc_get_state_vector(self._h, _ptr(out))
        return out

    def set_state_vector(self, x) -> "Oracle":
        xa = _c64(x)
        assert xa.shape == (N_STATE, self.ny, self.nx)
        lib().orc_set_state_vector(self._h, _ptr(xa))
        return self

    def adjoint_step(self, a_in) -> tuple[np.ndarray, np.ndarray]:
        """For the step from this state: (dX'/dX)^T a_in and (dX'/dtheta)^T a_in (the
        ADJ_PARAMS slots).  The state is left unchanged."""
        a = _c64(a_in)
        assert a.shape == (N_STATE, self.ny, self.nx)
        out = np.empty_like(a)
        dpar = np.zeros(len(ADJ_PARAMS))
        if lib().orc_adjoint_step(self._h, _ptr(a), _ptr(out), _ptr(dpar)) != 0:
            raise ValueError("no reverse mode for this configuration (ions, Debye-Hueckel closure, FD "
                             "potential or a residual-controlled potential)")
        return out, dpar

    def last_poisson(self):
        it, res, conv = C.c_int(0), C.c_double(0), C.c_int(0)
        lib().orc_last_poisson(self._h, C.byref(it), C.byref(res), C.byref(conv))
        return it.value, res.value, conv.value == 1

    def last_poisson_stalled(self) -> bool:
        """The last solve stopped on a stalled residual (not converged)."""
        it, res, conv = C.c_int(0), C.c_double(0), C.c_int(0)
        lib().orc_last_poisson(self._h, C.byref(it), C.byref(res), C.byref(conv))
        return conv.value == -1


def adjoint_init(params: dict, phi, a_in, u=None, q=None) -> tuple[np.ndarray, np.ndarray]:
    """Transpose of the state's creation from phi (u, q held fixed, noise additive):
    (dX0/dtheta)^T a_in over ADJ_PARAMS and (dX0/dphi)^T a_in as (3, ny, nx)."""
    ph, ua, qa, a = _c64(phi), _c64(u), _c64(q), _c64(a_in)
    pr = make_params(params)
    dpar = np.zeros(len(ADJ_PARAMS))
    dphi = np.zeros_like(ph)
    if lib().orc_adjoint_init(C.byref(pr), _ptr(ph), _ptr(ua), _ptr(qa), _ptr(a), _ptr(dpar), _ptr(dphi)) != 0:
        raise ValueError("no reverse mode for this configuration")
    return dpar, dphi


def deformation_seed(phi_of_state: np.ndarray, inner: int, matrix: int, which: str = "outer"):
    """D of the second moments of chi (chi = phi_inner, or 1 - phi_matrix for the
    outer drop) and dD/dphi as (3, ny, nx)."""
    ny, nx = phi_of_state.shape[1:]
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    chi = phi_of_state[inner] if which == "inner" else 1.0 - phi_of_state[matrix]
    A = chi.sum()
    xc, yc = (chi * x).sum() / A, (chi * y).sum() / A
    Ixx, Iyy = (chi * x * x).sum() / A - xc ** 2, (chi * y * y).sum() / A - yc ** 2
    a, b = 2.0 * np.sqrt(Iyy), 2.0 * np.sqrt(Ixx)
    D = (a - b) / (a + b)
    # chain rule through the moments: dI_xx/dchi = (x^2 - m3/A)/A - 2 xc (x - xc)/A
    dIxx = (x * x - (chi * x * x).sum() / A) / A - 2.0 * xc * (x - xc) / A
    dIyy = (y * y - (chi * y * y).sum() / A) / A - 2.0 * yc * (y - yc) / A
    dchi = 2.0 * (b * dIyy / np.sqrt(Iyy) - a * dIxx / np.sqrt(Ixx)) / (a + b) ** 2
    dphi = np.zeros_like(phi_of_state)
    if which == "inner":
        dphi[inner] = dchi
    else:
        dphi[matrix] = -dchi
    return D, dphi


def phi_of_state(x: np.ndarray) -> np.ndarray:
    """phi_i = sum_j f^i_j of a state vector."""
    f0, f1 = STATE_PLANES["f"]
    return x[f0:f1].reshape(3, 9, *x.shape[1:]).sum(axis=1)


def seed_from_phi(dphi: np.ndarray) -> np.ndarray:
    """The state-vector adjoint of an objective of phi = sum_j f^i_j."""
    ny, nx = dphi.shape[1:]
    a = np.zeros((N_STATE, ny, nx))
    f0 = STATE_PLANES["f"][0]
    for i in range(3):
        a[f0 + 9 * i:f0 + 9 * i + 9] = dphi[i]
    return a


def gradient(params: dict, phi, steps: int, objective, u=None, q=None):
    """Reverse-mode gradient of objective(phi of the final populations) after `steps`
    steps from the state created from phi.  `objective(phi) -> (J, dJ/dphi)`.
    Returns J, {parameter: dJ/dparameter}, dJ/dphi_init.  Every state is kept (small
    lattices only)."""
    o = Oracle(params, phi, u=u, q=q)
    states = []
    for _ in range(steps):
        states.append(o.clone())
        o.step(1)
    J, dphi = objective(phi_of_state(o.state_vector()))
    a = seed_from_phi(dphi)
    dpar = np.zeros(len(ADJ_PARAMS))
    for st in reversed(states):
        a, dp = st.adjoint_step(a)
        dpar += dp
    dp0, dphi0 = adjoint_init(params, phi, a, u=u, q=q)
    dpar += dp0
    return J, dict(zip(ADJ_PARAMS, dpar.tolist())), dphi0


def stencil(chi: np.ndarray, bc_y: int):
    chi = _c64(chi)
    ny, nx = chi.shape
    gx, gy, lap = np.empty_like(chi), np.empty_like(chi), np.empty_like(chi)
    lib().orc_stencil(nx, ny, bc_y, _ptr(chi), _ptr(gx), _ptr(gy), _ptr(lap))
    return gx, gy, lap


def lattice():
    cx, cy, opp = (C.c_int * 9)(), (C.c_int * 9)(), (C.c_int * 9)()
    w = (C.c_double * 9)()
    lib().orc_lattice(cx, cy, w, opp)
    return np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(opp[:])


class Oracle3D:
    """FP64 reference of the D3Q15 step.  ``params`` uses the two-dimensional keys
    plus ``nz``; ``bc_y`` gives the boundary of the z walls (the wall normal is z in
    three dimensions, x and y periodic), ``E_ext`` = (along x, along z).  Arrays are
    [.., nz, ny, nx]."""

    def __init__(self, params: dict, phi, u=None, q=None):
        self.params = dict(params)
        self.nx, self.ny, self.nz = int(params["nx"]), int(params["ny"]), int(params["nz"])
        self._keep = [_c64(phi), _c64(u), _c64(q)]
        pr = _Params3()
        for name, ctype in _Params3._fields_:
            v = params["bc_y"] if name == "bc" else params[name]
            if hasattr(ctype, "_length_"):
                getattr(pr, name)[:] = list(v)
            else:
                setattr(pr, name, v)
        self._p = pr
        st = C.c_int(0)
        h = lib().orc3_create(C.byref(pr), *(_ptr(a) for a in self._keep), C.byref(st))
        if not h:
            raise ValueError(f"oracle rejected parameters (status {st.value})")
        self._h = C.c_void_p(h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc3_destroy(self._h)
            self._h = None

    def step(self, n: int = 1):
        lib().orc3_step(self._h, int(n))
        return self

    @property
    def steps_done(self) -> int:
        return int(lib().orc3_step_count(self._h))

    def field(self, name: str) -> np.ndarray:
        out = np.empty((self.nz, self.ny, self.nx))
        if lib().orc3_get_field(self._h, FIELDS3[name], _ptr(out)) != 0:
            raise KeyError(name)
        return out

    def pop(self, set_name: str, j: int) -> np.ndarray:
        out = np.empty((self.nz, self.ny, self.nx))
        lib().orc3_get_field(self._h, POP_BASE + 15 * SETS[set_name] + j, _ptr(out))
        return out

    def observables(self) -> dict:
        out = np.zeros(11)
        lib().orc3_observables(self._h, _ptr(out))
        return dict(zip(OBS3_KEYS, out.tolist()))


def stencil3(chi: np.ndarray, bc: int):
    chi = _c64(chi)
    nz, ny, nx = chi.shape
    g, lap = np.empty((3,) + chi.shape), np.empty_like(chi)
    lib().orc3_stencil(nx, ny, nz, bc, _ptr(chi), _ptr(g), _ptr(lap))
    return g, lap


def lattice3():
    cx, cy, cz, opp = (C.c_int * 15)(), (C.c_int * 15)(), (C.c_int * 15)(), (C.c_int * 15)()
    w = (C.c_double * 15)()
    lib().orc3_lattice(cx, cy, cz, w, opp)
    return np.array(cx[:]), np.array(cy[:]), np.array(cz[:]), np.array(w[:]), np.array(opp[:])
