"""Python binding of liblb3e: the B300 three-phase EHD lattice Boltzmann step.

Argument marshalling only: every step of the method runs in the CUDA kernels of
``csrc/`` behind the C ABI of ``include/lb3e.h``.  PyTorch supplies the device
workspace and the stream.  There is no CPU fallback: if the library or a CUDA
device is missing, constructing a simulation raises.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
# the in-tree build; LB3E_LIBRARY may point at another build of the same sources
LIB_PATH = Path(os.environ.get("LB3E_LIBRARY", _HERE / "liblb3e.so"))

FIELDS = dict(phi1=0, phi2=1, phi3=2, ux=3, uy=4, p=5, q=6, psi=7, ex=8, ey=9,
              mu1=10, mu2=11, mu3=12, phinow1=13, phinow2=14, phinow3=15, qtilde=16, n1=17, n2=18,
              uz=19, ez=20)
SETS = dict(g=0, f1=1, f2=2, f3=3, l=4, h=5, n1=6, n2=7)
POP_BASE = 100
PRECISIONS = {0: "f64", 1: "f32", 2: "f32-compute/f16-store", 3: "f32 + 3 tangents", 4: "f64 + 1 tangent",
              5: "f32-compute/bf16-store"}
TANGENT = 1000
TANGENT_PARAMS = dict(V_top=0, eps1=1, eps2=2, eps3=3, gamma12=4, gamma13=5, gamma23=6)
# reverse mode: the parameter slots of dJ/dtheta and the planes of the state vector
ADJ_PARAMS = ("V_bottom", "V_top", "eps1", "eps2", "eps3", "sigma1", "sigma2", "sigma3",
              "gamma12", "gamma13", "gamma23")
N_STATE = 64
STATE_PLANES = dict(g=(0, 9), f=(9, 36), l=(36, 45), h=(45, 54), E=(54, 56), prev_phiu=(56, 62),
                    prev_qu=(62, 64))

KERNEL_CLASSES = ("moments", "prologue", "poisson", "reduce", "fields", "fused", "other", "ions", "anchor",
                  "coarse")


class Params(C.Structure):
    """Mirror of ``lb3e_params`` (include/lb3e.h)."""
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc_y", C.c_int32), ("electric", C.c_int32),
        ("precision", C.c_int32), ("_pad0", C.c_int32),
        ("rho", C.c_double * 3), ("visc", C.c_double * 3), ("tau_g", C.c_double),
        ("gamma12", C.c_double), ("gamma13", C.c_double), ("gamma23", C.c_double),
        ("width_D", C.c_double), ("tau_f", C.c_double),
        ("eps", C.c_double * 3), ("sigma", C.c_double * 3), ("eps_ref", C.c_double),
        ("alpha", C.c_double), ("V_bottom", C.c_double), ("V_top", C.c_double),
        ("E_ext", C.c_double * 2), ("u_wall_bottom", C.c_double), ("u_wall_top", C.c_double),
        ("charge_convection", C.c_int32), ("inner_phase", C.c_int32), ("matrix_phase", C.c_int32),
        ("_pad1", C.c_int32),
        ("poisson_tol", C.c_double), ("poisson_max_iter", C.c_int32),
        ("poisson_check_every", C.c_int32), ("poisson_fixed_iter", C.c_int32), ("_pad2", C.c_int32),
        ("tangent_param", C.c_int32 * 3), ("potential_solver", C.c_int32),
        ("ions", C.c_int32), ("_pad3", C.c_int32), ("ion_D", C.c_double * 2), ("ion_z", C.c_double * 2),
        ("ion_beta", C.c_double), ("ion_charge", C.c_double), ("nz", C.c_int32), ("_pad4", C.c_int32),
    ]
    # Nernst-Planck ion transport and the three-dimensional lattice are off unless
    # the dict asks for them
    _DEFAULTS = dict(ions=0, ion_D=(0.0, 0.0), ion_z=(1.0, -1.0), ion_beta=1.0, ion_charge=0.0, nz=0)

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        if d.get("debye_kappa2", 0.0):
            # a validation closure of the test oracle (electro-osmotic channel), not
            # part of the method this library implements
            raise ValueError("debye_kappa2 is an oracle-only validation closure; lb3e does not implement it")
        s = cls()
        for name, ctype in cls._fields_:
            if name.startswith("_pad"):
                continue
            v = d[name] if name in d or name not in cls._DEFAULTS else cls._DEFAULTS[name]
            if hasattr(ctype, "_length_"):
                conv = int if ctype._type_ is C.c_int32 else float
                getattr(s, name)[:] = [conv(a) for a in v]
            else:
                setattr(s, name, v)
        return s


class Observables(C.Structure):
    """Mirror of ``lb3e_observables_t``."""
    _fields_ = [
        ("mass", C.c_double * 3), ("charge", C.c_double), ("free_energy", C.c_double * 4),
        ("max_sum_dev", C.c_double), ("D_inner", C.c_double), ("D_outer", C.c_double),
        ("poisson_residual", C.c_double), ("nonfinite", C.c_int64), ("step", C.c_int64),
        ("poisson_iters", C.c_int32), ("poisson_converged", C.c_int32),
    ]

    def as_dict(self) -> dict:
        fe = list(self.free_energy)
        return dict(mass1=self.mass[0], mass2=self.mass[1], mass3=self.mass[2], charge=self.charge,
                    F_phi=fe[0], F_E=fe[1], F_u=fe[2], F_q=fe[3], max_sum_dev=self.max_sum_dev,
                    D_inner=self.D_inner, D_outer=self.D_outer, nonfinite=self.nonfinite,
                    step=self.step, poisson_iters=self.poisson_iters,
                    poisson_residual=self.poisson_residual,
                    poisson_converged=self.poisson_converged == 1,
                    poisson_stalled=self.poisson_converged == -1)


class LB3EError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {status_string(code)} ({code})")
        self.code = code


_lib = None


def lib() -> C.CDLL:
    """Load liblb3e.so (built in-tree by ``build.py``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2608_05787_b300.build`")
        L = C.CDLL(str(LIB_PATH))
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.lb3e_workspace_bytes.argtypes = [C.POINTER(Params), C.POINTER(C.c_size_t)]
        L.lb3e_init.argtypes = [C.POINTER(Params), vp, C.c_size_t, vp, vp, vp, vp, vp, C.POINTER(vp)]
        L.lb3e_step.argtypes = [vp, C.c_int32]
        L.lb3e_solve_potential.argtypes = [vp, vp, C.c_double, C.c_int32, C.c_int32,
                                           C.POINTER(C.c_int32), dp]
        L.lb3e_observables.argtypes = [vp, C.POINTER(Observables)]
        L.lb3e_get_field.argtypes = [vp, C.c_int32, vp]
        L.lb3e_state_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.lb3e_save_state.argtypes = [vp, vp]
        L.lb3e_load_state.argtypes = [vp, vp]
        L.lb3e_launch_count.restype = C.c_int64
        L.lb3e_launch_count.argtypes = [vp]
        L.lb3e_potential_iterations.restype = C.c_int64
        L.lb3e_potential_iterations.argtypes = [vp]
        L.lb3e_set_timing.argtypes = [vp, C.c_int32]
        L.lb3e_set_potential_chunk.argtypes = [vp, C.c_int32]
        L.lb3e_set_fused_tile.argtypes = [vp, C.c_int32]
        L.lb3e_set_staging.argtypes = [vp, C.c_int32]
        L.lb3e_set_ions.argtypes = [vp, vp]
        L.lb3e_potential_fd_residual.argtypes = [vp, dp]
        L.lb3e_deformation.argtypes = [vp, dp, dp]
        L.lb3e_shape_objective.argtypes = [vp, vp, dp, dp]
        L.lb3e_adjoint_workspace_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.lb3e_state_vector.argtypes = [vp, vp]
        L.lb3e_adjoint_step.argtypes = [vp, vp, vp, vp, dp, vp, C.c_size_t]
        L.lb3e_adjoint_init.argtypes = [vp, vp, vp, dp, vp, vp, C.c_size_t]
        L.lb3e_adjoint_step_x.argtypes = [vp, vp, C.c_int32, vp, vp, vp, vp, C.c_size_t]
        L.lb3e_is_first_step.argtypes = [vp, C.POINTER(C.c_int32)]
        L.lb3e_deformation_seed.argtypes = [vp, C.c_int32, dp, vp]
        L.lb3e_shape_seed.argtypes = [vp, vp, dp, vp]
        L.lb3e_potential_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), dp]
        L.lb3e_kernel_times.argtypes = [vp, dp, C.POINTER(C.c_int64)]
        L.lb3e_observables_noalloc.argtypes = [C.POINTER(Params), vp, vp, vp, vp, vp, C.POINTER(Observables)]
        L.lb3e_batch_workspace_bytes.argtypes = [C.POINTER(Params), C.c_int32, C.POINTER(C.c_size_t)]
        L.lb3e_batch_create.argtypes = [C.POINTER(Params), C.c_int32, C.POINTER(vp), vp, C.c_size_t, vp,
                                        C.POINTER(vp)]
        L.lb3e_batch_run.argtypes = [vp, C.c_int32]
        L.lb3e_batch_observables.argtypes = [vp, C.POINTER(Observables)]
        L.lb3e_batch_get_field.argtypes = [vp, C.c_int32, C.c_int32, vp]
        L.lb3e_batch_set_potential_chunk.argtypes = [vp, C.c_int32]
        L.lb3e_batch_set_fused_tile.argtypes = [vp, C.c_int32]
        L.lb3e_batch_launch_count.restype = C.c_int64
        L.lb3e_batch_launch_count.argtypes = [vp]
        L.lb3e_batch_destroy.argtypes = [vp]
        L.lb3e_batch_destroy.restype = None
        L.lb3e_destroy.argtypes = [vp]
        L.lb3e_destroy.restype = None
        L.lb3e_status_string.restype = C.c_char_p
        L.lb3e_status_string.argtypes = [C.c_int]
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().lb3e_status_string(code).decode()


def _check(fn: str, code: int):
    if code != 0:
        raise LB3EError(fn, code)


def workspace_bytes(params: dict) -> int:
    n = C.c_size_t(0)
    _check("lb3e_workspace_bytes", lib().lb3e_workspace_bytes(C.byref(Params.from_dict(params)), C.byref(n)))
    return n.value


def _addr(a):
    """Address of a host numpy array or a CUDA torch tensor (float64, contiguous)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a.ctypes.data, a
    import torch
    if isinstance(a, torch.Tensor):
        a = a.contiguous().to(torch.float64)
        return a.data_ptr(), a
    raise TypeError(type(a))


def observables_noalloc(params: dict, phi, q, E, u, stream=None) -> dict:
    """The observables reductions on caller-provided FP64 CUDA tensors, for callers
    that cannot allocate device memory: the scratch is a fixed array inside the
    library (lattices up to 2048 x 2048).  phi [3,ny,nx], q [ny,nx], E and u
    [2,ny,nx], all contiguous float64 CUDA tensors on one device, with nx and ny
    those of ``params`` (checked here: the C entry point cannot see the sizes)."""
    import torch
    ny, nx = int(params["ny"]), int(params["nx"])
    shapes = ((phi, (3, ny, nx)), (q, (ny, nx)), (E, (2, ny, nx)), (u, (2, ny, nx)))
    for t, shape in shapes:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError("lb3e_observables_noalloc takes contiguous float64 CUDA tensors")
        if tuple(t.shape) != shape:
            raise ValueError(f"lb3e_observables_noalloc: a field of shape {tuple(t.shape)}, expected {shape}")
        if t.device != phi.device:
            raise ValueError("lb3e_observables_noalloc: all fields must be on one device")
    # the library launches on the current device: make it the fields' device, and
    # take that device's current stream unless one is given
    with torch.cuda.device(phi.device):
        st = stream if stream is not None else torch.cuda.current_stream(phi.device)
        if st.device != phi.device:
            raise ValueError("lb3e_observables_noalloc: the stream is on another device than the fields")
        o = Observables()
        _check("lb3e_observables_noalloc",
               lib().lb3e_observables_noalloc(C.byref(Params.from_dict(params)), phi.data_ptr(), q.data_ptr(),
                                              E.data_ptr(), u.data_ptr(), st.cuda_stream, C.byref(o)))
    return o.as_dict()


class Sim:
    """One lattice, stepped on the GPU through the C ABI.

    ``params`` is a plain dict with the keys of ``lb3e_params``; initial arrays
    may be host numpy arrays or CUDA tensors (float64, ``[.., ny, nx]``).
    """

    def __init__(self, params: dict, phi, u=None, q=None, noise=None, stream=None, device=None, ions=None,
                 workspace=None):
        """``ions``: initial concentrations [2, ny, nx] of the Nernst-Planck species
        (parameters with ``ions`` = 1), set through ``lb3e_set_ions``.  ``workspace``:
        a caller-allocated uint8 CUDA tensor of at least ``workspace_bytes(params)``
        bytes to run in (allocated here if None)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lb3e needs a CUDA device (there is no CPU fallback)")
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self.nz = int(params.get("nz", 0))
        # arrays are [.., ny, nx], or [.., nz, ny, nx] on three-dimensional (D3Q15) lattices
        self.shape = (self.nz, self.ny, self.nx) if self.nz >= 2 else (self.ny, self.nx)
        self.q_dirs = 15 if self.nz >= 2 else 9
        self.device = torch.device(device or "cuda")
        self._p = Params.from_dict(self.params)
        nbytes = workspace_bytes(self.params)
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        elif not (isinstance(workspace, torch.Tensor) and workspace.is_cuda and workspace.dtype == torch.uint8
                  and workspace.numel() >= nbytes):
            raise ValueError(f"workspace: a uint8 CUDA tensor of at least {nbytes} bytes")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        keep = [_addr(a) for a in (phi, u, q, noise)]
        h = C.c_void_p(None)
        _check("lb3e_init", lib().lb3e_init(C.byref(self._p), self.workspace.data_ptr(), nbytes,
                                            *(k[0] for k in keep), self.stream.cuda_stream, C.byref(h)))
        self._h = h
        if ions is not None:
            addr, _keep = _addr(ions)
            _check("lb3e_set_ions", lib().lb3e_set_ions(self._h, addr))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lb3e_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> "Sim":
        _check("lb3e_step", lib().lb3e_step(self._h, int(n)))
        return self

    def observables(self) -> dict:
        o = Observables()
        _check("lb3e_observables", lib().lb3e_observables(self._h, C.byref(o)))
        return o.as_dict()

    def field(self, name: str, out=None, tangent: int = 0):
        """Field as a host float64 array (or written into ``out``, a CUDA tensor).
        In the tangent builds, ``tangent=k`` (1..3) gives its derivative along
        direction k."""
        fid = FIELDS[name] + TANGENT * int(tangent)
        return self._get(fid, out)

    def pop(self, set_name: str, j: int, out=None):
        return self._get(POP_BASE + self.q_dirs * SETS[set_name] + j, out)

    def _get(self, fid: int, out):
        if out is None:
            arr = np.empty(self.shape)
            _check("lb3e_get_field", lib().lb3e_get_field(self._h, fid, arr.ctypes.data))
            return arr
        _check("lb3e_get_field", lib().lb3e_get_field(self._h, fid, out.data_ptr()))
        return out

    def solve_potential(self, q=None, tol=1e-8, max_iter=100000, check=10):
        addr, _keep = _addr(q)
        it, res = C.c_int32(0), C.c_double(0)
        rc = lib().lb3e_solve_potential(self._h, addr, tol, max_iter, check, C.byref(it), C.byref(res))
        if rc not in (0, -4):
            _check("lb3e_solve_potential", rc)
        return it.value, res.value, rc == 0

    def potential_stats(self) -> dict:
        """Potential solves since the previous call: count, how many ended above the
        tolerance, the largest final residual (then cleared)."""
        n, bad, mx = C.c_int64(0), C.c_int64(0), C.c_double(0)
        _check("lb3e_potential_stats", lib().lb3e_potential_stats(self._h, C.byref(n), C.byref(bad), C.byref(mx)))
        return dict(solves=n.value, not_converged=bad.value, max_residual=mx.value)

    def deformation(self):
        """(D_inner, D_outer) of the current populations' phases and, in the tangent
        builds, ((dD_inner/dtheta_t), (dD_outer/dtheta_t)) along the tangent
        directions t = 0..2 (zeros in the plain builds)."""
        D = (C.c_double * 2)()
        dD = (C.c_double * 6)()
        _check("lb3e_deformation", lib().lb3e_deformation(self._h, D, dD))
        return (D[0], D[1]), (tuple(dD[0:3]), tuple(dD[3:6]))

    def shape_objective(self, phi_target):
        """J = sum (phi_i - target_i)^2 of the current populations' phases and, in the
        tangent builds, (dJ/dtheta_t) along the tangent directions (zeros otherwise).
        ``phi_target``: [3, ny, nx] float64, host numpy or CUDA tensor."""
        addr, _keep = _addr(phi_target)
        J = C.c_double(0)
        dJ = (C.c_double * 3)()
        _check("lb3e_shape_objective", lib().lb3e_shape_objective(self._h, addr, C.byref(J), dJ))
        return J.value, tuple(dJ)

    # ---------------------------------------------------------------- reverse mode
    @property
    def compute_dtype(self):
        import torch
        return torch.float64 if int(self.params.get("precision", 0)) == 0 else torch.float32

    def _adj_ws(self):
        ws = getattr(self, "_adj_workspace", None)
        if ws is None:
            n = C.c_size_t(0)
            _check("lb3e_adjoint_workspace_bytes", lib().lb3e_adjoint_workspace_bytes(self._h, C.byref(n)))
            import torch
            ws = self._adj_workspace = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        return ws

    def _state_tensor(self):
        import torch
        return torch.empty((N_STATE,) + self.shape, dtype=self.compute_dtype, device=self.device)

    def state_vector(self, out=None):
        """The state X as a (64, ny, nx) CUDA tensor in the build's arithmetic type
        (planes: STATE_PLANES)."""
        out = self._state_tensor() if out is None else out
        _check("lb3e_state_vector", lib().lb3e_state_vector(self._h, out.data_ptr()))
        return out

    def adjoint_step(self, a_in, state=None, out=None) -> np.ndarray:
        """One step backwards (lb3e_adjoint_step): writes dJ/dX^n into ``out`` (a
        (64, ny, nx) CUDA tensor, allocated if None) from a_in = dJ/dX^{n+1}, for the
        step from ``state`` (a snapshot from save_state; None: the current state).
        Returns (out, dJ/dtheta over ADJ_PARAMS through this step)."""
        out = self._state_tensor() if out is None else out
        ws = self._adj_ws()
        dpar = np.zeros(len(ADJ_PARAMS))
        _check("lb3e_adjoint_step",
               lib().lb3e_adjoint_step(self._h, None if state is None else state.data_ptr(), a_in.data_ptr(),
                                       out.data_ptr(), dpar.ctypes.data_as(C.POINTER(C.c_double)),
                                       ws.data_ptr(), ws.numel()))
        return out, dpar

    @property
    def is_first_step(self) -> bool:
        f = C.c_int32(0)
        _check("lb3e_is_first_step", lib().lb3e_is_first_step(self._h, C.byref(f)))
        return bool(f.value)

    def adjoint_step_x(self, X, first: bool, a_in, out, dparams):
        """One step backwards from a state vector X (lb3e_adjoint_step_x) into
        ``out``; ``dparams`` a float64 CUDA tensor of 11 slots, accumulated in stream
        order (no synchronisation)."""
        ws = self._adj_ws()
        _check("lb3e_adjoint_step_x",
               lib().lb3e_adjoint_step_x(self._h, X.data_ptr(), int(bool(first)), a_in.data_ptr(), out.data_ptr(),
                                         dparams.data_ptr(), ws.data_ptr(), ws.numel()))
        return out

    def adjoint_init(self, phi, a_in, want_dphi: bool = True):
        """The creation backwards (lb3e_adjoint_init): (dJ/dtheta over ADJ_PARAMS,
        dJ/dphi_init as a host (3, ny, nx) array or None)."""
        addr, _keep = _addr(phi)
        ws = self._adj_ws()
        dpar = np.zeros(len(ADJ_PARAMS))
        dphi = np.zeros((3,) + self.shape) if want_dphi else None
        _check("lb3e_adjoint_init",
               lib().lb3e_adjoint_init(self._h, addr, a_in.data_ptr(), dpar.ctypes.data_as(C.POINTER(C.c_double)),
                                       None if dphi is None else dphi.ctypes.data, ws.data_ptr(), ws.numel()))
        return dpar, dphi

    def deformation_seed(self, which: str = "outer"):
        """(D, dD/dX) of the current populations (lb3e_deformation_seed)."""
        a = self._state_tensor()
        D = C.c_double(0)
        _check("lb3e_deformation_seed",
               lib().lb3e_deformation_seed(self._h, 0 if which == "inner" else 1, C.byref(D), a.data_ptr()))
        return D.value, a

    def shape_seed(self, phi_target):
        """(J, dJ/dX) of the shape objective of the current populations (lb3e_shape_seed)."""
        addr, _keep = _addr(phi_target)
        a = self._state_tensor()
        J = C.c_double(0)
        _check("lb3e_shape_seed", lib().lb3e_shape_seed(self._h, addr, C.byref(J), a.data_ptr()))
        return J.value, a

    def fd_residual(self) -> float:
        """||b - A psi|| / ||b|| of the current potential in the finite-difference form
        of div(eps grad psi) + q = 0 (a diagnostic; see lb3e_potential_fd_residual)."""
        r = C.c_double(0)
        _check("lb3e_potential_fd_residual", lib().lb3e_potential_fd_residual(self._h, C.byref(r)))
        return r.value

    def state_bytes(self) -> int:
        n = C.c_size_t(0)
        _check("lb3e_state_bytes", lib().lb3e_state_bytes(self._h, C.byref(n)))
        return n.value

    def save_state(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        _check("lb3e_save_state", lib().lb3e_save_state(self._h, out.data_ptr()))
        return out

    def load_state(self, src):
        _check("lb3e_load_state", lib().lb3e_load_state(self._h, src.data_ptr()))

    def set_timing(self, enable: bool):
        _check("lb3e_set_timing", lib().lb3e_set_timing(self._h, int(bool(enable))))

    def set_chunk(self, k: int) -> "Sim":
        """LB potential iterations per kernel launch (1..8; speed only)."""
        _check("lb3e_set_potential_chunk", lib().lb3e_set_potential_chunk(self._h, int(k)))
        return self

    def set_tile(self, rows: int) -> "Sim":
        """Rows of the fused pass's 32 x rows tiles (4, 8, 16; speed only)."""
        _check("lb3e_set_fused_tile", lib().lb3e_set_fused_tile(self._h, int(rows)))
        return self

    def set_staging(self, planes: int) -> "Sim":
        """TMA staging of the D3Q15 potential iteration's inputs: z planes a block
        walks (0: per-thread loads; speed only)."""
        _check("lb3e_set_staging", lib().lb3e_set_staging(self._h, int(planes)))
        return self

    def kernel_times(self) -> dict:
        """{class: (total ms, launches)} since the last call (synchronises)."""
        ms = (C.c_double * len(KERNEL_CLASSES))()
        n = (C.c_int64 * len(KERNEL_CLASSES))()
        _check("lb3e_kernel_times", lib().lb3e_kernel_times(self._h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}

    @property
    def launches(self) -> int:
        return int(lib().lb3e_launch_count(self._h))

    @property
    def potential_iterations(self) -> int:
        return int(lib().lb3e_potential_iterations(self._h))


class Batch:
    """Many lattices (one precision, any sizes) stepped together through the C ABI.

    ``params_list[i]`` is instance i's parameter dict; ``phis[i]`` its initial
    [3, ny, nx] phase field (host numpy or CUDA float64).  Electric instances must
    share one ``poisson_fixed_iter``.
    """

    def __init__(self, params_list, phis, stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lb3e needs a CUDA device (there is no CPU fallback)")
        n = len(params_list)
        self.params = [dict(p) for p in params_list]
        self.shapes = [(int(p["ny"]), int(p["nx"])) for p in params_list]
        self._p = (Params * n)(*[Params.from_dict(p) for p in params_list])
        nb = C.c_size_t(0)
        _check("lb3e_batch_workspace_bytes", lib().lb3e_batch_workspace_bytes(self._p, n, C.byref(nb)))
        self.device = torch.device(device or "cuda")
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        keep = [_addr(a) for a in phis]
        ptrs = (C.c_void_p * n)(*[k[0] for k in keep])
        h = C.c_void_p(None)
        _check("lb3e_batch_create", lib().lb3e_batch_create(self._p, n, ptrs, self.workspace.data_ptr(), nb.value,
                                                            self.stream.cuda_stream, C.byref(h)))
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lb3e_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, nsteps: int) -> "Batch":
        _check("lb3e_batch_run", lib().lb3e_batch_run(self._h, int(nsteps)))
        return self

    def set_chunk(self, k: int) -> "Batch":
        """Potential pseudo-iterations per launch (1..8); see autotune.py."""
        _check("lb3e_batch_set_potential_chunk", lib().lb3e_batch_set_potential_chunk(self._h, int(k)))
        self.chunk = int(k)
        return self

    def set_tile(self, rows: int) -> "Batch":
        """Rows of the fused pass's 32 x rows tiles (4, 8, 16; speed only); see autotune.py."""
        _check("lb3e_batch_set_fused_tile", lib().lb3e_batch_set_fused_tile(self._h, int(rows)))
        self.tile = int(rows)
        return self

    def observables(self) -> list:
        out = (Observables * self.n)()
        _check("lb3e_batch_observables", lib().lb3e_batch_observables(self._h, out))
        return [o.as_dict() for o in out]

    def field(self, instance: int, name: str):
        ny, nx = self.shapes[instance]
        arr = np.empty((ny, nx))
        _check("lb3e_batch_get_field", lib().lb3e_batch_get_field(self._h, instance, FIELDS[name], arr.ctypes.data))
        return arr

    @property
    def launches(self) -> int:
        return int(lib().lb3e_batch_launch_count(self._h))
