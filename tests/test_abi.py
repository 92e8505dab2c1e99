"""The C ABI library loads and exports every entry point include/lb3e.h declares,
and its host-side validation works without a GPU (no compute calls here)."""
import ctypes as C
import re
from pathlib import Path

import pytest

import paper_2608_05787_b300 as L
import workloads as W

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(lb3e_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("lb3e_init", "lb3e_step", "lb3e_solve_potential", "lb3e_observables", "lb3e_get_field"):
        assert fn in names


def test_library_exports_every_declared_symbol():
    from paper_2608_05787_b300 import build
    build.build()
    lib = C.CDLL(str(L.LIB_PATH))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of lb3e_params / lb3e_observables_t have the C compiler's
    size and every field offset."""
    import subprocess
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "lb3e.h"', "int main(void) {"]
    for cname, py in (("lb3e_params", L.Params), ("lb3e_observables_t", L.Observables)):
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for py in (L.Params, L.Observables):
        want.append(C.sizeof(py))
        want += [getattr(py, f).offset for f, _ in py._fields_]
    assert got == want


@pytest.mark.parametrize("bad", [dict(tau_f=0.5), dict(nx=1), dict(bc_y=3), dict(precision=7),
                                 dict(gamma23=3e-3), dict(eps=(1.0, 0.0, 2.0)), dict(sigma=(-1, 0, 0)),
                                 dict(inner_phase=0), dict(V_top=float("nan")), dict(nx=2, ny=65535 * 8 + 1),
                                 dict(ions=2), dict(ions=1, ion_D=(0.0, 0.1)), dict(ions=1, precision=3),
                                 dict(ions=1, ion_beta=float("inf"))])
def test_invalid_parameters_rejected(bad):
    with pytest.raises(L.LB3EError) as e:
        L.workspace_bytes(W.params(**bad))
    assert e.value.code == -1


def test_workspace_scales_with_precision():
    p = W.params(nx=256, ny=128)
    b64 = L.workspace_bytes(dict(p, precision=0))
    b32 = L.workspace_bytes(dict(p, precision=1))
    b16 = L.workspace_bytes(dict(p, precision=2))
    assert b64 > b32 > b16 > 256 * 128 * 45 * 2 * 2


def test_ion_transport_adds_its_planes_to_the_workspace():
    """ions = 1 adds 2 x 18 population planes and 6 state planes (n_i, (n_i v_i)^{n-1})."""
    p = W.params(nx=256, ny=128)
    for prec, size in ((0, 8), (1, 4), (2, 4)):
        base = L.workspace_bytes(dict(p, precision=prec))
        ions = L.workspace_bytes(dict(p, precision=prec, ions=1))
        assert ions - base >= 42 * 256 * 128 * size
        assert ions - base < 42 * 256 * 128 * size + 3 * 256


def test_batches_refuse_ion_transport():
    p = W.params(nx=32, ny=32, poisson_fixed_iter=4, ions=1, ion_D=(0.1, 0.1))
    ps = (L.Params * 2)(L.Params.from_dict(p), L.Params.from_dict(p))
    nb = C.c_size_t(0)
    assert L.lib().lb3e_batch_workspace_bytes(ps, 2, C.byref(nb)) == -1
    ps[0].ions = ps[1].ions = 0
    assert L.lib().lb3e_batch_workspace_bytes(ps, 2, C.byref(nb)) == 0 and nb.value > 0


def test_three_dimensional_lattices_validated_and_sized():
    """nz >= 2 selects the D3Q15 step: FP64/FP32 and the LB potential only, no ions;
    the workspace holds 2 x 75 population planes, 2 x 15 potential planes and the
    fields (about 220 words a cell in FP32)."""
    p = dict(W.params(nx=64, ny=48), nz=40)
    n = 64 * 48 * 40
    b64 = L.workspace_bytes(dict(p, precision=0))
    b32 = L.workspace_bytes(dict(p, precision=1))
    assert 200 * 4 * n < b32 < 240 * 4 * n and b64 > 1.9 * b32
    for bad in (dict(precision=2), dict(precision=3), dict(potential_solver=1), dict(ions=1, ion_D=(0.1, 0.1)),
                dict(nz=70000)):
        with pytest.raises(L.LB3EError) as e:
            L.workspace_bytes(dict(p, **bad))
        assert e.value.code == -1
    # nz 0 or 1 is the two-dimensional step, and a dict without the key means 0
    assert L.workspace_bytes(dict(p, nz=1)) == L.workspace_bytes(W.params(nx=64, ny=48))
    ps = (L.Params * 2)(L.Params.from_dict(p), L.Params.from_dict(p))
    nb = C.c_size_t(0)
    assert L.lib().lb3e_batch_workspace_bytes(ps, 2, C.byref(nb)) == -1


def test_params_default_the_optional_fields():
    """Dicts written before the ion and three-dimensional fields existed still map:
    ions off, nz 0."""
    d = {k: v for k, v in W.params().items() if k not in ("ions", "ion_D", "ion_z", "ion_beta", "ion_charge")}
    s = L.Params.from_dict(d)
    assert s.ions == 0 and s.nz == 0 and s.precision == d["precision"]


@pytest.mark.parametrize("bad", [dict(potential_solver=2, nx=63), dict(potential_solver=2, bc_y=1),
                                 dict(potential_solver=3, precision=3), dict(potential_solver=2, precision=4),
                                 dict(potential_solver=4), dict(potential_solver=2, nz=8)])
def test_potential_solver_limits_are_checked(bad):
    """The anchored LB solves (2, 3) take the plain precisions; the coarse-corrected
    one (2) also needs electrodes and an even nx, like the multigrid solver."""
    p = W.config_deformation(n=64, r_out=16.0, r_in=8.0)["params"]
    with pytest.raises(L.LB3EError):
        L.workspace_bytes(dict(p, **bad))


def test_anchored_solver_workspace_holds_the_fp64_anchor():
    p = W.config_deformation(n=64, r_out=16.0, r_in=8.0, precision=1)["params"]
    plain, anch, coarse = (L.workspace_bytes(dict(p, potential_solver=s)) for s in (0, 3, 2))
    n = 64 * 64
    assert anch - plain >= 9 * n * 8 + 9 * n * 4   # the FP64 anchor and its FP32 increment
    assert coarse > anch                           # plus the multigrid levels


def test_staging_switch_checks_its_handle():
    """lb3e_set_staging validates on the host: a NULL handle is refused before any
    device work."""
    lib = L.lib()
    assert lib.lb3e_set_staging(None, 1) == -6
    assert lib.lb3e_set_staging(None, 0) == -6
