"""The LB potential solve (Eq. 43) run with 1 to 8 pseudo-iterations per launch:
one launch per iteration, or temporally blocked on a 4-cell or 8-cell halo.  The
blocking changes the launches, not the arithmetic of a cell, so FP64 states agree
bitwise; the walls cover the ghost-row bounce-back of the blocked kernels."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("phinow1", "phinow2", "phinow3", "psi", "ex", "ey", "q", "ux", "uy")


def _case(bc_y, precision=0, nx=67, ny=45, **kw):
    p = W.params(nx=nx, ny=ny, bc_y=bc_y, electric=1, precision=precision, eps=(1.0, 2.0, 4.0),
                 sigma=(1.0, 0.5, 0.25), eps_ref=4.0, V_top=0.03 if bc_y == 2 else 0.0,
                 E_ext=(0.0, 0.0) if bc_y == 2 else (0.0, 2e-3), **kw)
    return p, W.compound_droplet(nx, ny, 8.0, 15.0, 4.0)


def _run(p, phi, chunk, steps=5):
    import paper_2608_05787_b300 as L
    s = L.Sim(p, phi).set_chunk(chunk)
    s.step(steps)
    return s


@pytest.mark.parametrize("bc_y", [0, 1, 2])
@pytest.mark.parametrize("chunk", [2, 4, 5, 8])
def test_fp64_chunks_bitwise(bc_y, chunk):
    p, phi = _case(bc_y, poisson_fixed_iter=11)
    a, b = _run(p, phi, 1), _run(p, phi, chunk)
    for f in FIELDS:
        assert np.array_equal(a.field(f), b.field(f)), (bc_y, chunk, f)


@pytest.mark.parametrize("chunk", [3, 4, 8])
def test_fp64_chunks_converged_solve(chunk):
    """Tolerance-driven solves: the residual checks (every 5 iterations) fall inside
    or at the ends of chunks; iteration counts and states agree exactly.  The
    residual norm itself is summed over blocks of another shape (32 x 8 cells per
    launch of one iteration, 32 x 16 when blocked), so it agrees to rounding."""
    p, phi = _case(2, poisson_tol=1e-7, poisson_check_every=5, poisson_max_iter=4000)
    a, b = _run(p, phi, 1, steps=3), _run(p, phi, chunk, steps=3)
    oa, ob = a.observables(), b.observables()
    assert oa["poisson_iters"] == ob["poisson_iters"]
    assert abs(oa["poisson_residual"] - ob["poisson_residual"]) <= 1e-12 * oa["poisson_residual"]
    for f in FIELDS:
        assert np.array_equal(a.field(f), b.field(f)), (chunk, f)


@pytest.mark.parametrize("nx", [67, 66])
@pytest.mark.parametrize("bc_y", [0, 1, 2])
@pytest.mark.parametrize("chunk", [2, 4, 8])
@pytest.mark.parametrize("solver", [0, 3])
def test_fp32_chunks_bitwise(solver, chunk, bc_y, nx):
    """FP32: the blocked kernel runs a thread's two cells on packed FP32x2
    instructions, the per-iteration kernel one cell on scalar ones, in the same
    order of operations (each packed component rounds as the scalar instruction), so
    the iterates agree bitwise: the plain iteration (solver 0) and the iteration on
    the correction to the anchor (solver 3, refreshed every 5 iterations).  An odd nx
    takes the blocked kernel's scalar global accesses, an even one its 64-bit ones."""
    p, phi = _case(bc_y, precision=1, nx=nx, poisson_fixed_iter=13, potential_solver=solver, poisson_check_every=5)
    a, b = _run(p, phi, 1), _run(p, phi, chunk)
    for f in FIELDS:
        assert np.array_equal(a.field(f), b.field(f)), (solver, chunk, bc_y, f)
    for j in range(9):
        assert np.array_equal(a.pop("h", j), b.pop("h", j)), (solver, chunk, bc_y, j)


def test_chunk_out_of_range_is_rejected():
    import paper_2608_05787_b300 as L
    p, phi = _case(2, poisson_fixed_iter=3)
    s = L.Sim(p, phi)
    for bad in (0, 9, -1):
        with pytest.raises(RuntimeError):
            s.set_chunk(bad)
