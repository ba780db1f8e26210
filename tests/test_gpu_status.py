"""Failure statuses of the C ABI, driven by host-side inputs only (nothing
here faults, traps or hangs the GPU): a level set with no fluid, NaN in the
right-hand side or the iterate, a cycle cap below what the tolerance needs,
and calls out of order.  Each failure leaves a message in gp_last_error and
the iterate at the last completed cycle.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for

pytestmark = pytest.mark.gpu


def _solver(N=64, case="circle", **kw):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    return gpmg.Solver(N, x0, x0, L, levels=levels_for(N), **kw), shape, x0, L


@pytest.mark.parametrize("value", [1.0, 0.0])
def test_level_set_without_fluid_is_a_geometry_error(value):
    from paper_1911_00994_gb300 import gpmg
    s, shape, x0, L = _solver()
    N = s.N
    # paper sign: phi >= 0 everywhere is all object (no sign change, no fluid)
    phi = np.full((2 * N + 1, 2 * N + 1), value)
    st = s.geometry(phi)
    assert st == gpmg.GP_GEOMETRY
    assert len(s.error()) > 0
    # the solve refuses to run on a failed geometry
    x, b = s.new_vec(), s.new_vec()
    st, rep, hist = s.solve(x, b, 1e-10)
    assert st == gpmg.GP_INVALID and len(s.error()) > 0


def test_solve_before_geometry_is_invalid():
    from paper_1911_00994_gb300 import gpmg
    s, shape, x0, L = _solver()
    st, rep, hist = s.solve(s.new_vec(), s.new_vec(), 1e-10)
    assert st == gpmg.GP_INVALID and "geometry" in s.error()


def _built(**kw):
    s, shape, x0, L = _solver(**kw)
    phi = W.phi_half_lattice(shape, s.N, x0, x0, L)
    assert s.geometry(phi) == 0, s.error()
    t = s.types_flat(0)
    return s, t


@pytest.mark.parametrize("where", ["rhs", "iterate"])
def test_nan_input_reports_divergence(where):
    from paper_1911_00994_gb300 import gpmg
    s, t = _built()
    b = s.to_device(W.random_flat(s.N, t, 3))
    x0 = s.to_device(W.random_flat(s.N, t, 4))
    internal = np.where(t == W.INTERNAL)[0]
    k = int(s.maps(0)[int(internal[len(internal) // 2])])
    (b if where == "rhs" else x0)[k] = float("nan")
    x = x0.clone()
    st, rep, hist = s.solve(x, b, 1e-10)
    assert st == gpmg.GP_DIVERGED
    assert "diverged" in s.error()
    assert rep.cycles == 0
    # no cycle ran: the iterate is the input (inactive slots zeroed)
    a, c = x.cpu().numpy(), x0.cpu().numpy()
    same = (a == c) | (np.isnan(a) & np.isnan(c))
    act = s.maps(0).cpu().numpy()[t != W.INACTIVE]
    assert same[act].all()


@pytest.mark.parametrize("precision", [0, 1])
def test_cycle_cap_reports_not_converged_with_the_last_cycle(precision):
    from paper_1911_00994_gb300 import gpmg
    s, t = _built(max_cycles=1, precision=precision, graphs=False)
    b = s.to_device(W.random_flat(s.N, t, 3))
    x = s.new_vec()
    st, rep, hist = s.solve(x, b, 1e-14)
    assert st == gpmg.GP_NOT_CONVERGED
    assert "not converged" in s.error()
    assert rep.cycles == 1 and rep.iterations == 1
    assert rep.res > 1e-14
    if precision == gpmg.GP_FP64:
        # the iterate is one cycle from zero
        y = s.new_vec()
        s.cycle(y, b)
        a, c = x.cpu().numpy(), y.cpu().numpy()
        assert np.abs(a - c).max() <= 1e-13 * np.abs(c).max()
    r, nrm = s.residual(x, b)
    assert abs(nrm - rep.res) <= 1e-12 * rep.res0


def test_bad_arguments_are_invalid():
    from paper_1911_00994_gb300 import gpmg
    s, t = _built()
    x, b = s.new_vec(), s.new_vec()
    L = s.L
    import ctypes
    assert L.mg_solve(s.ctx, None, ctypes.c_void_p(b.data_ptr()), 1e-10, None) == gpmg.GP_INVALID
    assert L.mg_solve(s.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()), -1.0, None) == \
        gpmg.GP_INVALID
    assert L.gp_residual(s.ctx, s.levels, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                         ctypes.c_void_p(x.data_ptr()), None) == gpmg.GP_INVALID
    with pytest.raises(gpmg.GpmgError):
        s.set_alpha(-1.0)
