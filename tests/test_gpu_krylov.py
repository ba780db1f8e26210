"""BiCGSTAB preconditioned by one multigrid cycle on the GPU against the
oracle's BiCGSTAB, and on the bodies where plain V-cycles diverge (the
0.4 x 0.2 ellipse, the seven-petal flower)."""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle, manufactured

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


def setup(case, N, Re, precision=0):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / (2 * Re)
    lev = levels_for(N)
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=lev)
    assert st == 0
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha, krylov=True, precision=precision)
    assert s.geometry(phi) == 0, s.error()
    b, xe, t, gh = manufactured(o, W.taylor_green())
    return o, s, b


def test_krylov_matches_oracle_on_ellipse():
    o, s, b = setup("ellipse", 128, 100.0)
    st, xo, ho = o.solve_krylov(np.zeros_like(b), b, 1e-10, 60)
    assert st == 0
    x = s.new_vec()
    st, rep, hg = s.solve(x, s.to_device(b), 1e-10)
    assert st == 0, s.error()
    assert rel(s.to_flat(x), xo) <= 1e-8
    assert abs(rep.iterations - (len(ho) - 1)) <= 1
    assert rep.cycles == 2 * rep.iterations


@pytest.mark.parametrize("case,N,Re", [("flower7", 256, 500.0), ("flower5", 256, 1000.0), ("ellipse", 256, 100.0)])
def test_mixed_krylov_converges_where_cycles_diverge(case, N, Re):
    o, s, b = setup(case, N, Re, precision=1)
    x = s.new_vec()
    st, rep, hg = s.solve(x, s.to_device(b), 1e-10)
    assert st == 0, s.error()
    # the oracle's own residual of the GPU solution
    r, nrm = o.residual(s.to_flat(x), b)
    assert nrm <= 1.5e-10
