"""The cycle's residual restricted in the pass that computes it
(k_residual_restrict, `fuse_restrict=1`) against a residual pass followed by
a restriction pass (the default), and against the oracle.  The restricted
frames are the same bits (the same residual expressions, then Eq. restop /
restop5 in the same order); only the mean row's sum of p is added in another
order, so FP64 cycles agree to rounding.  N = 96 and 200 give coarse pitches
(64, 128) that leave ragged tiles at the right and top edges."""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle, manufactured

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


def solver(case, N, alpha, **kw):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    lev = levels_for(N)
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=lev)
    assert st == 0, o.error()
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha, **kw)
    assert s.geometry(phi, 0) == 0, s.error()
    return o, s


@pytest.mark.parametrize("case,N", [("flower5", 256), ("circle_off", 96), ("ellipse", 200)])
def test_fused_cycles_match_separate_passes_and_oracle(case, N):
    shape, x0, L = CASES[case]
    alpha = 2.0 * (L / N) ** 2
    o, s = solver(case, N, alpha, fuse_restrict=1)
    _, s2 = solver(case, N, alpha)
    b, xe, t, gh = manufactured(o, W.taylor_green())
    x = np.zeros_like(b)
    xg, bg = s.to_device(x), s.to_device(b)
    xg2, bg2 = s2.to_device(x), s2.to_device(b)
    for k in range(3):
        st, x = o.cycle(x, b)
        s.cycle(xg, bg)
        s2.cycle(xg2, bg2)
        got, sep = s.to_flat(xg), s2.to_flat(xg2)
        assert rel(got, sep) <= 1e-13, k
        assert rel(got, x) <= 1e-9, k


@pytest.mark.parametrize("case,N", [("flower5", 1024), ("ellipse", 200)])
def test_fused_mixed_solve_matches_separate_passes(case, N):
    # FP32 cycles inside FP64 residual correction: the same number of cycles
    # and FP64 residuals, both at the oracle's FP64 solution to the tolerance
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2000.0 if case == "flower5" else h / 200.0
    o, s = solver(case, N, alpha, precision=1, fuse_restrict=1)
    _, s2 = solver(case, N, alpha, precision=1)
    b, xe, t, gh = manufactured(o, W.taylor_green())
    xg, xg2 = s.new_vec(), s2.new_vec()
    st, rep, hist = s.solve(xg, s.to_device(b), 1e-10)
    st2, rep2, hist2 = s2.solve(xg2, s2.to_device(b), 1e-10)
    assert st == 0 and st2 == 0, (s.error(), s2.error())
    assert rep.cycles == rep2.cycles and rep.iterations == rep2.iterations
    assert rel(s.to_flat(xg), s2.to_flat(xg2)) <= 1e-9
    if N <= 256:
        st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 1e-10, 200)
        assert st_o == 0
        assert rel(s.to_flat(xg), x_o) <= 1e-8
