"""Pins of the GPU geometry (node types and ghost rows read back through the C
ABI) against facts of the paper and of mathematics, with no oracle call.

* Eq. (BCu): every boundary-condition row's nine weights are the products of
  the three-point Lagrange weights at the row's boundary point B, so they sum
  to 1 and reproduce every biquadratic at B (this also fixes the sign of
  theta).
* Algorithm 1 on a circle: B lies on the circle to within the bisection
  tolerance 0.01 h plus the error of the bilinear interpolant of phi, which
  for phi = R - r is below h^2 / (4 (R - 2 h)) near the circle.
* Algorithm LS: an internal node has phi < 0 (fluid) on its own level, and
  every node with phi > 0 is ghost, wall, box ghost or inactive.
* Extrapolation rows (p_G - 2 p_1 + p_2 and x_G - 3 x_1 + 3 x_2 - x_3 along an
  axis) and copy rows annihilate constants and, for the first two, linear
  functions along their axis.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for

pytestmark = pytest.mark.gpu

OFF = np.array([[0.0, 0.5], [0.5, 0.0], [0.5, 0.5]])


def _solver(case, N):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    lev = levels_for(N)
    s = gpmg.Solver(N, x0, x0, L, levels=lev)
    phi = W.phi_half_lattice(shape, N, x0, x0, L)
    assert s.geometry(phi) == 0, s.error()
    return s, phi, shape, x0, L


def _node_xy(s, lev, idx):
    """Coordinates of device-layout vector indices of level lev."""
    from paper_1911_00994_gb300 import gpmg
    Nl = s.N >> lev
    P, F = gpmg.pitch(Nl), gpmg.frame(Nl)
    h = s.len / Nl
    idx = np.asarray(idx, dtype=np.int64)
    g = idx // F
    rem = idx % F
    j = rem // P - 1
    i = rem % P - 1
    return g, s.x0 + (i + OFF[g, 0]) * h, s.y0 + (j + OFF[g, 1]) * h


@pytest.mark.parametrize("case,N", [("circle", 64), ("ellipse", 128), ("flower5", 256), ("flower7", 256)])
def test_bcu_rows_reproduce_biquadratics(case, N):
    s, phi, shape, x0, L = _solver(case, N)
    rng = np.random.default_rng(21)
    for lev in range(s.levels):
        gr = s.ghost_rows(lev)
        m = np.where(gr["kind"] == 0)[0]
        assert len(m) > 0
        w = gr["w"][m]
        assert np.abs(w.sum(axis=1) - 1.0).max() < 1e-13
        g, X, Y = _node_xy(s, lev, gr["st"][m].reshape(-1))
        X, Y = X.reshape(-1, 9), Y.reshape(-1, 9)
        g0, XG, YG = _node_xy(s, lev, gr["node"][m])
        assert np.array_equal(g.reshape(-1, 9)[:, 0], g0) and np.all(g0 < 2)
        # the first stencil entry is the ghost itself
        assert np.array_equal(gr["st"][m][:, 0], gr["node"][m])
        B = gr["B"][m]
        for _ in range(3):
            c = rng.standard_normal((3, 3))
            q = lambda x, y: sum(c[a, b] * x ** a * y ** b for a in range(3) for b in range(3))
            err = np.abs((w * q(X, Y)).sum(axis=1) - q(B[:, 0], B[:, 1]))
            assert err.max() < 1e-11 * (1 + np.abs(c).sum())


@pytest.mark.parametrize("N", [32, 64, 256, 1024])
def test_boundary_points_on_the_circle(N):
    s, phi, shape, x0, L = _solver("circle", N)
    R = 0.5
    for lev in range(s.levels):
        h = L / (N >> lev)
        gr = s.ghost_rows(lev)
        m = gr["kind"] == 0
        r = np.hypot(gr["B"][m, 0], gr["B"][m, 1])
        assert np.abs(r - R).max() <= 0.01 * h + h * h / (4 * (R - 2 * h)) + 1e-14


@pytest.mark.parametrize("case,N", [("circle", 64), ("flower5", 256), ("ellipse", 128)])
def test_types_follow_the_sign_of_phi(case, N):
    s, phi, shape, x0, L = _solver(case, N)
    for lev in range(s.levels):
        Nl = N >> lev
        t = s.types_flat(lev)[:-1].astype(int)
        g, i, j, X, Y = W.flat_coords(Nl, x0, x0, L)
        g, i, j, X, Y = g[:-1], i[:-1], j[:-1], X[:-1], Y[:-1]
        ph = shape(X, Y)                      # paper sign: > 0 inside the body
        assert np.all(ph[t == W.INTERNAL] < 0.0)
        assert not np.any((t == W.INTERNAL) & (ph > 0.0))
        # walls and box ghosts sit where Algorithm LS's box rows put them
        assert np.all((t == W.WALL) <= (((g == 0) & ((i == 0) | (i == Nl))) | ((g == 1) & ((j == 0) | (j == Nl)))))


@pytest.mark.parametrize("case,N", [("flower5", 256), ("flower7", 256)])
def test_extrapolation_rows_annihilate_polynomials(case, N):
    s, phi, shape, x0, L = _solver(case, N)
    rng = np.random.default_rng(5)
    for lev in range(s.levels):
        gr = s.ghost_rows(lev)
        for kind in (1, 2):
            m = np.where(gr["kind"] == kind)[0]
            if len(m) == 0:
                continue
            nst = gr["nst"][m]
            a = rng.standard_normal(3)
            for k in m[:500]:
                ns = gr["nst"][k]
                g, X, Y = _node_xy(s, lev, gr["st"][k][:ns])
                w = gr["w"][k][:ns]
                assert abs(w.sum()) < 1e-14                      # constants
                if kind == 1:
                    lin = a[0] + a[1] * X + a[2] * Y
                    assert abs(np.dot(w, lin)) < 1e-12          # linear along the axis
                    # nodes equally spaced on one axis line
                    d = np.hypot(np.diff(X), np.diff(Y))
                    assert np.allclose(d, d[0]) and (np.ptp(X) == 0 or np.ptp(Y) == 0)
            assert set(nst.tolist()) <= ({3, 4} if kind == 1 else {2})
