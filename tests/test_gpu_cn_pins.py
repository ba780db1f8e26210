"""Pins of the GPU's Crank-Nicolson pieces (gp_convective, gp_cn_rhs, cn_step)
against the mathematics of Sect. 2, with no oracle call.

* gp_convective: for affine (u, v) sampled at every node (ghost values
  included), u.grad u at every internal u and v node equals the analytic value
  (central differences and the four-point cross average are exact there);
  every other slot is 0.
* gp_cn_rhs: for a biquadratic state the five-point Laplacian is exact, so
  the momentum rows are u + alpha lap u + dt f - dt N; continuity rows carry
  the continuity source when one is set and 0 otherwise; the boundary rows
  carry the given values.
* cn_step with a linear-in-time convective history: the extrapolated step
  equals one solve with the history's mid-point value.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for

pytestmark = pytest.mark.gpu


def _solver(case, N, alpha=None):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    s = gpmg.Solver(N, x0, x0, L, levels=levels_for(N), alpha=alpha)
    assert s.geometry(W.phi_half_lattice(shape, N, x0, x0, L)) == 0, s.error()
    return s, x0, L


def _sample(s, N, x0, L, fu, fv, fp=None):
    g, i, j, X, Y = W.flat_coords(N, x0, x0, L)
    t = s.types_flat().astype(int)
    flat = np.zeros(g.size)
    act = (t != W.INACTIVE) & (g >= 0)
    for gg, f in ((0, fu), (1, fv), (2, fp)):
        if f is not None:
            m = act & (g == gg)
            flat[m] = f(X[m], Y[m])
    return flat, g, t, X, Y


@pytest.mark.parametrize("case,N", [("circle", 64), ("flower5", 128)])
def test_convective_exact_for_affine_fields(case, N):
    s, x0, L = _solver(case, N)
    rng = np.random.default_rng(31)
    a, c = rng.standard_normal(3), rng.standard_normal(3)
    fu = lambda X, Y: a[0] + a[1] * X + a[2] * Y
    fv = lambda X, Y: c[0] + c[1] * X + c[2] * Y
    flat, g, t, X, Y = _sample(s, N, x0, L, fu, fv)
    out = s.to_flat(s.convective(s.to_device(flat)))
    mu, mv = (g == 0) & (t == W.INTERNAL), (g == 1) & (t == W.INTERNAL)
    assert np.abs(out[mu] - (fu(X[mu], Y[mu]) * a[1] + fv(X[mu], Y[mu]) * a[2])).max() < 1e-12
    assert np.abs(out[mv] - (fu(X[mv], Y[mv]) * c[1] + fv(X[mv], Y[mv]) * c[2])).max() < 1e-12
    assert np.all(out[~(mu | mv)] == 0.0)


def _biquad(rng):
    k = rng.standard_normal((3, 3))
    f = lambda X, Y: sum(k[m, n] * X ** m * Y ** n for m in range(3) for n in range(3))
    lap = lambda X, Y: sum(k[m, n] * (m * (m - 1) * X ** max(m - 2, 0) * Y ** n
                                      + n * (n - 1) * X ** m * Y ** max(n - 2, 0))
                           for m in range(3) for n in range(3))
    return f, lap


def test_cn_rhs_exact_for_biquadratic_state():
    N = 128
    alpha = 0.41 / N
    s, x0, L = _solver("flower5", N, alpha=alpha)
    rng = np.random.default_rng(32)
    fu, lu = _biquad(rng)
    fv, lv = _biquad(rng)
    flat, g, t, X, Y = _sample(s, N, x0, L, fu, fv)
    n = flat.size
    f, Nh, bc, gsrc = (rng.standard_normal(n) for _ in range(4))
    dt = 0.017
    dev = s.to_device
    b = s.to_flat(s.cn_rhs(dev(flat), dev(Nh), dt, f=dev(f), bc=dev(bc)))
    for grid, ff, ll in ((0, fu, lu), (1, fv, lv)):
        m = (g == grid) & (t == W.INTERNAL)
        want = ff(X[m], Y[m]) + alpha * ll(X[m], Y[m]) + dt * f[m] - dt * Nh[m]
        assert np.abs(b[m] - want).max() < 1e-11
    mp = (g == 2) & (t == W.INTERNAL)
    assert np.all(b[mp] == 0.0)
    for tt in (W.WALL, W.BOXGHOST):
        m = (t == tt) & (g >= 0)
        assert np.array_equal(b[m], bc[m])
    # with a continuity source the continuity rows carry it
    gd = dev(gsrc)
    s.set_continuity_source(gd)
    b2 = s.to_flat(s.cn_rhs(dev(flat), dev(Nh), dt, f=dev(f), bc=dev(bc)))
    s.set_continuity_source(None)
    assert np.array_equal(b2[mp], gsrc[mp])
    assert np.array_equal(b2[~mp], b[~mp])


def test_extrapolated_step_uses_the_midpoint_of_a_linear_history():
    from paper_1911_00994_gb300 import gpmg
    N, Re = 64, 50.0
    shape, x0, L = CASES["circle"]
    dt = L / N
    s = gpmg.Solver(N, x0, x0, L, levels=levels_for(N), alpha=dt / (2 * Re), max_cycles=300)
    assert s.geometry(W.phi_half_lattice(shape, N, x0, x0, L)) == 0, s.error()
    ex = W.taylor_green()
    flat, g, t, X, Y = _sample(s, N, x0, L, lambda X, Y: 0.5 * ex.u(2 * X, 2 * Y), lambda X, Y: 0.5 * ex.v(2 * X, 2 * Y))
    xn = s.to_device(flat)
    Nn = s.convective(xn)
    D = s.to_device(W.random_flat(N, t, 9) * 0.3)
    N1, N2 = Nn - D, Nn - 2.0 * D
    x = xn.clone()
    st, rep = s.cn_step(x, N1.clone(), N2.clone(), 2, dt, Re, tol=5e-12, eps=0.0, kmax=1)
    assert st == 0, s.error()
    b = s.cn_rhs(xn, Nn + 0.5 * D, dt)
    y = xn.clone()
    st, rep2, _ = s.solve(y, b, 5e-12)
    assert st == 0, s.error()
    a, c = s.to_flat(x), s.to_flat(y)
    vel = (g < 2) & (t != W.INACTIVE)
    assert np.abs(a[vel] - c[vel]).max() <= 1e-9 * np.abs(c[vel]).max()
