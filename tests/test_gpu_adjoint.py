"""Adjoint of the multigrid solve on the GPU (M^T lam = c, the transposed
cycle) against the oracle's adjoint, element by element, and the gradient it
gives against central finite differences of the forward solves.

Tolerances as for the forward pieces: transposed residual 1e-13 relative,
relaxation stages 1e-12 (1e-11 for two relaxations), transfers 1e-14, cycles
1e-9, converged solves 1e-9 (both sides at ||r||_inf <= 1e-11).
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


def pair(case, N, alpha=None, **kw):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2.0 if alpha is None else alpha
    lev = levels_for(N)
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=lev)
    assert st == 0, o.error()
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha, adjoint=True, **kw)
    assert s.geometry(phi, 0) == 0, s.error()
    return o, s


@pytest.mark.parametrize("case,N", [("circle", 64), ("flower5", 128), ("ellipse", 128)])
def test_adjoint_pieces_match(case, N):
    o, s = pair(case, N)
    for lev in range(o.levels):
        Nl = N >> lev
        t = o.types(lev)
        rng = np.random.default_rng(40 + lev)
        lam = rng.standard_normal(o.n(lev))
        cc = rng.standard_normal(o.n(lev)) * 10
        lamd, ccd = s.to_device(lam, lev), s.to_device(cc, lev)
        r_o, n_o = o.residual_t(lam, cc, lev)
        r_g, n_g = s.residual_t(lamd, ccd, lev)
        assert rel(s.to_flat(r_g, lev), r_o) < 1e-13, lev
        assert abs(n_g - n_o) <= 1e-13 * n_o
        for name in ("box_sweep_t", "scalar_update_t", "ghost_sweep_t"):
            want = getattr(o, name)(lam, cc, lev)
            lg = s.to_device(lam, lev)
            getattr(s, name)(lg, ccd, lev)
            assert rel(s.to_flat(lg, lev), want) < 1e-12, (name, lev)
        want = o.smooth_t(lam, cc, 2, lev)
        lg = s.to_device(lam, lev)
        s.smooth_t(lg, ccd, 2, lev)
        assert rel(s.to_flat(lg, lev), want) < 1e-11, lev
        if lev + 1 < o.levels:
            yH = rng.standard_normal(o.n(lev + 1))
            want = o.restrict_t(yH, lam, lev)
            lg = s.to_device(lam, lev)
            s.restrict_t(s.to_device(yH, lev + 1), lg, lev)
            assert rel(s.to_flat(lg, lev), want) < 1e-14, lev
            want = o.prolong_t(cc, lev)
            got = s.to_flat(s.prolong_t(ccd, lev), lev + 1)
            assert rel(got, want) < 1e-14, lev
        assert Nl > 0


@pytest.mark.parametrize("case,N,ah2", [("circle", 64, None), ("flower5", 256, 2.0), ("circle_off", 128, None)])
def test_adjoint_cycles_match(case, N, ah2):
    shape, x0, L = CASES[case]
    h = L / N
    alpha = None if ah2 is None else ah2 * h * h
    o, s = pair(case, N, alpha=alpha)
    cc = np.random.default_rng(7).standard_normal(o.n())
    lam = np.zeros(o.n())
    lg, ccd = s.to_device(lam), s.to_device(cc)
    for k in range(3):
        st, lam = o.cycle_t(lam, cc)
        s.cycle_t(lg, ccd)
        assert rel(s.to_flat(lg), lam) < 1e-9, k


@pytest.mark.parametrize("case,N", [("circle", 32), ("flower5", 128)])
def test_adjoint_solve_matches_oracle(case, N):
    o, s = pair(case, N)
    cc = np.random.default_rng(8).standard_normal(o.n())
    st_o, lam_o, h_o = o.solve_t(np.zeros(o.n()), cc, 1e-11, 200)
    assert st_o == 0
    lg = s.new_vec()
    st, rep, h_g = s.solve_t(lg, s.to_device(cc), 1e-11)
    assert st == 0, s.error()
    assert rel(s.to_flat(lg), lam_o) <= 1e-9
    assert abs(len(h_g) - len(h_o)) <= 1
    if N == 32:
        A = o.dense_matrix(0)
        ref = np.linalg.solve(A.T, cc)
        assert rel(s.to_flat(lg), ref) <= 1e-9


@pytest.mark.parametrize("case,N", [("circle", 32), ("flower5", 128), ("ellipse", 128)])
def test_adjoint_krylov_matches_oracle(case, N):
    # BiCGSTAB on M^T lam = c preconditioned by one transposed cycle: the
    # oracle's adjoint solution (and at 32^2 the dense transpose solve), two
    # cycles per iteration, fewer cycles than the plain transposed cycles
    o, s = pair(case, N, krylov=True)
    cc = np.random.default_rng(9).standard_normal(o.n())
    st_o, lam_o, h_o = o.solve_t(np.zeros(o.n()), cc, 1e-11, 200)
    assert st_o == 0
    lg = s.new_vec()
    st, rep, h_g = s.solve_t(lg, s.to_device(cc), 1e-11)
    assert st == 0, s.error()
    assert rep.cycles == 2 * rep.iterations and len(h_g) == rep.iterations + 1
    assert rep.res <= 1e-11
    assert rel(s.to_flat(lg), lam_o) <= 1e-9
    assert rep.cycles < len(h_o) - 1
    if N == 32:
        A = o.dense_matrix(0)
        assert rel(s.to_flat(lg), np.linalg.solve(A.T, cc)) <= 1e-9


def test_forcing_gradient_matches_finite_differences():
    # J(f) = sum over a probe window of u^2 and v^2 after one extrapolated CN
    # step (Eq. extrUdU; the right-hand side is affine in f: dt f on internal
    # momentum rows), circle r = 0.25 at (0.2, 0) on [-1, 1]^2, N = 64,
    # Re = 100, dt = h.  dJ/df = dt lam on internal momentum rows with
    # M^T lam = dJ/dx = 2 x on the window.  J is quadratic in f, so central
    # differences are exact for any step; eps = 0.5 keeps the solver's
    # tolerance (1e-12) far below the compared digits.  8 seeded directions.
    from paper_1911_00994_gb300 import gpmg
    N, x0, L, Re = 64, -1.0, 2.0, 100.0
    h = L / N
    dt = h
    phi = W.phi_half_lattice(W.circle(0.25, 0.2, 0.0), N, x0, x0, L)
    s = gpmg.Solver(N, x0, x0, L, levels=levels_for(N), alpha=dt / (2 * Re), adjoint=True, max_cycles=200)
    assert s.geometry(phi, 0) == 0, s.error()
    tf = s.types_flat()
    n = len(tf)
    nU, nV = (N + 1) * (N + 2), (N + 2) * (N + 1)
    mom = np.zeros(n, dtype=bool)
    mom[:nU + nV] = tf[:nU + nV] == 1
    rng = np.random.default_rng(1234)
    xn = np.where(mom, 0.1 * rng.standard_normal(n), 0.0)
    N1 = np.where(mom, 0.1 * rng.standard_normal(n), 0.0)
    N2 = np.where(mom, 0.1 * rng.standard_normal(n), 0.0)
    f0 = np.where(mom, rng.standard_normal(n), 0.0)
    win = np.zeros(n)
    k = np.arange(nU)
    ju, iu = k // (N + 1) - 1, k % (N + 1)
    win[:nU] = (iu >= 40) & (iu < 56) & (ju >= 24) & (ju < 40)
    k = np.arange(nV)
    jv, iv = k // (N + 2), k % (N + 2) - 1
    win[nU:nU + nV] = (iv >= 40) & (iv < 56) & (jv >= 24) & (jv < 40)
    win *= mom

    def J(f):
        x, n1, n2 = s.to_device(xn), s.to_device(N1), s.to_device(N2)
        st, rep = s.cn_step(x, n1, n2, 2, dt, Re, f=s.to_device(f), body=(0.0, 0.0, 0.0, 0.2, 0.0), tol=1e-12)
        assert st == 0, s.error()
        xf = s.to_flat(x)
        return float(np.sum(win * xf * xf)), xf

    J0, xf0 = J(f0)
    assert J0 > 0.0
    lam = s.new_vec()
    st, rep, _ = s.solve_t(lam, s.to_device(2.0 * win * xf0), 1e-12)
    assert st == 0, s.error()
    grad = dt * np.where(mom, s.to_flat(lam), 0.0)
    eps = 0.5
    for k in range(8):
        d = np.where(mom, np.random.default_rng(k).standard_normal(n), 0.0)
        fd = (J(f0 + eps * d)[0] - J(f0 - eps * d)[0]) / (2 * eps)
        an = float(np.dot(grad, d))
        assert abs(fd - an) <= 1e-7 * abs(an) + 1e-12, (k, fd, an)
