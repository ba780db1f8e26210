"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
not by the oracle itself.

* Eq. (BCu): Lagrange weights reproduce biquadratics exactly at B (this is
  what fixes the sign of theta).
* Algorithm 1: B lies on the circle within the bisection tolerance 0.01 h
  plus the O(h^2) error of the bilinear interpolant.
* Polynomial exactness: for biquadratic u, v and linear p every row of the
  discrete system is exact, so the sampled field solves it (p up to the mean).
* Direct sparse solve (scipy) of the assembled system equals the oracle.
* Second-order decay of the velocity error and of xi (Sect. 5.1 claims).
* Eqs. (restop), (restop5): printed restriction stencils, incl. the 1/5 case.
* Bilinear prolongation is exact for linear fields.
* Multicolour box ordering is race free: a random order inside each colour
  gives a bitwise identical iterate.
* W-cycle (the cycle Sect. 4 adopts): with two levels it is the V-cycle
  bitwise (the coarse problem is solved exactly, so a second visit changes
  nothing); on more levels it is the pre-smoothing, restriction, two coarse
  cycles (from zero, then from the first's result), prolongation and
  post-smoothing composed from the pinned pieces; it converges to the dense
  solution.
* Eq. (LS) fixes the pressure only through the mean row: adding a constant to
  every internal and ghost pressure leaves every other row's residual
  unchanged (the momentum rows see pressure differences, the pressure ghost
  rows have weights summing to zero, no other row reads p), on every level.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, make_oracle, manufactured

OXY = {0: (0.0, 0.5), 1: (0.5, 0.0), 2: (0.5, 0.5)}


def node_xy(o, lev, g, i, j):
    h = o.len / (o.N >> lev)
    g = np.asarray(g)
    ox = np.where(g == 0, 0.0, 0.5)
    oy = np.where(g == 1, 0.0, 0.5)
    return o.x0 + (i + ox) * h, o.y0 + (j + oy) * h


@pytest.mark.parametrize("case,N", [("circle", 32), ("circle", 64), ("ellipse", 128), ("flower5", 128)])
def test_bcu_weights_reproduce_biquadratics(case, N):
    o, phi, st = make_oracle(case, N)
    assert st == 0, o.error()
    rng = np.random.default_rng(3)
    for lev in range(o.levels):
        gh = o.ghosts(lev)
        m = np.where((gh["grid"] < 2) & (gh["kind"] == 0))[0]
        assert len(m) > 0
        for _ in range(3):
            c = rng.standard_normal((3, 3))
            q = lambda x, y: sum(c[a, b] * x ** a * y ** b for a in range(3) for b in range(3))
            for k in m:
                st9 = gh["st"][k]
                xs, ys = node_xy(o, lev, gh["grid"][k], st9[:, 0], st9[:, 1])
                val = np.dot(gh["w"][k], q(xs, ys))
                assert abs(gh["w"][k].sum() - 1.0) < 1e-13
                assert abs(val - q(*gh["B"][k])) < 1e-12 * (1 + np.abs(c).sum() * 4)


def test_lagrange_nodes_and_theta_range():
    # theta of an Eq. (BCu) row lies in [0, 1] (B within one cell of G), or
    # down to -snap for a ghost snapped from inside the fluid (B beyond G)
    o, phi, st = make_oracle("circle", 64)
    gh = o.ghosts(0)
    m = (gh["grid"] < 2) & (gh["kind"] == 0)
    th = gh["theta"][m]
    assert th.min() > -(o.snap * np.sqrt(2.0) + 0.02) and th.max() <= 1.0
    assert (th.min(1) < 0).any() and (th.max(1) > 0.5).any()
    # a ghost on the boundary (theta = 0) gets the weights of the node itself
    w0 = gh["w"][m][np.argmin(np.abs(th).sum(1))]
    assert w0[0] > 0.9


def test_boundary_point_on_circle():
    R = 0.5
    for N in (32, 64, 128):
        o, phi, st = make_oracle("circle", N)
        h = 2.0 / N
        gh = o.ghosts(0)
        m = (gh["grid"] < 2) & (gh["kind"] == 0)
        B = gh["B"][m]
        r = np.hypot(B[:, 0], B[:, 1])
        # bilinear interpolant of R - r has error <= h^2 / (4 r) (second derivative 1/r)
        assert np.abs(r - R).max() <= 0.01 * h + h * h / (4 * (R - 2 * h))
        # and B is the foot of the normal through G within O(h^2)
        xs, ys = node_xy(o, 0, gh["grid"][m], gh["i"][m], gh["j"][m])
        G = np.stack([xs, ys], 1)
        Bstar = G * (R / np.hypot(xs, ys))[:, None]
        assert np.abs(B - Bstar).max() <= 0.01 * h + 2.0 * h * h / R


@pytest.mark.parametrize("case,N", [("circle", 32), ("circle", 64), ("ellipse", 128), ("circle_off", 128),
                                    ("flower5", 256), ("nobody", 32)])
def test_polynomial_exactness(case, N):
    o, phi, st = make_oracle(case, N)
    assert st == 0, o.error()
    ex = W.biquadratic(seed=7)
    b, xe, t, gh = manufactured(o, ex)
    r, nrm = o.residual(xe, b)
    assert nrm <= 1e-12 * max(1.0, np.abs(b).max())


def test_direct_and_multigrid_reproduce_biquadratic():
    o, phi, st = make_oracle("circle", 32)
    ex = W.biquadratic(seed=11)
    b, xe, t, gh = manufactured(o, ex)
    # direct sparse solve (library) of the assembled system
    ri, ci, v = o.assemble()
    A = sp.csr_matrix((v, (ri, ci)), shape=(o.n(), o.n()))
    xd = spla.spsolve(A.tocsc(), b)
    assert np.abs(xd - xe).max() < 1e-11
    # oracle dense LU
    st, xl = o.dense_solve(b)
    assert st == 0 and np.abs(xl - xe).max() < 1e-11
    # multigrid
    st, xm, hist = o.solve(np.zeros_like(b), b, 1e-12, 60)
    assert st == 0
    assert np.abs(xm - xe).max() < 1e-10


def test_assembled_matrix_matches_residual():
    o, phi, st = make_oracle("flower5", 64)
    rng = np.random.default_rng(0)
    t = o.types()
    x = W.random_flat(64, t, 1)
    b = rng.standard_normal(o.n())
    r, _ = o.residual(x, b)
    ri, ci, v = o.assemble()
    A = sp.csr_matrix((v, (ri, ci)), shape=(o.n(), o.n()))
    assert np.abs(r - (b - A @ x)).max() < 1e-12 * np.abs(b).max() * 100


def test_multigrid_equals_direct_circle32():
    # circle r = 0.5, 32 x 32 on [-1, 1]^2, Re = 1, dt = h -> alpha = h / 2
    o, phi, st = make_oracle("circle", 32)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st, xd = o.dense_solve(b)
    st, xm, hist = o.solve(np.zeros_like(b), b, 1e-12, 60)
    assert st == 0
    assert np.abs(xm - xd).max() / np.abs(xd).max() <= 1e-10


def test_second_order_velocity_and_divergence():
    errs, xis, hs = [], [], []
    for N in (32, 64, 128, 256):
        o, phi, st = make_oracle("circle", N)
        ex = W.taylor_green()
        b, xe, t, gh = manufactured(o, ex)
        st, x, hist = o.solve(np.zeros_like(b), b, 1e-12, 80)
        assert st == 0
        g, i, j, X, Y = W.flat_coords(N, o.x0, o.y0, o.len)
        m = (t == O.INTERNAL) & (g < 2)
        errs.append(np.abs(x[m] - xe[m]).max())
        xis.append(abs(x[-1]))
        hs.append(2.0 / N)
    order_u = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    order_xi = np.polyfit(np.log(hs), np.log(xis), 1)[0]
    assert order_u > 1.7, (errs, order_u)
    assert order_xi > 1.7, (xis, order_xi)


def test_divergence_minus_g_equals_xi_after_convergence():
    # Sect. 5.1: div u - g = xi at every internal cell once the system is solved
    o, phi, st = make_oracle("ellipse", 128)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st, x, hist = o.solve(np.zeros_like(b), b, 1e-11, 80)
    assert st == 0
    N, h = 128, 2.0 / 128
    u, v, p, xi = O.split(x, N)
    _, _, tp, _ = O.split(t.astype(float), N)
    _, _, bp, _ = O.split(b, N)
    div = (u[1:N + 1, 1:N + 1] - u[1:N + 1, 0:N] + v[1:N + 1, 1:N + 1] - v[0:N, 1:N + 1]) / h
    m = tp == O.INTERNAL
    assert np.abs(div[m] - bp[m] - xi).max() <= 2e-11
    assert abs(h * h * p[m].sum()) <= 1e-11


def test_mean_row_exact_after_scalar_update():
    o, phi, st = make_oracle("flower5", 64)
    t = o.types()
    x = W.random_flat(64, t, 2)
    b = np.zeros(o.n())
    b[-1] = 0.37
    x2 = o.scalar_update(x, b)
    r, _ = o.residual(x2, b)
    assert abs(r[-1]) < 1e-14


def _restrict_stencil(g, I, J):
    if g == 0:
        return [((2 * I + di, 2 * J + dj), (2.0 if di == 0 else 1.0) / 8) for dj in (0, 1) for di in (-1, 0, 1)]
    if g == 1:
        return [((2 * I + di, 2 * J + dj), (2.0 if dj == 0 else 1.0) / 8) for dj in (-1, 0, 1) for di in (0, 1)]
    return [((2 * I + di, 2 * J + dj), 0.25) for dj in (0, 1) for di in (0, 1)]


def test_restriction_printed_stencils_and_one_fifth_case():
    o, phi, st = make_oracle("circle", 64, levels=2)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(o.n(0))
    bH = o.restrict(r, 0)
    tf, tc = o.types(0), o.types(1)
    Nf, Nc = 64, 32
    seen_full, seen_five = 0, 0
    for k in range(len(tc) - 1):
        g, I, J = _gij(k, Nc)
        if tc[k] != O.INTERNAL:
            continue
        sten = _restrict_stencil(g, I, J)
        idx = [(W.flat_index(Nf, g, a, bb) if _inside(g, a, bb, Nf) else -1) for (a, bb), w in sten]
        internal = [q >= 0 and tf[q] == O.INTERNAL for q in idx]
        if all(internal):
            want = sum(w * r[q] for q, ((a, bb), w) in zip(idx, sten))
            assert abs(bH[k] - want) < 1e-14
            seen_full += 1
        elif g == 0 and sum(internal) == 5:
            want = np.mean([r[q] for q, ok in zip(idx, internal) if ok])  # Eq. (restop5)
            assert abs(bH[k] - want) < 1e-14
            seen_five += 1
    assert seen_full > 100 and seen_five > 0
    assert bH[-1] == r[-1]


def _inside(g, i, j, N):
    if g == 0:
        return 0 <= i <= N and -1 <= j <= N
    if g == 1:
        return -1 <= i <= N and 0 <= j <= N
    return 0 <= i < N and 0 <= j < N


def _gij(k, N):
    nU, nV, nP, n = W.flat_sizes(N)
    if k < nU:
        return 0, k % (N + 1), k // (N + 1) - 1
    k -= nU
    if k < nV:
        return 1, k % (N + 2) - 1, k // (N + 2)
    k -= nV
    return 2, k % N, k // N


def test_prolongation_exact_for_linear_fields():
    o, phi, st = make_oracle("nobody", 32, levels=2)
    a = np.array([0.3, -1.1, 0.7])
    f = lambda x, y: a[0] + a[1] * x + a[2] * y
    gC, iC, jC, XC, YC = W.flat_coords(16, o.x0, o.y0, o.len)
    tC = o.types(1)
    eH = np.where((tC != O.INACTIVE) & (gC >= 0), f(XC, YC), 0.0)
    eH[-1] = 0.0
    x = o.prolong(eH, np.zeros(o.n(0)), 0)
    g, i, j, X, Y = W.flat_coords(32, o.x0, o.y0, o.len)
    t = o.types(0)
    m = (t != O.INACTIVE) & (g >= 0)
    # velocity nodes next to a box corner interpolate from the
    # inactive corner node of the coarse grid (no value, weight renormalised away)
    near_x = (i <= 1) | (i >= 31)
    near_y = (j <= 1) | (j >= 31)
    corner = ((g == 0) | (g == 1)) & near_x & near_y
    m &= ~corner
    assert np.abs(x[m] - f(X[m], Y[m])).max() < 1e-13


def test_colour_order_is_race_free():
    o1, phi, st = make_oracle("flower5", 128, order_mode=0)
    o2, phi, st = make_oracle("flower5", 128, order_mode=1, seed=99)
    t = o1.types()
    x = W.random_flat(128, t, 4)
    b = W.random_flat(128, t, 5)
    y1 = o1.box_sweep(x, b)
    y2 = o2.box_sweep(x, b)
    assert np.array_equal(y1, y2)
    assert not np.array_equal(y1, x)


def test_w_cycle_on_two_levels_is_the_v_cycle():
    ex = W.taylor_green()
    out = []
    for gamma in (1, 2):
        o, phi, st = make_oracle("flower5", 64, levels=2, gamma=gamma)
        assert st == 0
        b, xe, t, gh = manufactured(o, ex)
        x = W.random_flat(64, t, 21)
        for _ in range(2):
            st, x = o.cycle(x, b)
            assert st == 0
        out.append(x)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_composed_from_its_pieces(gamma):
    # Sect. 4: nu1 relaxations, the residual restricted, the coarse residual
    # equation by gamma coarse cycles from a zero error (each from the last
    # one's result), the error prolonged and added, nu2 relaxations
    o, phi, st = make_oracle("flower5", 128, alpha=2.0 / 128 ** 2, levels=4, gamma=gamma)
    assert st == 0
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    x0 = W.random_flat(128, t, 22)
    st, xc = o.cycle(x0, b)
    assert st == 0
    x = o.smooth(x0, b, 2, 0)
    r, _ = o.residual(x, b, 0)
    bH = o.restrict(r, 0)
    eH = np.zeros(o.n(1))
    for _ in range(gamma):
        st, eH = o.cycle(eH, bH, 1)
    x = o.prolong(eH, x, 0)
    x = o.smooth(x, b, 1, 0)
    assert np.array_equal(x, xc)
    if gamma == 2:
        # one coarse cycle instead of two gives another iterate
        st, e1 = o.cycle(np.zeros(o.n(1)), bH, 1)
        assert not np.array_equal(e1, eH)


def test_w_cycles_converge_to_the_dense_solution():
    o, phi, st = make_oracle("circle", 32, gamma=2)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st, xd = o.dense_solve(b)
    st, xw, hw = o.solve(np.zeros_like(b), b, 1e-12, 60)
    assert st == 0
    assert np.abs(xw - xd).max() / np.abs(xd).max() <= 1e-10


def test_coarse_solve_matches_library_solve():
    o, phi, st = make_oracle("flower5", 64)
    lev = o.levels - 1
    A = o.dense_matrix(lev)
    rng = np.random.default_rng(8)
    b = rng.standard_normal(o.n(lev))
    x = o.coarse_solve(b)
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-9 * np.abs(x).max()


def test_krylov_equals_direct_solve():
    # BiCGSTAB preconditioned by one cycle reaches the dense solution of the
    # assembled system (the 32^2 circle)
    o, phi, st = make_oracle("circle", 32)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st, xd = o.dense_solve(b)
    st, xk, hist = o.solve_krylov(np.zeros_like(b), b, 1e-12, 60)
    assert st == 0
    assert np.abs(xk - xd).max() / np.abs(xd).max() <= 1e-10


def test_openmp_build_gives_the_same_iterate():
    # the multi-core CPU baseline's build: parallel loops only over
    # independent boxes of one colour and over rows with disjoint outputs,
    # so one V-cycle is bitwise that of the serial build
    o1, phi, st = make_oracle("flower5", 128)
    o4 = O.Oracle(128, 0.0, 0.0, 1.0, o1.levels, o1.alpha, threads=4)
    assert o4.geometry(phi) == 0 and o4.threads == 4
    t = o1.types()
    b = W.random_flat(128, t, 3)
    x = W.random_flat(128, t, 4)
    _, x1 = o1.cycle(x, b)
    _, x4 = o4.cycle(x, b)
    assert np.array_equal(x1, x4)
    assert np.array_equal(o1.residual(x1, b)[0], o4.residual(x4, b)[0])


@pytest.mark.parametrize("case,N", [("flower5", 128), ("circle_off", 128), ("ellipse", 256), ("flower7", 128),
                                    ("nobody", 64)])
def test_pressure_constant_only_changes_the_mean_row(case, N):
    shape, x0, L = CASES[case]
    o, phi, st = make_oracle(case, N, alpha=2.0 * (L / N) ** 2)
    assert st == 0, o.error()
    for lev in range(o.levels):
        Nl = N >> lev
        t = o.types(lev)
        n = t.size
        pbeg = n - 1 - Nl * Nl
        ind = np.zeros(n)
        pt = t[pbeg:n - 1]
        ind[pbeg:n - 1] = ((pt == 1) | (pt == 2)).astype(float)
        r, _ = o.residual(ind, np.zeros(n), lev=lev)
        assert np.abs(r[:-1]).max() <= 1e-9, lev
        # the mean row h^2 sum p over the internal cells sees it
        h = L / Nl
        assert abs(-r[-1] - h * h * np.count_nonzero(pt == 1)) <= 1e-9 * (1 + h * h * Nl * Nl), lev
