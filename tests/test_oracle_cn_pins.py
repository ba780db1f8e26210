"""Pins of the oracle's Crank-Nicolson pieces (Sect. 2) against facts of the
mathematics, not against the oracle itself.

* Convective term u.grad u (reading C18: central differences, the cross
  velocity averaged over the four nearest nodes of the other grid): for an
  affine velocity field, and for a biquadratic component with an affine
  cross velocity, every internal value equals the analytic u.grad u (central
  differences are exact for quadratics, the four-point average for affine
  fields).  A two-point cross average would miss it by |a_y b_y| h / 2.
* Right-hand side (Eqs. NSCN1, spaceprob): the five-point Laplacian is exact
  for biquadratics, so b = u + alpha lap u + dt f - dt N at every internal
  momentum node; continuity, extrapolation and mean rows 0; the boundary rows
  hold the given boundary values, or the rigid-body velocity at B and the
  wall velocities.
* Extrapolation (Eq. extrUdU): for a convective history that is linear in
  time, N^n + N^(n-1)/2 - N^(n-2)/2 is exactly its value at t^(n+1/2), so the
  step's solution is the solve with that mid-point value.
* Picard iteration (Eqs. NSitconv, iterativeNS): the returned state satisfies
  the stopping inequality, and with a tight eps it is the fixed point
  x = M^-1 b(N^(n+1/2)), N^(n+1/2) = (N(x^n) + N(x)) / 2.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_1911_00994_gb300 import workloads as W
from tests._cases import make_oracle


def _affine(rng):
    return rng.standard_normal(3)


def _fields(o, fu, fv, fp=None):
    """Flat vector with u, v (and p) sampled at every node of level 0 that
    is not inactive (ghost values included)."""
    N = o.N
    g, i, j, X, Y = W.flat_coords(N, o.x0, o.y0, o.len)
    t = o.types(0).astype(int)
    x = np.zeros(g.size)
    act = (t != W.INACTIVE) & (g >= 0)
    for gg, f in ((0, fu), (1, fv), (2, fp)):
        if f is None:
            continue
        m = act & (g == gg)
        x[m] = f(X[m], Y[m])
    return x, g, t, X, Y


def _internal(g, t, grid):
    return (g == grid) & (t == W.INTERNAL)


def test_convective_exact_for_affine_velocity():
    rng = np.random.default_rng(11)
    for case, N in (("circle", 32), ("flower5", 64), ("nobody", 32)):
        o, phi, st = make_oracle(case, N)
        assert st == 0, o.error()
        a, b = _affine(rng), _affine(rng)
        fu = lambda X, Y: a[0] + a[1] * X + a[2] * Y
        fv = lambda X, Y: b[0] + b[1] * X + b[2] * Y
        x, g, t, X, Y = _fields(o, fu, fv)
        out = o.convective(x)
        mu, mv = _internal(g, t, 0), _internal(g, t, 1)
        exu = fu(X[mu], Y[mu]) * a[1] + fv(X[mu], Y[mu]) * a[2]
        exv = fu(X[mv], Y[mv]) * b[1] + fv(X[mv], Y[mv]) * b[2]
        assert np.abs(out[mu] - exu).max() < 1e-12
        assert np.abs(out[mv] - exv).max() < 1e-12
        # every other slot is zero
        assert np.all(out[~(mu | mv)] == 0.0)
        # the pin separates the four-point cross average from a two-point
        # one: that would be off by |a_y b_y| h / 2 at every u node
        assert abs(a[2] * b[2]) * o.h / 2 > 1e3 * 1e-12


def test_convective_exact_for_quadratic_component():
    # u biquadratic, v affine: central differences of u are exact and the
    # averaged v is exact, so u.grad u at u nodes is exact; symmetrically
    # for v biquadratic and u affine at v nodes
    rng = np.random.default_rng(12)
    o, phi, st = make_oracle("circle_off", 64)
    assert st == 0, o.error()
    cq = rng.standard_normal((3, 3))
    q = lambda X, Y: sum(cq[m, n] * X ** m * Y ** n for m in range(3) for n in range(3))
    qx = lambda X, Y: sum(m * cq[m, n] * X ** (m - 1) * Y ** n for m in range(1, 3) for n in range(3))
    qy = lambda X, Y: sum(n * cq[m, n] * X ** m * Y ** (n - 1) for m in range(3) for n in range(1, 3))
    b = _affine(rng)
    lin = lambda X, Y: b[0] + b[1] * X + b[2] * Y
    x, g, t, X, Y = _fields(o, q, lin)
    out = o.convective(x)
    mu = _internal(g, t, 0)
    ex = q(X[mu], Y[mu]) * qx(X[mu], Y[mu]) + lin(X[mu], Y[mu]) * qy(X[mu], Y[mu])
    assert np.abs(out[mu] - ex).max() < 1e-11
    x, g, t, X, Y = _fields(o, lin, q)
    out = o.convective(x)
    mv = _internal(g, t, 1)
    ex = lin(X[mv], Y[mv]) * qx(X[mv], Y[mv]) + q(X[mv], Y[mv]) * qy(X[mv], Y[mv])
    assert np.abs(out[mv] - ex).max() < 1e-11


def _biquad(rng):
    c = rng.standard_normal((3, 3))
    f = lambda X, Y: sum(c[m, n] * X ** m * Y ** n for m in range(3) for n in range(3))
    lap = lambda X, Y: sum(c[m, n] * (m * (m - 1) * X ** max(m - 2, 0) * Y ** n
                                      + n * (n - 1) * X ** m * Y ** max(n - 2, 0))
                           for m in range(3) for n in range(3))
    return f, lap


def test_cn_rhs_exact_for_biquadratic_state():
    rng = np.random.default_rng(13)
    for case, N in (("circle", 32), ("flower5", 64)):
        o, phi, st = make_oracle(case, N, alpha=0.37 * (1.0 / 64))
        assert st == 0, o.error()
        fu, lu = _biquad(rng)
        fv, lv = _biquad(rng)
        xn, g, t, X, Y = _fields(o, fu, fv)
        n = xn.size
        f = rng.standard_normal(n)
        Nh = rng.standard_normal(n)
        bc = rng.standard_normal(n)
        dt = 0.013
        b = o.cn_rhs(xn, Nh, dt, f=f, bc=bc)
        mu, mv = _internal(g, t, 0), _internal(g, t, 1)
        for m, fx, lx in ((mu, fu, lu), (mv, fv, lv)):
            ex = fx(X[m], Y[m]) + o.alpha * lx(X[m], Y[m]) + dt * f[m] - dt * Nh[m]
            assert np.abs(b[m] - ex).max() < 1e-11
        # continuity rows and the mean row are 0
        assert np.all(b[_internal(g, t, 2)] == 0.0) and b[-1] == 0.0
        # boundary rows: the given values on Eq. (BCu) rows, walls and box
        # ghosts; 0 on extrapolation and copy rows and on pressure ghosts
        gh = o.ghosts(0)
        for gg, ii, jj, kd in zip(gh["grid"], gh["i"], gh["j"], gh["kind"]):
            k = W.flat_index(N, gg, ii, jj)
            assert b[k] == (bc[k] if (gg < 2 and kd == 0) else 0.0)
        for tt in (W.WALL, W.BOXGHOST):
            m = (t == tt) & (g >= 0)
            assert np.array_equal(b[m], bc[m])


def test_cn_rhs_rigid_body_and_walls():
    o, phi, st = make_oracle("circle_off", 64)
    assert st == 0, o.error()
    n = o.n()
    body = (0.3, -0.7, 1.9, 0.2, 0.0)
    walls = (0.11, 1.0, -0.4, 0.25)
    b = o.cn_rhs(np.zeros(n), np.zeros(n), 0.01, body=body, walls=walls)
    gh = o.ghosts(0)
    U, V, om, cx, cy = body
    for gg, ii, jj, kd, B in zip(gh["grid"], gh["i"], gh["j"], gh["kind"], gh["B"]):
        if gg == 2 or kd != 0:
            continue
        k = W.flat_index(o.N, gg, ii, jj)
        ub = U - om * (B[1] - cy) if gg == 0 else V + om * (B[0] - cx)
        assert abs(b[k] - ub) < 1e-15
    N = o.N
    for i in range(1, N):
        assert b[W.flat_index(N, 0, i, -1)] == walls[0]
        assert b[W.flat_index(N, 0, i, N)] == walls[1]
    for j in range(1, N):
        assert b[W.flat_index(N, 1, -1, j)] == walls[2]
        assert b[W.flat_index(N, 1, N, j)] == walls[3]
    # wall-normal velocities on the walls are 0
    for j in range(N):
        assert b[W.flat_index(N, 0, 0, j)] == 0.0 and b[W.flat_index(N, 0, N, j)] == 0.0


def _matrix(o):
    ri, ci, v = o.assemble(0)
    n = o.n()
    return sp.csc_matrix((v, (ri, ci)), shape=(n, n))


def _state(o, seed):
    """A smooth state with ghost values: Taylor-Green velocity scaled, p 0."""
    ex = W.taylor_green()
    x, g, t, X, Y = _fields(o, lambda X, Y: 0.5 * ex.u(2 * X, 2 * Y), lambda X, Y: 0.5 * ex.v(2 * X, 2 * Y))
    return x


def test_extrapolation_is_exact_for_linear_history():
    o, phi, st = make_oracle("circle", 32, alpha=1.0 / 16 / 2.0)
    assert st == 0, o.error()
    n = o.n()
    t = o.types(0).astype(int)
    xn = _state(o, 0)
    Nn = o.convective(xn)
    D = W.random_flat(o.N, t, 5) * 0.3       # dt dN/dt of the linear history
    N1, N2 = Nn - D, Nn - 2.0 * D             # N at t^(n-1), t^(n-2)
    dt = 1.0 / 16
    stt, x1, N1o, N2o, info = o.cn_step(xn.copy(), N1, N2, 2, dt, tol=1e-13)
    assert stt == 0
    # the history's value at t^(n+1/2)
    b = o.cn_rhs(xn, Nn + 0.5 * D, dt)
    xd = spla.spsolve(_matrix(o), b)
    act = t != W.INACTIVE
    vel = act & (np.arange(n) < n - 1 - o.N ** 2)
    assert np.abs(x1[vel] - xd[vel]).max() < 1e-10 * max(1.0, np.abs(xd[vel]).max())
    # a sign slip (N^n - N^(n-1)/2 + N^(n-2)/2) would give the value at t^(n-1/2)
    bw = o.cn_rhs(xn, Nn - 0.5 * D, dt)
    xw = spla.spsolve(_matrix(o), bw)
    assert np.abs(xw[vel] - xd[vel]).max() > 1e-4
    # history rotated: N1 <- N^n, N2 <- N^(n-1)
    assert np.array_equal(N1o, Nn) and np.array_equal(N2o, N1)


def test_picard_stops_on_iterativeNS_and_reaches_the_midpoint_fixed_point():
    o, phi, st = make_oracle("circle", 32, alpha=1.0 / 16 / 2.0)
    assert st == 0, o.error()
    t = o.types(0).astype(int)
    g = W.flat_coords(o.N, o.x0, o.y0, o.len)[0]
    mom = ((g == 0) | (g == 1)) & (t == W.INTERNAL)
    xn = _state(o, 0)
    dt = 1.0 / 16
    A = _matrix(o)
    Nn = o.convective(xn)
    ftil = o.cn_rhs(xn, np.zeros_like(xn), dt)
    fmax = np.abs(ftil[mom]).max()
    for eps in (1e-3, 1e-6):
        stt, x1, _, _, info = o.cn_step(xn.copy(), np.zeros_like(xn), np.zeros_like(xn), 0, dt, tol=1e-13,
                                        eps=eps, kmax=30)
        assert stt == 0 and 1 <= info[0] < 30
        # Eq. (iterativeNS) at the returned state, with its own new convective term
        b = o.cn_rhs(xn, 0.5 * (Nn + o.convective(x1)), dt)
        res = np.abs((b - A @ x1)[mom]).max()
        assert res < eps * max(1.0, fmax)
    # tight eps: the mid-point fixed point x = M^-1 b((N(x^n) + N(x)) / 2)
    stt, x1, _, _, info = o.cn_step(xn.copy(), np.zeros_like(xn), np.zeros_like(xn), 0, dt, tol=1e-13,
                                    eps=1e-12, kmax=60)
    assert stt == 0
    xf = spla.spsolve(A, o.cn_rhs(xn, 0.5 * (Nn + o.convective(x1)), dt))
    act = (t != W.INACTIVE) & (g >= 0) & (g < 2)
    assert np.abs(x1[act] - xf[act]).max() < 1e-9
    # and it is not the state of a single solve with N^n alone
    x0 = spla.spsolve(A, o.cn_rhs(xn, Nn, dt))
    assert np.abs(x0[act] - xf[act]).max() > 1e-6
