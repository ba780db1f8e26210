"""Pins of the 3-D MAC oracle (box domain) against mathematics, not itself.

* Polynomial exactness: for quadratic velocities and a linear pressure every
  row of the discrete system (momentum with the 7-point Laplacian, continuity,
  wall and box-ghost rows, the mean row) is exact, so the sampled field has
  zero residual against the right-hand side built from the continuous
  operator (Eqs. NSCN1, spaceprob in 3-D).
* The box solve makes the rows of every box of the colour just relaxed exact.
* The seven colours (i + 2j + 3k) mod 7 are conflict free: every offset at
  which two boxes share or read each other's unknowns is nonzero mod 7.
* Transfers: the restriction reproduces linear fields at interior coarse
  nodes; the prolongation reproduces linear coarse corrections in the interior.
* Multigrid reaches the dense solve of the assembled matrix.
* Among the wall and box-ghost rows the assembled matrix is diagonal, and a
  box-ghost row's other columns are interior nodes.
"""
import itertools

import numpy as np
import pytest

from oracle import mac3d as M


def coords(o, g, lev=0):
    N = o.N >> lev
    h = 1.0 / N
    r = np.arange(-1, N + 1)
    K, J, I = np.meshgrid(r, r, r, indexing="ij")
    off = [0.5, 0.5, 0.5]
    if g < 3:
        off[g] = 0.0
    return (I + off[0]) * h, (J + off[1]) * h, (K + off[2]) * h


def quad(c, x, y, z):
    # quadratic polynomial with coefficients c (10 of them)
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z + c[7] * x * y +
            c[8] * y * z + c[9] * x * z)


def lap_quad(c):
    return 2 * (c[4] + c[5] + c[6])


def grad_quad(c, x, y, z):
    return (c[1] + 2 * c[4] * x + c[7] * y + c[9] * z, c[2] + 2 * c[5] * y + c[7] * x + c[8] * z,
            c[3] + 2 * c[6] * z + c[8] * y + c[9] * x)


@pytest.mark.parametrize("N", [6, 8])
def test_polynomial_exactness(N):
    rng = np.random.default_rng(N)
    alpha = 0.37 / N ** 2
    o = M.Mac3D(N, alpha, 1)
    h = 1.0 / N
    cu = [rng.standard_normal(10) for _ in range(3)]
    cp = rng.standard_normal(4)
    pf = lambda x, y, z: cp[0] + cp[1] * x + cp[2] * y + cp[3] * z
    n = o.n()
    x = np.zeros(n)
    b = np.zeros(n)
    (xu, xv, xw, xp), xxi = o.split(x)
    (bu, bv, bw, bp), bm = o.split(b)
    t = o.types[0]
    for g, (xa, ba) in enumerate([(xu, bu), (xv, bv), (xw, bw)]):
        X, Y, Z = coords(o, g)
        val = quad(cu[g], X, Y, Z)
        act = t[g] != M.INACTIVE
        xa[act] = val[act]
        m = t[g] == M.INTERNAL
        # u - alpha lap u + dp/dx_g (the CN operator applied to the exact field)
        ba[m] = (val - alpha * lap_quad(cu[g]) + cp[1 + g])[m]
        m = t[g] == M.WALL
        ba[m] = val[m]
        # box-ghost rows: the exact value at the wall point between ghost and first node
        m = t[g] == M.BOXGHOST
        for ax in range(3):
            if ax == g:
                continue
            Xw = [X, Y, Z]
            for side, wall in ((0, 0.0), (N + 1, 1.0)):
                sel = np.zeros_like(m)
                idx = [slice(None)] * 3
                idx[2 - ax] = side
                sel[tuple(idx)] = True
                mm = m & sel
                P = [Xw[0].copy(), Xw[1].copy(), Xw[2].copy()]
                P[ax] = np.full_like(P[ax], wall)
                ba[mm] = quad(cu[g], *P)[mm]
    X, Y, Z = coords(o, 3)
    pv = pf(X, Y, Z)
    act = t[3] == M.INTERNAL
    xp[act] = pv[act]
    # continuity: the exact divergence at the cell centre (xi = 0)
    div = sum(grad_quad(cu[g], X, Y, Z)[g] for g in range(3))
    bp[act] = div[act]
    bm[0] = h ** 3 * xp[act].sum()
    r, nrm = o.residual(x, b)
    assert nrm <= 1e-11 * (1 + np.abs(b).max()), nrm


def test_box_rows_exact_after_their_colour():
    N = 8
    o = M.Mac3D(N, 0.4 / N ** 2, 1)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(o.n())
    b = rng.standard_normal(o.n())
    x2 = o.box_sweep(x, b)
    r, _ = o.residual(x2, b)
    S = N + 2
    F = S ** 3
    slot = lambda i, j, k: ((k + 1) * S + (j + 1)) * S + (i + 1)
    t = o.types[0].reshape(-1)
    worst = 0.0
    for k, j, i in itertools.product(range(N), range(N), range(N)):
        if M.colour(i, j, k) != M.NCOL - 1:
            continue
        rows = [M.G_U * F + slot(i, j, k), M.G_U * F + slot(i + 1, j, k), M.G_V * F + slot(i, j, k),
                M.G_V * F + slot(i, j + 1, k), M.G_W * F + slot(i, j, k), M.G_W * F + slot(i, j, k + 1)]
        rows = [rw for rw in rows if t[rw] == M.INTERNAL] + [M.G_P * F + slot(i, j, k)]
        worst = max(worst, np.abs(r[rows]).max())
    assert worst <= 1e-12


def test_seven_colours_are_conflict_free():
    # two boxes conflict when one writes a face or pressure that the other's
    # rows read or write: a common face or neighbouring face stencil along
    # one axis (offsets up to 2), or a face stencil in a transverse direction
    # (offsets of one along two axes)
    offs = set()
    for ax in range(3):
        for d in (1, 2):
            for s in (-1, 1):
                o = [0, 0, 0]
                o[ax] = s * d
                offs.add(tuple(o))
    for a1, a2 in itertools.combinations(range(3), 2):
        for s1, s2 in itertools.product((-1, 1), repeat=2):
            o = [0, 0, 0]
            o[a1], o[a2] = s1, s2
            offs.add(tuple(o))
    assert len(offs) == 6 + 6 + 12
    for o in offs:
        assert M.colour(*o) != 0, o


def test_transfers_linear_fields():
    N = 16
    o = M.Mac3D(N, 1.0 / N ** 2, 2)
    n0, n1 = o.n(0), o.n(1)
    c = np.array([0.3, -1.1, 0.7, 2.0])
    f = lambda X, Y, Z: c[0] + c[1] * X + c[2] * Y + c[3] * Z
    # restriction of a linear field sampled on interior rows: the field at the coarse node
    r = np.zeros(n0)
    parts, _ = o.split(r, 0)
    for g in range(4):
        parts[g][...] = f(*coords(o, g, 0))
    rH = o.restrict(r, 0)
    partsH, _ = o.split(rH, 1)
    tH = o.types[1]
    for g in range(4):
        want = f(*coords(o, g, 1))
        m = tH[g] == M.INTERNAL
        # interior coarse nodes whose whole fine stencil is interior
        inner = np.zeros_like(m)
        inner[2:-2, 2:-2, 2:-2] = True
        m &= inner
        assert m.any()
        assert np.abs(partsH[g][m] - want[m]).max() <= 1e-12
    # prolongation of a linear coarse field: the field at interior fine nodes
    e = np.zeros(n1)
    pe, _ = o.split(e, 1)
    for g in range(4):
        pe[g][...] = np.where(tH[g] != M.INACTIVE, f(*coords(o, g, 1)), 0.0)
    x = o.prolong(e, np.zeros(n0), 0)
    px, _ = o.split(x, 0)
    t0 = o.types[0]
    for g in range(4):
        want = f(*coords(o, g, 0))
        m = t0[g] == M.INTERNAL
        inner = np.zeros_like(m)
        inner[3:-3, 3:-3, 3:-3] = True
        m &= inner
        assert np.abs(px[g][m] - want[m]).max() <= 1e-12


def test_multigrid_reaches_the_dense_solution_and_converges_fast():
    N = 8
    o = M.Mac3D(N, 2.0 / N ** 2, 2)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(o.n())
    act = np.concatenate([o.types[0].reshape(-1) != M.INACTIVE, [True]])
    b[~act] = 0.0
    x, hist = o.solve(np.zeros(o.n()), b, 1e-10, 40)
    assert hist[-1] <= 1e-10
    xd = np.linalg.solve(o.assemble(0), b)
    assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
    # the box domain keeps the textbook rate of a box smoother (three relaxations)
    rho = (hist[-1] / hist[-5]) ** 0.25
    assert rho < 0.25, rho


@pytest.mark.parametrize("N", [4, 8])
def test_wall_and_box_ghost_rows_read_no_other_of_their_kind(N):
    # on the box domain a wall row (x = b) reads only its own node and a
    # box-ghost row (3/8, 3/4, -1/8 along the axis that leaves the box) its
    # own node and two interior nodes, so among these rows the matrix is
    # diagonal: lambda Jacobi sweeps over them equal lambda updates of each
    # row in turn, which the GPU's one-launch ghost sweeps rely on
    o = M.Mac3D(N, 2.0 / N ** 2, 1)
    A = o.assemble(0)
    t = o.types[0]
    rows = np.flatnonzero(np.concatenate([np.isin(t[:3].reshape(-1), (M.WALL, M.BOXGHOST)),
                                          np.zeros(t[3].size + 1, bool)]))
    assert rows.size == 3 * (6 * N * N - 4 * N)
    sub = A[np.ix_(rows, rows)]
    assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0
    assert np.all(np.diag(sub) != 0.0)
    # and the other nodes a box-ghost row reads are interior
    box = np.flatnonzero(np.concatenate([t[:3].reshape(-1) == M.BOXGHOST, np.zeros(t[3].size + 1, bool)]))
    internal = np.concatenate([t.reshape(-1) == M.INTERNAL, [False]])
    for e in box:
        cols = np.flatnonzero(A[e])
        assert np.all(internal[cols[cols != e]])
