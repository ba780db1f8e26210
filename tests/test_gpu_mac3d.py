"""The 3-D MAC extension on the GPU (gp3_* through the C ABI) against the 3-D
oracle (oracle/mac3d.py) on the same seeded inputs, and against mathematics
alone (the polynomial field the discrete system reproduces exactly)."""
import numpy as np
import pytest

from oracle import mac3d as M

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


def pair(N, levels, ah2=2.0):
    from paper_1911_00994_gb300 import mac3d
    alpha = ah2 / N ** 2
    o = M.Mac3D(N, alpha, levels)
    s = mac3d.Solver3D(N, levels, alpha)
    return o, s


def rand_vec(o, lev, seed, scale=1.0):
    # normals on the active rows of the level, zero elsewhere (plain layout)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(o.n(lev)) * scale
    act = np.concatenate([o.types[lev].reshape(-1) != M.INACTIVE, [True]])
    v[~act] = 0.0
    return v


@pytest.mark.parametrize("N,levels", [(16, 3), (24, 4)])
def test_types_and_pieces_match(N, levels):
    o, s = pair(N, levels)
    for lev in range(levels):
        assert np.array_equal(s.types(lev), o.types[lev].reshape(-1).astype(np.uint8)), lev
    for lev in range(levels - 1):
        x, b = rand_vec(o, lev, 10 + lev), rand_vec(o, lev, 20 + lev, 5.0)
        xg, bg = s.to_device(x, lev), s.to_device(b, lev)
        r_o, n_o = o.residual(x, b, lev)
        r_g, n_g = s.residual(xg, bg, lev)
        assert rel(s.to_flat(r_g, lev), r_o) <= 1e-13, lev
        assert abs(n_g - n_o) <= 1e-13 * n_o
        for nu in (1, 2):
            want = o.smooth(x, b, nu, lev)
            xs = s.to_device(x, lev)
            s.smooth(xs, bg, nu, lev)
            assert rel(s.to_flat(xs, lev), want) <= 1e-11, (lev, nu)
        bH = s.restrict(s.to_device(r_o, lev), lev)
        assert rel(s.to_flat(bH, lev + 1), o.restrict(r_o, lev)) <= 1e-13, lev
        e = rand_vec(o, lev + 1, 30 + lev)
        xp = s.to_device(x, lev)
        s.prolong(s.to_device(e, lev + 1), xp, lev)
        assert rel(s.to_flat(xp, lev), o.prolong(e, x, lev)) <= 1e-13, lev


def test_cycles_match_the_oracle():
    o, s = pair(16, 3)
    b = rand_vec(o, 0, 3)
    x = np.zeros_like(b)
    xg, bg = s.to_device(x), s.to_device(b)
    for k in range(3):
        x = o.cycle(x, b)
        s.cycle(xg, bg)
        assert rel(s.to_flat(xg), x) <= 1e-10, k


def test_solve_matches_the_dense_solve():
    o, s = pair(8, 2)
    b = rand_vec(o, 0, 4)
    xd = np.linalg.solve(o.assemble(0), b)
    xg = s.new_vec()
    st, cyc, res, hist = s.solve(xg, s.to_device(b), 1e-12, 60)
    assert st == 0, s.error()
    assert rel(s.to_flat(xg), xd) <= 1e-10
    # and the oracle's multigrid takes the same number of cycles
    xo, ho = o.solve(np.zeros_like(b), b, 1e-12, 60)
    assert abs(len(ho) - 1 - cyc) <= 1


def test_polynomial_field_is_the_discrete_solution():
    # quadratic velocities and a linear pressure satisfy every row exactly
    # (7-point Laplacian, central differences, the 3/8 3/4 -1/8 wall rows),
    # so the GPU's converged solution is the sampled field (pressure up to the
    # mean the mean row fixes) without reference to the oracle's arithmetic
    from paper_1911_00994_gb300 import mac3d
    N, levels = 16, 3
    alpha = 1.3 / N ** 2
    s = mac3d.Solver3D(N, levels, alpha)
    rng = np.random.default_rng(5)
    S = N + 2
    F = S ** 3
    h = 1.0 / N
    t = s.types(0).reshape(4, S, S, S)
    r = np.arange(-1, N + 1)
    K, J, I = np.meshgrid(r, r, r, indexing="ij")
    cu = [rng.standard_normal(10) for _ in range(3)]
    cp = rng.standard_normal(4)

    def q(c, x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z + c[7] * x * y +
                c[8] * y * z + c[9] * x * z)

    def grad(c, x, y, z):
        return (c[1] + 2 * c[4] * x + c[7] * y + c[9] * z, c[2] + 2 * c[5] * y + c[7] * x + c[8] * z,
                c[3] + 2 * c[6] * z + c[8] * y + c[9] * x)

    xe = np.zeros(4 * F + 1)
    b = np.zeros(4 * F + 1)
    for g in range(3):
        off = [0.5, 0.5, 0.5]
        off[g] = 0.0
        X, Y, Z = (I + off[0]) * h, (J + off[1]) * h, (K + off[2]) * h
        val = q(cu[g], X, Y, Z)
        tg = t[g]
        xg_ = np.where(tg != 0, val, 0.0)
        bg_ = np.zeros_like(val)
        m = tg == 1
        bg_[m] = (val - alpha * 2 * (cu[g][4] + cu[g][5] + cu[g][6]) + cp[1 + g])[m]
        m = tg == 3
        bg_[m] = val[m]
        m = tg == 4
        for ax, A in enumerate((I, J, K)):
            if ax == g:
                continue
            for side, wall in ((-1, 0.0), (N, 1.0)):
                mm = m & (A == side)
                P = [X.copy(), Y.copy(), Z.copy()]
                P[ax] = np.full_like(P[ax], wall)
                bg_[mm] = q(cu[g], *P)[mm]
        xe[g * F:(g + 1) * F] = xg_.reshape(-1)
        b[g * F:(g + 1) * F] = bg_.reshape(-1)
    X, Y, Z = (I + 0.5) * h, (J + 0.5) * h, (K + 0.5) * h
    pv = cp[0] + cp[1] * X + cp[2] * Y + cp[3] * Z
    cell = t[3] == 1
    p = np.where(cell, pv, 0.0)
    xe[3 * F:4 * F] = p.reshape(-1)
    div = sum(grad(cu[g], X, Y, Z)[g] for g in range(3))
    b[3 * F:4 * F] = np.where(cell, div, 0.0).reshape(-1)
    b[4 * F] = h ** 3 * p[cell].sum()
    xg = s.new_vec()
    st, cyc, res, hist = s.solve(xg, s.to_device(b), 1e-11, 80)
    assert st == 0, s.error()
    assert rel(s.to_flat(xg), xe) <= 1e-9


@pytest.mark.parametrize("inner", [1, 4])
def test_mixed_precision_solve_reaches_the_fp64_solution(inner):
    # FP32 cycles inside FP64 residual correction (the spec precision
    # scheme): the oracle's FP64 solution to the tolerance, with at most one
    # correction's worth of cycles more than the FP64 cycles
    from paper_1911_00994_gb300 import mac3d
    N, levels = 16, 3
    alpha = 2.0 / N ** 2
    o = M.Mac3D(N, alpha, levels)
    b = rand_vec(o, 0, 6)
    xo, ho = o.solve(np.zeros_like(b), b, 1e-12, 60)
    s64 = mac3d.Solver3D(N, levels, alpha)
    x64 = s64.new_vec()
    st, c64, r64, h64 = s64.solve(x64, s64.to_device(b), 1e-10, 80)
    assert st == 0, s64.error()
    s = mac3d.Solver3D(N, levels, alpha, precision=1, inner=inner)
    xg = s.new_vec()
    st, cyc, res, hist = s.solve(xg, s.to_device(b), 1e-10, 80)
    assert st == 0, s.error()
    assert res <= 1e-10 and hist[-1] <= 1e-10
    assert rel(s.to_flat(xg), xo) <= 1e-8
    assert cyc <= c64 + inner
    # one FP64 residual per correction: fewer than cycles once corrections run several
    if inner > 1:
        assert len(hist) - 1 < cyc
