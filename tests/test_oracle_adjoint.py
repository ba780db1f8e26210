"""Pins of the oracle's adjoint (transposed system M^T lam = c and the
transposed multigrid cycle) against the forward oracle and linear algebra.

Every forward stage used here (matrix-free residual, restriction,
interpolation, box sweep, (xi, mean) update, ghost sweep, relaxation, cycle)
is already pinned by test_oracle_pins.py; the transposed code is separate
code, and the identity <F b, c> = <b, F^T c> for random b, c fails for a
dropped term, a wrong sign, a wrong colour order or a transposed box solved
untransposed.  The adjoint solve is checked against a dense solve of the
assembled matrix's transpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle, manufactured

GEOMS = [("circle", 32, None), ("flower5", 64, 2.0), ("circle_off", 64, None), ("ellipse", 64, 8.0)]


def build(case, N, ah2, **kw):
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2.0 if ah2 is None else ah2 * h * h
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=levels_for(N), **kw)
    assert st == 0, o.error()
    return o


def close(a, b, tol):
    return abs(a - b) <= tol * max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("case,N,ah2", GEOMS)
def test_transposed_operator(case, N, ah2):
    o = build(case, N, ah2)
    rng = np.random.default_rng(1)
    for lev in range(o.levels):
        n = o.n(lev)
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        mx, _ = o.residual(x, np.zeros(n), lev)       # -M x (matrix-free rows)
        mty, _ = o.residual_t(y, np.zeros(n), lev)    # -M^T y (columns)
        assert close(np.dot(mx, y), np.dot(x, mty), 1e-13), lev


@pytest.mark.parametrize("case,N,ah2", GEOMS)
def test_transposed_transfers(case, N, ah2):
    o = build(case, N, ah2)
    rng = np.random.default_rng(2)
    for lev in range(o.levels - 1):
        n, nH = o.n(lev), o.n(lev + 1)
        r, yH = rng.standard_normal(n), rng.standard_normal(nH)
        assert close(np.dot(o.restrict(r, lev), yH), np.dot(r, o.restrict_t(yH, np.zeros(n), lev)), 1e-13)
        y = rng.standard_normal(n)
        assert close(np.dot(o.prolong(yH, np.zeros(n), lev), y), np.dot(yH, o.prolong_t(y, lev)), 1e-13)


@pytest.mark.parametrize("case,N,ah2", GEOMS)
def test_transposed_relaxation_stages(case, N, ah2):
    # one stage from zero is the linear map b -> Q b (Q of the stage's
    # x += Q (b - M x)); its transpose from zero is c -> Q^T c
    o = build(case, N, ah2)
    rng = np.random.default_rng(3)
    for lev in range(o.levels):
        n = o.n(lev)
        b, c = rng.standard_normal(n), rng.standard_normal(n)
        z = np.zeros(n)
        for fwd, tr in (("box_sweep", "box_sweep_t"), ("scalar_update", "scalar_update_t"),
                        ("ghost_sweep", "ghost_sweep_t")):
            Fb, Tc = getattr(o, fwd)(z, b, lev), getattr(o, tr)(z, c, lev)
            assert close(np.dot(Fb, c), np.dot(b, Tc), 1e-12), (fwd, lev)
        Fb, Tc = o.smooth(z, b, 2, lev), o.smooth_t(z, c, 2, lev)
        assert close(np.dot(Fb, c), np.dot(b, Tc), 1e-12), lev


@pytest.mark.parametrize("case,N,ah2,gamma", [g + (1,) for g in GEOMS] + [("flower5", 64, 2.0, 2)])
def test_transposed_cycle(case, N, ah2, gamma):
    o = build(case, N, ah2, gamma=gamma)
    rng = np.random.default_rng(4)
    n = o.n(0)
    b, c = rng.standard_normal(n), rng.standard_normal(n)
    st, Bb = o.cycle(np.zeros(n), b)
    assert st == 0
    st, Cc = o.cycle_t(np.zeros(n), c)
    assert st == 0
    # relative to |Bb| |c|: the dot product itself can be a small difference
    # of large terms
    scale = np.linalg.norm(Bb) * np.linalg.norm(c)
    assert abs(np.dot(Bb, c) - np.dot(b, Cc)) <= 1e-13 * scale


@pytest.mark.parametrize("case,N,ah2", [("circle", 32, None), ("flower5", 64, 2.0), ("circle_off", 64, None)])
def test_adjoint_solve_matches_dense_transpose(case, N, ah2):
    o = build(case, N, ah2)
    n = o.n(0)
    A = o.dense_matrix(0)
    c = np.random.default_rng(5).standard_normal(n)
    st, lam, hist = o.solve_t(np.zeros(n), c, 1e-11, 200)
    assert st == 0
    ref = np.linalg.solve(A.T, c)
    assert np.abs(lam - ref).max() <= 1e-9 * np.abs(ref).max()
    # the transposed cycle has the forward cycle's spectrum: about as many
    # cycles as the forward solve of a system of the same size
    b, xe, t, gh = manufactured(o, W.taylor_green())
    st, x, hf = o.solve(np.zeros(n), b * (np.abs(c).max() / np.abs(b).max()), 1e-11, 200)
    assert st == 0
    assert abs(len(hist) - len(hf)) <= 6
