"""Crank-Nicolson step (Sect. 2) on the GPU against the oracle: convective
term, right-hand side, and whole steps (mid-point Picard for steps 0 and 1,
extrapolation from step 2) of the 32^2 manufactured case (circle r = 0.5 on
[-1, 1]^2, Re = 1, dt = h, Taylor-Green velocity with the forcing that keeps it steady).
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


def setup(case, N, Re=1.0):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    h = L / N
    dt = h
    alpha = dt / (2 * Re)
    lev = levels_for(N)
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=lev)
    assert st == 0
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha)
    assert s.geometry(phi) == 0, s.error()
    return o, s, dt


def tg_forcing(Re):
    s, c = np.sin, np.cos
    fu = lambda x, y: 0.5 * np.sin(2 * x) + c(x) * s(y) + 2.0 * s(x) * c(y) / Re
    fv = lambda x, y: 0.5 * np.sin(2 * y) + s(x) * c(y) - 2.0 * c(x) * s(y) / Re
    return fu, fv


@pytest.mark.parametrize("case,N", [("circle", 32), ("flower5", 128)])
def test_convective_and_rhs_match(case, N):
    o, s, dt = setup(case, N)
    t = o.types()
    x = W.random_flat(N, t, 3)
    Nh = W.random_flat(N, t, 4)
    f = W.random_flat(N, t, 5)
    bc = W.random_flat(N, t, 6)
    want = o.convective(x)
    got = s.to_flat(s.convective(s.to_device(x)))
    g = W.flat_coords(N, 0, 0, 1)[0]
    m = g < 2
    assert rel(got[m], want[m]) < 1e-13
    for kw in (dict(bc=bc), dict(body=(0.3, -0.2, 1.1, 0.01, 0.02), walls=(0.5, 1.0, -0.25, 0.75))):
        want = o.cn_rhs(x, Nh, dt, f=f, **kw)
        kd = {k: (s.to_device(v) if k == "bc" else v) for k, v in kw.items()}
        got = s.to_flat(s.cn_rhs(s.to_device(x), s.to_device(Nh), dt, f=s.to_device(f), **kd))
        assert rel(got, want) < 1e-13


def test_circle32_cn_steps_match_oracle():
    Re = 1.0
    o, s, dt = setup("circle", 32, Re)
    N, x0, L = 32, -1.0, 2.0
    ex = W.taylor_green()
    t = o.types()
    gh = o.ghosts()
    bvec = W.manufactured_rhs(ex, N, x0, x0, L, o.alpha, t, gh["grid"], gh["i"], gh["j"], gh["B"], gh["kind"])
    xe = W.exact_flat(ex, N, x0, x0, L, t)
    x_init = xe.copy()
    g, i, j, X, Y = W.flat_coords(N, x0, x0, L)
    x_init[g == 2] *= dt  # the unknown is dt * p
    fu, fv = tg_forcing(Re)
    f = np.zeros_like(xe)
    f[g == 0] = fu(X[g == 0], Y[g == 0])
    f[g == 1] = fv(X[g == 1], Y[g == 1])
    # boundary values: the exact velocity (the same entries as the manufactured rhs)
    bc = bvec
    xo, N1o, N2o = x_init.copy(), np.zeros_like(xe), np.zeros_like(xe)
    xg, N1g, N2g = s.to_device(x_init), s.new_vec(), s.new_vec()
    fd, bcd = s.to_device(f), s.to_device(bc)
    for step in range(4):
        st, xo, N1o, N2o, info = o.cn_step(xo, N1o, N2o, step, dt, f=f, bc=bc, tol=1e-12)
        assert st == 0
        st, rep = s.cn_step(xg, N1g, N2g, step, dt, Re, f=fd, bc=bcd, tol=1e-12)
        assert st == 0, s.error()
        assert rep.picard == int(info[0]) or step >= 2
        assert rel(s.to_flat(xg), xo) < 1e-9, step
        assert rel(s.to_flat(N1g)[g < 2], N1o[g < 2]) < 1e-9
    # the scheme keeps the steady solution to discretisation accuracy
    m = (t == O.INTERNAL) & (g < 2)
    assert np.abs(xo[m] - xe[m]).max() < 5e-3
