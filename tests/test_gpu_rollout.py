"""Adjoint of a rollout of Crank-Nicolson steps around the orbiting circle
(the orbiting circle: r = 0.25, orbit radius 0.2, period 1, Re = 100) on the GPU:
the gradient of a windowed kinetic energy with respect to the forcing and the
body-velocity amplitude, against the oracle's adjoint (same geometry arrays),
against central differences of the forward rollout, and with and without
checkpoints.  Steps 0 and 1 use 4 Picard iterations, later steps the
extrapolated convective term; dt = 0.3 h (inside the paper's time-step bound).
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_00994_gb300 import workloads as W
from tests._cases import levels_for

pytestmark = pytest.mark.gpu

X0, LEN, RE, K = -1.0, 2.0, 100.0, 4


def moving(t):
    cx, cy = 0.2 * np.cos(2 * np.pi * t), 0.2 * np.sin(2 * np.pi * t)
    U, V = -0.2 * 2 * np.pi * np.sin(2 * np.pi * t), 0.2 * 2 * np.pi * np.cos(2 * np.pi * t)
    return W.circle(0.25, cx, cy), (U, V, 0.0, cx, cy)


def window(N, n):
    w = np.zeros(n)
    nU = (N + 1) * (N + 2)
    k = np.arange(nU)
    ju, iu = k // (N + 1) - 1, k % (N + 1)
    w[:nU] = (iu >= 5 * N // 8) & (iu < 7 * N // 8) & (ju >= 3 * N // 8) & (ju < 5 * N // 8)
    return w


def momentum_mask(types, N):
    nU, nV = (N + 1) * (N + 2), (N + 2) * (N + 1)
    m = np.zeros(len(types), dtype=bool)
    m[:nU + nV] = types[:nU + nV] == O.INTERNAL
    return m


def test_rollout_gradient_matches_oracle():
    from paper_1911_00994_gb300 import gpmg
    N, steps = 32, 5
    h = LEN / N
    dt, tol = 0.3 * h, 5e-13
    lev = levels_for(N)
    o = O.Oracle(N, X0, X0, LEN, lev, dt / (2 * RE), band=3)
    s = gpmg.Solver(N, X0, X0, LEN, levels=lev, alpha=dt / (2 * RE), band=3, adjoint=True, max_cycles=400)
    phis = [W.phi_half_lattice(moving(m * dt)[0], N, X0, X0, LEN) for m in range(steps + 1)]
    assert o.geometry(phis[0]) == 0 and s.geometry(phis[0]) == 0
    n = o.n()
    f = np.where(momentum_mask(o.types(), N), np.random.default_rng(1234).standard_normal(n), 0.0)
    w = window(N, n)
    xo, N1o, N2o = np.zeros(n), np.zeros(n), np.zeros(n)
    xg, N1g, N2g = s.new_vec(), s.new_vec(), s.new_vec()
    fg = s.to_device(f)
    xs_o, xs_g = [xo], [xg.clone()]
    for m in range(steps):
        body = moving((m + 1) * dt)[1]
        assert o.geometry(phis[m + 1]) == 0 and s.geometry(phis[m + 1]) == 0
        st, xo, N1o, N2o, info = o.cn_step(xo, N1o, N2o, m, dt, f=f, body=body, tol=tol, eps=0.0, kmax=K)
        assert st == 0
        st, rep = s.cn_step(xg, N1g, N2g, m, dt, RE, f=fg, body=body, tol=tol, eps=0.0, kmax=K)
        assert st == 0, s.error()
        xs_o.append(xo)
        xs_g.append(xg.clone())
    assert np.abs(s.to_flat(xg) - xo).max() <= 1e-9 * np.abs(xo).max()
    xbo = 2.0 * w * xo
    nbo = [np.zeros(n), np.zeros(n), np.zeros(n)]
    fbo, abo = np.zeros(n), 0.0
    xbg = s.to_device(2.0 * w * s.to_flat(xg))
    nbg = [s.new_vec(), s.new_vec(), s.new_vec()]
    fbg, abg = s.new_vec(), 0.0
    for m in reversed(range(steps)):
        body = moving((m + 1) * dt)[1]
        assert o.geometry(phis[m + 1]) == 0 and s.geometry(phis[m + 1]) == 0
        st, xbo, abo = o.cn_step_adjoint(m, xs_o[m], dt, xbo, nbo, fbo, abo, f=f, body=body, tol=tol, kmax=K)
        assert st == 0
        nbo = [nbo[1], nbo[2], np.zeros(n)]
        xm = s.new_vec()
        abg += s.cn_step_adjoint(m, xs_g[m], dt, RE, xbg, xm, nbg, fbg, f=fg, body=body, tol=tol, kmax=K)
        xbg = xm
        nbg = [nbg[1], nbg[2], s.new_vec()]
    assert np.abs(s.to_flat(fbg) - fbo).max() <= 1e-7 * np.abs(fbo).max()
    assert abs(abg - abo) <= 1e-7 * abs(abo)
    assert np.abs(s.to_flat(xbg) - xbo).max() <= 1e-7 * np.abs(xbo).max()


def bumps(N, types, scale):
    # 4 seeded Gaussian bumps (sigma = 0.1) on internal u, v nodes, centres
    # outside the orbit's reach
    g, i, j, X, Y = W.flat_coords(N, X0, X0, LEN)
    rng = np.random.default_rng(1234)
    f = np.zeros(len(types))
    for _ in range(4):
        while True:
            c = rng.uniform(-0.9, 0.9, 2)
            if np.hypot(c[0], c[1]) > 0.55:
                break
        a = rng.standard_normal(2)
        bump = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (2 * 0.1 ** 2))
        f += np.where(g == 0, a[0] * bump, 0.0) + np.where(g == 1, a[1] * bump, 0.0)
    return scale * np.where(momentum_mask(types, N), f, 0.0)


# At N = 64 the body speed is scaled by AMP = 0.3: with the full speed 0.4 pi
# the cell Reynolds number |u| h Re is 3.9 and the central convective term of
# the explicit steps grows without bound within ten steps (oracle and GPU
# alike); at 0.3 it is 1.2.
AMP = 0.3


def make_rollout(N, steps, every, krylov=False):
    from paper_1911_00994_gb300 import gpmg
    from paper_1911_00994_gb300.rollout import Rollout
    dt = 0.3 * LEN / N
    s = gpmg.Solver(N, X0, X0, LEN, levels=levels_for(N), alpha=dt / (2 * RE), band=3, adjoint=True,
                    max_cycles=400, krylov=krylov)
    shape = dict(kind=gpmg.GP_CIRCLE, a=0.25, orbit_r=0.2, orbit_period=1.0)
    st, body = s.geometry_shape(t=0.0, **shape)
    assert st == 0, s.error()
    return s, Rollout(s, shape, dt, RE, steps, kmax=K, tol=1e-10, every=every)


def test_checkpoints_do_not_change_the_gradient():
    N, steps = 64, 7
    s, ro = make_rollout(N, steps, 3)
    t = s.types_flat()
    n = len(t)
    f = s.to_device(bumps(N, t, 0.1))
    w = s.to_device(window(N, n))
    L3, f3, a3 = ro.loss_and_gradient(f, AMP, w)
    ro.every = 100
    L0, f0, a0 = ro.loss_and_gradient(f, AMP, w)
    assert L3 == L0 and a3 == a0
    assert np.array_equal(s.to_flat(f3), s.to_flat(f0))


def test_krylov_rollout_gradient_matches_plain_cycles():
    # BiCGSTAB for the forward and the adjoint solves (both to 1e-10): the
    # same loss and gradient as the plain cycles, to the solves' tolerance
    N, steps = 64, 7
    out = []
    for kry in (False, True):
        s, ro = make_rollout(N, steps, 3, krylov=kry)
        t = s.types_flat()
        f = s.to_device(bumps(N, t, 0.1))
        w = s.to_device(window(N, len(t)))
        L, fb, ab = ro.loss_and_gradient(f, AMP, w)
        out.append((L, s.to_flat(fb), ab))
    (L0, f0, a0), (L1, f1, a1) = out
    assert abs(L1 - L0) <= 1e-8 * abs(L0)
    assert abs(a1 - a0) <= 1e-6 * abs(a0)
    assert np.abs(f1 - f0).max() <= 1e-6 * np.abs(f0).max()


def test_rollout_gradient_matches_finite_differences():
    # central differences with eps = 1e-3 on 4 seeded forcing directions (node
    # noise of size 0.1 on internal momentum rows) and the amplitude
    # (truncation O(eps^2); solves to 1e-10 keep their noise below the
    # compared digits); N = 64, 12 steps, checkpoints every 5 steps
    N, steps = 64, 12
    s, ro = make_rollout(N, steps, 5)
    t = s.types_flat()
    n = len(t)
    mom = momentum_mask(t, N)
    f0 = bumps(N, t, 0.1)
    w = s.to_device(window(N, n))
    L0, fbar, abar = ro.loss_and_gradient(s.to_device(f0), AMP, w)
    assert L0 > 0.0
    grad = s.to_flat(fbar)

    def L(f, amp):
        x = ro.forward(s.to_device(f), amp)
        return float((w * x * x).sum())

    eps = 1e-3
    for k in range(4):
        d = np.where(mom, 0.1 * np.random.default_rng(100 + k).standard_normal(n), 0.0)
        fd = (L(f0 + eps * d, AMP) - L(f0 - eps * d, AMP)) / (2 * eps)
        an = float(np.dot(grad, d))
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-12, (k, fd, an)
    fd = (L(f0, AMP + eps) - L(f0, AMP - eps)) / (2 * eps)
    assert abs(fd - abar) <= 1e-5 * abs(abar) + 1e-12, (fd, abar)
