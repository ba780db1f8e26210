"""Pins of the oracle's adjoint of the Crank-Nicolson step (Sect. 2: Eqs.
NSCN1, extrUdU, NSitconv with a fixed number of Picard iterations) against
the oracle's forward step: the transposed convective Jacobian against exact
central differences of the convective term (quadratic in x), the transposed
explicit diffusion against the right-hand side, and the gradient of a
windowed kinetic energy after a short rollout of the orbiting circle (r = 0.25,
orbit radius 0.2) with respect to the forcing and the boundary-velocity amplitude
against central differences of the forward rollout."""
import numpy as np
import pytest

import oracle as O
from paper_1911_00994_gb300 import workloads as W
from tests._cases import levels_for

N, X0, LEN, RE = 32, -1.0, 2.0, 100.0


def moving(t):
    cx, cy = 0.2 * np.cos(2 * np.pi * t), 0.2 * np.sin(2 * np.pi * t)
    U, V = -0.2 * 2 * np.pi * np.sin(2 * np.pi * t), 0.2 * 2 * np.pi * np.cos(2 * np.pi * t)
    return W.circle(0.25, cx, cy), (U, V, 0.0, cx, cy)


def internal_mom(o):
    t = o.types()
    nU, nV = (N + 1) * (N + 2), (N + 2) * (N + 1)
    m = np.zeros(o.n(), dtype=bool)
    m[:nU + nV] = t[:nU + nV] == O.INTERNAL
    return m


def make(dt):
    o = O.Oracle(N, X0, X0, LEN, levels_for(N), dt / (2 * RE), band=3)
    shape, body = moving(0.0)
    assert o.geometry(W.phi_half_lattice(shape, N, X0, X0, LEN)) == 0
    return o


def test_convective_transpose_is_exact():
    o = make(0.3 * LEN / N)
    rng = np.random.default_rng(0)
    n = o.n()
    m = internal_mom(o)
    x, d = rng.standard_normal(n), rng.standard_normal(n)
    y = np.where(m, rng.standard_normal(n), 0.0)
    jd = (o.convective(x + d) - o.convective(x - d)) / 2.0   # exact: N is quadratic
    assert abs(np.dot(jd, y) - np.dot(d, o.convective_jt(x, y))) <= 1e-12 * np.abs(jd).sum() * np.abs(y).max()


def test_explicit_transpose():
    dt = 0.3 * LEN / N
    o = make(dt)
    rng = np.random.default_rng(1)
    n = o.n()
    m = internal_mom(o)
    x = rng.standard_normal(n)
    y = np.where(m, rng.standard_normal(n), 0.0)
    Ax = o.cn_rhs(x, np.zeros(n), dt)                        # x + alpha lap x on internal rows, 0 on the rest
    assert abs(np.dot(Ax, y) - np.dot(x, o.explicit_t(y))) <= 1e-12 * np.abs(Ax).sum() * np.abs(y).max()


def rollout(o, dt, steps, f, amp, K, tol):
    n = o.n()
    x, N1, N2 = np.zeros(n), np.zeros(n), np.zeros(n)
    xs = [x]
    for m in range(steps):
        shape, body = moving((m + 1) * dt)
        assert o.geometry(W.phi_half_lattice(shape, N, X0, X0, LEN)) == 0
        bd = (amp * body[0], amp * body[1], amp * body[2], body[3], body[4])
        st, x, N1, N2, info = o.cn_step(x, N1, N2, m, dt, f=f, body=bd, tol=tol, eps=0.0, kmax=K)
        assert st == 0
        xs.append(x)
    return xs


def gradient(o, dt, steps, f, amp, K, tol, w):
    n = o.n()
    xs = rollout(o, dt, steps, f, amp, K, tol)
    xbar = 2.0 * w * xs[-1]
    nb = [np.zeros(n), np.zeros(n), np.zeros(n)]
    fbar, abar = np.zeros(n), 0.0
    for m in reversed(range(steps)):
        shape, body = moving((m + 1) * dt)
        assert o.geometry(W.phi_half_lattice(shape, N, X0, X0, LEN)) == 0
        st, xbar, abar = o.cn_step_adjoint(m, xs[m], dt, xbar, nb, fbar, abar, f=f, body=body, amp=amp, tol=tol,
                                           kmax=K)
        assert st == 0
        nb = [nb[1], nb[2], np.zeros(n)]
    return float(np.sum(w * xs[-1] ** 2)), fbar, abar


@pytest.mark.parametrize("steps", [2, 5])
def test_rollout_gradient_matches_finite_differences(steps):
    # 2 steps: Picard only; 5 steps: Picard then extrapolation (the stored
    # convective terms of steps 0..2 feed steps 2..4)
    dt, K, tol = 0.3 * LEN / N, 4, 5e-13
    o = make(dt)
    n = o.n()
    m = internal_mom(o)
    rng = np.random.default_rng(1234)
    f = np.where(m, rng.standard_normal(n), 0.0)
    w = np.zeros(n)
    nU = (N + 1) * (N + 2)
    k = np.arange(nU)
    ju, iu = k // (N + 1) - 1, k % (N + 1)
    w[:nU] = ((iu >= 20) & (iu < 28) & (ju >= 12) & (ju < 20)).astype(float)
    amp = 1.0
    L0, fbar, abar = gradient(o, dt, steps, f, amp, K, tol, w)
    assert L0 > 0.0
    eps = 1e-4
    for s in range(3):
        d = np.where(m, np.random.default_rng(10 + s).standard_normal(n), 0.0)
        Lp = np.sum(w * rollout(o, dt, steps, f + eps * d, amp, K, tol)[-1] ** 2)
        Lm = np.sum(w * rollout(o, dt, steps, f - eps * d, amp, K, tol)[-1] ** 2)
        fd, an = (Lp - Lm) / (2 * eps), float(np.dot(fbar, d))
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-12, (s, fd, an)
    Lp = np.sum(w * rollout(o, dt, steps, f, amp + eps, K, tol)[-1] ** 2)
    Lm = np.sum(w * rollout(o, dt, steps, f, amp - eps, K, tol)[-1] ** 2)
    fd = (Lp - Lm) / (2 * eps)
    assert abs(fd - abar) <= 1e-5 * abs(abar) + 1e-12, (fd, abar)
