"""torch.autograd.Function wrappers of cn_step and of the checkpointed rollout
(autograd.py) on the GPU.

* One extrapolated CN step at 32^2: the gradients of L = sum w x^2 with
  respect to the forcing, the body-velocity amplitude and the convective
  history equal those given by a dense solve of the transposed system
  (numpy on the oracle's assembled matrix of the same level set):
  dL/df = dt lam, dL/damp = lam . g, dL/dN^(n-1) = -dt lam / 2,
  dL/dN^(n-2) = +dt lam / 2 on internal momentum rows, M^T lam = 2 w x.
* A chain of differentiable steps gives the rollout function's gradient.
* The rollout function's gradient agrees with central finite differences
  (eps = 1e-4, solves to 1e-12) on 8 seeded forcing directions and on the
  amplitude, to 1e-6 relative.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import levels_for, make_oracle

pytestmark = pytest.mark.gpu

X0, LEN, RE = -1.0, 2.0, 100.0


def _mom(t, N):
    nU, nV = (N + 1) * (N + 2), (N + 2) * (N + 1)
    m = np.zeros(len(t), dtype=bool)
    m[:nU + nV] = t[:nU + nV] == W.INTERNAL
    return m


def _window(N, n):
    w = np.zeros(n)
    nU = (N + 1) * (N + 2)
    k = np.arange(nU)
    ju, iu = k // (N + 1) - 1, k % (N + 1)
    w[:nU] = (iu >= 5 * N // 8) & (iu < 7 * N // 8) & (ju >= 3 * N // 8) & (ju < 5 * N // 8)
    return w


def test_cn_step_gradients_match_dense_transpose_solve():
    import torch
    from paper_1911_00994_gb300 import gpmg
    from paper_1911_00994_gb300.autograd import cn_step
    N = 32
    h = LEN / N
    dt = 0.3 * h
    alpha = dt / (2 * RE)
    o, phi, st = make_oracle("circle_off", N, alpha=alpha)
    assert st == 0, o.error()
    s = gpmg.Solver(N, X0, X0, LEN, levels=levels_for(N), alpha=alpha, adjoint=True, max_cycles=400)
    assert s.geometry(phi) == 0, s.error()
    t = o.types(0)
    n = len(t)
    mom = _mom(t, N)
    rng = np.random.default_rng(7)
    xm = np.where(mom, 0.2 * rng.standard_normal(n), 0.0)
    n1 = np.where(mom, rng.standard_normal(n), 0.0)
    n2 = np.where(mom, rng.standard_normal(n), 0.0)
    f0 = np.where(mom, rng.standard_normal(n), 0.0)
    body = (0.4, -0.3, 1.1, 0.2, 0.0)
    amp0 = 0.7
    w = _window(N, n)
    x = s.to_device(xm)
    N1 = s.to_device(n1).requires_grad_(True)
    N2 = s.to_device(n2).requires_grad_(True)
    f = s.to_device(f0).requires_grad_(True)
    amp = torch.tensor(amp0, dtype=torch.float64, requires_grad=True)
    xn, Nm = cn_step(x, N1, N2, f, amp, s, 2, dt, RE, body, tol=1e-13)
    wd = s.to_device(w)
    L = (wd * xn * xn).sum()
    L.backward()
    # dense transpose solve of the oracle's matrix
    A = o.dense_matrix(0)
    xf = s.to_flat(xn.detach())
    lam = np.linalg.solve(A.T, 2.0 * w * xf)
    g_body = o.cn_rhs(np.zeros(n), np.zeros(n), dt, body=body)   # the object's Eq. (BCu) values
    want_f = np.where(mom, dt * lam, 0.0)
    got_f = s.to_flat(f.grad)
    scale = np.abs(want_f).max()
    assert np.abs(got_f - want_f).max() <= 1e-9 * scale
    assert np.abs(s.to_flat(N1.grad) - np.where(mom, -0.5 * dt * lam, 0.0)).max() <= 1e-9 * scale
    assert np.abs(s.to_flat(N2.grad) - np.where(mom, 0.5 * dt * lam, 0.0)).max() <= 1e-9 * scale
    want_a = float(np.dot(lam, g_body))
    assert abs(float(amp.grad) - want_a) <= 1e-9 * abs(want_a)


def _moving(s, dt):
    from paper_1911_00994_gb300 import gpmg
    return dict(kind=gpmg.GP_CIRCLE, a=0.25, orbit_r=0.2, orbit_period=1.0)


def _rollout(N, steps, every, tol):
    from paper_1911_00994_gb300 import gpmg
    from paper_1911_00994_gb300.rollout import Rollout
    dt = 0.3 * LEN / N
    s = gpmg.Solver(N, X0, X0, LEN, levels=levels_for(N), alpha=dt / (2 * RE), band=3, adjoint=True,
                    max_cycles=600)
    shape = _moving(s, dt)
    st, body = s.geometry_shape(t=0.0, **shape)
    assert st == 0, s.error()
    return s, Rollout(s, shape, dt, RE, steps, kmax=4, tol=tol, every=every), shape, dt


def _bumps(N, t, seed=1234):
    g, i, j, X, Y = W.flat_coords(N, X0, X0, LEN)
    rng = np.random.default_rng(seed)
    f = np.zeros(len(t))
    for _ in range(4):
        while True:
            c = rng.uniform(-0.9, 0.9, 2)
            if np.hypot(c[0], c[1]) > 0.55:
                break
        a = rng.standard_normal(2)
        bump = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (2 * 0.1 ** 2))
        f += np.where(g == 0, a[0] * bump, 0.0) + np.where(g == 1, a[1] * bump, 0.0)
    return np.where(_mom(t, N), f, 0.0)


AMP = 0.3


def test_chain_of_steps_equals_rollout_function():
    import torch
    from paper_1911_00994_gb300.autograd import cn_step, rollout
    N, steps = 32, 5
    s, ro, shape, dt = _rollout(N, steps, 2, 1e-12)
    t = s.types_flat()
    w = s.to_device(_window(N, len(t)))
    f0 = s.to_device(0.1 * _bumps(N, t))
    # rollout function
    f = f0.clone().requires_grad_(True)
    amp = torch.tensor(AMP, dtype=torch.float64, requires_grad=True)
    x = rollout(f, amp, ro)
    L1 = (w * x * x).sum()
    L1.backward()
    gf1, ga1 = f.grad.clone(), float(amp.grad)
    # chain of steps
    f = f0.clone().requires_grad_(True)
    amp = torch.tensor(AMP, dtype=torch.float64, requires_grad=True)
    x, N1, N2 = s.new_vec(), s.new_vec(), s.new_vec()
    for m in range(steps):
        def geom(m=m):
            st, body = s.geometry_shape(t=(m + 1) * dt, **shape)
            assert st == 0, s.error()
            return body
        body = geom()
        x, Nm = cn_step(x, N1, N2, f, amp, s, m, dt, RE, body, tol=1e-12, kmax=4, geometry=geom)
        N1, N2 = Nm, N1
    L2 = (w * x * x).sum()
    L2.backward()
    assert abs(float(L2) - float(L1)) <= 1e-12 * abs(float(L1))
    a, b = s.to_flat(f.grad), s.to_flat(gf1)
    assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
    assert abs(float(amp.grad) - ga1) <= 1e-9 * abs(ga1)


def test_rollout_function_matches_central_differences_on_8_directions():
    import torch
    from paper_1911_00994_gb300.autograd import rollout
    N, steps = 64, 10
    tol = 1e-12
    s, ro, shape, dt = _rollout(N, steps, 4, tol)
    t = s.types_flat()
    n = len(t)
    mom = _mom(t, N)
    w = s.to_device(_window(N, n))
    f0 = 0.1 * _bumps(N, t)
    f = s.to_device(f0).requires_grad_(True)
    amp = torch.tensor(AMP, dtype=torch.float64, requires_grad=True)
    x = rollout(f, amp, ro)
    L = (w * x * x).sum()
    L.backward()
    grad = s.to_flat(f.grad)
    gamp = float(amp.grad)

    def loss(fv, a):
        with torch.no_grad():
            xx = rollout(s.to_device(fv), torch.tensor(a, dtype=torch.float64), ro)
            return float((w * xx * xx).sum())

    eps = 1e-4
    worst = 0.0
    for k in range(8):
        d = np.where(mom, np.random.default_rng(k).standard_normal(n), 0.0)
        fd = (loss(f0 + eps * d, AMP) - loss(f0 - eps * d, AMP)) / (2 * eps)
        an = float(np.dot(grad, d))
        worst = max(worst, abs(fd - an) / abs(an))
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)
    fd = (loss(f0, AMP + eps) - loss(f0, AMP - eps)) / (2 * eps)
    assert abs(fd - gamp) <= 1e-6 * abs(gamp), (fd, gamp)
