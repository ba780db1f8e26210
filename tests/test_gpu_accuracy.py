"""The accuracy study of Sect. 5.1 on the GPU (accuracy.py).

* Parity: the first CN steps of the manufactured solution of Eq. (sol:exa)
  (Picard steps, then extrapolated ones) with the continuity source and the
  exact boundary data, steady and rotating circle at 32^2, equal the oracle's
  steps on the same inputs.
* Second-order decay of the errors of u and v on a short horizon (t = 0.5),
  N = 60 -> 120, on the steady circle.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_00994_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("omega", [0.0, 2 * math.pi / 5])
def test_first_steps_match_the_oracle(omega):
    from paper_1911_00994_gb300.accuracy import AccuracyRun, X0, LEN
    # 64^2: the circle of Eq. (domains) has radius 1/sqrt(15), 8 cells, room for
    # the moving body's extra ghost band around its centre, where grad phi = 0
    N, steps = 64, 4
    r = AccuracyRun(N, "circle", omega=omega, tol=1e-12, levels=2)
    s, ex, dt = r.s, r.ex, r.dt
    o = O.Oracle(N, X0, X0, LEN, 2, dt / (2 * r.Re), band=3 if omega else 0)
    # the GPU run, keeping each step's device inputs for the oracle
    r._geometry(0.0)
    x = r._frames(lambda X, Y: ex.u(X, Y, 0.0), lambda X, Y: ex.v(X, Y, 0.0))
    assert o.geometry(W.phi_half_lattice(W.paper_shape("circle", omega, 0.0), N, X0, X0, LEN)) == 0
    t0 = o.types().astype(int)
    xo = s.to_flat(x)
    xo[t0 == W.INACTIVE] = 0.0
    xo[-1] = 0.0
    N1, N2 = s.new_vec(), s.new_vec()
    N1o, N2o = np.zeros(o.n()), np.zeros(o.n())
    for m in range(steps):
        t1, th = (m + 1) * dt, (m + 0.5) * dt
        r._geometry(t1)
        phi = W.phi_half_lattice(W.paper_shape("circle", omega, t1), N, X0, X0, LEN)
        assert o.geometry(phi) == 0, o.error()
        assert np.array_equal(o.types()[:-1], s.types_flat()[:-1])
        f = r._frames(lambda X, Y: ex.f_u(X, Y, th), lambda X, Y: ex.f_v(X, Y, th))
        r.g_dev.copy_(r._frames(None, None, lambda X, Y: ex.div(X, Y, t1)))
        bc = r._boundary(t1)
        st, rep = s.cn_step(x, N1, N2, m, dt, r.Re, f=f, bc=bc, tol=1e-12, eps=1e-8, kmax=10)
        assert st == 0, s.error()
        o.set_continuity_source(s.to_flat(r.g_dev))
        st, xo, N1o, N2o, info = o.cn_step(xo, N1o, N2o, m, dt, f=s.to_flat(f), bc=s.to_flat(bc), tol=1e-12,
                                           eps=1e-8, kmax=10)
        assert st == 0, o.error()
        xg = s.to_flat(x)
        act = o.types().astype(int) != W.INACTIVE
        vel = act.copy()
        vel[-1 - N * N:] = False
        assert np.abs(xg[vel] - xo[vel]).max() <= 1e-9 * np.abs(xo[vel]).max(), m
        assert abs(xg[-1] - xo[-1]) <= 1e-9 * max(1.0, abs(xo[-1]))


def test_second_order_on_a_short_horizon():
    # the six tests of Sect. 5.1 run to t = 10 are not reproduced (the
    # central convective term of reading C18 goes unstable where the exact
    # solution flows out through the body at cell Peclet numbers above 2, near
    # t = 2 for the steady circle at N = 60, whatever dt); on a horizon before
    # that, t = 0.5, the errors of u and v fall at second order from N = 60 to
    # 120 on the steady circle
    from paper_1911_00994_gb300.accuracy import AccuracyRun
    errs = {}
    for N in (60, 120):
        r = AccuracyRun(N, "circle", T=0.5, tol=1e-9)
        r.run()
        errs[N] = r.errors()
    for q in ("u", "v"):
        for n in range(2):
            order = math.log(errs[60][q][n] / errs[120][q][n]) / math.log(2.0)
            assert order > 1.5, (q, n, errs)
    # div u - g = xi is constant: equal L^1 and L^inf errors of div u (to the
    # solve tolerance on the continuity rows)
    for N in (60, 120):
        assert abs(errs[N]["div"][0] - errs[N]["div"][1]) <= 1e-8
