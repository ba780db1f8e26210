"""Moving bodies (Sect. 3.4): the device level set of a rigidly moving test
body against the closed form, and Crank-Nicolson steps of the orbiting circle
(circle r = 0.25 on an orbit of radius 0.2, period 1) with the geometry
rebuilt every step, against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1911_00994_gb300 import workloads as W
from tests._cases import levels_for

pytestmark = pytest.mark.gpu


def moving_circle(t):
    cx, cy = 0.2 * np.cos(2 * np.pi * t), 0.2 * np.sin(2 * np.pi * t)
    U, V = -0.2 * 2 * np.pi * np.sin(2 * np.pi * t), 0.2 * 2 * np.pi * np.cos(2 * np.pi * t)
    return W.circle(0.25, cx, cy), (U, V, 0.0, cx, cy)


@pytest.mark.parametrize("kind,a,b,k", [(0, 0.25, 0.0, 0), (1, 0.4, 0.2, 0), (2, 0.5, 0.1, 7)])
def test_shape_level_set_matches_closed_form(kind, a, b, k):
    from paper_1911_00994_gb300 import gpmg
    N, x0, L, t = 128, -1.0, 2.0, 0.37
    s = gpmg.Solver(N, x0, x0, L, levels=levels_for(N))
    st, body = s.geometry_shape(kind, a, b, k, orbit_r=0.3, orbit_period=1.0, omega=0.5, t=t)
    got = s.level_set().cpu().numpy()
    cx, cy = 0.3 * np.cos(2 * np.pi * t), 0.3 * np.sin(2 * np.pi * t)
    X, Y = W.half_lattice(N, x0, x0, L)
    ang = 0.5 * t
    dx, dy = X - cx, Y - cy
    qx, qy = np.cos(ang) * dx + np.sin(ang) * dy, -np.sin(ang) * dx + np.cos(ang) * dy
    r = np.hypot(qx, qy)
    want = {0: a - r, 1: 1 - np.sqrt(qx ** 2 / a ** 2 + qy ** 2 / max(b, 1e-300) ** 2) if kind == 1 else 0,
            2: a + b * np.sin(k * np.arctan2(qy, qx)) - r}[kind]
    assert np.abs(got - want).max() < 1e-12
    w = 2 * np.pi
    assert np.allclose(body, (-0.3 * w * np.sin(w * t), 0.3 * w * np.cos(w * t), 0.5, cx, cy), atol=1e-14)


def test_moving_circle_cn_steps_match_oracle():
    from paper_1911_00994_gb300 import gpmg
    # Sects. 3.4 and 5.1 bound the step by dt <= min(h, h / max |u|); the body moves at
    # 0.4 pi (about 1.26), and at this resolution the impulsively started
    # boundary layer makes the mid-point Picard iteration of Eq. (NSitconv)
    # diverge already at dt = 0.6 h, so the step is 0.3 h (0.38 h of motion)
    N, x0, L, Re = 64, -1.0, 2.0, 100.0
    h = L / N
    dt = 0.3 * h
    band = 3
    lev = levels_for(N)
    o = O.Oracle(N, x0, x0, L, lev, dt / (2 * Re), band=band)
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=dt / (2 * Re), band=band)
    xo, N1o, N2o = np.zeros(o.n()), np.zeros(o.n()), np.zeros(o.n())
    xg, N1g, N2g = s.new_vec(), s.new_vec(), s.new_vec()
    for step in range(4):
        shape, body = moving_circle((step + 1) * dt)
        phi = W.phi_half_lattice(shape, N, x0, x0, L)
        assert o.geometry(phi) == 0, o.error()
        assert s.geometry(phi) == 0, s.error()
        assert np.array_equal(o.types()[:-1], s.types_flat()[:-1])
        st, xo, N1o, N2o, info = o.cn_step(xo, N1o, N2o, step, dt, body=body, tol=1e-11)
        assert st == 0
        st, rep = s.cn_step(xg, N1g, N2g, step, dt, Re, body=body, tol=1e-11)
        assert st == 0, s.error()
        got = s.to_flat(xg)
        assert np.abs(got - xo).max() <= 1e-8 * max(1.0, np.abs(xo).max()), step
    assert np.abs(xo).max() > 1e-3  # the body has set the fluid in motion
