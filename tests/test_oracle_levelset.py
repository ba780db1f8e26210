"""Pins of the level-set transport reference (oracle/levelset.py) against the
mathematics of Eq. (sdf) and of the transport equation.

* A plane with |grad phi| = 1 is a fixed point of the reinitialisation, and
  first-order upwind differences advect it exactly (interior nodes).
* A plane with |grad phi| = 2 becomes a signed distance (|grad phi| = 1)
  inside the band the fictitious time has reached, its zero level moved by
  less than dx / 4.
* phi = R^2 - r^2 (the circle of Eq. domains, not a distance) becomes R - r
  near the circle to first order in dx.
* A disc carried by a constant velocity for time T keeps its radius and moves
  its centre by w T, to first order in dx.
"""
import math

import numpy as np

from oracle import levelset as LS
from paper_1911_00994_gb300 import workloads as W


def lattice(N, x0=-1.0, L=2.0):
    X, Y = W.half_lattice(N, x0, x0, L)
    return X, Y, 0.5 * L / N


def test_unit_plane_is_a_fixed_point_and_is_advected_exactly():
    X, Y, dx = lattice(32)
    th = 0.4
    phi = math.cos(th) * X + math.sin(th) * Y - 0.1
    out = LS.reinit(phi, dx, 10, 0.5 * dx)
    inner = (slice(12, -12), slice(12, -12))
    assert np.abs(out[inner] - phi[inner]).max() < 1e-13
    w = (0.3, -0.2)
    adv = LS.advect(phi, np.full_like(phi, w[0]), np.full_like(phi, w[1]), 0.5 * dx, dx, 10)
    T = 10 * 0.5 * dx
    exact = math.cos(th) * (X - w[0] * T) + math.sin(th) * (Y - w[1] * T) - 0.1
    assert np.abs(adv[inner] - exact[inner]).max() < 1e-13


def test_steep_plane_becomes_a_distance_in_the_reached_band():
    X, Y, dx = lattice(64)
    phi = 2.0 * (X - 0.05)
    out = LS.reinit(phi, dx, 80, 0.5 * dx)
    band = np.abs(X - 0.05) < 0.25           # fictitious time 80 * dx / 2 = 0.625 > 0.25 + margin
    gx = np.gradient(out, dx, axis=1)
    assert np.abs(gx[band] - 1.0).max() < 1e-6
    # the zero level moves by a fraction of dx (the scheme is first order
    # where the smoothed sign is not +-1), uniformly along the plane
    off = out[band] - (X[band] - 0.05)
    assert np.abs(off).max() < 0.25 * dx and np.ptp(off) < 1e-6
    # and stays between the same lattice columns
    assert np.array_equal(np.sign(out[:, 1:-1]), np.sign(phi[:, 1:-1]))


def test_circle_becomes_its_signed_distance():
    for N in (64, 128):
        X, Y, dx = lattice(N)
        R = 1.0 / math.sqrt(15.0)
        phi = R * R - (X * X + Y * Y)
        out = LS.reinit(phi, dx, 60, 0.5 * dx)
        near = np.abs(np.hypot(X, Y) - R) < 0.1
        err = np.abs(out[near] - (R - np.hypot(X[near], Y[near]))).max()
        assert err < 2.0 * dx, (N, err, dx)


def test_disc_carried_by_a_constant_velocity():
    X, Y, dx = lattice(128)
    R, w = 0.3, (0.5, 0.25)
    phi = R - np.hypot(X, Y)
    dt = 0.4 * dx / (abs(w[0]) + abs(w[1]))
    steps = 100
    T = steps * dt
    out = LS.advect(phi, np.full_like(phi, w[0]), np.full_like(phi, w[1]), dt, dx, steps)
    inside = out > 0
    cx, cy = X[inside].mean(), Y[inside].mean()
    assert abs(cx - w[0] * T) < 2 * dx and abs(cy - w[1] * T) < 2 * dx
    area = inside.sum() * dx * dx
    assert abs(area - math.pi * R * R) < 0.05 * math.pi * R * R
