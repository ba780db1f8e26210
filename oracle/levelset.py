"""Plain numpy reference of the level-set transport used for deforming bodies
(Sect. 3.1): reinitialisation to a signed distance function, Eq. (sdf), and
advection of phi by a velocity field.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and nothing in the product
path).  It shares no code with the CUDA kernels.

phi lives on the (2N+1) x (2N+1) half-cell lattice of the finest grid,
phi[b, a] at (x0 + a dx, y0 + b dx), dx = h / 2, paper sign (phi > 0 inside
the object).  One-sided differences:

    a = (phi[i] - phi[i-1]) / dx   (backward, x),   b = (phi[i+1] - phi[i]) / dx,
    c, d the same along y,

with the value beyond the lattice border taken equal to the border value
(zero normal gradient there).
"""
from __future__ import annotations

import numpy as np


def _one_sided(phi, dx):
    p = np.pad(phi, 1, mode="edge")
    a = (p[1:-1, 1:-1] - p[1:-1, :-2]) / dx     # backward x
    b = (p[1:-1, 2:] - p[1:-1, 1:-1]) / dx      # forward x
    c = (p[1:-1, 1:-1] - p[:-2, 1:-1]) / dx     # backward y
    d = (p[2:, 1:-1] - p[1:-1, 1:-1]) / dx      # forward y
    return a, b, c, d


def godunov_gradient(phi, s, dx):
    """|grad phi| by Godunov's upwind rule for the Hamilton-Jacobi equation
    phi_mu + s (|grad phi| - 1) = 0: information flows away from the zero
    level set, so for s > 0 the backward differences count when positive and
    the forward ones when negative, and the reverse for s < 0."""
    a, b, c, d = _one_sided(phi, dx)
    pos = np.sqrt(np.maximum(np.maximum(a, 0.0) ** 2, np.minimum(b, 0.0) ** 2)
                  + np.maximum(np.maximum(c, 0.0) ** 2, np.minimum(d, 0.0) ** 2))
    neg = np.sqrt(np.maximum(np.minimum(a, 0.0) ** 2, np.maximum(b, 0.0) ** 2)
                  + np.maximum(np.minimum(c, 0.0) ** 2, np.maximum(d, 0.0) ** 2))
    return np.where(s > 0, pos, np.where(s < 0, neg, 0.0))


def smoothed_sign(phi0, dx):
    """sgn(phi0) of Eq. (sdf), smoothed over one lattice spacing:
    phi0 / sqrt(phi0^2 + dx^2)."""
    return phi0 / np.sqrt(phi0 * phi0 + dx * dx)


def reinit(phi0, dx, iters, dtau):
    """`iters` forward-Euler steps in the fictitious time mu of Eq. (sdf),
    d phi / d mu = sgn(phi0) (1 - |grad phi|), from phi = phi0."""
    phi = np.array(phi0, dtype=np.float64)
    s = smoothed_sign(np.asarray(phi0, dtype=np.float64), dx)
    for _ in range(iters):
        phi = phi + dtau * s * (1.0 - godunov_gradient(phi, s, dx))
    return phi


def advect(phi, wx, wy, dt, dx, steps):
    """`steps` first-order upwind steps of phi_t + w . grad phi = 0 (the level
    set carried by the velocity w, given on the lattice)."""
    phi = np.array(phi, dtype=np.float64)
    for _ in range(steps):
        a, b, c, d = _one_sided(phi, dx)
        phi = phi - dt * (np.maximum(wx, 0.0) * a + np.minimum(wx, 0.0) * b
                          + np.maximum(wy, 0.0) * c + np.minimum(wy, 0.0) * d)
    return phi
