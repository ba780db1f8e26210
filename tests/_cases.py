"""Shared test cases: named geometries and problem parameters.

Every case is seeded and synthetic; see the input recipe in the design notes.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1911_00994_gb300 import workloads as W

CASES = {
    # name: (shape, x0, L)
    "circle": (W.circle(0.5), -1.0, 2.0),                           # the 32^2 manufactured case
    "circle_off": (W.circle(0.25, 0.2, 0.0), -1.0, 2.0),            # the orbiting circle at t = 0
    "ellipse": (W.ellipse(0.4, 0.2, 0.3, 0.0), -1.0, 2.0),          # the orbiting ellipse at t = 0
    "flower5": (W.flower(0.2, 0.05, 5, 0.5, 0.5), 0.0, 1.0),        # the cavity's five-petal flower
    "flower7": (W.flower(0.5, 0.1, 7), -1.0, 2.0),                  # the seven-petal flower
    "nobody": (lambda X, Y: -1.0 + 0.0 * X, -1.0, 2.0),             # empty box
}


def levels_for(N: int, nc: int = 16) -> int:
    lev = 1
    while (N >> lev) >= nc and (N >> (lev - 1)) > nc:
        lev += 1
    return lev


def make_oracle(case: str, N: int, alpha: float | None = None, levels: int | None = None, **kw):
    shape, x0, L = CASES[case]
    h = L / N
    if alpha is None:
        alpha = h / 2.0
    if levels is None:
        levels = levels_for(N)
    o = O.Oracle(N, x0, x0, L, levels, alpha, **kw)
    phi = W.phi_half_lattice(shape, N, x0, x0, L)
    st = o.geometry(phi)
    return o, phi, st


def manufactured(o: O.Oracle, ex: W.Exact, lev: int = 0):
    N = o.N >> lev
    L = o.len
    t = o.types(lev)
    gh = o.ghosts(lev)
    b = W.manufactured_rhs(ex, N, o.x0, o.y0, L, o.alpha, t, gh["grid"], gh["i"], gh["j"], gh["B"], gh["kind"])
    xe = W.exact_flat(ex, N, o.x0, o.y0, L, t)
    return b, xe, t, gh
