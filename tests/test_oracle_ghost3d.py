"""Pins of the 3-D ghost-point oracle (oracle/ghost3d.py) against
mathematics: the 27-point Eq. (BCu) weights reproduce every triquadratic at
the boundary point; Algorithm 1 puts B on the sphere within its bisection
tolerance plus the interpolation error of the trilinear level set; theta
lies in the span of the stencil."""
import itertools
import math

import numpy as np
import pytest

from oracle import ghost3d as G3


def triquad(c, x, y, z):
    return sum(c[a, b, d] * x ** a * y ** b * z ** d for a in range(3) for b in range(3) for d in range(3))


@pytest.mark.parametrize("N", [16, 32])
def test_weights_reproduce_triquadratics_and_b_on_the_sphere(N):
    c, R = (0.51, 0.47, 0.53), 0.27
    o = G3.Ghosts3D(N, c, R)
    h = 1.0 / N
    rng = np.random.default_rng(N)
    n = 0
    for g in range(3):
        rows = o.rows(g)
        assert len(rows) > 0
        cf = rng.standard_normal((3, 3, 3))
        for r in rows:
            n += 1
            xs = [G3.node_xyz(g, *nd, h) for nd in r["st"]]
            val = sum(w * triquad(cf, *p) for w, p in zip(r["w"], xs))
            assert abs(val - triquad(cf, *r["B"])) <= 1e-11 * (1 + np.abs(cf).sum() * 3)
            assert abs(r["w"].sum() - 1.0) <= 1e-13
            # B on the sphere: bisection tolerance plus the trilinear interpolation error
            d = math.sqrt(sum((r["B"][a] - c[a]) ** 2 for a in range(3)))
            assert abs(d - R) <= 0.01 * h + h * h / (R - 2 * h), (d - R) / h
            assert all(-1e-12 <= t <= 2.0 for t in r["theta"])
    assert n > 100


def test_ghosts_are_the_object_nodes_next_to_the_fluid():
    N = 16
    o = G3.Ghosts3D(N, (0.5, 0.5, 0.5), 0.3)
    for g in range(3):
        gh = set(o.ghost_nodes(g))
        for (i, j, k) in gh:
            assert o.phi_node(g, i, j, k) >= 0.0
        # every object node with a fluid neighbour is a ghost, no other node is
        for i, j, k in itertools.product(range(-1, N + 1), repeat=3):
            if not o.interior(g, i, j, k) or o.phi_node(g, i, j, k) < 0.0:
                assert (i, j, k) not in gh
