"""The 3-D ghost points of a sphere on the GPU (gp3_sphere_ghosts through
the C ABI) against the oracle (oracle/ghost3d.py), and against mathematics
alone (triquadratic reproduction at B, B on the sphere)."""
import math

import numpy as np
import pytest

from oracle import ghost3d as G3

pytestmark = pytest.mark.gpu

C, R = (0.51, 0.47, 0.53), 0.27


def oracle_rows(N):
    o = G3.Ghosts3D(N, C, R)
    S = N + 2
    F = S ** 3
    idx = lambda g, i, j, k: g * F + ((k + 1) * S + (j + 1)) * S + (i + 1)
    rows = []
    for g in range(3):
        for r in o.rows(g):
            rows.append((idx(g, *r["node"]), r["B"], r["theta"], [idx(g, *p) for p in r["st"]], r["w"]))
    rows.sort(key=lambda t: t[0])
    return rows


@pytest.mark.parametrize("N", [16, 32])
def test_ghost_rows_match_the_oracle(N):
    from paper_1911_00994_gb300 import mac3d
    got = mac3d.sphere_ghosts(N, C, R)
    want = oracle_rows(N)
    assert np.array_equal(got["node"], np.array([r[0] for r in want]))
    # the march and bisection take the same decisions: B and theta to rounding
    assert np.abs(got["B"] - np.array([r[1] for r in want])).max() <= 1e-14
    assert np.abs(got["theta"] - np.array([r[2] for r in want])).max() <= 1e-12
    assert np.array_equal(got["st"], np.array([r[3] for r in want]))
    assert np.abs(got["w"] - np.array([r[4] for r in want])).max() <= 1e-12


def test_gpu_rows_reproduce_triquadratics_at_b():
    # GPU data only: every row interpolates a random triquadratic exactly at
    # its B, and B lies on the sphere within the bisection tolerance plus the
    # trilinear interpolation error
    from paper_1911_00994_gb300 import mac3d
    N = 32
    h = 1.0 / N
    got = mac3d.sphere_ghosts(N, C, R)
    S = N + 2
    F = S ** 3
    rng = np.random.default_rng(9)
    cf = rng.standard_normal((3, 3, 3))
    q = lambda x, y, z: sum(cf[a, b, d] * x ** a * y ** b * z ** d for a in range(3) for b in range(3)
                            for d in range(3))

    def xyz(e):
        g, s = divmod(int(e), F)
        k, rem = divmod(s, S * S)
        j, i = divmod(rem, S)
        off = [0.5, 0.5, 0.5]
        off[g] = 0.0
        return (i - 1 + off[0]) * h, (j - 1 + off[1]) * h, (k - 1 + off[2]) * h

    assert len(got["node"]) > 1000
    for n in range(len(got["node"])):
        val = sum(w * q(*xyz(e)) for w, e in zip(got["w"][n], got["st"][n]))
        assert abs(val - q(*got["B"][n])) <= 1e-10 * (1 + np.abs(cf).sum() * 3), n
        d = math.sqrt(sum((got["B"][n][a] - C[a]) ** 2 for a in range(3)))
        assert abs(d - R) <= 0.01 * h + h * h / (R - 2 * h)
