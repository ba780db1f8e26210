"""Level-set transport on the GPU (gp_levelset_reinit, gp_levelset_advect;
Sect. 3.1, Eq. sdf) against the plain reference oracle/levelset.py, element
by element on the half-cell lattice, and the pipeline it serves: a body
carried by a velocity field, reinitialised, then built into the ghost-point
geometry."""
import math

import numpy as np
import pytest

from oracle import levelset as LS
from paper_1911_00994_gb300 import workloads as W
from tests._cases import levels_for

pytestmark = pytest.mark.gpu


def _solver(N):
    from paper_1911_00994_gb300 import gpmg
    return gpmg.Solver(N, -1.0, -1.0, 2.0, levels=levels_for(N))


@pytest.mark.parametrize("shape,N", [("circle", 64), ("flower", 128), ("ellipse", 96)])
def test_reinit_matches_the_reference(shape, N):
    import torch
    s = _solver(N)
    X, Y = W.half_lattice(N, -1.0, -1.0, 2.0)
    dx = 1.0 / N
    phi0 = W.paper_shape(shape)(X, Y)
    ref = LS.reinit(phi0, dx, 40, 0.5 * dx)
    d = torch.from_numpy(np.ascontiguousarray(phi0)).to(s.device)
    s.levelset_reinit(d, 40, 0.5 * dx)
    got = d.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_advection_matches_the_reference():
    import torch
    N = 128
    s = _solver(N)
    X, Y = W.half_lattice(N, -1.0, -1.0, 2.0)
    dx = 1.0 / N
    phi0 = W.paper_shape("flower")(X, Y)
    om = 2 * math.pi / 5
    wx, wy = -om * Y, om * X                     # rigid rotation about the origin
    dt = 0.4 * dx / (np.abs(wx).max() + np.abs(wy).max())
    ref = LS.advect(phi0, wx, wy, dt, dx, 25)
    dev = s.device
    d = torch.from_numpy(np.ascontiguousarray(phi0)).to(dev)
    s.levelset_advect(d, torch.from_numpy(np.ascontiguousarray(wx)).to(dev),
                      torch.from_numpy(np.ascontiguousarray(wy)).to(dev), dt, 25)
    got = d.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_carried_reinitialised_body_builds_a_geometry():
    # a disc carried by a uniform velocity, reinitialised, then classified:
    # its ghost rows' boundary points lie on the moved circle to O(dx)
    import torch
    N = 128
    s = _solver(N)
    X, Y = W.half_lattice(N, -1.0, -1.0, 2.0)
    dx = 1.0 / N
    R, w = 0.3, (0.4, -0.2)
    phi = torch.from_numpy(np.ascontiguousarray(R - np.hypot(X, Y))).to(s.device)
    dt = 0.4 * dx / (abs(w[0]) + abs(w[1]))
    steps = 120
    s.levelset_advect(phi, torch.full_like(phi, w[0]), torch.full_like(phi, w[1]), dt, steps)
    s.levelset_reinit(phi, 20, 0.5 * dx)
    assert s.geometry(phi.cpu().numpy()) == 0, s.error()
    T = steps * dt
    gr = s.ghost_rows(0)
    B = gr["B"][gr["kind"] == 0]
    r = np.hypot(B[:, 0] - w[0] * T, B[:, 1] - w[1] * T)
    assert np.abs(r - R).max() < 3 * dx
    with pytest.raises(Exception):
        s.levelset_reinit(phi, 5, 4.0 * dx)     # dtau above the lattice spacing
