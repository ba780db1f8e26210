"""W-cycles (gamma = 2, the cycle Sect. 4 adopts) on the GPU against the
oracle's W-cycles, element by element on identical seeded inputs.

Tolerances as for the V-cycle parity tests: cycles 1e-9 relative (FMA
contraction and summation order differ), converged FP64 solves 1e-9 after
both reach ||r||_inf <= 1e-10, mixed-precision solves 1e-8 against the
oracle's FP64 solution, transposed cycles 1e-9.  Graph replay is bitwise the
direct launches.  The solves use cases where the oracle's W-cycle converges
(it diverges on the five-petal flower at alpha / h^2 = 0.128, and at 1024^2
with seven levels at alpha / h^2 = 2.05, where the V-cycle converges); the
divergent 1024^2 history is matched cycle by cycle too.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle, manufactured

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


def pair(case, N, ah2=None, **kw):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2.0 if ah2 is None else ah2 * h * h
    lev = levels_for(N)
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=lev, gamma=2)
    assert st == 0, o.error()
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha, gamma=2, **kw)
    assert s.geometry(phi, 0) == 0, s.error()
    return o, s


@pytest.mark.parametrize("case,N,ah2", [("circle", 64, None), ("flower5", 256, 2.05), ("ellipse", 128, 8.0),
                                        ("flower5", 1024, 2.05)])
def test_w_cycle_history_matches(case, N, ah2):
    # the flower at 1024^2 (seven levels): the oracle's W-cycles make the
    # residual grow (about x2 per cycle after the first), and so do the GPU's
    o, s = pair(case, N, ah2)
    b, xe, t, gh = manufactured(o, W.taylor_green())
    x = np.zeros_like(b)
    xg, bd = s.to_device(x), s.to_device(b)
    for k in range(3):
        st, x = o.cycle(x, b)
        s.cycle(xg, bd)
        assert rel(s.to_flat(xg), x) < 1e-9, k
        _, no = o.residual(x, b)
        _, ng = s.residual(xg, bd)
        assert abs(ng - no) <= 1e-6 * no


@pytest.mark.parametrize("case,N,ah2", [("flower5", 256, 2.05), ("flower7", 256, 64.0)])
def test_w_cycle_solve_matches_oracle(case, N, ah2):
    # the seven-petal flower at alpha / h^2 = 64: W-cycles converge where
    # V-cycles stall at rho ~ 0.9
    o, s = pair(case, N, ah2)
    b, xe, t, gh = manufactured(o, W.taylor_green())
    st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 1e-10, 100)
    assert st_o == 0
    xg = s.new_vec()
    st, rep, h_g = s.solve(xg, s.to_device(b), 1e-10)
    assert st == 0, s.error()
    assert rep.res <= 1e-10
    assert rel(s.to_flat(xg), x_o) <= 1e-9
    assert abs(len(h_g) - len(h_o)) <= 1


@pytest.mark.parametrize("inner", [1, 0])
def test_w_cycle_mixed_tiled_solve_matches_oracle(inner):
    # FP32 W-cycles (levels from 128^2 tiled) inside FP64 residual correction:
    # the oracle's FP64 W-cycle solution to the tolerance
    o, s = pair("flower5", 256, 8.0, precision=1, tile_min=128, inner=inner)
    b, xe, t, gh = manufactured(o, W.taylor_green())
    st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 1e-10, 100)
    assert st_o == 0
    xg = s.new_vec()
    st, rep, h_g = s.solve(xg, s.to_device(b), 1e-10)
    assert st == 0, s.error()
    assert rep.res <= 1e-10
    assert rel(s.to_flat(xg), x_o) <= 1e-8
    assert rep.cycles <= len(h_o) - 1 + 2


def test_transposed_w_cycles_match():
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES["flower5"]
    N = 128
    h = L / N
    lev = levels_for(N)
    o, phi, st = make_oracle("flower5", N, alpha=h / 2.0, levels=lev, gamma=2)
    assert st == 0
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=h / 2.0, gamma=2, adjoint=True)
    assert s.geometry(phi, 0) == 0, s.error()
    cc = np.random.default_rng(11).standard_normal(o.n())
    lam = np.zeros(o.n())
    lg, ccd = s.to_device(lam), s.to_device(cc)
    for k in range(3):
        st, lam = o.cycle_t(lam, cc)
        s.cycle_t(lg, ccd)
        assert rel(s.to_flat(lg), lam) < 1e-9, k


@pytest.mark.parametrize("precision", [0, 1])
def test_w_cycle_graph_replay_matches_direct_launches(precision):
    # the captured W-cycle (every coarse visit in one graph) replays bitwise
    # the iterate of direct launches
    import torch
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES["flower5"]
    N = 128
    lev = levels_for(N)
    alpha = 8.0 * (L / N) ** 2
    o, phi, st = make_oracle("flower5", N, alpha=alpha, levels=lev, gamma=2)
    b, xe, t, gh = manufactured(o, W.taylor_green())
    out = []
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha, gamma=2, precision=precision, graphs=graphs,
                            stream=stream)
            assert s.geometry(phi) == 0, s.error()
            x = s.new_vec()
            bd = s.to_device(b)
            st, rep, hist = s.solve(x, bd, 1e-10)
            assert st == 0, s.error()
            x.zero_()
            st, rep2, hist2 = s.solve(x, bd, 1e-10)  # second solve replays the captured graphs
            stream.synchronize()
            out.append((s.to_flat(x), hist2))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
