"""The one-pass sweeps of the full boxes (Sect. 4.1.1, five colours in
shared memory, the result written to the level's other vector) against the
oracle's colour-by-colour sweep: the tile sweep (`wave_min=-1`) and the
sweep that streams down strips of rows (`wave_min=65`).  `tile_min` forces
the one-pass path on small levels; N = 96 and N = 200 leave ragged tiles
and strips at the right and top edges (frame pitch 128 and 224, 98 and 202
frame rows)."""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle, manufactured

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


def pair(case, N, alpha, **kw):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    lev = levels_for(N)
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=lev)
    assert st == 0, o.error()
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha, **kw)
    assert s.geometry(phi, 0) == 0, s.error()
    return o, s


WAVE = {"tiles": -1, "strips": 65}


@pytest.mark.parametrize("sweep", ["tiles", "strips"])
@pytest.mark.parametrize("case,N", [("flower5", 256), ("circle_off", 96), ("ellipse", 200), ("nobody", 128)])
def test_tiled_sweep_pieces_match(case, N, sweep):
    shape, x0, L = CASES[case]
    o, s = pair(case, N, alpha=(L / N) / 2.0, tile_min=65, wave_min=WAVE[sweep])
    for lev in range(o.levels):
        Nl = N >> lev
        if Nl < 65:
            break
        t = o.types(lev)
        x = W.random_flat(Nl, t, 500 + lev)
        b = W.random_flat(Nl, t, 600 + lev) * 10
        bd = s.to_device(b, lev)
        want = o.box_sweep(x, b, lev)
        xg = s.to_device(x, lev)
        s.box_sweep(xg, bd, lev)
        assert rel(s.to_flat(xg, lev), want) < 1e-12, lev
        for nu in (1, 2, 3):
            want = o.smooth(x, b, nu, lev)
            xg = s.to_device(x, lev)
            s.smooth(xg, bd, nu, lev)
            assert rel(s.to_flat(xg, lev), want) < 1e-11, (lev, nu)


@pytest.mark.parametrize("sweep", ["tiles", "strips"])
@pytest.mark.parametrize("case,N,ah2", [("flower5", 256, 2.0), ("circle_off", 200, None)])
def test_tiled_cycle_history_matches(case, N, ah2, sweep):
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2.0 if ah2 is None else ah2 * h * h
    o, s = pair(case, N, alpha=alpha, tile_min=65, wave_min=WAVE[sweep])
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    x = np.zeros_like(b)
    xg, bd = s.to_device(x), s.to_device(b)
    for k in range(4):
        st, x = o.cycle(x, b)
        s.cycle(xg, bd)
        assert rel(s.to_flat(xg), x) < 1e-9, k


@pytest.mark.parametrize("sweep", ["tiles", "strips"])
@pytest.mark.parametrize("case,N", [("flower5", 256), ("ellipse", 200)])
def test_tiled_mixed_solve_matches_oracle(case, N, sweep):
    # FP32 one-pass sweeps inside FP64 residual correction: the converged
    # solution is the oracle's FP64 solution to the tolerance
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2000.0 if case == "flower5" else h / 200.0
    o, s = pair(case, N, alpha=alpha, tile_min=65, precision=1, wave_min=WAVE[sweep])
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 1e-10, 200)
    assert st_o == 0
    xg = s.new_vec()
    st, rep, h_g = s.solve(xg, s.to_device(b), 1e-10)
    assert st == 0, s.error()
    assert rel(s.to_flat(xg), x_o) <= 1e-8
    # the same solve with the five colour passes takes as many cycles
    o2, s2 = pair(case, N, alpha=alpha, tile_min=-1, precision=1)
    xg2 = s2.new_vec()
    st2, rep2, h_g2 = s2.solve(xg2, s2.to_device(b), 1e-10)
    assert st2 == 0
    assert abs(len(h_g) - len(h_g2)) <= 1


@pytest.mark.parametrize("case,N", [("flower5", 256), ("ellipse", 200)])
def test_mixed_inner_cycles(case, N):
    # several FP32 cycles per FP64 residual correction, their number predicted
    # from the last correction's rate: the oracle's FP64 solution to the
    # tolerance, at most one cycle more than one cycle per correction, and
    # fewer FP64 residuals
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2000.0 if case == "flower5" else h / 200.0
    o, s1 = pair(case, N, alpha=alpha, precision=1, inner=1)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 1e-10, 200)
    assert st_o == 0
    x1 = s1.new_vec()
    st1, rep1, h1 = s1.solve(x1, s1.to_device(b), 1e-10)
    assert st1 == 0 and rep1.iterations == rep1.cycles
    for inner in (2, 4, 8):
        _, s3 = pair(case, N, alpha=alpha, precision=1, inner=inner)
        x3 = s3.new_vec()
        st3, rep3, h3 = s3.solve(x3, s3.to_device(b), 1e-10)
        assert st3 == 0, s3.error()
        assert rep3.res <= 1e-10 and h3[-1] <= 1e-10
        assert rel(s3.to_flat(x3), x_o) <= 1e-8
        assert rep3.cycles <= rep1.cycles + 1, (inner, rep3.cycles, rep1.cycles)
        assert rep3.iterations < rep1.iterations
        assert len(h3) == rep3.iterations + 1


@pytest.mark.parametrize("precision", [0, 1])
def test_strip_sweep_equals_tile_sweep(precision):
    # the two one-pass sweeps relax the same boxes in the same colour order
    # with the same box solve: the same iterate bit for bit, on a level of
    # several strips and segments (1024^2: 17 FP64 / 9 FP32 strips, segments
    # of a few dozen rows).  FP64: two cycles; FP32: six cycles of the mixed
    # solve (FP32 cycles inside the FP64 correction), iterate and history.
    import torch
    from paper_1911_00994_gb300 import gpmg
    case, N = "flower5", 1024
    shape, x0, L = CASES[case]
    h = L / N
    lev = levels_for(N)
    phi = W.phi_half_lattice(shape, N, x0, x0, L)
    out = []
    for wmin in (-1, 65):
        s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=2.0 * h * h, tile_min=65, wave_min=wmin,
                        precision=precision, max_cycles=6)
        assert s.geometry(phi, 0) == 0, s.error()
        t = s.types_flat(0)
        b = W.random_flat(N, t, 8) * 10
        bd = s.to_device(b)
        if precision == 0:
            xg = s.to_device(W.random_flat(N, t, 7))
            for k in range(2):
                s.cycle(xg, bd)
            hist = None
        else:
            xg = s.new_vec()
            st, rep, hist = s.solve(xg, bd, 1e-14)
            assert st == 4 and rep.cycles == 6, s.error()  # GP_NOT_CONVERGED after the cap
        torch.cuda.synchronize()
        out.append((s.to_flat(xg), hist))
    assert np.array_equal(out[0][0], out[1][0])
    if precision == 1:
        assert np.array_equal(out[0][1], out[1][1])
