"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on identical seeded inputs.

Tolerances: geometry decisions (node types, ghost row kinds, stencils) are
bit-exact; ghost weights and boundary points agree to 1e-13 (same formulas,
separately rounded operations on both sides); operator applications to
1e-12 relative (FMA contraction and summation order differ); full solves to
relative L-infinity 1e-10 after both reach the residual tolerance (1e-12 at
32^2; 5e-12, just above the rounding floor, at 128^2 and 256^2).
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle, manufactured

pytestmark = pytest.mark.gpu

GEOM_CASES = [("circle", 32), ("circle", 64), ("ellipse", 128), ("flower5", 128), ("circle_off", 128),
              ("flower7", 256), ("flower5", 512)]


def pair(case, N, alpha=None, **kw):
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / 2.0 if alpha is None else alpha
    lev = levels_for(N)
    o, phi, st = make_oracle(case, N, alpha=alpha, levels=lev, **{k: v for k, v in kw.items() if k in ("snap",)})
    assert st == 0, o.error()
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha, **kw)
    st = s.geometry(phi, 0)
    assert st == 0, s.error()
    return o, s


def rel(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


@pytest.mark.parametrize("case,N", GEOM_CASES)
def test_geometry_matches(case, N):
    o, s = pair(case, N)
    for lev in range(o.levels):
        Nl = N >> lev
        to = o.types(lev)
        tg = s.types_flat(lev)
        assert np.array_equal(to[:-1], tg[:-1]), "types differ on level %d" % lev
        go = o.ghosts(lev)
        gg = s.ghost_rows(lev)
        n = len(go["grid"])
        assert len(gg["node"]) == n
        m = s.maps(lev).cpu().numpy()
        inv = {int(v): k for k, v in enumerate(m)}
        flat_node = np.array([inv[int(v)] for v in gg["node"]])
        want_node = np.array([W.flat_index(Nl, g, i, j) for g, i, j in zip(go["grid"], go["i"], go["j"])])
        assert np.array_equal(flat_node, want_node)
        assert np.array_equal(gg["kind"], go["kind"])
        assert np.array_equal(gg["nst"], go["nst"])
        for k in range(n):
            ns = go["nst"][k]
            want = [W.flat_index(Nl, go["grid"][k], a, b) for a, b in go["st"][k][:ns]]
            got = [inv[int(v)] for v in gg["st"][k][:ns]]
            assert got == want
        assert np.abs(gg["w"] - go["w"]).max() < 1e-13
        bc = go["kind"] == 0
        if bc.any():
            assert np.abs(gg["B"][bc] - go["B"][bc]).max() < 1e-13
            assert np.abs(gg["theta"][bc] - go["theta"][bc]).max() < 1e-11


@pytest.mark.parametrize("case,N", [("circle", 64), ("flower5", 128), ("flower7", 256)])
def test_operator_pieces_match(case, N):
    o, s = pair(case, N)
    rng = np.random.default_rng(17)
    for lev in range(o.levels):
        Nl = N >> lev
        t = o.types(lev)
        x = W.random_flat(Nl, t, 100 + lev)
        b = W.random_flat(Nl, t, 200 + lev) * 10
        xd, bd = s.to_device(x, lev), s.to_device(b, lev)
        # residual, Eq. (LS)
        r_o, n_o = o.residual(x, b, lev)
        r_g, n_g = s.residual(xd, bd, lev)
        assert rel(s.to_flat(r_g, lev), r_o) < 1e-13
        assert abs(n_g - n_o) <= 1e-13 * n_o
        # relaxation pieces
        for name in ("box_sweep", "scalar_update", "ghost_sweep"):
            want = getattr(o, name)(x, b, lev)
            xg = s.to_device(x, lev)
            getattr(s, name)(xg, bd, lev)
            assert rel(s.to_flat(xg, lev), want) < 1e-12, (name, lev)
        want = o.smooth(x, b, 2, lev)
        xg = s.to_device(x, lev)
        s.smooth(xg, bd, 2, lev)
        assert rel(s.to_flat(xg, lev), want) < 1e-11
        if lev + 1 < o.levels:
            want = o.restrict(r_o, lev)
            got = s.to_flat(s.restrict(s.to_device(r_o, lev), lev), lev + 1)
            assert rel(got, want) < 1e-14
            tH = o.types(lev + 1)
            eH = W.random_flat(Nl // 2, tH, 300 + lev)
            want = o.prolong(eH, x, lev)
            xg = s.to_device(x, lev)
            s.prolong(s.to_device(eH, lev + 1), xg, lev)
            assert rel(s.to_flat(xg, lev), want) < 1e-14


@pytest.mark.parametrize("case,N", [("circle", 32), ("flower5", 128)])
def test_coarse_solve_matches(case, N):
    o, s = pair(case, N)
    lev = o.levels - 1
    t = o.types(lev)
    b = W.random_flat(N >> lev, t, 7)
    want = o.coarse_solve(b)
    got = s.to_flat(s.coarse_solve(s.to_device(b, lev)), lev)
    assert rel(got, want) < 1e-9


@pytest.mark.parametrize("case,N,ah2", [("circle", 64, None), ("flower5", 256, 2.0), ("ellipse", 128, 8.0)])
def test_cycle_history_matches(case, N, ah2):
    shape, x0, L = CASES[case]
    h = L / N
    alpha = None if ah2 is None else ah2 * h * h
    o, s = pair(case, N, alpha=alpha)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    x = np.zeros_like(b)
    xg, bd = s.to_device(x), s.to_device(b)
    for k in range(4):
        st, x = o.cycle(x, b)
        s.cycle(xg, bd)
        assert rel(s.to_flat(xg), x) < 1e-9, k
        _, no = o.residual(x, b)
        _, ng = s.residual(xg, bd)
        assert abs(ng - no) <= 1e-6 * no


def test_circle32_solve_matches_oracle():
    # circle r = 0.5, 32 x 32 on [-1, 1]^2, Re = 1, dt = h: alpha = h / 2;
    # Taylor-Green manufactured solution, solved to ||r||_inf <= 1e-12
    o, s = pair("circle", 32)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 1e-12, 100)
    assert st_o == 0
    xg = s.new_vec()
    st, rep, h_g = s.solve(xg, s.to_device(b), 1e-12)
    assert st == 0, s.error()
    assert rel(s.to_flat(xg), x_o) <= 1e-10
    assert len(h_g) == len(h_o)
    assert np.allclose(h_g, h_o, rtol=1e-6, atol=1e-13)


@pytest.mark.parametrize("case,N,Re", [("flower5", 256, 1000.0), ("circle_off", 256, 100.0)])
def test_solution_matches_oracle_config_params(case, N, Re):
    shape, x0, L = CASES[case]
    h = L / N
    alpha = h / (2.0 * Re)  # dt = h
    o, s = pair(case, N, alpha=alpha)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 1e-10, 100)
    assert st_o == 0
    xg = s.new_vec()
    st, rep, h_g = s.solve(xg, s.to_device(b), 1e-10)
    assert st == 0, s.error()
    assert rel(s.to_flat(xg), x_o) <= 1e-9
    assert abs(len(h_g) - len(h_o)) <= 1


@pytest.mark.parametrize("case,N,Re", [("flower5", 128, 1000.0), ("circle_off", 256, 100.0)])
def test_fp64_solutions_agree_near_the_rounding_floor(case, N, Re):
    # FP64 GPU and oracle both solved to ||r||_inf <= 5e-12: at these sizes the
    # residual's rounding floor is about 2.3e-12 (continuity rows carry 1/h),
    # so 1e-12 itself is out of reach; the solutions then agree to 1e-10
    shape, x0, L = CASES[case]
    alpha = (L / N) / (2.0 * Re)
    o, s = pair(case, N, alpha=alpha, max_cycles=200)
    b, xe, t, gh = manufactured(o, W.taylor_green())
    st_o, x_o, h_o = o.solve(np.zeros_like(b), b, 5e-12, 200)
    assert st_o == 0 and h_o[-1] <= 5e-12
    xg = s.new_vec()
    st, rep, h_g = s.solve(xg, s.to_device(b), 5e-12)
    assert st == 0, s.error()
    assert rel(s.to_flat(xg), x_o) <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(precision):
    # mg_solve replays each iteration as a captured CUDA graph on a side
    # stream; the iterate must be bitwise the one of direct launches
    import torch
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES["flower5"]
    N = 128
    lev = levels_for(N)
    h = L / N
    o, phi, st = make_oracle("flower5", N, alpha=h / 2000.0, levels=lev)
    ex = W.taylor_green()
    b, xe, t, gh = manufactured(o, ex)
    out = []
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=h / 2000.0, precision=precision, graphs=graphs,
                            stream=stream)
            assert s.geometry(phi) == 0, s.error()
            x = s.new_vec()
            bd = s.to_device(b)
            st, rep, hist = s.solve(x, bd, 1e-8)
            assert st == 0, s.error()
            x.zero_()
            st, rep2, hist2 = s.solve(x, bd, 1e-8)  # second solve replays the captured graph
            stream.synchronize()
            out.append((s.to_flat(x), hist2))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_large_level_relaxation_matches():
    # a level whose ghost-class rows (the walls alone give 4 N) exceed one
    # block's share: the box sweep, the (xi, mean) step and the fused ghost
    # sweeps of the multi-launch path, N = 1024
    o, s = pair("circle", 1024)
    t = o.types(0)
    x = W.random_flat(1024, t, 900)
    b = W.random_flat(1024, t, 901) * 10
    want = o.smooth(x, b, 1, 0)
    xg = s.to_device(x)
    s.smooth(xg, s.to_device(b), 1, 0)
    assert rel(s.to_flat(xg), want) < 1e-11
    want = o.ghost_sweep(x, b, 0)
    xg = s.to_device(x)
    s.ghost_sweep(xg, s.to_device(b), 0)
    assert rel(s.to_flat(xg), want) < 1e-12

