"""gp_residual_static against gp_residual and the oracle.

gp_residual_static serves callers that cannot allocate device memory (a
plug-in inside a host application that owns all device memory, or a caller
whose workspace was sized once for other work): its reduction scratch is a
fixed array inside the library.  It must return the same residual vector and
norm as gp_residual, and the oracle's residual, on consecutive calls (the
array keeps the previous call's contents), through the C ABI, and it must
allocate nothing.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle

pytestmark = pytest.mark.gpu


def _nan_vec(s, lev):
    r = s.new_vec(lev)
    r.fill_(float("nan"))
    return r


def test_static_scratch_residual_matches_workspace_residual_and_oracle():
    import torch
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES["flower5"]
    N = 128
    lev = levels_for(N)
    alpha = (L / N) / 2000.0
    o, phi, st = make_oracle("flower5", N, levels=lev, alpha=alpha)
    assert st == 0, o.error()
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=alpha)
    assert s.geometry(phi) == 0, s.error()
    t = o.types(0)
    assert np.array_equal(s.types_flat(0)[:-1], t[:-1])
    for call, seed in enumerate((1, 2)):
        xf = W.random_flat(N, t, 10 + seed)
        bf = W.random_flat(N, t, 20 + seed) * 5
        x, b = s.to_device(xf), s.to_device(bf)
        r_ws, n_ws = s.residual(x, b)
        r_out = _nan_vec(s, 0)
        torch.cuda.synchronize()
        mem0 = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        r_st, n_st = s.residual_static(x, b, r=r_out)
        torch.cuda.synchronize()
        # nothing allocated: torch's allocator holds no more memory and the
        # device's free memory is unchanged (a cudaMalloc would lower it)
        assert torch.cuda.memory_allocated() <= mem0, call
        assert torch.cuda.mem_get_info()[0] == free0, call
        assert r_st is r_out
        a, c = r_st.cpu().numpy(), r_ws.cpu().numpy()
        # every slot of the three frames and the mean row written (the 31
        # trailing scalar slots are padding), equal to the workspace residual
        assert np.isfinite(a[:3 * gpmg.frame(N) + 1]).all(), call
        a, c = a[:3 * gpmg.frame(N) + 1], c[:3 * gpmg.frame(N) + 1]
        assert np.abs(a - c).max() <= 1e-13 * np.abs(c).max(), call
        assert abs(n_st - n_ws) <= 1e-13 * n_ws, call
        # the oracle's residual of the same system (its own rows, FP64)
        r_or, n_or = o.residual(xf, bf)
        rf = s.to_flat(r_st)
        assert np.abs(rf - r_or).max() <= 1e-12 * np.abs(r_or).max(), call
        assert abs(n_st - n_or) <= 1e-12 * n_or, call
        # without a norm pointer: the same vector, no synchronisation
        r2, n2 = s.residual_static(x, b, r=_nan_vec(s, 0), want_norm=False)
        torch.cuda.synchronize()
        assert n2 is None
        assert np.array_equal(r2.cpu().numpy()[:a.size], a), call
    # a coarser level on the same array after the finer one
    Nc = N >> 2
    tc = o.types(2)
    xf, bf = W.random_flat(Nc, tc, 5), W.random_flat(Nc, tc, 6)
    x, b = s.to_device(xf, 2), s.to_device(bf, 2)
    r_ws, n_ws = s.residual(x, b, 2)
    r_st, n_st = s.residual_static(x, b, 2, r=_nan_vec(s, 2))
    n_used = 3 * gpmg.frame(Nc) + 1
    a, c = r_st.cpu().numpy()[:n_used], r_ws.cpu().numpy()[:n_used]
    assert np.isfinite(a).all()
    assert np.abs(a - c).max() <= 1e-13 * np.abs(c).max()
    assert abs(n_st - n_ws) <= 1e-13 * n_ws
    r_or, n_or = o.residual(xf, bf, lev=2)
    assert np.abs(s.to_flat(r_st, 2) - r_or).max() <= 1e-12 * np.abs(r_or).max()
