"""gp_residual_static against gp_residual.

gp_residual_static serves callers that cannot obtain device memory for
scratch (work recorded under a capture mode that forbids allocation, or a
fixed shared workspace): its reduction scratch is a fixed array inside the
library.  It must return the same residual vector and norm as gp_residual,
on consecutive calls (the array keeps the previous call's contents), through
the C ABI.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import CASES, levels_for, make_oracle

pytestmark = pytest.mark.gpu


def test_static_scratch_residual_matches_workspace_residual():
    from paper_1911_00994_gb300 import gpmg
    shape, x0, L = CASES["flower5"]
    N = 128
    lev = levels_for(N)
    o, phi, st = make_oracle("flower5", N, levels=lev)
    s = gpmg.Solver(N, x0, x0, L, levels=lev, alpha=(L / N) / 2000.0)
    assert s.geometry(phi) == 0, s.error()
    t = o.types(0)
    for call, seed in enumerate((1, 2)):
        x = s.to_device(W.random_flat(N, t, 10 + seed))
        b = s.to_device(W.random_flat(N, t, 20 + seed) * 5)
        r_ws, n_ws = s.residual(x, b)
        r_st, n_st = s.residual_static(x, b)
        a, c = r_st.cpu().numpy(), r_ws.cpu().numpy()
        assert np.abs(a - c).max() <= 1e-13 * np.abs(c).max(), call
        assert abs(n_st - n_ws) <= 1e-13 * n_ws, call
    # a coarser level on the same array after the finer one
    Nc = N >> 2
    tc = o.types(2)
    x = s.to_device(W.random_flat(Nc, tc, 5), 2)
    b = s.to_device(W.random_flat(Nc, tc, 6), 2)
    r_ws, n_ws = s.residual(x, b, 2)
    r_st, n_st = s.residual_static(x, b, 2)
    assert np.abs(r_st.cpu().numpy() - r_ws.cpu().numpy()).max() <= 1e-13 * np.abs(r_ws.cpu().numpy()).max()
    assert abs(n_st - n_ws) <= 1e-13 * n_ws
