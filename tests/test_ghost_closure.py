"""The closure argument behind the fused ghost sweeps, checked on the oracle's
ghost-class rows (Eq. ghostrelax: lambda Jacobi sweeps over the ghost rows with
the internal values fixed).

A block that owns a run of consecutive rows and relaxes them together with
every row within lambda - 1 stencil links (a link counts as zero once it leaves
that set) ends with exactly the owned rows' values after lambda plain sweeps,
because a row at link distance h stays exact for the first lambda - h sweeps.
The CUDA path lists these closures once per geometry, with room for 512 rows
per block of 128; the test geometries need far fewer.
"""
import numpy as np
import pytest

from paper_1911_00994_gb300 import workloads as W
from tests._cases import make_oracle

OWN, CAP, LAM, DTAU = 128, 512, 5, 0.9


def rows_of(o, lev):
    Nl = o.N >> lev
    go = o.ghosts(lev)
    n = len(go["grid"])
    node = [W.flat_index(Nl, g, i, j) for g, i, j in zip(go["grid"], go["i"], go["j"])]
    row_of = {v: k for k, v in enumerate(node)}
    st = [[W.flat_index(Nl, go["grid"][k], a, b) for a, b in go["st"][k][:go["nst"][k]]] for k in range(n)]
    w = [list(go["w"][k][:go["nst"][k]]) for k in range(n)]
    link = [[row_of.get(s, -1) for s in st[k]] for k in range(n)]
    return node, st, w, link


def sweeps(rows, node, st, w, link, x, b, lam):
    """lam sweeps over `rows` (list of row ids); links outside count as 0."""
    pos = {r: i for i, r in enumerate(rows)}
    d = [0.0] * len(rows)
    for s in range(lam):
        dn = []
        for c, k in enumerate(rows):
            res = b[node[k]]
            for q in range(len(st[k])):
                xq = x[st[k][q]]
                if s > 0 and link[k][q] in pos:
                    xq = xq + d[pos[link[k][q]]]
                res -= w[k][q] * xq
            dn.append(d[c] + DTAU * res)
        d = dn
    return dict(zip(rows, d))


@pytest.mark.parametrize("case,N,lev", [("flower7", 256, 0), ("flower5", 512, 0), ("ellipse", 256, 0)])
def test_closure_sweeps_equal_plain_sweeps(case, N, lev):
    o, phi, st = make_oracle(case, N)
    assert st == 0
    node, stn, w, link = rows_of(o, lev)
    n = len(node)
    assert n > OWN
    rng = np.random.default_rng(N + lev)
    x = rng.standard_normal(o.n(lev)).tolist()
    b = rng.standard_normal(o.n(lev)).tolist()
    want = sweeps(list(range(n)), node, stn, w, link, x, b, LAM)
    linked = 0
    for lo in range(0, n, OWN):
        own = set(range(lo, min(n, lo + OWN)))
        cl = set(own)
        for _ in range(LAM - 1):
            cl |= {l for r in cl for l in link[r] if l >= 0}
        assert len(cl) <= CAP
        linked += len(cl) > len(own)
        got = sweeps(sorted(cl), node, stn, w, link, x, b, LAM)
        for k in own:
            assert got[k] == want[k], (lo, k)
    # the rows are coupled, so the closures do reach past the owned runs
    assert linked > 0


def test_closure_needs_every_hop():
    # on the seven-petal flower some blocks' closures still grow at link
    # distance lambda - 1; stopping one hop short changes an owned row there
    o, phi, st = make_oracle("flower7", 256)
    assert st == 0
    node, stn, w, link = rows_of(o, 0)
    n = len(node)
    rng = np.random.default_rng(256)
    x = rng.standard_normal(o.n(0)).tolist()
    b = rng.standard_normal(o.n(0)).tolist()
    want = sweeps(list(range(n)), node, stn, w, link, x, b, LAM)
    grew = 0
    for lo in range(0, n, OWN):
        own = set(range(lo, min(n, lo + OWN)))
        short = set(own)
        for _ in range(LAM - 2):
            short |= {l for r in short for l in link[r] if l >= 0}
        full = short | {l for r in short for l in link[r] if l >= 0}
        if full == short:
            continue
        grew += 1
        got = sweeps(sorted(short), node, stn, w, link, x, b, LAM)
        assert any(got[k] != want[k] for k in own), lo
    assert grew > 0
