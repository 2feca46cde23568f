"""CUDA-graph replay of the apply: identical results to direct launches for both
precisions, across many (x, y) buffer pairs (more than the 64-graph cache holds, so
eviction is exercised), and in Davidson."""
import numpy as np
import pytest

import dmrg_synth as S

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_graph_equals_direct(tiny_problem, precision):
    import torch
    p = tiny_problem
    hg = lib.HEff.from_problem(p, precision=precision, max_nvec=2)
    hd = lib.HEff.from_problem(p, precision=precision, max_nvec=2, graphs=False)
    X = torch.from_numpy(p.random_vectors(2)).cuda()
    ys = []
    for _ in range(70):   # 70 distinct output buffers: beyond the 64-entry cache
        y = torch.empty_like(X)
        hg.apply(X, y, nvec=2)
        ys.append(y)
    yd = torch.empty_like(X)
    hd.apply(X, yd, nvec=2)
    torch.cuda.synchronize()
    for y in ys[::7] + [ys[-1]]:
        assert torch.equal(y, yd)
    # replay of a cached graph after new input values in the same buffer
    X.copy_(torch.from_numpy(p.random_vectors(2)[::-1].copy()))
    y0 = torch.empty_like(X)
    hg.apply(X, ys[-1], nvec=2)
    hd.apply(X, y0, nvec=2)
    torch.cuda.synchronize()
    assert torch.equal(ys[-1], y0)


def test_davidson_graph_equals_direct(tiny_problem):
    import torch
    p = tiny_problem
    res = []
    for graphs in (True, False):
        h = lib.HEff.from_problem(p, graphs=graphs)
        ev, info = h.davidson(torch.from_numpy(p.random_vectors(1)).cuda(), tol=1e-9)
        res.append((ev[0], info["iters"]))
    assert res[0] == res[1]
