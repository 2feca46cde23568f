"""GPU spin-adapted (SU(2)) H_eff*psi and eigensolvers against the SU(2) oracle, on
both precision paths: full products on the tiny workload for a triplet, a singlet
and a doublet target (several stacked vectors), the mid workload (1024 multiplets,
600 terms), the diagonal, the lowest eigenvalue from Davidson and Lanczos against the
dense reduced operator (tiny) and the converged oracle energy of the mid workload
(pinned in tests/golden), and the refusal of spin-adapted truncation."""
import json
import os

import numpy as np
import pytest

from dmrg_synth import su2 as G
from oracle import su2 as O
from tests.gpu_util import gpu_apply, rel_fro

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "synth_digests.json")
TOL = {"fp64": 1e-12, "split": 1e-11}
TARGETS = [(6, 2), (6, 0), (5, 1)]


@pytest.fixture(scope="module")
def mid():
    p = G.generate("su2_mid")
    X = p.random_vectors(2)
    return p, X, O.apply(p, X)


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("target", TARGETS, ids=["triplet", "singlet", "doublet"])
def test_tiny_apply(precision, target):
    p = G.generate("su2_tiny", target=target)
    X = p.random_vectors(3)
    ref = O.apply(p, X)
    h = lib.HEff.from_problem(p, precision=precision, max_nvec=3)
    for nv in (1, 3):
        Y = gpu_apply(h, X[:nv])
        for v in range(nv):
            assert rel_fro(Y[v], ref[v]) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_mid_apply(mid, precision):
    p, X, ref = mid
    h = lib.HEff.from_problem(p, precision=precision, max_nvec=2)
    Y = gpu_apply(h, X)
    for v in range(2):
        assert rel_fro(Y[v], ref[v]) <= TOL[precision]
    y1 = gpu_apply(h, X[1:2])[0]
    assert rel_fro(y1, ref[1]) <= TOL[precision]


@pytest.mark.parametrize("name", ["su2_tiny", "su2_mid"])
def test_diagonal(name):
    import torch
    p = G.generate(name)
    h = lib.HEff.from_problem(p)
    d = torch.empty(p.dim, dtype=torch.float64, device="cuda")
    h.diagonal(d)
    torch.cuda.synchronize()
    np.testing.assert_allclose(d.cpu().numpy(), O.diagonal(p), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("target", TARGETS, ids=["triplet", "singlet", "doublet"])
def test_tiny_lowest_eigenvalue(precision, target):
    import torch
    p = G.generate("su2_tiny", target=target)
    w0 = np.linalg.eigvalsh(O.apply(p, np.eye(p.dim)).T)[0]
    h = lib.HEff.from_problem(p, precision=precision)
    x = torch.from_numpy(p.random_vectors(1)).cuda()
    ev, info = h.davidson(x, tol=1e-9, max_iter=300)
    assert info["converged"] and abs(ev[0] - w0) <= 1e-10 * abs(w0)
    x = torch.from_numpy(p.random_vectors(1)[0]).cuda()
    ev, info = h.lanczos(x, tol=1e-9, max_iter=600, m_max=40)
    assert info["converged"] and abs(ev - w0) <= 1e-10 * abs(w0)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_mid_ground_state(precision):
    import torch
    e0 = json.load(open(GOLDEN))["su2_mid"]["e0"]
    p = G.generate("su2_mid")
    h = lib.HEff.from_problem(p, precision=precision)
    x = torch.from_numpy(p.random_vectors(1)).cuda()
    ev, info = h.davidson(x, tol=1e-9, max_iter=400)
    assert info["converged"] and abs(ev[0] - e0) <= 1e-10 * abs(e0)
    assert info["resid_max"] <= 1e-9


def test_truncation_refused():
    import torch
    p = G.generate("su2_tiny")
    h = lib.HEff.from_problem(p)
    with pytest.raises(lib.DmrgError):
        h.svd_truncate(torch.from_numpy(p.random_vectors(1)[0]).cuda(), 8)
