"""GPU restarted Lanczos (the eigensolver alternative the paper names beside Davidson)
on both precision paths: the lowest eigenvalue against the dense eigensolver (tiny),
the closed form of a free-fermion chain, the converged oracle ground-state energy of the
mid workload (pinned in tests/golden), the oracle Lanczos history step by step, the
restart path, and argument checks."""
import json
import os

import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from oracle.lanczos import lanczos as oracle_lanczos

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "synth_digests.json")


def gpu_lanczos(p, precision="fp64", **kw):
    import torch
    h = lib.HEff.from_problem(p, precision=precision)
    x = torch.from_numpy(p.random_vectors(1)[0]).cuda()
    ev, info = h.lanczos(x, **kw)
    return ev, info, x.cpu().numpy()


@pytest.mark.parametrize("precision,tol_e", [("fp64", 1e-12), ("split", 1e-10)])
def test_tiny_matches_dense(tiny_problem, tiny_dense, precision, tol_e):
    w = np.linalg.eigvalsh(tiny_dense)
    ev, info, x = gpu_lanczos(tiny_problem, precision, tol=1e-10, max_iter=400, m_max=12)
    assert info["converged"] and info["restarts"] >= 1
    assert abs(ev - w[0]) <= tol_e * abs(w[0])
    assert abs(np.linalg.norm(x) - 1.0) <= 1e-12
    assert info["resid_max"] <= 1e-8
    assert np.all(info["theta"] >= w[0] - 1e-10 * abs(w[0]))   # variational


def test_matches_oracle_history(tiny_problem):
    p = tiny_problem
    ev, info, _ = gpu_lanczos(p, "fp64", tol=0.0, max_iter=10, m_max=63)
    r = oracle_lanczos(lambda v: heff.apply(p, v), p.random_vectors(1)[0], tol=0.0, max_iter=10, m_max=63)
    assert not info["converged"] and info["iters"] == 10
    np.testing.assert_allclose(info["theta"], r["history"], rtol=1e-10)


def test_free_fermion_chain_closed_form():
    from tests.test_oracle_models import _hubbard_two_block
    p = _hubbard_two_block(3, 1.0, 0.0, (6, 0))
    eps = np.sort(-2 * np.cos(np.arange(1, 7) * np.pi / 7))
    e0 = 2 * eps[:3].sum()
    ev, info, _ = gpu_lanczos(p, "fp64", tol=1e-10, max_iter=300)
    assert info["converged"] and abs(ev - e0) <= 1e-10 * abs(e0)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_mid_ground_state(precision):
    e0 = json.load(open(GOLDEN))["mid"]["e0"]
    ev, info, _ = gpu_lanczos(S.generate("mid"), precision, tol=1e-9, max_iter=2000, m_max=63)
    assert info["converged"] and abs(ev - e0) <= 1e-10 * abs(e0)
    assert info["resid_max"] <= 1e-8


def test_arguments(tiny_problem):
    import torch
    h = lib.HEff.from_problem(tiny_problem)
    for kw in (dict(m_max=1), dict(m_max=64), dict(max_iter=0), dict(tol=-1.0)):
        with pytest.raises(lib.DmrgError):
            h.lanczos(torch.ones(tiny_problem.dim, dtype=torch.float64, device="cuda"), **kw)
    with pytest.raises(lib.DmrgError):
        h.lanczos(torch.zeros(tiny_problem.dim, dtype=torch.float64, device="cuda"))
