"""GPU spin-adapted (SU(2)) H_eff*psi and eigensolvers against the SU(2) oracle, on
both precision paths: full products on the tiny workload for a triplet, a singlet
and a doublet target (several stacked vectors), the mid workload (1024 multiplets,
600 terms), the diagonal, the lowest eigenvalue from Davidson and Lanczos against the
dense reduced operator (tiny) and the converged oracle energy of the mid workload
(pinned in tests/golden), a block Davidson for the two lowest, results bit-identical
across schedules and after autotuning, and the two-site decomposition per left sector."""
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


@pytest.mark.parametrize("name,target,D", [("su2_tiny", (6, 2), 30), ("su2_tiny", (5, 1), 12),
                                           ("su2_mid", None, 400)])
def test_truncation_matches_oracle(name, target, D):
    """Per left sector (its blocks side by side): singular values, kept counts,
    discarded weight and the kept bases through their projectors."""
    import torch
    p = G.generate(name, target=target)
    h = lib.HEff.from_problem(p)
    psi = p.random_vectors(1)[0]
    r = h.svd_truncate(torch.from_numpy(psi).cuda(), D)
    ref = O.truncate(p, psi, D)
    assert list(r["sectors"]) == ref["sectors"]
    smax = max(s[0] for s in ref["sv"])
    for s, t in zip(r["sv"], ref["sv"]):
        np.testing.assert_allclose(s, t, rtol=0, atol=1e-13 * smax)
    assert list(r["kept"]) == ref["kept"] and sum(ref["kept"]) == D
    assert abs(r["discarded"] - ref["discarded"]) <= 1e-12
    U = r["U"].cpu().numpy()
    mats = h.svd_matrices()
    for m, k in enumerate(r["kept"]):
        if k == 0:
            continue
        rows = int(mats[m, 1])
        Ug = U[r["u_off"][m]:r["u_off"][m] + rows * k].reshape(rows, k)
        np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-12)
        assert np.linalg.norm(Ug @ Ug.T - ref["U"][m] @ ref["U"][m].T) <= 1e-9


def test_split_schedules_and_autotune():
    """Spin-adapted plans under other schedules: the split result bit for bit, and the
    autotuned schedule within tolerance (same contract as the U(1) path)."""
    p = G.generate("su2_mid", n_terms=150, target=(20, 2))
    X = p.random_vectors(2)
    ref = O.apply(p, X)
    h = lib.HEff.from_problem(p, precision="split", max_nvec=2)
    y0 = gpu_apply(h, X)
    assert rel_fro(y0, ref) <= TOL["split"]
    base = dict(fp64_kchunk=[512, 512, 2048], fp64_ctas_per_sm=0, split_kchunk=[0, 0, 0], per_gemm=0, fp64_tile=0)
    for sched in (dict(base, split_kchunk=[8, 64, 256]), dict(base, per_gemm=1)):
        h.schedule = sched
        assert np.array_equal(gpu_apply(h, X), y0)
    r = h.autotune(nvec=2, reps=2)
    assert 0 < r["best_ms"] <= r["default_ms"] and h.schedule == r["best"]
    assert rel_fro(gpu_apply(h, X), ref) <= TOL["split"]


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_tiny_block_davidson_two_lowest(precision):
    import torch
    p = G.generate("su2_tiny", target=(6, 2))
    w = np.linalg.eigvalsh(O.apply(p, np.eye(p.dim)).T)
    h = lib.HEff.from_problem(p, precision=precision, max_nvec=2)
    x = torch.from_numpy(p.random_vectors(2)).cuda()
    ev, info = h.davidson(x, k_eig=2, tol=1e-9, max_iter=300, block=2)
    assert info["converged"]
    np.testing.assert_allclose(ev[:2], w[:2], rtol=1e-10)
