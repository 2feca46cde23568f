"""The large workload (D=8192 per block, 89 sectors, T=3500, |psi|=2,381,956, 114 GB of
FP64 operators, 10.5 TFLOP per H_eff*psi) on both paths, one vector per apply:

* FP64: 48 sampled output entries that the oracle forms one by one (relative Frobenius
  error over the samples <= 1e-12), the symmetry <x, H y> = <H x, y> on the full
  vectors;
* split: the operators streamed window by window through the slicer (no resident FP64
  copy), the output blocks in two chunks that share one intermediate buffer; the same
  sampled entries against the oracle (<= 1e-11), the full vectors against the FP64
  path's (<= 1e-11), the symmetry, and the diagonal bit for bit against the FP64
  path's (both form it with the same arithmetic)."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import rel_fro

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")


def _applies(h, X):
    import torch
    Y = np.empty_like(X)
    for v in range(X.shape[0]):
        xd = torch.from_numpy(X[v]).cuda()
        yd = torch.empty_like(xd)
        h.apply(xd, yd)
        torch.cuda.synchronize()
        Y[v] = yd.cpu().numpy()
    return Y


def _diag(h, dim):
    import torch
    d = torch.empty(dim, dtype=torch.float64, device="cuda")
    h.diagonal(d)
    torch.cuda.synchronize()
    return d.cpu().numpy()


def _symmetric(X, Y, tol):
    a, b = float(X[0] @ Y[1]), float(Y[0] @ X[1])
    return abs(a - b) <= tol * max(abs(a), abs(b), np.linalg.norm(Y[0]) * np.linalg.norm(X[1]))


@pytest.fixture(scope="module")
def large():
    p = S.generate("large")
    assert p.dim == 2381956 and p.n_terms == 3500
    X = p.random_vectors(2)
    idx = np.sort(np.random.default_rng(7).choice(p.dim, 48, replace=False))
    ref = heff.apply_entries(p, X[0], idx)
    h = lib.HEff.from_problem(p, precision="fp64")
    Y = _applies(h, X)
    diag = _diag(h, p.dim)
    h.close()
    return p, X, idx, ref, Y, diag


def test_large_fp64_sampled_and_symmetric(large):
    p, X, idx, ref, Y, _ = large
    assert rel_fro(Y[0][idx], ref) <= 1e-12
    assert _symmetric(X, Y, 1e-12)


def test_large_split_streamed_in_chunks(large):
    p, X, idx, ref, Y64, diag64 = large
    h = lib.HEff.from_problem(p, precision="split")
    mem = h.memory()
    assert mem["operators"] == 0 and mem["total"] < 280e9
    Y = _applies(h, X)
    diag = _diag(h, p.dim)
    h.close()
    assert np.all(np.isfinite(Y))
    assert rel_fro(Y[0][idx], ref) <= 1e-11
    for v in range(2):
        assert rel_fro(Y[v], Y64[v]) <= 1e-11
    assert _symmetric(X, Y, 1e-11)
    assert np.array_equal(diag, diag64)
