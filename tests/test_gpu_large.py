"""The large workload (D=8192 per block, 89 sectors, T=3500, |psi|=2,381,956, 114 GB of
FP64 operators, 10.5 TFLOP per H_eff*psi) on the FP64 path: one vector per apply, checked on 48 sampled output entries that the oracle
forms one by one (relative Frobenius error over the samples <= 1e-12), plus the
symmetry <x, H y> = <H x, y> on the full vectors.  The split path does not hold this
workload in HBM (operator and intermediate slices would need ~430 GB)."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import rel_fro

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")


def test_large_fp64_sampled_and_symmetric():
    import torch
    p = S.generate("large")
    assert p.dim == 2381956 and p.n_terms == 3500
    h = lib.HEff.from_problem(p, precision="fp64")   # one vector: 216 GB of the HBM
    X = p.random_vectors(2)
    Y = np.empty_like(X)
    for v in range(2):
        xd = torch.from_numpy(X[v]).cuda()
        yd = torch.empty_like(xd)
        h.apply(xd, yd)
        torch.cuda.synchronize()
        Y[v] = yd.cpu().numpy()
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(p.dim, 48, replace=False))
    assert rel_fro(Y[0][idx], heff.apply_entries(p, X[0], idx)) <= 1e-12
    # symmetry of H on the full vectors: <x0, H x1> = <H x0, x1>
    a, b = float(X[0] @ Y[1]), float(Y[0] @ X[1])
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b), np.linalg.norm(Y[0]) * np.linalg.norm(X[1]))
