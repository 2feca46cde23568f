"""Full-vector parity at the two D=4096 sizes, against the oracle's whole H_eff*psi
(not sampled entries):

* precision (D=4096, 78 sectors, T=2000, |psi|=598,090): the FP64 path within 1e-12
  and the split path within 1e-11 relative Frobenius error, one vector;
* heavy-tailed (D=4096 log-normal dims, T=3000) with 8 stacked vectors, the launch
  configuration of the batching measurement: two of the eight results against the
  oracle on both paths, and every one of the eight against a one-vector apply of the
  same handle (the stacking must not change a result beyond rounding)."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import gpu_apply, rel_fro

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "split": 1e-11}

lib = pytest.importorskip("paper_2407_07411_gb300")


@pytest.fixture(scope="module")
def precision_ref():
    p = S.generate("precision")
    x = p.random_vectors(1)[0]
    return p, x, heff.apply(p, x)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_precision_full_vector(precision_ref, prec):
    p, x, ref = precision_ref
    h = lib.HEff.from_problem(p, precision=prec)
    y = gpu_apply(h, x)[0]
    h.close()
    assert np.all(np.isfinite(y))
    assert rel_fro(y, ref) <= TOL[prec]


@pytest.fixture(scope="module")
def heavy_ref():
    p = S.generate("heavy")
    assert p.n_terms == 3000
    X = p.random_vectors(8)
    picked = (0, 5)
    return p, X, picked, {v: heff.apply(p, X[v]) for v in picked}


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_heavy_full_terms_eight_vectors(heavy_ref, prec):
    p, X, picked, refs = heavy_ref
    h = lib.HEff.from_problem(p, precision=prec, max_nvec=8)
    Y = gpu_apply(h, X)
    for v in picked:
        assert rel_fro(Y[v], refs[v]) <= TOL[prec]
    for v in range(8):
        assert rel_fro(Y[v], gpu_apply(h, X[v])[0]) <= 1e-13
    h.close()
