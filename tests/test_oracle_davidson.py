"""Oracle Davidson against LAPACK (numpy.linalg.eigh on the dense H) and ARPACK
(scipy.sparse.linalg.eigsh on the oracle operator), which are independent
eigensolvers."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import davidson, heff


@pytest.fixture(scope="module")
def tiny(tiny_problem):
    return tiny_problem


def test_tiny_lowest_matches_eigh(tiny, tiny_dense):
    w = np.linalg.eigvalsh(tiny_dense)
    r = davidson.davidson(lambda V: heff.apply(tiny, V), heff.diagonal(tiny),
                          tiny.random_vectors(1), tol=1e-9)
    assert r["converged"]
    assert abs(r["evals"][0] - w[0]) <= 1e-12 * abs(w[0])


@pytest.mark.parametrize("k_eig,block", [(3, 1), (3, 4), (1, 8)])
def test_tiny_block_and_several_eigs(tiny, tiny_dense, k_eig, block):
    H = tiny_dense
    w, U = np.linalg.eigh(H)
    r = davidson.davidson(lambda V: heff.apply(tiny, V), heff.diagonal(tiny),
                          tiny.random_vectors(block), k_eig=k_eig, tol=1e-9)
    assert r["converged"]
    np.testing.assert_allclose(r["evals"], w[:k_eig], rtol=1e-12, atol=0)
    for i in range(k_eig):
        # eigenvector sign is arbitrary; the lowest levels here are non-degenerate
        assert abs(abs(r["evecs"][i] @ U[:, i]) - 1.0) < 1e-8
        assert np.linalg.norm(H @ r["evecs"][i] - r["evals"][i] * r["evecs"][i]) <= 1e-9


def test_mid_reduced_matches_arpack():
    scipy_linalg = pytest.importorskip("scipy.sparse.linalg")
    p = S.generate("mid", n_terms=40)
    op = scipy_linalg.LinearOperator((p.dim, p.dim), matvec=lambda v: heff.apply(p, v), dtype=np.float64)
    ref = scipy_linalg.eigsh(op, k=1, which="SA", tol=1e-12, v0=p.random_vectors(1)[0])[0][0]
    r = davidson.davidson(lambda V: heff.apply(p, V), heff.diagonal(p), p.random_vectors(1),
                          tol=1e-8, max_iter=400)
    assert r["converged"]
    assert abs(r["evals"][0] - ref) <= 1e-10 * abs(ref)


def test_cgs2_orthonormal():
    rng = np.random.default_rng(3)
    cand = rng.standard_normal((6, 50))
    cand[5] = cand[0] + 1e-14 * rng.standard_normal(50)   # numerically dependent
    V, acc = davidson.cgs2_append(np.zeros((0, 50)), cand)
    assert acc == 5
    np.testing.assert_allclose(V @ V.T, np.eye(5), atol=1e-15)


def test_precondition_floor():
    r = np.ones(3)
    d = np.array([1.0, 2.0 + 1e-10, 2.0])
    out = davidson.precondition(r, d, 2.0)
    assert out[0] == -1.0 and out[1] == 1e8 and out[2] == 1e8
