"""Pins of the renormalisation oracle (O' = U_p^T O U_q per block) against facts it does
not compute: identity bases change nothing; square orthogonal bases keep Frobenius norms
and the spectrum of a symmetric diagonal block, and commute with products, (AB)' = A'B'
(a transposed or swapped basis breaks it); a basis of leading eigenvectors truncates a
symmetric block to the diagonal of its leading eigenvalues.  Plus the argument checks of
the C entry point, which run on the host before any device work."""
import ctypes

import numpy as np
import pytest

from oracle.renorm import basis_offsets, renormalise


def _orthogonal(rng, d, k):
    q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    return q[:, :k]


def _setup(rng, dims, dims_new):
    U = np.concatenate([_orthogonal(rng, d, k).ravel() for d, k in zip(dims, dims_new)])
    return U


def test_identity_bases():
    rng = np.random.default_rng(0)
    dims = [3, 5, 2]
    U = np.concatenate([np.eye(d).ravel() for d in dims])
    A = rng.standard_normal((5, 3))
    out = renormalise(dims, dims, U, [(0, 1, 0)], A.ravel())
    np.testing.assert_array_equal(out[0], A)


def test_orthogonal_bases_norm_spectrum_and_products():
    rng = np.random.default_rng(1)
    dims = [4, 6, 3]
    U = _setup(rng, dims, dims)
    A = rng.standard_normal((6, 4))          # A[1 <- 0]
    B = rng.standard_normal((4, 3))          # B[0 <- 2]
    S = rng.standard_normal((6, 6)); S = S + S.T   # S[1 <- 1]
    op = np.concatenate([A.ravel(), B.ravel(), (A @ B).ravel(), S.ravel()])
    blocks = [(0, 1, 0), (2, 0, 24), (2, 1, 36), (1, 1, 54)]
    Ap, Bp, ABp, Sp = renormalise(dims, dims, U, blocks, op)
    assert abs(np.linalg.norm(Ap) - np.linalg.norm(A)) <= 1e-13 * np.linalg.norm(A)
    np.testing.assert_allclose(ABp, Ap @ Bp, rtol=0, atol=1e-13 * np.abs(ABp).max())
    np.testing.assert_allclose(np.linalg.eigvalsh(Sp), np.linalg.eigvalsh(S), rtol=0, atol=1e-12)


def test_truncation_to_leading_eigenvectors():
    rng = np.random.default_rng(2)
    S = rng.standard_normal((7, 7)); S = S + S.T
    w, V = np.linalg.eigh(S)
    k = 3
    U = V[:, ::-1][:, :k].copy()             # eigenvectors of the k largest eigenvalues
    out = renormalise([7], [k], U.ravel(), [(0, 0, 0)], S.ravel())
    np.testing.assert_allclose(out[0], np.diag(w[::-1][:k]), rtol=0, atol=1e-12)
    assert list(basis_offsets([7, 2], [3, 1])) == [0, 21, 23]


def test_entry_point_rejects_bad_arguments():
    lib = pytest.importorskip("paper_2407_07411_gb300")
    f = lib._lib.dmrg_renormalise
    dims = (ctypes.c_int32 * 2)(4, 3)
    fake = ctypes.c_void_p(16)   # never dereferenced: the checks fail first
    off = (ctypes.c_int64 * 1)()

    def call(dn, blk, op_len=100, out_len=100):
        d2 = (ctypes.c_int32 * 2)(*dn)
        b = (ctypes.c_int64 * 3)(*blk)
        return f(2, dims, d2, fake, b, 1, fake, op_len, fake, out_len, off, None)

    bad = lib.ERR_INVALID_ARG
    assert call((5, 3), (0, 1, 0)) == bad          # new dim above the dim
    assert call((0, 3), (0, 1, 0)) == bad          # new dim below 1
    assert call((2, 2), (2, 1, 0)) == bad          # sector out of range
    assert call((2, 2), (0, 1, 90)) == bad         # 3 x 4 block beyond op_len = 100
    assert call((2, 2), (0, 1, 0), out_len=3) == bad   # 2 x 2 result does not fit
    assert f(2, dims, dims, None, None, 1, None, 0, None, 0, None, None) == bad   # null arrays
