"""Pins of the decomposition/truncation oracle against facts it does not compute
itself: squared singular values are the eigenvalues of M M^T (numpy eigh), a rank-one
block u v^T has the single singular value |u||v| with left vector +-u/|u|, a diagonal
block's singular values are its sorted absolute diagonal, the kept and discarded weights
add up to ||psi||^2, and ties go to the earlier block."""
import numpy as np

from oracle.svd import truncate


def _blocks(shapes):
    offs, o = [], 0
    for r, c in shapes:
        offs.append((o, r, c))
        o += r * c
    return offs, o


def test_singular_values_are_roots_of_gram_eigenvalues():
    rng = np.random.default_rng(0)
    blocks, n = _blocks([(5, 7), (6, 3), (4, 4)])
    psi = rng.standard_normal(n)
    r = truncate(blocks, psi, D=100)
    for (off, rows, cols), s in zip(blocks, r["sv"]):
        M = psi[off:off + rows * cols].reshape(rows, cols)
        ev = np.sort(np.linalg.eigvalsh(M @ M.T))[::-1][:min(rows, cols)]
        np.testing.assert_allclose(s ** 2, ev, rtol=1e-12, atol=1e-13)
    assert r["discarded"] <= 1e-12 * float(psi @ psi)
    # kept bases are orthonormal
    for u in r["U"]:
        np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)


def test_rank_one_and_diagonal_blocks():
    u, v = np.array([1.0, -2.0, 2.0]), np.array([3.0, 4.0])
    d = np.array([0.5, -3.0, 2.0])
    blocks, n = _blocks([(3, 2), (3, 3)])
    psi = np.concatenate([np.outer(u, v).ravel(), np.diag(d).ravel()])
    r = truncate(blocks, psi, D=2)
    assert abs(r["sv"][0][0] - 15.0) <= 1e-13 and r["sv"][0][1] <= 1e-14
    np.testing.assert_allclose(r["sv"][1], [3.0, 2.0, 0.5], rtol=1e-14)
    # D = 2 keeps 15 (block 0) and 3 (block 1); the rank-one basis is +-u / |u|
    assert r["kept"] == [1, 1]
    assert abs(abs(float(r["U"][0][:, 0] @ u)) - 3.0) <= 1e-13
    assert abs(r["discarded"] - (2.0 ** 2 + 0.5 ** 2)) <= 1e-12
    assert abs(sum(float(s @ s) for s in r["sv"]) - float(psi @ psi)) <= 1e-11


def test_ties_go_to_the_earlier_block():
    blocks, n = _blocks([(2, 2), (2, 2)])
    psi = np.concatenate([np.eye(2).ravel(), np.eye(2).ravel()])
    r = truncate(blocks, psi, D=3)
    assert r["kept"] == [2, 1] and abs(r["discarded"] - 1.0) <= 1e-13
