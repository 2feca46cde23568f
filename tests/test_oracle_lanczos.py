"""Pins of the Lanczos oracle against facts it does not compute itself: the dense
eigensolver (numpy eigh) on the tiny workload, the closed form of a free-fermion chain,
the tridiagonal structure Q^T H Q = T that defines the method (a wrong sign or index in
the three-term recurrence breaks it), and the invariant-subspace stop on an exact
eigenvector."""
import numpy as np

from oracle import heff
from oracle.lanczos import lanczos


def test_tiny_matches_dense_eigh(tiny_problem, tiny_dense):
    p = tiny_problem
    w = np.linalg.eigvalsh(tiny_dense)
    r = lanczos(lambda v: heff.apply(p, v), p.random_vectors(1)[0], tol=1e-10, max_iter=400, m_max=12)
    assert r["converged"] and r["restarts"] >= 1
    assert abs(r["eval"] - w[0]) <= 1e-12 * abs(w[0])
    assert r["resid"] <= 1e-9
    # the history is variational: every Ritz value lies above the ground state
    assert np.all(r["history"] >= w[0] - 1e-12 * abs(w[0]))


def test_free_fermion_chain_closed_form():
    from tests.test_oracle_models import _hubbard_two_block
    p = _hubbard_two_block(3, 1.0, 0.0, (6, 0))
    eps = np.sort(-2 * np.cos(np.arange(1, 7) * np.pi / 7))
    e0 = 2 * eps[:3].sum()
    x0 = np.random.default_rng(3).standard_normal(p.dim)
    r = lanczos(lambda v: heff.apply(p, v), x0, tol=1e-11, max_iter=300)
    assert r["converged"] and abs(r["eval"] - e0) <= 1e-12 * abs(e0)


def test_krylov_basis_is_orthonormal_and_tridiagonalises(tiny_problem, tiny_dense):
    # run a fixed number of steps by hand from the recurrence the oracle states and
    # compare with the dense operator: Q^T H Q must be the tridiagonal T
    H = tiny_dense
    p = tiny_problem
    q = p.random_vectors(1)[0]
    q = q / np.linalg.norm(q)
    seen = []
    r = lanczos(lambda v: (seen.append(v.copy()), heff.apply(p, v))[1], q, tol=0.0, max_iter=12, m_max=64)
    Q = np.array(seen[:12])   # the 13th apply is the final residual check
    assert len(seen) == 13 and np.allclose(Q @ Q.T, np.eye(12), atol=1e-13)
    T = Q @ H @ Q.T
    off = T - np.diag(np.diag(T)) - np.diag(np.diag(T, 1), 1) - np.diag(np.diag(T, -1), -1)
    assert np.abs(off).max() <= 1e-12 * np.abs(T).max()
    assert np.all(np.diag(T, 1) > 0)   # beta_j = ||w|| > 0
    # and its entries are the oracle's alpha_j = q_j.Hq_j and beta_j = ||w|| after reorth.
    np.testing.assert_allclose(np.diag(T), r["alpha"], rtol=0, atol=1e-12 * np.abs(T).max())
    np.testing.assert_allclose(np.diag(T, 1), r["beta"][:11], rtol=0, atol=1e-12 * np.abs(T).max())
    # its lowest eigenvalue is the oracle's Ritz value after 12 steps
    assert abs(np.linalg.eigvalsh(T)[0] - r["history"][-1]) <= 1e-12 * abs(r["history"][-1])


def test_exact_eigenvector_stops_at_once(tiny_problem, tiny_dense):
    w, V = np.linalg.eigh(tiny_dense)
    r = lanczos(lambda v: tiny_dense @ v, V[:, 0], tol=1e-12, max_iter=10)
    assert r["converged"] and r["iters"] == 1 and abs(r["eval"] - w[0]) <= 1e-13 * abs(w[0])
