"""Oracle: block Davidson for the lowest eigenpairs of H_eff.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper solves each local update as a large Hermitian eigenvalue problem with
Lanczos or Davidson (Numerical procedure, after Eq. 2) and names no variant.
The variant fixed here, step by step, is:

  0. V = CGS2-orthonormalised start block (b vectors), W = H V.
  1. Rayleigh-Ritz: S = V W^T (symmetrised), S U = U diag(theta), theta ascending.
  2. Ritz pairs i < kb = min(m, max(k_eig, b)): x_i = U_i^T V, Hx_i = U_i^T W,
     r_i = Hx_i - theta_i x_i.
  3. Converged when ||r_i|| <= tol for every i < k_eig (or after n_iter
     Rayleigh-Ritz steps when a fixed count is asked for).
  4. Corrections for the first b pairs i < kb with ||r_i|| > tol:
     delta_i = r_i / (diag - theta_i), a denominator of magnitude < 1e-8
     replaced by 1e-8 with its sign (+1e-8 for zero).
  5. Thick restart when m + (#corrections) > m_max: keep the lowest
     min(m, k_eig + b) Ritz vectors, V <- U[:, :r]^T V and W <- U[:, :r]^T W.
  6. Each correction, in order, is orthogonalised against the current basis
     twice (classical Gram-Schmidt, two passes), dropped if its norm fell
     below 1e-10 of its norm before, else normalised and appended; the
     accepted block is multiplied by H and appended to W.
  7. Stop without convergence if no correction was accepted.
m_max defaults to max(8 b, 24) and must be at least k_eig + 2 b.
"""
from __future__ import annotations

import numpy as np

DENOM_FLOOR = 1e-8
DROP_RATIO = 1e-10


def cgs2_append(V: np.ndarray, cand: np.ndarray) -> tuple[np.ndarray, int]:
    """Append each row of cand to the orthonormal rows of V after two passes
    of classical Gram-Schmidt; returns (new V, number accepted)."""
    rows = [V[i] for i in range(V.shape[0])]
    acc = 0
    for v in cand:
        v = np.array(v, np.float64)
        n0 = np.linalg.norm(v)
        if n0 == 0.0:
            continue
        for _ in range(2):
            if rows:
                B = np.array(rows)
                v = v - B.T @ (B @ v)
        n1 = np.linalg.norm(v)
        if n1 < DROP_RATIO * n0:
            continue
        rows.append(v / n1)
        acc += 1
    n = V.shape[1] if V.ndim == 2 else cand.shape[1]
    return (np.array(rows) if rows else np.zeros((0, n))), acc


def precondition(r: np.ndarray, diag: np.ndarray, theta: float) -> np.ndarray:
    den = diag - theta
    small = np.abs(den) < DENOM_FLOOR
    den = np.where(small, np.where(den < 0, -DENOM_FLOOR, DENOM_FLOOR), den)
    return r / den


def davidson(apply_fn, diag, X0, k_eig=1, tol=1e-8, max_iter=300, m_max=None, n_iter=None):
    """Lowest k_eig eigenpairs of the symmetric operator apply_fn ((b, n) -> (b, n)).

    Returns a dict with evals (k_eig,), evecs (k_eig, n), resid (k_eig,),
    iters (Rayleigh-Ritz steps), matvecs, converged, history (iters, k_eig) of
    the lowest Ritz values per step (nan while the basis is smaller than k_eig)."""
    X0 = np.atleast_2d(np.asarray(X0, np.float64))
    b, n = X0.shape
    m_max = m_max or max(8 * b, 24)
    if m_max < k_eig + 2 * b:
        raise ValueError("m_max must be at least k_eig + 2*block")
    V, acc = cgs2_append(np.zeros((0, n)), X0)
    if acc == 0:
        raise ValueError("start block is numerically zero")
    W = np.asarray(apply_fn(V), np.float64)
    matvecs = V.shape[0]
    history = []
    converged = False
    it = 0
    while it < max_iter:
        it += 1
        S = V @ W.T
        S = 0.5 * (S + S.T)
        theta, U = np.linalg.eigh(S)
        m = V.shape[0]
        kb = min(m, max(k_eig, b))
        X = U[:, :kb].T @ V
        HX = U[:, :kb].T @ W
        R = HX - theta[:kb, None] * X
        rn = np.linalg.norm(R, axis=1)
        h = np.full(k_eig, np.nan)
        h[:min(k_eig, kb)] = theta[:min(k_eig, kb)]
        history.append(h)
        if kb >= k_eig and np.all(rn[:k_eig] <= tol):
            converged = True
            break
        if n_iter is not None and it >= n_iter:
            break
        sel = [i for i in range(kb) if rn[i] > tol][:b]
        cand = np.array([precondition(R[i], diag, theta[i]) for i in sel])
        if m + len(sel) > m_max:
            r = min(m, k_eig + b)
            V = U[:, :r].T @ V
            W = U[:, :r].T @ W
        m_old = V.shape[0]
        V, acc = cgs2_append(V, cand)
        if acc == 0:
            break
        W = np.vstack([W, np.asarray(apply_fn(V[m_old:]), np.float64)])
        matvecs += acc
    k = min(k_eig, kb)
    return dict(evals=theta[:k].copy(), evecs=X[:k].copy(), resid=rn[:k].copy(), iters=it,
                matvecs=matvecs, converged=converged, history=np.array(history))
