"""Oracle: restarted Lanczos for the lowest eigenpair of H_eff.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper solves each local update as a large Hermitian eigenvalue problem with
Lanczos or Davidson (Numerical procedure, after Eq. 2) and names no variant.
The variant fixed here, step by step:

  0. q_0 = x0 / ||x0||, beta_{-1} = 0, j = 0.
  1. w = H q_j;  alpha_j = q_j . w;  w <- w - alpha_j q_j - beta_{j-1} q_{j-1}.
  2. Full reorthogonalisation: w against q_0 .. q_j, two passes of classical
     Gram-Schmidt.  beta_j = ||w||.
  3. Rayleigh-Ritz on the tridiagonal T_j (diagonal alpha_0 .. alpha_j, off-diagonal
     beta_0 .. beta_{j-1}): lowest eigenpair (theta, s).  The Ritz vector
     y = sum_i s_i q_i has the residual ||H y - theta y|| = beta_j |s_j|.
  4. Converged when beta_j |s_j| <= tol.  If beta_j < 1e-10 of the norm of w before
     step 2, the Krylov space is invariant and theta is exact: stop.
  5. Otherwise q_{j+1} = w / beta_j and j <- j + 1; when T_j has m_max rows, restart
     from q_0 = y / ||y||.
"""
from __future__ import annotations

import numpy as np

BREAKDOWN = 1e-10


def lanczos(apply_fn, x0, tol=1e-8, max_iter=300, m_max=64):
    """Lowest eigenpair of the symmetric operator apply_fn (vector -> vector).
    Returns dict(eval, x, iters, matvecs, restarts, converged, resid, history, alpha,
    beta) with history[k] the lowest Ritz value after step k + 1 and alpha, beta the
    tridiagonal of the last cycle."""
    q = np.asarray(x0, np.float64).ravel()
    q = q / np.linalg.norm(q)
    Q, alpha, beta = [q], [], []
    hist = []
    matvecs = restarts = 0
    theta, y, converged = None, q, False
    for it in range(max_iter):
        j = len(Q) - 1
        w = apply_fn(Q[j])
        matvecs += 1
        a = float(Q[j] @ w)
        w = w - a * Q[j]
        if j > 0:
            w = w - beta[j - 1] * Q[j - 1]
        n_before = np.linalg.norm(w)
        for _ in range(2):
            for qi in Q:
                w = w - float(qi @ w) * qi
        b = float(np.linalg.norm(w))
        alpha.append(a)
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        ev, U = np.linalg.eigh(T)
        theta, s = float(ev[0]), U[:, 0]
        hist.append(theta)
        y = np.array(Q).T @ s
        invariant = b < BREAKDOWN * n_before
        if b * abs(s[-1]) <= tol or invariant:
            converged = True
            break
        if len(Q) == m_max:   # restart from the Ritz vector
            y = y / np.linalg.norm(y)
            Q, alpha, beta = [y], [], []
            restarts += 1
            continue
        beta.append(b)
        Q.append(w / b)
    y = y / np.linalg.norm(y)
    resid = float(np.linalg.norm(apply_fn(y) - theta * y))
    return dict(eval=theta, x=y, iters=len(hist), matvecs=matvecs + 1, restarts=restarts,
                converged=converged, resid=resid, history=np.array(hist), alpha=np.array(alpha),
                beta=np.array(beta))
