"""Oracle: the two-site effective Hamiltonian in block-sparse form.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The operator is the restriction of the two-site Hamiltonian of the paper's
variational problem (Numerical procedure, Eq. 2) to the target symmetry sector,
solved by Lanczos/Davidson (the step right after Eq. 2).  In sector form

    H_eff = sum_t c_t (A_t (x) B_t) P_t ,   P_t = diag((-1)^{n_L}) on the input
                                              left index when the term carries
                                              the parity flag, identity otherwise,

restricted to V = span{|l>|r> : q(l) + q(r) = target}.  Block-wise, every term t
and every wave-function block q = (q_L, q_R) with q_L + Delta_t and q_R - Delta_t
present contributes

    y[q_L+Delta_t, q_R-Delta_t] += c_t s_t A_t[q_L+Delta_t <- q_L] x[q] B_t[q_R-Delta_t <- q_R]^T

with s_t = (-1)^{n(q_L)} for parity terms, else 1.
"""
from __future__ import annotations

import numpy as np

ORDER_A_FIRST = 0   # (A x) B^T
ORDER_B_FIRST = 1   # A (x B^T)


def _index(table):
    return {(int(n), int(s)): i for i, (n, s, _) in enumerate(table)}


def psi_blocks(problem):
    """Wave-function layout: blocks (q_L, q_R) with q_L + q_R = target, in
    ascending left-sector order, each stored row-major d(q_L) x d(q_R) and
    concatenated.  Returns a list of (iL, iR, offset, rows, cols)."""
    ridx = _index(problem.right)
    tn, ts = problem.target
    out, off = [], 0
    for iL, (n, s, d) in enumerate(problem.left):
        iR = ridx.get((tn - int(n), ts - int(s)))
        if iR is None:
            continue
        cols = int(problem.right[iR][2])
        out.append((iL, iR, off, int(d), cols))
        off += int(d) * cols
    return out


def _contributions(problem):
    """Every (term, input block, output block, a, b, c, d) that is present.
    a=d(q_L+Delta), b=d(q_L), c=d(q_R), d=d(q_R-Delta)."""
    lidx, ridx = _index(problem.left), _index(problem.right)
    blocks = psi_blocks(problem)
    by_left = {blk[0]: k for k, blk in enumerate(blocks)}
    items = []
    for t in range(problem.n_terms):
        dn, ds = int(problem.delta[t][0]), int(problem.delta[t][1])
        for k, (iL, iR, _, b, c) in enumerate(blocks):
            pL = lidx.get((int(problem.left[iL][0]) + dn, int(problem.left[iL][1]) + ds))
            pR = ridx.get((int(problem.right[iR][0]) - dn, int(problem.right[iR][1]) - ds))
            if pL is None or pR is None:
                continue
            if problem.a_off[t, iL] < 0 or problem.b_off[t, iR] < 0:
                continue
            kout = by_left[pL]
            items.append((t, k, kout, int(problem.left[pL][2]), b, c, int(problem.right[pR][2])))
    return items


def item_flops(a, b, c, d):
    """Flop counts of the two contraction orders of A(a x b) x(b x c) B^T(c x d):
    (A x) B^T costs 2abc + 2acd, A (x B^T) costs 2bcd + 2abd."""
    return 2 * a * b * c + 2 * a * c * d, 2 * b * c * d + 2 * a * b * d


def plan(problem) -> np.ndarray:
    """Contraction plan: one row (out_block, term, in_block, order, flops) per
    contributing (term, block) pair, order = the cheaper of the two (A-first
    on a tie), rows sorted by (out_block, term, in_block).  int64."""
    rows = []
    for t, k, kout, a, b, c, d in _contributions(problem):
        fa, fb = item_flops(a, b, c, d)
        order = ORDER_A_FIRST if fa <= fb else ORDER_B_FIRST
        rows.append((kout, t, k, order, min(fa, fb)))
    rows.sort()
    return np.array(rows, dtype=np.int64).reshape(-1, 5)


def plan_flops(problem) -> int:
    """Algorithmic flops of one H_eff*psi (one vector): the min-order sum."""
    p = plan(problem)
    return int(p[:, 4].sum()) if len(p) else 0


def _block(problem, off, rows, cols):
    return problem.op_data[off:off + rows * cols].reshape(rows, cols)


def apply(problem, x: np.ndarray) -> np.ndarray:
    """y = H_eff x for one vector (dim,) or several (nvec, dim), FP64, from the
    block-wise definition above.  Each term's product is formed as
    (A x_q) B^T with numpy matmul."""
    x = np.asarray(x, np.float64)
    single = x.ndim == 1
    X = x.reshape(1, -1) if single else x
    blocks = psi_blocks(problem)
    Y = np.zeros_like(X)
    for t, k, kout, a, b, c, d in _contributions(problem):
        iL, iR, off_in, _, _ = blocks[k]
        _, _, off_out, _, _ = blocks[kout]
        A = _block(problem, problem.a_off[t, iL], a, b)
        B = _block(problem, problem.b_off[t, iR], d, c)
        s = 1.0
        if problem.parity[t] and int(problem.left[iL][0]) % 2:
            s = -1.0
        coef = problem.coef[t] * s
        for v in range(X.shape[0]):
            xq = X[v, off_in:off_in + b * c].reshape(b, c)
            Y[v, off_out:off_out + a * d] += (coef * ((A @ xq) @ B.T)).ravel()
    return Y[0] if single else Y


def apply_entries(problem, x: np.ndarray, flat_idx) -> np.ndarray:
    """Selected entries y[flat_idx] of y = H_eff x (one vector), each formed
    from its own row of A and row of B, for spot checks at full size."""
    blocks = psi_blocks(problem)
    starts = np.array([b[2] for b in blocks])
    contrib = {}
    for t, k, kout, a, b, c, d in _contributions(problem):
        contrib.setdefault(kout, []).append((t, k, a, b, c, d))
    out = np.zeros(len(flat_idx))
    for n, g in enumerate(flat_idx):
        kout = int(np.searchsorted(starts, g, side="right") - 1)
        _, _, off_out, rows, cols = blocks[kout]
        i, j = divmod(int(g) - off_out, cols)
        acc = 0.0
        for t, k, a, b, c, d in contrib.get(kout, []):
            iL, iR, off_in, _, _ = blocks[k]
            A = _block(problem, problem.a_off[t, iL], a, b)
            B = _block(problem, problem.b_off[t, iR], d, c)
            xq = x[off_in:off_in + b * c].reshape(b, c)
            s = -1.0 if (problem.parity[t] and int(problem.left[iL][0]) % 2) else 1.0
            acc += problem.coef[t] * s * float(A[i, :] @ xq @ B[j, :])
        out[n] = acc
    return out


def diagonal(problem) -> np.ndarray:
    """Diagonal of H_eff in the wave-function layout.  Only Delta = 0 terms
    have diagonal entries: diag[(l, r)] = sum_t c_t s_t A_t[l, l] B_t[r, r]."""
    out = np.zeros(problem.dim)
    for iL, iR, off, rows, cols in psi_blocks(problem):
        for t in range(problem.n_terms):
            if problem.delta[t][0] != 0 or problem.delta[t][1] != 0:
                continue
            if problem.a_off[t, iL] < 0 or problem.b_off[t, iR] < 0:
                continue
            A = _block(problem, problem.a_off[t, iL], rows, rows)
            B = _block(problem, problem.b_off[t, iR], cols, cols)
            s = -1.0 if (problem.parity[t] and int(problem.left[iL][0]) % 2) else 1.0
            out[off:off + rows * cols] += problem.coef[t] * s * np.outer(np.diag(A), np.diag(B)).ravel()
    return out


def full_operator(problem, t: int, side: str) -> np.ndarray:
    """Dense D x D matrix of A_t (side 'A') or B_t (side 'B') assembled from its
    sector blocks, sectors in table order."""
    table = problem.left if side == "A" else problem.right
    offs = np.concatenate([[0], np.cumsum(table[:, 2])])
    idx = _index(table)
    D = int(offs[-1])
    M = np.zeros((D, D))
    dn, ds = int(problem.delta[t][0]), int(problem.delta[t][1])
    if side == "B":
        dn, ds = -dn, -ds
    off_tab = problem.a_off if side == "A" else problem.b_off
    for q, (n, s, dq) in enumerate(table):
        p = idx.get((int(n) + dn, int(s) + ds))
        if p is None or off_tab[t, q] < 0:
            continue
        dp = int(table[p][2])
        M[offs[p]:offs[p] + dp, offs[q]:offs[q] + int(dq)] = _block(problem, off_tab[t, q], dp, int(dq))
    return M


def target_indices(problem) -> np.ndarray:
    """Positions of the wave-function entries in the full left (x) right
    product space (index l * D_R + r), in wave-function order."""
    loffs = np.concatenate([[0], np.cumsum(problem.left[:, 2])])
    roffs = np.concatenate([[0], np.cumsum(problem.right[:, 2])])
    DR = int(roffs[-1])
    out = []
    for iL, iR, off, rows, cols in psi_blocks(problem):
        for i in range(rows):
            for j in range(cols):
                out.append((loffs[iL] + i) * DR + roffs[iR] + j)
    return np.array(out, dtype=np.int64)


def dense_h(problem) -> np.ndarray:
    """H_eff as a dense (dim x dim) matrix: sum_t c_t kron(A_t, B_t) P_t over
    the full product space, then restricted to the target entries.  Tiny
    problems only (D_L * D_R <= 4096)."""
    DL, DR = int(problem.left[:, 2].sum()), int(problem.right[:, 2].sum())
    if DL * DR > 4096:
        raise ValueError("dense_h is for tiny problems only")
    nL = np.repeat(problem.left[:, 0], problem.left[:, 2])
    par = np.kron(np.where(nL % 2 == 1, -1.0, 1.0), np.ones(DR))
    H = np.zeros((DL * DR, DL * DR))
    for t in range(problem.n_terms):
        K = np.kron(full_operator(problem, t, "A"), full_operator(problem, t, "B"))
        if problem.parity[t]:
            K = K * par[None, :]
        H += problem.coef[t] * K
    idx = target_indices(problem)
    return H[np.ix_(idx, idx)]
