"""Oracle: two-site decomposition and truncation of the wave function.

TEST INFRASTRUCTURE ONLY (see the package docstring).

After the local eigenproblem, the two-site wave function is factorised (the paper's
matrix factorisation step, Numerical procedure) and truncated to the bond dimension.
In sector form psi is block diagonal, one block psi_b = psi[q_L, target - q_L] per left
sector, and the reading used here is:

  1. per block the singular value decomposition psi_b = U_b S_b V_b^T (S descending);
  2. the D largest singular values over all blocks are kept, singular values below
     1e-13 of the largest one being treated as zero and never kept; ties go to the
     earlier block, then to the earlier position;
  3. the new left basis of sector q_L is U_b[:, :k_b] (k_b kept values of block b);
  4. the discarded weight is the sum of the squares of the singular values not kept.
"""
from __future__ import annotations

import numpy as np

ZERO = 1e-13


def truncate(blocks, psi, D):
    """blocks: (offset, rows, cols) of the psi blocks.  Returns dict(sv=[per-block
    descending singular values], kept=[k_b], U=[d_L x k_b arrays], discarded)."""
    sv, us = [], []
    for off, rows, cols in blocks:
        M = psi[off:off + rows * cols].reshape(rows, cols)
        u, s, _ = np.linalg.svd(M, full_matrices=False)
        sv.append(s)
        us.append(u)
    smax = max((s[0] for s in sv if s.size), default=0.0)
    cand = [(-s[i], b, i) for b, s in enumerate(sv) for i in range(s.size) if s[i] > ZERO * smax]
    cand.sort()
    keep = cand[:D]
    kept = [0] * len(blocks)
    for _, b, _ in keep:
        kept[b] += 1
    total = sum(float((s ** 2).sum()) for s in sv)
    discarded = total - sum(s * s for s, _, _ in keep)
    return dict(sv=sv, kept=kept, U=[u[:, :k] for u, k in zip(us, kept)], discarded=discarded)
