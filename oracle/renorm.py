"""Oracle: operator renormalisation in a truncated basis.

TEST INFRASTRUCTURE ONLY (see the package docstring).

After each local update the block operators are carried into the new, truncated
basis (the paper's renormalisation step, Numerical procedure).  Sector by sector, with
the basis U_q (d_q x d'_q) of sector q, a block O[p <- q] becomes

    O'[p <- q] = U_p^T O[p <- q] U_q          (d'_p x d'_q).

The definition is written out directly, one block at a time.
"""
from __future__ import annotations

import numpy as np


def basis_offsets(dims, dims_new):
    """Offsets of the row-major bases U_q in their concatenation, sector order."""
    sizes = np.asarray(dims, np.int64) * np.asarray(dims_new, np.int64)
    return np.concatenate([[0], np.cumsum(sizes)])


def renormalise(dims, dims_new, U, blocks, op):
    """List of the blocks U_p^T O[p <- q] U_q for blocks rows (q, p, offset)."""
    uo = basis_offsets(dims, dims_new)
    out = []
    for q, p, off in np.asarray(blocks, np.int64).reshape(-1, 3):
        dq, dp = int(dims[q]), int(dims[p])
        Uq = U[uo[q]:uo[q + 1]].reshape(dq, int(dims_new[q]))
        Up = U[uo[p]:uo[p + 1]].reshape(dp, int(dims_new[p]))
        O = op[off:off + dp * dq].reshape(dp, dq)
        out.append(Up.T @ O @ Uq)
    return out
