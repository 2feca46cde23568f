"""Many-body operators of spinful fermion sites, built in the occupation basis
with Jordan-Wigner strings, for textbook-model pins.  Independent of the
oracle: it never forms a block-sparse product.

Modes of a block of L sites are ordered (1 up, 1 down, 2 up, 2 down, ...);
basis state s is an integer whose bit j is the occupation of mode j."""
import numpy as np


def annihilator(n_modes: int, j: int) -> np.ndarray:
    dim = 1 << n_modes
    M = np.zeros((dim, dim))
    for s in range(dim):
        if s >> j & 1:
            sign = -1.0 if bin(s & ((1 << j) - 1)).count("1") % 2 else 1.0
            M[s ^ (1 << j), s] = sign
    return M


def quantum_numbers(n_modes: int):
    """(n, 2S_z) of every basis state; even modes are spin up."""
    out = []
    for s in range(1 << n_modes):
        up = sum(s >> j & 1 for j in range(0, n_modes, 2))
        dn = sum(s >> j & 1 for j in range(1, n_modes, 2))
        out.append((up + dn, up - dn))
    return out


class Block:
    """A block of L sites: its sector table and block extraction of operators."""

    def __init__(self, L: int):
        self.L = L
        self.nm = 2 * L
        qn = quantum_numbers(self.nm)
        self.sectors = sorted(set(qn))
        self.members = {q: [s for s in range(1 << self.nm) if qn[s] == q] for q in self.sectors}
        self.table = np.array([(n, s, len(self.members[(n, s)])) for n, s in self.sectors], np.int32)
        self.idx = {q: i for i, q in enumerate(self.sectors)}

    def c(self, site: int, spin: int) -> np.ndarray:       # spin 0 = up, 1 = down
        return annihilator(self.nm, 2 * site + spin)

    def hubbard(self, t: float, U: float) -> np.ndarray:
        H = np.zeros((1 << self.nm, 1 << self.nm))
        for i in range(self.L - 1):
            for sp in (0, 1):
                a, b = self.c(i, sp), self.c(i + 1, sp)
                H -= t * (a.T @ b + b.T @ a)
        for i in range(self.L):
            H += U * (self.c(i, 0).T @ self.c(i, 0)) @ (self.c(i, 1).T @ self.c(i, 1))
        return H

    def blocks(self, M: np.ndarray, shift) -> dict:
        """Sector blocks M[q+shift <- q], keyed by the input sector index."""
        out = {}
        for q in self.sectors:
            p = (q[0] + shift[0], q[1] + shift[1])
            if p not in self.idx:
                continue
            blk = M[np.ix_(self.members[p], self.members[q])]
            out[self.idx[q]] = blk
        return out


def full_fock_hubbard_chain(L: int, t: float, U: float, n: int, two_sz: int) -> np.ndarray:
    """Eigenvalues of the open L-site Hubbard chain in the (n, 2S_z) sector by
    exact diagonalisation in its full Fock space (global Jordan-Wigner order)."""
    B = Block(L)
    H = B.hubbard(t, U)
    sel = B.members[(n, two_sz)]
    return np.linalg.eigvalsh(H[np.ix_(sel, sel)])
