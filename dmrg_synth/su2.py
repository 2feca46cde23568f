"""Seeded synthetic spin-adapted (SU(2)) two-site problems (inputs only).

The paper works with spin-adapted DMRG (Introduction and Numerical procedure: the
SU(2) symmetry of the electronic Hamiltonian is used throughout).  There the bond
states are (n, S) multiplets and every operator is an irreducible tensor operator of
rank k, stored as reduced blocks only.  This module builds such inputs; like the
U(1) generator it holds no part of the method's arithmetic (no coupling
coefficients, no H_eff*psi, no planning).

Problem content:

* sector tables (n, 2S, dim) of the left and right enlarged blocks, dim = number
  of multiplets, ascending in (n, 2S), 2S >= 0;
* terms t = (c_t, 2k_t, dn_t, parity_t): the product of a rank-k tensor T_t on the
  left block (shifting n by +dn) and a rank-k tensor U_t on the right block
  (shifting n by -dn), coupled to a scalar;
* reduced blocks A_t[q' <- q] (left) and B_t[r' <- r] (right), row-major
  d(out) x d(in) in one flat FP64 array, listed as rows (term, in, out, offset).

Readings where the paper is silent:

* sector lattice (n, 2S) with 2S = n mod 2 and 0 <= 2S <= s_max;
* weights w = exp(-(n - n_target/2)^2 / sigma_n^2 - S^2 / sigma_s^2) and the U(1)
  keep-and-round rule (expected count D*w/sum(w) >= 1, at least one multiplet per
  kept sector, largest remainder, ties to the earlier sector);
* the right block has the left block's table;
* term kinds (dn, 2k) drawn uniformly from KINDS (the one-, two- and three-operator
  complementary operators of a quantum-chemistry Hamiltonian: creation-like
  (1, 1/2) and (1, 3/2), pair (2, 0) and (2, 1), and the dn = 0 ranks 0 and 1);
  dn = 0 gives one self-adjoint term, any other kind a pair (t, t') with
  dn' = -dn, the same rank and c' = c (dn even) or -c (dn odd, because of the
  parity sign (-1)^{n_L(input)});
* a block [out <- in] exists for every pair of sectors with the shifted n and
  (S_in, k, S_out) a triangle; entries N(0,1)/sqrt(d_in), c_t ~ N(0,1)/sqrt(T);
* adjoint blocks: A'[q <- q'] = phi_L A[q' <- q]^T and B'[r <- r'] = phi_R B[r' <- r]^T
  with phi = (-1)^e sqrt((2 S_out + 1) / (2 S_in + 1)) (in and out of the forward
  block), e_L = (2S_in - 2S_out + 2k)/2 and e_R = (2S_out - 2S_in - 2k)/2 for
  half-integer k, e_L = (2S_in - 2S_out)/2 and e_R = (2S_out - 2S_in)/2 for integer k.
  This is the adjoint relation of reduced matrix elements normalised by a
  Clebsch-Gordan coefficient (Wigner-Eckart), and it makes H symmetric; the
  oracle tests check that symmetry on the dense operator;
* random numbers: numpy's Philox keyed by (seed, stream), one stream per term.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np

from . import STREAM_PSI, STREAM_TERMS, _largest_remainder, philox

#: (dn, 2k) of the term kinds.
KINDS = ((0, 0), (0, 2), (1, 1), (-1, 1), (1, 3), (-1, 3), (2, 0), (-2, 0), (2, 2), (-2, 2))

#: Named spin-adapted workloads.
CONFIGS = {
    # 40 multiplets per block, n in [0,6], 2S in [0,4], target (6, 2S=2), 30 terms.
    "su2_tiny": dict(D=40, n_range=(0, 6), s_max=4, target=(6, 2), sigma_n=2.0, sigma_s=1.0,
                     T=30, keep_all=True),
    # 1024 multiplets per block, n in [0,20], 2S in [0,8], singlet target (20, 0), 600 terms.
    "su2_mid": dict(D=1024, n_range=(0, 20), s_max=8, target=(20, 0), sigma_n=3.0, sigma_s=1.5,
                    T=600, keep_all=False),
}


def triangle(a2: int, b2: int, c2: int) -> bool:
    """(a, b, c) (given as twice the spins) can couple: |a-b| <= c <= a+b, a+b+c integer."""
    return abs(a2 - b2) <= c2 <= a2 + b2 and (a2 + b2 + c2) % 2 == 0


@dataclasses.dataclass
class SU2Problem:
    """One spin-adapted two-site effective-Hamiltonian instance.

    left, right : int32 (nsec, 3) of (n, two_s, dim), ascending in (n, two_s).
    target      : (n, two_s) of the two-site wave function.
    coef, rank2, dn, parity : per term (float64, int32 x 3).
    a_blocks, b_blocks : int64 (n_blocks, 4) rows (term, in_sector, out_sector,
                  offset of the row-major d(out) x d(in) block in op_data), ascending.
    op_data     : float64 flat storage of all reduced blocks.
    dim         : number of entries of the reduced two-site wave function.
    """
    left: np.ndarray
    right: np.ndarray
    target: tuple
    coef: np.ndarray
    rank2: np.ndarray
    dn: np.ndarray
    parity: np.ndarray
    a_blocks: np.ndarray
    b_blocks: np.ndarray
    op_data: np.ndarray
    dim: int
    seed: int = 0
    name: str = "custom"

    @property
    def n_terms(self) -> int:
        return int(self.coef.shape[0])

    def random_vectors(self, k: int, stream0: int = STREAM_PSI) -> np.ndarray:
        """k seeded N(0,1) vectors of length dim, unit 2-norm, shape (k, dim)."""
        out = np.empty((k, self.dim))
        for i in range(k):
            v = philox(self.seed, stream0 + i).standard_normal(self.dim)
            out[i] = v / np.linalg.norm(v)
        return out

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.left, self.right, np.asarray(self.target, np.int32), self.coef, self.rank2, self.dn,
                  self.parity, self.a_blocks, self.b_blocks, self.op_data):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


def sector_table(cfg: dict) -> np.ndarray:
    secs = [(n, s) for n in range(cfg["n_range"][0], cfg["n_range"][1] + 1)
            for s in range(0, cfg["s_max"] + 1) if (s - n) % 2 == 0]
    nbar = cfg["target"][0] / 2.0
    w = np.array([np.exp(-(n - nbar) ** 2 / cfg["sigma_n"] ** 2 - (s / 2.0) ** 2 / cfg["sigma_s"] ** 2)
                  for n, s in secs])
    D = cfg["D"]
    keep = np.ones(len(secs), bool) if cfg["keep_all"] else (D * w / w.sum() >= 1.0)
    kept = [secs[i] for i in range(len(secs)) if keep[i]]
    wk = w[keep]
    dims = _largest_remainder(D * wk / wk.sum(), D)
    return np.array([(n, s, d) for (n, s), d in zip(kept, dims)], dtype=np.int32)


def wavefunction_dim(left, right, target) -> int:
    """Entries of the reduced two-site wave function: pairs of sectors with
    n_L + n_R = n_target whose spins couple to S_target (a count only)."""
    tot = 0
    for nl, sl, dl in left:
        for nr, sr, dr in right:
            if int(nl) + int(nr) == target[0] and triangle(int(sl), int(sr), target[1]):
                tot += int(dl) * int(dr)
    return tot


def block_pairs(table, dn: int, k2: int):
    """(in, out) sector pairs of a rank-k tensor shifting n by dn, in ascending
    (in, out) order."""
    out = []
    for q, (n, s, _) in enumerate(table):
        for p, (n2, s2, _) in enumerate(table):
            if int(n2) == int(n) + dn and triangle(int(s), k2, int(s2)):
                out.append((q, p))
    return out


def _phase_weight(s_in: int, s_out: int, k2: int, side: str) -> float:
    if k2 % 2:
        e = (s_in - s_out + k2) // 2 if side == "L" else (s_out - s_in - k2) // 2
    else:
        e = (s_in - s_out) // 2 if side == "L" else (s_out - s_in) // 2
    return (-1.0 if e % 2 else 1.0) * np.sqrt((s_out + 1.0) / (s_in + 1.0))


def pack(left, right, target, terms, seed=0, name="custom") -> SU2Problem:
    """Pack explicit terms into an SU2Problem.

    terms: list of (c, two_k, dn, parity, a_blocks, b_blocks), with a_blocks a dict
    {(in, out): dense d(out) x d(in) array} over left sector indices and b_blocks
    the same over right sector indices."""
    left = np.asarray(left, np.int32).reshape(-1, 3)
    right = np.asarray(right, np.int32).reshape(-1, 3)
    rows = {"A": [], "B": []}
    chunks, pos = [], 0
    for t, (c, k2, dn, par, ab, bb) in enumerate(terms):
        for side, blocks, tab, sh in (("A", ab, left, dn), ("B", bb, right, -dn)):
            for (q, p), blk in sorted(blocks.items()):
                if (int(tab[p][0]) != int(tab[q][0]) + sh or not triangle(int(tab[q][1]), k2, int(tab[p][1]))
                        or blk.shape != (tab[p][2], tab[q][2])):
                    raise ValueError("block shape or sector mismatch")
                rows[side].append((t, q, p, pos))
                chunks.append(np.ascontiguousarray(blk, np.float64).ravel())
                pos += blk.size
    op = np.concatenate(chunks) if chunks else np.zeros(0)
    T = len(terms)
    return SU2Problem(left=left, right=right, target=(int(target[0]), int(target[1])),
                      coef=np.array([t[0] for t in terms], np.float64),
                      rank2=np.array([t[1] for t in terms], np.int32).reshape(T),
                      dn=np.array([t[2] for t in terms], np.int32).reshape(T),
                      parity=np.array([t[3] for t in terms], np.int32).reshape(T),
                      a_blocks=np.array(rows["A"], np.int64).reshape(-1, 4),
                      b_blocks=np.array(rows["B"], np.int64).reshape(-1, 4),
                      op_data=op, dim=wavefunction_dim(left, right, target), seed=seed, name=name)


def generate(name: str, seed: int = 0, n_terms: int | None = None, target=None) -> SU2Problem:
    """Build the named spin-adapted workload (optionally fewer terms, or another
    target on the same sector tables).  Per term its A blocks then its B blocks, each
    in ascending (in, out); a forward term draws its blocks from its own Philox stream
    in that order, an adjoint partner takes the weighted transposes of its forward
    term's blocks."""
    cfg = dict(CONFIGS[name])
    if n_terms is not None:
        cfg["T"] = int(n_terms)
    table = sector_table(cfg)
    if target is not None:
        cfg["target"] = (int(target[0]), int(target[1]))
    dims = [int(x) for x in table[:, 2]]
    T = cfg["T"]
    g = philox(seed, STREAM_TERMS)
    kinds = []
    while len(kinds) < T:
        kd = (0, 0) if T - len(kinds) == 1 else KINDS[int(g.integers(len(KINDS)))]
        c = float(g.standard_normal()) / np.sqrt(T)
        if kd[0] == 0:
            kinds.append(("self", kd, c))
        else:
            kinds.append(("fwd", kd, c))
            kinds.append(("adj", (-kd[0], kd[1]), c if kd[0] % 2 == 0 else -c))
    rows = {"A": [], "B": []}
    where = {}
    pos = 0
    for t, (_, (dn, k2), _) in enumerate(kinds):
        for side, sh in (("A", dn), ("B", -dn)):
            for q, p in block_pairs(table, sh, k2):
                rows[side].append((t, q, p, pos))
                where[(t, side, q, p)] = pos
                pos += dims[p] * dims[q]
    op = np.empty(pos, np.float64)

    def blk(t, side, q, p):
        o = where[(t, side, q, p)]
        return op[o:o + dims[p] * dims[q]].reshape(dims[p], dims[q])

    for t, (kind, (dn, k2), _) in enumerate(kinds):
        if kind == "adj":   # [q <- p] = phi * (forward [p <- q])^T, phi of the forward block
            for side, sh in (("A", -dn), ("B", dn)):
                for p, q in block_pairs(table, sh, k2):   # forward block [q <- p]
                    phi = _phase_weight(int(table[p][1]), int(table[q][1]), k2, "L" if side == "A" else "R")
                    blk(t, side, q, p)[...] = phi * blk(t - 1, side, p, q).T
            continue
        gt = philox(seed, 1 + t)
        for side, sh in (("A", dn), ("B", -dn)):
            pairs = block_pairs(table, sh, k2)
            for q, p in pairs:
                m = gt.standard_normal((dims[p], dims[q])) / np.sqrt(float(dims[q]))
                if kind == "self":
                    if p < q:      # filled from its partner block [q <- p]
                        continue
                    if p == q:
                        m = 0.5 * (m + m.T)
                blk(t, side, q, p)[...] = m
            if kind == "self":
                for q, p in pairs:
                    if p < q:
                        phi = _phase_weight(int(table[p][1]), int(table[q][1]), k2, "L" if side == "A" else "R")
                        blk(t, side, q, p)[...] = phi * blk(t, side, p, q).T
    T = len(kinds)
    return SU2Problem(left=table.copy(), right=table.copy(), target=(int(cfg["target"][0]), int(cfg["target"][1])),
                      coef=np.array([k[2] for k in kinds], np.float64),
                      rank2=np.array([k[1][1] for k in kinds], np.int32),
                      dn=np.array([k[1][0] for k in kinds], np.int32),
                      parity=np.array([1 if k[1][0] % 2 else 0 for k in kinds], np.int32),
                      a_blocks=np.array(rows["A"], np.int64).reshape(-1, 4),
                      b_blocks=np.array(rows["B"], np.int64).reshape(-1, 4),
                      op_data=op, dim=wavefunction_dim(table, table, cfg["target"]), seed=seed, name=name)
