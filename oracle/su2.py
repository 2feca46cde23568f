"""Oracle: the spin-adapted (SU(2)) two-site effective Hamiltonian.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's DMRG is spin-adapted (Introduction; Numerical procedure): bond states
are (n, S) multiplets, operators are irreducible tensor operators stored as
reduced blocks, and H_eff acts on the reduced two-site wave function of total spin
S.  The reading fixed here (all spins below as twice their value in the code):

* Wigner-Eckart, Clebsch-Gordan normalised: a rank-k tensor T with reduced block
  A[q' <- q] has the matrix elements
      <a' S' m'| T_mu |a S m> = <S m; k mu | S' m'> A[q' <- q][a', a];
* term t is c_t O_t P_t with the scalar coupling
      O_t = sum_mu (-1)^{k - mu} T_mu (left) U_{-mu} (right)      (a real scalar),
  P_t = (-1)^{n_L(input)} for parity terms, else 1;
* the reduced wave function holds, per pair of sectors (q_L, q_R) with
  n_L + n_R = n_target and (S_L, S_R, S) a triangle, the coefficients of the
  coupled states |(a S_L)(b S_R); S M>; blocks in (q_L, q_R) order, row-major
  d(q_L) x d(q_R), concatenated;
* then, for every term, A block [q_L' <- q_L], B block [q_R' <- q_R] and pair of
  wave-function blocks (q_L, q_R) -> (q_L', q_R'):
      y[q_L', q_R'] += c_t s_t W A x[q_L, q_R] B^T,
  W = <(S_L' S_R') S M | O (unit reduced blocks) | (S_L S_R) S M>, which does not
  depend on M (the operator is a scalar).

The oracle computes W from that definition, a sum of products of four
Clebsch-Gordan coefficients over the magnetic quantum numbers at M = S, and the
coefficients themselves from Racah's closed form in exact rational arithmetic.
The M-resolved helpers build the full operator of tiny problems, so that the
tests can check the reduced form against it.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

ORDER_A_FIRST = 0
ORDER_B_FIRST = 1


def triangle(a2: int, b2: int, c2: int) -> bool:
    return abs(a2 - b2) <= c2 <= a2 + b2 and (a2 + b2 + c2) % 2 == 0


@lru_cache(maxsize=None)
def cg(j1: int, m1: int, j2: int, m2: int, J: int, M: int) -> float:
    """<j1 m1; j2 m2 | J M> (Condon-Shortley phases), arguments twice the spins,
    by Racah's closed form: sqrt of a factorial ratio times an alternating sum."""
    if m1 + m2 != M or not triangle(j1, j2, J):
        return 0.0
    for j, m in ((j1, m1), (j2, m2), (J, M)):
        if abs(m) > j or (j + m) % 2:
            return 0.0
    f = math.factorial
    h = lambda x2: x2 // 2   # noqa: E731 (all combinations below are even)
    pre = Fraction((J + 1) * f(h(J + j1 - j2)) * f(h(J - j1 + j2)) * f(h(j1 + j2 - J)), f(h(j1 + j2 + J) + 1))
    pre *= f(h(J + M)) * f(h(J - M)) * f(h(j1 - m1)) * f(h(j1 + m1)) * f(h(j2 - m2)) * f(h(j2 + m2))
    s = Fraction(0)
    for k in range(0, h(j1 + j2 - J) + 1):
        args = (h(j1 + j2 - J) - k, h(j1 - m1) - k, h(j2 + m2) - k, h(J - j2 + m1) + k, h(J - j1 - m2) + k)
        if min(args) < 0:
            continue
        den = f(k)
        for a in args:
            den *= f(a)
        s += Fraction(-1 if k % 2 else 1, den)
    if s == 0:
        return 0.0
    return math.copysign(math.sqrt(pre * s * s), s)


@lru_cache(maxsize=None)
def recoupling(sl_out: int, sr_out: int, sl_in: int, sr_in: int, k2: int, s2: int) -> float:
    """W of the reading above, from its definition at M = S (twice the spins)."""
    if not (triangle(sl_in, sr_in, s2) and triangle(sl_out, sr_out, s2)
            and triangle(sl_in, k2, sl_out) and triangle(sr_in, k2, sr_out)):
        return 0.0
    M = s2
    w = 0.0
    for ml in range(-sl_in, sl_in + 1, 2):
        mr = M - ml
        if abs(mr) > sr_in:
            continue
        c_in = cg(sl_in, ml, sr_in, mr, s2, M)
        if c_in == 0.0:
            continue
        for mu in range(-k2, k2 + 1, 2):
            ml2, mr2 = ml + mu, mr - mu
            if abs(ml2) > sl_out or abs(mr2) > sr_out:
                continue
            sign = -1.0 if ((k2 - mu) // 2) % 2 else 1.0
            w += (cg(sl_out, ml2, sr_out, mr2, s2, M) * c_in * sign * cg(sl_in, ml, k2, mu, sl_out, ml2)
                  * cg(sr_in, mr, k2, -mu, sr_out, mr2))
    return w


def psi_blocks(problem):
    """Reduced wave-function layout: (iL, iR, offset, rows, cols) for every pair of
    sectors with n_L + n_R = n_target and (S_L, S_R, S) a triangle, in (iL, iR) order."""
    tn, ts = problem.target
    out, off = [], 0
    for iL, (nl, sl, dl) in enumerate(problem.left):
        for iR, (nr, sr, dr) in enumerate(problem.right):
            if int(nl) + int(nr) == tn and triangle(int(sl), int(sr), ts):
                out.append((iL, iR, off, int(dl), int(dr)))
                off += int(dl) * int(dr)
    return out


def _blocks_by_term(rows, T):
    out = [[] for _ in range(T)]
    for t, q, p, off in rows:
        out[int(t)].append((int(q), int(p), int(off)))
    return out


def _contributions(problem):
    """(term, in block, out block, W, A offset, B offset, a, b, c, d) for every
    present contribution; a = d(q_L'), b = d(q_L), c = d(q_R), d = d(q_R')."""
    blocks = psi_blocks(problem)
    bidx = {(b[0], b[1]): k for k, b in enumerate(blocks)}
    T = problem.n_terms
    A = _blocks_by_term(problem.a_blocks, T)
    B = _blocks_by_term(problem.b_blocks, T)
    L, R = problem.left, problem.right
    items = []
    for t in range(T):
        k2 = int(problem.rank2[t])
        for qa, pa, oa in A[t]:
            for qb, pb, ob in B[t]:
                kin, kout = bidx.get((qa, qb)), bidx.get((pa, pb))
                if kin is None or kout is None:
                    continue
                w = recoupling(int(L[pa][1]), int(R[pb][1]), int(L[qa][1]), int(R[qb][1]), k2, problem.target[1])
                items.append((t, kin, kout, w, oa, ob, int(L[pa][2]), int(L[qa][2]), int(R[qb][2]), int(R[pb][2])))
    return items


def plan(problem) -> np.ndarray:
    """One row (out_block, term, in_block, order, flops) per contribution, order the
    cheaper of (A x) B^T = 2abc + 2acd and A (x B^T) = 2bcd + 2abd (A-first on a
    tie), sorted.  int64."""
    rows = []
    for t, kin, kout, _, _, _, a, b, c, d in _contributions(problem):
        fa, fb = 2 * a * b * c + 2 * a * c * d, 2 * b * c * d + 2 * a * b * d
        rows.append((kout, t, kin, ORDER_A_FIRST if fa <= fb else ORDER_B_FIRST, min(fa, fb)))
    rows.sort()
    return np.array(rows, dtype=np.int64).reshape(-1, 5)


def _sign(problem, t, iL):
    return -1.0 if (problem.parity[t] and int(problem.left[iL][0]) % 2) else 1.0


def apply(problem, x: np.ndarray) -> np.ndarray:
    """y = H_eff x (one vector (dim,) or several (nvec, dim)) from the blockwise
    form above, FP64, numpy matmul per contribution."""
    x = np.asarray(x, np.float64)
    single = x.ndim == 1
    X = x.reshape(1, -1) if single else x
    blocks = psi_blocks(problem)
    Y = np.zeros_like(X)
    op = problem.op_data
    for t, kin, kout, w, oa, ob, a, b, c, d in _contributions(problem):
        iL, _, off_in, _, _ = blocks[kin]
        off_out = blocks[kout][2]
        Am = op[oa:oa + a * b].reshape(a, b)
        Bm = op[ob:ob + d * c].reshape(d, c)
        f = problem.coef[t] * _sign(problem, t, iL) * w
        for v in range(X.shape[0]):
            xq = X[v, off_in:off_in + b * c].reshape(b, c)
            Y[v, off_out:off_out + a * d] += (f * ((Am @ xq) @ Bm.T)).ravel()
    return Y[0] if single else Y


def apply_entries(problem, x: np.ndarray, flat_idx) -> np.ndarray:
    """Selected entries y[flat_idx] of y = H_eff x, each from its own rows of A and B."""
    blocks = psi_blocks(problem)
    starts = np.array([b[2] for b in blocks])
    by_out = {}
    for it in _contributions(problem):
        by_out.setdefault(it[2], []).append(it)
    op = problem.op_data
    out = np.zeros(len(flat_idx))
    for n, g in enumerate(flat_idx):
        kout = int(np.searchsorted(starts, g, side="right") - 1)
        _, _, off_out, rows, cols = blocks[kout]
        i, j = divmod(int(g) - off_out, cols)
        acc = 0.0
        for t, kin, _, w, oa, ob, a, b, c, d in by_out.get(kout, []):
            iL, _, off_in, _, _ = blocks[kin]
            xq = x[off_in:off_in + b * c].reshape(b, c)
            arow = op[oa + i * b:oa + (i + 1) * b]
            brow = op[ob + j * c:ob + (j + 1) * c]
            acc += problem.coef[t] * _sign(problem, t, iL) * w * float(arow @ xq @ brow)
        out[n] = acc
    return out


def diagonal(problem) -> np.ndarray:
    """Diagonal of the reduced H_eff: contributions whose output block is their input
    block, diag[(l, r)] += c_t s_t W A[l, l] B[r, r]."""
    blocks = psi_blocks(problem)
    out = np.zeros(problem.dim)
    op = problem.op_data
    for t, kin, kout, w, oa, ob, a, b, c, d in _contributions(problem):
        if kin != kout:
            continue
        iL, _, off, rows, cols = blocks[kin]
        Am = op[oa:oa + a * b].reshape(a, b)
        Bm = op[ob:ob + d * c].reshape(d, c)
        f = problem.coef[t] * _sign(problem, t, iL) * w
        out[off:off + rows * cols] += f * np.outer(np.diag(Am), np.diag(Bm)).ravel()
    return out


def truncate(problem, psi, D):
    """Two-site decomposition of the reduced wave function: per left sector the matrix of
    its blocks side by side (in block order), then the rule of oracle.svd.truncate over
    these matrices.  Returns its dict plus sectors (the left sector of each matrix).
    Reading: the squared singular values of that matrix are the eigenvalues of the left
    block's density matrix summed over the magnetic sublevels (the tests check this on the
    full space), so a kept singular vector is a kept multiplet."""
    from . import svd
    groups = []
    for iL, _, off, rows, cols in psi_blocks(problem):
        if groups and groups[-1][0] == iL:
            groups[-1][2].append((off, cols))
        else:
            groups.append((iL, rows, [(off, cols)]))
    flat, mats, pos = [], [], 0
    for _, rows, parts in groups:
        M = np.hstack([psi[o:o + rows * c].reshape(rows, c) for o, c in parts])
        flat.append(M.ravel())
        mats.append((pos, rows, M.shape[1]))
        pos += M.size
    r = svd.truncate(mats, np.concatenate(flat) if flat else np.zeros(0), D)
    r["sectors"] = [g[0] for g in groups]
    return r


# ---------------------------------------------------------------------------
# M-resolved (full) space of tiny problems


def m_basis(table):
    """States (sector, a, 2m) of one block with every magnetic sublevel, sector-major."""
    return [(q, a, m) for q, (_, s, d) in enumerate(table) for a in range(int(d))
            for m in range(-int(s), int(s) + 1, 2)]


def m_tensor(table, rows, op, t, k2, mu):
    """Dense matrix of component mu (twice) of the rank-k tensor of term t on one
    block, built from its reduced blocks by the Wigner-Eckart rule above: the
    sub-matrix of sectors (p <- q) is kron(A[p <- q], C) with
    C[m', m] = <S_q m; k mu | S_p m'>."""
    offs = np.concatenate([[0], np.cumsum([int(d) * (int(s) + 1) for _, s, d in table])])
    M = np.zeros((offs[-1], offs[-1]))
    for tt, q, p, off in rows:
        if int(tt) != t:
            continue
        q, p, off = int(q), int(p), int(off)
        sq, sp, dq, dp = int(table[q][1]), int(table[p][1]), int(table[q][2]), int(table[p][2])
        C = np.array([[cg(sq, m, k2, mu, sp, m2) for m in range(-sq, sq + 1, 2)] for m2 in range(-sp, sp + 1, 2)])
        M[offs[p]:offs[p + 1], offs[q]:offs[q + 1]] = np.kron(op[off:off + dp * dq].reshape(dp, dq), C)
    return M


def m_spin(table):
    """Dense S_z and S_+ of one block (each multiplet a spin-S irrep)."""
    basis = m_basis(table)
    idx = {st: i for i, st in enumerate(basis)}
    Sz = np.diag([m / 2.0 for _, _, m in basis])
    Sp = np.zeros((len(basis), len(basis)))
    for i, (q, a, m) in enumerate(basis):
        s = int(table[q][1])
        if m + 2 <= s:
            j, mm = s / 2.0, m / 2.0
            Sp[idx[(q, a, m + 2)], i] = math.sqrt(j * (j + 1) - mm * (mm + 1))
    return Sz, Sp


def full_space(problem):
    """The full operator on the n_target subspace of left (x) right with every
    magnetic sublevel: returns dict(H, Sz, Sp, E, index) with H the dense operator,
    Sz and Sp the total spin operators there and E the isometry from the reduced
    wave function to the coupled states with M = S."""
    L, R, op = problem.left, problem.right, problem.op_data
    bl, br = m_basis(L), m_basis(R)
    nL = np.array([int(L[q][0]) for q, _, _ in bl])
    nR = np.array([int(R[q][0]) for q, _, _ in br])
    keep = [i * len(br) + j for i in range(len(bl)) for j in range(len(br)) if nL[i] + nR[j] == problem.target[0]]
    keep = np.array(keep, dtype=np.int64)
    H = np.zeros((len(keep), len(keep)))
    par = np.kron(np.where(nL % 2 == 1, -1.0, 1.0), np.ones(len(br)))[keep]
    ki, kj = keep // len(br), keep % len(br)
    for t in range(problem.n_terms):
        k2 = int(problem.rank2[t])
        K = np.zeros((len(keep), len(keep)))
        for mu in range(-k2, k2 + 1, 2):   # (T (x) U)[keep, keep] = T[ki, ki] * U[kj, kj]
            sign = -1.0 if ((k2 - mu) // 2) % 2 else 1.0
            Tm = m_tensor(L, problem.a_blocks, op, t, k2, mu)
            Um = m_tensor(R, problem.b_blocks, op, t, k2, -mu)
            K += sign * Tm[np.ix_(ki, ki)] * Um[np.ix_(kj, kj)]
        if problem.parity[t]:
            K = K * par[None, :]
        H += problem.coef[t] * K
    SzL, SpL = m_spin(L)
    SzR, SpR = m_spin(R)
    IL, IR = np.eye(len(bl)), np.eye(len(br))
    Sz = (np.kron(SzL, IR) + np.kron(IL, SzR))[np.ix_(keep, keep)]
    Sp = (np.kron(SpL, IR) + np.kron(IL, SpR))[np.ix_(keep, keep)]
    pos = {int(g): i for i, g in enumerate(keep)}
    il = {st: i for i, st in enumerate(bl)}
    ir = {st: i for i, st in enumerate(br)}
    s2 = problem.target[1]
    E = np.zeros((len(keep), problem.dim))
    for iL, iR, off, rows, cols in psi_blocks(problem):
        sl, sr = int(L[iL][1]), int(R[iR][1])
        for a in range(rows):
            for b in range(cols):
                col = off + a * cols + b
                for ml in range(-sl, sl + 1, 2):
                    mr = s2 - ml
                    if abs(mr) > sr:
                        continue
                    c = cg(sl, ml, sr, mr, s2, s2)
                    if c != 0.0:
                        E[pos[il[(iL, a, ml)] * len(br) + ir[(iR, b, mr)]], col] += c
    return dict(H=H, Sz=Sz, Sp=Sp, E=E, index=keep)
