"""Oracle: split-precision (Ozaki-style) products of FP64 matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper computes in FP64 (its FP64 bound lines, Performance assessment, Fig. 1).
An FP64 product can be reached on low-precision tensor cores by splitting each
operand into slices whose pairwise products are exact (Ozaki, Ogita, Oishi and Rump,
Numer. Algorithms 59 (2012): error-free splitting of matrix products).  The split
used here, written from that idea:

* a vector along the contraction index (a row of the left factor, a column of the
  right factor) gets the exponent E with |a| < 2^E for all its entries;
* each entry becomes S balanced base-256 digits of round(|a| 2^(7 + 8(S-1) - E)):
  a ~= 2^(E-7) sum_k d_k 2^(-8k), d_0 in [-128, 128], d_k in [-127, 128];
* the product keeps the digit pairs (i, j) with i + j <= S - 1:
  (L R)_rc ~= 2^(E_r + E_c - 14) sum_{i+j<=S-1} sum_K d_i(L_rK) d_j(R_Kc) 2^(-8(i+j)).

Sums are formed exactly (Python integers / Fractions), so this is the value the
split path reaches before any rounding of its own accumulators.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

S_DEFAULT = 6


def vector_exponent(vec) -> int | None:
    """E with |a| < 2^E for every entry (None for an all-zero vector)."""
    a = np.asarray(vec, np.float64)
    nz = a[a != 0]
    if nz.size == 0:
        return None
    return int(np.max(np.frexp(nz)[1]))


def digits(vec, S: int = S_DEFAULT):
    """(E, D): D[i, k] is digit k of entry i, most significant first."""
    a = np.asarray(vec, np.float64)
    E = vector_exponent(a)
    D = np.zeros((a.size, S), np.int64)
    if E is None:
        return 0, D
    shift = 7 + 8 * (S - 1) - E
    for i, v in enumerate(a):
        R = round(abs(Fraction(float(v))) * Fraction(2) ** shift)
        for k in range(S - 1, -1, -1):
            t = R & 255
            R >>= 8
            if t > 128:
                t -= 256
                R += 1
            D[i, k] = -t if v < 0 else t
        assert R == 0
    return E, D


def reconstruct(E: int, D: np.ndarray) -> list:
    """Exact value (Fractions) of each entry's digits."""
    S = D.shape[1]
    w = [Fraction(2) ** (E - 7 - 8 * k) for k in range(S)]
    return [sum(int(D[i, k]) * w[k] for k in range(S)) for i in range(D.shape[0])]


def split_product(L, R, S: int = S_DEFAULT, max_pair: int | None = None) -> np.ndarray:
    """Split product of L (M x K) and R (K x N) with the pairs i + j <= max_pair
    (default S - 1), summed exactly, rounded once to FP64."""
    L = np.atleast_2d(np.asarray(L, np.float64))
    R = np.atleast_2d(np.asarray(R, np.float64))
    max_pair = S - 1 if max_pair is None else max_pair
    rows = [digits(L[i], S) for i in range(L.shape[0])]
    cols = [digits(R[:, j], S) for j in range(R.shape[1])]
    out = np.zeros((L.shape[0], R.shape[1]))
    for i, (Ei, Di) in enumerate(rows):
        for j, (Ej, Dj) in enumerate(cols):
            acc = 0
            for p in range(S):
                for q in range(S):
                    if p + q <= max_pair:
                        acc += int(np.dot(Di[:, p], Dj[:, q])) << (8 * (max_pair - p - q))
            out[i, j] = float(Fraction(acc) * Fraction(2) ** (Ei + Ej - 14 - 8 * max_pair))
    return out


def exact_product(L, R) -> np.ndarray:
    """L R with exact rational sums, rounded once to FP64."""
    L = np.atleast_2d(np.asarray(L, np.float64))
    R = np.atleast_2d(np.asarray(R, np.float64))
    out = np.zeros((L.shape[0], R.shape[1]))
    for i in range(L.shape[0]):
        for j in range(R.shape[1]):
            out[i, j] = float(sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(L[i], R[:, j])))
    return out
