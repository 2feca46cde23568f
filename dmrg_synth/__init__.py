"""Seeded synthetic two-site DMRG problems (inputs only).

This module builds the *inputs* of the effective-Hamiltonian product: the
(n, 2S_z) sector tables of the left and right enlarged blocks, a list of terms
(coefficient c_t, quantum-number shift Delta_t, fermion-parity flag) with their
dense FP64 operator blocks A_t and B_t, and random start vectors.  It holds no
part of the method's arithmetic: no H_eff*psi, no planning, no ordering of
contractions.  Both the CPU oracle and the GPU library consume exactly the
bytes produced here, so the two sides always see identical inputs.

The workload shapes follow the two-site problem of the paper (Numerical
procedure, Eq. 2 and the Davidson/Lanczos step after it): a block-sparse
Hermitian operator over symmetry sectors whose dimensions have the Gaussian
profile in (n, S_z) that a quantum-chemistry U(1) bond shows.  Where the paper
is silent the readings are:

* sectors (n, 2S_z) on the lattice 2S_z = n (mod 2) with n and 2S_z in the
  given ranges (|2S_z| <= n is not imposed);
* weights w = exp(-(n - n_target/2)^2 / sigma_n^2 - S_z^2 / sigma_s^2),
  S_z = 2S_z / 2;
* sectors whose expected count D*w/sum(w) is >= 1 are kept (or all of them),
  each kept sector gets max(1, floor(D*w/sum_kept(w))) states and the rest is
  handed out by largest fractional part, ties to the earlier sector;
* the right block has the same table as the left block;
* terms: Delta drawn uniformly from {(0,0), (+-1,+-1), (+-2,0), (0,+-2)};
  Delta = 0 gives one self-adjoint term (A and B blocks symmetrised), any other
  Delta gives a pair (t, t') with Delta' = -Delta, A' = A^T, B' = B^T and
  c' = c for even Delta_n, c' = -c for odd Delta_n, which keeps
  H = sum_t c_t (A_t (x) B_t) P_t symmetric when P_t = (-1)^{n_L(input)};
* block entries N(0,1)/sqrt(d_in), c_t ~ N(0,1)/sqrt(T);
* random numbers come from numpy's Philox counter-based generator keyed by
  (seed, stream), one stream per term so that any term can be rebuilt alone.

The spin-adapted ((n, S) multiplet) inputs are built by ``dmrg_synth.su2``.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np

#: The nine quantum-number shifts (dn, d2sz) a term can carry.
DELTAS = ((0, 0), (1, 1), (1, -1), (-1, 1), (-1, -1), (2, 0), (-2, 0), (0, 2), (0, -2))

#: Named workloads: two-site problems shaped like quantum-chemistry DMRG.
CONFIGS = {
    # D=64 per block, n in [0,8], 2sz in [-2,2], target (8,0), 40 terms.
    "tiny": dict(D=64, n_range=(0, 8), s_range=(-2, 2), target=(8, 0), sigma_n=2.0,
                 sigma_s=1.0, T=40, keep_all=True, dims="gauss"),
    # D=1024, n in [0,20], 2sz in [-4,4], target (20,0), 600 terms.
    "mid": dict(D=1024, n_range=(0, 20), s_range=(-4, 4), target=(20, 0), sigma_n=3.0,
                sigma_s=1.5, T=600, keep_all=False, dims="gauss"),
    # D=4096, n in [0,38], 2sz in [-6,6], target (38,0), 2000 terms.
    "precision": dict(D=4096, n_range=(0, 38), s_range=(-6, 6), target=(38, 0), sigma_n=3.0,
                      sigma_s=1.5, T=2000, keep_all=False, dims="gauss"),
    # D=4096 on the sectors of "precision", log-normal(0, 1.2) dims clipped to [1, 900],
    # 3000 terms.
    "heavy": dict(D=4096, n_range=(0, 38), s_range=(-6, 6), target=(38, 0), sigma_n=3.0,
                  sigma_s=1.5, T=3000, keep_all=False, dims="lognormal", ln_sigma=1.2,
                  d_max=900),
    # D=8192, n in [0,56], 2sz in [-8,8], target (56,0), 3500 terms.
    "large": dict(D=8192, n_range=(0, 56), s_range=(-8, 8), target=(56, 0), sigma_n=3.0,
                  sigma_s=1.5, T=3500, keep_all=False, dims="gauss"),
}

STREAM_TERMS = 0            # Delta and coefficient draws
STREAM_PSI = 1 << 40        # start vectors (stream + k for vector k)
STREAM_DIMS = (1 << 40) - 1  # log-normal sector dimensions


def philox(seed: int, stream: int) -> np.random.Generator:
    """Counter-based generator for one (seed, stream) pair."""
    if seed < 0 or stream < 0:
        raise ValueError("seed and stream must be non-negative")
    return np.random.Generator(np.random.Philox(key=(int(stream) << 64) | int(seed)))


@dataclasses.dataclass
class Problem:
    """One two-site effective-Hamiltonian instance.

    left, right : int32 arrays (nsec, 3) of (n, two_sz, dim), sorted by (n, two_sz).
    target      : (n, two_sz) of the two-site wave function.
    coef        : float64 (T,) term coefficients c_t.
    delta       : int32 (T, 2) shifts (dn, d2sz) applied to the left block; the
                  right block is shifted by -delta.
    parity      : int32 (T,) 1 if the term carries the sign (-1)^{n_L(input)}.
    a_off       : int64 (T, nl) offset in op_data of A_t[q+delta <- q] for left
                  input sector q (row-major d(q+delta) x d(q)), -1 if absent.
    b_off       : int64 (T, nr) offset in op_data of B_t[q-delta <- q] for right
                  input sector q (row-major d(q-delta) x d(q)), -1 if absent.
    op_data     : float64 flat storage of all operator blocks.
    dim         : number of entries of the two-site wave function.
    """
    left: np.ndarray
    right: np.ndarray
    target: tuple
    coef: np.ndarray
    delta: np.ndarray
    parity: np.ndarray
    a_off: np.ndarray
    b_off: np.ndarray
    op_data: np.ndarray
    dim: int
    seed: int = 0
    name: str = "custom"

    @property
    def n_terms(self) -> int:
        return int(self.coef.shape[0])

    def random_vectors(self, k: int, stream0: int = STREAM_PSI) -> np.ndarray:
        """k seeded N(0,1) vectors of length dim, each scaled to unit 2-norm,
        shape (k, dim).  Vector 0 is the start vector psi0."""
        out = np.empty((k, self.dim))
        for i in range(k):
            v = philox(self.seed, stream0 + i).standard_normal(self.dim)
            out[i] = v / np.linalg.norm(v)
        return out

    def digest(self) -> str:
        """sha256 over every input byte (tables, terms, offsets, operator data)."""
        h = hashlib.sha256()
        for a in (self.left, self.right, np.asarray(self.target, np.int32), self.coef,
                  self.delta, self.parity, self.a_off, self.b_off, self.op_data):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()

    def structure_digest(self) -> str:
        """sha256 over the integer structure only (no floating-point values)."""
        h = hashlib.sha256()
        for a in (self.left, self.right, np.asarray(self.target, np.int32), self.delta,
                  self.parity, self.a_off, self.b_off):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


def sector_lattice(n_range, s_range):
    """All (n, two_sz) with two_sz = n mod 2, sorted by (n, two_sz)."""
    return [(n, s) for n in range(n_range[0], n_range[1] + 1)
            for s in range(s_range[0], s_range[1] + 1) if (s - n) % 2 == 0]


def _largest_remainder(x: np.ndarray, total: int) -> np.ndarray:
    base = np.maximum(1, np.floor(x)).astype(np.int64)
    rest = total - int(base.sum())
    if rest < 0:
        raise ValueError("sector minimum of one state exceeds the bond dimension")
    frac = x - np.floor(x)
    order = sorted(range(len(x)), key=lambda i: (-frac[i], i))
    for i in order[:rest]:
        base[i] += 1
    return base


def sector_table(cfg: dict, seed: int = 0) -> np.ndarray:
    """(nsec, 3) int32 table of (n, two_sz, dim) for one enlarged block."""
    secs = sector_lattice(cfg["n_range"], cfg["s_range"])
    nbar = cfg["target"][0] / 2.0
    w = np.array([np.exp(-(n - nbar) ** 2 / cfg["sigma_n"] ** 2
                         - (s / 2.0) ** 2 / cfg["sigma_s"] ** 2) for n, s in secs])
    D = cfg["D"]
    keep = np.ones(len(secs), bool) if cfg["keep_all"] else (D * w / w.sum() >= 1.0)
    kept = [secs[i] for i in range(len(secs)) if keep[i]]
    if cfg.get("dims", "gauss") == "gauss":
        wk = w[keep]
        dims = _largest_remainder(D * wk / wk.sum(), D)
    else:
        g = philox(seed, STREAM_DIMS)
        raw = g.lognormal(0.0, cfg["ln_sigma"], size=len(kept))
        x = raw * D / raw.sum()
        for _ in range(100):           # clip to [1, d_max] and rescale until stable
            x = np.clip(x, 1.0, cfg["d_max"])
            x = x * D / x.sum()
            if x.max() <= cfg["d_max"] and x.min() >= 1.0:
                break
        x = np.clip(x, 1.0, cfg["d_max"])
        dims = _largest_remainder(x * D / x.sum(), D)
        while dims.max() > cfg["d_max"]:   # hand clipped states to the smallest sectors
            i = int(np.argmax(dims)); dims[i] -= 1; dims[int(np.argmin(dims))] += 1
    return np.array([(n, s, d) for (n, s), d in zip(kept, dims)], dtype=np.int32)


def _index(table):
    return {(int(n), int(s)): i for i, (n, s, _) in enumerate(table)}


def wavefunction_dim(left, right, target) -> int:
    """Number of two-site entries with q_L + q_R = target (a count only)."""
    ridx = _index(right)
    tot = 0
    for n, s, d in left:
        j = ridx.get((target[0] - int(n), target[1] - int(s)))
        if j is not None:
            tot += int(d) * int(right[j][2])
    return tot


def assemble(left, right, target, terms, seed=0, name="custom") -> Problem:
    """Pack explicit terms into a Problem.

    terms: list of (c, (dn, d2sz), parity, a_blocks, b_blocks) where a_blocks maps
    a left input sector index q to the dense block A[q+delta <- q] and b_blocks
    maps a right input sector index q to B[q-delta <- q].  Missing keys are
    absent blocks."""
    left = np.asarray(left, np.int32).reshape(-1, 3)
    right = np.asarray(right, np.int32).reshape(-1, 3)
    T = len(terms)
    a_off = -np.ones((T, len(left)), np.int64)
    b_off = -np.ones((T, len(right)), np.int64)
    chunks, pos = [], 0
    lidx, ridx = _index(left), _index(right)
    for t, (c, dl, par, ab, bb) in enumerate(terms):
        for q, blk in sorted(ab.items()):
            p = lidx.get((int(left[q][0]) + dl[0], int(left[q][1]) + dl[1]))
            if p is None or blk.shape != (left[p][2], left[q][2]):
                raise ValueError("A block shape or sector mismatch")
            a_off[t, q] = pos; chunks.append(np.ascontiguousarray(blk, np.float64).ravel())
            pos += blk.size
        for q, blk in sorted(bb.items()):
            p = ridx.get((int(right[q][0]) - dl[0], int(right[q][1]) - dl[1]))
            if p is None or blk.shape != (right[p][2], right[q][2]):
                raise ValueError("B block shape or sector mismatch")
            b_off[t, q] = pos; chunks.append(np.ascontiguousarray(blk, np.float64).ravel())
            pos += blk.size
    op = np.concatenate(chunks) if chunks else np.zeros(0)
    return Problem(left=left, right=right, target=(int(target[0]), int(target[1])),
                   coef=np.array([t[0] for t in terms], np.float64),
                   delta=np.array([t[1] for t in terms], np.int32).reshape(T, 2),
                   parity=np.array([t[2] for t in terms], np.int32),
                   a_off=a_off, b_off=b_off, op_data=op,
                   dim=wavefunction_dim(left, right, target), seed=seed, name=name)


def _shift_pairs(table, shift):
    """(q, p) for every sector q whose shifted sector p = q + shift exists, q ascending."""
    idx = _index(table)
    out = []
    for q, (n, s, _) in enumerate(table):
        p = idx.get((int(n) + shift[0], int(s) + shift[1]))
        if p is not None:
            out.append((q, p))
    return out


def generate(name: str, seed: int = 0, n_terms: int | None = None) -> Problem:
    """Build the named workload with the given seed (optionally fewer terms).

    The operator data is laid out first (per term its A blocks, then its B blocks, each
    in ascending input sector) and every block is drawn straight into that one array,
    so the peak host memory is the operator data itself.  Term t's blocks come from
    its own Philox stream in layout order (A then B); an adjoint partner's blocks are
    the transposes of the forward term's."""
    cfg = dict(CONFIGS[name])
    if n_terms is not None:
        cfg["T"] = int(n_terms)
    table = sector_table(cfg, seed)
    left = right = table
    T = cfg["T"]
    g = philox(seed, STREAM_TERMS)
    kinds = []
    while len(kinds) < T:
        d = (0, 0) if T - len(kinds) == 1 else DELTAS[int(g.integers(len(DELTAS)))]
        c = float(g.standard_normal()) / np.sqrt(T)
        if d == (0, 0):
            kinds.append(("self", d, c))
        else:
            kinds.append(("fwd", d, c))
            kinds.append(("adj", (-d[0], -d[1]), c if d[0] % 2 == 0 else -c))
    dims = [int(x) for x in table[:, 2]]
    a_off = -np.ones((T, len(left)), np.int64)
    b_off = -np.ones((T, len(right)), np.int64)
    pairs = {}
    pos = 0
    for t, (_, d, _) in enumerate(kinds):
        for off, shift in ((a_off, d), (b_off, (-d[0], -d[1]))):
            if shift not in pairs:
                pairs[shift] = _shift_pairs(table, shift)
            for q, p in pairs[shift]:
                off[t, q] = pos
                pos += dims[p] * dims[q]
    op = np.empty(pos, np.float64)

    def block(off, t, q, p):
        return op[off[t, q]:off[t, q] + dims[p] * dims[q]].reshape(dims[p], dims[q])

    for t, (kind, d, _) in enumerate(kinds):
        if kind == "adj":   # A'[q <- p] = A[p <- q]^T of the forward partner, B likewise
            dn, ds = -d[0], -d[1]      # the partner's (forward) shift
            for off, shift in ((a_off, (dn, ds)), (b_off, (-dn, -ds))):
                for q, p in pairs[shift]:
                    block(off, t, p, q)[...] = block(off, t - 1, q, p).T
            continue
        gt = philox(seed, 1 + t)
        for off, shift in ((a_off, d), (b_off, (-d[0], -d[1]))):
            for q, p in pairs[shift]:
                m = gt.standard_normal((dims[p], dims[q])) / np.sqrt(float(dims[q]))
                if kind == "self":
                    m = 0.5 * (m + m.T)
                block(off, t, q, p)[...] = m
    return Problem(left=np.asarray(left, np.int32).reshape(-1, 3), right=np.asarray(right, np.int32).reshape(-1, 3),
                   target=(int(cfg["target"][0]), int(cfg["target"][1])),
                   coef=np.array([k[2] for k in kinds], np.float64),
                   delta=np.array([k[1] for k in kinds], np.int32).reshape(T, 2),
                   parity=np.array([1 if k[1][0] % 2 else 0 for k in kinds], np.int32),
                   a_off=a_off, b_off=b_off, op_data=op,
                   dim=wavefunction_dim(left, right, cfg["target"]), seed=seed, name=name)
