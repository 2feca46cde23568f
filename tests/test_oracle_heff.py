"""Oracle H_eff*psi, planner and diagonal against definitions computed another
way: dense Kronecker assembly (numpy.kron over full block matrices), library
matmul for one-block special cases, invariants, and a hand-computed plan."""
import json
import os

import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny(tiny_problem):
    return tiny_problem


@pytest.fixture(scope="module")
def mid_small():
    return S.generate("mid", n_terms=60)


def test_tiny_matches_dense_kronecker(tiny, tiny_dense):
    H = tiny_dense
    X = tiny.random_vectors(3)
    for x in X:
        y = heff.apply(tiny, x)
        assert np.linalg.norm(H @ x - y) <= 1e-14 * np.linalg.norm(y)
    assert np.array_equal(H, H.T)


def test_tiny_diagonal_matches_dense(tiny, tiny_dense):
    np.testing.assert_allclose(heff.diagonal(tiny), np.diag(tiny_dense), rtol=0, atol=1e-15)


def test_symmetry_and_linearity(mid_small):
    p = mid_small
    x, z = p.random_vectors(2)
    hx, hz = heff.apply(p, x), heff.apply(p, z)
    lhs, rhs = x @ hz, hx @ z
    assert abs(lhs - rhs) <= 1e-13 * (np.linalg.norm(x) * np.linalg.norm(hz))
    a, b = 0.37, -2.1
    h_lin = heff.apply(p, a * x + b * z)
    assert np.linalg.norm(h_lin - (a * hx + b * hz)) <= 1e-13 * np.linalg.norm(h_lin)


def test_batched_equals_single(mid_small):
    X = mid_small.random_vectors(3)
    Y = heff.apply(mid_small, X)
    for v in range(3):
        assert np.array_equal(Y[v], heff.apply(mid_small, X[v]))


def test_sector_conservation(tiny):
    blocks = heff.psi_blocks(tiny)
    lidx = {(int(n), int(s)): i for i, (n, s, _) in enumerate(tiny.left)}
    deltas = {(int(a), int(b)) for a, b in tiny.delta}
    for k, (iL, iR, off, r, c) in enumerate(blocks):
        x = np.zeros(tiny.dim)
        x[off:off + r * c] = np.arange(1, r * c + 1)
        y = heff.apply(tiny, x)
        n, s = int(tiny.left[iL][0]), int(tiny.left[iL][1])
        reach = {lidx.get((n + dn, s + ds)) for dn, ds in deltas} - {None}
        for k2, (jL, _, off2, r2, c2) in enumerate(blocks):
            if jL not in reach:
                assert not np.any(y[off2:off2 + r2 * c2])


def test_single_term_single_sector_is_matmul():
    rng = np.random.default_rng(5)
    A, B, x = rng.standard_normal((7, 7)), rng.standard_normal((5, 5)), rng.standard_normal((7, 5))
    tabL, tabR = np.array([(2, 0, 7)], np.int32), np.array([(2, 0, 5)], np.int32)
    p = S.assemble(tabL, tabR, (4, 0), [(0.3, (0, 0), 0, {0: A}, {0: B})])
    y = heff.apply(p, x.ravel())
    np.testing.assert_allclose(y, (0.3 * A @ x @ B.T).ravel(), rtol=1e-15, atol=1e-15)


def test_identity_operators_scale(tiny):
    terms = []
    ab = {q: np.eye(int(d)) for q, (_, _, d) in enumerate(tiny.left)}
    bb = {q: np.eye(int(d)) for q, (_, _, d) in enumerate(tiny.right)}
    p = S.assemble(tiny.left, tiny.right, tiny.target, [(-1.25, (0, 0), 0, ab, bb)])
    x = tiny.random_vectors(1)[0]
    assert np.array_equal(heff.apply(p, x), -1.25 * x)


def test_parity_sign_on_one_hot():
    # left sectors n = 0..3 (one state each), right the mirror; one odd term
    # A = B = 1 per block with Delta = (1, 1): y[out] = (-1)^{n_L(in)} x[in].
    tab = np.array([(0, 0, 1), (1, 1, 1), (2, 2, 1), (3, 3, 1)], np.int32)
    one = np.ones((1, 1))
    ab = {q: one for q in range(3)}
    bb = {q: one for q in range(1, 4)}
    p = S.assemble(tab, tab, (3, 3), [(1.0, (1, 1), 1, ab, bb)])
    for k in range(3):
        x = np.zeros(4); x[k] = 1.0
        y = heff.apply(p, x)
        expect = np.zeros(4); expect[k + 1] = (-1.0) ** k
        assert np.array_equal(y, expect)


def test_plan_hand_computed():
    g = json.load(open(os.path.join(GOLDEN, "plan_small.json")))
    one = lambda r, c: np.ones((r, c))
    L, R = np.array(g["left"], np.int32), np.array(g["right"], np.int32)
    dims = {(int(n), int(s)): int(d) for n, s, d in L}
    dimsR = {(int(n), int(s)): int(d) for n, s, d in R}
    terms = []
    for dn, ds in g["terms"]:
        ab = {}
        for q, (n, s, d) in enumerate(L):
            pq = (int(n) + dn, int(s) + ds)
            if pq in dims:
                ab[q] = one(dims[pq], int(d))
        bb = {}
        for q, (n, s, d) in enumerate(R):
            pq = (int(n) - dn, int(s) - ds)
            if pq in dimsR:
                bb[q] = one(dimsR[pq], int(d))
        terms.append((1.0, (dn, ds), dn % 2, ab, bb))
    p = S.assemble(L, R, tuple(g["target"]), terms)
    plan = heff.plan(p)
    assert plan.tolist() == g["plan"]
    assert heff.plan_flops(p) == g["total_flops"]


def test_item_flops_closed_form():
    # For a square problem a=b=c=d=n both orders cost 4 n^3 (the D^3 cost of
    # the eigensolver step).
    for n in (1, 7, 64):
        fa, fb = heff.item_flops(n, n, n, n)
        assert fa == fb == 4 * n ** 3


def test_apply_entries_match(mid_small):
    x = mid_small.random_vectors(1)[0]
    y = heff.apply(mid_small, x)
    idx = np.random.default_rng(1).choice(mid_small.dim, 40, replace=False)
    np.testing.assert_allclose(heff.apply_entries(mid_small, x, idx), y[idx], rtol=1e-12, atol=1e-14)
