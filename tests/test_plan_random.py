"""Randomised planning checks (CPU, plan-only handles): on seeded random small problems of
both symmetries -- random sector tables, term kinds and subsets of present blocks -- the
library's plan, wave-function size and flop total equal the oracle's independent
planner bit for bit, and the split planner proves its bounds."""
import numpy as np
import pytest

import dmrg_synth as S
from dmrg_synth import su2 as G
from oracle import heff
from oracle import su2 as O

lib = pytest.importorskip("paper_2407_07411_gb300")


def _common_sum(pairs, rng):
    """One of the three most frequent sector sums (a target with many blocks)."""
    vals, counts = np.unique(np.array(pairs), axis=0, return_counts=True)
    top = np.argsort(-counts, kind="stable")[:3]
    v = vals[top[int(rng.integers(len(top)))]]
    return int(v[0]), int(v[1])


def _u1_problem(rng):
    secs = [(n, s) for n in range(0, 6) for s in range(-3, 4) if (s - n) % 2 == 0]
    keep = sorted(rng.choice(len(secs), size=int(rng.integers(6, 16)), replace=False))
    table = [(secs[i][0], secs[i][1], int(rng.integers(1, 6))) for i in keep]
    idx = {(n, s): i for i, (n, s, _) in enumerate(table)}
    target = _common_sum([(n1 + n2, s1 + s2) for n1, s1, _ in table for n2, s2, _ in table], rng)
    terms = []
    for _ in range(int(rng.integers(4, 20))):
        d = S.DELTAS[int(rng.integers(len(S.DELTAS)))]
        ab, bb = {}, {}
        for q, (n, s, dq) in enumerate(table):
            p = idx.get((n + d[0], s + d[1]))
            if p is not None and rng.random() < 0.8:
                ab[q] = rng.standard_normal((table[p][2], dq))
            p = idx.get((n - d[0], s - d[1]))
            if p is not None and rng.random() < 0.8:
                bb[q] = rng.standard_normal((table[p][2], dq))
        terms.append((float(rng.standard_normal()), d, int(d[0] % 2), ab, bb))
    return S.assemble(table, table, target, terms)


def _su2_problem(rng):
    secs = [(n, s) for n in range(0, 6) for s in range(0, 6) if (s - n) % 2 == 0]
    keep = sorted(rng.choice(len(secs), size=int(rng.integers(5, 14)), replace=False))
    table = [(secs[i][0], secs[i][1], int(rng.integers(1, 5))) for i in keep]
    target = _common_sum([(n1 + n2, s) for n1, s1, _ in table for n2, s2, _ in table
                          for s in range(abs(s1 - s2), s1 + s2 + 1, 2)], rng)
    terms = []
    for _ in range(int(rng.integers(3, 14))):
        dn, k2 = G.KINDS[int(rng.integers(len(G.KINDS)))]
        blocks = []
        for sh in (dn, -dn):
            b = {}
            for q, p in G.block_pairs(np.array(table), sh, k2):
                if rng.random() < 0.7:
                    b[(q, p)] = rng.standard_normal((table[p][2], table[q][2]))
            blocks.append(b)
        terms.append((float(rng.standard_normal()), k2, dn, int(dn % 2), blocks[0], blocks[1]))
    return G.pack(table, table, target, terms)


@pytest.mark.parametrize("seed", range(40))
def test_u1_random_plan(seed):
    p = _u1_problem(np.random.default_rng(1000 + seed))
    h = lib.HEff.from_problem(p, plan_only=True)
    ref = heff.plan(p)
    assert h.dim == p.dim
    assert np.array_equal(h.plan_dump(), ref)
    assert h.flops == (int(ref[:, 4].sum()) if len(ref) else 0)


@pytest.mark.parametrize("seed", range(40))
def test_su2_random_plan(seed):
    p = _su2_problem(np.random.default_rng(2000 + seed))
    h = lib.HEff.from_problem(p, plan_only=True)
    ref = O.plan(p)
    assert h.dim == p.dim == sum(b[3] * b[4] for b in O.psi_blocks(p))
    assert np.array_equal(h.plan_dump(), ref)
    assert h.flops == (int(ref[:, 4].sum()) if len(ref) else 0)


@pytest.mark.parametrize("seed", range(20))
@pytest.mark.parametrize("nvec", [1, 3])
def test_random_split_plans_prove_bounds(seed, nvec):
    """The split planner's host-side bounds proof (every copy, slice write, exponent and
    store in range) on the random shapes above, both symmetries."""
    for p in (_u1_problem(np.random.default_rng(1000 + seed)), _su2_problem(np.random.default_rng(2000 + seed))):
        lib.HEff.from_problem(p, precision="split", plan_only=True, max_nvec=nvec).close()
