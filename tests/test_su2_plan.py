"""Host logic of the spin-adapted path (no GPU): the recoupling coefficient the
planner computes from the 6j closed form against the oracle's definition as a sum
over magnetic quantum numbers, the plan against the oracle's independent planner
(bit-exact), the split plan's bounds proof, and argument checks of
dmrg_heff_create_su2 / dmrg_su2_recoupling."""
import itertools

import numpy as np
import pytest

from dmrg_synth import su2 as G
from oracle import su2 as O

lib = pytest.importorskip("paper_2407_07411_gb300")


def test_recoupling_matches_definition():
    n = 0
    for sl, sr, k2, s2 in itertools.product(range(0, 7), range(0, 7), range(0, 5), range(0, 9)):
        for slo, sro in itertools.product(range(max(0, sl - k2), sl + k2 + 1, 2), range(max(0, sr - k2), sr + k2 + 1, 2)):
            assert lib.su2_recoupling(slo, sro, sl, sr, k2, s2) == pytest.approx(
                O.recoupling(slo, sro, sl, sr, k2, s2), abs=2e-15)
            n += 1
    assert n > 10000
    # larger spins: relative agreement where the coefficient is not tiny
    for sl, sr, k2, s2 in ((12, 10, 2, 6), (16, 16, 3, 1), (9, 13, 3, 8), (20, 20, 4, 0)):
        for slo in range(max(0, sl - k2), sl + k2 + 1, 2):
            for sro in range(max(0, sr - k2), sr + k2 + 1, 2):
                a, b = lib.su2_recoupling(slo, sro, sl, sr, k2, s2), O.recoupling(slo, sro, sl, sr, k2, s2)
                assert abs(a - b) <= 1e-13 * max(1.0, abs(b))


@pytest.mark.parametrize("name,target,n_terms", [("su2_tiny", None, None), ("su2_tiny", (6, 0), None),
                                                 ("su2_tiny", (5, 1), None), ("su2_mid", None, 120)])
def test_plan_bit_exact(name, target, n_terms):
    p = G.generate(name, target=target, n_terms=n_terms)
    h = lib.HEff.from_problem(p, plan_only=True)
    assert h.dim == p.dim
    ref = O.plan(p)
    got = h.plan_dump()
    assert got.dtype == np.int64 and np.array_equal(got, ref)
    assert h.flops == int(ref[:, 4].sum())
    blocks = h.psi_blocks()
    ob = O.psi_blocks(p)
    assert [tuple(r) for r in blocks[:, :2]] == [(b[0], b[1]) for b in ob]
    assert list(blocks[:, 4]) == [b[2] for b in ob]


@pytest.mark.parametrize("n_terms,nvec", [(60, 1), (60, 4), (None, 1), (None, 8)])
def test_split_plan_bounds_proof(n_terms, nvec):
    p = G.generate("su2_mid", n_terms=n_terms)
    lib.HEff.from_problem(p, precision="split", plan_only=True, max_nvec=nvec).close()


def _with(p, **kw):
    d = dict(left=p.left, right=p.right, target=p.target, coef=p.coef, rank2=p.rank2, dn=p.dn, parity=p.parity,
             a_blocks=p.a_blocks, b_blocks=p.b_blocks, op_data=p.op_data)
    d.update(kw)

    class P:
        pass
    q = P()
    for k, v in d.items():
        setattr(q, k, v)
    return q


def test_rejects_malformed_inputs():
    p = G.generate("su2_tiny")
    bad_rank = p.rank2.copy(); bad_rank[2] += 2            # block triangles no longer hold
    dup = np.concatenate([p.a_blocks, p.a_blocks[:1]])
    off = p.a_blocks.copy(); off[0, 3] = p.op_data.size   # block past the end
    neg = p.left.copy(); neg[0, 1] = -2
    unsorted = p.left[::-1].copy()
    cases = [(dict(rank2=bad_rank), lib.DmrgError), (dict(a_blocks=dup), lib.DmrgError),
             (dict(a_blocks=off), lib.DmrgError), (dict(left=neg), lib.DmrgError),
             (dict(left=unsorted), lib.DmrgError), (dict(parity=p.parity * 2), lib.DmrgError),
             (dict(target=(6, -2)), lib.DmrgError)]
    for kw, exc in cases:
        with pytest.raises(exc):
            lib.HEff.from_su2(_with(p, **kw), plan_only=True)
    for args in ((-1, 0, 0, 0, 0, 0), (0, 0, 0, 0, 42, 0), (0, 0, 0, 0, 0, 81)):
        with pytest.raises(lib.DmrgError):
            lib.su2_recoupling(*args)


def test_empty_target():
    p = G.generate("su2_tiny", target=(30, 0))
    h = lib.HEff.from_problem(p, plan_only=True)
    assert h.dim == 0 and h.flops == 0 and len(h.plan_dump()) == 0


@pytest.mark.parametrize("target", [(6, 2), (6, 0), (5, 1)])
def test_svd_matrices_group_blocks_by_left_sector(target):
    p = G.generate("su2_tiny", target=target)
    h = lib.HEff.from_problem(p, plan_only=True)
    mats = h.svd_matrices()
    blocks = O.psi_blocks(p)
    lefts = sorted({b[0] for b in blocks})
    assert list(mats[:, 0]) == lefts
    for iL, rows, cols, off in mats:
        mine = [b for b in blocks if b[0] == iL]
        assert rows == mine[0][3] and cols == sum(b[4] for b in mine) and off == mine[0][2]
    if target[1] > 0:
        assert len(mats) < len(blocks)


def test_full_mid_plan_bit_exact():
    p = G.generate("su2_mid")
    h = lib.HEff.from_problem(p, plan_only=True)
    ref = O.plan(p)
    assert np.array_equal(h.plan_dump(), ref) and h.flops == int(ref[:, 4].sum()) == 13631489180


def test_bench_workload_dispatch():
    """bench.py serves the spin-adapted workloads: generator, oracle and description."""
    import argparse
    import bench
    p = bench.load_workload("su2_tiny", 0)
    assert hasattr(p, "rank2") and bench.oracle_for(p) is O
    args = argparse.Namespace(config="su2_tiny", terms=None, seed=0, nvec=1)
    cfg = bench.workload_config(p, args, "split_bf16")
    assert cfg["psi_dim"] == p.dim and "spin-adapted" in cfg["workload"]
    assert all(isinstance(k, tuple) and len(k) == 2 for k in bench.NCU_TRAFFIC)
