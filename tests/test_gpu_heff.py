"""GPU parity of H_eff*psi (FP64 DMMA path) against the CPU oracle, through the
C ABI: element-wise relative Frobenius error <= 1e-12 on tiny, mid and
heavy-tailed problems (full-vector checks at the D=4096 sizes are in
test_gpu_full_size.py), edge cases (empty
sector, no terms, absent blocks, one-state sectors, blocks spanning several tiles
with ragged tails, long split-K reductions), bit-exact plans and determinism."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import gpu_apply, rel_fro

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-12

lib = pytest.importorskip("paper_2407_07411_gb300")


@pytest.fixture(scope="module")
def mid():
    return S.generate("mid")


@pytest.mark.parametrize("nvec", [1, 3])
def test_tiny(tiny_problem, nvec):
    p = tiny_problem
    h = lib.HEff.from_problem(p, max_nvec=nvec)
    X = p.random_vectors(nvec)
    assert rel_fro(gpu_apply(h, X), heff.apply(p, X)) <= TOL_FP64
    assert h.plan_dump().tobytes() == heff.plan(p).tobytes()


def test_mid_full(mid):
    h = lib.HEff.from_problem(mid, max_nvec=2)
    X = mid.random_vectors(2)
    Y = gpu_apply(h, X)
    Yr = heff.apply(mid, X)
    for v in range(2):
        assert rel_fro(Y[v], Yr[v]) <= TOL_FP64
    # deterministic: no atomics in any accumulation
    assert np.array_equal(gpu_apply(h, X), Y)
    assert h.flops == heff.plan_flops(mid)


def test_heavy_tailed_reduced():
    p = S.generate("heavy", n_terms=240)
    h = lib.HEff.from_problem(p)
    x = p.random_vectors(1)
    assert rel_fro(gpu_apply(h, x)[0], heff.apply(p, x[0])) <= TOL_FP64


def test_apply_host_matches_device(mid):
    h = lib.HEff.from_problem(mid, max_nvec=2)
    X = mid.random_vectors(2)
    assert np.array_equal(h.apply_host(X), gpu_apply(h, X))


def test_diagonal(mid):
    import torch
    h = lib.HEff.from_problem(mid)
    d = torch.empty(mid.dim, dtype=torch.float64, device="cuda")
    h.diagonal(d)
    torch.cuda.synchronize()
    ref = heff.diagonal(mid)
    assert rel_fro(d.cpu().numpy(), ref) <= 1e-14


def test_edge_empty_sector_and_no_terms(tiny_problem):
    p = tiny_problem
    h = lib.HEff(p.left, p.right, (100, 0), p.coef, p.delta, p.parity, p.a_off, p.b_off, p.op_data)
    assert h.dim == 0
    h.apply_host(np.zeros(0))
    h0 = lib.HEff(p.left, p.right, p.target, np.zeros(0), np.zeros((0, 2)), np.zeros(0),
                  np.zeros((0, len(p.left))), np.zeros((0, len(p.right))), np.zeros(0))
    x = p.random_vectors(1)
    assert not np.any(gpu_apply(h0, x))


def test_edge_absent_blocks(tiny_problem):
    p = tiny_problem
    rng = np.random.default_rng(11)
    a_off = p.a_off.copy(); b_off = p.b_off.copy()
    a_off[rng.random(a_off.shape) < 0.3] = -1
    b_off[rng.random(b_off.shape) < 0.3] = -1
    q = S.Problem(**{**p.__dict__, "a_off": a_off, "b_off": b_off})
    h = lib.HEff.from_problem(q, max_nvec=2)
    X = q.random_vectors(2)
    assert rel_fro(gpu_apply(h, X), heff.apply(q, X)) <= TOL_FP64


@pytest.mark.parametrize("dl,dr", [(1, 1), (100, 70), (33, 257), (17, 5)])
def test_edge_single_sector_matmul(dl, dr):
    # one sector per side, one Delta=0 term: y = c A x B^T; shapes span several
    # 32-wide tiles with ragged tails, or are a single 1x1 entry
    rng = np.random.default_rng(dl * 1000 + dr)
    A, B = rng.standard_normal((dl, dl)), rng.standard_normal((dr, dr))
    x = rng.standard_normal((dl, dr))
    p = S.assemble([(2, 0, dl)], [(2, 0, dr)], (4, 0), [(0.7, (0, 0), 0, {0: A}, {0: B})])
    h = lib.HEff.from_problem(p)
    y = gpu_apply(h, x.ravel())[0]
    assert rel_fro(y, (0.7 * A @ x @ B.T).ravel()) <= TOL_FP64


def test_edge_long_reduction():
    # many Delta=0 terms on one small block: stage 2 has K = T*c >> the split-K
    # chunk, exercising the fixed-order partial reduction
    rng = np.random.default_rng(2)
    d = 9
    terms = [(float(rng.standard_normal()), (0, 0), 0, {0: rng.standard_normal((d, d))},
              {0: rng.standard_normal((d, d))}) for _ in range(400)]
    p = S.assemble([(1, 1, d)], [(1, -1, d)], (2, 0), terms)
    h = lib.HEff.from_problem(p)
    x = rng.standard_normal(p.dim)
    assert rel_fro(gpu_apply(h, x)[0], heff.apply(p, x)) <= TOL_FP64


def test_hubbard_chain_model():
    from tests.test_oracle_models import _hubbard_two_block
    p = _hubbard_two_block(2, 1.0, 4.0, (4, 0))
    h = lib.HEff.from_problem(p)
    x = np.random.default_rng(0).standard_normal(p.dim)
    assert rel_fro(gpu_apply(h, x)[0], heff.dense_h(p) @ x) <= TOL_FP64
