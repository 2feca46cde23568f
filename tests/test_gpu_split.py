"""GPU parity of the split-precision (Ozaki, BF16 slices on tcgen05) H_eff*psi
against the FP64 oracle: relative Frobenius error <= 1e-11, bit-exact results
when every slice product and partial sum is an exactly representable integer,
determinism, edge cases, and Davidson eigenvalues within 1e-10."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import gpu_apply, rel_fro

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-11

lib = pytest.importorskip("paper_2407_07411_gb300")


def split_handle(p, nvec=1):
    return lib.HEff.from_problem(p, precision="split", max_nvec=nvec)


@pytest.mark.parametrize("nvec", [1, 2])
def test_tiny(tiny_problem, nvec):
    p = tiny_problem
    X = p.random_vectors(nvec)
    assert rel_fro(gpu_apply(split_handle(p, nvec), X), heff.apply(p, X)) <= TOL_SPLIT


def test_mid_full_and_deterministic():
    p = S.generate("mid")
    h = split_handle(p)
    x = p.random_vectors(1)
    y = gpu_apply(h, x)
    assert rel_fro(y[0], heff.apply(p, x[0])) <= TOL_SPLIT
    assert np.array_equal(gpu_apply(h, x), y)


@pytest.mark.parametrize("nvec", [1, 3])
def test_output_chunks_bit_identical(nvec):
    # the output blocks in chunks that reuse one intermediate buffer (a 1-byte cap puts
    # every block in a chunk of its own; 2 MB groups a few): the same bits as one chunk,
    # under the default schedule and one launch per GEMM; the streamed diagonal equals
    # the FP64 handle's bit for bit
    import torch
    p = S.generate("mid")
    X = p.random_vectors(nvec)
    one = split_handle(p, nvec)
    ref = gpu_apply(one, X)
    assert rel_fro(ref[0], heff.apply(p, X[0])) <= TOL_SPLIT
    d_split = torch.empty(p.dim, dtype=torch.float64, device="cuda")
    one.diagonal(d_split)
    one.close()
    h64 = lib.HEff.from_problem(p, precision="fp64")
    d_fp64 = torch.empty_like(d_split)
    h64.diagonal(d_fp64)
    torch.cuda.synchronize()
    h64.close()
    assert torch.equal(d_split, d_fp64)
    for cap in (1, 2 << 20):
        h = lib.HEff.from_problem(p, precision="split", max_nvec=nvec, split_mid_bytes=cap)
        assert np.array_equal(gpu_apply(h, X), ref)
        h.schedule = dict(h.schedule, per_gemm=1)
        assert np.array_equal(gpu_apply(h, X), ref)
        h.close()


@pytest.mark.parametrize("name,n_terms,nvec", [("mid", 300, 8), ("heavy", 120, 8), ("tiny", None, 5)])
def test_stacked_vectors(name, n_terms, nvec):
    # nvec vectors stacked inside every slice GEMM; every call size up to max_nvec
    p = S.generate(name, n_terms=n_terms)
    h = split_handle(p, nvec)
    X = p.random_vectors(nvec)
    ref = heff.apply(p, X)
    for nv in sorted({1, 2, nvec}):
        Y = gpu_apply(h, X[:nv])
        for v in range(nv):
            assert rel_fro(Y[v], ref[v]) <= TOL_SPLIT


def test_davidson_split_block8(tiny_problem, tiny_dense):
    import torch
    w = np.linalg.eigvalsh(tiny_dense)
    h = split_handle(tiny_problem, 8)
    ev, info = h.davidson(torch.from_numpy(tiny_problem.random_vectors(8)).cuda(), k_eig=3, block=8, tol=1e-9)
    assert info["converged"]
    np.testing.assert_allclose(ev, w[:3], rtol=1e-10, atol=0)


def test_heavy_tailed_reduced():
    p = S.generate("heavy", n_terms=240)
    x = p.random_vectors(1)
    assert rel_fro(gpu_apply(split_handle(p), x)[0], heff.apply(p, x[0])) <= TOL_SPLIT


def _integer_problem(rng, dims, n_terms, coef_choices=(1.0, -1.0, 2.0)):
    # one (n, 2Sz) sector lattice with integer operator entries |v| <= 127 and
    # power-of-two coefficients: every slice product and partial sum is an exact
    # integer below 2^24, so the split result must equal exact arithmetic
    tab = np.array(sorted((n, s, d) for (n, s), d in dims), np.int32)
    keys = {(int(n), int(s)): i for i, (n, s, _) in enumerate(tab)}
    deltas = [(0, 0), (1, 1), (-1, -1), (1, -1), (-1, 1), (0, 2), (0, -2)]
    terms = []
    for t in range(n_terms):
        dl = deltas[t % len(deltas)]
        ab, bb = {}, {}
        for q, (n, s, d) in enumerate(tab):
            p = keys.get((int(n) + dl[0], int(s) + dl[1]))
            if p is not None:
                ab[q] = rng.integers(-127, 128, (int(tab[p][2]), int(d))).astype(np.float64)
            p = keys.get((int(n) - dl[0], int(s) - dl[1]))
            if p is not None:
                bb[q] = rng.integers(-127, 128, (int(tab[p][2]), int(d))).astype(np.float64)
        terms.append((float(rng.choice(coef_choices)), dl, dl[0] % 2, ab, bb))
    return S.assemble(tab, tab, (4, 0), terms)


def test_exact_integer_arithmetic():
    rng = np.random.default_rng(7)
    dims = [((1, -1), 70), ((1, 1), 90), ((2, 0), 130), ((3, 1), 40), ((3, -1), 200), ((2, 2), 20), ((2, -2), 3)]
    p = _integer_problem(rng, dims, 14)
    x = rng.integers(-127, 128, p.dim).astype(np.float64)
    y = gpu_apply(split_handle(p), x)[0]
    ref = heff.apply(p, x)
    assert np.all(np.abs(ref) < 2 ** 52)
    assert np.array_equal(y, ref)


@pytest.mark.parametrize("dl,dr", [(1, 1), (100, 70), (33, 257), (130, 65)])
def test_edge_single_sector(dl, dr):
    rng = np.random.default_rng(dl * 1000 + dr)
    A, B = rng.standard_normal((dl, dl)), rng.standard_normal((dr, dr))
    x = rng.standard_normal((dl, dr))
    p = S.assemble([(2, 0, dl)], [(2, 0, dr)], (4, 0), [(0.7, (0, 0), 0, {0: A}, {0: B})])
    y = gpu_apply(split_handle(p), x.ravel())[0]
    assert rel_fro(y, (0.7 * A @ x @ B.T).ravel()) <= TOL_SPLIT


def test_edge_long_reduction_and_scales():
    # 400 terms on one block, coefficients over 12 decades: stage 2 runs over K =
    # 3600 (several exact drains) and the per-vector scales must absorb the range
    rng = np.random.default_rng(3)
    d = 9
    terms = [(float(10.0 ** rng.uniform(-6, 6) * rng.choice([-1, 1])), (0, 0), 0,
              {0: rng.standard_normal((d, d))}, {0: rng.standard_normal((d, d))}) for _ in range(400)]
    p = S.assemble([(1, 1, d)], [(1, -1, d)], (2, 0), terms)
    x = rng.standard_normal(p.dim)
    assert rel_fro(gpu_apply(split_handle(p), x)[0], heff.apply(p, x)) <= TOL_SPLIT


def test_edge_subnormal_vector(tiny_problem):
    # every entry of x subnormal: x is sliced relative to its own (subnormal) exponent,
    # not flushed to zero; both sides round y to the subnormal grid (about 2^-44 of its
    # entries here), far inside the tolerance
    p = tiny_problem
    x = p.random_vectors(1)[0] * 2.0 ** -1030
    assert np.all(np.abs(x) < np.finfo(np.float64).tiny)
    y = gpu_apply(split_handle(p), x)[0]
    ref = heff.apply(p, x)
    assert np.count_nonzero(y) == np.count_nonzero(ref) > 0
    assert rel_fro(y, ref) <= TOL_SPLIT


def test_edge_absent_blocks_and_zero_vector(tiny_problem):
    p = tiny_problem
    rng = np.random.default_rng(12)
    a_off = p.a_off.copy(); b_off = p.b_off.copy()
    a_off[rng.random(a_off.shape) < 0.3] = -1
    b_off[rng.random(b_off.shape) < 0.3] = -1
    q = S.Problem(**{**p.__dict__, "a_off": a_off, "b_off": b_off})
    h = split_handle(q, 2)
    X = q.random_vectors(2)
    X[1] = 0.0
    Y = gpu_apply(h, X)
    assert rel_fro(Y[0], heff.apply(q, X[0])) <= TOL_SPLIT
    assert not np.any(Y[1])


def test_davidson_split_tiny_and_mid(tiny_problem, tiny_dense):
    import json
    import os
    import torch
    w0 = np.linalg.eigvalsh(tiny_dense)[0]
    h = split_handle(tiny_problem)
    ev, info = h.davidson(torch.from_numpy(tiny_problem.random_vectors(1)).cuda(), tol=1e-9)
    assert info["converged"] and abs(ev[0] - w0) <= 1e-10 * abs(w0)
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "synth_digests.json")))
    p = S.generate("mid")
    h = split_handle(p)
    ev, info = h.davidson(torch.from_numpy(p.random_vectors(1)).cuda(), tol=1e-9, max_iter=600)
    assert info["converged"] and abs(ev[0] - g["mid"]["e0"]) <= 1e-10 * abs(g["mid"]["e0"])
