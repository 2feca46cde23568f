"""GPU side of the work-list schedule (batching step): every schedule computes the
same H_eff*psi -- the split path bit for bit, the FP64 path bit for bit when only the
launch grouping changes (one launch per GEMM) and within 1e-12 of the oracle for other
split-K extents -- and the autotuner leaves in place a schedule it measured, no slower
than the one it started from, under which the results stay within tolerance."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import gpu_apply, rel_fro

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")
DEFAULT = dict(fp64_kchunk=[512, 512, 2048], fp64_ctas_per_sm=0, split_kchunk=[0, 0, 0], per_gemm=0, fp64_tile=0)


@pytest.mark.parametrize("name,n_terms", [("mid", 200), ("heavy", 80)])
def test_fp64_schedules(name, n_terms):
    p = S.generate(name, n_terms=n_terms)
    X = p.random_vectors(2)
    ref = heff.apply(p, X)
    h = lib.HEff.from_problem(p, precision="fp64", max_nvec=2)
    y0 = gpu_apply(h, X)
    assert rel_fro(y0, ref) <= 1e-12
    h.schedule = dict(DEFAULT, per_gemm=1)
    assert np.array_equal(gpu_apply(h, X), y0)
    for sched in (dict(DEFAULT, fp64_kchunk=[256, 1024, 0], fp64_ctas_per_sm=2),
                  dict(DEFAULT, fp64_kchunk=[0, 0, 0], per_gemm=1)):
        h.schedule = sched
        assert rel_fro(gpu_apply(h, X), ref) <= 1e-12
        assert rel_fro(gpu_apply(h, X[:1]), ref[:1]) <= 1e-12
    # the output tile: each element's sum runs in the same order whatever the tile, so
    # with the same K chunks the results are the same bits
    for tile in (1, 2):
        h.schedule = dict(DEFAULT, fp64_tile=tile)
        assert np.array_equal(gpu_apply(h, X), y0)
        h.schedule = dict(DEFAULT, fp64_tile=tile, per_gemm=1, fp64_ctas_per_sm=3)
        assert np.array_equal(gpu_apply(h, X), y0)


@pytest.mark.parametrize("name,n_terms,nvec", [("heavy", 120, 4), ("mid", 200, 2)])
def test_split_schedules_bit_identical(name, n_terms, nvec):
    p = S.generate(name, n_terms=n_terms)
    X = p.random_vectors(nvec)
    h = lib.HEff.from_problem(p, precision="split", max_nvec=nvec)
    y0 = gpu_apply(h, X)
    y1 = gpu_apply(h, X[:1])
    assert rel_fro(y0, heff.apply(p, X)) <= 1e-11
    for sched in (dict(DEFAULT, split_kchunk=[8, 64, 256]),
                  dict(DEFAULT, split_kchunk=[256, 16, 8], per_gemm=1),
                  dict(DEFAULT, per_gemm=1)):
        h.schedule = sched
        assert np.array_equal(gpu_apply(h, X), y0)
        assert np.array_equal(gpu_apply(h, X[:1]), y1)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("split", 1e-11)])
def test_autotune(prec, tol):
    p = S.generate("mid", n_terms=200)
    h = lib.HEff.from_problem(p, precision=prec, max_nvec=2)
    r = h.autotune(nvec=2, reps=2)
    assert r["nvec"] == 2 and r["trials"] >= 2
    assert 0 < r["best_ms"] <= r["default_ms"]
    assert h.schedule == r["best"] and r["best"]["per_gemm"] == 0
    want = [(32, 32), (64, 32), (32, 64)][r["best"]["fp64_tile"]] if prec == "fp64" else (128, 96)
    assert tuple(r["tile"]) == want
    X = p.random_vectors(2)
    assert rel_fro(gpu_apply(h, X), heff.apply(p, X)) <= tol
    with pytest.raises(lib.DmrgError):
        h.autotune(nvec=3)
