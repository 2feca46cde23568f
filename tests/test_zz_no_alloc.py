"""The entry point that allocates no GPU memory (dmrg_heff_apply_noalloc), for
callers whose device memory is owned by someone else (a host framework's pool, an
embedding application) and who therefore cannot call cudaMalloc.  Called through
the C ABI, twice in a row, its result must match the oracle and the handle-based
entry point (dmrg_heff_apply) within the FP64 tolerance of the other parity tests,
also on a non-default stream with work still queued on it.  This file sorts last so
that a run stopping at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import gpu_apply, rel_fro

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-12

lib = pytest.importorskip("paper_2407_07411_gb300")


def _noalloc(p, op_dev, x_dev, y_dev, stream=None):
    arr = lambda a, dt: np.ascontiguousarray(np.asarray(a, dt))
    left, right = arr(p.left, np.int32), arr(p.right, np.int32)
    coef, delta, parity = arr(p.coef, np.float64), arr(p.delta, np.int32), arr(p.parity, np.int32)
    a_off, b_off = arr(p.a_off, np.int64), arr(p.b_off, np.int64)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a.size else None
    rc = lib._lib.dmrg_heff_apply_noalloc(
        ptr(left), len(left), ptr(right), len(right), int(p.target[0]), int(p.target[1]),
        ptr(coef), ptr(delta), ptr(parity), ptr(a_off), ptr(b_off), p.n_terms,
        ctypes.c_void_p(op_dev.data_ptr()), op_dev.numel(), ctypes.c_void_p(x_dev.data_ptr()),
        ctypes.c_void_p(y_dev.data_ptr()), stream)
    return rc


@pytest.mark.parametrize("name,n_terms", [("tiny", None), ("mid", 200)])
def test_noalloc_matches_oracle_and_handle_twice(name, n_terms):
    import torch
    p = S.generate(name, n_terms=n_terms)
    h = lib.HEff.from_problem(p)
    op = torch.from_numpy(p.op_data).cuda()
    X = p.random_vectors(2)
    for v in range(2):                       # two calls in a row, different inputs
        x = torch.from_numpy(X[v]).cuda()
        y = torch.full_like(x, float("nan"))
        assert _noalloc(p, op, x, y) == 0
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert rel_fro(got, heff.apply(p, X[v])) <= TOL_FP64
        assert rel_fro(got, gpu_apply(h, X[v])[0]) <= TOL_FP64


def test_noalloc_on_a_stream_with_queued_work():
    # x is written by a kernel still queued on the stream when the call is made: the
    # call must order itself after it and leave its result on that stream
    import torch
    p = S.generate("mid", n_terms=120)
    op = torch.from_numpy(p.op_data).cuda()
    xs = p.random_vectors(1)[0]
    src = torch.from_numpy(xs).cuda()
    x = torch.zeros_like(src)
    y = torch.full_like(src, float("nan"))
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        torch.cuda._sleep(2_000_000)         # keep the stream busy before the copy
        x.copy_(src)
        assert _noalloc(p, op, x, y, ctypes.c_void_p(s.cuda_stream)) == 0
        out = y.to("cpu", non_blocking=False)
    s.synchronize()
    assert rel_fro(out.numpy(), heff.apply(p, xs)) <= TOL_FP64


def test_noalloc_rejects_overlap_and_oversized_problem():
    import torch
    p = S.generate("tiny")
    op = torch.from_numpy(p.op_data).cuda()
    x = torch.from_numpy(p.random_vectors(1)[0]).cuda()
    assert _noalloc(p, op, x, x) == -1
    assert b"overlap" in lib._lib.dmrg_last_error()
    # one sector of 3000 states per block: one intermediate block alone is 72 MB
    d = 3000
    q = S.assemble([(2, 0, d)], [(2, 0, d)], (4, 0), [(1.0, (0, 0), 0, {0: np.eye(d)}, {0: np.eye(d)})])
    op = torch.from_numpy(q.op_data).cuda()
    x = torch.zeros(q.dim, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(q, op, x, y) == -1
    assert b"32 MiB" in lib._lib.dmrg_last_error()
