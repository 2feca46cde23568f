"""Failure detection on the GPU without a fault: a bounded wait that runs out must
return DMRG_ERR_DEVICE_TIMEOUT through the status word and leave the CUDA context
usable for the next call."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff
from tests.gpu_util import gpu_apply, rel_fro

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")


def test_bounded_wait_times_out_and_context_survives(tiny_problem):
    rc = lib._lib.dmrg_selftest_wait_timeout(20_000_000)    # ~10 ms of SM clock
    assert rc == -5
    assert b"ran out" in lib._lib.dmrg_last_error()
    x = tiny_problem.random_vectors(1)
    for prec in ("fp64", "split"):
        h = lib.HEff.from_problem(tiny_problem, precision=prec)
        assert rel_fro(gpu_apply(h, x)[0], heff.apply(tiny_problem, x[0])) <= 1e-11


def test_selftest_rejects_bad_range():
    assert lib._lib.dmrg_selftest_wait_timeout(0) == -1
