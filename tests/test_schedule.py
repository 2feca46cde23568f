"""Host side of the work-list schedule (batching step): defaults, range checks, and
that every schedule keeps the plan bit-exact and passes the split planner's bounds
proof (plan-only handles, no GPU)."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff

lib = pytest.importorskip("paper_2407_07411_gb300")

DEFAULT = dict(fp64_kchunk=[512, 512, 2048], fp64_ctas_per_sm=0, split_kchunk=[0, 0, 0], per_gemm=0, fp64_tile=0)


def test_default_schedule():
    p = S.generate("tiny")
    for prec in ("fp64", "split"):
        h = lib.HEff.from_problem(p, precision=prec, plan_only=True)
        assert h.schedule == DEFAULT


@pytest.mark.parametrize("bad", [
    dict(fp64_kchunk=[500, 512, 512]),          # not a multiple of 16
    dict(fp64_kchunk=[-16, 512, 512]),
    dict(split_kchunk=[12, 0, 0]),              # not a multiple of 8
    dict(split_kchunk=[0, 0, 264]),             # above 256 K tiles (32 drains)
    dict(fp64_ctas_per_sm=65),
    dict(per_gemm=2),
    dict(fp64_tile=3),                          # tile shapes 0..2
])
def test_schedule_range_checks(bad):
    h = lib.HEff.from_problem(S.generate("tiny"), precision="split", plan_only=True)
    with pytest.raises(lib.DmrgError) as ei:
        h.schedule = {**DEFAULT, **bad}
    assert ei.value.code == lib.ERR_INVALID_ARG
    assert h.schedule == DEFAULT


@pytest.mark.parametrize("name,n_terms", [("mid", 200), ("heavy", 80)])
def test_schedules_keep_plan_and_bounds(name, n_terms):
    # the split planner re-proves its buffer bounds for every stacked-vector plan
    p = S.generate(name, n_terms=n_terms)
    ref = heff.plan(p)
    for prec, nv in (("fp64", 1), ("split", 4)):
        h = lib.HEff.from_problem(p, precision=prec, max_nvec=nv, plan_only=True)
        for sched in (dict(DEFAULT, fp64_kchunk=[256, 1024, 0], fp64_ctas_per_sm=3),
                      dict(DEFAULT, fp64_tile=1, fp64_kchunk=[0, 256, 512]),
                      dict(DEFAULT, fp64_tile=2, per_gemm=1),
                      dict(DEFAULT, split_kchunk=[8, 64, 256]),
                      dict(DEFAULT, split_kchunk=[256, 16, 8], per_gemm=1)):
            h.schedule = sched
            assert h.schedule == sched
            assert h.plan_dump().tobytes() == ref.tobytes()
