"""Device-memory figures of a handle (dmrg_heff_memory) and the output chunks of the
split path, on plan-only handles (no GPU): the FP64 operator copy is one stacked A and
B block per plan row; the split path keeps no FP64 copy and its figures add up; a
smaller intermediate cap splits the output blocks into more chunks (smaller apply
buffers) and the planner's bounds proof still holds for every chunk."""
import numpy as np
import pytest

import dmrg_synth as S

lib = pytest.importorskip("paper_2407_07411_gb300")


def _ops_len(h):
    blocks = h.psi_blocks()
    rows, cols = blocks[:, 2], blocks[:, 3]
    plan = h.plan_dump()
    o, k = plan[:, 0], plan[:, 2]
    return int(np.sum(rows[o] * rows[k] + cols[o] * cols[k]))


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_fp64_memory_is_the_operator_copy(name):
    p = S.generate(name)
    h = lib.HEff.from_problem(p, precision="fp64", plan_only=True)
    m = h.memory()
    assert m["operators"] == 8 * _ops_len(h)
    assert m["operator_slices"] == 0 and m["setup_peak"] == 0
    assert m["total"] == m["operators"] + m["apply_buffers"]
    h.close()


@pytest.mark.parametrize("name,nvec", [("tiny", 1), ("mid", 3)])
def test_split_memory_keeps_no_fp64_copy(name, nvec):
    p = S.generate(name)
    h = lib.HEff.from_problem(p, precision="split", plan_only=True, max_nvec=nvec)
    m = h.memory()
    ops = 8 * _ops_len(h)
    assert m["operators"] == 0
    assert m["operator_slices"] >= 1.5 * ops          # 6 BF16 digits per FP64 entry, plus padding
    assert 0 < m["setup_peak"] <= ops                  # one window of the FP64 layout
    assert m["total"] == m["operator_slices"] + m["apply_buffers"]
    h.close()


@pytest.mark.parametrize("nvec", [1, 2])
def test_split_output_chunks_share_the_intermediates(nvec):
    p = S.generate("mid")
    one = lib.HEff.from_problem(p, precision="split", plan_only=True, max_nvec=nvec)
    m1 = one.memory()
    one.close()
    prev = m1["apply_buffers"]
    for cap in (32 << 20, 4 << 20, 1):   # a cap below one block's needs gives one block per chunk
        h = lib.HEff.from_problem(p, precision="split", plan_only=True, max_nvec=nvec, split_mid_bytes=cap)
        m = h.memory()
        assert m["operator_slices"] == m1["operator_slices"]
        assert m["apply_buffers"] <= prev
        prev = m["apply_buffers"]
        h.close()
    assert prev < m1["apply_buffers"] / 4


def test_options_outside_the_built_path_are_refused():
    p = S.generate("tiny")
    with pytest.raises(lib.DmrgError) as e:
        lib.HEff.from_problem(p, precision="split", plan_only=True, n_slices=5)
    assert e.value.code == -8
    with pytest.raises(lib.DmrgError) as e:
        lib.HEff.from_problem(p, precision="split", plan_only=True, split_mid_bytes=-1)
    assert e.value.code == -1
    lib.HEff.from_problem(p, precision="split", plan_only=True, n_slices=6).close()
