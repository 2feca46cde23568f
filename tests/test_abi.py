"""The C-ABI library without a GPU: it loads, exports every function declared in
include/dmrg_heff.h, validates its inputs on the host, and its host-only planner
reproduces the oracle plan bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

import dmrg_synth as S
from oracle import heff

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
lib = pytest.importorskip("paper_2407_07411_gb300")


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(dmrg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert "dmrg_heff_apply" in names and "dmrg_davidson" in names
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert set(names) <= set(lib.SYMBOLS) | set(names)


def test_strerror():
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib._lib.dmrg_strerror(code)
    assert lib._lib.dmrg_strerror(-99) == b"unknown error code"


@pytest.mark.parametrize("name,n_terms", [("tiny", None), ("mid", 120), ("heavy", 60)])
def test_host_plan_bit_exact(name, n_terms):
    p = S.generate(name, n_terms=n_terms)
    h = lib.HEff.from_problem(p, plan_only=True)
    assert h.dim == p.dim
    ref = heff.plan(p)
    got = h.plan_dump()
    assert got.dtype == np.int64 and got.tobytes() == ref.tobytes()
    assert h.flops == heff.plan_flops(p)


def _tiny_args(p):
    return dict(left=p.left, right=p.right, target=p.target, coef=p.coef, delta=p.delta,
                parity=p.parity, a_off=p.a_off, b_off=p.b_off, op_data=p.op_data)


def test_rejects_malformed_inputs():
    p = S.generate("tiny")
    base = _tiny_args(p)

    def code(**kw):
        args = dict(base, **kw)
        with pytest.raises(lib.DmrgError) as e:
            lib.HEff(**args, plan_only=True)
        return e.value.code

    bad_left = p.left.copy(); bad_left[[0, 1]] = bad_left[[1, 0]]
    assert code(left=bad_left) == -1                       # unsorted sectors
    zero_dim = p.left.copy(); zero_dim[3, 2] = 0
    assert code(left=zero_dim) == -1                       # empty sector
    par = p.parity.copy(); par[0] = 2
    assert code(parity=par) == -1                          # parity not 0/1
    a = p.a_off.copy(); a[0, np.argmax(a[0] >= 0)] = p.op_data.size
    assert code(a_off=a) == -1                             # offset past the end
    c = p.coef.copy(); c[1] = np.nan
    assert code(coef=c) == -1                              # non-finite coefficient
    # a block present for a shift whose output sector does not exist
    t = int(np.argmax(p.delta[:, 0] == 2))
    q = int(np.argmax(p.a_off[t] < 0))
    a = p.a_off.copy(); a[t, q] = 0
    assert code(a_off=a) == -2


def test_empty_target_sector():
    p = S.generate("tiny")
    h = lib.HEff(p.left, p.right, (100, 0), p.coef, p.delta, p.parity, p.a_off, p.b_off, p.op_data,
                 plan_only=True)
    assert h.dim == 0 and h.flops == 0 and h.plan_dump().shape == (0, 5)


def test_plan_only_handle_refuses_compute():
    p = S.generate("tiny")
    h = lib.HEff.from_problem(p, plan_only=True)
    with pytest.raises(lib.DmrgError) as e:
        h.apply_host(np.zeros(p.dim))
    assert e.value.code == -1


@pytest.mark.parametrize("name,n_terms,nvec", [("tiny", None, 1), ("tiny", None, 8), ("mid", None, 4),
                                               ("heavy", 120, 8), ("precision", 24, 2)])
def test_split_plan_bounds_proof(name, n_terms, nvec):
    # the split planner proves on the host that every copy, slice write, exponent
    # access and output store of its kernels stays inside its buffer, for every number
    # of stacked vectors up to nvec
    p = S.generate(name, n_terms=n_terms)
    h = lib.HEff.from_problem(p, precision="split", plan_only=True, max_nvec=nvec)
    assert h.dim == p.dim and h.plan_dump().tobytes() == heff.plan(p).tobytes()


def test_renorm_plan_argument_checks_on_the_host():
    # every argument error of the renormalisation plan is reported before any device
    # work (these run without a GPU); an empty block list needs no device at all
    d, dn = np.array([3, 4], np.int32), np.array([2, 4], np.int32)
    good = np.array([[0, 1, 0]], np.int64)
    for dims, dims_new, blocks, op_len, out_len in [
            (d, np.array([4, 4], np.int32), good, 100, 100),          # new dim above the dim
            (d, dn, np.array([[2, 1, 0]], np.int64), 100, 100),       # sector out of range
            (d, dn, np.array([[0, 1, 95]], np.int64), 100, 100),      # block outside op
            (d, dn, good, 100, 7)]:                                   # out too small (needs 8)
        with pytest.raises(lib.DmrgError) as e:
            lib.Renorm(dims, dims_new, blocks, op_len, out_len)
        assert e.value.code == -1
    r = lib.Renorm(d, dn, np.zeros((0, 3), np.int64), 0, 0)
    assert len(r.out_off) == 0
    r.close()
