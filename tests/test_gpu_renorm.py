"""GPU operator renormalisation (O' = U_p^T O U_q for every listed block, two stages of
the FP64 grouped tile kernel) against the oracle block by block: all A_t blocks of the mid
workload carried into random orthonormal bases with ~60 % of each sector's states, plus
square bases on the tiny workload; relative Frobenius error <= 1e-12 over all blocks."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle.renorm import renormalise as oracle_renormalise
from tests.gpu_util import rel_fro

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")


def _case(p, frac, seed):
    rng = np.random.default_rng(seed)
    dims = p.left[:, 2].astype(np.int32)
    dims_new = np.maximum(1, np.ceil(frac * dims)).astype(np.int32)
    U = np.concatenate([np.linalg.qr(rng.standard_normal((d, d)))[0][:, :k].ravel()
                        for d, k in zip(dims, dims_new)])
    idx = {(int(n), int(s)): i for i, (n, s, _) in enumerate(p.left)}
    blocks = []
    for t in range(p.n_terms):
        dn, ds = int(p.delta[t][0]), int(p.delta[t][1])
        for q in range(len(p.left)):
            if p.a_off[t, q] >= 0:
                blocks.append((q, idx[(int(p.left[q][0]) + dn, int(p.left[q][1]) + ds)], int(p.a_off[t, q])))
    return dims, dims_new, U, np.array(blocks, np.int64)


@pytest.mark.parametrize("name,frac", [("mid", 0.6), ("tiny", 1.0)])
def test_matches_oracle(name, frac):
    import torch
    p = S.generate(name)
    dims, dims_new, U, blocks = _case(p, frac, seed=5)
    n_out = int(sum(int(dims_new[q]) * int(dims_new[pp]) for q, pp, _ in blocks))
    Ud = torch.from_numpy(U).cuda()
    opd = torch.from_numpy(p.op_data).cuda()
    out = torch.full((n_out,), float("nan"), dtype=torch.float64, device="cuda")
    offs = lib.renormalise(dims, dims_new, Ud, blocks, opd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle_renormalise(dims, dims_new, U, blocks, p.op_data)
    assert np.all(np.isfinite(got))
    g = np.concatenate([got[o:o + r.size] for o, r in zip(offs, ref)])
    assert rel_fro(g, np.concatenate([r.ravel() for r in ref])) <= 1e-12


def test_plan_runs_match_one_shot_call():
    # a plan built once and run twice on a non-default stream (new bases for the second
    # run) gives the one-shot call's results bit for bit
    import torch
    p = S.generate("mid")
    dims, dims_new, U, blocks = _case(p, 0.6, seed=5)
    _, _, U2, _ = _case(p, 0.6, seed=6)
    n_out = int(sum(int(dims_new[q]) * int(dims_new[pp]) for q, pp, _ in blocks))
    opd = torch.from_numpy(p.op_data).cuda()
    plan = lib.Renorm(dims, dims_new, blocks, opd.numel(), n_out)
    st = torch.cuda.Stream()
    for Uh in (U, U2):
        Ud = torch.from_numpy(Uh).cuda()
        ref = torch.full((n_out,), float("nan"), dtype=torch.float64, device="cuda")
        off = lib.renormalise(dims, dims_new, Ud, blocks, opd, ref)
        out = torch.full_like(ref, float("nan"))
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            plan.run(Ud, opd, out, stream=st)
        st.synchronize()
        assert np.array_equal(off, plan.out_off)
        assert torch.equal(out, ref)
    plan.close()
