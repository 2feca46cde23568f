"""One local DMRG update on the GPU, end to end: the Davidson ground state of the mid
workload, its decomposition and truncation to D states, and the left operators carried
into the kept bases; each result is checked against the oracle taking the GPU's
preceding output as its input (energy against the pinned oracle E0, singular values
and discarded weight against the oracle decomposition, renormalised blocks against
the oracle definition with the GPU bases); the same on the spin-adapted mid workload."""
import json
import os

import numpy as np
import pytest

import dmrg_synth as S
from oracle.renorm import renormalise as oracle_renormalise
from oracle.svd import truncate as oracle_truncate
from tests.gpu_util import rel_fro

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "synth_digests.json")


def test_mid_update_chain():
    import torch
    p = S.generate("mid")
    h = lib.HEff.from_problem(p, precision="split")
    x = torch.from_numpy(p.random_vectors(1)).cuda()
    ev, info = h.davidson(x, tol=1e-9, max_iter=800)
    e0 = json.load(open(GOLDEN))["mid"]["e0"]
    assert info["converged"] and abs(ev[0] - e0) <= 1e-10 * abs(e0)
    psi = x[0].contiguous()
    D = 300
    r = h.svd_truncate(psi, D)
    blk = h.psi_blocks()
    ref = oracle_truncate([(int(o), int(rw), int(c)) for _, _, rw, c, o in blk], psi.cpu().numpy(), D)
    assert list(r["kept"]) == ref["kept"] and sum(r["kept"]) == D
    assert abs(r["discarded"] - ref["discarded"]) <= 1e-12
    # the kept left bases, sector by sector, and the A blocks between kept sectors
    Uall = r["U"].cpu().numpy()
    dims = p.left[:, 2].astype(np.int32)
    k_of = {int(b[0]): int(k) for b, k in zip(blk, r["kept"])}
    sect = [q for q in range(len(dims)) if k_of.get(q, 0) > 0]
    new_id = {q: i for i, q in enumerate(sect)}
    sub_dims = dims[sect]
    sub_new = np.array([k_of[q] for q in sect], np.int32)
    bases = []
    for q in sect:
        b = [i for i, row in enumerate(blk) if int(row[0]) == q][0]
        bases.append(Uall[r["u_off"][b]:r["u_off"][b] + dims[q] * k_of[q]])
    U = np.concatenate(bases)
    idx = {(int(n), int(s)): i for i, (n, s, _) in enumerate(p.left)}
    blocks = []
    for t in range(p.n_terms):
        for q in sect:
            if p.a_off[t, q] < 0:
                continue
            out = idx[(int(p.left[q][0]) + int(p.delta[t][0]), int(p.left[q][1]) + int(p.delta[t][1]))]
            if out in new_id:
                blocks.append((new_id[q], new_id[out], int(p.a_off[t, q])))
    blocks = np.array(blocks, np.int64)
    n_out = int(sum(int(sub_new[a]) * int(sub_new[b]) for a, b, _ in blocks))
    out = torch.empty(n_out, dtype=torch.float64, device="cuda")
    offs = lib.renormalise(sub_dims, sub_new, torch.from_numpy(U).cuda(), blocks, torch.from_numpy(p.op_data).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = oracle_renormalise(sub_dims, sub_new, U, blocks, p.op_data)
    g = np.concatenate([got[o:o + w.size] for o, w in zip(offs, want)])
    assert len(blocks) > 100 and rel_fro(g, np.concatenate([w.ravel() for w in want])) <= 1e-12


@pytest.mark.parametrize("target,D", [(None, 300), ((20, 2), 300)], ids=["singlet", "triplet"])
def test_su2_mid_update_chain(target, D):
    """The same chain on the spin-adapted mid workload: Davidson (split), truncation per
    left sector (blocks side by side), and the reduced A blocks carried into the kept
    multiplet bases (the basis change acts inside each (n, S) sector, so reduced blocks
    transform like U(1) blocks)."""
    import torch
    from dmrg_synth import su2 as G
    from oracle import su2 as O
    p = G.generate("su2_mid", target=target)
    h = lib.HEff.from_problem(p, precision="split")
    x = torch.from_numpy(p.random_vectors(1)).cuda()
    ev, info = h.davidson(x, tol=1e-9, max_iter=800)
    assert info["converged"]
    if target is None:
        e0 = json.load(open(GOLDEN))["su2_mid"]["e0"]
        assert abs(ev[0] - e0) <= 1e-10 * abs(e0)
    psi = x[0].contiguous()
    r = h.svd_truncate(psi, D)
    ref = O.truncate(p, psi.cpu().numpy(), D)
    assert list(r["sectors"]) == ref["sectors"] and list(r["kept"]) == ref["kept"] and sum(r["kept"]) == D
    assert abs(r["discarded"] - ref["discarded"]) <= 1e-12
    Uall = r["U"].cpu().numpy()
    dims = p.left[:, 2].astype(np.int32)
    k_of = {int(q): int(k) for q, k in zip(r["sectors"], r["kept"])}
    m_of = {int(q): m for m, q in enumerate(r["sectors"])}
    sect = [q for q in range(len(dims)) if k_of.get(q, 0) > 0]
    new_id = {q: i for i, q in enumerate(sect)}
    sub_new = np.array([k_of[q] for q in sect], np.int32)
    U = np.concatenate([Uall[r["u_off"][m_of[q]]:r["u_off"][m_of[q]] + dims[q] * k_of[q]] for q in sect])
    blocks = np.array([(new_id[int(q)], new_id[int(pp)], int(off)) for _, q, pp, off in p.a_blocks
                       if int(q) in new_id and int(pp) in new_id], np.int64)
    n_out = int(sum(int(sub_new[a]) * int(sub_new[b]) for a, b, _ in blocks))
    out = torch.empty(n_out, dtype=torch.float64, device="cuda")
    offs = lib.renormalise(dims[sect], sub_new, torch.from_numpy(U).cuda(), blocks,
                           torch.from_numpy(p.op_data).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = oracle_renormalise(dims[sect], sub_new, U, blocks, p.op_data)
    g = np.concatenate([got[o:o + w.size] for o, w in zip(offs, want)])
    assert len(blocks) > 100 and rel_fro(g, np.concatenate([w.ravel() for w in want])) <= 1e-12
