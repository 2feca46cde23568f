"""GPU two-site decomposition and truncation (one-sided Jacobi SVD per wave-function
block, D largest singular values over all blocks) against the oracle: singular values
(1e-13 of the largest), kept counts, discarded weight, and the kept left bases through
their projectors U U^T (independent of signs and of rotations inside degenerate
singular subspaces); truncation to more than the rank discards nothing.  Matrices
above 64 KB (precision's larger blocks) run on the cluster kernel, beside the one-CTA
kernel on a second stream."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle.svd import truncate as oracle_truncate

pytestmark = pytest.mark.gpu
lib = pytest.importorskip("paper_2407_07411_gb300")


@pytest.mark.parametrize("name,D", [("tiny", 40), ("mid", 500), ("mid", 40000), ("precision", 20000)])
def test_matches_oracle(name, D):
    # precision's wave function (its operators cut to 4 terms: the blocks are the same)
    # has blocks of up to 260 x 260, above the 64 KB limit of the one-CTA kernel: both
    # kernels run
    import torch
    p = S.generate(name, n_terms=4 if name == "precision" else None)
    h = lib.HEff.from_problem(p, plan_only=False)
    psi = p.random_vectors(1)[0]
    r = h.svd_truncate(torch.from_numpy(psi).cuda(), D)
    blk = h.psi_blocks()
    ref = oracle_truncate([(int(o), int(rw), int(c)) for _, _, rw, c, o in blk], psi, D)
    smax = max(s[0] for s in ref["sv"])
    for s, t in zip(r["sv"], ref["sv"]):
        np.testing.assert_allclose(s, t, rtol=0, atol=1e-13 * smax)
    assert list(r["kept"]) == ref["kept"]
    assert abs(r["discarded"] - ref["discarded"]) <= 1e-12 * float(psi @ psi)
    U = r["U"].cpu().numpy()
    for b, (row, k) in enumerate(zip(blk, r["kept"])):
        if k == 0:
            continue
        Ug = U[r["u_off"][b]:r["u_off"][b] + int(row[2]) * k].reshape(int(row[2]), k)
        Ur = ref["U"][b]
        np.testing.assert_allclose(Ug.T @ Ug, np.eye(k), atol=1e-12)
        assert np.linalg.norm(Ug @ Ug.T - Ur @ Ur.T) <= 1e-9
    if D >= 40000:
        assert r["discarded"] <= 1e-12 and list(r["kept"]) == [int(min(b[2], b[3])) for b in blk]
