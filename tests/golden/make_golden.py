"""Writes tests/golden/synth_digests.json: structure and full byte digests of the
seeded workloads, their oracle plan flop totals and the oracle ground-state energies
of the mid workloads (U(1) and spin-adapted).  Calls only dmrg_synth and
oracle; run from the repository root:  python tests/golden/make_golden.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import dmrg_synth as S  # noqa: E402
from dmrg_synth import su2 as G  # noqa: E402
from oracle import davidson, heff  # noqa: E402
from oracle import su2 as O  # noqa: E402

out = {}
for name in ("tiny", "mid"):
    p = S.generate(name, seed=0)
    plan = heff.plan(p)
    out[name] = dict(structure_sha256=p.structure_digest(), sha256=p.digest(), dim=p.dim, n_terms=p.n_terms,
                     op_len=int(p.op_data.size), plan_items=int(len(plan)),
                     plan_flops=int(plan[:, 4].sum()))
    if name == "mid":
        # converged lowest eigenvalue (residual <= 1e-10, so the eigenvalue error is
        # ~||r||^2 / gap, far below 1e-12 relative)
        r = davidson.davidson(lambda V: heff.apply(p, V), heff.diagonal(p), p.random_vectors(1),
                              tol=1e-10, max_iter=600)
        assert r["converged"]
        out[name]["e0"] = float(r["evals"][0])
        out[name]["e0_residual"] = float(r["resid"][0])
for name in ("su2_tiny", "su2_mid"):
    p = G.generate(name, seed=0)
    plan = O.plan(p)
    out[name] = dict(sha256=p.digest(), dim=p.dim, n_terms=p.n_terms, op_len=int(p.op_data.size),
                     plan_items=int(len(plan)), plan_flops=int(plan[:, 4].sum()))
    if name == "su2_mid":   # converged like the U(1) mid value above
        r = davidson.davidson(lambda V: O.apply(p, V), O.diagonal(p), p.random_vectors(1), tol=1e-10,
                              max_iter=600)
        assert r["converged"]
        out[name]["e0"] = float(r["evals"][0])
        out[name]["e0_residual"] = float(r["resid"][0])
json.dump(out, open(os.path.join(ROOT, "tests", "golden", "synth_digests.json"), "w"), indent=1)
print(json.dumps(out, indent=1))
