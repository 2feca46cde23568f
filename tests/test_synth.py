"""Seeded input generator: determinism, the integer size table of the named
workloads, and the symmetry-preserving term construction."""
import json
import os

import numpy as np

import dmrg_synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Integer columns (sectors, d_min, d_max, psi blocks, psi entries) of the size
# table, computed by an independent model of the same sector reading.
SIZE_TABLE = {
    "tiny": (23, 1, 10, 23, 322),
    "mid": (51, 2, 76, 51, 39928),
    "precision": (78, 1, 260, 78, 598090),
    "large": (89, 2, 580, 89, 2381956),
}


def test_size_table():
    for name, (ns, dmin, dmax, nb, dim) in SIZE_TABLE.items():
        cfg = S.CONFIGS[name]
        tab = S.sector_table(cfg)
        assert len(tab) == ns and tab[:, 2].min() == dmin and tab[:, 2].max() == dmax
        assert int(tab[:, 2].sum()) == cfg["D"]
        assert S.wavefunction_dim(tab, tab, cfg["target"]) == dim
        tn, ts = cfg["target"]
        keys = {(int(n), int(s)) for n, s, _ in tab}
        assert sum((tn - int(n), ts - int(s)) in keys for n, s, _ in tab) == nb
        order = [(int(n), int(s)) for n, s, _ in tab]
        assert order == sorted(order) and all((s - n) % 2 == 0 for n, s in order)


def test_heavy_tailed_dims():
    tab = S.sector_table(S.CONFIGS["heavy"], seed=0)
    assert len(tab) == 78 and int(tab[:, 2].sum()) == 4096
    assert tab[:, 2].min() >= 1 and tab[:, 2].max() <= 900
    assert tab[:, 2].max() / np.median(tab[:, 2]) > 5          # heavy tail


def test_deterministic_and_pinned():
    g = json.load(open(os.path.join(GOLDEN, "synth_digests.json")))
    for name in ("tiny", "mid"):
        p1, p2 = S.generate(name), S.generate(name)
        assert p1.digest() == p2.digest()
        assert p1.structure_digest() == g[name]["structure_sha256"]
        assert p1.digest() == g[name]["sha256"]   # every value byte
        assert p1.dim == g[name]["dim"] and p1.op_data.size == g[name]["op_len"]
    assert S.generate("tiny", seed=1).digest() != S.generate("tiny", seed=0).digest()


def test_pairs_are_adjoint():
    p = S.generate("tiny")
    T = p.n_terms
    t = 0
    while t < T:
        d = tuple(int(v) for v in p.delta[t])
        if d == (0, 0):
            t += 1
            continue
        assert tuple(int(v) for v in p.delta[t + 1]) == (-d[0], -d[1])
        sign = -1.0 if d[0] % 2 else 1.0
        assert p.coef[t + 1] == sign * p.coef[t]
        assert p.parity[t] == p.parity[t + 1] == d[0] % 2
        t += 2


def test_random_vectors_unit_norm():
    p = S.generate("tiny")
    V = p.random_vectors(3)
    np.testing.assert_allclose(np.linalg.norm(V, axis=1), 1.0, rtol=1e-15)
    assert not np.array_equal(V[0], V[1])


def test_su2_pinned():
    from dmrg_synth import su2 as G
    g = json.load(open(os.path.join(GOLDEN, "synth_digests.json")))
    for name in ("su2_tiny", "su2_mid"):
        p = G.generate(name, seed=0)
        assert p.digest() == g[name]["sha256"]
        assert (p.dim, p.n_terms, p.op_data.size) == (g[name]["dim"], g[name]["n_terms"], g[name]["op_len"])
    t = G.generate("su2_mid").left
    assert len(t) == 38 and int(t[:, 2].sum()) == 1024 and int(t[:, 1].min()) >= 0
    assert all((int(s) - int(n)) % 2 == 0 for n, s, _ in t)
