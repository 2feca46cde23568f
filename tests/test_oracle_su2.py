"""Pins of the spin-adapted oracle (oracle/su2.py) to things other than itself:
Clebsch-Gordan coefficients against sympy and their orthonormality and textbook
values; the Heisenberg dimer S_L . S_R, whose energies are the closed form
[J(J+1) - j_L(j_L+1) - j_R(j_R+1)] / 2; the full operator with every magnetic
sublevel, assembled from the reduced blocks by Wigner-Eckart, which must commute
with the total spin (built from the ladder formula alone) and reproduce the reduced
operator on the coupled states; the reduction to the U(1) oracle when every spin is
0; symmetry and linearity; the truncation weights against the density matrix of the
full state."""
import itertools
import math

import numpy as np
import pytest

from dmrg_synth import su2 as G
from dmrg_synth import assemble
from oracle import heff
from oracle import su2 as O


def test_cg_textbook_values():
    h = 1 / math.sqrt(2)
    assert O.cg(1, 1, 1, -1, 0, 0) == pytest.approx(h, abs=1e-15)
    assert O.cg(1, -1, 1, 1, 0, 0) == pytest.approx(-h, abs=1e-15)
    assert O.cg(1, 1, 1, -1, 2, 0) == pytest.approx(h, abs=1e-15)
    assert O.cg(1, 1, 1, 1, 2, 2) == pytest.approx(1.0, abs=1e-15)
    # <j m; 1 0 | j m> = m / sqrt(j(j+1))
    for j2 in range(1, 7):
        j = j2 / 2
        for m2 in range(-j2, j2 + 1, 2):
            assert O.cg(j2, m2, 2, 0, j2, m2) == pytest.approx((m2 / 2) / math.sqrt(j * (j + 1)), abs=1e-14)


def test_cg_against_sympy():
    wig = pytest.importorskip("sympy.physics.wigner")
    from sympy import Rational
    for j1, j2 in itertools.product(range(0, 5), range(0, 5)):
        for J in range(abs(j1 - j2), j1 + j2 + 1, 2):
            for m1, m2 in itertools.product(range(-j1, j1 + 1, 2), range(-j2, j2 + 1, 2)):
                M = m1 + m2
                if abs(M) > J:
                    continue
                ref = float(wig.clebsch_gordan(Rational(j1, 2), Rational(j2, 2), Rational(J, 2),
                                               Rational(m1, 2), Rational(m2, 2), Rational(M, 2)))
                assert O.cg(j1, m1, j2, m2, J, M) == pytest.approx(ref, abs=1e-14)


def test_cg_orthonormal():
    for j1, j2 in itertools.product(range(0, 6), range(0, 6)):
        Js = list(range(abs(j1 - j2), j1 + j2 + 1, 2))
        for M in range(-(j1 + j2), j1 + j2 + 1, 2):
            pairs = [(m1, M - m1) for m1 in range(-j1, j1 + 1, 2) if abs(M - m1) <= j2]
            C = np.array([[O.cg(j1, m1, j2, m2, J, M) for J in Js] for m1, m2 in pairs])
            C = C[:, [k for k, J in enumerate(Js) if abs(M) <= J]]
            np.testing.assert_allclose(C.T @ C, np.eye(C.shape[1]), atol=1e-14)
            np.testing.assert_allclose(C @ C.T, np.eye(C.shape[0]), atol=1e-14)


def test_recoupling_rank0_is_identity():
    for sl, sr in itertools.product(range(0, 7), range(0, 7)):
        for s in range(abs(sl - sr), sl + sr + 1, 2):
            assert O.recoupling(sl, sr, sl, sr, 0, s) == pytest.approx(1.0, abs=1e-14)
    assert O.recoupling(2, 2, 2, 2, 0, 6) == 0.0   # (1, 1, 3) is no triangle


def _dimer(jl2, jr2, s2):
    """S_L . S_R of two multiplets (one each), coupled to total spin s2/2.  The
    reduced block of the spin vector is sqrt(j(j+1)); the scalar coupling
    sum_mu (-1)^{1-mu} T_mu U_-mu is -T.U, hence the coefficient -1."""
    left = [(1, jl2, 1)]
    right = [(1, jr2, 1)]
    a = np.array([[math.sqrt(jl2 / 2 * (jl2 / 2 + 1))]])
    b = np.array([[math.sqrt(jr2 / 2 * (jr2 / 2 + 1))]])
    return G.pack(left, right, (2, s2), [(-1.0, 2, 0, 0, {(0, 0): a}, {(0, 0): b})])


@pytest.mark.parametrize("jl2,jr2", [(1, 1), (2, 2), (1, 2), (3, 2), (4, 3)])
def test_heisenberg_dimer_closed_form(jl2, jr2):
    jl, jr = jl2 / 2, jr2 / 2
    for s2 in range(abs(jl2 - jr2), jl2 + jr2 + 1, 2):
        p = _dimer(jl2, jr2, s2)
        assert p.dim == 1
        J = s2 / 2
        e = (J * (J + 1) - jl * (jl + 1) - jr * (jr + 1)) / 2
        assert O.apply(p, np.ones(1))[0] == pytest.approx(e, abs=1e-14)
        assert O.diagonal(p)[0] == pytest.approx(e, abs=1e-14)


@pytest.fixture(scope="module", params=[(6, 2), (6, 0), (5, 1)], ids=["triplet", "singlet", "doublet"])
def tiny_full(request):
    p = G.generate("su2_tiny", target=request.param)
    return p, O.full_space(p), O.apply(p, np.eye(p.dim)).T


def test_full_operator_is_spin_invariant(tiny_full):
    p, F, _ = tiny_full
    H, Sz, Sp = F["H"], F["Sz"], F["Sp"]
    assert np.abs(H).max() > 0.1
    np.testing.assert_allclose(H, H.T, atol=1e-14)
    np.testing.assert_allclose(H @ Sp, Sp @ H, atol=1e-13)
    np.testing.assert_allclose(H @ Sz, Sz @ H, atol=1e-13)


def test_coupled_states_are_highest_weight(tiny_full):
    p, F, _ = tiny_full
    E = F["E"]
    np.testing.assert_allclose(E.T @ E, np.eye(p.dim), atol=1e-14)
    np.testing.assert_allclose(F["Sp"] @ E, 0.0, atol=1e-14)
    np.testing.assert_allclose(F["Sz"] @ E, (p.target[1] / 2) * E, atol=1e-14)


def test_reduced_operator_is_the_projection(tiny_full):
    p, F, Hr = tiny_full
    H, E = F["H"], F["E"]
    np.testing.assert_allclose(Hr, E.T @ H @ E, atol=1e-13)
    np.testing.assert_allclose(H @ E, E @ Hr, atol=1e-13)   # the coupled states span an invariant space
    np.testing.assert_allclose(Hr, Hr.T, atol=1e-14)
    wf = np.linalg.eigvalsh(H)
    for w in np.linalg.eigvalsh(Hr):
        assert np.abs(wf - w).min() <= 1e-12


def test_diagonal_and_entries(tiny_full):
    p, _, Hr = tiny_full
    np.testing.assert_allclose(O.diagonal(p), np.diag(Hr), atol=1e-14)
    x = p.random_vectors(1)[0]
    idx = np.arange(0, p.dim, 7)
    np.testing.assert_allclose(O.apply_entries(p, x, idx), (Hr @ x)[idx], atol=1e-13)


def test_spin_zero_reduces_to_u1():
    """With every spin 0 and rank-0 terms W = 1 and every block is a U(1) block."""
    rng = np.random.default_rng(5)
    table = [(0, 0, 2), (2, 0, 3), (4, 0, 2)]
    u1_terms, su2_terms = [], []
    for c, dn in ((0.7, 0), (-0.4, 2), (-0.4, -2), (1.1, 0)):
        ab, bb, ua, ub = {}, {}, {}, {}
        for q, (n, _, d) in enumerate(table):
            for p_, (n2, _, d2) in enumerate(table):
                if n2 == n + dn:
                    ab[(q, p_)] = rng.standard_normal((d2, d))
                    ua[q] = ab[(q, p_)]
                if n2 == n - dn:
                    bb[(q, p_)] = rng.standard_normal((d2, d))
                    ub[q] = bb[(q, p_)]
        su2_terms.append((c, 0, dn, 0, ab, bb))
        u1_terms.append((c, (dn, 0), 0, ua, ub))
    ps = G.pack(table, table, (4, 0), su2_terms)
    pu = assemble(table, table, (4, 0), u1_terms)
    assert ps.dim == pu.dim
    x = np.random.default_rng(1).standard_normal(ps.dim)
    np.testing.assert_allclose(O.apply(ps, x), heff.apply(pu, x), rtol=1e-14, atol=1e-14)


def test_symmetry_and_linearity_mid_subset():
    p = G.generate("su2_mid", n_terms=24)
    x, y = p.random_vectors(2)
    hx, hy = O.apply(p, x), O.apply(p, y)
    assert abs(x @ hy - hx @ y) <= 1e-13 * np.linalg.norm(hx) * np.linalg.norm(y)
    np.testing.assert_allclose(O.apply(p, 2.0 * x - 3.0 * y), 2.0 * hx - 3.0 * hy, rtol=1e-12, atol=1e-13)


def test_generator_is_deterministic():
    a, b = G.generate("su2_tiny"), G.generate("su2_tiny")
    assert a.digest() == b.digest()
    assert G.generate("su2_tiny", seed=1).digest() != a.digest()


def test_truncation_weights_are_the_summed_density_matrix(tiny_full):
    """Per left sector the stacked matrix M_q = [psi_b ...] satisfies
    M_q M_q^T = sum_m rho_L[(q, ., m), (q, ., m)], rho_L the left density matrix of the
    full state E psi; its squared singular values are therefore the multiplet weights."""
    p, F, _ = tiny_full
    psi = p.random_vectors(1)[0]
    full = F["E"] @ psi
    bl, br = O.m_basis(p.left), O.m_basis(p.right)
    Psi = np.zeros((len(bl), len(br)))
    Psi.ravel()[F["index"]] = full
    rho = Psi @ Psi.T
    r = O.truncate(p, psi, 10 ** 6)
    assert abs(sum(float((s ** 2).sum()) for s in r["sv"]) - 1.0) <= 1e-13
    for q, sv in zip(r["sectors"], r["sv"]):
        d = int(p.left[q][2])
        acc = np.zeros((d, d))
        for m in range(-int(p.left[q][1]), int(p.left[q][1]) + 1, 2):
            idx = [i for i, st in enumerate(bl) if st[0] == q and st[2] == m]
            acc += rho[np.ix_(idx, idx)]
        w = np.sort(np.linalg.eigvalsh(acc))[::-1][:len(sv)]
        np.testing.assert_allclose(w, sv ** 2, atol=1e-14)
    assert r["discarded"] <= 1e-12
    n_blocks = len(O.psi_blocks(p))   # S > 0: some left sectors own several blocks
    assert len(r["sectors"]) < n_blocks if p.target[1] > 0 else len(r["sectors"]) == n_blocks


def test_plan_hand_computed():
    """Two multiplet sectors per block, (n, 2S) = (1, 1) dim 2 and (1, 3) dim 1, target
    (2, 2S=2): the four sector pairs all couple to S = 1, blocks b0 = (0,0) 2x2,
    b1 = (0,1) 2x1, b2 = (1,0) 1x2, b3 = (1,1) 1x1.  Term 0 (rank 1) has only
    A[1 <- 0] (1x2) and B[1 <- 1] (1x1): one contribution b1 -> b3 with a=1, b=2, c=1,
    d=1, (A x) B^T = 2*1*2*1 + 2*1*1*1 = 6 < A (x B^T) = 8.  Term 1 (rank 0) has A[0 <- 0]
    and B[0 <- 0] (2x2): b0 -> b0, 2*8 + 2*8 = 32 either way, a tie, so A-first."""
    table = [(1, 1, 2), (1, 3, 1)]
    rng = np.random.default_rng(2)
    terms = [(0.5, 2, 0, 0, {(0, 1): rng.standard_normal((1, 2))}, {(1, 1): rng.standard_normal((1, 1))}),
             (0.3, 0, 0, 0, {(0, 0): rng.standard_normal((2, 2))}, {(0, 0): rng.standard_normal((2, 2))})]
    p = G.pack(table, table, (2, 2), terms)
    assert [(b[0], b[1], b[2], b[3], b[4]) for b in O.psi_blocks(p)] == \
        [(0, 0, 0, 2, 2), (0, 1, 4, 2, 1), (1, 0, 6, 1, 2), (1, 1, 8, 1, 1)]
    assert p.dim == 9
    np.testing.assert_array_equal(O.plan(p), np.array([[0, 1, 0, 0, 32], [3, 0, 1, 0, 6]]))
