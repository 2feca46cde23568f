"""Oracle pins against textbook models with known spectra.

Each model is written as a two-block problem (left block (x) right block) with
explicit terms c_t (A_t (x) B_t) P_t, P_t the fermion-parity sign of the input
left block for odd Delta_n.  The expected values come from closed forms or from
exact diagonalisation in the full Fock space, never from the oracle itself.
Together the models use every shift of the term set: Delta = (0,0), (+-1,+-1),
(0,+-2) and (+-2,0)."""
import numpy as np
import pytest

import dmrg_synth as S
from oracle import davidson, heff
from tests.fermions import Block, full_fock_hubbard_chain


def _spectrum(p):
    return np.linalg.eigvalsh(heff.dense_h(p))


def test_heisenberg_dimer_closed_form():
    # J S1.S2 on two spin-1/2 sites: singlet -3J/4, triplet +J/4.  Each block is
    # one singly occupied site: sectors (1,-1), (1,1).
    J = 1.7
    tab = np.array([(1, -1, 1), (1, 1, 1)], np.int32)
    one = np.ones((1, 1))
    sz = {0: -0.5 * one, 1: 0.5 * one}
    terms = [
        (J, (0, 0), 0, sz, sz),
        (J / 2, (0, 2), 0, {0: one}, {1: one}),      # S+ (x) S-
        (J / 2, (0, -2), 0, {1: one}, {0: one}),     # S- (x) S+
    ]
    p = S.assemble(tab, tab, (2, 0), terms)
    assert p.dim == 2
    np.testing.assert_allclose(_spectrum(p), [-0.75 * J, 0.25 * J], rtol=0, atol=1e-14)


def test_eta_pairing_dimer_closed_form():
    # J eta1.eta2 with eta+ = c+_up c+_dn: the same SU(2) algebra on the empty /
    # doubly occupied states, so the spectrum is again -3J/4 and +J/4.
    J = 0.9
    tab = np.array([(0, 0, 1), (2, 0, 1)], np.int32)
    one = np.ones((1, 1))
    ez = {0: -0.5 * one, 1: 0.5 * one}
    terms = [
        (J, (0, 0), 0, ez, ez),
        (J / 2, (2, 0), 0, {0: one}, {1: one}),
        (J / 2, (-2, 0), 0, {1: one}, {0: one}),
    ]
    p = S.assemble(tab, tab, (2, 0), terms)
    np.testing.assert_allclose(_spectrum(p), [-0.75 * J, 0.25 * J], rtol=0, atol=1e-14)


def _hubbard_two_block(L: int, t: float, U: float, target):
    """Open Hubbard chain of 2L sites split into two blocks of L sites.
    Boundary hopping -t (c+_L c_R1 + c+_R1 c_L) becomes, per spin,
    -t (c+_L (x) c_R1) P and +t (c_L (x) c+_R1) P."""
    B = Block(L)
    I = np.eye(1 << B.nm)
    H = B.hubbard(t, U)
    terms = [(1.0, (0, 0), 0, B.blocks(H, (0, 0)), B.blocks(I, (0, 0))),
             (1.0, (0, 0), 0, B.blocks(I, (0, 0)), B.blocks(H, (0, 0)))]
    for sp, dsz in ((0, 1), (1, -1)):
        cl, cr = B.c(L - 1, sp), B.c(0, sp)
        terms.append((-t, (1, dsz), 1, B.blocks(cl.T, (1, dsz)), B.blocks(cr, (-1, -dsz))))
        terms.append((t, (-1, -dsz), 1, B.blocks(cl, (-1, -dsz)), B.blocks(cr.T, (1, dsz))))
    return S.assemble(B.table, B.table, target, terms)


@pytest.mark.parametrize("U", [0.0, 2.5, 8.0])
def test_hubbard_dimer_closed_form(U):
    t = 1.3
    p = _hubbard_two_block(1, t, U, (2, 0))
    e0 = (U - np.sqrt(U * U + 16 * t * t)) / 2
    assert abs(_spectrum(p)[0] - e0) < 1e-13


def test_free_fermion_chain_closed_form():
    # 6-site open tight-binding chain (3 + 3 sites, D = 64 per block) at half
    # filling, S_z = 0: E0 = 2 * sum of the three lowest -2t cos(k pi / 7).
    t = 1.0
    p = _hubbard_two_block(3, t, 0.0, (6, 0))
    eps = np.sort(-2 * t * np.cos(np.arange(1, 7) * np.pi / 7))
    e0 = 2 * eps[:3].sum()
    assert abs(_spectrum(p)[0] - e0) < 1e-12
    # the same through the oracle Davidson
    r = davidson.davidson(lambda V: heff.apply(p, V), heff.diagonal(p),
                          p.random_vectors(1), tol=1e-10, max_iter=300)
    assert r["converged"] and abs(r["evals"][0] - e0) < 1e-12


@pytest.mark.parametrize("target", [(4, 0), (3, 1), (5, -1)])
def test_hubbard_chain_matches_full_fock_ed(target):
    # 2 + 2 sites, interacting: the two-block spectrum equals the full-space
    # exact diagonalisation with global Jordan-Wigner strings in that sector.
    t, U = 1.0, 4.0
    p = _hubbard_two_block(2, t, U, target)
    ref = full_fock_hubbard_chain(4, t, U, *target)
    np.testing.assert_allclose(_spectrum(p), ref, rtol=0, atol=1e-12)
