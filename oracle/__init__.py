"""CPU FP64 oracle for the two-site effective-Hamiltonian product and its
Davidson eigensolver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library (``paper_2407_07411_gb300``); the two meet
only through the inputs produced by ``dmrg_synth``.

Modules
  heff     sector indexing, contraction-order planner, H_eff*psi from its
           blockwise definition, dense Kronecker H (tiny cases), diagonal of H.
  davidson block Davidson with CGS2 orthogonalisation and thick restart.
  lanczos  restarted Lanczos with full reorthogonalisation.
  ozaki    split-precision (Ozaki) slicing and the exact slice-product sum.
  svd      two-site decomposition and truncation to the D largest singular values.
  renorm   operator renormalisation O' = U_p^T O U_q in per-sector bases.
  su2      the spin-adapted form: Clebsch-Gordan coefficients, the recoupling
           coefficient from its definition, the reduced H_eff*psi, its planner and
           diagonal, the truncation per left sector, and the full operator with every
           magnetic sublevel (tiny cases).

Pins (what ties each function to something other than itself) live in
``tests/test_oracle_*.py``: dense Kronecker assembly through ``numpy.kron``,
closed-form ground-state energies of textbook models (Heisenberg, eta-pairing
and Hubbard dimers, the free-fermion chain), exact diagonalisation of a
four-site Hubbard chain in its full Fock space, ``numpy.linalg.eigh`` and
ARPACK (``scipy.sparse.linalg.eigsh``), Hermiticity, linearity, sector
conservation, hand-computed plans, exact integer arithmetic for the slices, and for
the spin-adapted form sympy's Clebsch-Gordan coefficients, the Heisenberg dimer and
the total-spin invariance of the full operator.
"""
