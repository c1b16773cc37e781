"""Oracle: a plain, slow, FP64 CPU restatement of the POLFED hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
execute anything in this package.  The CUDA product path never imports it, and
this package never imports the CUDA path: the two share nothing except the
seeded input generators in ``pf_inputs`` (random draws only, no arithmetic of
the method).

Each function cites the passage of the paper (arXiv 2605.10191, "Computing
eigenpairs of quantum many-body systems with Polfed.jl") it restates:

  basis.py        Hilbert-space bases (Sec. 2 intro, App. A, Eq. qsun)
  hamiltonian.py  CSR Hamiltonians: XXZ (Eq. xxz), quantum sun (Eq. qsun),
                  Fermi-Hubbard (not in the paper; conventions documented there)
  chebyshev.py    rescaling (Eq. rescaledMatrix), delta filter (Eq. transformation,
                  Eq. transformationCoefficients), Clenshaw (Eq. clenshaw_chebyshev_prod)
  dos.py          Gaussian DOS (Eq. dos_gaussian), window (Eq. Nev), K (Eq. K_approx,
                  Eq. condition_for_K), expected Krylov dimension (Sec. 5.5)
  dense.py        dense reference spectra: LAPACK eigh, cyclic Jacobi, closed forms
  lanczos.py      plain Lanczos (Eq. lanczos_recurrence) and POLFED block Lanczos
                  (Sec. 2.2, Sec. 4.3, Eq. blocklan_criterion, Sec. 4.6 workflow)

Parity status: every function is pinned by tests in tests/test_oracle_*.py
against closed forms, invariants, brute force or values the paper prints,
except the completeness of the eigenpair set at dimensions where dense
diagonalisation is infeasible (parity unpinned there; see polfed()).
"""
