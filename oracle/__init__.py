"""Plain FP64 CPU oracle for the null-space-free Maxwell eigenproblem.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import anything from this package.  The
product path (the CUDA library and its Python binding) never imports it and
shares no code with it.

Every function follows the paper (Huang, Li, Li, Lin, Lin, Tian, "Eigenvalue
problems of discrete curl operators on various lattices for simulating three
dimensional photonic crystals", arXiv:1806.10284) and names the section,
equation, theorem or algorithm it restates.  It is written to be read against
the paper, not to be fast: numpy FFTs and scipy sparse/dense linear algebra are
the only library steps.

Modules
-------
lattice   Section 2.2: canonical ordering, grid offsets m1, m2, m3 with the
          angle correction, eq. (transvec), the index-shift lattice.
curl      Section 3: the Yee curl C and gradient G assembled by quasi-periodic
          index wrapping (Theorems period1-period3), plus the paper's printed
          K1, K2/J2 and K3/J3 forms (eqs. K1, K2, J2, J1, acuteJ3, obtuseJ3).
spectral  Section 4: the twist phases, Lambda_1..3, the unitary T, and the
          FFT matvecs T q (Algorithm 5.2) and T^* p (Algorithm 5.1).
nfsep     Section 5.1-5.2: Pi_0, Pi_1, Pi_2, Sigma_r, the reduced operator
          A_r (eq. NFSEP), its dense form, and the dense GEP (eq. GEP).
eigs      A plain FP64 block LOBPCG (Knyazev 2001) and dense eigensolves of
          A_r for the few smallest eigenvalues.
grad      Hellmann-Feynman eps-gradient of the eigenvalues through B^{-1}.

Parity status: every function is pinned by a ``-m "not gpu"`` test under
``tests/test_oracle_*.py``; none is "parity unpinned".
"""
