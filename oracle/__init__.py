"""CPU oracle for the exact-diagonalization hot path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, FP64 restatement of what the method computes.
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path (the CUDA library and its Python
binding) never does, and fails loudly when its extension is missing.

Modules
-------
``fock``      Fock basis of a sector (Sec. 2.3, Sec. 6.3), fermionic signs
              (Sec. 2.3), per-spin hopping matrices, the diagonal and the
              sector Hamiltonian split of Eq. Hdecomp / Eq. Hbuild (Sec. 2.4),
              the factorised product of Sec. 3.2 without MPI, and the
              non-factorisable part H_nd of Eq. Ham1 (spin exchange J_X,
              pair hopping J_P) applied term by term to every basis state.
``fullfock``  Independent checkers: the whole Fock space built from
              Jordan-Wigner operator matrices (Eq. Ham1, Ns <= 6) and a
              sector Hamiltonian built state by state with the full mode
              ordering (no spin factorisation).
``lanczos``   Plain Lanczos without re-orthogonalisation (Sec. 6.6), the
              lowest eigenpair of the tridiagonal matrix by Sturm bisection and
              inverse iteration, the second pass for the ground-state vector
              and an FP64 Rayleigh-quotient polish.
``gf``        Impurity Green's function from c^+|gs> and c|gs> Lanczos chains
              and continued fractions (Sec. 6.8, Eq. KLgf) at Matsubara or
              arbitrary complex frequencies (the real axis), plus the exact
              Lehmann sum from dense eigenvectors for small sectors.
``observables`` The non-interacting impurity function of the normal bath, the
              self-energy by the Dyson equation, the Hartree limit of the
              self-energy, and local densities, density-density correlators
              and the interaction energy of a ground state (Sec. 6.8, App. B).

``eph``       The electron-phonon (Holstein) extension of Sec. 4: the coupled
              sector of Eq. HephBuild with the phonon index slowest (Eq.
              Vdecomp2), its product slice by slice, c / c^+ on every phonon
              slice and the T = 0 Green's function from chains.

``thermal``   Several low-lying states of a sector (ARPACK on the sector
              operator, Sec. 5), the eigenspace list with the annealing
              truncation of Sec. 6.2, the finite-temperature Green's function
              as the Boltzmann-weighted sum of per-state chains (App. A), and
              the exact finite-temperature Lehmann sum for pins.

``chi``       Spin, charge and s-wave pair susceptibilities at T = 0 (Sec. 6.8,
              Eq. KLgf with the bosonic sign) from two Lanczos chains, and the
              exact Lehmann sum for small sectors.

Every function cites the passage of the paper it follows.  Pins (tests under
``tests/test_oracle_*.py``) tie each function to something other than itself:
binomial dimensions, brute force, closed forms and symmetry invariants.
Parity unpinned: the individual Lanczos coefficients after loss of
orthogonality (rounding dependent); only E0, G(i w_n) and residuals are
compared.
"""
