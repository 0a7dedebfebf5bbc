"""Plain, slow FP64 CPU oracle for the SQ3 hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import anything from this package; the
product (the CUDA library and its Python binding) never does, and shares no
code with it.

What it computes, and where the paper defines it:

* ``fd``          -- 12th-order central finite-difference Laplacian on a
                     periodic grid (Sec. 5, simulation setup).
* ``hamiltonian`` -- H = -1/2 Lap + V + sum_J sum_lm gamma_Jl |c><c|
                     (Sec. 2, Eq. (KSeqn) and Eq. (nonlocaloperator)).
* ``fermi``       -- Fermi-Dirac occupations, Fermi level from 2 Tr D = Ne,
                     rho = 2 D(x, x), band and entropy energies
                     (Sec. 2, Eq. (TraceD), (rhoDensMat), (ON:FreeEnergy)) by
                     exact diagonalisation: the plain definition the method
                     converges to.
* ``chebyshev``   -- Chebyshev coefficients c_j, d_j, e_j (Sec. 4,
                     Eq. (ChebyshevCoeff) and the band/entropy expansions),
                     the Fermi-operator expansion of the density kernel in the
                     paper's order (Eq. (ChebyshevExpansion), (DMCFinal),
                     (ThreeTermRecurrenceRelation), (FermiLevelCalc)), and the
                     Chebyshev filter p_m(H) X by its plain definition.
* ``subspace``    -- orthonormalisation by Cholesky QR, Hs = X^T H X
                     (Sec. 3, Eq. (DsHsRelation)), and rho from the kernel
                     (Eq. (phi_tilde), Eq. (density:NewForm)).
* ``scf``         -- the self-consistent loop around the fixed-potential
                     iteration: Gaussian pseudocharges and the FD Poisson
                     equation (Sec. 2, Eq. (poisson)), the LDA, Kerker-
                     preconditioned periodic Pulay mixing (cited in Sec. 5)
                     and the free energy (Eq. (ON:FreeEnergy),
                     Eq. (FreeEnergy:NewForm)).
* ``forces``      -- Hellmann-Feynman forces on the nuclei, Eq. (force:NewForm)
                     (Sec. 3; Eq. (ON:forces) in Sec. 2): the pseudocharge
                     term and the nonlocal term in the paper's form.
* ``degree``      -- the minimal Chebyshev degree of the Fermi-operator
                     expansion for a tolerance on the occupations, by brute
                     force over the Fermi level (Sec. 4; the trend with
                     temperature in Sec. 5).
* ``guess``       -- starting densities for the SCF: uniform, atomic
                     superposition, and a small learned model (not in the
                     paper; the comparison the learned guess is built for).
* ``qmd``         -- velocity-Verlet dynamics of the nuclei on those forces,
                     with the isokinetic option of the paper's QMD (Sec. 5).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, library routines or brute force; none is marked "parity
unpinned".
"""
