"""FP64 CPU oracle for the contour-integral sign function and overlap operator.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of Nagai & Tomiya, "Extensively parallelizable chiral
fermion" (arXiv:2204.01583), written to check the CUDA library against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the library never does, and the two share no code.

Modules
-------
gamma      chiral-basis Euclidean gamma matrices (the paper fixes none).
wilson     the hermitian Wilson-Dirac operator H_W = gamma5 D_W(-m0) (Eq. 1 and
           the sentence defining H_W after it), applied to vectors and as a dense matrix.
contour    quadrature nodes z_j and weights w_j of the elliptic contour (Eq. 7),
           the coefficient lists for sgn (Eqs. 3, 5) and the scalar rational
           function r_N they define.
sign       resolvent solves (Eq. 6), the quadrature sum (Eqs. 5, 7), the overlap
           operator (Eq. 1), the spectral sign function (Eq. 2), the quality
           measure sigma and the Ginsparg-Wilson residual (Sec. "Numerical
           experiments").
freefield  the U = 1 closed form in momentum space (exact at any lattice size).
force      gradient of Re<eta, S_N b> with respect to b and the SU(3) links
           (derivative of Eq. 4 through the resolvents).
cimpl      the same H_W and per-node CGNR resolvent solves as plain C (OpenMP over
           nodes), for lattices where dense algebra is too slow.

Parity status: every function here is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, invariants, dense LAPACK eigendecompositions, finite differences).
The paper's own sigma values (Table 1) are on a gauge ensemble that is not
available, so matching them is "parity unpinned"; the tests use the paper's contour
on synthetic fields instead.
"""
