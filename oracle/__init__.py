"""Oracle: a plain, slow, FP64 CPU statement of the SP2 density / response /
susceptibility path, written from the paper (arXiv 2409.17033).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this package. The product path (the
CUDA library and its Python binding) never imports, calls or falls back to it,
and this package imports nothing from the product path; the two share only the
seeded input generators in ``workloads``.

Contents (each function cites the passage it follows):

* ``sp2``       -- Eq. DM0 (SP2 expansion), the spectral-bound scaling and the
                   trace-based branch choice of Sec. II, Eq. DM1 (first-order
                   density-matrix response), Eq. DM2 (backward susceptibility),
                   Eq. DM3 (forward susceptibility), the merged forms of the
                   Appendix (Eq. DMSuscept, Eq. DMPert), the expectation and
                   response contractions (Eqs. expectation, direct, dual).
* ``exact``     -- the closed forms the recursion approximates: D = theta(mu I - H)
                   (Sec. II, Eq. 1) and the Daleckii-Krein / Loewner form of the
                   first-order response (Appendix, proof of Eq. Equivalence),
                   plus the same recursion carried out exactly on the
                   eigenvalues (finite-M reference).
* ``split``     -- the hi/lo half-precision splitting of Eq. doubleHalf and the
                   three-product mixed-precision multiplication of Eq. MixPrecMult
                   with the lo*lo term dropped (Eq. mults); the three-plane
                   bfloat16 split and its six-term product (tunable accuracy).
* ``fermi``     -- the finite-temperature recursion of Sec. V.B and its responses.
* ``scf``       -- the site-charge self-consistent response (Appendix, Eq.
                   DM_CP_SCF), its exact solve, mixers and the MLP.
* ``nonorth``   -- non-orthonormal representations (Sec. V.A): Loewdin factor,
                   congruences, and the dual three-contraction form of the
                   basis-set dependent derivative (Eq. NonOrthDer).
* ``sparse``    -- Eq. DM0 in blockwise thresholded sparse algebra (Sec. II's
                   remark on thresholded sparse matrix products).

Parity status: every function here is pinned by a `-m "not gpu"` test against
a closed form, an invariant, brute force or a library routine (see
``tests/test_oracle_*.py``). None is marked "parity unpinned".
"""
from . import exact, fermi, nonorth, scf, sp2, sparse, split  # noqa: F401
