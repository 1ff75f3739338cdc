"""CPU oracle for the HODLR/HSS matrix-times-block product (TEST INFRASTRUCTURE).

This package is test infrastructure only.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it; the library under
``paper_1909_07909_gb300/`` never does, and it shares no code with it.

What it computes.  The fast product of Sec. 4.1 reaches exactly (up to the
order of rounding) ``Y = A X`` with ``A`` the dense matrix the generators
define, so the oracle is that definition written out in float64:

* ``tree``     -- cluster trees (Def. 2.1) from the leaf-end vector ``c``
                  (Sec. 3.7) or the default ceil(n/2) split (Sec. 3.1).
* ``dense``    -- dense expansion of HODLR generators (Def. 2.2 and the
                  ``hodlr`` class of Sec. 2.1) and of HSS generators (nested
                  bases of Eq. 2.2, core blocks of Sec. 2.2, Def. 2.3).
* ``matmat``   -- ``Y = A X`` streamed one leaf row block at a time (a BLAS
                  matmul is the only library primitive used), plus sampled rows
                  for sizes whose dense matrix does not fit in memory.
* ``expkernel``-- exact product with the exponential kernel by its O(nK)
                  two-pass recurrence (full-vector reference at any n).
* ``bounds``   -- the componentwise forward-error envelope
                  ``|D||X| + sum |U|(|V|^T |X|)`` (HSS: with |R| and |S|).
* ``transpose``-- generators of A^T by the block definition
                  (A^T)(I, J) = A(J, I)^T and the product Y = A^T X.
* ``convert``  -- hss2hodlr (Sec. 3.5): HODLR generators of an HSS matrix from
                  its explicit nested bases.
* ``hadamard`` -- generators of A o B (Sec. 4.4, Eq. 4.1, Fig. 4.3): transpose
                  Khatri-Rao factors, Kronecker couplings and translations.
* ``solve``    -- Y = A^{-1} B by a dense LU solve of the defining matrix
                  (Sec. 4.3), and the backward error of a candidate solution.
* ``fig41``    -- the recursive HODLR product and the four-step HSS product of
                  Fig. 4.1, kept only to show which reading of the printed
                  coupling loop agrees with the definition.

Every function is pinned by ``tests/test_oracle_*.py`` against brute force,
closed forms and exact-rank fixtures; none is "parity unpinned".
"""

from . import tree, dense, matmat, expkernel, bounds, fig41, transpose, convert, hadamard, solve  # noqa: F401
