"""Y = A^{-1} B for a HODLR or HSS matrix A.  Test infrastructure.

The HSS solver of Sec. 4.3 (implicit ULV, Fig. 4.4-4.5; `A\\v` and `ulv(A)` in
Table 4.2) reaches exactly, up to rounding, the solution of A Y = B.  So the
oracle is that definition written out: the dense matrix A of the generators
(``dense``) and a float64 LU solve with partial pivoting (LAPACK, the one
library primitive used), for sizes whose dense matrix fits in memory.

For any size, ``residual`` gives the normwise backward error of a candidate
solution through the streamed product of ``matmat``:
``||A Y - B||_F / (||A||_F ||Y||_F + ||B||_F)``, with ||A||_F from the
generators block by block.
"""

import numpy as np

from . import dense, matmat as M, tree as T


def solve_dense(c, g, B):
    """A^{-1} B from the dense matrix (n x r float64 B)."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    A = dense.dense(c, g)
    return np.linalg.solve(A, B)


def frobenius(c, g):
    """||A||_F, summed over leaf row blocks (A is never formed whole)."""
    p = T.depth(c)
    cache = dense.hss_bases(c, g) if g["kind"] == "hss" else None
    tot = 0.0
    for i in range(1 << p):
        a, b = T.leaf_range(c, i)
        if b > a:
            tot += float(np.sum(dense.leaf_rowblock(c, g, i, cache) ** 2))
    return np.sqrt(tot)


def residual(c, g, Y, B):
    """Normwise backward error of Y as a solution of A Y = B."""
    Y = np.asarray(Y, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    if B.ndim == 1:
        B = B[:, None]
    R = M.matmat(c, g, Y) - B
    den = frobenius(c, g) * np.linalg.norm(Y) + np.linalg.norm(B)
    return float(np.linalg.norm(R) / den) if den > 0 else float(np.linalg.norm(R))
