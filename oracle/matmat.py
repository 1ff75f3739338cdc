"""Y = A X by the plain definition, streamed per leaf row block.  Test infrastructure.

``A`` is never formed whole: each leaf row block ``A(I_i^p, :)`` is assembled
from the generators (``dense.leaf_rowblock``) and multiplied by X with a
float64 BLAS matmul (the one library primitive used).  Memory is O(m n).
"""

import numpy as np

from . import dense, tree as T


def matmat(c, g, X):
    """Y = A X for an n x r float64 block X (any memory order)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    n = int(c[-1])
    if X.shape[0] != n:
        raise ValueError("X must have n rows")
    p = T.depth(c)
    Y = np.zeros((n, X.shape[1]), order="F")
    cache = dense.hss_bases(c, g) if g["kind"] == "hss" else None
    for i in range(1 << p):
        a, b = T.leaf_range(c, i)
        if b > a:
            Y[a:b] = dense.leaf_rowblock(c, g, i, cache) @ X
    return Y


def matmat_rows(c, g, X, idx):
    """Rows ``idx`` of A X, each computed from the explicit row A(idx, :)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    return dense.rows(c, g, idx) @ X


def matmat_leaves(c, g, X, leaves):
    """Y restricted to the rows of the given leaves (used for bounded CPU samples)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    cache = dense.hss_bases(c, g) if g["kind"] == "hss" else None
    out = []
    for i in leaves:
        out.append(dense.leaf_rowblock(c, g, i, cache) @ X)
    return out
