"""The fast products of Fig. 4.1, in the paper's order.  Test infrastructure.

These are not the reference the CUDA path is compared with (that is the dense
definition in ``matmat``).  They exist to pin one reading: the printed HSS
coupling loop runs over levels 1..p-1, which leaves the sibling leaves
uncoupled; the definition (Def. 2.3, every sibling pair on levels 1..p) needs
levels 1..p.  ``hss_matvec(..., couple_to=p)`` is the reading we use and
``couple_to=p-1`` is the loop as printed; the tests show that only the former
equals the dense product.
"""

import numpy as np

from . import tree as T


def hodlr_matvec(c, g, X):
    """Recursive HODLR product (Fig. 4.1, left)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    p = T.depth(c)
    L = 1 << p

    def rec(q):
        lvl, j = T.level_pos(q)
        a, b = T.node_range(c, lvl, j)
        if lvl == p:
            return np.asarray(g["D"][q - (L - 1)]) @ X[a:b]
        la, lb = T.children(q)
        a1, b1 = T.node_range(c, lvl + 1, 2 * j)
        a2, b2 = T.node_range(c, lvl + 1, 2 * j + 1)
        y1 = rec(la)
        y2 = g["U12"][q] @ (g["V12"][q].T @ X[a2:b2])
        y3 = g["U21"][q] @ (g["V21"][q].T @ X[a1:b1])
        y4 = rec(lb)
        return np.vstack([y1 + y2, y3 + y4])

    return rec(0)


def hss_matvec(c, g, X, couple_to=None):
    """Four-step HSS product (Fig. 4.1, right) with the coupling loop over 1..couple_to."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    p = T.depth(c)
    L = 1 << p
    if couple_to is None:
        couple_to = p
    v = {}
    d = {}
    for i in range(L):
        a, b = T.leaf_range(c, i)
        v[L - 1 + i] = np.asarray(g["V"][i]).T @ X[a:b]
        d[i] = np.asarray(g["D"][i]) @ X[a:b]
    for lvl in range(p - 1, 0, -1):          # upsweep
        for j in range(1 << lvl):
            q = T.node_id(lvl, j)
            a, b = T.children(q)
            v[q] = g["RV"][q].T @ np.vstack([v[a], v[b]])
    # Couplings.  Read as two arrays (x-hat from the upsweep, y-hat here): a node
    # that no coupling reaches has y-hat = 0.  The printed loop overwrites v in
    # place, so a level it skips keeps its x-hat; ``couple_to < p`` models that.
    xh = v
    v = {q: (xh[q] if couple_to < p else np.zeros_like(xh[q])) for q in xh}
    for lvl in range(1, couple_to + 1):
        for j in range(1 << (lvl - 1)):
            q = T.node_id(lvl - 1, j)
            a, b = T.children(q)
            v[a] = g["B12"][q] @ xh[b]
            v[b] = g["B21"][q] @ xh[a]
    for lvl in range(1, p):                  # downsweep
        for j in range(1 << lvl):
            q = T.node_id(lvl, j)
            a, b = T.children(q)
            t = g["RU"][q] @ v[q]
            ka = v[a].shape[0]
            v[a] = v[a] + t[:ka]
            v[b] = v[b] + t[ka:]
    out = []
    for i in range(L):
        out.append(np.asarray(g["U"][i]) @ v[L - 1 + i] + d[i])
    return np.vstack(out)
