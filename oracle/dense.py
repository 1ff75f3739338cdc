"""Dense expansion of HODLR and HSS generators.  Test infrastructure.

HODLR (Def. 2.2; ``hodlr`` class of Sec. 2.1): the leaves hold the dense
diagonal blocks ``A(I_i^p, I_i^p) = D_i``; every internal node q with
children a (left) and b (right) holds the two sibling blocks
``A(I_a, I_b) = U12_q V12_q^T`` and ``A(I_b, I_a) = U21_q V21_q^T``.

HSS (Sec. 2.2, Eq. 2.2, Def. 2.3; ``hss`` class): the leaf bases U_i, V_i are
given; a non-root internal node q gets
``U_q = blkdiag(U_a, U_b) R_{U,q}`` and ``V_q = blkdiag(V_a, V_b) R_{V,q}``
with ``R_{U,q} = [Rl; Rr]`` and ``R_{V,q} = [Wl; Wr]``; sibling blocks are
``A(I_a, I_b) = U_a B12_q V_b^T`` and ``A(I_b, I_a) = U_b B21_q V_a^T`` on every
level 1..p; the leaves hold D_i.  ``^*`` is read as ``^T`` (real data).
"""

import numpy as np

from . import tree as T


def hodlr_dense(c, g):
    p = T.depth(c)
    L = 1 << p
    n = int(c[-1])
    A = np.zeros((n, n))
    for i in range(L):
        a, b = T.leaf_range(c, i)
        A[a:b, a:b] = g["D"][i]
    for q in range(L - 1):
        lvl, j = T.level_pos(q)
        a1, b1 = T.node_range(c, lvl + 1, 2 * j)
        a2, b2 = T.node_range(c, lvl + 1, 2 * j + 1)
        A[a1:b1, a2:b2] = g["U12"][q] @ g["V12"][q].T
        A[a2:b2, a1:b1] = g["U21"][q] @ g["V21"][q].T
    return A


def hss_bases(c, g):
    """Explicit U_q, V_q for every non-root node q (Eq. 2.2, applied bottom-up)."""
    p = T.depth(c)
    L = 1 << p
    Ub, Vb = {}, {}
    for i in range(L):
        Ub[L - 1 + i] = np.asarray(g["U"][i], dtype=np.float64)
        Vb[L - 1 + i] = np.asarray(g["V"][i], dtype=np.float64)
    for lvl in range(p - 1, 0, -1):
        for j in range(1 << lvl):
            q = T.node_id(lvl, j)
            a, b = T.children(q)
            Ub[q] = _blkdiag(Ub[a], Ub[b]) @ g["RU"][q]
            Vb[q] = _blkdiag(Vb[a], Vb[b]) @ g["RV"][q]
    return Ub, Vb


def _blkdiag(X, Y):
    out = np.zeros((X.shape[0] + Y.shape[0], X.shape[1] + Y.shape[1]))
    out[:X.shape[0], :X.shape[1]] = X
    out[X.shape[0]:, X.shape[1]:] = Y
    return out


def hss_dense(c, g):
    p = T.depth(c)
    L = 1 << p
    n = int(c[-1])
    A = np.zeros((n, n))
    for i in range(L):
        a, b = T.leaf_range(c, i)
        A[a:b, a:b] = g["D"][i]
    Ub, Vb = hss_bases(c, g)
    for q in range(L - 1):
        lvl, j = T.level_pos(q)
        la, lb = T.children(q)
        a1, b1 = T.node_range(c, lvl + 1, 2 * j)
        a2, b2 = T.node_range(c, lvl + 1, 2 * j + 1)
        A[a1:b1, a2:b2] = Ub[la] @ g["B12"][q] @ Vb[lb].T
        A[a2:b2, a1:b1] = Ub[lb] @ g["B21"][q] @ Vb[la].T
    return A


def dense(c, g):
    return hodlr_dense(c, g) if g["kind"] == "hodlr" else hss_dense(c, g)


def leaf_rowblock(c, g, i, hss_cache=None):
    """A(I_i^p, :) assembled from the generators without forming all of A.

    For each level l = 1..p the leaf's ancestor a at level l and its sibling b
    (children of q) contribute the sibling block restricted to the leaf's rows.
    """
    n = int(c[-1])
    a0, b0 = T.leaf_range(c, i)
    out = np.zeros((b0 - a0, n))
    out[:, a0:b0] = g["D"][i]
    if g["kind"] == "hss":
        Ub, Vb = hss_cache if hss_cache is not None else hss_bases(c, g)
    for (anc, sib, q) in T.ancestors(c, i):
        lvl, j = T.level_pos(anc)
        sa, _ = T.node_range(c, lvl, j)
        sl, sj = T.level_pos(sib)
        s0, s1 = T.node_range(c, sl, sj)
        rows = slice(a0 - sa, b0 - sa)
        is_left = anc % 2 == 1
        if g["kind"] == "hodlr":
            if is_left:
                out[:, s0:s1] = g["U12"][q][rows] @ g["V12"][q].T
            else:
                out[:, s0:s1] = g["U21"][q][rows] @ g["V21"][q].T
        else:
            S = g["B12"][q] if is_left else g["B21"][q]
            out[:, s0:s1] = Ub[anc][rows] @ S @ Vb[sib].T
    return out


def rows(c, g, idx, hss_cache=None):
    """A(idx, :) for a list of 0-based row indices (each row from its leaf row block)."""
    import bisect
    idx = [int(v) for v in idx]
    n = int(c[-1])
    out = np.zeros((len(idx), n))
    if g["kind"] == "hss" and hss_cache is None:
        hss_cache = hss_bases(c, g)
    by_leaf = {}
    for pos, r in enumerate(idx):
        if not 0 <= r < n:
            raise IndexError(r)
        leaf = bisect.bisect_right([int(v) for v in c], r)
        by_leaf.setdefault(leaf, []).append(pos)
    for leaf, poss in by_leaf.items():
        a0, _ = T.leaf_range(c, leaf)
        blk = _leaf_rows_subset(c, g, leaf, [idx[p_] - a0 for p_ in poss], hss_cache)
        out[poss] = blk
    return out


def _leaf_rows_subset(c, g, i, local_rows, hss_cache):
    n = int(c[-1])
    a0, b0 = T.leaf_range(c, i)
    lr = np.asarray(local_rows, dtype=np.int64)
    out = np.zeros((len(lr), n))
    out[:, a0:b0] = np.asarray(g["D"][i])[lr]
    if g["kind"] == "hss":
        Ub, Vb = hss_cache
    for (anc, sib, q) in T.ancestors(c, i):
        lvl, j = T.level_pos(anc)
        sa, _ = T.node_range(c, lvl, j)
        sl, sj = T.level_pos(sib)
        s0, s1 = T.node_range(c, sl, sj)
        rr = lr + (a0 - sa)
        is_left = anc % 2 == 1
        if g["kind"] == "hodlr":
            if is_left:
                out[:, s0:s1] = g["U12"][q][rr] @ g["V12"][q].T
            else:
                out[:, s0:s1] = g["U21"][q][rr] @ g["V21"][q].T
        else:
            S = g["B12"][q] if is_left else g["B21"][q]
            out[:, s0:s1] = Ub[anc][rr] @ S @ Vb[sib].T
    return out
