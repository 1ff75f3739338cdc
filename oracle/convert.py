"""HSS to HODLR conversion (hss2hodlr, Sec. 3.5).  Test infrastructure.

An HSS matrix is also HODLR on the same cluster tree: the nested bases of
Eq. 2.2, written out explicitly for every node (``dense.hss_bases``), give the
sibling blocks of Def. 2.3 as ``A(I_a, I_b) = U_a B12_q V_b^T`` and
``A(I_b, I_a) = U_b B21_q V_a^T``.  Taking the HODLR factors (Def. 2.2)

    U12_q = U_a B12_q,  V12_q = V_b,  U21_q = U_b B21_q,  V21_q = V_a

reproduces every block; the diagonal blocks D_i are kept.
"""

from . import dense, tree as T


def hss_to_hodlr(c, g):
    """HODLR generators of the HSS matrix ``g`` (same tree ``c``)."""
    if g["kind"] != "hss":
        raise ValueError("hss_to_hodlr needs HSS generators")
    Ub, Vb = dense.hss_bases(c, g)
    L = len(c)
    h = {"kind": "hodlr", "D": list(g["D"]), "U12": [], "V12": [], "U21": [], "V21": []}
    for q in range(L - 1):
        a, b = T.children(q)
        h["U12"].append(Ub[a] @ g["B12"][q])
        h["V12"].append(Vb[b])
        h["U21"].append(Ub[b] @ g["B21"][q])
        h["V21"].append(Vb[a])
    return h
