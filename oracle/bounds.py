"""Componentwise forward-error envelope of the product.  Test infrastructure.

For HODLR, ``B = |D||X| + sum_l |U|(|V|^T |X|)``; for HSS the same with every
factor of the nested bases (Eq. 2.2) and every core block taken in absolute
value.  Both equal the product of the matrix built from the absolute-valued
generators with |X|, so ``envelope`` is the oracle product applied to them.
A computed product whose generators, inputs and intermediates were each
rounded with unit roundoff u and whose sums were accumulated with unit
roundoff u_acc over at most L terms satisfies, to first order,

    |Y_hat - Y| <= (c_round * u + gamma_L(u_acc)) * B,   gamma_L(u) = L u / (1 - L u)

where c_round counts the rounded factors on the longest product chain.
"""

import numpy as np

from . import matmat as M


def abs_gens(g):
    out = {"kind": g["kind"]}
    for key, val in g.items():
        if key == "kind":
            continue
        out[key] = [None if v is None else np.abs(np.asarray(v, dtype=np.float64)) for v in val]
    return out


def envelope(c, g, X):
    return M.matmat(c, abs_gens(g), np.abs(np.asarray(X, dtype=np.float64)))


def envelope_rows(c, g, X, idx):
    return M.matmat_rows(c, abs_gens(g), np.abs(np.asarray(X, dtype=np.float64)), idx)


def gamma(L, u):
    Lu = L * u
    if Lu >= 1:
        return float("inf")
    return Lu / (1.0 - Lu)
