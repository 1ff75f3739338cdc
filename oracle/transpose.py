"""Generators of the transposed matrix and Y = A^T X.  Test infrastructure.

The constructors of Sec. 3.2 and Sec. 3.3 (Table 3.1) need products with
A^* as well as with A; the data here are real, so A^* = A^T.  The oracle
takes the definition (A^T)(I, J) = A(J, I)^T block by block:

* HODLR (Def. 2.2): the diagonal blocks become D_i^T; for the children a, b
  of node q, A^T(I_a, I_b) = A(I_b, I_a)^T = V21_q U21_q^T and
  A^T(I_b, I_a) = V12_q U12_q^T, so U12' = V21, V12' = U21, U21' = V12 and
  V21' = U12.
* HSS (Def. 2.3, Eq. 2.2): A^T(I_a, I_b) = (U_b B21_q V_a^T)^T
  = V_a B21_q^T U_b^T.  The row bases of A^T are the column bases of A at
  every level, which the nested form gives by taking U' = V on the leaves
  and R_U' = R_V on the internal nodes (and V' = U, R_V' = R_U), with
  B12' = B21^T and B21' = B12^T.

The product is then the plain streamed product of ``matmat`` on these
generators.
"""

import numpy as np

from . import matmat as M


def _t(b):
    return None if b is None else np.asfortranarray(np.asarray(b, dtype=np.float64).T)


def transpose_gens(c, g):
    """Generators of A^T (same cluster tree ``c``)."""
    if g["kind"] == "hodlr":
        return {"kind": "hodlr", "D": [_t(D) for D in g["D"]],
                "U12": list(g["V21"]), "V12": list(g["U21"]),
                "U21": list(g["V12"]), "V21": list(g["U12"])}
    return {"kind": "hss", "D": [_t(D) for D in g["D"]],
            "U": list(g["V"]), "V": list(g["U"]),
            "RU": list(g["RV"]), "RV": list(g["RU"]),
            "B12": [_t(B) for B in g["B21"]], "B21": [_t(B) for B in g["B12"]]}


def matmat_transpose(c, g, X):
    """Y = A^T X for an n x r float64 block X."""
    return M.matmat(c, transpose_gens(c, g), X)


def matmat_transpose_rows(c, g, X, idx):
    """Rows ``idx`` of A^T X."""
    return M.matmat_rows(c, transpose_gens(c, g), X, idx)
