"""Hadamard product C = A o B of two HODLR or HSS matrices on the same
cluster tree (Sec. 4.4, Eq. 4.1, Fig. 4.3).  Test infrastructure.

For low-rank blocks, (U1 B1 V1^T) o (U2 B2 V2^T) = (U1 (.)^T U2)(B1 (x) B2)(V1 (.)^T V2)^T
(Eq. 4.1), with (x) the Kronecker product and (.)^T the transpose Khatri-Rao
product: row i of C (.)^T D is kron(c_i, d_i).  So:

* HODLR: D_C = D_A o D_B; every factor U12, V12, U21, V21 of C is the
  transpose Khatri-Rao product of A's and B's (Fig. 4.3 left); ranks multiply.
* HSS: D_C = D_A o D_B; leaf bases U_C = U_A (.)^T U_B, V_C = V_A (.)^T V_B;
  couplings B12_C = B12_A (x) B12_B, B21_C likewise (Fig. 4.3 right).  The
  translation operators are stacked, R_U = [R_l; R_r], one block per child;
  the derivation in Sec. 4.4 holds for each child's block, so the reading
  here is R_U,C = [R_l,A (x) R_l,B; R_r,A (x) R_r,B] (and the same for R_V),
  not the Kronecker product of the two stacked matrices.

Column a1 * k_B + a2 of a Khatri-Rao factor pairs column a1 of A's factor
with column a2 of B's, matching the Kronecker index order of R and B.
"""

import numpy as np

from . import tree as T


def khatri_rao_t(C, D):
    """Transpose Khatri-Rao product: row i is kron(C[i], D[i])."""
    C = np.asarray(C, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    n = C.shape[0]
    out = np.zeros((n, C.shape[1] * D.shape[1]), order="F")
    for i in range(n):
        out[i] = np.kron(C[i], D[i])
    return out


def _kron_halves(RA, RB, ka, kb, ka2, kb2):
    """[R_l,A (x) R_l,B; R_r,A (x) R_r,B] for stacked R_A = [R_l,A; R_r,A] with
    child ranks ka, kb (A) and ka2, kb2 (B)."""
    RA = np.asarray(RA, dtype=np.float64)
    RB = np.asarray(RB, dtype=np.float64)
    top = np.kron(RA[:ka], RB[:ka2])
    bot = np.kron(RA[ka:ka + kb], RB[ka2:ka2 + kb2])
    return np.asfortranarray(np.vstack([top, bot]))


def hadamard_gens(c, gA, gB):
    """Generators of A o B (same tree ``c``, same kind)."""
    if gA["kind"] != gB["kind"]:
        raise ValueError("A and B must be of the same kind")
    D = [np.asfortranarray(np.asarray(a) * np.asarray(b)) for a, b in zip(gA["D"], gB["D"])]
    if gA["kind"] == "hodlr":
        return {"kind": "hodlr", "D": D,
                **{key: [khatri_rao_t(a, b) for a, b in zip(gA[key], gB[key])]
                   for key in ("U12", "V12", "U21", "V21")}}
    p = T.depth(c)
    L = 1 << p

    def rank(g, key, rkey, q):
        if q >= L - 1:
            return np.asarray(g[key][q - (L - 1)]).shape[1]
        return g[rkey][q].shape[1]

    RU = [None] * (2 * L - 1)
    RV = [None] * (2 * L - 1)
    for q in range(1, L - 1):
        a, b = T.children(q)
        RU[q] = _kron_halves(gA["RU"][q], gB["RU"][q], rank(gA, "U", "RU", a), rank(gA, "U", "RU", b),
                             rank(gB, "U", "RU", a), rank(gB, "U", "RU", b))
        RV[q] = _kron_halves(gA["RV"][q], gB["RV"][q], rank(gA, "V", "RV", a), rank(gA, "V", "RV", b),
                             rank(gB, "V", "RV", a), rank(gB, "V", "RV", b))
    return {"kind": "hss", "D": D,
            "U": [khatri_rao_t(a, b) for a, b in zip(gA["U"], gB["U"])],
            "V": [khatri_rao_t(a, b) for a, b in zip(gA["V"], gB["V"])],
            "RU": RU, "RV": RV,
            "B12": [np.asfortranarray(np.kron(a, b)) for a, b in zip(gA["B12"], gB["B12"])],
            "B21": [np.asfortranarray(np.kron(a, b)) for a, b in zip(gA["B21"], gB["B21"])]}
