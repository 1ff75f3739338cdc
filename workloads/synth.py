"""Seeded generators of HODLR/HSS inputs (random and closed-form fixtures).

All arrays are float64 numpy arrays; blocks are stored column-major
(Fortran order), as Matlab would hold them.  Nothing here multiplies a
matrix by a vector: the functions only shape random draws or evaluate the
closed-form factor formulas of the fixture matrices.
"""

import math

import numpy as np

__all__ = [
    "SEED_BASE", "rng_for", "node_bounds", "uniform_leaf_ends",
    "gaussian_block", "random_hodlr", "random_hss",
    "exp_points", "exp_params", "exp_kernel_hodlr", "exp_kernel_hss",
    "tridiag_inverse_hodlr", "tridiag_inverse_hss", "tridiag_hodlr",
    "ones_hodlr", "ones_hss", "diagonal_hodlr", "diagonal_hss",
    "lowrank_hodlr", "lowrank_hss", "zeros_like_gens",
    "batch_spec", "serve_spec", "CONFIGS", "workload", "rng_named",
]

SEED_BASE = 1909_07909


def rng_for(config_id, salt=0):
    """numpy PCG64 stream for a configuration id and a salt."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + int(config_id), int(salt)]))


def _depth(c):
    L = len(c)
    p = L.bit_length() - 1
    if L < 1 or (1 << p) != L:
        raise ValueError("leaf count must be a power of two")
    return p


def node_bounds(c, level):
    """(start, end) row ranges of the 2**level nodes at ``level``."""
    p = _depth(c)
    span = 1 << (p - level)
    ends = [0] + [int(v) for v in c]
    return [(ends[j * span], ends[(j + 1) * span]) for j in range(1 << level)]


def uniform_leaf_ends(n_leaves, m):
    return [m * (i + 1) for i in range(n_leaves)]


def _F(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def gaussian_block(rng, rows, cols, std=1.0):
    return _F(rng.standard_normal((rows, cols)) * std)


def _rank_of(k, q):
    return int(k(q)) if callable(k) else int(k)


def random_hodlr(rng, c, k, d_shift=8.0, uv_var=None):
    """Gaussian HODLR generators: D ~ N(0,1) + d_shift*I, U, V ~ N(0, uv_var).

    ``uv_var`` is a variance (default 1/sqrt(n)); ``k`` is an int or a
    function of the internal node id giving its rank (used for both k12 and
    k21; pass a pair-returning function via ``k=lambda q: (k12, k21)``).
    """
    n = int(c[-1]) if len(c) else 0
    p = _depth(c)
    if uv_var is None:
        uv_var = 1.0 / math.sqrt(max(n, 1))
    std = math.sqrt(uv_var)
    leaves = node_bounds(c, p)
    D = []
    for (a, b) in leaves:
        m = b - a
        D.append(_F(rng.standard_normal((m, m)) + d_shift * np.eye(m)))
    U12, V12, U21, V21 = [], [], [], []
    for lvl in range(p):
        kids = node_bounds(c, lvl + 1)
        for j in range(1 << lvl):
            q = (1 << lvl) - 1 + j
            kq = k(q) if callable(k) else k
            k12, k21 = (kq if isinstance(kq, tuple) else (kq, kq))
            (a1, b1), (a2, b2) = kids[2 * j], kids[2 * j + 1]
            U12.append(gaussian_block(rng, b1 - a1, k12, std))
            V12.append(gaussian_block(rng, b2 - a2, k12, std))
            U21.append(gaussian_block(rng, b2 - a2, k21, std))
            V21.append(gaussian_block(rng, b1 - a1, k21, std))
    return {"kind": "hodlr", "D": D, "U12": U12, "V12": V12, "U21": U21, "V21": V21}


def _orthonormal_cols(rng, m, k):
    """Q factor of a Gaussian m x k draw, zero-padded to k columns if m < k."""
    G = rng.standard_normal((m, k))
    if m == 0 or k == 0:
        return _F(np.zeros((m, k)))
    Q, _ = np.linalg.qr(G)
    if Q.shape[1] < k:
        Q = np.hstack([Q, np.zeros((m, k - Q.shape[1]))])
    return _F(Q)


def random_hss(rng, c, k, d_shift=8.0, rb_var=1.0 / 32.0, orthonormal=True):
    """Gaussian HSS generators.

    Leaf U, V have orthonormal columns (Q of a Gaussian QR); translations
    R_U, R_V and couplings B12, B21 are iid N(0, rb_var) (a variance);
    D ~ N(0,1) + d_shift*I.  ``k`` is an int or a function of the node id
    returning the rank of that node's row and column bases (``(ku, kv)`` or
    one int for both).
    """
    p = _depth(c)
    L = 1 << p
    N = 2 * L - 1
    std = math.sqrt(rb_var)

    def ranks(q):
        kq = k(q) if callable(k) else k
        return kq if isinstance(kq, tuple) else (kq, kq)

    leaves = node_bounds(c, p)
    D, U, V = [], [], []
    for i, (a, b) in enumerate(leaves):
        m = b - a
        ku, kv = ranks(L - 1 + i)
        D.append(_F(rng.standard_normal((m, m)) + d_shift * np.eye(m)))
        if orthonormal:
            U.append(_orthonormal_cols(rng, m, ku))
            V.append(_orthonormal_cols(rng, m, kv))
        else:
            U.append(gaussian_block(rng, m, ku))
            V.append(gaussian_block(rng, m, kv))
    RU = [None] * N
    RV = [None] * N
    for q in range(1, L - 1):
        l, r = 2 * q + 1, 2 * q + 2
        ku, kv = ranks(q)
        RU[q] = gaussian_block(rng, ranks(l)[0] + ranks(r)[0], ku, std)
        RV[q] = gaussian_block(rng, ranks(l)[1] + ranks(r)[1], kv, std)
    B12, B21 = [], []
    for q in range(L - 1):
        l, r = 2 * q + 1, 2 * q + 2
        B12.append(gaussian_block(rng, ranks(l)[0], ranks(r)[1], std))
        B21.append(gaussian_block(rng, ranks(r)[0], ranks(l)[1], std))
    return {"kind": "hss", "D": D, "U": U, "V": V, "RU": RU, "RV": RV, "B12": B12, "B21": B21}


# ---------------------------------------------------------------------------
# Exponential kernel a_ij = sum_k c_k exp(-|t_i - t_j| / l_k)  (exact rank K)
# ---------------------------------------------------------------------------

def exp_points(rng, n):
    """n points sorted, iid Uniform[0, 1]."""
    return np.sort(rng.uniform(0.0, 1.0, size=n))


def exp_params(K=8, lmin=1e-2, lmax=1.0):
    """c_k = 1/K and l_k log-spaced between lmin and lmax."""
    ck = np.full(K, 1.0 / K)
    lk = np.logspace(math.log10(lmin), math.log10(lmax), K) if K > 1 else np.array([lmin])
    return ck, lk


def _expm(d, lk):
    """exp(-d / l_k) for d >= 0 (clamped), shape (len(d), K)."""
    d = np.maximum(np.asarray(d, dtype=np.float64), 0.0)
    return np.exp(-d[:, None] / lk[None, :])


def _exp_dense_block(ti, tj, ck, lk):
    d = np.abs(ti[:, None] - tj[None, :])
    out = np.zeros(d.shape)
    for c_, l_ in zip(ck, lk):
        out += c_ * np.exp(-d / l_)
    return out


def exp_kernel_hodlr(t, c, ck, lk):
    """Exact rank-K HODLR factors, centred at each split so entries lie in (0, 1].

    For internal node q with left child rows I and right child columns J and
    s = last point of I: A(I, J) has U = c_k e^{-(s - t_i)/l_k},
    V = e^{-(t_j - s)/l_k}; A(J, I) has U = c_k e^{-(t_i - s)/l_k},
    V = e^{-(s - t_j)/l_k}.
    """
    t = np.asarray(t, dtype=np.float64)
    p = _depth(c)
    D = [_F(_exp_dense_block(t[a:b], t[a:b], ck, lk)) for (a, b) in node_bounds(c, p)]
    U12, V12, U21, V21 = [], [], [], []
    for lvl in range(p):
        kids = node_bounds(c, lvl + 1)
        for j in range(1 << lvl):
            (a1, b1), (a2, b2) = kids[2 * j], kids[2 * j + 1]
            if b1 > a1:
                s = t[b1 - 1]
            elif b2 > a2:
                s = t[a2]
            else:
                s = 0.0
            tl, tr = t[a1:b1], t[a2:b2]
            U12.append(_F(_expm(s - tl, lk) * ck[None, :]))
            V12.append(_F(_expm(tr - s, lk)))
            U21.append(_F(_expm(tr - s, lk) * ck[None, :]))
            V21.append(_F(_expm(s - tl, lk)))
    return {"kind": "hodlr", "D": D, "U12": U12, "V12": V12, "U21": U21, "V21": V21}


def exp_kernel_hss(t, c, ck, lk):
    """Exact rank-2K HSS generators of the exponential kernel.

    A node spanning points [a, b] has basis columns e^{-(b - t)/l_k}
    (right-facing) and e^{-(t - a)/l_k} (left-facing); translations are
    diagonal scalings by e^{-gap/l_k}; couplings carry c_k e^{-gap/l_k} in one
    K x K corner.  Every leaf must be non-empty.
    """
    t = np.asarray(t, dtype=np.float64)
    p = _depth(c)
    L = 1 << p
    K = len(ck)
    span = {}
    for lvl in range(p + 1):
        for j, (a, b) in enumerate(node_bounds(c, lvl)):
            if b <= a:
                raise ValueError("exp_kernel_hss needs non-empty leaves")
            span[(1 << lvl) - 1 + j] = (t[a], t[b - 1])
    leaves = node_bounds(c, p)
    D, U, V = [], [], []
    for i, (a, b) in enumerate(leaves):
        ta, tb = span[L - 1 + i]
        tt = t[a:b]
        D.append(_F(_exp_dense_block(tt, tt, ck, lk)))
        B = np.hstack([_expm(tb - tt, lk), _expm(tt - ta, lk)])
        U.append(_F(B))
        V.append(_F(B))
    RU = [None] * (2 * L - 1)
    RV = [None] * (2 * L - 1)
    B12, B21 = [], []
    for q in range(L - 1):
        l, r = 2 * q + 1, 2 * q + 2
        a, b = span[q]
        a1, b1 = span[l]
        a2, b2 = span[r]
        if q > 0:
            Rl = np.diag(np.concatenate([np.exp(-(b - b1) / lk), np.ones(K)]))
            Rr = np.diag(np.concatenate([np.ones(K), np.exp(-(a2 - a) / lk)]))
            RU[q] = _F(np.vstack([Rl, Rr]))
            RV[q] = _F(np.vstack([Rl, Rr]))
        g = ck * np.exp(-(a2 - b1) / lk)
        S12 = np.zeros((2 * K, 2 * K))
        S21 = np.zeros((2 * K, 2 * K))
        S12[np.arange(K), K + np.arange(K)] = g
        S21[K + np.arange(K), np.arange(K)] = g
        B12.append(_F(S12))
        B21.append(_F(S21))
    return {"kind": "hss", "D": D, "U": U, "V": V, "RU": RU, "RV": RV, "B12": B12, "B21": B21}


# ---------------------------------------------------------------------------
# tridiag(-1, 2, -1) and its inverse min(i,j)(n+1-max(i,j))/(n+1)
# ---------------------------------------------------------------------------

def _tinv_block(rows1, cols1, n):
    """Closed-form entries of the inverse of tridiag(-1,2,-1); 1-based indices."""
    i = np.asarray(rows1, dtype=np.float64)[:, None]
    j = np.asarray(cols1, dtype=np.float64)[None, :]
    return np.minimum(i, j) * (n + 1 - np.maximum(i, j)) / (n + 1)


def tridiag_inverse_hodlr(c):
    """Rank-1 HODLR factors of T^{-1}: above the diagonal U = i, V = (n+1-j)/(n+1)."""
    n = int(c[-1])
    p = _depth(c)
    D = [_F(_tinv_block(np.arange(a, b) + 1, np.arange(a, b) + 1, n)) for (a, b) in node_bounds(c, p)]
    U12, V12, U21, V21 = [], [], [], []
    for lvl in range(p):
        kids = node_bounds(c, lvl + 1)
        for j in range(1 << lvl):
            (a1, b1), (a2, b2) = kids[2 * j], kids[2 * j + 1]
            il = np.arange(a1, b1, dtype=np.float64) + 1
            ir = np.arange(a2, b2, dtype=np.float64) + 1
            U12.append(_F(il[:, None]))
            V12.append(_F(((n + 1 - ir) / (n + 1))[:, None]))
            U21.append(_F(((n + 1 - ir) / (n + 1))[:, None]))
            V21.append(_F(il[:, None]))
    return {"kind": "hodlr", "D": D, "U12": U12, "V12": V12, "U21": U21, "V21": V21}


def tridiag_inverse_hss(c):
    """Rank-2 HSS generators of T^{-1}: bases [i, n+1-i], identity translations."""
    n = int(c[-1])
    p = _depth(c)
    L = 1 << p
    leaves = node_bounds(c, p)
    D, U, V = [], [], []
    for (a, b) in leaves:
        i = np.arange(a, b, dtype=np.float64) + 1
        D.append(_F(_tinv_block(i, i, n)))
        B = np.stack([i, n + 1 - i], axis=1) if b > a else np.zeros((0, 2))
        U.append(_F(B))
        V.append(_F(B))
    RU = [None] * (2 * L - 1)
    RV = [None] * (2 * L - 1)
    for q in range(1, L - 1):
        RU[q] = _F(np.vstack([np.eye(2), np.eye(2)]))
        RV[q] = _F(np.vstack([np.eye(2), np.eye(2)]))
    S12 = _F([[0.0, 1.0 / (n + 1)], [0.0, 0.0]])
    S21 = _F([[0.0, 0.0], [1.0 / (n + 1), 0.0]])
    return {"kind": "hss", "D": D, "U": U, "V": V, "RU": RU, "RV": RV,
            "B12": [S12.copy() for _ in range(L - 1)], "B21": [S21.copy() for _ in range(L - 1)]}


def tridiag_hodlr(c):
    """Exact rank-1 HODLR representation of the banded T = tridiag(-1, 2, -1)."""
    n = int(c[-1])
    p = _depth(c)
    D = []
    for (a, b) in node_bounds(c, p):
        m = b - a
        D.append(_F(2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)))
    U12, V12, U21, V21 = [], [], [], []
    for lvl in range(p):
        kids = node_bounds(c, lvl + 1)
        for j in range(1 << lvl):
            (a1, b1), (a2, b2) = kids[2 * j], kids[2 * j + 1]
            ml, mr = b1 - a1, b2 - a2
            u12 = np.zeros((ml, 1)); v12 = np.zeros((mr, 1))
            u21 = np.zeros((mr, 1)); v21 = np.zeros((ml, 1))
            if ml and mr:
                u12[-1, 0] = 1.0; v12[0, 0] = -1.0
                u21[0, 0] = 1.0; v21[-1, 0] = -1.0
            U12.append(_F(u12)); V12.append(_F(v12)); U21.append(_F(u21)); V21.append(_F(v21))
    del n
    return {"kind": "hodlr", "D": D, "U12": U12, "V12": V12, "U21": U21, "V21": V21}


# ---------------------------------------------------------------------------
# Structured constructors of Sec. 3.4 with exactly known products
# ---------------------------------------------------------------------------

def ones_hodlr(c):
    p = _depth(c)
    D = [_F(np.ones((b - a, b - a))) for (a, b) in node_bounds(c, p)]
    U12, V12, U21, V21 = [], [], [], []
    for lvl in range(p):
        kids = node_bounds(c, lvl + 1)
        for j in range(1 << lvl):
            (a1, b1), (a2, b2) = kids[2 * j], kids[2 * j + 1]
            U12.append(_F(np.ones((b1 - a1, 1)))); V12.append(_F(np.ones((b2 - a2, 1))))
            U21.append(_F(np.ones((b2 - a2, 1)))); V21.append(_F(np.ones((b1 - a1, 1))))
    return {"kind": "hodlr", "D": D, "U12": U12, "V12": V12, "U21": U21, "V21": V21}


def ones_hss(c):
    p = _depth(c)
    L = 1 << p
    leaves = node_bounds(c, p)
    RU = [None] * (2 * L - 1)
    RV = [None] * (2 * L - 1)
    for q in range(1, L - 1):
        RU[q] = _F([[1.0], [1.0]]); RV[q] = _F([[1.0], [1.0]])
    return {"kind": "hss", "D": [_F(np.ones((b - a, b - a))) for (a, b) in leaves],
            "U": [_F(np.ones((b - a, 1))) for (a, b) in leaves],
            "V": [_F(np.ones((b - a, 1))) for (a, b) in leaves],
            "RU": RU, "RV": RV, "B12": [_F([[1.0]]) for _ in range(L - 1)],
            "B21": [_F([[1.0]]) for _ in range(L - 1)]}


def diagonal_hodlr(c, d):
    """Rank-0 HODLR representation of diag(d)."""
    p = _depth(c)
    D = [_F(np.diag(d[a:b])) for (a, b) in node_bounds(c, p)]
    U12, V12, U21, V21 = [], [], [], []
    for lvl in range(p):
        kids = node_bounds(c, lvl + 1)
        for j in range(1 << lvl):
            (a1, b1), (a2, b2) = kids[2 * j], kids[2 * j + 1]
            U12.append(_F(np.zeros((b1 - a1, 0)))); V12.append(_F(np.zeros((b2 - a2, 0))))
            U21.append(_F(np.zeros((b2 - a2, 0)))); V21.append(_F(np.zeros((b1 - a1, 0))))
    return {"kind": "hodlr", "D": D, "U12": U12, "V12": V12, "U21": U21, "V21": V21}


def diagonal_hss(c, d):
    p = _depth(c)
    L = 1 << p
    leaves = node_bounds(c, p)
    RU = [None] * (2 * L - 1)
    RV = [None] * (2 * L - 1)
    for q in range(1, L - 1):
        RU[q] = _F(np.zeros((0, 0))); RV[q] = _F(np.zeros((0, 0)))
    return {"kind": "hss", "D": [_F(np.diag(d[a:b])) for (a, b) in leaves],
            "U": [_F(np.zeros((b - a, 0))) for (a, b) in leaves],
            "V": [_F(np.zeros((b - a, 0))) for (a, b) in leaves],
            "RU": RU, "RV": RV, "B12": [_F(np.zeros((0, 0))) for _ in range(L - 1)],
            "B21": [_F(np.zeros((0, 0))) for _ in range(L - 1)]}


def lowrank_hodlr(c, Ug, Vg):
    """Exact HODLR representation of Ug @ Vg.T (Sec. 3.4 'low-rank')."""
    p = _depth(c)
    D = [_F(Ug[a:b] @ Vg[a:b].T) for (a, b) in node_bounds(c, p)]
    U12, V12, U21, V21 = [], [], [], []
    for lvl in range(p):
        kids = node_bounds(c, lvl + 1)
        for j in range(1 << lvl):
            (a1, b1), (a2, b2) = kids[2 * j], kids[2 * j + 1]
            U12.append(_F(Ug[a1:b1])); V12.append(_F(Vg[a2:b2]))
            U21.append(_F(Ug[a2:b2])); V21.append(_F(Vg[a1:b1]))
    return {"kind": "hodlr", "D": D, "U12": U12, "V12": V12, "U21": U21, "V21": V21}


def lowrank_hss(c, Ug, Vg):
    """Exact HSS representation of Ug @ Vg.T with identity translations/couplings."""
    p = _depth(c)
    L = 1 << p
    k = Ug.shape[1]
    leaves = node_bounds(c, p)
    RU = [None] * (2 * L - 1)
    RV = [None] * (2 * L - 1)
    for q in range(1, L - 1):
        RU[q] = _F(np.vstack([np.eye(k), np.eye(k)])); RV[q] = _F(np.vstack([np.eye(k), np.eye(k)]))
    return {"kind": "hss", "D": [_F(Ug[a:b] @ Vg[a:b].T) for (a, b) in leaves],
            "U": [_F(Ug[a:b]) for (a, b) in leaves], "V": [_F(Vg[a:b]) for (a, b) in leaves],
            "RU": RU, "RV": RV, "B12": [_F(np.eye(k)) for _ in range(L - 1)],
            "B21": [_F(np.eye(k)) for _ in range(L - 1)]}


def zeros_like_gens(g, keep_D=False):
    """Same shapes as ``g`` with every generator zero (or only the D blocks kept)."""
    out = {"kind": g["kind"]}
    for key, val in g.items():
        if key == "kind":
            continue
        if key == "D" and keep_D:
            out[key] = [_F(v) for v in val]
        else:
            out[key] = [None if v is None else _F(np.zeros_like(v)) for v in val]
    return out


# ---------------------------------------------------------------------------
# The five workload shapes (a configuration id picks the seed)
# ---------------------------------------------------------------------------

CONFIGS = {
    1: dict(name="hodlr_n4096_m128_k8_r1_f64", kind="hodlr", n=4096, m=128, k=8, r=1),
    2: dict(name="hss_n65536_m256_k32_r64", kind="hss", n=65536, m=256, k=32, r=64),
    3: dict(name="hodlr_exp_n262144_m256_K8", kind="hodlr", n=262144, m=256, K=8, r=(1, 128)),
    4: dict(name="batched_512", count=512, nmin=1024, nmax=32768, ranks=(4, 8, 16, 32, 64),
            rmax=32, m=256),
    5: dict(name="serving_64_hss", count=64, log2n=(12, 18), ranks=(16, 32, 48, 64), rmax=16,
            m=256, rates=(1000, 5000, 10000, 20000, 50000), budget=100 << 30),
}


def batch_spec(rng, count=512, nmin=1024, nmax=32768, ranks=(4, 8, 16, 32, 64), rmax=32):
    """Shapes of the batched workload: n log-uniform, rank and RHS count uniform.

    Returns a list of dicts {kind, n, k, r}; half HODLR and half HSS, chosen
    by the seed.
    """
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        k = int(rng.choice(ranks))
        r = int(rng.integers(1, rmax + 1))
        kind = "hodlr" if rng.uniform() < 0.5 else "hss"
        out.append(dict(kind=kind, n=n, k=k, r=r))
    return out


def serve_spec(rng, count=64, log2n=(12, 18), ranks=(16, 32, 48, 64)):
    """Resident matrices of the serving workload: n = 2^e, e uniform; rank uniform."""
    return [dict(kind="hss", n=1 << int(rng.integers(log2n[0], log2n[1] + 1)),
                 k=int(rng.choice(ranks))) for _ in range(count)]


def workload(name):
    """The synthetic workload called `name` (its sizes and shapes)."""
    for cfg in CONFIGS.values():
        if cfg["name"] == name:
            return cfg
    raise KeyError(name)


def rng_named(name, salt=0):
    """The seeded stream of the workload called `name` (same seed as its id)."""
    for key, cfg in CONFIGS.items():
        if cfg["name"] == name:
            return rng_for(key, salt)
    raise KeyError(name)
