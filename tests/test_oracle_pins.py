"""Pins of the CPU oracle against brute force, closed forms and exact-rank fixtures.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
swapped B12/B21, a transposed factor, a wrong half of a translation operator,
the coupling loop stopping one level early) fails at least one of them;
``test_planted_mistakes`` plants such slips in the oracle and checks that the
brute-force pin catches each one.
"""

import bisect
import os

import numpy as np
import pytest

import workloads as W
from oracle import bounds, convert as CV, dense, expkernel, fig41, hadamard as HD, matmat as M, solve as SV, transpose as TR, tree as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")

# Small trees: uniform, ragged (non power of two) and with empty leaves (Fig. 3.2 style).
SMALL_TREES = [
    ("uniform_p3", [8, 16, 24, 32, 40, 48, 56, 64]),
    ("ragged_p3", T.default_leaf_ends(45, 6)),
    ("empty_leaves_p2", [5, 9, 17, 17]),
    ("empty_first_p2", [0, 7, 12, 20]),
    ("single_leaf", [13]),
    ("p1", [7, 13]),
]


# --------------------------------------------------------------------------
# Brute force: every entry evaluated on its own from the generators.
# --------------------------------------------------------------------------

def _leaf_of(c, r):
    return bisect.bisect_right([int(v) for v in c], r)


def _start(c, q):
    lvl, j = T.level_pos(q)
    return T.node_range(c, lvl, j)[0]


def brute_entry(c, g, r, s):
    """A(r, s) from the generators: the deepest common ancestor q of rows r and s
    decides which sibling block holds the entry (Def. 2.2 / Def. 2.3)."""
    p = T.depth(c)
    L = 1 << p
    li, lj = _leaf_of(c, r), _leaf_of(c, s)
    if li == lj:
        a0 = _start(c, L - 1 + li)
        return float(np.asarray(g["D"][li])[r - a0, s - a0])
    a, b = L - 1 + li, L - 1 + lj
    while (a - 1) // 2 != (b - 1) // 2:
        a, b = (a - 1) // 2, (b - 1) // 2
    q = (a - 1) // 2
    left = a % 2 == 1
    if g["kind"] == "hodlr":
        Uq, Vq = (g["U12"][q], g["V12"][q]) if left else (g["U21"][q], g["V21"][q])
        return float(Uq[r - _start(c, a)] @ Vq[s - _start(c, b)])
    u = _basis_row(c, g, "U", "RU", li, r, a)
    v = _basis_row(c, g, "V", "RV", lj, s, b)
    S = g["B12"][q] if left else g["B21"][q]
    return float(u @ S @ v)


def _basis_row(c, g, leafkey, rkey, leaf, row, stop):
    """Row `row` of the nested basis of node `stop`, walking up from the leaf with
    the child's half of each translation operator (Eq. 2.2)."""
    p = T.depth(c)
    L = 1 << p
    x = L - 1 + leaf
    u = np.asarray(g[leafkey][leaf])[row - _start(c, x)]
    while x != stop:
        y = (x - 1) // 2
        R = g[rkey][y]
        left_rank = _rank(g, leafkey, rkey, 2 * y + 1, L)
        if x % 2 == 1:
            u = u @ R[:left_rank]
        else:
            u = u @ R[left_rank:]
        x = y
    return u


def _rank(g, leafkey, rkey, q, L):
    if q >= L - 1:
        return np.asarray(g[leafkey][q - (L - 1)]).shape[1]
    return g[rkey][q].shape[1]


def brute_dense(c, g):
    n = int(c[-1])
    A = np.zeros((n, n))
    for r in range(n):
        for s in range(n):
            A[r, s] = brute_entry(c, g, r, s)
    return A


def _gens(kind, c, seed, k=3):
    rng = np.random.default_rng(seed)
    if kind == "hodlr":
        return W.random_hodlr(rng, c, k)
    return W.random_hss(rng, c, k, orthonormal=False)


# --------------------------------------------------------------------------
# P1: brute force on tiny trees
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SMALL_TREES)
def test_dense_equals_brute_force(kind, name, c):
    g = _gens(kind, c, 7)
    A = dense.dense(c, g)
    B = brute_dense(c, g)
    assert np.allclose(A, B, rtol=1e-13, atol=1e-13), name


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_variable_ranks_brute_force(kind):
    c = T.default_leaf_ends(40, 5)
    rng = np.random.default_rng(3)
    if kind == "hodlr":
        g = W.random_hodlr(rng, c, lambda q: (1 + q % 3, 2 + q % 2))
    else:
        g = W.random_hss(rng, c, lambda q: (1 + q % 4, 1 + (q * 7) % 3), orthonormal=False)
    assert np.allclose(dense.dense(c, g), brute_dense(c, g), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_every_entry_set_once(kind):
    """HODLR/HSS partition: diagonal leaves + one sibling block per level cover A exactly once."""
    c = T.default_leaf_ends(37, 4)
    g = W.ones_hodlr(c) if kind == "hodlr" else W.ones_hss(c)
    A = dense.dense(c, g)
    assert np.array_equal(A, np.ones((37, 37)))


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SMALL_TREES)
def test_matmat_and_rows_vs_brute(kind, name, c):
    g = _gens(kind, c, 11)
    n = int(c[-1])
    X = np.random.default_rng(5).standard_normal((n, 3))
    Ab = brute_dense(c, g)
    Y = M.matmat(c, g, X)
    assert np.allclose(Y, Ab @ X, rtol=1e-12, atol=1e-12)
    if n:
        idx = [0, n - 1, n // 2]
        assert np.allclose(M.matmat_rows(c, g, X, idx), (Ab @ X)[idx], rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# P2: exact-rank exponential kernel
# --------------------------------------------------------------------------

def _exp_case(n, nmin, seed=2):
    rng = np.random.default_rng(seed)
    t = W.exp_points(rng, n)
    ck, lk = W.exp_params(8)
    c = T.default_leaf_ends(n, nmin)
    return t, ck, lk, c


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_exp_kernel_generators_are_exact(fmt):
    t, ck, lk, c = _exp_case(300, 32)
    g = W.exp_kernel_hodlr(t, c, ck, lk) if fmt == "hodlr" else W.exp_kernel_hss(t, c, ck, lk)
    A = dense.dense(c, g)
    E = expkernel.entries(t, ck, lk, np.arange(300), np.arange(300))
    assert np.max(np.abs(A - E)) <= 1e-14
    # entries of the centred factors lie in (0, 1]
    for key in ("U12", "V12", "U21", "V21", "U", "V"):
        for blk in g.get(key, []):
            if blk.size:
                assert blk.min() >= 0.0 and blk.max() <= 1.0


def test_exp_kernel_ranks():
    """Off-diagonal sibling blocks have rank <= K; HSS block rows rank <= 2K."""
    t, ck, lk, c = _exp_case(256, 32)
    E = expkernel.entries(t, ck, lk, np.arange(256), np.arange(256))
    K = len(ck)
    for lvl in range(1, T.depth(c) + 1):
        for j in range(0, 1 << lvl, 2):
            a1, b1 = T.node_range(c, lvl, j)
            a2, b2 = T.node_range(c, lvl, j + 1)
            assert np.linalg.matrix_rank(E[a1:b1, a2:b2], tol=1e-12) <= K
            rows = E[a1:b1]
            blockrow = np.hstack([rows[:, :a1], rows[:, b1:]])
            assert np.linalg.matrix_rank(blockrow, tol=1e-12) <= 2 * K


def test_exp_recurrence_vs_brute_force():
    t, ck, lk, c = _exp_case(500, 64)
    X = np.random.default_rng(9).standard_normal((500, 4))
    E = expkernel.entries(t, ck, lk, np.arange(500), np.arange(500))
    Y = expkernel.apply(t, ck, lk, X)
    assert np.allclose(Y, E @ X, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_exp_matmat_vs_recurrence(fmt):
    t, ck, lk, c = _exp_case(1000, 64)
    g = W.exp_kernel_hodlr(t, c, ck, lk) if fmt == "hodlr" else W.exp_kernel_hss(t, c, ck, lk)
    X = np.random.default_rng(4).standard_normal((1000, 2))
    Y = M.matmat(c, g, X)
    Z = expkernel.apply(t, ck, lk, X)
    assert np.linalg.norm(Y - Z) <= 1e-13 * np.linalg.norm(Z)


# --------------------------------------------------------------------------
# P3: closed forms
# --------------------------------------------------------------------------

def _tridiag(n):
    return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
@pytest.mark.parametrize("n,nmin", [(64, 8), (77, 9), (130, 16)])
def test_tridiag_inverse_is_inverse(fmt, n, nmin):
    c = T.default_leaf_ends(n, nmin)
    g = W.tridiag_inverse_hodlr(c) if fmt == "hodlr" else W.tridiag_inverse_hss(c)
    A = dense.dense(c, g)
    assert np.max(np.abs(_tridiag(n) @ A - np.eye(n))) <= 1e-12 * n


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_tridiag_inverse_exact_answer(fmt):
    n = 200
    c = T.default_leaf_ends(n, 16)
    g = W.tridiag_inverse_hodlr(c) if fmt == "hodlr" else W.tridiag_inverse_hss(c)
    z = np.random.default_rng(1).integers(-5, 6, size=(n, 3)).astype(np.float64)
    x = 2 * z
    x[1:] -= z[:-1]
    x[:-1] -= z[1:]
    y = M.matmat(c, g, x)
    env = bounds.envelope(c, g, x)
    assert np.all(np.abs(y - z) <= bounds.gamma(2 * n, 2.0 ** -53) * env + 1e-300)


def test_tridiag_banded_integer_exact():
    c = T.default_leaf_ends(97, 8)
    g = W.tridiag_hodlr(c)
    X = np.random.default_rng(2).integers(-9, 10, size=(97, 5)).astype(np.float64)
    Y = M.matmat(c, g, X)
    S = 2 * X
    S[1:] -= X[:-1]
    S[:-1] -= X[1:]
    assert np.array_equal(Y, S)


def _read_ranks():
    out = []
    with open(os.path.join(GOLD, "structured_ranks.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                name, bl, bu, hr, sr = [s.strip() for s in line.split("|")]
                out.append((name, int(bl), int(bu), int(hr), int(sr)))
    return out


@pytest.mark.parametrize("name,bl,bu,hodlr_rank,hss_rank", _read_ranks())
def test_banded_ranks_stated_in_paper(name, bl, bu, hodlr_rank, hss_rank):
    n = 64
    rng = np.random.default_rng(0)
    A = np.zeros((n, n))
    for d in range(-bl, bu + 1):
        A += np.diag(rng.uniform(1, 2, n - abs(d)), k=d)
    c = T.default_leaf_ends(n, 8)
    hmax, smax = 0, 0
    for lvl in range(1, T.depth(c) + 1):
        for j in range(1 << lvl):
            a, b = T.node_range(c, lvl, j)
            sa, sb = T.node_range(c, lvl, j ^ 1)
            hmax = max(hmax, np.linalg.matrix_rank(A[a:b, sa:sb]))
            br = np.hstack([A[a:b, :a], A[a:b, b:]])
            bc = np.vstack([A[:a, a:b], A[b:, a:b]])
            smax = max(smax, np.linalg.matrix_rank(br), np.linalg.matrix_rank(bc))
    assert hmax == hodlr_rank
    assert smax == hss_rank


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_structured_exact_products(fmt):
    c = T.default_leaf_ends(50, 6)
    n = 50
    X = np.random.default_rng(8).integers(-4, 5, size=(n, 3)).astype(np.float64)
    ones = W.ones_hodlr(c) if fmt == "hodlr" else W.ones_hss(c)
    assert np.array_equal(M.matmat(c, ones, X), np.tile(X.sum(axis=0), (n, 1)))
    d = np.arange(1, n + 1, dtype=np.float64)
    diag = W.diagonal_hodlr(c, d) if fmt == "hodlr" else W.diagonal_hss(c, d)
    assert np.array_equal(M.matmat(c, diag, X), d[:, None] * X)
    eye = W.diagonal_hodlr(c, np.ones(n)) if fmt == "hodlr" else W.diagonal_hss(c, np.ones(n))
    assert np.array_equal(M.matmat(c, eye, X), X)
    zg = W.zeros_like_gens(ones)
    assert np.array_equal(M.matmat(c, zg, X), np.zeros((n, 3)))
    rng = np.random.default_rng(3)
    Ug, Vg = rng.standard_normal((n, 4)), rng.standard_normal((n, 4))
    lr = W.lowrank_hodlr(c, Ug, Vg) if fmt == "hodlr" else W.lowrank_hss(c, Ug, Vg)
    assert np.allclose(M.matmat(c, lr, X), Ug @ (Vg.T @ X), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# P4: invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_linearity_and_columns(kind):
    c = T.default_leaf_ends(90, 10)
    g = _gens(kind, c, 21, k=4)
    rng = np.random.default_rng(6)
    X, Z = rng.standard_normal((90, 3)), rng.standard_normal((90, 3))
    lhs = M.matmat(c, g, 2.5 * X - 0.5 * Z)
    rhs = 2.5 * M.matmat(c, g, X) - 0.5 * M.matmat(c, g, Z)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    Y = M.matmat(c, g, X)
    for j in range(3):
        assert np.allclose(M.matmat(c, g, X[:, j])[:, 0], Y[:, j], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("name,c", SMALL_TREES)
def test_fig41_hodlr_recursion(name, c):
    g = _gens("hodlr", c, 13)
    X = np.random.default_rng(1).standard_normal((int(c[-1]), 2))
    assert np.allclose(fig41.hodlr_matvec(c, g, X), M.matmat(c, g, X), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name,c", SMALL_TREES)
def test_fig41_hss_couplings_through_level_p(name, c):
    """Reading of the coupling loop: levels 1..p agree with the definition;
    levels 1..p-1 (as printed) do not once leaf siblings couple."""
    g = _gens("hss", c, 17)
    n = int(c[-1])
    X = np.random.default_rng(2).standard_normal((n, 2))
    Y = M.matmat(c, g, X)
    assert np.allclose(fig41.hss_matvec(c, g, X), Y, rtol=1e-12, atol=1e-12)
    p = T.depth(c)
    if p >= 1 and n > 0:
        Yp = fig41.hss_matvec(c, g, X, couple_to=p - 1)
        assert np.linalg.norm(Yp - Y) > 1e-3 * np.linalg.norm(Y)


def test_hss_to_hodlr_expansion():
    """hss2hodlr (Sec. 3.5): explicit factors U_a B12 and V_b give the same matrix."""
    c = T.default_leaf_ends(70, 8)
    g = _gens("hss", c, 5, k=3)
    Ub, Vb = dense.hss_bases(c, g)
    L = len(c)
    h = {"kind": "hodlr", "D": g["D"], "U12": [], "V12": [], "U21": [], "V21": []}
    for q in range(L - 1):
        a, b = T.children(q)
        h["U12"].append(Ub[a] @ g["B12"][q]); h["V12"].append(Vb[b])
        h["U21"].append(Ub[b] @ g["B21"][q]); h["V21"].append(Vb[a])
    assert np.allclose(dense.hodlr_dense(c, h), dense.hss_dense(c, g), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_envelope_dominates(kind):
    c = T.default_leaf_ends(60, 7)
    g = _gens(kind, c, 23)
    X = np.random.default_rng(3).standard_normal((60, 2))
    assert np.all(bounds.envelope(c, g, X) >= np.abs(M.matmat(c, g, X)) * (1 - 1e-14))
    ag = bounds.abs_gens(g)
    assert np.allclose(bounds.envelope(c, g, X), M.matmat(c, ag, np.abs(X)))


def test_float32_model_within_envelope():
    """The error model: generators and X rounded to float32 and float32 sums stay
    inside (c_round u + gamma_L(u)) * envelope."""
    c = T.default_leaf_ends(128, 16)
    g = _gens("hodlr", c, 29, k=4)
    X = np.random.default_rng(4).standard_normal((128, 2))
    g32 = {k: (v if k == "kind" else [None if b is None else b.astype(np.float32) for b in v])
           for k, v in g.items()}
    A32 = dense.dense(c, g32).astype(np.float32)
    Y32 = A32 @ X.astype(np.float32)
    Y = M.matmat(c, g, X)
    u = 2.0 ** -24
    tol = (4 * u + bounds.gamma(200, u)) * bounds.envelope(c, g, X)
    assert np.all(np.abs(Y32 - Y) <= tol)


# --------------------------------------------------------------------------
# Planted mistakes: each must be caught by the brute-force pin.
# --------------------------------------------------------------------------

def _hss_bases_wrong_half(c, g):
    p = T.depth(c)
    L = 1 << p
    Ub, Vb = {}, {}
    for i in range(L):
        Ub[L - 1 + i] = np.asarray(g["U"][i]); Vb[L - 1 + i] = np.asarray(g["V"][i])
    for lvl in range(p - 1, 0, -1):
        for j in range(1 << lvl):
            q = T.node_id(lvl, j)
            a, b = T.children(q)
            Ub[q] = dense._blkdiag(Ub[b], Ub[a]) @ g["RU"][q]   # children swapped
            Vb[q] = dense._blkdiag(Vb[a], Vb[b]) @ g["RV"][q]
    return Ub, Vb


_ORIG_HSS_BASES = dense.hss_bases


def _hss_bases_ru_for_v(c, g):
    return _ORIG_HSS_BASES(c, dict(g, RV=g["RU"]))


@pytest.mark.parametrize("plant", ["swap_couplings", "wrong_half", "ru_for_v", "drop_level",
                                   "transpose_hodlr"])
def test_planted_mistakes(monkeypatch, plant):
    c = [6, 12, 18, 24, 30, 36, 42, 48]
    kind = "hodlr" if plant == "transpose_hodlr" else "hss"
    g = _gens(kind, c, 31, k=3)
    ref = brute_dense(c, g)
    if plant == "swap_couplings":
        orig = dense.hss_dense
        monkeypatch.setattr(dense, "hss_dense", lambda c_, g_: orig(c_, dict(g_, B12=g_["B21"], B21=g_["B12"])))
    elif plant == "wrong_half":
        monkeypatch.setattr(dense, "hss_bases", _hss_bases_wrong_half)
    elif plant == "ru_for_v":
        monkeypatch.setattr(dense, "hss_bases", _hss_bases_ru_for_v)
    elif plant == "drop_level":
        orig = dense.hss_dense

        def dropped(c_, g_):
            A = orig(c_, g_)
            a1, b1 = T.node_range(c_, 3, 0)
            a2, b2 = T.node_range(c_, 3, 1)
            A[a1:b1, a2:b2] = 0.0
            return A
        monkeypatch.setattr(dense, "hss_dense", dropped)
    elif plant == "transpose_hodlr":
        orig = dense.hodlr_dense
        monkeypatch.setattr(dense, "hodlr_dense",
                            lambda c_, g_: orig(c_, dict(g_, U21=g_["V21"], V21=g_["U21"])))
    A = dense.dense(c, g)
    assert not np.allclose(A, ref, rtol=1e-6, atol=1e-6), plant


# --------------------------------------------------------------------------
# Transposed product (A^T X; products with A^* in Sec. 3.2-3.3, Table 3.1)
# --------------------------------------------------------------------------

def _mixed_gens(kind, c, seed):
    """Per-node ranks that differ between rows and columns (ku != kv), so a
    swapped pair of factors cannot pass by symmetry."""
    rng = np.random.default_rng(seed)
    if kind == "hodlr":
        return W.random_hodlr(rng, c, lambda q: (1 + q % 3, 2 + q % 2))
    return W.random_hss(rng, c, lambda q: (1 + q % 4, 1 + (q * 7) % 3), orthonormal=False)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SMALL_TREES + [("variable_p3", T.default_leaf_ends(40, 5))])
def test_transpose_gens_brute_force(kind, name, c):
    """Every entry of the relabelled generators, evaluated on its own, is the
    mirrored entry of A."""
    g = _mixed_gens(kind, c, 17)
    gt = TR.transpose_gens(c, g)
    assert np.allclose(brute_dense(c, gt), brute_dense(c, g).T, rtol=1e-13, atol=1e-13), name


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_transpose_adjoint_identity(kind):
    """<Z, A X> = <A^T Z, X> through the streamed products."""
    c = T.default_leaf_ends(90, 7)
    g = _mixed_gens(kind, c, 23)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((90, 3))
    Z = rng.standard_normal((90, 2))
    lhs = Z.T @ M.matmat(c, g, X)
    rhs = TR.matmat_transpose(c, g, Z).T @ X
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    idx = [0, 45, 89]
    assert np.allclose(TR.matmat_transpose_rows(c, g, Z, idx), TR.matmat_transpose(c, g, Z)[idx],
                       rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_transpose_is_an_involution(kind):
    c = T.default_leaf_ends(40, 5)
    g = _mixed_gens(kind, c, 29)
    gtt = TR.transpose_gens(c, TR.transpose_gens(c, g))
    for key, blocks in g.items():
        if key == "kind":
            continue
        for a, b in zip(blocks, gtt[key]):
            assert (a is None and b is None) or np.array_equal(np.asarray(a), np.asarray(b)), key


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_transpose_of_symmetric_closed_form(fmt):
    """T^{-1} of tridiag(-1, 2, -1) is symmetric: A^T X = A X (closed form,
    min(i,j)(n+1-max(i,j))/(n+1))."""
    n = 77
    c = T.default_leaf_ends(n, 9)
    g = W.tridiag_inverse_hodlr(c) if fmt == "hodlr" else W.tridiag_inverse_hss(c)
    X = np.random.default_rng(6).standard_normal((n, 2))
    i = np.arange(1, n + 1)
    Tinv = np.minimum.outer(i, i) * (n + 1 - np.maximum.outer(i, i)) / (n + 1)
    assert np.allclose(TR.matmat_transpose(c, g, X), Tinv @ X, rtol=1e-12, atol=1e-12)


def _bad_transpose(plant):
    orig = TR.transpose_gens

    def bad(c_, g_):
        gt = orig(c_, g_)
        if plant == "hss_b12_not_b21":
            gt["B12"] = [np.asfortranarray(B.T) for B in g_["B12"]]
        elif plant == "hss_ru_kept":
            gt["RU"] = list(g_["RU"])
        elif plant == "hss_untransposed_coupling":
            gt["B12"] = list(g_["B21"])
        elif plant == "hodlr_u12_from_v12":
            gt["U12"] = list(g_["V12"])
        elif plant == "leaf_d_kept":
            gt["D"] = list(g_["D"])
        return gt
    return bad


@pytest.mark.parametrize("plant", ["hss_b12_not_b21", "hss_ru_kept", "hss_untransposed_coupling",
                                   "hodlr_u12_from_v12", "leaf_d_kept"])
def test_transpose_planted_mistakes(monkeypatch, plant):
    c = [6, 12, 18, 24, 30, 36, 42, 48]
    kind = "hodlr" if plant.startswith("hodlr") else "hss"
    rng = np.random.default_rng(37)
    if kind == "hodlr":
        g = W.random_hodlr(rng, c, 3)
    else:
        g = W.random_hss(rng, c, 3, orthonormal=False)
    ref = brute_dense(c, g).T
    monkeypatch.setattr(TR, "transpose_gens", _bad_transpose(plant))
    got = brute_dense(c, TR.transpose_gens(c, g))
    assert not np.allclose(got, ref, rtol=1e-6, atol=1e-6), plant


# --------------------------------------------------------------------------
# hss2hodlr (Sec. 3.5)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,c", SMALL_TREES + [("variable_p3", T.default_leaf_ends(40, 5))])
def test_hss_to_hodlr_brute_force(name, c):
    """Every entry of the converted HODLR generators, evaluated on its own,
    equals the HSS entry (rank per node differs between rows and columns)."""
    g = _mixed_gens("hss", c, 41)
    h = CV.hss_to_hodlr(c, g)
    assert np.allclose(brute_dense(c, h), brute_dense(c, g), rtol=1e-13, atol=1e-13), name
    L = len(c)
    for q in range(L - 1):
        a, b = T.children(q)
        kv = lambda x: (np.asarray(g["V"][x - (L - 1)]).shape[1] if x >= L - 1 else g["RV"][x].shape[1])
        assert h["U12"][q].shape[1] == kv(b) and h["U21"][q].shape[1] == kv(a)


def test_hss_to_hodlr_products_and_rejects_hodlr():
    c = T.default_leaf_ends(120, 9)
    g = _mixed_gens("hss", c, 43)
    X = np.random.default_rng(8).standard_normal((120, 4))
    assert np.allclose(M.matmat(c, CV.hss_to_hodlr(c, g), X), M.matmat(c, g, X), rtol=1e-12, atol=1e-12)
    with pytest.raises(ValueError):
        CV.hss_to_hodlr(c, _mixed_gens("hodlr", c, 1))


@pytest.mark.parametrize("plant", ["b12_for_b21", "v_from_wrong_child", "rv_in_row_bases"])
def test_hss_to_hodlr_planted_mistakes(monkeypatch, plant):
    c = [6, 12, 18, 24, 30, 36, 42, 48]
    g = W.random_hss(np.random.default_rng(47), c, 3, orthonormal=False)
    ref = brute_dense(c, g)
    orig = CV.hss_to_hodlr

    def bad(c_, g_):
        h = orig(c_, g_)
        Ub, Vb = dense.hss_bases(c_, g_)
        for q in range(len(c_) - 1):
            a, b = T.children(q)
            if plant == "b12_for_b21":
                h["U21"][q] = Ub[b] @ g_["B12"][q].T
            elif plant == "v_from_wrong_child":
                h["V12"][q] = Vb[a] if Vb[a].shape == Vb[b].shape else h["V12"][q]
            elif plant == "rv_in_row_bases":
                Uw, _ = dense.hss_bases(c_, dict(g_, RU=g_["RV"]))
                h["U12"][q] = Uw[a] @ g_["B12"][q]
        return h
    monkeypatch.setattr(CV, "hss_to_hodlr", bad)
    got = brute_dense(c, CV.hss_to_hodlr(c, g))
    assert not np.allclose(got, ref, rtol=1e-6, atol=1e-6), plant


# --------------------------------------------------------------------------
# Hadamard product (Sec. 4.4, Eq. 4.1, Fig. 4.3)
# --------------------------------------------------------------------------

def test_khatri_rao_t_definition():
    C_ = np.arange(6.0).reshape(3, 2)
    D_ = np.arange(9.0).reshape(3, 3) + 1
    KR = HD.khatri_rao_t(C_, D_)
    for i in range(3):
        for a1 in range(2):
            for a2 in range(3):
                assert KR[i, a1 * 3 + a2] == C_[i, a1] * D_[i, a2]


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SMALL_TREES + [("variable_p3", T.default_leaf_ends(40, 5))])
def test_hadamard_brute_force(kind, name, c):
    """Every entry of the Hadamard generators, evaluated on its own, is the
    product of the entries of A and B (ranks differ per node and between A and B)."""
    gA = _mixed_gens(kind, c, 51)
    rng = np.random.default_rng(52)
    if kind == "hodlr":
        gB = W.random_hodlr(rng, c, lambda q: (1 + (q * 5) % 2, 1 + q % 2))
    else:
        gB = W.random_hss(rng, c, lambda q: (1 + (q * 5) % 2, 2 + q % 2), orthonormal=False)
    gC = HD.hadamard_gens(c, gA, gB)
    assert np.allclose(brute_dense(c, gC), brute_dense(c, gA) * brute_dense(c, gB), rtol=1e-12, atol=1e-12), name


def test_hadamard_with_ones_is_identity_map():
    """A o ones = A, with the all-ones matrix in its exact rank-1 form."""
    c = T.default_leaf_ends(37, 4)
    for kind in ("hodlr", "hss"):
        gA = _gens(kind, c, 55)
        gO = W.ones_hodlr(c) if kind == "hodlr" else W.ones_hss(c)
        X = np.random.default_rng(2).standard_normal((37, 3))
        assert np.allclose(M.matmat(c, HD.hadamard_gens(c, gA, gO), X), M.matmat(c, gA, X), rtol=1e-12, atol=1e-12)


def test_hadamard_rejects_mixed_kinds():
    c = T.default_leaf_ends(20, 5)
    with pytest.raises(ValueError):
        HD.hadamard_gens(c, _gens("hodlr", c, 1), _gens("hss", c, 2))


@pytest.mark.parametrize("plant", ["kron_of_stacked_r", "swapped_kr_order", "b12_from_b21"])
def test_hadamard_planted_mistakes(monkeypatch, plant):
    c = [6, 12, 18, 24, 30, 36, 42, 48]
    rng = np.random.default_rng(57)
    gA = W.random_hss(rng, c, 2, orthonormal=False)
    gB = W.random_hss(rng, c, 3, orthonormal=False)
    ref = brute_dense(c, gA) * brute_dense(c, gB)
    orig = HD.hadamard_gens

    def bad(c_, a_, b_):
        gC = orig(c_, a_, b_)
        for q in range(1, len(c_) - 1):
            if plant == "kron_of_stacked_r":
                K = np.kron(a_["RU"][q], b_["RU"][q])
                gC["RU"][q] = K[:gC["RU"][q].shape[0]]
        if plant == "swapped_kr_order":
            gC["U"] = [HD.khatri_rao_t(b, a) for a, b in zip(a_["U"], b_["U"])]
        if plant == "b12_from_b21":
            gC["B12"] = [np.kron(a, b) for a, b in zip(a_["B21"], b_["B21"])]
        return gC
    monkeypatch.setattr(HD, "hadamard_gens", bad)
    got = brute_dense(c, HD.hadamard_gens(c, gA, gB))
    assert not np.allclose(got, ref, rtol=1e-6, atol=1e-6), plant


# --------------------------------------------------------------------------
# Y = A^{-1} B (Sec. 4.3, `A\\v` of Table 4.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", [t for t in SMALL_TREES if int(t[1][-1]) > 0])
def test_solve_against_brute_force(kind, name, c):
    """The independently evaluated dense A times the oracle's solution gives B."""
    g = _gens(kind, c, 61)
    n = int(c[-1])
    B = np.random.default_rng(3).standard_normal((n, 3))
    Y = SV.solve_dense(c, g, B)
    Ab = brute_dense(c, g)
    assert np.allclose(Ab @ Y, B, rtol=1e-10, atol=1e-10), name


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_solve_closed_form_tridiag_inverse(fmt):
    """A = T^{-1} for T = tridiag(-1, 2, -1): A^{-1} b = T b."""
    n = 77
    c = T.default_leaf_ends(n, 9)
    g = W.tridiag_inverse_hodlr(c) if fmt == "hodlr" else W.tridiag_inverse_hss(c)
    b = np.random.default_rng(2).standard_normal((n, 2))
    Y = SV.solve_dense(c, g, b)
    assert np.allclose(Y, _tridiag(n) @ b, rtol=1e-9, atol=1e-9)


def test_solve_frobenius_and_residual():
    c = T.default_leaf_ends(60, 8)
    for kind in ("hodlr", "hss"):
        g = _mixed_gens(kind, c, 63)
        Ab = brute_dense(c, g)
        assert np.isclose(SV.frobenius(c, g), np.linalg.norm(Ab), rtol=1e-13)
        B = np.random.default_rng(4).standard_normal((60, 2))
        Y = SV.solve_dense(c, g, B)
        assert SV.residual(c, g, Y, B) <= 1e-14
        assert SV.residual(c, g, Y + 1e-3, B) > 1e-6
        assert np.isclose(SV.residual(c, g, np.zeros_like(B), B), 1.0)


def test_solve_planted_mistake_transposed_matrix(monkeypatch):
    """Solving with A^T instead of A fails the brute-force pin (A is not symmetric)."""
    c = [6, 12, 18, 24, 30, 36, 42, 48]
    g = _gens("hss", c, 65, k=3)
    B = np.random.default_rng(5).standard_normal((48, 2))
    orig = dense.dense
    monkeypatch.setattr(dense, "dense", lambda c_, g_: orig(c_, g_).T)
    Y = SV.solve_dense(c, g, B)
    assert not np.allclose(brute_dense(c, g) @ Y, B, rtol=1e-6, atol=1e-6)
