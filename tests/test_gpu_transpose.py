"""Parity of the transposed product A^T X (hm_matrix_transpose, then the
ordinary product) with the oracle's A^T X through the C ABI.

The oracle relabels the generators by the block definition
(A^T)(I, J) = A(J, I)^T (oracle/transpose.py, pinned by brute force); the
CUDA side permutes A's device storage.  Tolerances are those of the
parity tests: FP64 per-column relative error <= 1e-12 and every entry inside
the componentwise bound; reduced storage inside (c_round u_s + gamma_L) times
the envelope of the transposed generators.
"""

import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, matmat as OM, transpose as OTR, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")

SMALL = [
    ("uniform_p3", [32 * (i + 1) for i in range(8)]),
    ("ragged", OT.default_leaf_ends(301, 40)),
    ("empty_leaves", [5, 9, 17, 17]),
    ("empty_first", [0, 70, 120, 200]),
    ("single_leaf", [57]),
    ("p1", [100, 190]),
    ("deep_p6", OT.default_leaf_ends(700, 11)),
]


def _mixed(kind, c, seed):
    """Row and column ranks that differ per node, so swapped factors show."""
    rng = np.random.default_rng(seed)
    if kind == "hodlr":
        return W.random_hodlr(rng, c, lambda q: (2 + q % 5, 4 + q % 3))
    return W.random_hss(rng, c, lambda q: (3 + q % 6, 9 + (q * 7) % 5), orthonormal=False)


def _transposed(c, g, storage):
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    return A, A.transpose()


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SMALL)
@pytest.mark.parametrize("r", [1, 8, 33])
def test_f64_transpose_small_trees(kind, name, c, r):
    g = _mixed(kind, c, 200 + r)
    n = int(c[-1])
    X = np.random.default_rng(r).standard_normal((n, r))
    _, At = _transposed(c, g, "f64")
    Y = H.to_host(At.matmat(H.to_dev(X, "f64"), out_dtype=torch.float64))
    gt = OTR.transpose_gens(c, g)
    ref = OM.matmat(c, gt, X)
    assert H.col_rel_err(Y, ref) <= 1e-12, name
    info = At.info()
    H.check_bound(Y, ref, OB.envelope(c, gt, X),
                  H.bound_factor("f64", kind, info["depth"], H.acc_length(info, kind)), name)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("storage,xt", [("f32", "f32"), ("bf16", "bf16"), ("bf16", "f32"), ("bf16x2", "f32")])
@pytest.mark.parametrize("r", [5, 40])
def test_reduced_precision_transpose_within_bound(kind, storage, xt, r):
    c = OT.default_leaf_ends(777, 64)
    g = _mixed(kind, c, 9 + r)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), xt)
    _, At = _transposed(c, g, storage)
    Y = H.to_host(At.matmat(H.to_dev(X, xt), out_dtype=torch.float32))
    gt = OTR.transpose_gens(c, g)
    ref = OM.matmat(c, gt, X)
    info = At.info()
    H.check_bound(Y, ref, OB.envelope(c, gt, X),
                  H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=True),
                  storage)


TC_CASES = [
    ("hss_uniform_m256_r64", "hss", [256 * (i + 1) for i in range(16)], 64),
    ("hodlr_ragged_m144_r20", "hodlr", OT.default_leaf_ends(4600, 150), 20),
    ("hss_ragged_r33", "hss", OT.default_leaf_ends(3001, 200), 33),
    ("hss_empty_leaf_r48", "hss", [300, 600, 600, 900], 48),
]


@pytest.mark.parametrize("storage", ["bf16", "bf16x2"])
@pytest.mark.parametrize("name,kind,c,r", TC_CASES)
def test_transpose_tensor_core_and_simt(storage, name, kind, c, r):
    g = _mixed(kind, c, 43)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), "f32")
    _, At = _transposed(c, g, storage)
    Xd = H.to_dev(X, "f32")
    At.set_path(2)
    Yt = H.to_host(At.matmat(Xd, out_dtype=torch.float32))
    At.set_path(1)
    Ys = H.to_host(At.matmat(Xd, out_dtype=torch.float32))
    hm.device_status()
    gt = OTR.transpose_gens(c, g)
    ref = OM.matmat(c, gt, X)
    info = At.info()
    fac = H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=True)
    env = OB.envelope(c, gt, X)
    H.check_bound(Yt, ref, env, fac, name + " tensor cores")
    H.check_bound(Ys, ref, env, fac, name + " simt")


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "bf16x2"])
def test_transpose_twice_is_bit_identical(kind, storage):
    """Every stored value is copied: (A^T)^T multiplies exactly like A."""
    c = OT.default_leaf_ends(2100, 200)
    g = _mixed(kind, c, 51)
    A, At = _transposed(c, g, storage)
    Att = At.transpose()
    xt = "f64" if storage == "f64" else "f32"
    X = H.to_dev(np.random.default_rng(2).standard_normal((2100, 24)), xt)
    od = torch.float64 if storage == "f64" else torch.float32
    Y1 = A.matmat(X, out_dtype=od)
    Y2 = Att.matmat(X, out_dtype=od)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)
    ia, it, itt = A.info(), At.info(), Att.info()
    assert A.generator_bytes() == At.generator_bytes() == Att.generator_bytes()
    assert (it["depth"], it["num_leaves"]) == (ia["depth"], ia["num_leaves"])
    assert itt == ia


def test_transpose_swaps_row_and_column_ranks():
    c = OT.default_leaf_ends(1024, 128)
    rng = np.random.default_rng(8)
    g = W.random_hss(rng, c, (8, 24), orthonormal=False)
    A, At = _transposed(c, g, "f32")
    ia, it = A.info(), At.info()
    assert (ia["rank_total"], ia["rank_col"]) == (8, 24)
    assert (it["rank_total"], it["rank_col"]) == (24, 8)


def test_transpose_adjoint_identity_full_size():
    """<Z, A X> = <A^T Z, X> on the n = 65536, leaf 256, rank 32 HSS matrix (FP64)."""
    cfg = W.workload("hss_n65536_m256_k32_r64")
    rng = W.rng_named("hss_n65536_m256_k32_r64", salt=5)
    c = OT.default_leaf_ends(cfg["n"], cfg["m"])
    g = W.random_hss(rng, c, cfg["k"])
    A, At = _transposed(c, g, "f64")
    X = rng.standard_normal((cfg["n"], 4))
    Z = rng.standard_normal((cfg["n"], 3))
    AX = H.to_host(A.matmat(H.to_dev(X, "f64"), out_dtype=torch.float64))
    ATZ = H.to_host(At.matmat(H.to_dev(Z, "f64"), out_dtype=torch.float64))
    lhs = Z.T @ AX
    rhs = ATZ.T @ X
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-9 * np.abs(lhs).max())


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_transpose_full_size_sampled_rows(storage):
    """A^T X for the HSS n = 65536, leaf 256, rank 32, r = 64 matrix; oracle on sampled rows."""
    cfg = W.workload("hss_n65536_m256_k32_r64")
    rng = W.rng_named("hss_n65536_m256_k32_r64")
    c = OT.default_leaf_ends(cfg["n"], cfg["m"])
    g = W.random_hss(rng, c, cfg["k"])
    X = rng.standard_normal((cfg["n"], cfg["r"]))
    xt = "f64" if storage == "f64" else "bf16"
    Xe = H.exact_input(X, xt)
    _, At = _transposed(c, g, storage)
    Y = H.to_host(At.matmat(H.to_dev(Xe, xt), out_dtype=torch.float64 if storage == "f64" else torch.float32))
    rs = np.random.default_rng(3)
    rows = sorted(set([0, cfg["n"] - 1, 255, 256, 32767, 32768] + [int(v) for v in rs.integers(0, cfg["n"], 90)]))
    gt = OTR.transpose_gens(c, g)
    ref = OM.matmat_rows(c, gt, Xe, rows)
    info = At.info()
    if storage == "f64":
        assert H.col_rel_err(Y[rows], ref) <= 1e-12
    H.check_bound(Y[rows], ref, OB.envelope_rows(c, gt, Xe, rows),
                  H.bound_factor(storage, "hss", info["depth"], H.acc_length(info, "hss"), tensor_core=True),
                  storage)


def test_transpose_in_a_batch_matches_alone():
    c1 = OT.default_leaf_ends(3000, 256)
    c2 = OT.default_leaf_ends(1500, 128)
    A1, T1 = _transposed(c1, _mixed("hss", c1, 61), "bf16")
    A2, T2 = _transposed(c2, _mixed("hodlr", c2, 62), "f32")
    mats = [A1, T1, A2, T2]
    rs = [16, 16, 5, 5]
    gen = torch.Generator(device="cuda").manual_seed(4)
    Xs = [torch.randn((r, m.tree.shape()[0]), generator=gen, device="cuda").t() for r, m in zip(rs, mats)]
    B = hm.Batch(mats, rs)
    Ys = [torch.full((r, X.shape[0]), float("nan"), dtype=torch.float32, device="cuda").t() for r, X in zip(rs, Xs)]
    B.run(Xs, Ys)
    singles = [m.matmat(X, out_dtype=torch.float32) for m, X in zip(mats, Xs)]
    torch.cuda.synchronize()
    for j in range(len(mats)):
        assert torch.equal(Ys[j], singles[j]), j


def test_transpose_bad_arguments():
    lib = hm._lib.lib
    out = C.c_void_p()
    assert lib.hm_matrix_transpose(None, C.byref(out)) == hm._lib.HM_EINVAL
    assert out.value is None
    c = [64, 128]
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), _mixed("hodlr", c, 1), "f64")
    assert lib.hm_matrix_transpose(A._h, None) == hm._lib.HM_EINVAL
    tree = hm.Tree.from_leaf_ends(c)
    assert lib.hm_matrix_transpose(tree._h, C.byref(out)) == hm._lib.HM_EINVAL
