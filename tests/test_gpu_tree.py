"""The tree phases in one cluster launch against the per-level kernels.

Both run the same sums in the same order (Sec. 4.1, Fig. 4.1: the HSS
upsweep through R_V with the B couplings and the downsweep through R_U; the
HODLR per-level sums), so the products must agree bit for bit; the cluster
results are also held to the oracle's bound.  Shapes cover trees shallower
than a full cluster (p = 1, 2), subtrees of one leaf, uneven ranks
(Kp != Ke), ragged column chunks and shapes that do not fit (the level
kernels then run).
"""

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, matmat as OM, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")


def _gens(kind, c, seed, k):
    rng = np.random.default_rng(seed)
    if kind == "hodlr":
        return W.random_hodlr(rng, c, k)
    return W.random_hss(rng, c, k, orthonormal=False)


CASES = [
    ("hss_p1", "hss", [100, 200], 8, 3),
    ("hss_p2", "hss", OT.default_leaf_ends(400, 100), 8, 5),
    ("hss_p3_one_leaf_subtrees", "hss", OT.default_leaf_ends(800, 100), 16, 9),
    ("hss_p5", "hss", OT.default_leaf_ends(3200, 100), 8, 16),
    ("hss_p8_r64", "hss", OT.default_leaf_ends(65536 // 4, 64), 32, 64),
    ("hss_p6_r1", "hss", OT.default_leaf_ends(4096, 64), 16, 1),
    ("hss_p7_r33", "hss", OT.default_leaf_ends(8192, 64), 8, 33),
    ("hodlr_p2", "hodlr", OT.default_leaf_ends(400, 100), 4, 3),
    ("hodlr_p4_r17", "hodlr", OT.default_leaf_ends(1600, 100), 6, 17),
    ("hodlr_p8_r64", "hodlr", OT.default_leaf_ends(16384, 64), 4, 64),
    ("hss_empty_leaf", "hss", [300, 600, 600, 900], 8, 6),
]


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("name,kind,c,k,r", CASES)
def test_cluster_tree_matches_level_kernels(storage, name, kind, c, k, r):
    g = _gens(kind, c, 7, k)
    n = int(c[-1])
    xt = "f64" if storage == "f64" else "f32"
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), xt)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    Xd = H.to_dev(X, xt)
    od = torch.float64 if storage == "f64" else torch.float32
    A.set_tree(1)
    y_level = H.to_host(A.matmat(Xd, out_dtype=od))
    A.set_tree(2)
    y_cluster = H.to_host(A.matmat(Xd, out_dtype=od))
    A.set_tree(0)
    y_auto = H.to_host(A.matmat(Xd, out_dtype=od))
    hm.device_status()
    assert np.array_equal(y_level, y_cluster), name + ": cluster and level tree kernels differ"
    assert np.array_equal(y_cluster, y_auto)
    ref = OM.matmat(c, g, X)
    info = A.info()
    tc = storage in ("bf16", "bf16x2") and r >= 16
    fac = H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=tc)
    H.check_bound(y_cluster, ref, OB.envelope(c, g, X), fac, name)
    if storage == "f64":
        assert H.col_rel_err(y_cluster, ref) <= 1e-12


@pytest.mark.parametrize("ranks", [lambda q: (16, 8), lambda q: (8, 16),
                                   lambda q: (4 + 4 * (q % 3), 8 + 8 * (q % 2))])
def test_cluster_tree_uneven_ranks(ranks):
    """HSS with U and V ranks that differ (Kp != Ke) and vary by node."""
    c = OT.default_leaf_ends(4096, 128)
    rng = np.random.default_rng(11)
    g = W.random_hss(rng, c, ranks, orthonormal=False)
    n = int(c[-1])
    X = H.exact_input(rng.standard_normal((n, 24)), "f32")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f32")
    Xd = H.to_dev(X, "f32")
    A.set_tree(1)
    y1 = H.to_host(A.matmat(Xd))
    A.set_tree(2)
    y2 = H.to_host(A.matmat(Xd))
    hm.device_status()
    assert np.array_equal(y1, y2)
    ref = OM.matmat(c, g, X)
    info = A.info()
    H.check_bound(y2, ref, OB.envelope(c, g, X),
                  H.bound_factor("f32", "hss", info["depth"], H.acc_length(info, "hss")), "uneven ranks")


def test_cluster_tree_deep_tree_falls_back():
    """p = 11 is deeper than the cluster layout takes: mode 2 runs the level kernels."""
    c = OT.default_leaf_ends(2048 * 8, 8)
    g = _gens("hss", c, 3, 4)
    X = H.exact_input(np.random.default_rng(2).standard_normal((2048 * 8, 8)), "f64")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    assert A.info()["depth"] == 11
    Xd = H.to_dev(X, "f64")
    A.set_tree(1)
    y1 = H.to_host(A.matmat(Xd))
    A.set_tree(2)
    y2 = H.to_host(A.matmat(Xd))
    hm.device_status()
    assert np.array_equal(y1, y2)
    assert H.col_rel_err(y2, OM.matmat(c, g, X)) <= 1e-12


def test_set_tree_rejects_bad_mode():
    c = OT.default_leaf_ends(256, 64)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), _gens("hss", c, 1, 4), "f32")
    with pytest.raises(hm.HMError):
        A.set_tree(3)


@pytest.mark.parametrize("storage", ["f64", "bf16"])
@pytest.mark.parametrize("name,kind,c,k,r", [CASES[3], CASES[4], CASES[8]])
def test_tuned_tree_shape_changes_no_bit(storage, name, kind, c, k, r):
    """hm_matrix_tune_tree picks a launch shape by timing; every shape sums in
    the same order, so the product is bit-identical to the per-level kernels'."""
    g = _gens(kind, c, 9, k)
    n = int(c[-1])
    xt = "f64" if storage == "f64" else "f32"
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), xt)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    Xd = H.to_dev(X, xt)
    od = torch.float64 if storage == "f64" else torch.float32
    A.set_tree(1)
    y_level = H.to_host(A.matmat(Xd, out_dtype=od))
    A.set_tree(0)
    ms = A.tune_tree(r)
    assert ms is not None and ms > 0
    y_tuned = H.to_host(A.matmat(Xd, out_dtype=od))
    info = A.info()
    assert info["tree_cluster"] > 0
    assert np.array_equal(y_level, y_tuned), name


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_pinned_tree_shapes_change_no_bit(storage):
    """hm_matrix_set_tree_shape: every shape that fits gives the per-level
    kernels' bits; values outside the allowed sets are rejected."""
    c = OT.default_leaf_ends(4096, 64)
    g = _gens("hss", c, 9, 12)
    n = int(c[-1])
    r = 8
    xt = "f64" if storage == "f64" else "f32"
    X = H.exact_input(np.random.default_rng(5).standard_normal((n, r)), xt)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    Xd = H.to_dev(X, xt)
    od = torch.float64 if storage == "f64" else torch.float32
    A.set_tree(1)
    y_level = H.to_host(A.matmat(Xd, out_dtype=od))
    A.set_tree(0)
    tried = 0
    for cl in (2, 4, 8, 16):
        for cols in (1, 2, 4, 8):
            for ns in (2, 3, 5, 8, 12):
                try:
                    A.set_tree_shape(r, cl, cols, ns)
                except hm.HMError as e:
                    assert e.status == hm._lib.HM_EUNSUPPORTED, (cl, cols, ns, e)
                    continue
                tried += 1
                y = H.to_host(A.matmat(Xd, out_dtype=od))
                info = A.info()
                assert (info["tree_cluster"], info["tree_columns"], info["tree_ring"]) == (cl, cols, ns)
                assert np.array_equal(y_level, y), (cl, cols, ns)
    assert tried >= 8
    for bad in ((3, 8, 3), (32, 8, 3), (4, 3, 3), (4, 8, 1), (4, 8, 13)):
        with pytest.raises(hm.HMError) as ei:
            A.set_tree_shape(r, *bad)
        assert ei.value.status == hm._lib.HM_EINVAL, bad
