"""Batched products: one persistent launch per phase over many matrices.

Every product keeps its own blocking in the batch, so each batched result
must be bit-identical to the same product run alone; a few are also checked
against the oracle.  Graph replay, tuning and the tuning cache are covered.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, matmat as OM, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")


def _mixed(seed=0, count=12):
    rng = np.random.default_rng(seed)
    spec = [("hodlr", "f32", 900, 4, 1), ("hss", "bf16", 2048, 16, 20), ("hodlr", "bf16", 3000, 8, 33),
            ("hss", "f32", 1500, 8, 7), ("hss", "bf16x2", 4096, 32, 16), ("hodlr", "bf16x2", 777, 6, 3),
            ("hss", "bf16", 1024, 4, 1), ("hodlr", "f32", 5000, 16, 12), ("hss", "f32", 300, 8, 40),
            ("hodlr", "bf16", 2600, 12, 64), ("hss", "bf16x2", 1800, 8, 2), ("hodlr", "f32", 64, 2, 5)]
    out = []
    for kind, st, n, k, r in spec[:count]:
        c = OT.default_leaf_ends(n, 256 if n > 1000 else 64)
        g = W.random_hodlr(rng, c, k) if kind == "hodlr" else W.random_hss(rng, c, k, orthonormal=False)
        X = H.exact_input(rng.standard_normal((n, r)), "f32")
        out.append((kind, st, c, g, X))
    return out


def _make(items):
    mats = [hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, st) for (_, st, c, g, _) in items]
    Xs = [H.to_dev(X, "f32") for (*_, X) in items]
    rs = [X.shape[1] for (*_, X) in items]
    return mats, Xs, rs


def test_batch_bit_identical_to_single_products():
    items = _mixed()
    mats, Xs, rs = _make(items)
    B = hm.Batch(mats, rs)
    Ys = [torch.full((r, X.shape[0]), float("nan"), dtype=torch.float32, device="cuda").t() for r, X in zip(rs, Xs)]
    B.run(Xs, Ys)
    singles = [A.matmat(X, out_dtype=torch.float32) for A, X in zip(mats, Xs)]
    torch.cuda.synchronize()
    for j, (Yb, Ys1) in enumerate(zip(Ys, singles)):
        assert torch.equal(Yb, Ys1), j
    info = B.info()
    assert info["launches_per_run"] <= 6
    hm.device_status()
    # a few against the oracle
    for j in (0, 1, 4):
        kind, st, c, g, X = items[j]
        ref = OM.matmat(c, g, X)
        inf = mats[j].info()
        H.check_bound(H.to_host(Ys[j]), ref, OB.envelope(c, g, X),
                      H.bound_factor(st, kind, inf["depth"], H.acc_length(inf, kind), True), "batch %d" % j)


def test_batch_graph_replay_new_inputs():
    items = _mixed(seed=3, count=8)
    mats, Xs, rs = _make(items)
    B = hm.Batch(mats, rs)
    Ys = [torch.empty((r, X.shape[0]), dtype=torch.float32, device="cuda").t() for r, X in zip(rs, Xs)]
    for rep in range(3):
        Xr = [X * (rep + 1) - rep for X in Xs]
        Xr = [hm.colmajor(x) for x in Xr]
        B.run(Xr, Ys)
        singles = [A.matmat(X, out_dtype=torch.float32) for A, X in zip(mats, Xr)]
        torch.cuda.synchronize()
        for j in range(len(mats)):
            assert torch.equal(Ys[j], singles[j]), (rep, j)
    info = B.info()
    assert info["graph"] == 1, info["capture_error"]


def test_batch_tune_and_cache(tmp_path):
    items = _mixed(seed=5, count=6)
    mats, Xs, rs = _make(items)
    cache = str(tmp_path / "tune.txt")
    B = hm.Batch(mats, rs)
    B.tune(cache)
    assert B.info()["tuned"] == 1
    assert os.path.exists(cache) and open(cache).read().strip()
    B2 = hm.Batch(mats, rs)
    B2.tune(cache)
    i2 = B2.info()
    assert i2["tuned"] == 2
    assert (i2["grid_mult"], i2["rc_cap"], i2["rct_cap"], i2["tile_rows"]) == tuple(
        B.info()[k] for k in ("grid_mult", "rc_cap", "rct_cap", "tile_rows"))
    Ys = [torch.empty((r, X.shape[0]), dtype=torch.float32, device="cuda").t() for r, X in zip(rs, Xs)]
    B2.run(Xs, Ys)
    singles = [A.matmat(X, out_dtype=torch.float32) for A, X in zip(mats, Xs)]
    torch.cuda.synchronize()
    for j in range(len(mats)):
        assert torch.equal(Ys[j], singles[j]), j


def test_batch_rejects_f64_and_empty():
    c = OT.default_leaf_ends(300, 64)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), W.random_hodlr(np.random.default_rng(0), c, 3), "f64")
    with pytest.raises(hm.HMError):
        hm.Batch([A], [2])
    with pytest.raises(hm.HMError):
        hm.Batch([], [])
