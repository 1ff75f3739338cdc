"""Parity of hss2hodlr on the GPU (hm_hss_to_hodlr): the converted HODLR
matrix multiplies like the HSS matrix it came from.

References: the oracle's product with the HSS generators and with the
oracle's own converted generators (oracle/convert.py, pinned by brute
force).  FP64: per-column relative error <= 1e-12.  Reduced storage: every
entry inside the HSS bound of the parity tests plus two more roundings to the
storage type (the converted U and V factors are rounded once each).
"""

import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, convert as OCV, matmat as OM, tree as OT
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


def _mixed(c, seed):
    rng = np.random.default_rng(seed)
    return W.random_hss(rng, c, lambda q: (3 + q % 6, 9 + (q * 7) % 5), orthonormal=False)


def _convert(c, g, storage):
    S = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    return S, S.to_hodlr()


@pytest.mark.parametrize("name,c", SMALL)
@pytest.mark.parametrize("r", [1, 8, 33])
def test_f64_converted_small_trees(name, c, r):
    g = _mixed(c, 300 + r)
    n = int(c[-1])
    X = np.random.default_rng(r).standard_normal((n, r))
    _, Hm = _convert(c, g, "f64")
    Y = H.to_host(Hm.matmat(H.to_dev(X, "f64"), out_dtype=torch.float64))
    ref = OM.matmat(c, g, X)
    assert H.col_rel_err(Y, ref) <= 1e-12, name
    assert H.col_rel_err(Y, OM.matmat(c, OCV.hss_to_hodlr(c, g), X)) <= 1e-12, name


def _reduced_factor(storage, info, p):
    return H.bound_factor(storage, "hss", p, H.acc_length(info, "hodlr"), tensor_core=True) + 2 * H.UNIT[storage]


@pytest.mark.parametrize("storage,xt", [("f32", "f32"), ("bf16", "bf16"), ("bf16", "f32"), ("bf16x2", "f32")])
@pytest.mark.parametrize("r", [5, 40])
def test_reduced_converted_within_bound(storage, xt, r):
    c = OT.default_leaf_ends(777, 64)
    g = _mixed(c, 19 + r)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), xt)
    _, Hm = _convert(c, g, storage)
    Y = H.to_host(Hm.matmat(H.to_dev(X, xt), out_dtype=torch.float32))
    ref = OM.matmat(c, g, X)
    info = Hm.info()
    H.check_bound(Y, ref, OB.envelope(c, g, X), _reduced_factor(storage, info, info["depth"]), storage)


@pytest.mark.parametrize("storage", ["bf16", "bf16x2"])
@pytest.mark.parametrize("name,c,r", [("uniform_m256_r64", [256 * (i + 1) for i in range(16)], 64),
                                      ("ragged_r33", OT.default_leaf_ends(3001, 200), 33)])
def test_converted_tensor_core_and_simt(storage, name, c, r):
    g = _mixed(c, 53)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), "f32")
    _, Hm = _convert(c, g, storage)
    Xd = H.to_dev(X, "f32")
    Hm.set_path(2)
    Yt = H.to_host(Hm.matmat(Xd, out_dtype=torch.float32))
    Hm.set_path(1)
    Ys = H.to_host(Hm.matmat(Xd, out_dtype=torch.float32))
    hm.device_status()
    ref = OM.matmat(c, g, X)
    info = Hm.info()
    fac = _reduced_factor(storage, info, info["depth"])
    env = OB.envelope(c, g, X)
    H.check_bound(Yt, ref, env, fac, name + " tensor cores")
    H.check_bound(Ys, ref, env, fac, name + " simt")


def test_converted_structure():
    c = OT.default_leaf_ends(2048, 256)
    g = W.random_hss(np.random.default_rng(3), c, (8, 16), orthonormal=False)
    S, Hm = _convert(c, g, "f32")
    si, hi = S.info(), Hm.info()
    assert hi["kind"] == hm.HM_HODLR and si["kind"] == hm.HM_HSS
    assert (hi["depth"], hi["num_leaves"], hi["leaf_pad"], hi["n"]) == (si["depth"], si["num_leaves"],
                                                                        si["leaf_pad"], si["n"])
    assert hi["rank_total"] == si["depth"] * si["rank_col"] == 3 * 16
    m = 256
    assert hi["generator_elements"] == 2048 * m + 2 * 2048 * 3 * 16
    assert Hm.generator_bytes() == hi["generator_elements"] * 4


def test_converted_full_size_sampled_rows():
    """HSS n = 65536, leaf 256, rank 32, r = 64, BF16: converted product on sampled rows."""
    cfg = W.workload("hss_n65536_m256_k32_r64")
    rng = W.rng_named("hss_n65536_m256_k32_r64")
    c = OT.default_leaf_ends(cfg["n"], cfg["m"])
    g = W.random_hss(rng, c, cfg["k"])
    X = rng.standard_normal((cfg["n"], cfg["r"]))
    Xe = H.exact_input(X, "bf16")
    _, Hm = _convert(c, g, "bf16")
    Y = H.to_host(Hm.matmat(H.to_dev(Xe, "bf16"), out_dtype=torch.float32))
    rows = sorted(set([0, cfg["n"] - 1, 255, 256, 32767, 32768] +
                      [int(v) for v in np.random.default_rng(5).integers(0, cfg["n"], 90)]))
    ref = OM.matmat_rows(c, g, Xe, rows)
    info = Hm.info()
    H.check_bound(Y[rows], ref, OB.envelope_rows(c, g, Xe, rows), _reduced_factor("bf16", info, info["depth"]),
                  "bf16")


def test_converted_then_transposed_matches_transposed_then_converted_f64():
    c = OT.default_leaf_ends(900, 100)
    g = _mixed(c, 71)
    S = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    A1 = S.to_hodlr().transpose()
    A2 = S.transpose().to_hodlr()
    X = H.to_dev(np.random.default_rng(9).standard_normal((900, 6)), "f64")
    Y1 = H.to_host(A1.matmat(X, out_dtype=torch.float64))
    Y2 = H.to_host(A2.matmat(X, out_dtype=torch.float64))
    assert H.col_rel_err(Y1, Y2) <= 1e-13


def test_convert_rejects_bad_input():
    lib = hm._lib.lib
    out = C.c_void_p()
    c = [64, 128]
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), W.random_hodlr(np.random.default_rng(1), c, 3), "f64")
    assert lib.hm_hss_to_hodlr(A._h, C.byref(out)) == hm._lib.HM_EINVAL
    assert out.value is None
    assert lib.hm_hss_to_hodlr(None, C.byref(out)) == hm._lib.HM_EINVAL
    S = hm.Matrix.create(hm.Tree.from_leaf_ends(c), _mixed(c, 2), "f64")
    assert lib.hm_hss_to_hodlr(S._h, None) == hm._lib.HM_EINVAL
