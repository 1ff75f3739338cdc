"""Parity of the Hadamard product on the GPU (hm_hadamard): C = A o B built
in device memory multiplies like the oracle's Hadamard generators
(oracle/hadamard.py, pinned by brute force against dense(A) o dense(B)).

FP64: per-column relative error <= 1e-12.  Reduced storage: every entry
inside the parity tests' bound for C's generators plus two more roundings
(each stored product of two entries is rounded once to the storage type).
"""

import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, hadamard as OHD, matmat as OM, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")

SMALL = [
    ("uniform_p3", [32 * (i + 1) for i in range(8)]),
    ("ragged", OT.default_leaf_ends(301, 40)),
    ("empty_leaves", [5, 9, 17, 17]),
    ("single_leaf", [57]),
    ("p1", [100, 190]),
    ("deep_p5", OT.default_leaf_ends(700, 22)),
]


def _pair(kind, c, seed):
    rng = np.random.default_rng(seed)
    if kind == "hodlr":
        return (W.random_hodlr(rng, c, lambda q: (2 + q % 3, 1 + q % 2)),
                W.random_hodlr(rng, c, lambda q: (1 + (q * 5) % 3, 2)))
    return (W.random_hss(rng, c, lambda q: (2 + q % 3, 1 + (q * 7) % 3), orthonormal=False),
            W.random_hss(rng, c, lambda q: (1 + (q * 5) % 2, 2 + q % 2), orthonormal=False))


def _hadamard(c, gA, gB, storage):
    t = hm.Tree.from_leaf_ends(c)
    A = hm.Matrix.create(t, gA, storage)
    B = hm.Matrix.create(t, gB, storage)
    return A, B, A.hadamard(B)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SMALL)
@pytest.mark.parametrize("r", [1, 7, 33])
def test_f64_hadamard_small_trees(kind, name, c, r):
    gA, gB = _pair(kind, c, 400 + r)
    n = int(c[-1])
    X = np.random.default_rng(r).standard_normal((n, r))
    _, _, Cm = _hadamard(c, gA, gB, "f64")
    Y = H.to_host(Cm.matmat(H.to_dev(X, "f64"), out_dtype=torch.float64))
    gC = OHD.hadamard_gens(c, gA, gB)
    ref = OM.matmat(c, gC, X)
    assert H.col_rel_err(Y, ref) <= 1e-12, name
    info = Cm.info()
    H.check_bound(Y, ref, OB.envelope(c, gC, X),
                  H.bound_factor("f64", kind, info["depth"], H.acc_length(info, kind)), name)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("storage,xt", [("f32", "f32"), ("bf16", "bf16"), ("bf16x2", "f32")])
@pytest.mark.parametrize("r", [5, 40])
def test_reduced_hadamard_within_bound(kind, storage, xt, r):
    c = OT.default_leaf_ends(777, 64)
    gA, gB = _pair(kind, c, 29 + r)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), xt)
    _, _, Cm = _hadamard(c, gA, gB, storage)
    Y = H.to_host(Cm.matmat(H.to_dev(X, xt), out_dtype=torch.float32))
    gC = OHD.hadamard_gens(c, gA, gB)
    ref = OM.matmat(c, gC, X)
    info = Cm.info()
    fac = H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=True) + \
        2 * H.UNIT[storage]
    H.check_bound(Y, ref, OB.envelope(c, gC, X), fac, storage)


@pytest.mark.parametrize("storage", ["bf16", "bf16x2"])
@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_hadamard_tensor_core_and_simt(storage, kind):
    c = [256 * (i + 1) for i in range(16)]
    gA, gB = _pair(kind, c, 61)
    X = H.exact_input(np.random.default_rng(3).standard_normal((4096, 48)), "f32")
    _, _, Cm = _hadamard(c, gA, gB, storage)
    Xd = H.to_dev(X, "f32")
    Cm.set_path(2)
    Yt = H.to_host(Cm.matmat(Xd, out_dtype=torch.float32))
    Cm.set_path(1)
    Ys = H.to_host(Cm.matmat(Xd, out_dtype=torch.float32))
    hm.device_status()
    gC = OHD.hadamard_gens(c, gA, gB)
    ref = OM.matmat(c, gC, X)
    info = Cm.info()
    fac = H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=True) + \
        2 * H.UNIT[storage]
    env = OB.envelope(c, gC, X)
    H.check_bound(Yt, ref, env, fac, "tensor cores")
    H.check_bound(Ys, ref, env, fac, "simt")


def test_hadamard_ranks_multiply():
    c = OT.default_leaf_ends(2048, 256)
    rng = np.random.default_rng(5)
    gA = W.random_hss(rng, c, (8, 16), orthonormal=False)
    gB = W.random_hss(rng, c, (2, 3), orthonormal=False)
    A, B, Cm = _hadamard(c, gA, gB, "f32")
    ia, ib, ic = A.info(), B.info(), Cm.info()
    # unpadded ranks multiply (8 x 2, 16 x 3), then pad to 8
    assert (ia["rank_total"], ia["rank_col"], ib["rank_total"], ib["rank_col"]) == (8, 16, 8, 8)
    assert (ic["rank_total"], ic["rank_col"]) == (16, 48)
    h1 = W.random_hodlr(rng, c, 3)
    h2 = W.random_hodlr(rng, c, 2)
    _, _, Ch = _hadamard(c, h1, h2, "f32")
    assert Ch.info()["rank_total"] == 24                 # three levels of rank 6, total padded to 8


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_hadamard_with_ones_is_a(kind):
    c = OT.default_leaf_ends(1000, 120)
    rng = np.random.default_rng(7)
    gA = W.random_hodlr(rng, c, 4) if kind == "hodlr" else W.random_hss(rng, c, 4, orthonormal=False)
    gO = W.ones_hodlr(c) if kind == "hodlr" else W.ones_hss(c)
    A, _, Cm = _hadamard(c, gA, gO, "f64")
    X = H.to_dev(np.random.default_rng(1).standard_normal((1000, 5)), "f64")
    Y1 = H.to_host(A.matmat(X, out_dtype=torch.float64))
    Y2 = H.to_host(Cm.matmat(X, out_dtype=torch.float64))
    assert H.col_rel_err(Y2, Y1) <= 1e-13


def test_hadamard_full_size_sampled_rows():
    """HSS n = 65536, leaf 256: rank 8 o rank 4 = rank 32, BF16, r = 64."""
    cfg = W.workload("hss_n65536_m256_k32_r64")
    rng = W.rng_named("hss_n65536_m256_k32_r64", salt=9)
    c = OT.default_leaf_ends(cfg["n"], cfg["m"])
    gA = W.random_hss(rng, c, 8)
    gB = W.random_hss(rng, c, 4)
    X = rng.standard_normal((cfg["n"], cfg["r"]))
    Xe = H.exact_input(X, "bf16")
    _, _, Cm = _hadamard(c, gA, gB, "bf16")
    assert Cm.info()["rank_total"] == 32
    Y = H.to_host(Cm.matmat(H.to_dev(Xe, "bf16"), out_dtype=torch.float32))
    rows = sorted(set([0, cfg["n"] - 1, 255, 256, 32767, 32768] +
                      [int(v) for v in np.random.default_rng(4).integers(0, cfg["n"], 60)]))
    gC = OHD.hadamard_gens(c, gA, gB)
    ref = OM.matmat_rows(c, gC, Xe, rows)
    info = Cm.info()
    fac = H.bound_factor("bf16", "hss", info["depth"], H.acc_length(info, "hss"), tensor_core=True) + \
        2 * H.UNIT["bf16"]
    H.check_bound(Y[rows], ref, OB.envelope_rows(c, gC, Xe, rows), fac, "bf16")


def test_hadamard_rejects_mismatched_operands():
    lib = hm._lib.lib
    out = C.c_void_p()
    c = [64, 128]
    t = hm.Tree.from_leaf_ends(c)
    Ah = hm.Matrix.create(t, W.random_hodlr(np.random.default_rng(1), c, 2), "f64")
    As = hm.Matrix.create(t, W.random_hss(np.random.default_rng(2), c, 2, orthonormal=False), "f64")
    Af = hm.Matrix.create(t, W.random_hodlr(np.random.default_rng(3), c, 2), "f32")
    c2 = [60, 128]
    Ao = hm.Matrix.create(hm.Tree.from_leaf_ends(c2), W.random_hodlr(np.random.default_rng(4), c2, 2), "f64")
    for B in (As, Af, Ao):
        assert lib.hm_hadamard(Ah._h, B._h, C.byref(out)) == hm._lib.HM_EINVAL
        assert out.value is None
    assert lib.hm_hadamard(Ah._h, Ah._h, None) == hm._lib.HM_EINVAL
    assert lib.hm_hadamard(None, Ah._h, C.byref(out)) == hm._lib.HM_EINVAL
