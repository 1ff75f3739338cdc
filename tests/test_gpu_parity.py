"""Parity of the CUDA path with the CPU oracle (through the C ABI).

FP64: per-column relative error <= 1e-12 and every entry inside the
componentwise bound gamma_L(2^-53) * envelope.  FP32 / BF16 / BF16X2: every
entry inside (c_round u_s + gamma_L(u_acc)) * envelope, the bound written out in
tests/hmtest.py.  Integer work (tridiag with integer X) is bit-exact.
"""

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, expkernel as OE, matmat as OM, tree as OT
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


def _gens(kind, c, seed, k):
    rng = np.random.default_rng(seed)
    return W.random_hodlr(rng, c, k) if kind == "hodlr" else W.random_hss(rng, c, k, orthonormal=False)


def _run(c, g, X, storage, xt, yt="f64"):
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    Xd = H.to_dev(X, xt)
    td = torch.float64 if yt == "f64" else torch.float32
    Y = A.matmat(Xd, out_dtype=td)
    return H.to_host(Y), A


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SMALL)
@pytest.mark.parametrize("r", [1, 3, 8, 20, 33, 64, 70])
def test_f64_small_trees(kind, name, c, r):
    g = _gens(kind, c, 100 + r, 5)
    n = int(c[-1])
    X = np.random.default_rng(r).standard_normal((n, r))
    Y, A = _run(c, g, X, "f64", "f64")
    ref = OM.matmat(c, g, X)
    assert H.col_rel_err(Y, ref) <= 1e-12
    info = A.info()
    H.check_bound(Y, ref, OB.envelope(c, g, X),
                  H.bound_factor("f64", kind, info["depth"], H.acc_length(info, kind)), name)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("storage,xt", [("f32", "f32"), ("bf16", "f32"), ("bf16", "bf16"),
                                        ("bf16x2", "f32"), ("f32", "f64")])
@pytest.mark.parametrize("r", [1, 5, 16, 40])
def test_reduced_precision_within_bound(kind, storage, xt, r):
    c = OT.default_leaf_ends(777, 64)
    g = _gens(kind, c, 7 + r, 6)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), xt)
    Y, A = _run(c, g, X, storage, xt, "f32")
    ref = OM.matmat(c, g, X)
    info = A.info()
    H.check_bound(Y, ref, OB.envelope(c, g, X),
                  H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind)), storage)


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_variable_ranks(kind):
    c = OT.default_leaf_ends(500, 50)
    rng = np.random.default_rng(3)
    if kind == "hodlr":
        g = W.random_hodlr(rng, c, lambda q: (1 + q % 5, 3 + q % 4))
    else:
        g = W.random_hss(rng, c, lambda q: (2 + q % 6, 1 + (q * 7) % 5), orthonormal=False)
    X = np.random.default_rng(1).standard_normal((500, 9))
    Y, _ = _run(c, g, X, "f64", "f64")
    assert H.col_rel_err(Y, OM.matmat(c, g, X)) <= 1e-12


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "bf16x2"])
def test_tridiag_integer_exact(storage):
    """T = tridiag(-1,2,-1) with small-integer X: exact in every precision."""
    c = OT.default_leaf_ends(1000, 64)
    g = W.tridiag_hodlr(c)
    X = np.random.default_rng(2).integers(-9, 10, size=(1000, 6)).astype(np.float64)
    xt = "f64" if storage == "f64" else "f32"
    Y, _ = _run(c, g, X, storage, xt, "f64" if storage == "f64" else "f32")
    S = 2 * X
    S[1:] -= X[:-1]
    S[:-1] -= X[1:]
    assert np.array_equal(Y, S)


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_tridiag_inverse_exact_answer(fmt):
    n = 3000
    c = OT.default_leaf_ends(n, 100)
    g = W.tridiag_inverse_hodlr(c) if fmt == "hodlr" else W.tridiag_inverse_hss(c)
    z = np.random.default_rng(1).integers(-5, 6, size=(n, 2)).astype(np.float64)
    x = 2 * z
    x[1:] -= z[:-1]
    x[:-1] -= z[1:]
    Y, A = _run(c, g, x, "f64", "f64")
    info = A.info()
    env = OB.envelope(c, g, x)
    H.check_bound(Y, z, env, H.bound_factor("f64", fmt, info["depth"], H.acc_length(info, fmt) + n), fmt)


@pytest.mark.parametrize("fmt", ["hodlr", "hss"])
def test_structured_products(fmt):
    c = OT.default_leaf_ends(640, 64)
    X = np.random.default_rng(8).integers(-4, 5, size=(640, 4)).astype(np.float64)
    ones = W.ones_hodlr(c) if fmt == "hodlr" else W.ones_hss(c)
    Y, _ = _run(c, ones, X, "f64", "f64")
    assert np.array_equal(Y, np.tile(X.sum(axis=0), (640, 1)))
    d = np.arange(1, 641, dtype=np.float64)
    diag = W.diagonal_hodlr(c, d) if fmt == "hodlr" else W.diagonal_hss(c, d)
    Y, _ = _run(c, diag, X, "f64", "f64")
    assert np.array_equal(Y, d[:, None] * X)
    rng = np.random.default_rng(3)
    Ug, Vg = rng.standard_normal((640, 4)), rng.standard_normal((640, 4))
    lr = W.lowrank_hodlr(c, Ug, Vg) if fmt == "hodlr" else W.lowrank_hss(c, Ug, Vg)
    Y, _ = _run(c, lr, X, "f64", "f64")
    assert H.col_rel_err(Y, Ug @ (Vg.T @ X)) <= 1e-12


def test_exp_kernel_hss_exact_rank():
    rng = np.random.default_rng(5)
    t = W.exp_points(rng, 2048)
    ck, lk = W.exp_params(8)
    c = OT.default_leaf_ends(2048, 128)
    g = W.exp_kernel_hss(t, c, ck, lk)
    X = rng.standard_normal((2048, 3))
    Y, _ = _run(c, g, X, "f64", "f64")
    assert H.col_rel_err(Y, OE.apply(t, ck, lk, X)) <= 1e-12


def test_empty_and_zero_sizes():
    c = [0]
    g = W.random_hodlr(np.random.default_rng(0), c, 2)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    Xd = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    A.matmat_raw(3, Xd.data_ptr(), 1, hm.HM_F64, Xd.data_ptr() + 8, 1, hm.HM_F64,
                 torch.cuda.current_stream().cuda_stream)
    c = OT.default_leaf_ends(100, 10)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), _gens("hss", c, 1, 3), "f64")
    Y = torch.full((100, 2), 7.0, dtype=torch.float64, device="cuda")
    X = torch.zeros((100, 2), dtype=torch.float64, device="cuda")
    A.matmat_raw(0, X.data_ptr(), 100, hm.HM_F64, Y.data_ptr(), 100, hm.HM_F64, None)
    torch.cuda.synchronize()
    assert float(Y.min()) == 7.0                      # r = 0 writes nothing


def test_bad_arguments_rejected():
    c = OT.default_leaf_ends(200, 32)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), _gens("hodlr", c, 1, 3), "f32")
    X = torch.zeros((200, 2), dtype=torch.float32, device="cuda")
    Y = torch.zeros((200, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(hm.HMError):
        A.matmat_raw(2, X.data_ptr(), 100, hm.HM_F32, Y.data_ptr(), 200, hm.HM_F32, None)   # ldx < n
    with pytest.raises(hm.HMError):
        A.matmat_raw(2, X.data_ptr(), 200, hm.HM_F32, X.data_ptr(), 200, hm.HM_F32, None)   # overlap
    with pytest.raises(hm.HMError):
        A.matmat_raw(2, X.data_ptr(), 200, hm.HM_F32, Y.data_ptr(), 200, hm.HM_BF16, None)  # Y type
    B = hm.Matrix.create(hm.Tree.from_leaf_ends(c), _gens("hodlr", c, 1, 3), "f64")
    with pytest.raises(hm.HMError):
        B.matmat_raw(2, X.data_ptr(), 200, hm.HM_F32, Y.data_ptr(), 200, hm.HM_F32, None)   # F64 needs F64
    from paper_1909_07909_gb300 import _lib as L
    assert L.lib.hm_hss_matmat(A._h, 2, X.data_ptr(), 200, L.HM_F32, Y.data_ptr(), 200, L.HM_F32,
                               None) == L.HM_EINVAL                                      # wrong kind


def test_host_buffers_and_leading_dimension():
    c = OT.default_leaf_ends(900, 100)
    g = _gens("hss", c, 4, 7)
    X = np.random.default_rng(0).standard_normal((900, 5))
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    Yh = A.matmat(np.asfortranarray(X))                       # host in, host out
    big = torch.zeros((5, 1000), dtype=torch.float64, device="cuda")
    big[:, :900] = torch.from_numpy(X.T).cuda()
    Xd = big.t()[:900]                                        # ldx = 1000
    Yd = A.matmat(Xd)
    ref = OM.matmat(c, g, X)
    assert H.col_rel_err(Yh, ref) <= 1e-12
    assert np.array_equal(Yh, H.to_host(Yd))


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_deterministic(kind, storage):
    c = OT.default_leaf_ends(3000, 128)
    g = _gens(kind, c, 9, 8)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    xt = "f64" if storage == "f64" else "f32"
    X = H.to_dev(np.random.default_rng(2).standard_normal((3000, 24)), xt)
    Y1 = A.matmat(X)
    Y2 = A.matmat(X)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)


# ---------------------------------------------------------------------------
# The workload shapes at full size
# ---------------------------------------------------------------------------

def test_config_hodlr_n4096_f64_dense_oracle():
    """HODLR n=4096, leaf 128 (p=5), rank 8, r=1, FP64: full-vector dense oracle."""
    cfg = W.workload("hodlr_n4096_m128_k8_r1_f64")
    rng = W.rng_named("hodlr_n4096_m128_k8_r1_f64")
    c = OT.default_leaf_ends(cfg["n"], cfg["m"])
    g = W.random_hodlr(rng, c, cfg["k"])
    X = rng.standard_normal((cfg["n"], 1))
    Y, A = _run(c, g, X, "f64", "f64")
    ref = OM.matmat(c, g, X)
    assert A.info()["depth"] == 5
    assert H.col_rel_err(Y, ref) <= 1e-12


def _sample_rows(c, count, seed):
    rng = np.random.default_rng(seed)
    n = int(c[-1])
    edges = set()
    for v in c:
        for d in (-1, 0):
            if 0 <= v + d < n:
                edges.add(v + d)
    rows = sorted(edges)[: count // 2]
    rows += list(rng.integers(0, n, size=count - len(rows)))
    return sorted(set(int(v) for v in rows))


@pytest.mark.parametrize("storage,xt", [("f64", "f64"), ("f32", "f32"), ("bf16", "f32"), ("bf16", "bf16"),
                                        ("bf16x2", "f32")])
def test_config_hss_n65536_sampled_rows(storage, xt):
    """HSS n=65536, leaf 256, rank 32, r=64 at full size; oracle on sampled rows
    (BF16 storage also with bf16 X, the TMA-loaded operand the bench times)."""
    cfg = W.workload("hss_n65536_m256_k32_r64")
    rng = W.rng_named("hss_n65536_m256_k32_r64")
    c = OT.default_leaf_ends(cfg["n"], cfg["m"])
    g = W.random_hss(rng, c, cfg["k"])
    X = rng.standard_normal((cfg["n"], cfg["r"]))
    Xe = H.exact_input(X, xt)
    Y, A = _run(c, g, Xe, storage, xt, "f64" if storage == "f64" else "f32")
    rows = _sample_rows(c, 192, 3)
    ref = OM.matmat_rows(c, g, Xe, rows)
    info = A.info()
    if storage == "f64":
        assert H.col_rel_err(Y[rows], ref) <= 1e-12
    env = OB.envelope_rows(c, g, Xe, rows)
    H.check_bound(Y[rows], ref, env, H.bound_factor(storage, "hss", info["depth"], H.acc_length(info, "hss")),
                  storage)


@pytest.mark.parametrize("storage,r", [("f64", 1), ("f32", 1), ("bf16x2", 1), ("f32", 128), ("bf16x2", 128)])
def test_config_exp_kernel_n262144(storage, r):
    """HODLR exp kernel n=262144, leaf 256, K=8: recurrence (r=1, all rows) or sampled rows."""
    rng = W.rng_named("hodlr_exp_n262144_m256_K8")
    n = 262144
    t = W.exp_points(rng, n)
    ck, lk = W.exp_params(8)
    c = OT.default_leaf_ends(n, 256)
    g = W.exp_kernel_hodlr(t, c, ck, lk)
    X = rng.standard_normal((n, r))
    xt = "f64" if storage == "f64" else "f32"
    Xe = H.exact_input(X, xt)
    Y, A = _run(c, g, Xe, storage, xt, "f64" if storage == "f64" else "f32")
    info = A.info()
    fac = H.bound_factor(storage, "hodlr", info["depth"], H.acc_length(info, "hodlr"))
    if r == 1:
        ref = OE.apply(t, ck, lk, Xe)
        if storage == "f64":
            assert H.col_rel_err(Y, ref) <= 1e-12
        # all entries of kernel and X magnitudes: envelope = A |x|
        env = OE.apply(t, ck, lk, np.abs(Xe))
        H.check_bound(Y, ref, env, fac, storage)
    else:
        rows = _sample_rows(c, 160, 4)
        ref = OM.matmat_rows(c, g, Xe, rows)
        env = OB.envelope_rows(c, g, Xe, rows)
        H.check_bound(Y[rows], ref, env, fac, storage)


# ---------------------------------------------------------------------------
# Tensor-core expansion (tcgen05) against the oracle and against the SIMT path
# ---------------------------------------------------------------------------

TC_CASES = [
    ("hss_uniform_m256_r64", "hss", [256 * (i + 1) for i in range(16)], 32, 64),
    ("hodlr_ragged_m144_r20", "hodlr", OT.default_leaf_ends(4600, 150), 6, 20),
    ("hodlr_deep_K80_r128", "hodlr", OT.default_leaf_ends(8192, 256), 8, 128),
    ("hss_ragged_r33", "hss", OT.default_leaf_ends(3001, 200), 16, 33),
    ("hss_leaf512_r16", "hss", [512 * (i + 1) for i in range(4)], 24, 16),
    ("hodlr_r300_chunks", "hodlr", OT.default_leaf_ends(2048, 256), 8, 300),
    ("hss_empty_leaf_r48", "hss", [300, 600, 600, 900], 8, 48),
]


@pytest.mark.parametrize("storage", ["bf16", "bf16x2"])
@pytest.mark.parametrize("name,kind,c,k,r", TC_CASES)
def test_tensor_core_expansion(storage, name, kind, c, k, r):
    g = _gens(kind, c, 41, k)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r).standard_normal((n, r)), "f32")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    Xd = H.to_dev(X, "f32")
    A.set_path(2)                                   # tensor cores whenever supported
    Yt = H.to_host(A.matmat(Xd, out_dtype=torch.float32))
    A.set_path(1)                                   # SIMT only
    Ys = H.to_host(A.matmat(Xd, out_dtype=torch.float32))
    hm.device_status()
    ref = OM.matmat(c, g, X)
    info = A.info()
    fac = H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=True)
    env = OB.envelope(c, g, X)
    H.check_bound(Yt, ref, env, fac, name + " tensor cores")
    H.check_bound(Ys, ref, env, fac, name + " simt")


def test_tensor_core_split_f64_output_and_bf16_input():
    c = OT.default_leaf_ends(2048, 256)
    g = _gens("hss", c, 5, 16)
    X = H.exact_input(np.random.default_rng(0).standard_normal((2048, 32)), "bf16")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "bf16x2")
    A.set_path(2)
    Y = H.to_host(A.matmat(H.to_dev(X, "bf16"), out_dtype=torch.float64))
    ref = OM.matmat(c, g, X)
    info = A.info()
    H.check_bound(Y, ref, OB.envelope(c, g, X),
                  H.bound_factor("bf16x2", "hss", info["depth"], H.acc_length(info, "hss"), True), "split f64 out")
    assert H.col_rel_err(Y, ref) <= 1e-4


TMA_CASES = [
    ("hss_full_leaves_m256_r64", "hss", [256 * (i + 1) for i in range(16)], 16, 64),
    ("hodlr_full_leaves_m144_r33", "hodlr", [144 * (i + 1) for i in range(16)], 6, 33),
    ("hss_mixed_full_ragged_r16", "hss", OT.default_leaf_ends(4600, 150), 12, 16),
    ("hodlr_r130_chunks", "hodlr", [256 * (i + 1) for i in range(8)], 8, 130),
]


@pytest.mark.parametrize("storage", ["bf16", "bf16x2"])
@pytest.mark.parametrize("name,kind,c,k,r", TMA_CASES)
def test_tensor_core_bf16_x_tma_matches_staged(storage, name, kind, c, k, r):
    """bf16 X read by TMA (ld a multiple of 8, aligned) and bf16 X staged by the
    threads (odd ld, or a base off the 16-byte grid) build the same operand, so
    the products agree bit for bit; both stay within the bound."""
    g = _gens(kind, c, 17, k)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r + 5).standard_normal((n, r)), "bf16")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    A.set_path(2)
    xt = torch.from_numpy(np.ascontiguousarray(X.T)).to(H.torch_dev()).to(torch.bfloat16)
    x_tma = xt.t()                                                   # ld = n
    pad = torch.zeros((r, n + 3), dtype=torch.bfloat16, device=xt.device)
    pad[:, :n] = xt
    x_odd_ld = pad.t()[:n]                                           # ld = n + 3
    flat = torch.zeros(r * n + 1, dtype=torch.bfloat16, device=xt.device)
    flat[1:] = xt.reshape(-1)
    x_shift = flat[1:].view(r, n).t()                                # base 2 bytes off
    ys = [H.to_host(A.matmat(x, out_dtype=torch.float32)) for x in (x_tma, x_odd_ld, x_shift)]
    hm.device_status()
    assert np.array_equal(ys[0], ys[1]), name + ": TMA and odd-ld staging differ"
    assert np.array_equal(ys[0], ys[2]), name + ": TMA and shifted-base staging differ"
    ref = OM.matmat(c, g, X)
    info = A.info()
    fac = H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=True)
    H.check_bound(ys[0], ref, OB.envelope(c, g, X), fac, name)


@pytest.mark.parametrize("storage", ["bf16", "bf16x2"])
def test_tensor_core_deterministic_and_streams(storage):
    c = OT.default_leaf_ends(16384, 256)
    g = _gens("hss", c, 3, 32)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    X = H.to_dev(np.random.default_rng(1).standard_normal((16384, 64)), "f32")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Y1 = A.matmat(X)
        Y2 = A.matmat(X)
    s.synchronize()
    assert torch.equal(Y1, Y2)
    hm.device_status()
