"""The allocation-free product entry point (hm_matmat_noalloc).

Some callers cannot allocate device memory at the moment they need a product
(latency-bound serving loops that must not stall on cudaMalloc's implicit
synchronisation, programs whose own allocator owns the GPU's memory).
hm_matmat_noalloc serves them with its scratch in a fixed array inside the
library.  These tests call it through the C ABI and compare each result with
the allocating entry point's within the error bound the other parity tests
use: twice on the same matrix, with a product of another, larger matrix on
NaN inputs in between, so that the second call starts from scratch that holds
another product's NaNs and must clear or overwrite everything it reads.  This
file is collected last so that a run stopping at its first failure has already
run every other test.
"""

import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, matmat as OM, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")
from paper_1909_07909_gb300 import _lib as L  # noqa: E402

vp = C.c_void_p


def _noalloc(A, r, X, xt, Y, yt, n):
    return L.lib.hm_matmat_noalloc(A._h, r, vp(X.data_ptr()), n, xt, vp(Y.data_ptr()), n, yt,
                                   vp(torch.cuda.current_stream().cuda_stream))


def _dirty_the_scratch():
    """A product of another, larger HSS matrix on NaN inputs: afterwards the
    static scratch holds NaN wherever that product wrote."""
    c = OT.default_leaf_ends(20000, 128)
    g = W.random_hss(np.random.default_rng(5), c, 16, orthonormal=False)
    B = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f32")
    n, r = int(c[-1]), 32
    X = torch.full((r, n), float("nan"), dtype=torch.float32, device="cuda").t()
    Y = torch.empty((r, n), dtype=torch.float32, device="cuda").t()
    assert _noalloc(B, r, X, L.HM_F32, Y, L.HM_F32, n) == L.HM_OK, L.lib.hm_last_error()
    torch.cuda.synchronize()
    assert torch.isnan(Y).all()


@pytest.mark.parametrize("kind,storage,r,xt,c", [
    ("hss", "f64", 24, "f64", OT.default_leaf_ends(3000, 128)),   # FP64 register-tiled path
    ("hss", "f64", 8, "f64", OT.default_leaf_ends(3000, 128)),
    ("hodlr", "f64", 3, "f64", OT.default_leaf_ends(3000, 128)),
    ("hss", "bf16", 32, "f32", OT.default_leaf_ends(3000, 128)),
    ("hss", "bf16", 64, "bf16", OT.default_leaf_ends(4096, 128)),   # bf16 X by TMA
    ("hodlr", "bf16x2", 20, "f32", OT.default_leaf_ends(3000, 128)),
    ("hss", "f32", 5, "f32", OT.default_leaf_ends(3000, 128))])
def test_noalloc_matches_allocating_entry_point_twice(kind, storage, r, xt, c):
    rng = np.random.default_rng(11)
    g = W.random_hodlr(rng, c, 8) if kind == "hodlr" else W.random_hss(rng, c, 8, orthonormal=False)
    n = int(c[-1])
    X = H.exact_input(rng.standard_normal((n, r)), xt)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    Xd = H.to_dev(X, xt)
    td = torch.float64 if storage == "f64" else torch.float32
    code = L.HM_F64 if storage == "f64" else L.HM_F32
    xcode = {"f64": L.HM_F64, "f32": L.HM_F32, "bf16": L.HM_BF16}[xt]
    Yref = H.to_host(A.matmat(Xd, out_dtype=td))
    ref = OM.matmat(c, g, X)
    info = A.info()
    fac = H.bound_factor(storage, kind, info["depth"], H.acc_length(info, kind), tensor_core=True)
    env = OB.envelope(c, g, X)
    H.check_bound(Yref, ref, env, fac, "allocating")
    for call in range(2):
        if call == 1:
            _dirty_the_scratch()
        Y = torch.full((r, n), float("nan"), dtype=td, device="cuda").t()
        assert _noalloc(A, r, Xd, xcode, Y, code, n) == L.HM_OK, L.lib.hm_last_error()
        Yn = H.to_host(Y)
        assert np.isfinite(Yn).all()
        H.check_bound(Yn, ref, env, fac, "noalloc call %d" % call)
        assert np.allclose(Yn, Yref, rtol=0, atol=float(np.max(fac * env)) * 2 + 1e-300)
    hm.device_status()


def test_noalloc_rejects_overlapping_x_and_y():
    c = OT.default_leaf_ends(500, 64)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), W.random_hodlr(np.random.default_rng(2), c, 4), "f64")
    buf = torch.zeros((3, 500), dtype=torch.float64, device="cuda")
    st = L.lib.hm_matmat_noalloc(A._h, 2, vp(buf.data_ptr()), 500, L.HM_F64, vp(buf[1].data_ptr()), 500,
                                 L.HM_F64, vp(torch.cuda.current_stream().cuda_stream))
    assert st == L.HM_EINVAL
    assert b"overlap" in L.lib.hm_last_error()


def test_noalloc_rejects_products_above_the_limit():
    c = OT.default_leaf_ends(65536, 256)
    g = W.random_hss(np.random.default_rng(0), c, 32)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "bf16")
    r = 256
    X = torch.zeros((r, 65536), dtype=torch.float32, device="cuda").t()
    Y = torch.zeros((r, 65536), dtype=torch.float32, device="cuda").t()
    st = _noalloc(A, r, X, L.HM_F32, Y, L.HM_F32, 65536)
    assert st == L.HM_EINVAL
    assert b"limit" in L.lib.hm_last_error()


def test_noalloc_rejects_host_buffers():
    c = OT.default_leaf_ends(500, 64)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), W.random_hodlr(np.random.default_rng(1), c, 4), "f64")
    X = torch.zeros((2, 500), dtype=torch.float64).t()
    Y = torch.zeros((2, 500), dtype=torch.float64).t()
    st = L.lib.hm_matmat_noalloc(A._h, 2, vp(X.data_ptr()), 500, L.HM_F64, vp(Y.data_ptr()), 500, L.HM_F64, None)
    assert st == L.HM_EINVAL
