"""HSS solves X = A^{-1} B by the implicit ULV factorization (Sec. 4.3) on the
GPU, against the oracle (the dense LU solve of the defining matrix), the
closed form of tridiag(-1,2,-1)^{-1} (whose inverse is the tridiagonal
matrix itself), and the backward error through the FP64 product at full
size."""

import numpy as np
import pytest

import workloads as W
from oracle import matmat as OM, solve as SV, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")
from paper_1909_07909_gb300 import _lib as L  # noqa: E402

SHAPES = [
    ("uniform_p3", [64 * (i + 1) for i in range(8)]),
    ("ragged", OT.default_leaf_ends(777, 50)),
    ("p1", [100, 190]),
    ("deep_p6", OT.default_leaf_ends(1500, 20)),
    ("leaf_below_rank", [6 * (i + 1) for i in range(16)]),   # leaves smaller than the rank: padded
]


def _solve(c, g, B):
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    F = A.ulv()
    X = F.solve(H.to_dev(B, "f64"))
    return H.to_host(X), A, F


@pytest.mark.parametrize("name,c", SHAPES)
@pytest.mark.parametrize("r", [1, 7, 33])
def test_ulv_solve_matches_dense_solve(name, c, r):
    rng = np.random.default_rng(17 + r)
    g = W.random_hss(rng, c, 8, orthonormal=False)
    B = rng.standard_normal((int(c[-1]), r))
    X, A, F = _solve(c, g, B)
    ref = SV.solve_dense(c, g, B)
    assert H.col_rel_err(X, ref) <= 1e-11, name
    assert SV.residual(c, g, X, B) <= 1e-14
    hm.device_status()


def test_ulv_variable_ranks_and_repeated_solves():
    c = OT.default_leaf_ends(900, 64)
    rng = np.random.default_rng(3)
    g = W.random_hss(rng, c, lambda q: (3 + q % 6, 3 + q % 6), orthonormal=False)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    F = A.ulv()
    for r in (4, 9, 4):                               # the work space grows, then is reused
        B = rng.standard_normal((900, r))
        X = H.to_host(F.solve(H.to_dev(B, "f64")))
        assert H.col_rel_err(X, SV.solve_dense(c, g, B)) <= 1e-11


@pytest.mark.parametrize("n,leaf", [(1000, 64), (4096, 256)])
def test_ulv_tridiag_inverse_closed_form(n, leaf):
    """A = T^{-1} with T = tridiag(-1, 2, -1) (HSS rank 2): A^{-1} B = T B exactly."""
    c = OT.default_leaf_ends(n, leaf)
    g = W.tridiag_inverse_hss(c)
    B = np.random.default_rng(1).integers(-5, 6, size=(n, 3)).astype(np.float64)
    X, _, _ = _solve(c, g, B)
    TB = 2 * B
    TB[1:] -= B[:-1]
    TB[:-1] -= B[1:]
    cond = (n + 1) ** 2 / 4                            # ||T|| ||T^-1|| up to a constant
    assert np.max(np.abs(X - TB)) <= 64 * cond * 2.0 ** -53 * np.max(np.abs(TB)) + 1e-9


def test_ulv_full_size_backward_error():
    """HSS n=65536, leaf 256, rank 32, 64 right-hand sides: ||A X - B|| / ||B||
    through the FP64 product (itself held to the oracle by the parity tests)."""
    rng = W.rng_named("hss_n65536_m256_k32_r64")
    c = OT.default_leaf_ends(65536, 256)
    g = W.random_hss(rng, c, 32)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    F = A.ulv()
    B = H.to_dev(rng.standard_normal((65536, 64)), "f64")
    X = F.solve(B)
    R = A.matmat(X) - B
    torch.cuda.synchronize()
    rel = (torch.linalg.norm(R) / torch.linalg.norm(B)).item()
    assert rel <= 1e-12, rel
    # spot rows against the oracle's product of the computed X
    rows = [0, 255, 256, 40000, 65535]
    Xh = H.to_host(X)
    AX = OM.matmat_rows(c, g, Xh, rows)
    Bh = H.to_host(B)
    assert np.max(np.abs(AX - Bh[rows])) <= 1e-10 * np.max(np.abs(Bh))


def test_ulv_rejects_what_it_cannot_factor():
    c = OT.default_leaf_ends(500, 64)
    rng = np.random.default_rng(0)
    Ah = hm.Matrix.create(hm.Tree.from_leaf_ends(c), W.random_hodlr(rng, c, 4), "f64")
    with pytest.raises(hm.HMError) as e:
        Ah.ulv()
    assert e.value.status == L.HM_EINVAL
    As = hm.Matrix.create(hm.Tree.from_leaf_ends(c), W.random_hss(rng, c, 4), "f32")
    with pytest.raises(hm.HMError) as e:
        As.ulv()
    assert e.value.status == L.HM_EUNSUPPORTED
