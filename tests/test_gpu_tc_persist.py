"""The persistent tensor-core leaf kernels (BF16 storage, many leaves).

When the one-item-per-CTA projection or expansion would need more than one
wave of CTAs, single products run the persistent kernels (k_tc_persist.cuh):
same MMA sequence, B chunks from TMA, from the Z block fetched into shared
memory, or converted from global memory.  The batched path still runs the one-item-per-CTA
tile code, so a batch of the same matrix must give the same bits; the results
are also held to the oracle's bound (Sec. 4.1, Def. 2.2 / 2.3) on sampled
rows.  Cases cover bf16 X by TMA, f32 X and bf16 X at an odd leading
dimension (converted by the threads), ragged leaves, a Ke that is not a
multiple of 4 (4-byte copies of the Z block), HODLR and HSS, and the full-size
exponential-kernel workload at 128 columns.
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
    return W.random_hodlr(rng, c, k) if kind == "hodlr" else W.random_hss(rng, c, k, orthonormal=False)


def _rows(c, count, seed):
    rng = np.random.default_rng(seed)
    n = int(c[-1])
    rows = {0, n - 1}
    for v in c[: count // 4]:
        rows.update({int(v) - 1, int(v)})
    rows.update(int(v) for v in rng.integers(0, n, size=count))
    return sorted(v for v in rows if 0 <= v < n)


CASES = [
    # name, kind, leaf ends, rank, columns
    ("hodlr_l64_r128", "hodlr", OT.default_leaf_ends(65536, 64), 4, 128),
    ("hss_l128_r48", "hss", OT.default_leaf_ends(65536, 128), 16, 48),
    ("hodlr_ragged_r64", "hodlr", OT.default_leaf_ends(50001, 100), 4, 64),
    ("hss_ke6_r96", "hss", OT.default_leaf_ends(32768, 64), 6, 96),
]


@pytest.mark.parametrize("name,kind,c,k,r", CASES)
def test_persistent_expansion_matches_batched_tiles(name, kind, c, k, r):
    g = _gens(kind, c, 23, k)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r + 1).standard_normal((n, r)), "f32")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "bf16")
    Xd = H.to_dev(X, "f32")
    y1 = A.matmat(Xd, out_dtype=torch.float32)
    y2 = A.matmat(Xd, out_dtype=torch.float32)                    # again: nothing carried over
    B = hm.Batch([A], [r])
    yb = torch.full((r, n), float("nan"), dtype=torch.float32, device=Xd.device).t()
    B.run([Xd], [yb])
    torch.cuda.synchronize()
    hm.device_status()
    assert torch.equal(y1, y2), name
    assert torch.equal(y1, yb), name + ": persistent expansion and batched tiles differ"
    rows = _rows(c, 96, 7)
    Y = H.to_host(y1)
    ref = OM.matmat_rows(c, g, X, rows)
    info = A.info()
    fac = H.bound_factor("bf16", kind, info["depth"], H.acc_length(info, kind), tensor_core=True)
    H.check_bound(Y[rows], ref, OB.envelope_rows(c, g, X, rows), fac, name)


@pytest.mark.parametrize("name,kind,c,k,r", [CASES[0], CASES[3]])
def test_persistent_expansion_bf16_x_tma_matches_staged(name, kind, c, k, r):
    """bf16 X by TMA (ld = n) and converted by the threads (ld = n + 3) give the
    same bits in the persistent kernel."""
    g = _gens(kind, c, 29, k)
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(r + 2).standard_normal((n, r)), "bf16")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "bf16")
    xt = torch.from_numpy(np.ascontiguousarray(X.T)).to(H.torch_dev()).to(torch.bfloat16)
    pad = torch.zeros((r, n + 3), dtype=torch.bfloat16, device=xt.device)
    pad[:, :n] = xt
    y_tma = A.matmat(xt.t(), out_dtype=torch.float32)
    y_odd = A.matmat(pad.t()[:n], out_dtype=torch.float32)
    torch.cuda.synchronize()
    hm.device_status()
    assert torch.equal(y_tma, y_odd), name
    rows = _rows(c, 64, 3)
    ref = OM.matmat_rows(c, g, X, rows)
    info = A.info()
    fac = H.bound_factor("bf16", kind, info["depth"], H.acc_length(info, kind), tensor_core=True)
    H.check_bound(H.to_host(y_tma)[rows], ref, OB.envelope_rows(c, g, X, rows), fac, name)


def test_exp_kernel_n262144_bf16_r128():
    """The exponential-kernel HODLR workload (n = 262144, leaf 256, K = 8) at
    128 columns in BF16 storage with bf16 X, as the bench times it: sampled rows
    against the oracle."""
    rng = W.rng_named("hodlr_exp_n262144_m256_K8")
    n, r = 262144, 128
    t = W.exp_points(rng, n)
    ck, lk = W.exp_params(8)
    c = OT.default_leaf_ends(n, 256)
    g = W.exp_kernel_hodlr(t, c, ck, lk)
    X = H.exact_input(rng.standard_normal((n, r)), "bf16")
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "bf16")
    Xd = H.to_dev(X, "bf16")
    y = A.matmat(Xd, out_dtype=torch.float32)
    torch.cuda.synchronize()
    hm.device_status()
    Y = H.to_host(y)
    rows = _rows(c, 160, 4)
    ref = OM.matmat_rows(c, g, X, rows)
    info = A.info()
    fac = H.bound_factor("bf16", "hodlr", info["depth"], H.acc_length(info, "hodlr"), tensor_core=True)
    H.check_bound(Y[rows], ref, OB.envelope_rows(c, g, X, rows), fac, "exp bf16 r128")
