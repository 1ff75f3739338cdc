"""The precision gates of the parity tests, checked on the CPU with the
oracle: a BF16-rounded product passes them, and a product with one coupling
level dropped (a mistake planted in the oracle's input) fails them.

The componentwise bound (c_round u_s + gamma) * envelope is loose for HSS
matrices (the envelope multiplies absolute values through every nested
factor); the normwise per-column gate of tests/hmtest.py is what a dropped
level trips."""

import copy

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, matmat as OM, tree as OT
from tests import hmtest as H


def _bf16(a):
    """Round to nearest even bfloat16 (float64 in, float64 out)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rounded(g):
    out = {"kind": g["kind"]}
    for key, v in g.items():
        if key == "kind":
            continue
        out[key] = [None if b is None else np.asfortranarray(_bf16(b)) for b in v]
    return out


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(0)
    c = OT.default_leaf_ends(4096, 256)
    g = W.random_hss(rng, c, 32)
    X = rng.standard_normal((4096, 8))
    fac = H.bound_factor("bf16", "hss", 4, H.acc_length({"leaf_pad": 256, "rank_total": 32, "depth": 4}, "hss"),
                         tensor_core=True)
    return c, g, X, OM.matmat(c, g, X), OB.envelope(c, g, X), fac


def test_bf16_rounded_product_passes_both_gates(case):
    c, g, X, ref, env, fac = case
    Y = OM.matmat(c, _rounded(g), _bf16(X))
    H.check_bound(Y, ref, env, fac, "bf16-rounded")
    assert H.col_rel_err(Y, ref) < H.NORMWISE["bf16"] / 2


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_dropped_coupling_level_fails_the_normwise_gate(case, level):
    c, g, X, ref, env, fac = case
    g2 = copy.deepcopy(g)
    for j in range(1 << (level - 1)):
        q = (1 << (level - 1)) - 1 + j
        g2["B12"][q] = np.zeros_like(g2["B12"][q])
        g2["B21"][q] = np.zeros_like(g2["B21"][q])
    Y = OM.matmat(c, g2, X)
    with pytest.raises(AssertionError, match="normwise"):
        H.check_bound(Y, ref, env, fac, "dropped level %d" % level)
