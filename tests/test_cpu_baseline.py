"""The CPU fast product (cpu_baseline, the timed CPU baseline of bench.py)
against the oracle: it runs the tree algorithms of Fig. 4.1 in float64, so
on every tree shape it must agree with the dense definition to rounding.
Runs on the CPU (no GPU marker); builds the baseline library if needed."""

import numpy as np
import pytest

import cpu_baseline as CB
import workloads as W
from oracle import matmat as OM, tree as OT
from tests import hmtest as H

SHAPES = [
    ("uniform_p3", [32 * (i + 1) for i in range(8)]),
    ("ragged", OT.default_leaf_ends(301, 40)),
    ("empty_leaves", [5, 9, 17, 17]),
    ("empty_first", [0, 70, 120, 200]),
    ("single_leaf", [57]),
    ("p1", [100, 190]),
    ("deep_p6", OT.default_leaf_ends(700, 11)),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    CB.build()


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
@pytest.mark.parametrize("name,c", SHAPES)
@pytest.mark.parametrize("r", [1, 5, 9])
def test_cpu_fast_product_matches_oracle(kind, name, c, r):
    rng = np.random.default_rng(31 + r)
    g = W.random_hodlr(rng, c, 5) if kind == "hodlr" else W.random_hss(rng, c, 5, orthonormal=False)
    X = rng.standard_normal((int(c[-1]), r))
    Y = CB.CpuMatrix(c, g).matmat(X)
    assert H.col_rel_err(Y, OM.matmat(c, g, X)) <= 1e-13, name


@pytest.mark.parametrize("kind", ["hodlr", "hss"])
def test_cpu_fast_product_variable_ranks(kind):
    c = OT.default_leaf_ends(500, 50)
    rng = np.random.default_rng(3)
    if kind == "hodlr":
        g = W.random_hodlr(rng, c, lambda q: (1 + q % 5, 3 + q % 4))
    else:
        g = W.random_hss(rng, c, lambda q: (2 + q % 6, 1 + (q * 7) % 5), orthonormal=False)
    X = rng.standard_normal((500, 6))
    M = CB.CpuMatrix(c, g)
    Y1 = M.matmat(X)
    Y2 = M.matmat(X)      # the work space is reused, not cleared
    assert H.col_rel_err(Y1, OM.matmat(c, g, X)) <= 1e-13
    assert np.array_equal(Y1, Y2)


def test_cpu_fast_product_tridiag_integer_exact():
    c = OT.default_leaf_ends(1000, 64)
    X = np.random.default_rng(2).integers(-9, 10, size=(1000, 4)).astype(np.float64)
    Y = CB.CpuMatrix(c, W.tridiag_hodlr(c)).matmat(X)
    S = 2 * X
    S[1:] -= X[:-1]
    S[:-1] -= X[1:]
    assert np.array_equal(Y, S)


def test_cpu_fast_product_reports_threads():
    assert CB.threads() >= 1
