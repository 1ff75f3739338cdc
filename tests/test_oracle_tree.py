"""Pins of the oracle's cluster trees (Def. 2.1, Sec. 3.1, Sec. 3.7)."""

import os

import pytest

from oracle import tree as T

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_trees():
    out = []
    with open(os.path.join(GOLD, "trees.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, c, nodes = [s.strip() for s in line.split("|")]
            c = [int(v) for v in c.split()]
            spec = []
            for tok in nodes.split():
                lv, rest = tok.split(":")
                i, rng = rest.split("=")
                if rng == "empty":
                    spec.append((int(lv), int(i), None))
                else:
                    a, b = rng.split("-")
                    spec.append((int(lv), int(i), (int(a), int(b))))
            out.append((name, c, spec))
    return out


@pytest.mark.parametrize("name,c,spec", _read_trees())
def test_paper_trees(name, c, spec):
    for lvl, i, want in spec:
        a, b = T.node_range(c, lvl, i - 1)
        if want is None:
            assert a == b, (name, lvl, i)
        else:
            assert (a + 1, b) == want, (name, lvl, i)


def test_fig21_is_default_tree():
    # Fig. 2.1 is the default construction for n = 8, n_min = 1 (Sec. 2.1, Sec. 3.7).
    assert T.default_leaf_ends(8, 1) == [1, 2, 3, 4, 5, 6, 7, 8]


@pytest.mark.parametrize("n,nmin,p", [(4096, 128, 5), (65536, 256, 8), (262144, 256, 10),
                                      (256, 256, 0), (257, 256, 1), (0, 256, 0)])
def test_config_depths(n, nmin, p):
    c = T.default_leaf_ends(n, nmin)
    assert len(c) == 1 << p
    assert c[-1] == n


@pytest.mark.parametrize("n", list(range(0, 70)) + [1000, 1023, 1025, 9159, 32768])
@pytest.mark.parametrize("nmin", [1, 3, 16, 256])
def test_default_tree_invariants(n, nmin):
    """Invariants that fix the ceil(n/2) rule: balanced, left >= right by at most one,
    every leaf <= n_min, and the depth minimal."""
    c = T.default_leaf_ends(n, nmin)
    p = T.depth(c)
    assert c[-1] == n
    for lvl in range(p):
        for j in range(1 << lvl):
            a, b = T.node_range(c, lvl, j)
            a1, b1 = T.node_range(c, lvl + 1, 2 * j)
            a2, b2 = T.node_range(c, lvl + 1, 2 * j + 1)
            assert a1 == a and b1 == a2 and b2 == b
            assert (b1 - a1) - (b2 - a2) in (0, 1)          # {1..ceil(s/2)} first
    sizes = [T.leaf_range(c, i)[1] - T.leaf_range(c, i)[0] for i in range(1 << p)]
    assert max(sizes) <= nmin
    if p > 0:
        above = [T.node_range(c, p - 1, j) for j in range(1 << (p - 1))]
        assert max(b - a for a, b in above) > nmin


def test_depth_rejects_bad_vectors():
    with pytest.raises(ValueError):
        T.depth([1, 2, 3])
    with pytest.raises(ValueError):
        T.depth([3, 2])


def test_ancestors_chain():
    c = T.default_leaf_ends(8, 1)
    ch = T.ancestors(c, 5)              # leaf 6 (1-based), id 12
    assert [a for a, _, _ in ch] == [2, 5, 12]
    assert [s for _, s, _ in ch] == [1, 6, 11]
    assert [q for _, _, q in ch] == [0, 2, 5]
