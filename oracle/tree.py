"""Cluster trees (Def. 2.1) and their leaf-end vector c (Sec. 3.7).  Test infrastructure.

A tree of depth p is given by c = [n_1, ..., n_{2^p}], the last index of
each leaf (1-based), i.e. leaf i (0-based) holds rows c[i-1] .. c[i]-1
(0-based, c[-1] of the empty prefix being 0).  Every node at level l is the
union of 2^(p-l) consecutive leaves.  Leaves may be empty (Def. 2.1, Fig. 3.2).
"""


def depth(c):
    L = len(c)
    p = L.bit_length() - 1
    if L < 1 or (1 << p) != L:
        raise ValueError("the number of leaves must be a power of two (Def. 2.1)")
    prev = 0
    for v in c:
        if v < prev:
            raise ValueError("leaf ends must be non-decreasing (Def. 2.1)")
        prev = v
    return p


def default_leaf_ends(n, n_min):
    """Default tree of Sec. 3.1.

    {1..n} is split into {1..ceil(n/2)} and the rest; every node of a level
    is split while some node of that level is larger than n_min, so all
    leaves sit at the same depth (completely balanced tree, Def. 2.1).
    """
    if n < 0 or n_min < 1:
        raise ValueError("n >= 0 and n_min >= 1 required")
    intervals = [(0, n)]
    while max(b - a for a, b in intervals) > n_min:
        nxt = []
        for a, b in intervals:
            h = (b - a + 1) // 2          # ceil((b - a) / 2)
            nxt.append((a, a + h))
            nxt.append((a + h, b))
        intervals = nxt
    return [b for _, b in intervals]


def node_id(level, j):
    return (1 << level) - 1 + j


def level_pos(q):
    level = (q + 1).bit_length() - 1
    return level, q - ((1 << level) - 1)


def node_range(c, level, j):
    """0-based half-open row range [start, end) of node I_{j+1}^{level}."""
    p = len(c).bit_length() - 1
    span = 1 << (p - level)
    first, last = j * span, (j + 1) * span - 1
    start = c[first - 1] if first > 0 else 0
    return int(start), int(c[last])


def leaf_range(c, i):
    return node_range(c, len(c).bit_length() - 1, i)


def children(q):
    return 2 * q + 1, 2 * q + 2


def parent(q):
    return (q - 1) // 2


def ancestors(c, leaf):
    """For leaf i: list over levels l = 1..p of (node id at level l, sibling id, parent id)."""
    p = depth(c)
    out = []
    q = node_id(p, leaf)
    chain = []
    while q > 0:
        chain.append(q)
        q = parent(q)
    for q in reversed(chain):
        par = parent(q)
        sib = q + 1 if q % 2 == 1 else q - 1
        out.append((q, sib, par))
    return out
