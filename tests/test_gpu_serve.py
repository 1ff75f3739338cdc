"""Serving: resident matrices, admission, continuous batching.

The key property: a request's result is the same alone and merged with other
requests (bit-identical here, since each matrix's kernel family is fixed at
registration and columns are independent).  Also admission by slots and by
memory budget, bounded waits, and the latency statistics.
"""

import threading

import numpy as np
import pytest

import workloads as W
from oracle import bounds as OB, matmat as OM, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")


def _matrices(rng):
    out = []
    for kind, st, n, k in [("hss", "bf16", 4096, 16), ("hodlr", "f32", 3000, 8), ("hss", "bf16x2", 2048, 32),
                           ("hss", "bf16", 8192, 64), ("hodlr", "bf16", 1500, 4)]:
        c = OT.default_leaf_ends(n, 256)
        g = W.random_hodlr(rng, c, k) if kind == "hodlr" else W.random_hss(rng, c, k, orthonormal=False)
        out.append((kind, st, c, g, hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, st)))
    return out


def test_alone_equals_in_the_mix():
    rng = np.random.default_rng(0)
    mats = _matrices(rng)
    S = hm.Server(8 << 30, 512)
    ids = [S.register(m[4]) for m in mats]
    reqs = []
    for q in range(120):
        j = int(rng.integers(0, len(mats)))
        r = int(rng.integers(1, 17))
        n = mats[j][2][-1]
        X = H.to_dev(H.exact_input(rng.standard_normal((n, r)), "f32"), "f32")
        Y = torch.full((r, n), float("nan"), dtype=torch.float32, device="cuda").t()
        reqs.append((j, r, X, Y))
    # alone: each request as its own product (same kernel family as registered)
    alone = [mats[j][4].matmat(X, out_dtype=torch.float32) for (j, r, X, Y) in reqs]
    torch.cuda.synchronize()
    tickets = [S.submit(ids[j], r, X.data_ptr(), Y.data_ptr()) for (j, r, X, Y) in reqs]
    assert all(t is not None for t in tickets)
    for t in tickets:
        S.wait(t, 20000)
    torch.cuda.synchronize()
    for q, ((j, r, X, Y), Ya) in enumerate(zip(reqs, alone)):
        assert torch.equal(Y, Ya), q
    st = S.stats()
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    assert st["p99_us"] >= st["p50_us"] > 0
    assert st["launches"] <= len(reqs)
    # spot-check against the oracle
    kind, sto, c, g, A = mats[0]
    for (j, r, X, Y) in reqs:
        if j == 0:
            Xh = H.to_host(X)
            ref = OM.matmat(c, g, Xh)
            inf = A.info()
            H.check_bound(H.to_host(Y), ref, OB.envelope(c, g, Xh),
                          H.bound_factor(sto, kind, inf["depth"], H.acc_length(inf, kind), True), "served")
            break
    S.close()


def test_concurrent_submitters_merge():
    rng = np.random.default_rng(1)
    mats = _matrices(rng)[:2]
    S = hm.Server(8 << 30, 1024)
    ids = [S.register(m[4]) for m in mats]
    bufs = []
    for q in range(200):
        j = q % 2
        n = mats[j][2][-1]
        X = H.to_dev(rng.standard_normal((n, 4)), "f32")
        Y = torch.empty((4, n), dtype=torch.float32, device="cuda").t()
        bufs.append((j, X, Y))
    torch.cuda.synchronize()
    tickets = [None] * len(bufs)

    def submitter(lo, hi):
        for q in range(lo, hi):
            j, X, Y = bufs[q]
            tickets[q] = S.submit(ids[j], 4, X.data_ptr(), Y.data_ptr())

    th = [threading.Thread(target=submitter, args=(a, a + 50)) for a in range(0, 200, 50)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for t in tickets:
        S.wait(t, 20000)
    torch.cuda.synchronize()
    for q, (j, X, Y) in enumerate(bufs):
        assert torch.equal(Y, mats[j][4].matmat(X, out_dtype=torch.float32)), q
    assert S.stats()["completed"] == 200
    S.close()


def test_admission_by_slots_budget_and_bounded_wait():
    rng = np.random.default_rng(2)
    c = OT.default_leaf_ends(65536, 256)
    g = W.random_hss(rng, c, 32)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "bf16")
    small = hm.Server(1 << 20, 4)
    with pytest.raises(hm.HMError):
        small.register(A)                      # the matrix does not fit a 1 MiB budget
    small.close()
    S = hm.Server(4 << 30, 3)
    mid = S.register(A)
    X = torch.zeros((64, 65536), dtype=torch.float32, device="cuda").t()
    Ys = [torch.empty((64, 65536), dtype=torch.float32, device="cuda").t() for _ in range(5)]
    got = [S.submit(mid, 64, X.data_ptr(), Y.data_ptr()) for Y in Ys]
    assert any(t is None for t in got)         # slots exhausted: refused, not queued
    live = [t for t in got if t is not None]
    assert len(live) <= 3
    S.wait(live[0], 20000)
    for t in live[1:]:
        S.wait(t, 20000)
    st = S.stats()
    assert st["rejected"] >= 1 and st["completed"] == len(live)
    t = S.submit(mid, 64, X.data_ptr(), Ys[0].data_ptr())
    with pytest.raises(hm.HMError) as e:
        S.wait(t, 0)                           # not finished yet: a bounded wait returns
    assert e.value.status == hm._lib.HM_ETIMEOUT or S.poll(t)
    S.wait(t, 20000) if not S.poll(t) else None
    with pytest.raises(hm.HMError):
        S.submit(99, 1, X.data_ptr(), Ys[0].data_ptr())
    with pytest.raises(hm.HMError):
        S.submit(mid, 0, X.data_ptr(), Ys[0].data_ptr())
    S.close()
