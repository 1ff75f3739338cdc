"""Failure detection without a GPU fault.

Device side: the library's bounded waits take a runtime limit; a self-test
kernel whose waits can never be satisfied (an mbarrier transaction that is
never issued, a flag that nothing sets) must give up after that limit,
record its codes, exit normally and leave the context usable, and
hm_device_status must report HM_ETIMEOUT.  Host side: injected allocation
failures surface as HM_ENOMEM from the call that needed the memory, which
can be retried; a stalled serving worker makes hm_serve_wait time out and a
queued request can be cancelled.  Nothing here faults, traps or hangs the GPU.
"""

import numpy as np
import pytest

import workloads as W
from oracle import matmat as OM, tree as OT
from tests import hmtest as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hm = pytest.importorskip("paper_1909_07909_gb300")
from paper_1909_07909_gb300 import _lib as L  # noqa: E402

DEFAULT_NS = 2_000_000_000


@pytest.fixture(autouse=True)
def _restore():
    yield
    hm.set_device_wait_limit(DEFAULT_NS)
    hm.inject_alloc_failures(0)


def _small_hss(seed=1, n=1500, k=6):
    c = OT.default_leaf_ends(n, 128)
    g = W.random_hss(np.random.default_rng(seed), c, k, orthonormal=False)
    return c, g


def _check_product(c, g, storage="f64", r=5):
    n = int(c[-1])
    X = np.random.default_rng(3).standard_normal((n, r))
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, storage)
    Y = H.to_host(A.matmat(H.to_dev(X, "f64")))
    assert H.col_rel_err(Y, OM.matmat(c, g, X)) <= 1e-12


def test_device_wait_runs_out_and_the_context_stays_usable():
    s = torch.cuda.current_stream().cuda_stream
    hm.set_device_wait_limit(2_000_000)          # 2 ms
    assert hm.device_wait_limit() == 2_000_000
    hm.selftest_device_timeout(s)
    with pytest.raises(hm.HMError) as e:
        hm.device_status(s)
    assert e.value.status == L.HM_ETIMEOUT
    assert b"code 3" in L.lib.hm_last_error()
    hm.device_status(s)                          # the flag was cleared
    hm.set_device_wait_limit(DEFAULT_NS)
    c, g = _small_hss()
    _check_product(c, g)                          # products still run and are correct
    hm.device_status(s)


@pytest.mark.parametrize("limit_ms", [5, 40])
def test_wait_limit_is_honoured(limit_ms):
    st = torch.cuda.current_stream()
    hm.set_device_wait_limit(limit_ms * 1_000_000)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    hm.selftest_device_timeout(st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # two waits, each given up after the limit
    assert 2 * limit_ms * 0.95 <= ms <= 2 * limit_ms + 200, ms
    with pytest.raises(hm.HMError):
        hm.device_status(st.cuda_stream)


def test_injected_allocation_failure_at_create_and_retry():
    c, g = _small_hss(2)
    hm.inject_alloc_failures(1)
    with pytest.raises(hm.HMError) as e:
        hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f32")
    assert e.value.status == L.HM_ENOMEM
    _check_product(c, g)                          # the next create succeeds


def test_injected_allocation_failure_in_product_scratch_and_retry():
    c, g = _small_hss(4)
    n = int(c[-1])
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f64")
    X = np.random.default_rng(5).standard_normal((n, 7))
    Xd = H.to_dev(X, "f64")
    hm.inject_alloc_failures(1)                   # the product's scratch allocation fails
    with pytest.raises(hm.HMError) as e:
        A.matmat(Xd)
    assert e.value.status == L.HM_ENOMEM
    Y = H.to_host(A.matmat(Xd))                   # retried: allocates and runs
    assert H.col_rel_err(Y, OM.matmat(c, g, X)) <= 1e-12


def test_injected_allocation_failure_at_serve_register():
    c, g = _small_hss(6)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f32")
    S = hm.Server(1 << 30, 16)
    hm.inject_alloc_failures(1)
    with pytest.raises(hm.HMError) as e:
        S.register(A)
    assert e.value.status == L.HM_ENOMEM
    assert S.register(A) >= 0
    S.close()


def _server_with_matrix():
    c, g = _small_hss(8, n=2048, k=8)
    A = hm.Matrix.create(hm.Tree.from_leaf_ends(c), g, "f32")
    S = hm.Server(1 << 30, 16)
    mid = S.register(A)
    return S, mid, A, c, g


def test_stalled_worker_wait_times_out_then_completes():
    S, mid, A, c, g = _server_with_matrix()
    n = int(c[-1])
    X = H.exact_input(np.random.default_rng(9).standard_normal((n, 3)), "f32")
    Xd = H.to_dev(X, "f32")
    Y = torch.full((3, n), float("nan"), dtype=torch.float32, device="cuda").t()
    S.pause(True)
    t = S.submit(mid, 3, Xd.data_ptr(), Y.data_ptr())
    assert t is not None
    with pytest.raises(hm.HMError) as e:
        S.wait(t, 50)
    assert e.value.status == L.HM_ETIMEOUT
    assert not S.poll(t)
    S.pause(False)
    S.wait(t, 20000)
    torch.cuda.synchronize()
    alone = A.matmat(Xd, out_dtype=torch.float32)
    torch.cuda.synchronize()
    assert torch.equal(Y, alone)
    S.close()


def test_cancel_a_queued_request():
    S, mid, A, c, g = _server_with_matrix()
    n = int(c[-1])
    X = H.to_dev(np.random.default_rng(10).standard_normal((n, 2)), "f32")
    Y1 = torch.full((2, n), float("nan"), dtype=torch.float32, device="cuda").t()
    Y2 = torch.full((2, n), float("nan"), dtype=torch.float32, device="cuda").t()
    S.pause(True)
    t1 = S.submit(mid, 2, X.data_ptr(), Y1.data_ptr())
    t2 = S.submit(mid, 2, X.data_ptr(), Y2.data_ptr())
    assert S.stats()["pending"] == 2
    assert S.cancel(t1)
    assert S.stats()["pending"] == 1
    with pytest.raises(hm.HMError) as e:          # the ticket is released
        S.wait(t1, 10)
    assert e.value.status == L.HM_EINVAL
    S.pause(False)
    S.wait(t2, 20000)
    torch.cuda.synchronize()
    assert torch.isnan(Y1).all()                  # the cancelled request never ran
    assert torch.isfinite(Y2).all()
    assert S.stats()["pending"] == 0
    with pytest.raises(hm.HMError):               # finished and collected: unknown
        S.cancel(t2)
    S.close()
