"""The multi-process path of bench.py on CPU (gloo, world size 2).

Each rank runs its own replica of the product (weak scaling, no collective
on the data path); the job's time is the longest rank's timed region (MAX
all-reduce) and the job's throughput counts every rank's products.  The
reference arm runs on rank 0 only.
"""

import importlib.util
import multiprocessing as mp
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        local = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        ms = b.max_over_ranks(local, world, "cpu")
        b.rank_barrier(world)
        q.put((rank, ms, b.job_throughput(2e9, 4, ms, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]           # both ranks see the longest timed region
    expect = 2 * 2e9 * 4 / 15e-3 / 1e9                   # both ranks' products over that time
    assert all(abs(o[2] - expect) < 1e-9 * expect for o in out)


def test_single_process_helpers():
    b = _bench()
    assert b.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert abs(b.job_throughput(1e9, 10, 5.0, 1) - 2000.0) < 1e-9
    b.rank_barrier(1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        cpu_leaves = 6
        steps = 1
        warmup = 0
    assert b.run_reference(A()) == 0                     # no work, exit code 0


def test_guarded_variant_records_its_error():
    """A failing secondary workload becomes an entry with its error; the
    entries before it and the line's headline are kept."""
    b = _bench()
    variants = {"f32": {"value": 1.0}}
    b.guarded(variants, "served", lambda: {"served_64": {"value": 2.0}})
    assert variants["served_64"] == {"value": 2.0}

    def fail():
        raise RuntimeError("request refused")
    b.guarded(variants, "workloads", fail)
    assert variants["workloads"]["error"] == "RuntimeError: request refused"
    assert variants["f32"] == {"value": 1.0}
