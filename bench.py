#!/usr/bin/env python3
"""Throughput of the HSS matrix-times-block product on GB300.

Workload (one "step" = one product Y = A X through the C ABI):
  HSS, n = 65536, leaf 256 (p = 8), nested rank 32, 64 right-hand sides;
  leaf U, V orthonormal (Q of a Gaussian QR), translations R and couplings B
  iid N(0, 1/32) (variance), D ~ N(0,1) + 8 I, X ~ N(0,1); seeded.
  Headline storage: --precision (default bf16) with float32 X and Y; the
  other storages (f64, f32, bf16x2) are timed as variants in the same run.

Timing: W untimed steps, then exactly K steps bracketed by a barrier and
torch.cuda.synchronize() on both sides, CUDA events on the launching stream,
max over ranks.  The inputs rotate over several resident copies whose total
exceeds the 135 MB L2, so every step streams its generators from HBM.

--impl reference times the CPU oracle (the FP64 dense-definition product)
on a bounded sample of the same workload.  N > 1 (torchrun): each rank runs
its own replica (weak scaling, no collective on the data path).
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HSS/HODLR matvec GB/s, % of roofline, mixed vs FP64 at stated err; p99 ms"
N_, LEAF, RANK, RHS = 65536, 256, 32, 64
WORKLOAD = "hss_matmat n=65536 leaf=256 rank=32 rhs=64"
ESZ = {"f64": 8, "f32": 4, "bf16": 2, "bf16x2": 4}
# Right-hand-side format per storage: the BF16 tensor-core path rounds X to
# bf16 in its operand anyway, so it takes X in bf16 (same result, half the
# bytes, TMA-loaded); split BF16 needs the float X for its lo part.
X_DTYPE = {"f64": "f64", "f32": "f32", "bf16": "bf16", "bf16x2": "f32"}
XSZ = {"f64": 8, "f32": 4, "bf16": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="hm", choices=["hm", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "f32", "f64", "bf16x2"])
    ap.add_argument("--copies", type=int, default=0, help="resident copies (0 = enough to exceed L2)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-leaves", type=int, default=6, help="leaf row blocks in the CPU sample")
    ap.add_argument("--workload", default="hss", choices=["hss", "batched", "serve"],
                    help="hss: the HSS n=65536 headline; batched: 512 uneven matrices; serve: Poisson requests")
    ap.add_argument("--count", type=int, default=0, help="matrices in the batched / serving workload")
    ap.add_argument("--rates", default="1000,5000,10000,20000,50000")
    ap.add_argument("--seconds", type=float, default=1.0, help="arrival window per rate (serve)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), \
        int(os.environ.get("WORLD_SIZE", "1"))


def rank_barrier(world):
    """All ranks meet (no-op for one process)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ms_local, world, device):
    """The whole job's timed region: the longest rank's (a MAX all-reduce,
    then a barrier); `device` is where the reduction tensor lives ("cuda" for
    NCCL, "cpu" for gloo)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    return float(t.item())


def job_throughput(bytes_per_step, steps, ms_max, world):
    """Whole-job GB/s: every rank runs `steps` products of `bytes_per_step`
    (weak scaling) within the longest rank's `ms_max`."""
    return world * bytes_per_step * steps / (ms_max * 1e-3) / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 / FP32 FMA peaks of this GPU model (FMA-throughput probe, profiles/fma_peaks_probe.txt).
FP64_TFLOPS = 1.199
FP32_TFLOPS = 74.9


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        loaded = [v for v in sm if v > 0.5 * (mx or max(sm))] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs():
    import workloads as W
    rng = W.rng_named("hss_n65536_m256_k32_r64")
    import paper_1909_07909_gb300 as hm
    tree = hm.Tree.default(N_, LEAF)
    c = tree.leaf_ends
    g = W.random_hss(rng, c, RANK)
    X = rng.standard_normal((N_, RHS))
    return tree, c, g, X


def step_bytes(A, storage, xs=4, ys=4):
    return A.generator_bytes() + N_ * RHS * (xs + ys)


# Phase slots of hm_matrix_phase_times: the leaf projection, the tree (the
# cluster kernel runs upsweep, couplings and downsweep in this one slot; the
# per-level kernels use it for the upsweep), the per-level downsweep, the
# leaf expansion.
PHASES = ["project", "tree", "tree_down", "expand"]


def phase_bytes(storage, c):
    """Algorithmic bytes per launch: the expansion reads D and U, X and writes
    Y; the projection reads V and X; the tree kernels read their operators
    once (R_V, B12, B21 upward; R_U downward; held in FP64 for FP64 storage,
    else FP32).  Per-node k x r intermediates are excluded, as for the whole
    step."""
    s = ESZ[storage]
    xs = XSZ[X_DTYPE[storage]]
    ys = 8 if storage == "f64" else 4
    ts = 8 if storage == "f64" else 4
    L = len(c)
    sizes = [c[0]] + [c[i] - c[i - 1] for i in range(1, L)]
    d_elems = sum(m * m for m in sizes)
    expand = (d_elems + N_ * RANK) * s + N_ * RHS * (xs + ys)
    project = N_ * RANK * s + N_ * RHS * xs
    internal = L - 1
    tree = internal * (2 * RANK * RANK + 2 * RANK * RANK) * ts + internal * 2 * RANK * RANK * ts
    return {"project": project, "tree": tree, "tree_down": 0, "expand": expand}


def tree_flops(c):
    """FLOPs of the HSS tree for the workload: R_V^T on every internal node
    but the root, B12 and B21 on every internal node, one R_U half per node
    of levels 2 .. p (2 flops per multiply-add, every right-hand side)."""
    L = len(c)
    k2 = RANK * RANK
    return 2 * RHS * ((L - 2) * 2 * k2 + (L - 1) * 2 * k2 + (2 * L - 4) * k2)


def time_variant(hm, torch, tree, g, storage, steps, warmup, copies, want_phases, clock_index=None,
                 prof_steps=None, world=1, form=None, g_b=None):
    """Device throughput of one storage type (timed region without profiling
    events, so consecutive kernels overlap), then a profiled pass that brackets
    every kernel with CUDA events for per-kernel durations.  form="transpose"
    times Y = A^T X (matrices from hm_matrix_transpose); form="hodlr" times
    the HODLR form of the HSS matrix (hm_hss_to_hodlr); form="hadamard"
    times the Hadamard product of g and g_b (hm_hadamard)."""
    td = torch.float64 if storage == "f64" else torch.float32
    xd = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[X_DTYPE[storage]]
    dev = torch.device("cuda", torch.cuda.current_device())
    mats = []
    for _ in range(copies):
        A0 = hm.Matrix.create(tree, g, storage)
        if form == "hadamard":
            B0 = hm.Matrix.create(tree, g_b, storage)
            mats.append(A0.hadamard(B0))
            del B0
        else:
            mats.append(A0.transpose() if form == "transpose" else A0.to_hodlr() if form == "hodlr" else A0)
        del A0
    Xh = torch.from_numpy(g["_X"].T.copy())
    Xs = [Xh.to(dev).to(xd).t() for _ in range(copies)]
    Ys = [torch.empty((RHS, N_), dtype=td, device=dev).t() for _ in range(copies)]
    for A in mats:
        A.reserve(RHS)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    code = hm.HM_F64 if storage == "f64" else hm.HM_F32
    xcode = {"f64": hm.HM_F64, "f32": hm.HM_F32, "bf16": hm.HM_BF16}[X_DTYPE[storage]]

    def run(i):
        j = i % copies
        mats[j].matmat_raw(RHS, Xs[j].data_ptr(), N_, xcode, Ys[j].data_ptr(), N_, code, sptr)

    for i in range(warmup):
        run(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(clock_index) if clock_index is not None else None
    if sampler:
        sampler.__enter__()
    torch.cuda.synchronize()
    rank_barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(steps):
        run(i)
    e1.record(stream)
    torch.cuda.synchronize()
    rank_barrier(world)
    if sampler:
        sampler.__exit__()
    ms_total = e0.elapsed_time(e1)
    phases = None
    if want_phases:
        ps = prof_steps or steps
        for A in mats:
            A.profile(True)
            A.phase_times()
        for i in range(ps):
            run(i)
        torch.cuda.synchronize()
        acc_ms = [0.0] * 4
        acc_n = [0] * 4
        for A in mats:
            ms, n = A.phase_times()
            A.profile(False)
            for k in range(4):
                acc_ms[k] += ms[k]
                acc_n[k] += n[k]
        phases = {"ms": acc_ms, "launches": acc_n, "steps": ps}
    es = 8 if storage == "f64" else 4
    res = {"ms_total": ms_total, "ms_per_step": ms_total / steps,
           "bytes_per_step": step_bytes(mats[0], storage, XSZ[X_DTYPE[storage]], es),
           "phases": phases, "clocks": sampler.summary() if sampler else None,
           "generator_bytes": mats[0].generator_bytes()}
    res["gbs"] = res["bytes_per_step"] / (res["ms_per_step"] * 1e-3) / 1e9
    Y0 = Ys[0].to(torch.float64).cpu().numpy()
    del mats
    return res, Y0


def e2e_host(hm, torch, tree, g, storage, steps):
    """Same product through the C ABI with pinned host buffers (copies inside)."""
    import numpy as np
    A = hm.Matrix.create(tree, g, storage)
    A.reserve(RHS)
    f64 = storage == "f64"
    td = torch.float64 if f64 else torch.float32
    xd = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[X_DTYPE[storage]]
    Xp = torch.from_numpy(g["_X"].T.copy()).to(xd).pin_memory()
    Yp = torch.empty((RHS, N_), dtype=td).pin_memory()
    code = hm.HM_F64 if f64 else hm.HM_F32
    xcode = {"f64": hm.HM_F64, "f32": hm.HM_F32, "bf16": hm.HM_BF16}[X_DTYPE[storage]]
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        A.matmat_raw(RHS, Xp.data_ptr(), N_, xcode, Yp.data_ptr(), N_, code, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        A.matmat_raw(RHS, Xp.data_ptr(), N_, xcode, Yp.data_ptr(), N_, code, stream)
    dt = (time.perf_counter() - t0) / steps
    es = 8 if f64 else 4
    xs = XSZ[X_DTYPE[storage]]
    b = A.generator_bytes() + N_ * RHS * (xs + es)
    del np
    return {"value": b / dt / 1e9, "unit": "GB/s", "h2d_bytes_per_step": N_ * RHS * xs,
            "d2h_bytes_per_step": N_ * RHS * es, "ms_per_step": dt * 1e3}


def fp64_step_bytes(c):
    """Algorithmic bytes of one FP64 product: all generators read once, X read, Y written."""
    L = len(c)
    sizes = [c[0]] + [c[i] - c[i - 1] for i in range(1, L)]
    elems = sum(m * m for m in sizes) + 2 * N_ * RANK + max(L - 2, 0) * 4 * RANK * RANK + \
        max(2 * L - 2, 0) * RANK * RANK
    return 8 * elems + N_ * RHS * 16


def cpu_oracle_sample(c, g, X, leaves):
    """Oracle (dense-definition product) on `leaves` leaf row blocks; returns
    (seconds, rows, Yrows, cores)."""
    import numpy as np
    from oracle import matmat as OM
    from oracle import tree as OT
    t0 = time.perf_counter()
    blocks = OM.matmat_leaves(c, g, X, leaves)
    dt = time.perf_counter() - t0
    rows = []
    for i in leaves:
        a, b = OT.leaf_range(c, i)
        rows.extend(range(a, b))
    return dt, rows, np.vstack(blocks)


def traffic_for(kernel_key):
    """ncu DRAM bytes per launch recorded in profiles/traffic.json, if the kernel
    source has not changed since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    ent = rec.get(kernel_key)
    if not ent:
        return None
    h = hashlib.sha256()
    for f in ent.get("sources", []):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != ent.get("sha256"):
        return None
    return ent.get("bytes_per_launch")


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import workloads as W
    from oracle import tree as OT
    rng = W.rng_named("hss_n65536_m256_k32_r64")
    c = OT.default_leaf_ends(N_, LEAF)
    g = W.random_hss(rng, c, RANK)
    X = rng.standard_normal((N_, RHS))
    L = len(c)
    per = max(1, args.cpu_leaves)
    for i in range(args.warmup):
        cpu_oracle_sample(c, g, X, [(i * per + j) % L for j in range(per)])
    t = 0.0
    for i in range(args.steps):
        dt, _, _ = cpu_oracle_sample(c, g, X, [((i + args.warmup) * per + j) % L for j in range(per)])
        t += dt
    frac = per / L
    nbytes = fp64_step_bytes(c)
    step_s = t / args.steps / frac
    val = nbytes / step_s / 1e9
    cores = os.cpu_count()
    sample = "%d of %d leaf row blocks per step (scaled by %d)" % (per, L, L // per)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "storage": "f64", "oracle": "dense definition, FP64 numpy/BLAS"},
           "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    del np
    return 0


# ---------------------------------------------------------------------------
# Batched workload: 512 matrices, n log-uniform in [1024, 32768], rank in
# {4, 8, 16, 32, 64}, 1..32 right-hand sides, half HODLR and half HSS.
# ---------------------------------------------------------------------------

def run_batched(args):
    import numpy as np
    import torch
    import workloads as W
    import paper_1909_07909_gb300 as hm
    torch.cuda.set_device(0)
    rng = W.rng_named("batched_512")
    count = args.count or 512
    spec = W.batch_spec(rng, count=count)
    out = {"metric": METRIC, "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
           "config": {"workload": "batched %d matrices, n log-uniform [1024,32768], rank {4..64}, r 1..32, "
                                  "half HODLR/HSS, leaf 256" % count}}
    res = {}
    allm = {"bf16": [], "f32": [], "f64": []}
    rs = []
    for sp in spec:
        tree = hm.Tree.default(sp["n"], 256)
        c = tree.leaf_ends
        g = (W.random_hodlr(rng, c, sp["k"]) if sp["kind"] == "hodlr" else W.random_hss(rng, c, sp["k"]))
        for stg in allm:
            allm[stg].append(hm.Matrix.create(tree, g, stg))
        rs.append(sp["r"])
        del g
    for storage in ("bf16", "f32", "f64"):
        mats = allm[storage]
        td = torch.float64 if storage == "f64" else torch.float32
        Xs = [torch.randn((sp["r"], sp["n"]), dtype=td, device="cuda").t() for sp in spec]
        Ys = [torch.empty((sp["r"], sp["n"]), dtype=td, device="cuda").t() for sp in spec]
        gen_bytes = sum(A.generator_bytes() for A in mats)
        es = 8 if storage == "f64" else 4
        io_bytes = sum(sp["n"] * sp["r"] * 2 * es for sp in spec)
        step_bytes = gen_bytes + io_bytes
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        entry = {"bytes_per_run": step_bytes}
        if storage != "f64":
            B = hm.Batch(mats, rs)
            t0 = time.perf_counter()
            B.tune(None)
            entry["tune_s"] = time.perf_counter() - t0
            for _ in range(args.warmup):
                B.run(Xs, Ys)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(args.steps):
                B.run(Xs, Ys)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            info = B.info()          # after the runs: the first run after tuning records the graph
            entry.update({"batched_ms": ms, "batched_gbs": step_bytes / (ms * 1e-3) / 1e9,
                          "launches_per_run": info["launches_per_run"], "graph": info["graph"],
                          "capture_error": info["capture_error"],
                          "tuned": {k: info[k] for k in ("grid_mult", "rc_cap", "rct_cap", "tile_rows")}})
        loops = max(1, args.steps // 4)
        for _ in range(2):
            for A, X, Y in zip(mats, Xs, Ys):
                A.matmat(X, Y)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(loops):
            for A, X, Y in zip(mats, Xs, Ys):
                A.matmat(X, Y)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / loops
        entry.update({"loop_ms": ms, "loop_gbs": step_bytes / (ms * 1e-3) / 1e9})
        res[storage] = entry
        del Xs, Ys
        allm[storage] = []
        del mats
        torch.cuda.empty_cache()
    out["value"] = res["bf16"]["batched_gbs"]
    out["ms_per_step"] = res["bf16"]["batched_ms"]
    out["dtype"] = "bf16"
    out["variants"] = res
    out["batched_vs_fp64_unbatched"] = res["bf16"]["batched_gbs"] / res["f64"]["loop_gbs"]
    out["gpu_launches"] = res["bf16"]["launches_per_run"] * args.steps
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# Serving workload: 64 resident HSS matrices (n = 2^12..2^18, rank 16..64,
# BF16), Poisson arrivals, 1..16 right-hand sides per request.
# ---------------------------------------------------------------------------

def run_serve(args):
    import numpy as np
    import torch
    import workloads as W
    import paper_1909_07909_gb300 as hm
    torch.cuda.set_device(0)
    rng = W.rng_named("serving_64_hss")
    count = args.count or 64
    spec = W.serve_spec(rng, count=count)
    server = hm.Server(100 << 30, 4096)
    mats, ids, pools = [], [], []
    for sp in spec:
        tree = hm.Tree.default(sp["n"], 256)
        g = W.random_hss(rng, tree.leaf_ends, sp["k"])
        A = hm.Matrix.create(tree, g, "bf16")
        del g
        mats.append(A)
        ids.append(server.register(A))
        X = torch.randn((16, sp["n"]), dtype=torch.float32, device="cuda").t()
        Ys = [torch.empty((16, sp["n"]), dtype=torch.float32, device="cuda").t() for _ in range(48)]
        pools.append((X, Ys))
    torch.cuda.synchronize()
    rates = [int(v) for v in args.rates.split(",") if v]
    by_rate = {}
    for rate in rates:
        nreq = max(50, int(rate * args.seconds))
        gaps = rng.exponential(1.0 / rate, size=nreq)
        which = rng.integers(0, count, size=nreq)
        rr = rng.integers(1, 17, size=nreq)
        server.reset_stats()
        tickets = []
        busy = 0
        t0 = time.perf_counter()
        due = t0
        slot = [0] * count
        for q in range(nreq):
            due += gaps[q]
            while time.perf_counter() < due:
                pass
            j = int(which[q])
            X, Ys = pools[j]
            Y = Ys[slot[j] % len(Ys)]
            slot[j] += 1
            t = server.submit(ids[j], int(rr[q]), X.data_ptr(), Y.data_ptr())
            if t is None:
                busy += 1
            else:
                tickets.append(t)
            if len(tickets) > 2048:
                server.wait(tickets.pop(0), 60000)
        for t in tickets:
            server.wait(t, 60000)
        wall = time.perf_counter() - t0
        stt = server.stats()
        by_rate[str(rate)] = {"offered_rps": rate, "requests": nreq, "refused": busy,
                              "p50_ms": stt["p50_us"] / 1e3, "p99_ms": stt["p99_us"] / 1e3,
                              "throughput_rps": stt["throughput_rps"], "gbs": stt["gbs"],
                              "launches": stt["launches"], "max_merged": stt["max_merged"], "wall_s": wall}
    # FP64 unbatched reference on the same GPU: each request alone, one after another
    f64 = []
    for j in range(min(count, 8)):
        tree = mats[j].tree
        g = W.random_hss(W.rng_named("serving_64_hss", 100 + j), tree.leaf_ends, spec[j]["k"])
        A64 = hm.Matrix.create(tree, g, "f64")
        X = torch.randn((8, spec[j]["n"]), dtype=torch.float64, device="cuda").t()
        A64.matmat(X)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            A64.matmat(X)
        torch.cuda.synchronize()
        f64.append((time.perf_counter() - t0) / 5)
    f64_ms = 1e3 * float(np.mean(f64))
    # headline: the p99 latency at the highest offered rate the server sustains
    # (completes at least 95 % of what is offered); also the saturation throughput
    sustained = [rt for rt in rates if by_rate[str(rt)]["throughput_rps"] >= 0.95 * rt]
    top_rate = max(sustained) if sustained else min(rates)
    top = by_rate[str(top_rate)]
    out = {"metric": METRIC, "value": top["p99_ms"], "unit": "ms (p99)", "n_gpus": 1, "steps": len(rates),
           "warmup": 0, "ms_per_step": top["p50_ms"], "higher_is_better": False, "scaling": "weak",
           "sustained_rps": top_rate,
           "saturation_throughput_rps": max(v["throughput_rps"] for v in by_rate.values()),
           "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": "serving %d resident HSS matrices n=2^12..2^18 rank 16..64 BF16, Poisson "
                                  "arrivals, 1..16 RHS per request, 100 GB budget" % count},
           "by_rate": by_rate, "fp64_unbatched_ms_per_request_r8": f64_ms,
           "resident_bytes": server.stats()["resident_bytes"]}
    server.close()
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    rank, local, world = dist_env()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args) if rank == 0 else 0
    if args.workload == "serve":
        return run_serve(args) if rank == 0 else 0
    os.environ.setdefault("OPENBLAS_NUM_THREADS", str(os.cpu_count()))
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    import paper_1909_07909_gb300 as hm

    peaks, peak_src = measured_peaks()
    tree, c, g, X = make_inputs()
    g["_X"] = X
    prec = args.precision
    gen_bytes_est = {"bf16": 45e6, "f32": 90e6, "bf16x2": 90e6, "f64": 180e6}[prec]
    io = N_ * RHS * (16 if prec == "f64" else 8)
    copies = args.copies or max(2, math.ceil(2.2 * 135.5e6 / (gen_bytes_est + io)))

    if world > 1:
        torch.distributed.barrier()
    head, Yh = time_variant(hm, torch, tree, g, prec, args.steps, args.warmup, copies, True,
                            clock_index=local, prof_steps=min(args.steps, 200), world=world)
    # whole-job time: max over ranks of this rank's timed region
    ms_max = max_over_ranks(head["ms_total"], world, "cuda")
    value = job_throughput(head["bytes_per_step"], args.steps, ms_max, world)

    # dominant kernel roofline (per-kernel durations from the profiled pass)
    pb = phase_bytes(prec, c)
    ph = head["phases"]
    dom = max(range(4), key=lambda k: ph["ms"][k])
    avg_ms = ph["ms"][dom] / max(ph["launches"][dom], 1)
    achieved = pb[PHASES[dom]] / (avg_ms * 1e-3) / 1e9
    kernel_key = "%s_%s" % (PHASES[dom], prec)
    if prec == "f64":
        flops = {"project": 2 * N_ * RANK * RHS, "tree": tree_flops(c), "tree_down": 0,
                 "expand": 2 * (N_ * LEAF + N_ * RANK) * RHS}[PHASES[dom]]
        roof = {"bound": "alu", "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": FP64_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "FP64 FMA probe (profiles/fma_peaks_probe.txt)"}
    elif PHASES[dom] == "tree":
        # FP32 small products: bound by the FMA pipes (and their shared-memory
        # operands), not by HBM; the denominator is the scalar FFMA peak
        roof = {"bound": "alu", "achieved": tree_flops(c) / (avg_ms * 1e-3) / 1e12, "peak": FP32_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "FP32 FMA probe (profiles/fma_peaks_probe.txt)"}
    else:
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "peak_source": peak_src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_for(kernel_key)
    roof["kernel"] = kernel_key
    roof["ms_per_launch"] = avg_ms
    roof["phase_ms_per_step"] = {PHASES[k]: ph["ms"][k] / ph["steps"] for k in range(4)}
    roof["expand_frac_of_hbm"] = (pb["expand"] / (ph["ms"][3] / max(ph["launches"][3], 1) * 1e-3) / 1e9
                                  / peaks["hbm_gbs"]) if ph["launches"][3] else None

    out = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16",
                                                              "bf16x2": "bf16x2"}[prec],
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N_, "leaf": LEAF, "rank": RANK, "rhs": RHS, "storage": prec,
                      "x_dtype": X_DTYPE[prec], "y_dtype": "f64" if prec == "f64" else "f32",
                      "l2": "inputs larger than L2: %d rotating resident copies of %.1f MB" %
                            (copies, head["bytes_per_step"] / 1e6),
                      "generators": "leaf U,V orthonormal; R,B iid N(0,1/32) (variance); D=N(0,1)+8I; X=N(0,1)",
                      "parallelism": "replicas" if world > 1 else "single"},
           "roofline": roof,
           "gpu_launches": int(sum(ph["launches"]) * args.steps / ph["steps"]),
           "clocks": head["clocks"]}

    if rank == 0:
        out["e2e"] = e2e_host(hm, torch, tree, g, prec, max(5, min(50, args.steps // 4)))
        variants = {}
        ys = {prec: Yh}
        if not args.no_variants:
            for v in ["f64", "f32", "bf16", "bf16x2"]:
                if v == prec:
                    continue
                eb = {"bf16": 45e6, "f32": 90e6, "bf16x2": 90e6, "f64": 180e6}[v] + N_ * RHS * (16 if v == "f64" else 8)
                cps = max(2, math.ceil(2.2 * 135.5e6 / eb))
                st = 20 if v == "f64" else max(20, args.steps // 4)
                r_, yv = time_variant(hm, torch, tree, g, v, st, 3, cps, True, prof_steps=min(st, 20))
                ys[v] = yv
                pbv = phase_bytes(v, c)
                d = max(range(4), key=lambda k: r_["phases"]["ms"][k])
                am = r_["phases"]["ms"][d] / max(r_["phases"]["launches"][d], 1)
                variants[v] = {"value": r_["gbs"], "ms_per_step": r_["ms_per_step"], "steps": st,
                               "dominant_kernel": PHASES[d],
                               "phase_ms_per_step": {PHASES[k]: r_["phases"]["ms"][k] / r_["phases"]["steps"]
                                                     for k in range(4)}}
                if pbv[PHASES[d]]:
                    variants[v]["dominant_gbs"] = pbv[PHASES[d]] / (am * 1e-3) / 1e9
            # the transposed product A^T X on the headline storage
            st = max(20, args.steps // 4)
            r_, yt = time_variant(hm, torch, tree, g, prec, st, 3, copies, True, prof_steps=min(st, 20),
                                  form="transpose")
            d = max(range(4), key=lambda k: r_["phases"]["ms"][k])
            variants["transpose"] = {"value": r_["gbs"], "ms_per_step": r_["ms_per_step"], "steps": st,
                                     "storage": prec, "dominant_kernel": PHASES[d],
                                     "phase_ms_per_step": {PHASES[k]: r_["phases"]["ms"][k] / r_["phases"]["steps"]
                                                           for k in range(4)}}
            # the same matrix in HODLR form (hss2hodlr on the device): more bytes, no tree recursion
            r_, yh = time_variant(hm, torch, tree, g, prec, st, 3, copies, True, prof_steps=min(st, 20),
                                  form="hodlr")
            ys["hodlr_from_hss"] = yh
            d = max(range(4), key=lambda k: r_["phases"]["ms"][k])
            variants["hodlr_from_hss"] = {"value": r_["gbs"], "ms_per_step": r_["ms_per_step"], "steps": st,
                                          "storage": prec, "generator_bytes": r_["generator_bytes"],
                                          "dominant_kernel": PHASES[d],
                                          "phase_ms_per_step": {PHASES[k]: r_["phases"]["ms"][k] /
                                                                r_["phases"]["steps"] for k in range(4)}}
            # the Hadamard product of two HSS matrices of ranks 8 and 4 (rank 32), same tree and X
            import workloads as W
            rng_h = W.rng_named("hss_n65536_m256_k32_r64", salt=11)
            gA8 = W.random_hss(rng_h, c, 8)
            gB4 = W.random_hss(rng_h, c, 4)
            gA8["_X"] = X
            r_, yhd = time_variant(hm, torch, tree, gA8, prec, st, 3, copies, True, prof_steps=min(st, 20),
                                   form="hadamard", g_b=gB4)
            d = max(range(4), key=lambda k: r_["phases"]["ms"][k])
            variants["hadamard"] = {"value": r_["gbs"], "ms_per_step": r_["ms_per_step"], "steps": st,
                                    "storage": prec, "ranks": "8 o 4 = 32", "generator_bytes": r_["generator_bytes"],
                                    "dominant_kernel": PHASES[d],
                                    "phase_ms_per_step": {PHASES[k]: r_["phases"]["ms"][k] /
                                                          r_["phases"]["steps"] for k in range(4)}}
        if not args.no_cpu and world == 1:
            if "hadamard" in variants:
                from oracle import hadamard as OHD
                from oracle import matmat as OMM
                hrows = sorted(set([0, N_ - 1] + list(range(255, N_, N_ // 190))))[:192]
                Yh_o = OMM.matmat_rows(c, OHD.hadamard_gens(c, gA8, gB4), X, hrows)
                variants["hadamard"]["err_vs_oracle"] = float(np.max(
                    np.linalg.norm(yhd[hrows] - Yh_o, axis=0) / np.linalg.norm(Yh_o, axis=0)))
                variants["hadamard"]["err_rows"] = len(hrows)
            if "transpose" in variants:
                from oracle import transpose as OTR
                trows = sorted(set([0, N_ - 1] + list(range(255, N_, N_ // 190))))[:192]
                Yt_o = OTR.matmat_transpose_rows(c, g, X, trows)
                variants["transpose"]["err_vs_oracle"] = float(np.max(
                    np.linalg.norm(yt[trows] - Yt_o, axis=0) / np.linalg.norm(Yt_o, axis=0)))
                variants["transpose"]["err_rows"] = len(trows)
            leaves = [0, 1, 127, 128, 200, 255][: max(1, args.cpu_leaves)]
            dt, rows, Yo = cpu_oracle_sample(c, g, X, leaves)
            frac = len(leaves) / len(c)
            bytes64 = fp64_step_bytes(c)
            est = dt / frac
            out["cpu_baseline"] = {"value": bytes64 / est / 1e9, "unit": "GB/s", "cores": os.cpu_count(),
                                   "kind": "oracle",
                                   "sample": "%d of %d leaf row blocks of one product, %.2f s, scaled by %.1f"
                                             % (len(leaves), len(c), dt, 1 / frac)}
            errs = {}
            for v, Yv in ys.items():
                num = np.linalg.norm(Yv[rows] - Yo, axis=0)
                den = np.linalg.norm(Yo, axis=0)
                errs[v] = float(np.max(num / den))
            out["err_vs_oracle"] = {"metric": "max over columns of ||y - y_oracle||_2/||y_oracle||_2 on %d sampled rows"
                                              % len(rows), **errs}
            for v in variants:
                if v in errs:
                    variants[v]["err_vs_oracle"] = errs[v]
        if variants:
            out["variants"] = variants
            if "f64" in variants and prec != "f64":
                out["mixed_vs_fp64_speedup"] = value / world / variants["f64"]["value"]
        print(json.dumps(out))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
