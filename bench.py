#!/usr/bin/env python3
"""Throughput of the HSS matrix-times-block product on GB300.

Workload (one "step" = one product Y = A X through the C ABI):
  HSS, n = 65536, leaf 256 (p = 8), nested rank 32, 64 right-hand sides;
  leaf U, V orthonormal (Q of a Gaussian QR), translations R and couplings B
  iid N(0, 1/32) (variance), D ~ N(0,1) + 8 I, X ~ N(0,1); seeded.
  Headline: FP64 storage, FP64 X and Y (the paper's arithmetic); the other
  storages (BF16, split BF16, FP32) are timed as variants in the same run,
  each with its time ratio to FP64 and its error against the FP64 oracle,
  next to the HODLR n=4096 FP64 r=1 and exponential-kernel n=262144
  (r = 1 and 128) workloads.

Timing: W untimed steps, then exactly K steps bracketed by a barrier and
torch.cuda.synchronize() on both sides, CUDA events on the launching stream,
max over ranks.  The inputs rotate over several resident copies whose total
exceeds the 135 MB L2, so every step streams its generators from HBM.

Rooflines: the FP64 products are bound by the FP64 pipe (about 1/64 of the
FP32 rate on this GPU), so their denominator is the FP64 FMA throughput that
libhm_probe.so measures in this process; the FP32 tree kernel's is the FP32
FMA throughput; the reduced-precision leaf kernels are HBM-bound and use the
measured copy bandwidth of MEASURED_PEAKS.json.

--impl reference times the CPU oracle (the FP64 dense-definition product)
on a bounded sample of the same workload.  N > 1 (torchrun): each rank runs
its own replica (weak scaling, no collective on the data path).
"""

import argparse
import ctypes
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
L2_BYTES = 135.5e6
# FP64 FMA rate from the recipe's unit counts: 152 SMs x 2 FMA/cycle x 2 flops
# x 2.07 GHz (NVIDIA's stated 1.25 TFLOP/s), and the FP32 SIMT rate: 152 SMs x
# 128 lanes x 2 flops x 2.07 GHz.  Context for the measured denominators.
FP64_NOMINAL_TFLOPS = 1.25
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hm", choices=["hm", "reference"])
    ap.add_argument("--precision", default="f64", choices=["bf16", "f32", "f64", "bf16x2"])
    ap.add_argument("--copies", type=int, default=0, help="resident copies (0 = enough to exceed L2)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-workloads", action="store_true", help="skip the n=4096 and n=262144 workloads")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tree-shape", default="", help="pin the tree kernel shape 'cluster,columns,slots' (no tuning)")
    ap.add_argument("--no-solve", action="store_true", help="skip the HSS solve variant")
    ap.add_argument("--cpu-leaves", type=int, default=6, help="leaf row blocks in the CPU oracle sample")
    ap.add_argument("--workload", default="hss", choices=["hss", "exp", "hodlr4096", "batched", "serve"],
                    help="hss: the HSS n=65536 headline; exp: the exponential-kernel HODLR n=262144; "
                         "hodlr4096: HODLR n=4096 FP64 r=1; batched: 512 uneven matrices; serve: Poisson requests")
    ap.add_argument("--storages", default="", help="exp: comma-separated storages (default all)")
    ap.add_argument("--rhs", default="", help="exp: comma-separated right-hand-side counts (default 1,128)")
    ap.add_argument("--count", type=int, default=0, help="matrices in the batched / serving workload")
    ap.add_argument("--rates", default="1000,5000,10000,20000,50000")
    ap.add_argument("--seconds", type=float, default=1.0, help="arrival window per rate (serve)")
    ap.add_argument("--probe-sweep", action="store_true",
                    help="only print the FP32 / FP64 / FP64-mma pipe throughput over several launch shapes")
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


PROBE_SHAPE = {"fp32": (0, 2, 256, 20000), "fp64": (1, 2, 256, 400)}


def _probe_lib():
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1909_07909_gb300", "libhm_probe.so"))
    lib.hm_probe_peak.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_double),
                                                       ctypes.POINTER(ctypes.c_double),
                                                       ctypes.POINTER(ctypes.c_int)]
    return lib


def probe_sweep():
    """Pipe throughput over launch shapes (FP32 FMA, FP64 FMA, FP64 mma.sync)."""
    import torch
    torch.cuda.set_device(0)
    lib = _probe_lib()
    rows = []
    for which, name, iters in ((0, "fp32_fma", 20000), (1, "fp64_fma", 400), (2, "fp64_mma", 400)):
        for bps, thr in ((1, 128), (1, 256), (2, 256), (4, 256), (8, 256)):
            tf, ms, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
            rc = lib.hm_probe_peak(which, bps, thr, iters, 3, ctypes.byref(tf), ctypes.byref(ms), ctypes.byref(sms))
            rows.append({"probe": name, "blocks_per_sm": bps, "threads": thr, "rc": rc, "tflops": tf.value,
                         "ms": ms.value, "sms": sms.value})
    print(json.dumps({"pipe_probe_sweep": rows}))
    return 0


def probe_pipes():
    """FP32 and FP64 FMA throughput of this GPU, measured now by libhm_probe.so
    (paper_1909_07909_gb300/probe/peak_probe.cu): SMs x 2 blocks x 256
    threads, 8 independent FMA chains per thread, best of 3 launches after a
    warm-up launch.  Returns {name: {"tflops", "ms", "shape"}}."""
    lib = _probe_lib()
    out = {}
    for name, (which, bps, thr, iters) in PROBE_SHAPE.items():
        tf, ms, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        rc = lib.hm_probe_peak(which, bps, thr, iters, 3, ctypes.byref(tf), ctypes.byref(ms), ctypes.byref(sms))
        if rc != 0:
            raise RuntimeError("pipe probe %s failed with CUDA error %d" % (name, rc))
        out[name] = {"tflops": tf.value, "ms": ms.value,
                     "shape": "%d SMs x %d blocks x %d threads, 8 FMA chains per thread, %d x 4 FMAs per "
                              "chain, best of 3" % (sms.value, bps, thr, iters)}
    return out


# ---------------------------------------------------------------------------
# Algorithmic work of one product, per phase (the roofline's numerators)
# ---------------------------------------------------------------------------

def _elems(blocks):
    import numpy as np
    return int(sum(np.asarray(b).size for b in blocks if b is not None))


def gen_counts(g):
    """Generator element counts of a workload's generator dict (unpadded)."""
    if g["kind"] == "hodlr":
        return {"D": _elems(g["D"]), "U": _elems(g["U12"]) + _elems(g["U21"]),
                "V": _elems(g["V12"]) + _elems(g["V21"]), "tree": 0}
    return {"D": _elems(g["D"]), "U": _elems(g["U"]), "V": _elems(g["V"]),
            "tree": _elems(g["RU"]) + _elems(g["RV"]) + _elems(g["B12"]) + _elems(g["B21"])}


def phase_work(g, n, r, storage):
    """Algorithmic bytes and flops per launch of every phase of one product
    (generators read once in the storage type, X read, Y written; per-node
    k x r intermediates excluded).  The tree operators are held in FP64 for
    FP64 storage and in FP32 otherwise.  Phase names follow
    hm_matrix_phase_times: project, tree, tree_down, expand, dpart (the FP64
    diagonal-block product D X; the expansion then adds E Z to Y)."""
    gc = gen_counts(g)
    s = ESZ[storage]
    xs = XSZ[X_DTYPE[storage]]
    ys = 8 if storage == "f64" else 4
    ts = 8 if storage == "f64" else 4
    io = n * r
    w = {"project": {"bytes": gc["V"] * s + io * xs, "flops": 2 * gc["V"] * r},
         "tree": {"bytes": gc["tree"] * ts, "flops": 2 * gc["tree"] * r},
         "tree_down": {"bytes": 0, "flops": 0},
         "expand": {"bytes": (gc["D"] + gc["U"]) * s + io * (xs + ys), "flops": 2 * (gc["D"] + gc["U"]) * r},
         "dpart": {"bytes": 0, "flops": 0}}
    return w, gc


def split_work(w, gc, n, r, storage):
    """The FP64 wide-block path runs D X as its own launch (phase dpart) and
    the expansion as Y += E Z (reading and writing Y)."""
    s, xs, ys = ESZ[storage], XSZ[X_DTYPE[storage]], 8
    w = dict(w)
    w["dpart"] = {"bytes": gc["D"] * s + n * r * (xs + ys), "flops": 2 * gc["D"] * r}
    w["expand"] = {"bytes": gc["U"] * s + n * r * 2 * ys, "flops": 2 * gc["U"] * r}
    return w


PHASES = ["project", "tree", "tree_down", "expand", "dpart"]
KERNEL_NAMES = {
    ("f64", "dpart"): "k_leaf_f64<1, 32> (FP64 diagonal-block product D X, register-tiled)",
    ("f64", "expand"): "k_leaf_f64<2, *> / k_expand<F64> (FP64 leaf expansion)",
    ("f64", "project"): "k_leaf_f64<0, *> / k_project<F64> (FP64 leaf projection)",
    ("f64", "tree"): "k_tree_cluster<double, *> (FP64 tree)",
}


def roofline(w, phases, storage, peaks, pipes, tc):
    """Roofline of the dominant kernel of one product from the profiled
    pass's per-launch CUDA-event durations.  FP64: every phase is bound by
    the FP64 pipe.  Otherwise the bound is the one the kernel's arithmetic
    intensity puts it under: FP32 FMA pipe (SIMT and the FP32 tree), BF16
    tensor pipe (tensor-core leaf kernels, `tc`), or HBM."""
    ms, ln = phases["ms"], phases["launches"]
    dom = max(range(len(PHASES)), key=lambda k: ms[k])
    name = PHASES[dom]
    avg_ms = ms[dom] / max(ln[dom], 1)
    wk = w[name]
    hbm = peaks["hbm_gbs"]
    if storage == "f64":
        bound, peak, unit, ach = "alu", pipes["fp64"]["tflops"], "TFLOP/s", wk["flops"] / (avg_ms * 1e-3) / 1e12
        src = "FP64 FMA throughput measured in this run (libhm_probe.so, %s)" % pipes["fp64"]["shape"]
    else:
        if name == "tree" or not tc:
            pk_f = pipes["fp32"]["tflops"]
            src_f = "FP32 FMA throughput measured in this run (libhm_probe.so, %s)" % pipes["fp32"]["shape"]
        else:
            pk_f = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
            src_f = "BF16 dense tensor peak (MEASURED_PEAKS.json, sustained)"
        intensity = wk["flops"] / max(wk["bytes"], 1)
        if wk["bytes"] == 0 or intensity * hbm * 1e9 >= pk_f * 1e12:
            bound, peak, unit, src = ("alu" if name == "tree" or not tc else "tensor"), pk_f, "TFLOP/s", src_f
            ach = wk["flops"] / (avg_ms * 1e-3) / 1e12
        else:
            bound, peak, unit, src = "hbm", hbm, "GB/s", "copy bandwidth (MEASURED_PEAKS.json)"
            ach = wk["bytes"] / (avg_ms * 1e-3) / 1e9
    return {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
            "peak_source": src, "phase": name, "ms_per_launch": avg_ms,
            "bytes_per_launch": wk["bytes"], "flops_per_launch": wk["flops"]}


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

# --tree-shape: a pinned launch shape of the tree kernel (cluster CTAs,
# columns, ring slots) instead of timing every shape; for profiler runs,
# where the timings that pick a shape are distorted.
TREE_SHAPE = None


def pick_tree(A, r, storage):
    """Pin the --tree-shape launch shape when given (and it fits), else time
    every shape and keep the fastest; returns the tuned ms or None."""
    if TREE_SHAPE is not None:
        try:
            A.set_tree_shape(r, *TREE_SHAPE)
            return None
        except Exception:
            pass
    return A.tune_tree(r, X_DTYPE[storage], "f64" if storage == "f64" else "f32")


def make_inputs():
    import workloads as W
    rng = W.rng_named("hss_n65536_m256_k32_r64")
    import paper_1909_07909_gb300 as hm
    tree = hm.Tree.default(N_, LEAF)
    c = tree.leaf_ends
    g = W.random_hss(rng, c, RANK)
    X = rng.standard_normal((N_, RHS))
    return tree, c, g, X


def fp64_step_bytes(c):
    """Algorithmic bytes of one FP64 product: all generators read once, X read, Y written."""
    L = len(c)
    sizes = [c[0]] + [c[i] - c[i - 1] for i in range(1, L)]
    elems = sum(m * m for m in sizes) + 2 * N_ * RANK + max(L - 2, 0) * 4 * RANK * RANK + \
        max(2 * L - 2, 0) * RANK * RANK
    return 8 * elems + N_ * RHS * 16


def step_bytes(A, storage, n, r):
    ys = 8 if storage == "f64" else 4
    return A.generator_bytes() + n * r * (XSZ[X_DTYPE[storage]] + ys)


def copies_for(bytes_per_step, want=0):
    return want or max(1 if bytes_per_step > 1.5 * L2_BYTES else 2, math.ceil(2.2 * L2_BYTES / bytes_per_step))


def time_variant(hm, torch, tree, g, storage, X, steps, warmup, copies, clock_index=None, prof_steps=None,
                 world=1, form=None, g_b=None):
    """Device throughput of one storage type on the product Y = A X (timed
    region without profiling events, so consecutive kernels overlap), then a
    profiled pass that brackets every kernel with CUDA events for per-kernel
    durations.  form="transpose" times Y = A^T X (matrices from
    hm_matrix_transpose); form="hodlr" the HODLR form of the HSS matrix
    (hm_hss_to_hodlr); form="hadamard" the Hadamard product of g and g_b."""
    n, r = X.shape
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
    Xh = torch.from_numpy(X.T.copy())
    Xs = [Xh.to(dev).to(xd).t() for _ in range(copies)]
    Ys = [torch.empty((r, n), dtype=td, device=dev).t() for _ in range(copies)]
    tree_ms = None
    for A in mats:
        A.reserve(r)
        # the fastest launch shape of the tree kernel for this product (no result changes)
        tree_ms = pick_tree(A, r, storage)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    code = hm.HM_F64 if storage == "f64" else hm.HM_F32
    xcode = {"f64": hm.HM_F64, "f32": hm.HM_F32, "bf16": hm.HM_BF16}[X_DTYPE[storage]]

    def run(i):
        j = i % copies
        mats[j].matmat_raw(r, Xs[j].data_ptr(), n, xcode, Ys[j].data_ptr(), n, code, sptr)

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
    ps = prof_steps or steps
    for A in mats:
        A.profile(True)
        A.phase_times()
    for i in range(ps):
        run(i)
    torch.cuda.synchronize()
    acc_ms = [0.0] * len(PHASES)
    acc_n = [0] * len(PHASES)
    for A in mats:
        ms, nl = A.phase_times()
        A.profile(False)
        for k in range(len(PHASES)):
            acc_ms[k] += ms[k]
            acc_n[k] += nl[k]
    info = mats[0].info()
    res = {"ms_total": ms_total, "ms_per_step": ms_total / steps,
           "bytes_per_step": step_bytes(mats[0], storage, n, r),
           "phases": {"ms": acc_ms, "launches": acc_n, "steps": ps},
           "clocks": sampler.summary() if sampler else None,
           "generator_bytes": mats[0].generator_bytes(), "info": info,
           "launches_per_step": sum(acc_n) / ps,
           "tree_shape": {"cluster_ctas": info["tree_cluster"], "columns": info["tree_columns"],
                          "ring_slots": info["tree_ring"], "tuned_ms": tree_ms}}
    res["gbs"] = res["bytes_per_step"] / (res["ms_per_step"] * 1e-3) / 1e9
    Y0 = Ys[0].to(torch.float64).cpu().numpy()
    del mats
    return res, Y0


def e2e_host(hm, torch, tree, g, storage, X, steps, copies):
    """The same product through the C ABI with pinned host buffers: every
    call copies X to the device and Y back inside the timed region.  The
    matrices rotate over the same number of resident copies as the device
    arm, so every product streams its generators from HBM."""
    n, r = X.shape
    mats = [hm.Matrix.create(tree, g, storage) for _ in range(copies)]
    for A in mats:
        A.reserve(r)
        pick_tree(A, r, storage)
    f64 = storage == "f64"
    td = torch.float64 if f64 else torch.float32
    xd = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[X_DTYPE[storage]]
    Xp = torch.from_numpy(X.T.copy()).to(xd).pin_memory()
    Yp = torch.empty((r, n), dtype=td).pin_memory()
    code = hm.HM_F64 if f64 else hm.HM_F32
    xcode = {"f64": hm.HM_F64, "f32": hm.HM_F32, "bf16": hm.HM_BF16}[X_DTYPE[storage]]
    stream = torch.cuda.current_stream().cuda_stream
    for i in range(max(3, copies)):
        mats[i % copies].matmat_raw(r, Xp.data_ptr(), n, xcode, Yp.data_ptr(), n, code, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        mats[i % copies].matmat_raw(r, Xp.data_ptr(), n, xcode, Yp.data_ptr(), n, code, stream)
    dt = (time.perf_counter() - t0) / steps
    ys = 8 if f64 else 4
    xs = XSZ[X_DTYPE[storage]]
    b = mats[0].generator_bytes() + n * r * (xs + ys)
    del mats
    return {"value": b / dt / 1e9, "unit": "GB/s", "h2d_bytes_per_step": n * r * xs,
            "d2h_bytes_per_step": n * r * ys, "ms_per_step": dt * 1e3,
            "l2": "%d rotating resident matrices" % copies}


def time_ulv(hm, torch, tree, g, X, steps):
    """The HSS solve X = A^{-1} B (Sec. 4.3, implicit ULV) on the headline
    matrix in FP64: the factorization once (host-timed, synchronous), then
    `steps` solves with the 64 right-hand sides (CUDA events), and the backward
    error ||A X - B||_F / ||B||_F through the FP64 product."""
    A = hm.Matrix.create(tree, g, "f64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F = A.ulv()
    t_factor = time.perf_counter() - t0
    n, r = X.shape
    B = torch.from_numpy(X.T.copy()).cuda().t()
    Xs = F.solve(B)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        F.solve(B, Xs)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    R = A.matmat(Xs) - B
    rel = (torch.linalg.norm(R) / torch.linalg.norm(B)).item()
    F.close()
    return {"storage": "f64", "rhs": r, "factor_ms": t_factor * 1e3, "ms_per_solve": ms, "steps": steps,
            "backward_error": rel, "metric": "||A X - B||_F / ||B||_F through the FP64 product"}


def cpu_fast_baseline(c, g, X, runs=3):
    """The paper's fast product (Fig. 4.1) in FP64 C++/OpenMP on all host
    cores (cpu_baseline/libhm_cpu.so): one warm-up product, then the best of
    `runs` full products.  Returns (seconds, threads, Y)."""
    import cpu_baseline as CB
    M = CB.CpuMatrix(c, g)
    Y = M.matmat(X)
    best = 1e30
    for _ in range(runs):
        t0 = time.perf_counter()
        M.matmat(X, out=Y)
        best = min(best, time.perf_counter() - t0)
    M.close()
    return best, CB.threads(), Y


def cpu_oracle_sample(c, g, X, leaves):
    """Oracle (dense-definition product) on `leaves` leaf row blocks; returns
    (seconds, rows, Yrows)."""
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


def col_err(Y, ref):
    import numpy as np
    num = np.linalg.norm(Y - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(num / np.where(den == 0, 1.0, den)))


def summarize(res, w, storage, peaks, pipes, tc, extra=None):
    ph = res["phases"]
    roof = roofline(w, ph, storage, peaks, pipes, tc)
    out = {"value": res["gbs"], "unit": "GB/s", "ms_per_step": res["ms_per_step"],
           "bytes_per_step": res["bytes_per_step"], "tree_shape": res.get("tree_shape"),
           "phase_ms_per_step": {PHASES[k]: ph["ms"][k] / ph["steps"] for k in range(len(PHASES))},
           "roofline": roof}
    if extra:
        out.update(extra)
    return out


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
    print(json.dumps(batched_result(args)))
    return 0


def batched_result(args):
    """The batched workload (one JSON object; args: steps, warmup, count)."""
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
    return out


# ---------------------------------------------------------------------------
# Serving workload: 64 resident HSS matrices (n = 2^12..2^18, rank 16..64,
# BF16), Poisson arrivals, 1..16 right-hand sides per request.
# ---------------------------------------------------------------------------

def run_serve(args):
    print(json.dumps(serve_result(args)))
    return 0


def serve_result(args):
    """The serving workload (one JSON object; args: count, rates, seconds)."""
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
    return out


def guarded(variants, name, fn):
    """Adds fn()'s entries to variants; an exception (a refused request, a
    timed-out device wait) becomes {name: {"error": ...}} and a traceback on
    stderr, so that the headline measured before it is still printed."""
    try:
        variants.update(fn())
    except Exception as e:  # noqa: BLE001 - recorded in the output line, not swallowed
        import traceback
        traceback.print_exc()
        variants[name] = {"error": "%s: %s" % (type(e).__name__, e)}


def batched_and_served(args, torch):
    """Compact entries for the batched (512 matrices) and served (64 resident
    matrices, Poisson arrivals) workloads, run after the single-matrix ones."""
    import types
    torch.cuda.empty_cache()
    ns = types.SimpleNamespace(steps=max(3, min(10, args.steps)), warmup=2, count=0, rates=args.rates,
                               seconds=min(args.seconds, 0.5))
    b = batched_result(ns)
    keep = ("batched_ms", "batched_gbs", "loop_ms", "loop_gbs", "launches_per_run", "bytes_per_run")
    out = {"batched_512": {"value": b["value"], "unit": "GB/s", "ms_per_step": b["ms_per_step"],
                           "config": b["config"]["workload"],
                           "batched_vs_fp64_unbatched": b["batched_vs_fp64_unbatched"],
                           "storages": {k: {f: v[f] for f in keep if f in v} for k, v in b["variants"].items()}}}
    torch.cuda.empty_cache()
    sv = serve_result(ns)
    out["served_64"] = {"value": sv["value"], "unit": sv["unit"], "p50_ms": sv["ms_per_step"],
                        "sustained_rps": sv["sustained_rps"],
                        "saturation_throughput_rps": sv["saturation_throughput_rps"],
                        "fp64_unbatched_ms_per_request_r8": sv["fp64_unbatched_ms_per_request_r8"],
                        "config": sv["config"]["workload"],
                        "by_rate": {k: {f: v[f] for f in ("p50_ms", "p99_ms", "throughput_rps", "refused")}
                                    for k, v in sv["by_rate"].items()}}
    torch.cuda.empty_cache()
    return out


def run_workloads(hm, torch, np, peaks, pipes, steps, warmup, with_cpu, which=("hodlr4096", "exp"), storages=None,
                  rhs=None):
    """The other single-matrix workloads, each with its own roofline:
    HODLR n=4096 leaf 128 rank 8 r=1 FP64 (L2-resident: 48 rotating copies)
    and the exact rank-8 exponential kernel HODLR n=262144 leaf 256 at r=1 and
    r=128 in every storage; errors against the oracle (the O(nK) recurrence
    for r=1, sampled dense rows for r=128, the dense product for n=4096)."""
    out = {}
    if "hodlr4096" in which:
        out.update(_run_hodlr4096(hm, torch, np, peaks, pipes, steps, warmup, with_cpu))
    if "exp" in which:
        out.update(_run_exp(hm, torch, np, peaks, pipes, steps, warmup, with_cpu, storages, rhs))
    return out


def _run_hodlr4096(hm, torch, np, peaks, pipes, steps, warmup, with_cpu):
    import workloads as W
    from oracle import matmat as OM
    out = {}
    rng = W.rng_named("hodlr_n4096_m128_k8_r1_f64")
    tree = hm.Tree.default(4096, 128)
    c = tree.leaf_ends
    g = W.random_hodlr(rng, c, 8)
    X = rng.standard_normal((4096, 1))
    w, _ = phase_work(g, 4096, 1, "f64")
    res, Y = time_variant(hm, torch, tree, g, "f64", X, max(steps, 200), warmup, 48, prof_steps=50)
    ent = summarize(res, w, "f64", peaks, pipes, False,
                    {"workload": "hodlr n=4096 leaf=128 rank=8 r=1", "storage": "f64",
                     "l2": "48 rotating copies of %.1f MB (one matrix fits in L2)" % (res["bytes_per_step"] / 1e6),
                     "launches_per_step": res["launches_per_step"]})
    if with_cpu:
        ent["err_vs_oracle"] = col_err(Y, OM.matmat(c, g, X))
    out["hodlr_n4096_r1_f64"] = ent
    return out


def _run_exp(hm, torch, np, peaks, pipes, steps, warmup, with_cpu, storages=None, rhs=None):
    import workloads as W
    from oracle import expkernel as OE, matmat as OM
    out = {}
    rng = W.rng_named("hodlr_exp_n262144_m256_K8")
    n = 262144
    t = W.exp_points(rng, n)
    ck, lk = W.exp_params(8)
    tree = hm.Tree.default(n, 256)
    c = tree.leaf_ends
    g = W.exp_kernel_hodlr(t, c, ck, lk)
    rows = sorted(set([0, n - 1] + [int(v) for v in np.linspace(255, n - 2, 158)]))
    for r, sts in ((1, ("f32", "bf16", "bf16x2", "f64")), (128, ("bf16", "bf16x2", "f32", "f64"))):
        X = rng.standard_normal((n, r))
        if rhs and r not in rhs:
            continue
        for st in sts:
            if storages and st not in storages:
                continue
            w, _ = phase_work(g, n, r, st)
            f64_split = st == "f64" and r >= 12
            if f64_split:
                w = split_work(w, gen_counts(g), n, r, st)
            nst = max(3, steps // 2) if (st == "f64" and r > 1) else max(steps, 20)
            res, Y = time_variant(hm, torch, tree, g, st, X, nst, 2, 1, prof_steps=min(nst, 10))
            ent = summarize(res, w, st, peaks, pipes, st in ("bf16", "bf16x2") and r >= 16,
                            {"workload": "hodlr exp kernel n=262144 leaf=256 K=8 r=%d" % r, "storage": st,
                             "x_dtype": X_DTYPE[st],
                             "l2": "one matrix of %.0f MB per product (larger than L2)" % (res["generator_bytes"] / 1e6),
                             "launches_per_step": res["launches_per_step"]})
            if with_cpu:
                Xe = X if st == "f64" else np.asarray(
                    torch.from_numpy(X).to({"f32": torch.float32, "bf16": torch.bfloat16}[X_DTYPE[st]])
                    .to(torch.float64).numpy())
                if r == 1:
                    ent["err_vs_oracle"] = col_err(Y, OE.apply(t, ck, lk, Xe))
                    ent["err_rows"] = "all %d (O(nK) recurrence)" % n
                else:
                    ent["err_vs_oracle"] = col_err(Y[rows], OM.matmat_rows(c, g, Xe, rows))
                    ent["err_rows"] = "%d sampled rows (dense oracle)" % len(rows)
            out["exp_n262144_r%d_%s" % (r, st)] = ent
            del Y
        del X
    return out


def run_workload_only(args):
    """One of the other single-matrix workloads on its own (one JSON line)."""
    import numpy as np
    import torch
    import paper_1909_07909_gb300 as hm
    torch.cuda.set_device(0)
    peaks, _ = measured_peaks()
    pipes = probe_pipes()
    storages = [v for v in args.storages.split(",") if v] or None
    rhs = [int(v) for v in args.rhs.split(",") if v] or None
    res = run_workloads(hm, torch, np, peaks, pipes, args.steps, args.warmup, not args.no_cpu, (args.workload,),
                        storages, rhs)
    print(json.dumps({"metric": METRIC, "workload": args.workload, "unit": "GB/s", "data": "synthetic",
                      "variants": res, "pipe_probe": pipes}))
    return 0


def main():
    global TREE_SHAPE
    args = parse()
    if args.tree_shape:
        TREE_SHAPE = tuple(int(v) for v in args.tree_shape.split(","))
    rank, local, world = dist_env()
    if args.impl == "reference":
        return run_reference(args)
    if args.probe_sweep:
        return probe_sweep() if rank == 0 else 0
    if args.workload in ("exp", "hodlr4096"):
        return run_workload_only(args) if rank == 0 else 0
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
    pipes = probe_pipes()
    tree, c, g, X = make_inputs()
    prec = args.precision
    w, gc = phase_work(g, N_, RHS, prec)
    if prec == "f64":
        w = split_work(w, gc, N_, RHS, prec)
    est = {"bf16": 45e6, "f32": 90e6, "bf16x2": 90e6, "f64": 180e6}[prec] + N_ * RHS * (16 if prec == "f64" else 8)
    copies = copies_for(est, args.copies)

    if world > 1:
        torch.distributed.barrier()
    head, Yh = time_variant(hm, torch, tree, g, prec, X, args.steps, args.warmup, copies, clock_index=local,
                            prof_steps=min(args.steps, 20), world=world)
    # whole-job time: max over ranks of this rank's timed region
    ms_max = max_over_ranks(head["ms_total"], world, "cuda")
    value = job_throughput(head["bytes_per_step"], args.steps, ms_max, world)

    tc = prec in ("bf16", "bf16x2")
    roof = roofline(w, head["phases"], prec, peaks, pipes, tc)
    roof["kernel"] = KERNEL_NAMES.get((prec, roof["phase"]), "%s (%s storage)" % (roof["phase"], prec))
    roof["traffic"] = traffic_for("hss_n65536:%s_%s" % (roof["phase"], prec))
    step_flops = sum(v["flops"] for v in w.values())
    if prec == "f64":
        roof["peak_nominal"] = FP64_NOMINAL_TFLOPS
        roof["step"] = {"flops": step_flops, "achieved": step_flops / (ms_max / args.steps * 1e-3) / 1e12,
                        "unit": "TFLOP/s"}
        roof["step"]["frac"] = roof["step"]["achieved"] / roof["peak"]
    ph = head["phases"]
    roof["phase_ms_per_step"] = {PHASES[k]: ph["ms"][k] / ph["steps"] for k in range(len(PHASES))}
    roof["tree_shape"] = head.get("tree_shape")

    out = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N_, "leaf": LEAF, "rank": RANK, "rhs": RHS, "storage": prec,
                      "x_dtype": X_DTYPE[prec], "y_dtype": "f64" if prec == "f64" else "f32",
                      "l2": "inputs larger than L2: %d rotating resident copies of %.1f MB" %
                            (copies, head["bytes_per_step"] / 1e6),
                      "generators": "leaf U,V orthonormal; R,B iid N(0,1/32) (variance); D=N(0,1)+8I; X=N(0,1)",
                      "parallelism": "replicas" if world > 1 else "single"},
           "roofline": roof,
           "gpu_launches": int(round(head["launches_per_step"] * args.steps)),
           "clocks": head["clocks"],
           "pipe_probe": pipes}

    if rank == 0:
        out["e2e"] = e2e_host(hm, torch, tree, g, prec, X, max(5, min(20, args.steps)), copies)
        variants = {}
        ys = {prec: Yh}
        if not args.no_variants:
            for v in ["bf16", "bf16x2", "f32", "f64"]:
                if v == prec:
                    continue
                wv, _ = phase_work(g, N_, RHS, v)
                if v == "f64":
                    wv = split_work(wv, gc, N_, RHS, v)
                ev = {"bf16": 45e6, "f32": 90e6, "bf16x2": 90e6, "f64": 180e6}[v] + N_ * RHS * (16 if v == "f64" else 8)
                st = max(10, args.steps) if v == "f64" else max(20, args.steps)
                r_, yv = time_variant(hm, torch, tree, g, v, X, st, 3, copies_for(ev), prof_steps=min(st, 20))
                ys[v] = yv
                variants[v] = summarize(r_, wv, v, peaks, pipes, v in ("bf16", "bf16x2"),
                                        {"steps": st, "x_dtype": X_DTYPE[v]})
                variants[v]["time_ratio_vs_" + prec] = (ms_max / args.steps) / r_["ms_per_step"]
            # derived matrices on BF16 storage: the transposed product, the
            # HODLR form (hss2hodlr) and a Hadamard product (ranks 8 o 4)
            st = max(20, args.steps)
            ebf = 45e6 + N_ * RHS * 6
            for form in ("transpose", "hodlr"):
                r_, yf = time_variant(hm, torch, tree, g, "bf16", X, st, 3, copies_for(ebf), prof_steps=min(st, 20),
                                      form=form)
                key = "transpose" if form == "transpose" else "hodlr_from_hss"
                ys[key] = yf
                variants[key] = {"value": r_["gbs"], "ms_per_step": r_["ms_per_step"], "steps": st, "storage": "bf16",
                                 "generator_bytes": r_["generator_bytes"],
                                 "phase_ms_per_step": {PHASES[k]: r_["phases"]["ms"][k] / r_["phases"]["steps"]
                                                       for k in range(len(PHASES))}}
            import workloads as W
            rng_h = W.rng_named("hss_n65536_m256_k32_r64", salt=11)
            gA8 = W.random_hss(rng_h, c, 8)
            gB4 = W.random_hss(rng_h, c, 4)
            r_, yhd = time_variant(hm, torch, tree, gA8, "bf16", X, st, 3, copies_for(ebf), prof_steps=min(st, 20),
                                   form="hadamard", g_b=gB4)
            variants["hadamard"] = {"value": r_["gbs"], "ms_per_step": r_["ms_per_step"], "steps": st,
                                    "storage": "bf16", "ranks": "8 o 4 = 32", "generator_bytes": r_["generator_bytes"],
                                    "phase_ms_per_step": {PHASES[k]: r_["phases"]["ms"][k] / r_["phases"]["steps"]
                                                          for k in range(len(PHASES))}}
        if not args.no_variants and not args.no_solve:
            guarded(variants, "ulv_solve_f64", lambda: {"ulv_solve_f64": time_ulv(hm, torch, tree, g, X,
                                                                                 max(5, min(20, args.steps)))})
        if not args.no_workloads:
            guarded(variants, "workloads", lambda: run_workloads(hm, torch, np, peaks, pipes, args.steps, 3,
                                                                 not args.no_cpu and world == 1))
            guarded(variants, "batched_and_served", lambda: batched_and_served(args, torch))
        if not args.no_cpu and world == 1:
            # the timed CPU baseline: the fast tree product on every host core
            secs, thr, Ycpu = cpu_fast_baseline(c, g, X)
            b64 = fp64_step_bytes(c)
            out["cpu_baseline"] = {"value": b64 / secs / 1e9, "unit": "GB/s", "cores": thr, "kind": "fast_matvec",
                                   "ms_per_step": secs * 1e3,
                                   "sample": "the whole product (n=65536, r=64, FP64): Fig. 4.1 in C++/OpenMP "
                                             "(cpu_baseline/hm_cpu.cpp), best of 3 after a warm-up product"}
            # the oracle itself, on a bounded sample
            leaves = [0, 1, 127, 128, 200, 255][: max(1, args.cpu_leaves)]
            dt, rows, Yo = cpu_oracle_sample(c, g, X, leaves)
            frac = len(leaves) / len(c)
            out["cpu_oracle"] = {"value": b64 / (dt / frac) / 1e9, "unit": "GB/s", "cores": os.cpu_count(),
                                 "kind": "oracle",
                                 "sample": "%d of %d leaf row blocks of one product, %.2f s, scaled by %.1f"
                                           % (len(leaves), len(c), dt, 1 / frac)}
            errs = {"cpu_fast_matvec": col_err(Ycpu[rows], Yo)}
            for v, Yv in ys.items():
                if v in ("transpose", "hodlr_from_hss"):
                    continue
                errs[v] = col_err(Yv[rows], Yo)
            errs["hodlr_from_hss"] = col_err(ys["hodlr_from_hss"][rows], Yo) if "hodlr_from_hss" in ys else None
            out["err_vs_oracle"] = {"metric": "max over columns of ||y - y_oracle||_2/||y_oracle||_2 on %d "
                                              "sampled rows" % len(rows), **errs}
            for v in variants:
                if v in errs and errs[v] is not None:
                    variants[v]["err_vs_oracle"] = errs[v]
            if "hadamard" in variants:
                from oracle import hadamard as OHD
                from oracle import matmat as OMM
                hrows = sorted(set([0, N_ - 1] + list(range(255, N_, N_ // 190))))[:192]
                Yh_o = OMM.matmat_rows(c, OHD.hadamard_gens(c, gA8, gB4), X, hrows)
                variants["hadamard"]["err_vs_oracle"] = col_err(yhd[hrows], Yh_o)
                variants["hadamard"]["err_rows"] = len(hrows)
            if "transpose" in ys:
                from oracle import transpose as OTR
                trows = sorted(set([0, N_ - 1] + list(range(255, N_, N_ // 190))))[:192]
                Yt_o = OTR.matmat_transpose_rows(c, g, X, trows)
                variants["transpose"]["err_vs_oracle"] = col_err(ys["transpose"][trows], Yt_o)
                variants["transpose"]["err_rows"] = len(trows)
        if variants:
            out["variants"] = variants
        print(json.dumps(out))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
