"""CPU fast product of HODLR/HSS matrices (Sec. 4.1, Fig. 4.1) in float64 on
all host cores: the timed CPU baseline next to the GPU library.

``libhm_cpu.so`` is built from ``hm_cpu.cpp`` with g++ and OpenMP by
:func:`build` (called from the repository's ``build()``).  It is neither the
oracle (which expands the defining matrix) nor part of the GPU library, and
shares no code with either.  Generators use the dictionaries of
``workloads`` (lists of column-major float64 blocks in node order).
"""

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hm_cpu.cpp")
LIB = os.path.join(HERE, "libhm_cpu.so")

_lib = None


def build(force=False):
    """Compiles libhm_cpu.so in-tree (portable flags: no -march=native)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("g++ failed for %s:\n%s%s" % (SRC, res.stdout, res.stderr))
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libhm_cpu.so is not built: run cpu_baseline.build()")
        h = C.CDLL(LIB)
        pp = C.POINTER(C.c_void_p)
        i64p = C.POINTER(C.c_int64)
        i32p = C.POINTER(C.c_int32)
        h.hmc_threads.restype = C.c_int
        h.hmc_destroy.argtypes = [C.c_void_p]
        h.hmc_hodlr_create.restype = C.c_void_p
        h.hmc_hodlr_create.argtypes = [C.c_int64, C.c_int32, i64p, pp, pp, pp, pp, pp, i32p, i32p]
        h.hmc_hss_create.restype = C.c_void_p
        h.hmc_hss_create.argtypes = [C.c_int64, C.c_int32, i64p, pp, pp, pp, pp, pp, pp, pp, i32p, i32p]
        h.hmc_matmat.restype = C.c_int
        h.hmc_matmat.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]
        _lib = h
    return _lib


def threads():
    """OpenMP threads a product uses (the cores of the timed baseline)."""
    return int(lib().hmc_threads())


class CpuMatrix:
    """A HODLR or HSS matrix held by the CPU baseline (copies the generators)."""

    def __init__(self, c, g):
        h = lib()
        self._keep = []
        c = [int(v) for v in c]
        L = len(c)
        n = c[-1] if L else 0
        self.n = n
        ends = (C.c_int64 * L)(*c)

        def blocks(lst):
            arr = (C.c_void_p * max(len(lst), 1))()
            for i, b in enumerate(lst):
                if b is None:
                    arr[i] = None
                    continue
                a = np.asfortranarray(np.asarray(b, dtype=np.float64))
                self._keep.append(a)
                arr[i] = a.ctypes.data if a.size else None
            return arr

        if g["kind"] == "hodlr":
            k12 = (C.c_int32 * max(L - 1, 1))(*[int(np.asarray(u).shape[1]) for u in g["U12"]])
            k21 = (C.c_int32 * max(L - 1, 1))(*[int(np.asarray(u).shape[1]) for u in g["U21"]])
            self._h = h.hmc_hodlr_create(n, L, ends, blocks(g["D"]), blocks(g["U12"]), blocks(g["V12"]),
                                         blocks(g["U21"]), blocks(g["V21"]), k12, k21)
        else:
            N = 2 * L - 1
            ku = [0] * N
            kv = [0] * N
            for i in range(L):
                ku[L - 1 + i] = int(np.asarray(g["U"][i]).shape[1])
                kv[L - 1 + i] = int(np.asarray(g["V"][i]).shape[1])
            for q in range(1, L - 1):
                ku[q] = int(np.asarray(g["RU"][q]).shape[1])
                kv[q] = int(np.asarray(g["RV"][q]).shape[1])
            RU = [None] + [g["RU"][q] for q in range(1, N)]
            RV = [None] + [g["RV"][q] for q in range(1, N)]
            self._h = h.hmc_hss_create(n, L, ends, blocks(g["D"]), blocks(g["U"]), blocks(g["V"]),
                                       blocks(RU[:N]), blocks(RV[:N]), blocks(g["B12"]), blocks(g["B21"]),
                                       (C.c_int32 * N)(*ku), (C.c_int32 * N)(*kv))
        self._keep = []
        if not self._h:
            raise MemoryError("hmc create failed (bad generators or out of memory)")

    def matmat(self, X, out=None):
        """Y = A X for an n x r float64 block (returned column-major)."""
        X = np.asfortranarray(np.asarray(X, dtype=np.float64))
        if X.ndim == 1:
            X = X[:, None]
        r = X.shape[1]
        Y = out if out is not None else np.empty((self.n, r), order="F")
        st = lib().hmc_matmat(self._h, r, X.ctypes.data, max(self.n, 1), Y.ctypes.data, max(self.n, 1))
        if st != 0:
            raise RuntimeError("hmc_matmat failed with status %d" % st)
        return Y

    def close(self):
        if getattr(self, "_h", None):
            lib().hmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
