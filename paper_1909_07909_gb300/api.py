"""Python objects over the C ABI: trees, HODLR/HSS matrices and their products.

Only argument marshalling happens here; every step of a product runs in the
library's CUDA kernels.  Blocks are passed as float64 column-major numpy
arrays; right-hand sides are (n, r) column-major torch tensors (device or
host) or Fortran-ordered numpy arrays (host).
"""

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import check, lib

vp = C.c_void_p

try:  # torch is only needed for device tensors
    import torch
except Exception:  # pragma: no cover
    torch = None


def _dtype_code(d):
    if isinstance(d, int):
        return d
    if isinstance(d, str):
        return L.DTYPES[d]
    if torch is not None:
        if d == torch.float64:
            return L.HM_F64
        if d == torch.float32:
            return L.HM_F32
        if d == torch.bfloat16:
            return L.HM_BF16
    if d == np.float64:
        return L.HM_F64
    if d == np.float32:
        return L.HM_F32
    raise ValueError("unsupported dtype %r" % (d,))


class Tree:
    """Cluster tree (Def. 2.1) given by its leaf-end vector c (Sec. 3.7)."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def from_leaf_ends(cls, c):
        c = [int(v) for v in c]
        arr = (C.c_int64 * len(c))(*c)
        h = vp()
        check(lib.hm_tree_create(c[-1] if c else 0, arr, len(c), C.byref(h)), "hm_tree_create")
        return cls(h)

    @classmethod
    def default(cls, n, n_min=256):
        h = vp()
        check(lib.hm_tree_default(int(n), int(n_min), C.byref(h)), "hm_tree_default")
        return cls(h)

    def shape(self):
        n, p, L_ = C.c_int64(), C.c_int32(), C.c_int32()
        check(lib.hm_tree_shape(self._h, C.byref(n), C.byref(p), C.byref(L_)), "hm_tree_shape")
        return n.value, p.value, L_.value

    @property
    def leaf_ends(self):
        _, _, L_ = self.shape()
        arr = (C.c_int64 * L_)()
        check(lib.hm_tree_leaf_ends(self._h, arr), "hm_tree_leaf_ends")
        return [int(v) for v in arr]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.hm_destroy(h)
            self._h = None


def _ptrs(blocks, keep):
    arr = (vp * max(len(blocks), 1))()
    for i, b in enumerate(blocks):
        if b is None:
            arr[i] = None
            continue
        a = np.asfortranarray(np.asarray(b, dtype=np.float64))
        keep.append(a)
        arr[i] = a.ctypes.data if a.size else None
    keep.append(arr)
    return C.cast(arr, C.POINTER(vp))


def _ints(vals, keep):
    arr = (C.c_int32 * max(len(vals), 1))(*[int(v) for v in vals])
    keep.append(arr)
    return C.cast(arr, C.POINTER(C.c_int32))


def _cols(b):
    return 0 if b is None else int(np.asarray(b).shape[1])


class Matrix:
    """A HODLR or HSS matrix resident on the current CUDA device."""

    def __init__(self, handle, kind, tree):
        self._h = handle
        self.kind = kind
        self.tree = tree

    @classmethod
    def hodlr(cls, tree, g, storage="f64"):
        keep = []
        gens = L.hm_hodlr_gens(
            D=_ptrs(g["D"], keep), U12=_ptrs(g["U12"], keep), V12=_ptrs(g["V12"], keep),
            U21=_ptrs(g["U21"], keep), V21=_ptrs(g["V21"], keep),
            k12=_ints([_cols(b) for b in g["U12"]], keep), k21=_ints([_cols(b) for b in g["U21"]], keep))
        h = vp()
        check(lib.hm_hodlr_create(tree._h, C.byref(gens), _dtype_code(storage), C.byref(h)), "hm_hodlr_create")
        return cls(h, "hodlr", tree)

    @classmethod
    def hss(cls, tree, g, storage="f64"):
        keep = []
        Lv = len(g["D"])
        N = 2 * Lv - 1
        ku = [0] * N
        kv = [0] * N
        for i in range(Lv):
            ku[Lv - 1 + i] = _cols(g["U"][i])
            kv[Lv - 1 + i] = _cols(g["V"][i])
        for q in range(1, Lv - 1):
            ku[q] = _cols(g["RU"][q])
            kv[q] = _cols(g["RV"][q])
        gens = L.hm_hss_gens(
            D=_ptrs(g["D"], keep), U=_ptrs(g["U"], keep), V=_ptrs(g["V"], keep),
            RU=_ptrs(g["RU"], keep), RV=_ptrs(g["RV"], keep),
            B12=_ptrs(g["B12"], keep), B21=_ptrs(g["B21"], keep),
            ku=_ints(ku, keep), kv=_ints(kv, keep))
        h = vp()
        check(lib.hm_hss_create(tree._h, C.byref(gens), _dtype_code(storage), C.byref(h)), "hm_hss_create")
        return cls(h, "hss", tree)

    @classmethod
    def create(cls, tree, g, storage="f64"):
        return cls.hodlr(tree, g, storage) if g["kind"] == "hodlr" else cls.hss(tree, g, storage)

    def info(self):
        inf = L.hm_matrix_info_t()
        check(lib.hm_matrix_info(self._h, C.byref(inf)), "hm_matrix_info")
        return {f: getattr(inf, f) for f, _ in L.hm_matrix_info_t._fields_}

    def generator_bytes(self):
        b = C.c_size_t()
        check(lib.hm_matrix_bytes(self._h, C.byref(b)), "hm_matrix_bytes")
        return b.value

    def transpose(self):
        """A^T as a new matrix on the same device (generators relabelled in
        device memory; values copied exactly)."""
        h = vp()
        check(lib.hm_matrix_transpose(self._h, C.byref(h)), "hm_matrix_transpose")
        return Matrix(h, self.kind, self.tree)

    def to_hodlr(self):
        """The HODLR form of this HSS matrix (hss2hodlr) as a new matrix."""
        h = vp()
        check(lib.hm_hss_to_hodlr(self._h, C.byref(h)), "hm_hss_to_hodlr")
        return Matrix(h, "hodlr", self.tree)

    def hadamard(self, other):
        """The entrywise product of this matrix and ``other`` (same kind, tree
        and storage) as a new matrix; ranks multiply."""
        h = vp()
        check(lib.hm_hadamard(self._h, other._h, C.byref(h)), "hm_hadamard")
        return Matrix(h, self.kind, self.tree)

    def ulv(self):
        """Implicit ULV factorization of this HSS matrix (Sec. 4.3) for solves."""
        h = vp()
        check(lib.hm_ulv_factor(self._h, C.byref(h)), "hm_ulv_factor")
        return Ulv(h, self)

    def reserve(self, r_max):
        check(lib.hm_matrix_reserve(self._h, int(r_max)), "hm_matrix_reserve")

    def set_path(self, path):
        check(lib.hm_matrix_set_path(self._h, int(path)), "hm_matrix_set_path")

    def set_tree(self, mode):
        """Tree-phase kernels: 0 automatic, 1 per-level launches, 2 one cluster launch (when it fits)."""
        check(lib.hm_matrix_set_tree(self._h, int(mode)), "hm_matrix_set_tree")

    def tune_tree(self, r, xt=None, yt=None):
        """Time the product for r columns with every tree-kernel launch shape and
        keep the fastest; returns its time per product in ms (None when the tree
        runs per level).  xt, yt: X and Y types (default F64 for F64 storage,
        else F32)."""
        info = self.info()
        f64 = info["storage"] == L.HM_F64
        xt = _dtype_code(xt) if xt is not None else (L.HM_F64 if f64 else L.HM_F32)
        yt = _dtype_code(yt) if yt is not None else (L.HM_F64 if f64 else L.HM_F32)
        ms = C.c_double()
        st = lib.hm_matrix_tune_tree(self._h, int(r), int(xt), int(yt), C.byref(ms))
        if st == L.HM_EUNSUPPORTED:
            return None
        check(st, "hm_matrix_tune_tree")
        return ms.value

    def set_tree_shape(self, r, cluster_ctas, columns, ring_slots):
        """Pin the tree kernel's launch shape for products of r columns
        (clusters of cluster_ctas CTAs, `columns` columns per cluster,
        ring_slots operator slots; 0 for HODLR)."""
        check(lib.hm_matrix_set_tree_shape(self._h, int(r), int(cluster_ctas), int(columns), int(ring_slots)),
              "hm_matrix_set_tree_shape")

    def profile(self, enable=True):
        """Bracket every kernel launch of later products with CUDA events."""
        check(lib.hm_matrix_profile(self._h, 1 if enable else 0), "hm_matrix_profile")

    def phase_times(self):
        """(ms[5], launches[5]) per phase since the last read: projection, tree up,
        HSS down, expansion, and the diagonal-block product when it is a launch
        of its own (FP64 with wide X)."""
        ms = (C.c_double * 5)()
        n = (C.c_int64 * 5)()
        check(lib.hm_matrix_phase_times(self._h, ms, n), "hm_matrix_phase_times")
        return list(ms), list(n)

    def matmat_raw(self, r, X, ldx, xt, Y, ldy, yt, stream=None):
        """Direct C call with raw pointers (ints) and dtype codes."""
        f = lib.hm_hodlr_matmat if self.kind == "hodlr" else lib.hm_hss_matmat
        return check(f(self._h, int(r), vp(X), int(ldx), int(xt), vp(Y), int(ldy), int(yt),
                       vp(stream) if stream else None), "hm_%s_matmat" % self.kind)

    def matmat(self, X, Y=None, out_dtype=None, stream=None):
        """Y = A X for an (n, r) column-major tensor/array X; returns Y."""
        n = self.tree.shape()[0]
        if torch is not None and isinstance(X, torch.Tensor):
            X2 = X if X.dim() == 2 else X.reshape(-1, 1)
            if X2.shape[0] != n:
                raise ValueError("X must have n rows")
            r = X2.shape[1]
            if r > 1 and X2.stride(0) != 1:
                raise ValueError("X must be column-major (stride(0) == 1); use colmajor()")
            ldx = X2.stride(1) if r > 1 else max(n, 1)
            if Y is None:
                od = out_dtype or (torch.float64 if X2.dtype == torch.float64 else torch.float32)
                Y = torch.empty((r, n), dtype=od, device=X2.device).t()
            Y2 = Y if Y.dim() == 2 else Y.reshape(-1, 1)
            if r > 1 and Y2.stride(0) != 1:
                raise ValueError("Y must be column-major")
            ldy = Y2.stride(1) if r > 1 else max(n, 1)
            if stream is None and X2.is_cuda:
                stream = torch.cuda.current_stream(X2.device).cuda_stream
            self.matmat_raw(r, X2.data_ptr(), ldx, _dtype_code(X2.dtype), Y2.data_ptr(), ldy,
                            _dtype_code(Y2.dtype), stream)
            return Y
        Xn = np.asarray(X)
        if Xn.ndim == 1:
            Xn = Xn[:, None]
        Xn = np.asfortranarray(Xn)
        r = Xn.shape[1]
        if Y is None:
            od = out_dtype or (np.float64 if Xn.dtype == np.float64 else np.float32)
            Y = np.zeros((n, r), dtype=od, order="F")
        self.matmat_raw(r, Xn.ctypes.data, max(n, 1), _dtype_code(Xn.dtype.type), Y.ctypes.data, max(n, 1),
                        _dtype_code(Y.dtype.type), stream)
        return Y

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.hm_destroy(h)
            self._h = None


class Batch:
    """Many products Y_j = A_j X_j run as one persistent launch per phase."""

    def __init__(self, mats, rs):
        self.mats = list(mats)
        self.rs = [int(v) for v in rs]
        hs = (vp * len(self.mats))(*[m._h for m in self.mats])
        rr = (C.c_int64 * len(self.rs))(*self.rs)
        h = vp()
        check(lib.hm_batch_create(hs, rr, len(self.mats), C.byref(h)), "hm_batch_create")
        self._h = h

    def tune(self, cache_path=None):
        check(lib.hm_batch_tune(self._h, cache_path.encode() if cache_path else None), "hm_batch_tune")

    def run(self, Xs, Ys, xt=L.HM_F32, yt=L.HM_F32, stream=None):
        """Xs, Ys: sequences of device pointers (ints) or column-major tensors."""
        xp = [x.data_ptr() if hasattr(x, "data_ptr") else int(x) for x in Xs]
        yp = [y.data_ptr() if hasattr(y, "data_ptr") else int(y) for y in Ys]
        xa = (vp * len(xp))(*xp)
        ya = (vp * len(yp))(*yp)
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        check(lib.hm_batch_run(self._h, xa, ya, _dtype_code(xt), _dtype_code(yt), vp(stream) if stream else None),
              "hm_batch_run")

    def info(self):
        inf = L.hm_batch_info_t()
        check(lib.hm_batch_info(self._h, C.byref(inf)), "hm_batch_info")
        out = {f: getattr(inf, f) for f, _ in L.hm_batch_info_t._fields_}
        out["items"] = list(out["items"])
        out["grid"] = list(out["grid"])
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.hm_destroy(h)
            self._h = None


class Ulv:
    """A factorization for solves X = A^{-1} B (keeps its matrix alive)."""

    def __init__(self, handle, matrix):
        self._h = handle
        self.matrix = matrix

    def solve(self, B, X=None, stream=None):
        """X = A^{-1} B for an (n, r) float64 column-major device tensor B."""
        n = self.matrix.tree.shape()[0]
        if B.dim() == 1:
            B = B.reshape(-1, 1)
        r = B.shape[1]
        if X is None:
            X = torch.empty((r, n), dtype=torch.float64, device=B.device).t()
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        check(lib.hm_ulv_solve(self._h, int(r), vp(B.data_ptr()), int(B.stride(1)) if r > 1 else n,
                               vp(X.data_ptr()), int(X.stride(1)) if r > 1 else n, vp(st)), "hm_ulv_solve")
        return X

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib.hm_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


class Server:
    """Resident matrices and continuously batched product requests."""

    def __init__(self, mem_budget, max_slots):
        h = vp()
        check(lib.hm_serve_create(int(mem_budget), int(max_slots), C.byref(h)), "hm_serve_create")
        self._h = h
        self.mats = []

    def register(self, A):
        i = C.c_int32()
        check(lib.hm_serve_register(self._h, A._h, C.byref(i)), "hm_serve_register")
        self.mats.append(A)
        return i.value

    def submit(self, mid, r, X, Y):
        """Returns a ticket, or None when the server refuses (HM_EBUSY)."""
        t = C.c_uint64()
        st = lib.hm_serve_submit(self._h, int(mid), int(r), vp(X), vp(Y), C.byref(t))
        if st == L.HM_EBUSY:
            return None
        check(st, "hm_serve_submit")
        return t.value

    def wait(self, ticket, timeout_ms=10000):
        return check(lib.hm_serve_wait(self._h, int(ticket), int(timeout_ms)), "hm_serve_wait")

    def poll(self, ticket):
        st = lib.hm_serve_poll(self._h, int(ticket))
        if st == L.HM_EBUSY:
            return False
        check(st, "hm_serve_poll")
        return True

    def cancel(self, ticket):
        """True if the queued request was withdrawn, False if it already runs or ran."""
        st = lib.hm_serve_cancel(self._h, int(ticket))
        if st == L.HM_EBUSY:
            return False
        check(st, "hm_serve_cancel")
        return True

    def pause(self, paused=True):
        """Stop (True) or resume (False) the worker's intake of queued requests."""
        check(lib.hm_serve_pause(self._h, 1 if paused else 0), "hm_serve_pause")

    def stats(self):
        sst = L.hm_serve_stats_t()
        check(lib.hm_serve_stats(self._h, C.byref(sst)), "hm_serve_stats")
        return {f: getattr(sst, f) for f, _ in L.hm_serve_stats_t._fields_}

    def reset_stats(self):
        check(lib.hm_serve_reset_stats(self._h), "hm_serve_reset_stats")

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib.hm_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


def colmajor(t):
    """Column-major copy of a 2-D torch tensor (layout helper for callers)."""
    return t.t().contiguous().t()


def device_status(stream=None):
    check(lib.hm_device_status(vp(stream) if stream else None), "hm_device_status")


def set_device_wait_limit(ns):
    """Device-side bounded waits give up after `ns` nanoseconds (default 2e9)."""
    check(lib.hm_set_device_wait_limit(int(ns)), "hm_set_device_wait_limit")


def device_wait_limit():
    v = C.c_uint64()
    check(lib.hm_get_device_wait_limit(C.byref(v)), "hm_get_device_wait_limit")
    return v.value


def selftest_device_timeout(stream=None):
    """Queues the kernel whose bounded waits always run out (see hm.h)."""
    check(lib.hm_selftest_device_timeout(vp(stream) if stream else None), "hm_selftest_device_timeout")


def inject_alloc_failures(count):
    """The next `count` device allocations of the library fail (HM_ENOMEM)."""
    check(lib.hm_inject_alloc_failures(int(count)), "hm_inject_alloc_failures")
