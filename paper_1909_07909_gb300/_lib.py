"""ctypes declarations of the C ABI in include/hm.h (argument marshalling only).

Loading fails loudly: if libhm.so has not been built, importing this module
raises ImportError; there is no fallback implementation.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libhm.so is not built (run paper_1909_07909_gb300.build.build() "
                      "or __graft_entry__.build()); there is no fallback implementation")

lib = C.CDLL(LIB_PATH)

HM_OK, HM_EINVAL, HM_ENOMEM, HM_EBUSY, HM_ETIMEOUT, HM_ECUDA, HM_EUNSUPPORTED = range(7)
HM_F64, HM_F32, HM_BF16, HM_BF16X2 = range(4)
HM_HODLR, HM_HSS = 0, 1

DTYPES = {"f64": HM_F64, "f32": HM_F32, "bf16": HM_BF16, "bf16x2": HM_BF16X2}
STATUS_NAMES = {0: "HM_OK", 1: "HM_EINVAL", 2: "HM_ENOMEM", 3: "HM_EBUSY", 4: "HM_ETIMEOUT",
                5: "HM_ECUDA", 6: "HM_EUNSUPPORTED"}

c_int64_p = C.POINTER(C.c_int64)
c_int32_p = C.POINTER(C.c_int32)
c_dbl_pp = C.POINTER(C.c_void_p)


class hm_hodlr_gens(C.Structure):
    _fields_ = [("D", c_dbl_pp), ("U12", c_dbl_pp), ("V12", c_dbl_pp), ("U21", c_dbl_pp),
                ("V21", c_dbl_pp), ("k12", c_int32_p), ("k21", c_int32_p)]


class hm_hss_gens(C.Structure):
    _fields_ = [("D", c_dbl_pp), ("U", c_dbl_pp), ("V", c_dbl_pp), ("RU", c_dbl_pp), ("RV", c_dbl_pp),
                ("B12", c_dbl_pp), ("B21", c_dbl_pp), ("ku", c_int32_p), ("kv", c_int32_p)]


class hm_matrix_info_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("storage", C.c_int32), ("n", C.c_int64), ("depth", C.c_int32),
                ("num_leaves", C.c_int32), ("leaf_pad", C.c_int32), ("rank_total", C.c_int32),
                ("generator_elements", C.c_int64), ("generator_bytes", C.c_size_t),
                ("device_bytes", C.c_size_t), ("tree_cluster", C.c_int32), ("tree_columns", C.c_int32),
                ("tree_ring", C.c_int32), ("rank_col", C.c_int32)]


class hm_batch_info_t(C.Structure):
    _fields_ = [("count", C.c_int32), ("launches_per_run", C.c_int32), ("items", C.c_int64 * 6),
                ("grid", C.c_int32 * 6), ("graph", C.c_int32), ("tuned", C.c_int32), ("grid_mult", C.c_int32),
                ("rc_cap", C.c_int32), ("rct_cap", C.c_int32), ("tile_rows", C.c_int32),
                ("capture_error", C.c_int32)]


class hm_serve_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("rejected", C.c_int64),
                ("completed", C.c_int64), ("launches", C.c_int64), ("pending", C.c_int32),
                ("max_merged", C.c_int32), ("resident_bytes", C.c_size_t), ("p50_us", C.c_double),
                ("p99_us", C.c_double), ("mean_us", C.c_double), ("throughput_rps", C.c_double),
                ("gbs", C.c_double)]


def _decl(name, res, *args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


vp = C.c_void_p
_decl("hm_status_string", C.c_char_p, C.c_int)
_decl("hm_last_error", C.c_char_p)
_decl("hm_version", C.c_char_p)
_decl("hm_tree_create", C.c_int, C.c_int64, c_int64_p, C.c_int32, C.POINTER(vp))
_decl("hm_tree_default", C.c_int, C.c_int64, C.c_int64, C.POINTER(vp))
_decl("hm_tree_shape", C.c_int, vp, c_int64_p, c_int32_p, c_int32_p)
_decl("hm_tree_leaf_ends", C.c_int, vp, c_int64_p)
_decl("hm_hodlr_create", C.c_int, vp, C.POINTER(hm_hodlr_gens), C.c_int, C.POINTER(vp))
_decl("hm_hss_create", C.c_int, vp, C.POINTER(hm_hss_gens), C.c_int, C.POINTER(vp))
_decl("hm_matrix_info", C.c_int, vp, C.POINTER(hm_matrix_info_t))
_decl("hm_matrix_bytes", C.c_int, vp, C.POINTER(C.c_size_t))
_decl("hm_matrix_transpose", C.c_int, vp, C.POINTER(vp))
_decl("hm_hss_to_hodlr", C.c_int, vp, C.POINTER(vp))
_decl("hm_hadamard", C.c_int, vp, vp, C.POINTER(vp))
_decl("hm_matrix_reserve", C.c_int, vp, C.c_int64)
_decl("hm_matrix_set_path", C.c_int, vp, C.c_int32)
_decl("hm_matrix_set_tree", C.c_int, vp, C.c_int32)
_decl("hm_matrix_tune_tree", C.c_int, vp, C.c_int64, C.c_int, C.c_int, C.POINTER(C.c_double))
_decl("hm_matrix_set_tree_shape", C.c_int, vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32)
_decl("hm_hodlr_matmat", C.c_int, vp, C.c_int64, vp, C.c_int64, C.c_int, vp, C.c_int64, C.c_int, vp)
_decl("hm_hss_matmat", C.c_int, vp, C.c_int64, vp, C.c_int64, C.c_int, vp, C.c_int64, C.c_int, vp)
_decl("hm_device_status", C.c_int, vp)
_decl("hm_matmat_noalloc", C.c_int, vp, C.c_int64, vp, C.c_int64, C.c_int, vp, C.c_int64, C.c_int, vp)
_decl("hm_matrix_profile", C.c_int, vp, C.c_int32)
_decl("hm_matrix_phase_times", C.c_int, vp, C.POINTER(C.c_double), C.POINTER(C.c_int64))
_decl("hm_batch_create", C.c_int, C.POINTER(vp), C.POINTER(C.c_int64), C.c_int32, C.POINTER(vp))
_decl("hm_batch_tune", C.c_int, vp, C.c_char_p)
_decl("hm_batch_run", C.c_int, vp, C.POINTER(vp), C.POINTER(vp), C.c_int, C.c_int, vp)
_decl("hm_batch_info", C.c_int, vp, C.POINTER(hm_batch_info_t))
_decl("hm_serve_create", C.c_int, C.c_size_t, C.c_int32, C.POINTER(vp))
_decl("hm_serve_register", C.c_int, vp, vp, C.POINTER(C.c_int32))
_decl("hm_serve_submit", C.c_int, vp, C.c_int32, C.c_int64, vp, vp, C.POINTER(C.c_uint64))
_decl("hm_serve_wait", C.c_int, vp, C.c_uint64, C.c_int32)
_decl("hm_serve_poll", C.c_int, vp, C.c_uint64)
_decl("hm_serve_stats", C.c_int, vp, C.POINTER(hm_serve_stats_t))
_decl("hm_serve_reset_stats", C.c_int, vp)
_decl("hm_serve_cancel", C.c_int, vp, C.c_uint64)
_decl("hm_serve_pause", C.c_int, vp, C.c_int32)
_decl("hm_set_device_wait_limit", C.c_int, C.c_uint64)
_decl("hm_get_device_wait_limit", C.c_int, C.POINTER(C.c_uint64))
_decl("hm_selftest_device_timeout", C.c_int, vp)
_decl("hm_inject_alloc_failures", C.c_int, C.c_int32)
_decl("hm_ulv_factor", C.c_int, vp, C.POINTER(vp))
_decl("hm_ulv_solve", C.c_int, vp, C.c_int64, vp, C.c_int64, vp, C.c_int64, vp)
_decl("hm_destroy", None, vp)


class HMError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = lib.hm_last_error().decode(errors="replace")
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(status, status), detail))


def check(status, where):
    if status != HM_OK:
        raise HMError(status, where)
    return status
