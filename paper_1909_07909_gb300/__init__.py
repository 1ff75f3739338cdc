"""GB300-native HODLR/HSS matrix-times-block products (sm_103a CUDA kernels).

Python binding of libhm (include/hm.h).  The library must be built first
(``paper_1909_07909_gb300.build.build()``); importing without it raises.
"""

from ._lib import (HM_BF16, HM_BF16X2, HM_F32, HM_F64, HM_HODLR, HM_HSS, HMError,  # noqa: F401
                   LIB_PATH, lib)
from .api import (Batch, Matrix, Server, Tree, Ulv, colmajor, device_status, device_wait_limit,  # noqa: F401
                  inject_alloc_failures, selftest_device_timeout, set_device_wait_limit)

__all__ = ["Tree", "Matrix", "Batch", "Server", "Ulv", "colmajor", "device_status", "set_device_wait_limit",
           "device_wait_limit", "selftest_device_timeout", "inject_alloc_failures", "HMError", "lib", "LIB_PATH",
           "HM_F64", "HM_F32", "HM_BF16", "HM_BF16X2", "HM_HODLR", "HM_HSS"]
