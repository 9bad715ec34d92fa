"""ctypes binding of include/spider.h -- argument marshalling only.

Every function of the C ABI is exposed under its own name.  Loading fails
loudly (``ImportError``) when the in-tree library has not been built: there
is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_int64, c_size_t, c_void_p, c_double, c_uint32, c_uint64 = (
    ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_double, ctypes.c_uint32,
    ctypes.c_uint64)

# spider_status
SPIDER_OK, SPIDER_ERR_INVALID, SPIDER_ERR_UNSUPPORTED, SPIDER_ERR_OOM, SPIDER_ERR_CUDA, SPIDER_ERR_TIMEOUT, \
    SPIDER_ERR_BUSY = range(7)
STATUS_NAMES = {0: "SPIDER_OK", 1: "SPIDER_ERR_INVALID", 2: "SPIDER_ERR_UNSUPPORTED", 3: "SPIDER_ERR_OOM",
                4: "SPIDER_ERR_CUDA", 5: "SPIDER_ERR_TIMEOUT", 6: "SPIDER_ERR_BUSY"}
# spider_shape
SPIDER_STAR, SPIDER_BOX = 0, 1
# spider_precision
SPIDER_TF32, SPIDER_F16X2, SPIDER_BF16X3, SPIDER_AUTO = 0, 1, 2, 3
# spider_engine
SPIDER_ENGINE_SPARSE_TC, SPIDER_ENGINE_DENSE_TC, SPIDER_ENGINE_CUDA_CORE, SPIDER_ENGINE_SPARSE_TC_COPY = 0, 1, 2, 3
SPIDER_ENGINE_SPARSE_TC_NO_CO = 4

# name -> (restype, argtypes); the complete list of entry points of spider.h
SIGNATURES = {
    "spider_plan_create": (c_int, [c_int, ctypes.POINTER(c_int64), c_int, c_int, ctypes.POINTER(ctypes.c_float),
                                   c_int, ctypes.POINTER(c_void_p)]),
    "spider_plan_set_engine": (c_int, [c_void_p, c_int]),
    "spider_plan_set_steps_per_pass": (c_int, [c_void_p, c_int]),
    "spider_plan_set_tile_variant": (c_int, [c_void_p, c_int]),
    "spider_plan_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, ctypes.POINTER(c_int),
                                     ctypes.POINTER(c_int)]),
    "spider_plan_autotune_arithmetic": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.c_double, c_void_p,
                                                ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                                ctypes.POINTER(ctypes.c_double)]),
    "spider_plan_operands": (c_int, [c_void_p, ctypes.POINTER(c_uint32), c_size_t, ctypes.POINTER(c_size_t),
                                     ctypes.POINTER(c_uint32), c_size_t, ctypes.POINTER(c_size_t)]),
    "spider_run": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "spider_run_host": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "spider_run_host_async": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "spider_run_static": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "spider_plan_sync": (c_int, [c_void_p, c_void_p]),
    "spider_plan_device_bytes": (c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "spider_plan_error_bound": (c_int, [c_void_p, c_int, c_int, c_int64, ctypes.POINTER(c_double)]),
    "spider_plan_destroy": (None, [c_void_p]),
    "spider_set_wait_limit": (c_int, [ctypes.c_longlong]),
    "spider_batch_drop_item": (c_int, [ctypes.c_longlong]),
    "spider_batch_configure": (c_int, [ctypes.c_longlong, c_int]),
    "spider_batch": (c_int, [c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                             ctypes.POINTER(c_int64), c_void_p]),
    "spider_domain_create": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(c_void_p)]),
    "spider_domain_slab": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                   ctypes.POINTER(c_int64), ctypes.POINTER(c_int64)]),
    "spider_domain_run": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "spider_domain_sync": (c_int, [c_void_p, c_void_p]),
    "spider_domain_destroy": (None, [c_void_p]),
    "spider_norms_fp64": (c_int, [c_void_p, c_void_p, c_int64, ctypes.POINTER(c_double), c_void_p]),
    "spider_constant_check_fp64": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64), c_int64, c_double,
                                           ctypes.POINTER(c_double), c_void_p]),
    "spider_measure_mma_rate": (c_int, [c_int, ctypes.POINTER(c_double), c_void_p]),
    "spider_server_create": (c_int, [c_size_t, ctypes.POINTER(c_void_p)]),
    "spider_submit": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_double, ctypes.POINTER(c_uint64)]),
    "spider_poll": (c_int, [c_void_p, c_uint64, c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    "spider_server_job_arithmetic": (c_int, [c_void_p, c_uint64, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                             ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    "spider_server_wait": (c_int, [c_void_p, c_double, ctypes.POINTER(c_uint64), ctypes.POINTER(c_int)]),
    "spider_server_destroy": (None, [c_void_p]),
    "spider_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Loads the in-tree libspider.so (raises ImportError if it is missing)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libspider.so is not built ({path}); run paper_2506_22035_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class SpiderError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, fn: str) -> None:
    if status != SPIDER_OK:
        raise SpiderError(status, fn, load().spider_last_error().decode(errors="replace"))


def __getattr__(name):
    # spider_* functions resolve to the loaded library's symbols
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
