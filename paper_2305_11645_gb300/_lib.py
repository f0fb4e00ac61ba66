"""ctypes declarations of the C ABI in include/qmc.h (libqmc_gb300.so)."""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import POINTER, c_double, c_int, c_size_t, c_uint32, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libqmc_gb300.so")

QMC_OK, QMC_ERR_INVALID_ARG, QMC_ERR_UNSUPPORTED, QMC_ERR_NO_MEMORY, QMC_ERR_CUDA, QMC_ERR_DEVICE, QMC_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "QMC_OK", 1: "QMC_ERR_INVALID_ARG", 2: "QMC_ERR_UNSUPPORTED", 3: "QMC_ERR_NO_MEMORY",
                4: "QMC_ERR_CUDA", 5: "QMC_ERR_DEVICE", 6: "QMC_ERR_TIMEOUT"}
QMC_FP64, QMC_FP32, QMC_SPLIT, QMC_BF16 = range(4)
QMC_LAYOUT_FULL, QMC_LAYOUT_DISTINCT = 0, 1
QMC_OP_GEN_POINTS, QMC_OP_REDUCED_MATMUL, QMC_OP_INTEGRATE, QMC_OP_INTEGRATE_BWD = range(4)
QMC_BWD_REUSE_FORWARD = 1

EXPORTS = ["qmc_version", "qmc_last_error", "qmc_validate_rule", "qmc_workspace_size", "qmc_gen_points",
           "qmc_reduced_matmul", "qmc_integrate", "qmc_integrate_backward", "qmc_integrate_noalloc",
           "qmc_trace_enable", "qmc_trace_collect", "qmc_trace_entry", "qmc_device_status",
           "qmc_selftest_wait_timeout", "qmc_autotune", "qmc_tune_set", "qmc_tune_save", "qmc_tune_load",
           "qmc_tune_clear"]
PRECISIONS = {"fp64": QMC_FP64, "fp32": QMC_FP32, "split": QMC_SPLIT, "bf16": QMC_BF16}


class QmcRule(ctypes.Structure):
    _fields_ = [("kind", c_int), ("b", c_uint32), ("m", c_uint32), ("s", c_uint32),
                ("w", POINTER(c_uint32)), ("z", POINTER(c_uint32)), ("C", POINTER(c_uint32)),
                ("R", c_uint32), ("shift", POINTER(c_uint32)), ("transform", c_int),
                ("d_gen", c_void_p), ("d_shift", c_void_p)]


class QmcIntegrand(ctypes.Structure):
    _fields_ = [("kind", c_int), ("params", c_double * 4)]


class QmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library; raises if it has not been built (there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libqmc_gb300.so not found at {path}: build it with "
                               "`python -m paper_2305_11645_gb300.build` (the CUDA path has no CPU fallback)")
        lib = ctypes.CDLL(path)
        lib.qmc_version.restype = ctypes.c_char_p
        lib.qmc_last_error.restype = ctypes.c_char_p
        lib.qmc_validate_rule.argtypes = [POINTER(QmcRule)]
        lib.qmc_workspace_size.argtypes = [c_int, POINTER(QmcRule), POINTER(c_uint32), c_uint32,
                                           POINTER(QmcIntegrand), c_int, POINTER(c_size_t)]
        lib.qmc_gen_points.argtypes = [POINTER(QmcRule), c_uint32, c_int, c_void_p, c_size_t, c_void_p, c_size_t,
                                       c_void_p]
        lib.qmc_reduced_matmul.argtypes = [POINTER(QmcRule), c_void_p, c_uint32, c_int, c_void_p, c_void_p, c_size_t,
                                           c_void_p]
        lib.qmc_integrate.argtypes = [POINTER(QmcRule), POINTER(c_void_p), POINTER(c_uint32), c_uint32,
                                      POINTER(QmcIntegrand), c_int, c_void_p, POINTER(c_void_p), c_void_p, c_size_t,
                                      c_void_p]
        lib.qmc_integrate_backward.argtypes = [POINTER(QmcRule), POINTER(c_void_p), POINTER(c_uint32), c_uint32,
                                               POINTER(QmcIntegrand), c_int, c_void_p, POINTER(c_void_p), c_uint32,
                                               c_void_p, c_size_t, c_void_p]
        lib.qmc_integrate_noalloc.argtypes = [POINTER(QmcRule), c_void_p, c_uint32, POINTER(QmcIntegrand), c_int,
                                              c_void_p, c_void_p]
        lib.qmc_autotune.argtypes = [POINTER(QmcRule), c_void_p, c_uint32, POINTER(QmcIntegrand), c_int, c_void_p,
                                     c_void_p, c_void_p, c_size_t, c_void_p, POINTER(c_uint32)]
        lib.qmc_tune_set.argtypes = [POINTER(QmcRule), c_uint32, POINTER(QmcIntegrand), c_int, c_int, c_int, c_int,
                                     c_int]
        lib.qmc_tune_save.argtypes = [ctypes.c_char_p]
        lib.qmc_tune_load.argtypes = [ctypes.c_char_p, POINTER(c_uint32)]
        lib.qmc_tune_clear.argtypes = []
        lib.qmc_device_status.argtypes = [c_int]
        lib.qmc_selftest_wait_timeout.argtypes = [c_uint32, c_void_p]
        lib.qmc_trace_enable.argtypes = [c_int]
        lib.qmc_trace_collect.argtypes = [POINTER(c_uint32)]
        lib.qmc_trace_entry.argtypes = [c_uint32, POINTER(ctypes.c_char_p), POINTER(ctypes.c_uint64),
                                        POINTER(c_double)]
        for name in EXPORTS[2:]:
            getattr(lib, name).restype = c_int
        _lib = lib
        return lib


def check(status: int) -> None:
    if status != QMC_OK:
        raise QmcError(status, load().qmc_last_error().decode())


def device_status(clear: bool = True) -> None:
    """Synchronise the device and raise QmcError(QMC_ERR_TIMEOUT) if a tensor-core kernel gave up
    a bounded wait since the last check (the error word is cleared when `clear`)."""
    check(load().qmc_device_status(1 if clear else 0))


def trace_enable(on: bool) -> None:
    check(load().qmc_trace_enable(1 if on else 0))


def trace_collect() -> dict:
    """{kernel name: (launches, total device ms)} of the launches recorded since trace_enable(True)."""
    lib = load()
    n = c_uint32(0)
    check(lib.qmc_trace_collect(ctypes.byref(n)))
    out = {}
    for i in range(n.value):
        name, cnt, ms = ctypes.c_char_p(), ctypes.c_uint64(0), c_double(0)
        check(lib.qmc_trace_entry(i, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)))
        out[name.value.decode()] = (int(cnt.value), float(ms.value))
    return out
