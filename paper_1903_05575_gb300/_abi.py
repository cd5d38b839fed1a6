"""ctypes declarations of the C ABI in include/qgemm.h.

Loads paper_1903_05575_gb300/lib/libqgemm.so (building it first when it is
missing or stale).  The library has no CPU fallback; if it cannot be loaded
the import fails loudly.
"""
import ctypes
import os

from . import build as _build

OP = {"N": 0, "T": 1, "C": 2, "H": 3}
LAYOUT = {"interleaved": 0, "planes": 1}
PRECISION = {"fp64": 0, "split_bf16": 1, "fp64_sliced": 2}

SUCCESS = 0
ERR_UNSUPPORTED = 1
ERR_CUDA = 2
ERR_TIMEOUT = 3
ERR_NO_DEVICE = 4
ERR_WORKSPACE = 5
NOALLOC_SCRATCH_BYTES = 64 << 20

i32, i64, sz, vp, dp = (ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p,
                        ctypes.POINTER(ctypes.c_double))


class QgemmProblem(ctypes.Structure):
    """Mirror of struct qgemm_problem."""
    _fields_ = [("opA", ctypes.c_int32), ("opB", ctypes.c_int32),
                ("m", i64), ("n", i64), ("k", i64),
                ("alpha", ctypes.c_double * 4), ("beta", ctypes.c_double * 4),
                ("A", vp), ("lda", i64), ("psA", i64),
                ("B", vp), ("ldb", i64), ("psB", i64),
                ("C", vp), ("ldc", i64), ("psC", i64)]


class QgemmGroupedPlan(ctypes.Structure):
    """Mirror of struct qgemm_grouped_plan."""
    _fields_ = [("workspace", vp), ("workspace_bytes", sz), ("layout", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("count", i64), ("tiles", i64),
                ("grid", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("desc_offset", i64), ("tile_offset", i64), ("data_offset", i64),
                ("reserved", i64 * 4)]


# name -> (restype, argtypes)
SIGNATURES = {
    "qgemm": (i32, [i32, i32, i64, i64, i64, dp, vp, i64, i64, vp, i64, i64, dp, vp, i64, i64,
                    i32, i32, vp, sz, vp]),
    "qgemm_workspace_bytes": (sz, [i32, i32, i64, i64, i64, i32, i32]),
    "qgemm_split_noalloc": (i32, [i32, i32, i64, i64, i64, dp, vp, i64, i64, vp, i64, i64, dp,
                                  vp, i64, i64, i32, vp]),
    "qgemm_batched_grouped": (i32, [ctypes.POINTER(QgemmProblem), i64, i32, i32, vp, sz, vp]),
    "qgemm_grouped_workspace_bytes": (sz, [ctypes.POINTER(QgemmProblem), i64, i32, i32]),
    "qgemm_grouped_prepare": (i32, [ctypes.POINTER(QgemmProblem), i64, i32, i32, vp, sz, vp,
                                    ctypes.POINTER(QgemmGroupedPlan)]),
    "qgemm_grouped_launch": (i32, [ctypes.POINTER(QgemmGroupedPlan), vp]),
    "qgemm_grouped_set_tile_table": (i32, [i32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "qgemm_grouped_tile_info": (i32, [ctypes.POINTER(ctypes.c_int32)] * 5),
    "qherk": (i32, [i32, i32, i64, i64, ctypes.c_double, vp, i64, i64, ctypes.c_double, vp, i64,
                    i64, i32, i32, vp, sz, vp]),
    "qherk_workspace_bytes": (sz, [i32, i32, i64, i64, i32, i32]),
    "qtrmm": (i32, [i32, i32, i32, i32, i64, i64, dp, vp, i64, i64, vp, i64, i64, vp, i64, i64,
                    i32, i32, vp, sz, vp]),
    "qtrmm_workspace_bytes": (sz, [i32, i32, i32, i32, i64, i64, i32, i32]),
    "qgemm_mixed": (i32, [i32, i32, i32, i32, i64, i64, i64, dp, vp, i64, i64, vp, i64, i64, dp,
                          vp, i64, i64, i32, i32, vp, sz, vp]),
    "qgemm_mixed_workspace_bytes": (sz, [i32, i32, i32, i32, i64, i64, i64, i32, i32]),
    "qgemm_backward": (i32, [i64, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64,
                             vp, i64, i64, vp, i64, i64, i32, i32, i32, vp, sz, vp]),
    "qgemm_backward_workspace_bytes": (sz, [i64, i64, i64, i32, i32]),
    "qgemm_get_last_device_error": (i32, []),
    "qgemm_status_string": (ctypes.c_char_p, [i32]),
    "qgemm_last_cuda_error": (ctypes.c_char_p, []),
    "qgemm_debug_unsatisfied_wait": (i32, [ctypes.c_uint64, vp]),
    "qgemm_debug_arm_fault": (i32, [i32, i32, ctypes.c_uint64]),
    "qgemm_probe_peak": (i32, [i32, ctypes.c_double, dp, vp]),
    "qgemm_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library with every entry point declared."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def lib_path():
    return _build.LIB


def q4(x):
    """Host double[4] for alpha / beta."""
    vals = [float(v) for v in x]
    if len(vals) != 4:
        raise ValueError("a quaternion scalar has 4 components")
    return (ctypes.c_double * 4)(*vals)


def status_string(rc):
    return lib().qgemm_status_string(rc).decode()


class QgemmError(RuntimeError):
    def __init__(self, rc, what=""):
        self.rc = rc
        detail = status_string(rc)
        if rc == ERR_CUDA:
            detail += ": " + lib().qgemm_last_cuda_error().decode()
        super().__init__("%s failed: %d (%s)" % (what or "qgemm", rc, detail))


def check(rc, what=""):
    if rc != 0:
        raise QgemmError(rc, what)
    return rc
