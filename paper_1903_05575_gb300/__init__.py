"""GB300 (sm_103a) quaternion GEMM: C = alpha op(A) op(B) + beta C over H.

The compute path is the CUDA library built from csrc/ behind the C ABI of
include/qgemm.h; this package only marshals arguments to it.
"""
from . import _abi  # noqa: F401
from .autograd import QLinear, QLinearFunction, qlinear  # noqa: F401
from .ops import (GroupedBatch, geometry, last_device_error, probe_peak, qgemm,  # noqa: F401
                  qgemm_backward, qgemm_mixed, qherk, qtrmm, set_tile_table, tile_info,
                  workspace)

__all__ = ["GroupedBatch", "set_tile_table", "tile_info", "QLinear", "QLinearFunction", "qlinear", "qgemm", "qgemm_mixed", "qherk", "qtrmm", "qgemm_backward", "geometry", "workspace", "last_device_error",
           "probe_peak"]
