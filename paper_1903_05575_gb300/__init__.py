"""GB300 (sm_103a) quaternion GEMM: C = alpha op(A) op(B) + beta C over H.

The compute path is the CUDA library built from csrc/ behind the C ABI of
include/qgemm.h; this package only marshals arguments to it.
"""
from . import _abi  # noqa: F401
from .autograd import QLinear, QLinearFunction, qlinear  # noqa: F401
from .ops import (geometry, last_device_error, probe_peak, qgemm,  # noqa: F401
                  qgemm_backward, workspace)

__all__ = ["QLinear", "QLinearFunction", "qlinear", "qgemm", "qgemm_backward", "geometry", "workspace", "last_device_error",
           "probe_peak"]
