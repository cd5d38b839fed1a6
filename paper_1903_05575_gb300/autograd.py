"""torch.autograd binding of a quaternion linear map Y = X W.

Shapes (column-major quaternion matrices, see ops.py):
  interleaved: X (k, mb, 4), W (n, k, 4), Y (n, mb, 4)
  planes:      X (4, k, mb), W (4, n, k), Y (4, n, mb)
The loss is real; gradients are componentwise, dL/dX^s_{ij}.  With the real
inner product <P, Q> = Re tr(P^H Q) (the sum of component products) and
Re tr(PQ) = Re tr(QP) over H, dX = dY W^H and dW = X^H dY (conjugate
transpose of Sec. 2.2), computed by the C ABI's qgemm_backward with the
conjugate transpose folded into the tile loads.  float64 tensors use the FP64
path (or the digit-sliced FP64 path with precision="fp64_sliced"), float32
the split-BF16 path.
"""
import torch

from . import ops

ONE = (1.0, 0.0, 0.0, 0.0)
ZERO = (0.0, 0.0, 0.0, 0.0)


def _dims(X, W, layout):
    if layout == "interleaved":
        k, mb = X.shape[0], X.shape[1]
        n = W.shape[0]
        if W.shape[1] != k:
            raise ValueError("X is mb x k and W is k x n")
    else:
        k, mb = X.shape[1], X.shape[2]
        n = W.shape[1]
        if W.shape[2] != k:
            raise ValueError("X is mb x k and W is k x n")
    return mb, k, n


class QLinearFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, W, layout="interleaved", precision=None):
        X, W = X.contiguous(), W.contiguous()
        mb, k, n = _dims(X, W, layout)
        shape = (n, mb, 4) if layout == "interleaved" else (4, n, mb)
        Y = torch.empty(shape, dtype=X.dtype, device=X.device)
        ops.qgemm("N", "N", mb, n, k, ONE, X, W, ZERO, Y, layout=layout, precision=precision)
        ctx.save_for_backward(X, W)
        ctx.layout = layout
        ctx.precision = precision
        return Y

    @staticmethod
    def backward(ctx, dY):
        X, W = ctx.saved_tensors
        layout = ctx.layout
        mb, k, n = _dims(X, W, layout)
        dX = torch.empty_like(X) if ctx.needs_input_grad[0] else None
        dW = torch.empty_like(W) if ctx.needs_input_grad[1] else None
        if dX is not None or dW is not None:
            ops.qgemm_backward(X, W, dY.contiguous(), mb, k, n, dX=dX, dW=dW, layout=layout,
                               precision=ctx.precision)
        return dX, dW, None, None


def qlinear(X, W, layout="interleaved", precision=None):
    return QLinearFunction.apply(X, W, layout, precision)


class QLinear(torch.nn.Module):
    """Quaternion linear layer: Y = X W with W a k x n quaternion matrix."""

    def __init__(self, in_features, out_features, dtype=torch.float32, device="cuda",
                 layout="interleaved", std=None, precision=None):
        super().__init__()
        self.layout = layout
        self.precision = precision
        shape = ((out_features, in_features, 4) if layout == "interleaved"
                 else (4, out_features, in_features))
        std = (1.0 / (4.0 * in_features)) ** 0.5 if std is None else std
        self.weight = torch.nn.Parameter(torch.randn(shape, dtype=dtype, device=device) * std)

    def forward(self, X):
        return qlinear(X, self.weight, self.layout, self.precision)
