"""Quaternion linear layer Y = X W: gradients of the C-ABI backward
(dX = dY W^H, dW = X^H dY) through torch.autograd.

Expected values never come from the CUDA path: finite differences use the
FP64 oracle's forward, and the second reference is torch float64 CPU autograd
of the real 4x4-block form built from the Hamilton table in tests/golden."""
import os

import numpy as np
import pytest
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import QLinearFunction, ops
from tests.gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hamilton_table.txt")


def _sign_table():
    s = np.zeros((4, 4))
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            i, j, sg, k = (int(float(x)) for x in line.split())
            s[i, j] = sg
    return s


def real_block_loss_grads(Xc, Wc):
    """torch float64 CPU autograd of L = sum(Y_r^2), Y_r = Lexp(X) W_r.
    Xc: (mb, k, 4) components, Wc: (k, n, 4)."""
    S = _sign_table()
    X = torch.tensor(Xc, dtype=torch.float64, requires_grad=True)
    W = torch.tensor(Wc, dtype=torch.float64, requires_grad=True)
    mb, k, _ = Xc.shape
    n = Wc.shape[1]
    rows = []
    for c in range(4):
        cols = [S[c ^ j, j] * X[:, :, c ^ j] for j in range(4)]  # each (mb, k)
        rows.append(torch.stack(cols, dim=2))                    # (mb, k, 4 [j])
    Xbig = torch.stack(rows, dim=1).reshape(4 * mb, 4 * k)       # rows (i, c), cols (kappa, j)
    Wr = W.permute(0, 2, 1).reshape(4 * k, n)                    # rows (kappa, j)
    Yr = Xbig @ Wr                                               # rows (i, c)
    L = (Yr * Yr).sum()
    L.backward()
    return X.grad.numpy(), W.grad.numpy(), float(L)


def oracle_loss(Xs, Ws, mb, k, n):
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    Y = qsynth.empty(mb, n)
    orc.qgemm("N", "N", mb, n, k, one, Xs, Ws, zero, Y)
    return float(np.sum(Y * Y))


def gpu_grads(Xs, Ws, dtype, precision=None):
    X = to_dev(Xs, dtype).requires_grad_(True)
    W = to_dev(Ws, dtype).requires_grad_(True)
    Y = QLinearFunction.apply(X, W, "interleaved", precision)
    L = (Y.double() * Y.double()).sum()
    L.backward()
    return X.grad.double().cpu().numpy(), W.grad.double().cpu().numpy(), float(L)


def test_grad_vs_finite_differences_fp64():
    """16 x 16 x 16 slice, central differences of the oracle's loss, step 1e-3
    (the loss is quadratic in each entry, so the difference is exact up to
    rounding)."""
    mb = k = n = 16
    Xs = qsynth.normal(mb, k, 51)
    Ws = qsynth.normal(k, n, 52, scale=0.25)
    gX, gW, _ = gpu_grads(Xs, Ws, torch.float64)
    h = 1e-3
    g = qsynth.rng(53)
    for arr, grad in ((Xs, gX), (Ws, gW)):
        idx = [tuple(int(v) for v in (g.integers(0, arr.shape[0]), g.integers(0, arr.shape[1]),
                                      g.integers(0, 4))) for _ in range(48)]
        fd = []
        for t in idx:
            old = arr[t]
            arr[t] = old + h
            lp = oracle_loss(Xs, Ws, mb, k, n)
            arr[t] = old - h
            lm = oracle_loss(Xs, Ws, mb, k, n)
            arr[t] = old
            fd.append((lp - lm) / (2 * h))
        got = np.array([grad[t] for t in idx])
        fd = np.array(fd)
        assert rel_fro(got, fd) <= 1e-9, rel_fro(got, fd)


@pytest.mark.parametrize("dtype,tol,precision", [(torch.float64, 1e-12, None),
                                                 (torch.float32, 2e-6, None),
                                                 (torch.float64, 1e-12, "fp64_sliced")])
def test_grad_vs_real_block_form(dtype, tol, precision):
    mb, k, n = 70, 40, 36
    Xs = qsynth.normal(mb, k, 61)
    Ws = qsynth.normal(k, n, 62, scale=1.0 / 16)
    if dtype == torch.float32:
        Xs, Ws = Xs.astype(np.float32).astype(np.float64), Ws.astype(np.float32).astype(np.float64)
    gX, gW, L = gpu_grads(Xs, Ws, dtype, precision)
    rX, rW, Lr = real_block_loss_grads(qsynth.components(Xs, mb, "interleaved"),
                                       qsynth.components(Ws, k, "interleaved"))
    assert abs(L - Lr) <= 10 * tol * Lr
    assert rel_fro(qsynth.components(gX, mb, "interleaved"), rX) <= tol
    assert rel_fro(qsynth.components(gW, k, "interleaved"), rW) <= tol


def test_backward_accumulate_and_skip():
    mb, k, n = 33, 20, 17
    Xs, Ws, dYs = qsynth.normal(mb, k, 71), qsynth.normal(k, n, 72), qsynth.normal(mb, n, 73)
    X, W, dY = to_dev(Xs), to_dev(Ws), to_dev(dYs)
    dX0, dW0 = to_dev(qsynth.normal(mb, k, 74)), to_dev(qsynth.normal(k, n, 75))
    dX, dW = dX0.clone(), dW0.clone()
    ops.qgemm_backward(X, W, dY, mb, k, n, dX=dX, dW=dW, accumulate=True)
    one = np.array([1.0, 0, 0, 0])
    refX = dX0.cpu().numpy().copy()
    orc.qgemm("N", "H", mb, k, n, one, dYs, Ws, one, refX)
    refW = dW0.cpu().numpy().copy()
    orc.qgemm("H", "N", k, n, mb, one, Xs, dYs, one, refW)
    assert rel_fro(dX.cpu().numpy(), refX) <= 1e-12
    assert rel_fro(dW.cpu().numpy(), refW) <= 1e-12
    dW2 = dW0.clone()
    ops.qgemm_backward(X, W, dY, mb, k, n, dX=None, dW=dW2)
    refW2 = qsynth.empty(k, n)
    orc.qgemm("H", "N", k, n, mb, one, Xs, dYs, np.zeros(4), refW2)
    assert rel_fro(dW2.cpu().numpy(), refW2) <= 1e-12


def test_linear_layer_8192x1024x1024_split():
    """X 8192 x 1024, W 1024 x 1024 (W ~ N(0, 1/4096)), FP32 split path:
    forward Y and backward dX, dW for a seeded dY, sampled against the oracle."""
    mb, k, n = 8192, 1024, 1024
    Xs = qsynth.normal(mb, k, 81, pad=0.0).astype(np.float32).astype(np.float64)
    Ws = qsynth.normal(k, n, 82, scale=1.0 / 64, pad=0.0).astype(np.float32).astype(np.float64)
    dYs = qsynth.normal(mb, n, 83, pad=0.0).astype(np.float32).astype(np.float64)
    X, W, dY = to_dev(Xs, torch.float32), to_dev(Ws, torch.float32), to_dev(dYs, torch.float32)
    Y = QLinearFunction.apply(X, W)
    dX, dW = torch.empty_like(X), torch.empty_like(W)
    ops.qgemm_backward(X, W, dY, mb, k, n, dX=dX, dW=dW)
    torch.cuda.synchronize()
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    g = qsynth.rng(84)
    for (got, opA, opB, M, N, K, A, B) in (
            (Y, "N", "N", mb, n, k, Xs, Ws),
            (dX, "N", "H", mb, k, n, dYs, Ws),
            (dW, "H", "N", k, n, mb, Xs, dYs)):
        rows, cols = g.integers(0, M, 1024), g.integers(0, N, 1024)
        ref = orc.qgemm_entries(opA, opB, M, N, K, one, A, B, zero, qsynth.empty(M, N),
                                rows, cols)
        G = qsynth.components(got.double().cpu().numpy(), M, "interleaved")[rows, cols]
        err = rel_fro(G, ref)
        print("linear layer %s%s rel err %.3e" % (opA, opB, err))
        assert err <= 2e-6
