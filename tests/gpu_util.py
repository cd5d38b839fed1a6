"""Helpers for the GPU parity tests: move seeded inputs to the device, run
the library through its C ABI, and compare with the FP64 oracle."""
import numpy as np
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import ops


def to_dev(X, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(X))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def padding(X, rows, layout):
    return X[:, rows:, :] if layout == "interleaved" else X[:, :, rows:]


def make_case(opA, opB, m, n, k, layout, seed, kind="normal", pad=(1, 2, 3), dtype=np.float64):
    """Stored A, B, C (numpy FP64, NaN padding rows) for op(A) m x k, op(B) k x n."""
    make = {"normal": qsynth.normal, "int": qsynth.small_int, "scaled": qsynth.scaled}[kind]
    ra, ca = qsynth.stored_shape(opA, m, k)
    rb, cb = qsynth.stored_shape(opB, k, n)
    A = make(ra, ca, seed, layout, ld=ra + pad[0])
    B = make(rb, cb, seed + 1, layout, ld=rb + pad[1])
    C = make(m, n, seed + 2, layout, ld=m + pad[2])
    if dtype != np.float64:
        A, B, C = (X.astype(dtype).astype(np.float64) for X in (A, B, C))  # exact in dtype
    return A, B, C


def oracle_full(opA, opB, m, n, k, alpha, A, B, beta, C, layout):
    R = C.copy()
    orc.qgemm(opA, opB, m, n, k, alpha, A, B, beta, R, layout=layout)
    return R


def gpu_run(opA, opB, m, n, k, alpha, A, B, beta, C, layout, dtype=torch.float64):
    dA, dB, dC = to_dev(A, dtype), to_dev(B, dtype), to_dev(C, dtype)
    ops.qgemm(opA, opB, m, n, k, alpha, dA, dB, beta, dC, layout=layout)
    torch.cuda.synchronize()
    return dC.cpu().double().numpy()


def rel_fro(X, Ref):
    d = np.linalg.norm((X - Ref).ravel())
    r = np.linalg.norm(Ref.ravel())
    return d / r if r > 0 else d
