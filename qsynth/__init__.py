"""Seeded synthetic inputs for quaternion GEMM.

This module only draws numbers and lays them out in memory.  It holds none
of the product's arithmetic, so both the FP64 oracle and the GPU tests can
use it without sharing any of the method's code.

Array conventions (numpy, C-contiguous), column-major quaternion matrices
with leading dimension ``ld`` (rows <= ld):
  interleaved  shape (cols, ld, 4): component s of element (r, c) at [c, r, s]
  planes       shape (4, cols, ld): component s of element (r, c) at [s, c, r]
Padding rows r >= rows are filled with ``pad`` (NaN by default) so that a
kernel that reads or writes them is caught.
"""
import numpy as np

LAYOUTS = ("interleaved", "planes")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def empty(rows, cols, layout="interleaved", ld=None, dtype=np.float64, pad=np.nan):
    ld = rows if ld is None else ld
    ld = max(ld, 1)
    if ld < rows:
        raise ValueError("ld < rows")
    shape = (cols, ld, 4) if layout == "interleaved" else (4, cols, ld)
    return np.full(shape, pad, dtype=dtype)


def _place(vals, rows, cols, layout, ld, dtype, pad):
    """vals: (rows, cols, 4) component array -> storage layout."""
    out = empty(rows, cols, layout, ld, dtype, pad)
    if layout == "interleaved":
        out[:, :rows, :] = np.transpose(vals, (1, 0, 2))
    else:
        out[:, :, :rows] = np.transpose(vals, (2, 1, 0))
    return out


def components(X, rows, layout):
    """Storage layout -> (rows, cols, 4) array of components (a copy)."""
    if layout == "interleaved":
        return np.ascontiguousarray(np.transpose(X[:, :rows, :], (1, 0, 2)))
    return np.ascontiguousarray(np.transpose(X[:, :, :rows], (2, 1, 0)))


def normal(rows, cols, seed, layout="interleaved", ld=None, dtype=np.float64, pad=np.nan,
           scale=1.0):
    """Components iid N(0, scale^2)."""
    v = rng(seed).standard_normal((rows, cols, 4)) * scale
    return _place(v, rows, cols, layout, ld, dtype, pad)


def small_int(rows, cols, seed, layout="interleaved", ld=None, dtype=np.float64, pad=np.nan,
              bound=8):
    """Integer components uniform in [-bound, bound] (exact in any summation order
    while the partial sums stay below 2^53 (FP64) or 2^24 (FP32))."""
    v = rng(seed).integers(-bound, bound + 1, size=(rows, cols, 4)).astype(np.float64)
    return _place(v, rows, cols, layout, ld, dtype, pad)


def scaled(rows, cols, seed, layout="interleaved", ld=None, dtype=np.float64, pad=np.nan,
           urange=20):
    """Components N(0,1) * 2^(u_r + v_c), u_r and v_c integers uniform in
    [-urange, urange] drawn per row and per column (wide dynamic range, also
    along the summation index)."""
    g = rng(seed)
    v = g.standard_normal((rows, cols, 4))
    ur = g.integers(-urange, urange + 1, size=rows)
    vc = g.integers(-urange, urange + 1, size=cols)
    v = v * np.ldexp(1.0, ur)[:, None, None] * np.ldexp(1.0, vc)[None, :, None]
    return _place(v, rows, cols, layout, ld, dtype, pad)


def unit_quaternion(seed):
    """A random quaternion of unit norm (4 iid N(0,1), normalised)."""
    q = rng(seed).standard_normal(4)
    return q / np.sqrt(np.sum(q * q))


def grouped_problems(count, seed, lo=8, hi=256, ops=("N", "H")):
    """Sizes and op flags for a grouped batch: m, n, k iid uniform integers in
    [lo, hi], opA and opB iid from ``ops``; alpha, beta random unit quaternions."""
    g = rng(seed)
    mnk = g.integers(lo, hi + 1, size=(count, 3))
    oa = g.integers(0, len(ops), size=count)
    ob = g.integers(0, len(ops), size=count)
    ab = g.standard_normal((count, 2, 4))
    ab /= np.sqrt(np.sum(ab * ab, axis=2, keepdims=True))
    probs = []
    for i in range(count):
        probs.append(dict(m=int(mnk[i, 0]), n=int(mnk[i, 1]), k=int(mnk[i, 2]),
                          opA=ops[oa[i]], opB=ops[ob[i]],
                          alpha=ab[i, 0].copy(), beta=ab[i, 1].copy(),
                          seed=int(seed * 1000003 + i)))
    return probs


def stored_shape(op, rows, cols):
    """(stored rows, stored cols) of X such that op(X) is rows x cols."""
    return (cols, rows) if op in ("T", "H") else (rows, cols)


WIDTH = {"H": 4, "C": 2, "R": 1}


def typed(rows, cols, seed, typ, layout="interleaved", ld=None, kind="normal", pad=np.nan,
          dtype=np.float64):
    """A quaternion ("H"), complex ("C") or real ("R") matrix with iid N(0,1)
    (kind "normal") or small-integer (kind "int", |x| <= 8) components:
    interleaved (cols, ld, width), planes (width, cols, ld)."""
    w = WIDTH[typ]
    g = rng(seed)
    if kind == "int":
        v = g.integers(-8, 9, size=(rows, cols, w)).astype(np.float64)
    else:
        v = g.standard_normal((rows, cols, w))
    ld = rows if ld is None else ld
    ld = max(ld, 1)
    if layout == "interleaved":
        out = np.full((cols, ld, w), pad, dtype=dtype)
        out[:, :rows, :] = np.transpose(v, (1, 0, 2))
    else:
        out = np.full((w, cols, ld), pad, dtype=dtype)
        out[:, :, :rows] = np.transpose(v, (2, 1, 0))
    return out


def typed_components(X, rows, typ, layout):
    """Typed storage -> (rows, cols, 4) quaternion components (missing ones 0)."""
    w = WIDTH[typ]
    if layout == "interleaved":
        v = np.transpose(X[:, :rows, :], (1, 0, 2))
    else:
        v = np.transpose(X[:, :, :rows], (2, 1, 0))
    out = np.zeros(v.shape[:2] + (4,))
    out[..., :w] = v
    return out
