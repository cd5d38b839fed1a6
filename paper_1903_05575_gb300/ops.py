"""Thin torch-facing binding over the C ABI (argument marshalling only).

Tensors are column-major quaternion matrices:
  interleaved: shape (cols, ld, 4), C-contiguous; component s of element
               (r, c) at [c, r, s] -- four contiguous reals per element (Sec. 4)
  planes:      shape (4, cols, ld), C-contiguous; plane s at [s] (Sec. 2.2)
Row counts are given explicitly (rows <= ld).  float64 tensors run the FP64
path (DMMA) unless precision="fp64_sliced" asks for the digit-sliced FP64
path on the BF16 tensor cores; float32 tensors run the split-BF16 path.
Every call goes to the CUDA library on torch's current stream; there is no
CPU fallback.
"""
import torch

from . import _abi

_workspaces = {}


def geometry(X, layout):
    """(ld, plane_stride, stored_cols) of a tensor in the given layout."""
    if not X.is_contiguous():
        raise ValueError("quaternion tensors must be contiguous")
    if layout == "interleaved":
        if X.dim() != 3 or X.shape[2] != 4:
            raise ValueError("interleaved tensors have shape (cols, ld, 4)")
        return X.shape[1], 0, X.shape[0]
    if X.dim() != 3 or X.shape[0] != 4:
        raise ValueError("split-plane tensors have shape (4, cols, ld)")
    return X.shape[2], X.shape[1] * X.shape[2], X.shape[1]


def precision_of(dtype, precision=None):
    """The library precision for a tensor dtype: float64 -> "fp64" (or
    "fp64_sliced" when asked), float32 -> "split_bf16"."""
    if dtype == torch.float64:
        if precision in (None, "fp64", "fp64_sliced"):
            return precision or "fp64"
    elif dtype == torch.float32:
        if precision in (None, "split_bf16"):
            return "split_bf16"
    else:
        raise TypeError("quaternion GEMM takes float64 (FP64 paths) or float32 (split-BF16 path)")
    raise ValueError("precision %r does not take %s data" % (precision, dtype))


def _stream_of(stream, device=None):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return stream


def _stream_handle(stream):
    return _stream_of(stream).cuda_stream


def workspace(nbytes, device, stream=None):
    """A cached device workspace of at least nbytes for calls on `stream`
    (torch's current stream when None), grown on demand.  Each (device,
    stream) pair has its own buffer, allocated on that stream, so calls on
    unordered streams never share a workspace, and a buffer replaced by a
    larger one goes back to torch's allocator on the stream that used it."""
    if nbytes == 0:
        return None
    dev = torch.device(device)
    s = _stream_of(stream, dev)
    key = (dev.index or 0, s.cuda_stream)
    ws = _workspaces.get(key)
    if ws is None or ws.numel() < nbytes:
        with torch.cuda.stream(s):
            ws = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=dev)
        _workspaces[key] = ws
    return ws


def qgemm(opA, opB, m, n, k, alpha, A, B, beta, C, layout="interleaved", ws=None,
          stream=None, precision=None):
    """C <- alpha op(A) op(B) + beta C on the GPU (C is updated in place).

    ws: a uint8 device tensor, or None for the module's cached workspace of
    the size qgemm_workspace_bytes reports.  That size includes the optional
    part that lets a product with a small C and a long k split K across CTAs
    (the only workspace the FP64 path uses); a smaller ws runs K unsplit, or
    fails with the ABI's -20 below the tensor-core paths' minimum."""
    prec = precision_of(C.dtype, precision)
    if A.dtype != C.dtype or B.dtype != C.dtype:
        raise TypeError("A, B and C must share a dtype")
    L = _abi.lib()
    lda, psA, _ = geometry(A, layout)
    ldb, psB, _ = geometry(B, layout)
    ldc, psC, _ = geometry(C, layout)
    need = L.qgemm_workspace_bytes(_abi.OP[opA], _abi.OP[opB], m, n, k, _abi.LAYOUT[layout],
                                   _abi.PRECISION[prec])
    if ws is None:
        ws = workspace(need, C.device, stream)
    wptr = ws.data_ptr() if ws is not None else None
    wbytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = L.qgemm(_abi.OP[opA], _abi.OP[opB], m, n, k, _abi.q4(alpha), A.data_ptr(), lda, psA,
                 B.data_ptr(), ldb, psB, _abi.q4(beta), C.data_ptr(), ldc, psC,
                 _abi.LAYOUT[layout], _abi.PRECISION[prec], wptr, wbytes, _stream_handle(stream))
    _abi.check(rc, "qgemm")
    return C


def qherk(uplo, trans, n, k, alpha, A, beta, C, layout="interleaved", ws=None, stream=None,
          precision=None):
    """Hermitian rank-k update on one triangle of C (real alpha, beta):
    trans N: C <- alpha A A^H + beta C;  trans H: C <- alpha A^H A + beta C."""
    prec = precision_of(C.dtype, precision)
    L = _abi.lib()
    lda, psA, _ = geometry(A, layout)
    ldc, psC, _ = geometry(C, layout)
    up, tr = {"L": 0, "U": 1}[uplo], _abi.OP[trans]
    need = L.qherk_workspace_bytes(up, tr, n, k, _abi.LAYOUT[layout], _abi.PRECISION[prec])
    if ws is None:
        ws = workspace(need, C.device, stream)
    wptr = ws.data_ptr() if ws is not None else None
    wbytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = L.qherk(up, tr, n, k, float(alpha), A.data_ptr(), lda, psA, float(beta), C.data_ptr(),
                 ldc, psC, _abi.LAYOUT[layout], _abi.PRECISION[prec], wptr, wbytes,
                 _stream_handle(stream))
    _abi.check(rc, "qherk")
    return C


_WIDTH = {"H": 4, "C": 2, "R": 1}
_TYPE = {"H": 0, "C": 1, "R": 2}


def typed_geometry(X, layout, typ):
    """(ld, plane_stride) of a quaternion ("H"), complex ("C") or real ("R")
    tensor: interleaved (cols, ld, width) (a real one may be (cols, ld));
    planes (width, cols, ld)."""
    if not X.is_contiguous():
        raise ValueError("tensors must be contiguous")
    w = _WIDTH[typ]
    if layout == "interleaved":
        if typ == "R" and X.dim() == 2:
            return X.shape[1], 0
        if X.dim() != 3 or X.shape[2] != w:
            raise ValueError("interleaved %s tensors have shape (cols, ld, %d)" % (typ, w))
        return X.shape[1], 0
    if X.dim() != 3 or X.shape[0] != w:
        raise ValueError("split-plane %s tensors have shape (%d, cols, ld)" % (typ, w))
    return X.shape[2], X.shape[1] * X.shape[2]


def qgemm_mixed(typeA, typeB, opA, opB, m, n, k, alpha, A, B, beta, C, layout="interleaved",
                ws=None, stream=None, precision=None):
    """C <- alpha op(A) op(B) + beta C with A, B quaternion ("H"), complex ("C")
    or real ("R") and C quaternion (in place)."""
    prec = precision_of(C.dtype, precision)
    if A.dtype != C.dtype or B.dtype != C.dtype:
        raise TypeError("A, B and C must share a dtype")
    L = _abi.lib()
    lda, psA = typed_geometry(A, layout, typeA)
    ldb, psB = typed_geometry(B, layout, typeB)
    ldc, psC, _ = geometry(C, layout)
    head = (_TYPE[typeA], _TYPE[typeB], _abi.OP[opA], _abi.OP[opB], m, n, k)
    need = L.qgemm_mixed_workspace_bytes(*head, _abi.LAYOUT[layout], _abi.PRECISION[prec])
    if ws is None:
        ws = workspace(need, C.device, stream)
    wptr = ws.data_ptr() if ws is not None else None
    wbytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = L.qgemm_mixed(*head, _abi.q4(alpha), A.data_ptr(), lda, psA, B.data_ptr(), ldb, psB,
                       _abi.q4(beta), C.data_ptr(), ldc, psC, _abi.LAYOUT[layout],
                       _abi.PRECISION[prec], wptr, wbytes, _stream_handle(stream))
    _abi.check(rc, "qgemm_mixed")
    return C


def qtrmm(side, uplo, trans, diag, m, n, alpha, A, B, C, layout="interleaved", ws=None,
          stream=None, precision=None):
    """Triangular product into C (written, not read, must not be B):
    side "L": C = alpha op(tri(A)) B;  side "R": C = alpha B op(tri(A));
    tri(A) = the uplo ("L"/"U") triangle of A, unit diagonal if diag == "U"."""
    prec = precision_of(C.dtype, precision)
    if A.dtype != C.dtype or B.dtype != C.dtype:
        raise TypeError("A, B and C must share a dtype")
    L = _abi.lib()
    lda, psA, _ = geometry(A, layout)
    ldb, psB, _ = geometry(B, layout)
    ldc, psC, _ = geometry(C, layout)
    args = ({"L": 0, "R": 1}[side], {"L": 0, "U": 1}[uplo], _abi.OP[trans],
            {"N": 0, "U": 1}[diag], m, n)
    need = L.qtrmm_workspace_bytes(*args, _abi.LAYOUT[layout], _abi.PRECISION[prec])
    if ws is None:
        ws = workspace(need, C.device, stream)
    wptr = ws.data_ptr() if ws is not None else None
    wbytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = L.qtrmm(*args, _abi.q4(alpha), A.data_ptr(), lda, psA, B.data_ptr(), ldb, psB,
                 C.data_ptr(), ldc, psC, _abi.LAYOUT[layout], _abi.PRECISION[prec], wptr, wbytes,
                 _stream_handle(stream))
    _abi.check(rc, "qtrmm")
    return C


def qgemm_backward(X, W, dY, mb, k, n, dX=None, dW=None, accumulate=False,
                   layout="interleaved", ws=None, stream=None, precision=None):
    """dX = dY W^H and dW = X^H dY for Y = X W (either output may be None)."""
    prec = precision_of(X.dtype, precision)
    L = _abi.lib()
    ldx, psx, _ = geometry(X, layout)
    ldw, psw, _ = geometry(W, layout)
    lddy, psdy, _ = geometry(dY, layout)
    lddx, psdx = (geometry(dX, layout)[:2] if dX is not None else (max(mb, 1), 0))
    lddw, psdw = (geometry(dW, layout)[:2] if dW is not None else (max(k, 1), 0))
    need = L.qgemm_backward_workspace_bytes(mb, k, n, _abi.LAYOUT[layout], _abi.PRECISION[prec])
    if ws is None:
        ws = workspace(need, X.device, stream)
    wptr = ws.data_ptr() if ws is not None else None
    wbytes = ws.numel() * ws.element_size() if ws is not None else 0
    rc = L.qgemm_backward(mb, k, n, X.data_ptr(), ldx, psx, W.data_ptr(), ldw, psw,
                          dY.data_ptr(), lddy, psdy,
                          dX.data_ptr() if dX is not None else None, lddx, psdx,
                          dW.data_ptr() if dW is not None else None, lddw, psdw,
                          1 if accumulate else 0, _abi.LAYOUT[layout], _abi.PRECISION[prec],
                          wptr, wbytes, _stream_handle(stream))
    _abi.check(rc, "qgemm_backward")
    return dX, dW


class GroupedBatch:
    """Many independent problems C_p <- alpha_p op(A_p) op(B_p) + beta_p C_p in
    one persistent launch (C ABI qgemm_grouped_prepare / qgemm_grouped_launch).

    problems: sequence of dicts with keys opA, opB, m, n, k, alpha, beta, A, B,
    C (tensors of one dtype and layout); float64 batches take precision
    "fp64" (DMMA) or "fp64_sliced".  prepare() runs once (not during
    graph capture); launch() only resets a counter and launches, so it can be
    captured in a CUDA graph and replayed.  The tensors must stay alive.
    """

    def __init__(self, problems, layout="interleaved", ws=None, stream=None, precision=None):
        import ctypes

        from . import autotune
        autotune.ensure_plan_loaded()
        self.problems = list(problems)
        if not self.problems:
            raise ValueError("empty batch")
        self.layout = layout
        self.prec = precision_of(self.problems[0]["C"].dtype, precision)
        arr = (_abi.QgemmProblem * len(self.problems))()
        for i, p in enumerate(self.problems):
            q = arr[i]
            q.opA, q.opB = _abi.OP[p["opA"]], _abi.OP[p["opB"]]
            q.m, q.n, q.k = p["m"], p["n"], p["k"]
            for s in range(4):
                q.alpha[s] = float(p["alpha"][s])
                q.beta[s] = float(p["beta"][s])
            for name in ("A", "B", "C"):
                X = p[name]
                ld, ps, _ = geometry(X, layout)
                setattr(q, name, X.data_ptr())
                setattr(q, "ld" + name.lower(), ld)
                setattr(q, "ps" + name, ps)
        self._arr = arr
        L = _abi.lib()
        n = len(self.problems)
        need = L.qgemm_grouped_workspace_bytes(arr, n, _abi.LAYOUT[layout],
                                               _abi.PRECISION[self.prec])
        if need == 0:
            raise _abi.QgemmError(_abi.ERR_UNSUPPORTED, "qgemm_grouped_workspace_bytes")
        dev = self.problems[0]["C"].device
        self.ws = ws if ws is not None else torch.empty(need, dtype=torch.uint8, device=dev)
        self.plan = _abi.QgemmGroupedPlan()
        rc = L.qgemm_grouped_prepare(arr, n, _abi.LAYOUT[layout], _abi.PRECISION[self.prec],
                                     self.ws.data_ptr(), self.ws.numel(), _stream_handle(stream),
                                     ctypes.byref(self.plan))
        _abi.check(rc, "qgemm_grouped_prepare")

    def launch(self, stream=None):
        import ctypes
        rc = _abi.lib().qgemm_grouped_launch(ctypes.byref(self.plan), _stream_handle(stream))
        _abi.check(rc, "qgemm_grouped_launch")


def set_tile_table(table, precision="fp64"):
    """Install a per-bucket tile-shape table (None restores the default).  An
    explicit table takes precedence over a stored autotuner plan."""
    import ctypes

    from . import autotune
    autotune._loaded = True
    L = _abi.lib()
    if table is None:
        rc = L.qgemm_grouped_set_tile_table(_abi.PRECISION[precision], None, 0)
    else:
        arr = (ctypes.c_int32 * len(table))(*[int(x) for x in table])
        rc = L.qgemm_grouped_set_tile_table(_abi.PRECISION[precision], arr, len(table))
    _abi.check(rc, "qgemm_grouped_set_tile_table")


def tile_info():
    """(shapes [(rows, cols)], number of buckets, bucket edges)."""
    import ctypes
    ns, nb = ctypes.c_int32(0), ctypes.c_int32(0)
    rows, cols, edges = (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 4)()
    _abi.lib().qgemm_grouped_tile_info(ctypes.byref(ns), rows, cols, ctypes.byref(nb), edges)
    return ([(rows[i], cols[i]) for i in range(ns.value)], nb.value, list(edges))


def last_device_error():
    return _abi.lib().qgemm_get_last_device_error()


def probe_peak(which, seconds=0.3, stream=None):
    """Measured TFLOP/s of a pipe: 0 DMMA, 1 DFMA, 2 FFMA, 3 tcgen05 BF16."""
    import ctypes
    out = ctypes.c_double(0.0)
    rc = _abi.lib().qgemm_probe_peak(which, seconds, ctypes.byref(out), _stream_handle(stream))
    _abi.check(rc, "qgemm_probe_peak")
    return out.value
