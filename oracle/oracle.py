"""ctypes wrapper around the plain C FP64 oracle (``qgemm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the library.

Array conventions (numpy, float64, C-contiguous):
  interleaved  shape (cols, ld, 4): component s of element (r, c) at [c, r, s]
  split planes shape (4, cols, ld): component s of element (r, c) at [s, c, r]
Both are column-major quaternion matrices with leading dimension ``ld``
(Sec. 3.1 column-major storage; Sec. 4 interleaved element; Sec. 2.2 planes).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qgemm_oracle.c")
_LIB = os.path.join(_HERE, "libqgemm_oracle.so")

OPS = {"N": 0, "T": 1, "C": 2, "H": 3}
LAYOUTS = {"interleaved": 0, "planes": 1}


def build(force=False, src=_SRC, out=_LIB):
    """Compile the oracle with gcc (-O2, OpenMP).  No BLAS, no CUDA."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load_variant(path):
    """Load another compiled copy of the oracle (the mutation test plants
    mistakes in a copy of the C source and checks the pins catch them)."""
    return _bind(path)


_lib = None


def _bind(path):
    """Load a compiled oracle and declare its C signatures."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.oracle_hamilton.argtypes = [dp, dp, dp]
    lib.oracle_hamilton.restype = None
    lib.oracle_qgemm.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64, dp,
                                 dp, i64, i64, dp, i64, i64, dp, dp, i64, i64,
                                 ctypes.c_int, ctypes.c_int]
    lib.oracle_qgemm.restype = ctypes.c_int
    lib.oracle_qgemm_entries.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64, dp,
                                         dp, i64, i64, dp, i64, i64, dp, dp, i64, i64,
                                         ctypes.c_int, ctypes.POINTER(i64),
                                         ctypes.POINTER(i64), i64, dp, ctypes.c_int]
    lib.oracle_qgemm_entries.restype = ctypes.c_int
    lib.oracle_qherk.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, ctypes.c_double, dp, i64,
                                 i64, ctypes.c_double, dp, i64, i64, ctypes.c_int, ctypes.c_int]
    lib.oracle_qherk.restype = ctypes.c_int
    lib.oracle_qtrmm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, i64,
                                 dp, dp, i64, i64, dp, i64, i64, dp, i64, i64, ctypes.c_int,
                                 ctypes.c_int]
    lib.oracle_qtrmm.restype = ctypes.c_int
    lib.oracle_qgemm_mixed.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       i64, i64, i64, dp, dp, i64, i64, dp, i64, i64, dp, dp,
                                       i64, i64, ctypes.c_int, ctypes.c_int]
    lib.oracle_qgemm_mixed.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(_LIB)
    return _lib




def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _q4(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(4))
    return a


def geometry(X, layout):
    """(ld, plane_stride, stored_cols) of a quaternion array."""
    if layout == "interleaved":
        assert X.ndim == 3 and X.shape[2] == 4, X.shape
        return X.shape[1], 0, X.shape[0]
    assert X.ndim == 3 and X.shape[0] == 4, X.shape
    return X.shape[2], X.shape[1] * X.shape[2], X.shape[1]


def _check(X):
    if X.dtype != np.float64 or not X.flags.c_contiguous:
        raise TypeError("oracle arrays must be C-contiguous float64")


def max_threads(lib=None):
    return (lib or _load()).oracle_max_threads()


def hamilton(p, q, lib=None):
    """Hamilton product of two quaternions (Sec. 2.1, Eq. quaternion_prod)."""
    lib = lib or _load()
    p, q = _q4(p), _q4(q)
    r = np.zeros(4)
    lib.oracle_hamilton(_dptr(p), _dptr(q), _dptr(r))
    return r


def qgemm(opA, opB, m, n, k, alpha, A, B, beta, C, layout="interleaved", nthreads=0,
          lib=None):
    """C <- alpha op(A) op(B) + beta C in place (FP64, Eq. general_gemm)."""
    lib = lib or _load()
    for X in (A, B, C):
        _check(X)
    lda, psA, _ = geometry(A, layout)
    ldb, psB, _ = geometry(B, layout)
    ldc, psC, _ = geometry(C, layout)
    al, be = _q4(alpha), _q4(beta)
    rc = lib.oracle_qgemm(OPS[opA], OPS[opB], m, n, k, _dptr(al), _dptr(A), lda, psA,
                          _dptr(B), ldb, psB, _dptr(be), _dptr(C), ldc, psC,
                          LAYOUTS[layout], int(nthreads))
    if rc != 0:
        raise ValueError("oracle_qgemm returned %d" % rc)
    return C


def qgemm_entries(opA, opB, m, n, k, alpha, A, B, beta, C, rows, cols,
                  layout="interleaved", nthreads=0, lib=None):
    """Entries (rows[e], cols[e]) of alpha op(A) op(B) + beta C; C untouched."""
    lib = lib or _load()
    for X in (A, B, C):
        _check(X)
    lda, psA, _ = geometry(A, layout)
    ldb, psB, _ = geometry(B, layout)
    ldc, psC, _ = geometry(C, layout)
    al, be = _q4(alpha), _q4(beta)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    assert rows.shape == cols.shape
    out = np.zeros((rows.size, 4))
    i64p = ctypes.POINTER(ctypes.c_int64)
    rc = lib.oracle_qgemm_entries(OPS[opA], OPS[opB], m, n, k, _dptr(al), _dptr(A), lda, psA,
                                  _dptr(B), ldb, psB, _dptr(be), _dptr(C), ldc, psC,
                                  LAYOUTS[layout], rows.ctypes.data_as(i64p),
                                  cols.ctypes.data_as(i64p), rows.size, _dptr(out),
                                  int(nthreads))
    if rc != 0:
        raise ValueError("oracle_qgemm_entries returned %d" % rc)
    return out


def qherk(uplo, trans, n, k, alpha, A, beta, C, layout="interleaved", nthreads=0, lib=None):
    """Hermitian rank-k update on one triangle of C, in place (real alpha, beta):
    trans N: C <- alpha A A^H + beta C;  trans H: C <- alpha A^H A + beta C."""
    lib = lib or _load()
    for X in (A, C):
        _check(X)
    lda, psA, _ = geometry(A, layout)
    ldc, psC, _ = geometry(C, layout)
    rc = lib.oracle_qherk({"L": 0, "U": 1}[uplo], OPS[trans], n, k, float(alpha), _dptr(A), lda,
                          psA, float(beta), _dptr(C), ldc, psC, LAYOUTS[layout], int(nthreads))
    if rc != 0:
        raise ValueError("oracle_qherk returned %d" % rc)
    return C


def qtrmm(side, uplo, trans, diag, m, n, alpha, A, B, C, layout="interleaved", nthreads=0,
          lib=None):
    """Triangular product into C (written, not read): side L: C = alpha op(tri(A)) B,
    side R: C = alpha B op(tri(A)); tri(A) = the uplo triangle of A, unit
    diagonal when diag is "U"."""
    lib = lib or _load()
    for X in (A, B, C):
        _check(X)
    lda, psA, _ = geometry(A, layout)
    ldb, psB, _ = geometry(B, layout)
    ldc, psC, _ = geometry(C, layout)
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(4))
    rc = lib.oracle_qtrmm({"L": 0, "R": 1}[side], {"L": 0, "U": 1}[uplo], OPS[trans],
                          {"N": 0, "U": 1}[diag], m, n, _dptr(al), _dptr(A), lda, psA, _dptr(B),
                          ldb, psB, _dptr(C), ldc, psC, LAYOUTS[layout], int(nthreads))
    if rc != 0:
        raise ValueError("oracle_qtrmm returned %d" % rc)
    return C


TYPES = {"H": 0, "C": 1, "R": 2}
WIDTH = {"H": 4, "C": 2, "R": 1}


def typed_geometry(X, layout, typ):
    """(ld, plane_stride) of a typed operand: interleaved (cols, ld, width)
    (a real operand may also be (cols, ld)); planes (width, cols, ld)."""
    w = WIDTH[typ]
    if layout == "interleaved":
        if typ == "R" and X.ndim == 2:
            return X.shape[1], 0
        assert X.ndim == 3 and X.shape[2] == w
        return X.shape[1], 0
    assert X.ndim == 3 and X.shape[0] == w
    return X.shape[2], X.shape[1] * X.shape[2]


def qgemm_mixed(typeA, typeB, opA, opB, m, n, k, alpha, A, B, beta, C, layout="interleaved",
                nthreads=0, lib=None):
    """C <- alpha op(A) op(B) + beta C with A, B quaternion ("H"), complex ("C")
    or real ("R"); C quaternion, in place."""
    lib = lib or _load()
    for X in (A, B, C):
        _check(X)
    lda, psA = typed_geometry(A, layout, typeA)
    ldb, psB = typed_geometry(B, layout, typeB)
    ldc, psC, _ = geometry(C, layout)
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(4))
    be = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(4))
    rc = lib.oracle_qgemm_mixed(TYPES[typeA], TYPES[typeB], OPS[opA], OPS[opB], m, n, k,
                                _dptr(al), _dptr(A), lda, psA, _dptr(B), ldb, psB, _dptr(be),
                                _dptr(C), ldc, psC, LAYOUTS[layout], int(nthreads))
    if rc != 0:
        raise ValueError("oracle_qgemm_mixed returned %d" % rc)
    return C
