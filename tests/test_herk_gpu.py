"""Hermitian rank-k update (qherk) against the FP64 oracle, through the C ABI:
one triangle of C written, the other untouched, the diagonal real."""
import numpy as np
import pytest
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import _abi, ops
from tests.gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu


def run(uplo, trans, n, k, layout, dtype, seed, alpha=1.5, beta=-0.5, kind="normal"):
    make = qsynth.small_int if kind == "int" else qsynth.normal
    ra, ca = (n, k) if trans == "N" else (k, n)
    A = make(ra, ca, seed, layout, ld=ra + 2)
    C = make(n, n, seed + 1, layout, ld=n + 1)
    if dtype == torch.float32:
        A, C = A.astype(np.float32).astype(np.float64), C.astype(np.float32).astype(np.float64)
    ref = C.copy()
    orc.qherk(uplo, trans, n, k, alpha, A, beta, ref, layout=layout)
    dA, dC = to_dev(A, dtype), to_dev(C, dtype)
    ops.qherk(uplo, trans, n, k, alpha, dA, beta, dC, layout=layout)
    torch.cuda.synchronize()
    got = dC.double().cpu().numpy()
    G, R, C0 = (qsynth.components(X, n, layout) for X in (got, ref, C))
    tri = np.tril(np.ones((n, n), bool)) if uplo == "L" else np.triu(np.ones((n, n), bool))
    assert np.array_equal(G[~tri], C0[~tri]), "other triangle modified"
    assert np.all(G[np.arange(n), np.arange(n), 1:] == 0.0), "diagonal not real"
    pad = got[:, n:, :] if layout == "interleaved" else got[:, :, n:]
    assert np.all(np.isnan(pad))
    return rel_fro(G[tri], R[tri]), G, R


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("trans", ["N", "H"])
def test_herk_fp64(uplo, trans, layout):
    err, _, _ = run(uplo, trans, 77, 45, layout, torch.float64, 10)
    assert err <= 1e-12


@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("trans", ["N", "H"])
def test_herk_fp64_small_int_exact(uplo, trans):
    _, G, R = run(uplo, trans, 40, 30, "interleaved", torch.float64, 20, alpha=2.0, beta=3.0,
                  kind="int")
    tri = np.tril(np.ones((40, 40), bool)) if uplo == "L" else np.triu(np.ones((40, 40), bool))
    assert np.array_equal(G[tri], R[tri])


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("trans", ["N", "H"])
def test_herk_split(uplo, trans, layout):
    err, _, _ = run(uplo, trans, 300, 70, layout, torch.float32, 30)
    assert err <= 2e-6


def test_herk_k_zero_and_alpha_zero():
    for k, alpha in ((0, 1.0), (9, 0.0)):
        err, _, _ = run("L", "N", 20, k, "interleaved", torch.float64, 40, alpha=alpha)
        assert err <= 1e-15


def test_herk_argument_codes():
    L = _abi.lib()
    assert L.qherk(2, 0, 4, 4, 1.0, 64, 4, 0, 0.0, 64, 4, 0, 0, 0, None, 0, None) == -1
    assert L.qherk(0, 1, 4, 4, 1.0, 64, 4, 0, 0.0, 64, 4, 0, 0, 0, None, 0, None) == -2
    assert L.qherk(0, 0, 4, 4, 1.0, 64, 3, 0, 0.0, 64, 4, 0, 0, 0, None, 0, None) == -7
    assert L.qherk(0, 0, 4, 4, 1.0, 64, 4, 0, 0.0, 64, 2, 0, 0, 0, None, 0, None) == -11


def test_herk_sampled_4096_split():
    """n = 4096, k = 1024, FP32 split path, sampled triangle entries."""
    n, k = 4096, 1024
    A = qsynth.normal(n, k, 50, pad=0.0).astype(np.float32).astype(np.float64)
    C = qsynth.normal(n, n, 51, pad=0.0).astype(np.float32).astype(np.float64)
    dA, dC = to_dev(A, torch.float32), to_dev(C, torch.float32)
    ops.qherk("L", "N", n, k, 1.0, dA, 0.5, dC)
    torch.cuda.synchronize()
    G = qsynth.components(dC.double().cpu().numpy(), n, "interleaved")
    g = qsynth.rng(52)
    i, j = g.integers(0, n, 2048), g.integers(0, n, 2048)
    lo, hi = np.maximum(i, j), np.minimum(i, j)
    # entry (lo, hi) of A A^H through the GEMM oracle's sampled entries
    ref = orc.qgemm_entries("N", "H", n, n, k, [1.0, 0, 0, 0], A, A, [0.5, 0, 0, 0], C, lo, hi)
    ref[lo == hi, 1:] = 0.0
    err = rel_fro(G[lo, hi], ref)
    print("herk 4096 split sampled rel err %.3e" % err)
    assert err <= 2e-6


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("uplo", ["L", "U"])
@pytest.mark.parametrize("trans", ["N", "H"])
def test_herk_fp64_split_k(uplo, trans, layout):
    """A small, long update (n = 50, k = 8000): qherk_workspace_bytes lets
    the FP64 path split K; the triangle, the real diagonal and the untouched
    other triangle hold as unsplit."""
    assert _abi.lib().qherk_workspace_bytes(0 if uplo == "L" else 1, 0 if trans == "N" else 3,
                                            50, 8000, _abi.LAYOUT[layout], 0) > 0
    err, _, _ = run(uplo, trans, 50, 8000, layout, torch.float64, 50)
    assert err <= 1e-12


@pytest.mark.parametrize("uplo", ["L", "U"])
def test_herk_fp64_split_k_small_int_exact(uplo):
    _, G, R = run(uplo, "H", 37, 3000, "interleaved", torch.float64, 60, alpha=2.0, beta=3.0,
                  kind="int")
    tri = np.tril(np.ones((37, 37), bool)) if uplo == "L" else np.triu(np.ones((37, 37), bool))
    assert np.array_equal(G[tri], R[tri])
