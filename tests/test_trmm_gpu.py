"""Triangular product qtrmm (side L/R, lower/upper, every op, unit or not)
on every precision, through the C ABI, against the FP64 oracle.

Bar: FP64 within 1e-12 (bit-exact on small integers), digit-sliced FP64
within 1e-12, split-BF16 within 2e-6 relative Frobenius error."""
import numpy as np
import pytest
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import _abi, ops
from tests.gpu_util import padding, rel_fro, to_dev

pytestmark = pytest.mark.gpu
ALPHA = qsynth.unit_quaternion(61)
TOL = {"fp64": 1e-12, "fp64_sliced": 1e-12, "split_bf16": 2e-6}


def run_case(side, uplo, trans, diag, m, n, layout, seed, precision="fp64", kind="normal",
             alpha=ALPHA):
    K = m if side == "L" else n
    make = qsynth.small_int if kind == "int" else qsynth.normal
    A = make(K, K, seed, layout, ld=K + 1)
    B = make(m, n, seed + 1, layout, ld=m + 2)
    if precision == "split_bf16":
        A, B = (X.astype(np.float32).astype(np.float64) for X in (A, B))
    C = qsynth.empty(m, n, layout, ld=m + 3)
    ref = orc.qtrmm(side, uplo, trans, diag, m, n, alpha, A, B, C.copy(), layout=layout)
    dt = torch.float32 if precision == "split_bf16" else torch.float64
    dA, dB, dC = to_dev(A, dt), to_dev(B, dt), to_dev(C, dt)
    ops.qtrmm(side, uplo, trans, diag, m, n, alpha, dA, dB, dC, layout=layout,
              precision=None if precision == "split_bf16" else precision)
    torch.cuda.synchronize()
    got = dC.double().cpu().numpy()
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    if kind == "int":
        assert np.array_equal(g, r)
    else:
        err = rel_fro(g, r)
        assert err <= TOL[precision], "%s %s%s%s%s err %.3e" % (precision, side, uplo, trans,
                                                                  diag, err)
    assert np.all(np.isnan(padding(got, m, layout)))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("side", ("L", "R"))
@pytest.mark.parametrize("uplo", ("L", "U"))
@pytest.mark.parametrize("trans", "NTCH")
@pytest.mark.parametrize("diag", ("N", "U"))
def test_fp64_every_variant(side, uplo, trans, diag, layout):
    """Ragged shapes spanning several FP64 tiles and k-blocks."""
    run_case(side, uplo, trans, diag, 70, 45, layout, seed=10 + "NTCH".index(trans))


@pytest.mark.parametrize("side", ("L", "R"))
@pytest.mark.parametrize("uplo", ("L", "U"))
def test_fp64_small_int_exact(side, uplo):
    run_case(side, uplo, "H", "N", 50, 37, "interleaved", seed=30, kind="int",
             alpha=np.array([1.0, -2.0, 0.0, 1.0]))


@pytest.mark.parametrize("precision", ("fp64_sliced", "split_bf16"))
@pytest.mark.parametrize("side", ("L", "R"))
@pytest.mark.parametrize("uplo", ("L", "U"))
@pytest.mark.parametrize("trans", "NH")
@pytest.mark.parametrize("diag", ("N", "U"))
def test_tensor_core_precisions(precision, side, uplo, trans, diag):
    """The split-BF16 and digit-sliced paths: several 128-row tiles and
    256-k chunks, ragged."""
    run_case(side, uplo, trans, diag, 300, 150, "interleaved", seed=40, precision=precision)


@pytest.mark.parametrize("precision", ("fp64", "fp64_sliced", "split_bf16"))
def test_large_ragged(precision):
    run_case("L", "L", "N", "N", 1000, 300, "interleaved", seed=50, precision=precision)
    run_case("R", "U", "H", "U", 300, 1000, "interleaved", seed=51, precision=precision)


def test_in_place_rejected_and_alpha_zero():
    m, n = 20, 10
    A = to_dev(qsynth.normal(m, m, 1))
    B = to_dev(qsynth.normal(m, n, 2))
    L = _abi.lib()
    ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    rc = L.qtrmm(0, 0, 0, 0, m, n, _abi.q4(ALPHA), A.data_ptr(), m, 0, B.data_ptr(), m, 0,
                 B.data_ptr(), m, 0, 0, 0, ws.data_ptr(), ws.numel(), None)
    assert rc == -14
    C = torch.full((n, m, 4), float("nan"), dtype=torch.float64, device="cuda")
    rc = L.qtrmm(0, 0, 0, 0, m, n, _abi.q4([0, 0, 0, 0]), None, m, 0, None, m, 0, C.data_ptr(),
                 m, 0, 0, 0, None, 0, None)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.all(C == 0)
