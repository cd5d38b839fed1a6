"""Mixed-type products qgemm_mixed (quaternion, complex or real factors, C
quaternion) on every precision, through the C ABI, against the FP64 oracle.

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
ALPHA = qsynth.unit_quaternion(71)
BETA = qsynth.unit_quaternion(72)
TOL = {"fp64": 1e-12, "fp64_sliced": 1e-12, "split_bf16": 2e-6}
PAIRS = [("H", "C"), ("C", "H"), ("H", "R"), ("R", "H"), ("C", "C"), ("R", "C"), ("C", "R")]


def run_case(tA, tB, opA, opB, m, n, k, layout, seed, precision="fp64", kind="normal",
             alpha=ALPHA, beta=BETA):
    ra, ca = qsynth.stored_shape(opA, m, k)
    rb, cb = qsynth.stored_shape(opB, k, n)
    A = qsynth.typed(ra, ca, seed, tA, layout, ld=ra + 1, kind=kind)
    B = qsynth.typed(rb, cb, seed + 1, tB, layout, ld=rb + 2, kind=kind)
    C = (qsynth.small_int if kind == "int" else qsynth.normal)(m, n, seed + 2, layout, ld=m + 3)
    if precision == "split_bf16":
        A, B, C = (X.astype(np.float32).astype(np.float64) for X in (A, B, C))
    ref = orc.qgemm_mixed(tA, tB, opA, opB, m, n, k, alpha, A, B, beta, C.copy(), layout=layout)
    dt = torch.float32 if precision == "split_bf16" else torch.float64
    dA, dB, dC = to_dev(A, dt), to_dev(B, dt), to_dev(C, dt)
    ops.qgemm_mixed(tA, tB, opA, opB, m, n, k, alpha, dA, dB, beta, dC, layout=layout,
                    precision=None if precision == "split_bf16" else precision)
    torch.cuda.synchronize()
    got = dC.double().cpu().numpy()
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    if kind == "int":
        assert np.array_equal(g, r)
    else:
        err = rel_fro(g, r)
        assert err <= TOL[precision], "%s %s%s %s%s err %.3e" % (precision, tA, tB, opA, opB, err)
    assert np.all(np.isnan(padding(got, m, layout)))
    return g, r


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("types", PAIRS)
@pytest.mark.parametrize("ops_", [("N", "N"), ("H", "T"), ("C", "H"), ("T", "C")])
def test_fp64(types, ops_, layout):
    run_case(*types, *ops_, 70, 45, 37, layout, seed=100 + PAIRS.index(types))


@pytest.mark.parametrize("types", PAIRS)
def test_fp64_small_int_exact(types):
    run_case(*types, "H", "N", 40, 33, 50, "interleaved", seed=200, kind="int",
             alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0, 1.0, -1.0]))


@pytest.mark.parametrize("precision", ("fp64_sliced", "split_bf16"))
@pytest.mark.parametrize("types", PAIRS)
@pytest.mark.parametrize("ops_", [("N", "N"), ("H", "T"), ("C", "H")])
def test_tensor_core_precisions(precision, types, ops_):
    """The narrow factor on the left of the real form (turned around with
    (AB)^H = B^H A^H when it is B): several 128-row tiles and 256-k chunks."""
    run_case(*types, *ops_, 200, 70, 300, "interleaved", seed=300 + PAIRS.index(types),
             precision=precision)


@pytest.mark.parametrize("precision", ("fp64_sliced", "split_bf16"))
def test_tensor_core_planes(precision):
    for types in (("H", "C"), ("R", "H")):
        run_case(*types, "H", "N", 150, 40, 100, "planes", seed=400, precision=precision)


def test_quaternion_pair_matches_qgemm():
    """typeA = typeB = quaternion is qgemm itself."""
    run_case("H", "H", "N", "H", 60, 50, 40, "interleaved", seed=500)


def test_argument_numbers():
    L = _abi.lib()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    rc = L.qgemm_mixed(3, 0, 0, 0, 4, 4, 4, _abi.q4([1, 0, 0, 0]), x.data_ptr(), 4, 0,
                       x.data_ptr(), 4, 0, _abi.q4([0, 0, 0, 0]), x.data_ptr(), 4, 0, 0, 0, None,
                       0, None)
    assert rc == -1
    rc = L.qgemm_mixed(0, 1, 0, 0, 4, 4, 4, _abi.q4([1, 0, 0, 0]), x.data_ptr(), 3, 0,
                       x.data_ptr(), 4, 0, _abi.q4([0, 0, 0, 0]), x.data_ptr(), 4, 0, 0, 0, None,
                       0, None)
    assert rc == -10   # lda, argument 8 of qgemm
