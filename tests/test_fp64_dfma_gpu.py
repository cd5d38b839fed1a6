"""FP64 products large enough for the FP64 FMA-pipe kernel (fp64_dfma.cu:
32 x 32-quaternion tiles, taken when the grid has at least 8 tiles per SM
and its waves are at least 90 % full)
against the FP64 oracle, through the C ABI.

Shapes are ragged in every dimension (2049 x 2433 x 37: 65 x 77 tiles) with
a short k so the oracle stays fast.  Bar as for the FP64 path: N(0,1) within
1e-12 relative Frobenius error, small integers bit-exact, padding rows (NaN
guard) untouched, beta = 0 never reading C."""
import numpy as np
import pytest

import qsynth
from tests.gpu_util import gpu_run, make_case, oracle_full, rel_fro
from tests.test_fp64_gpu import ALPHA, BETA, OPS, check

pytestmark = pytest.mark.gpu

M, N, K = 2049, 2433, 37


@pytest.mark.parametrize("opA", OPS)
@pytest.mark.parametrize("opB", OPS)
def test_op_pairs_interleaved(opA, opB):
    check(opA, opB, M, N, K, "interleaved", seed=601 + 4 * OPS.index(opA) + OPS.index(opB))


@pytest.mark.parametrize("opA,opB", [("N", "N"), ("T", "H"), ("C", "T"), ("H", "C")])
def test_op_pairs_planes(opA, opB):
    check(opA, opB, M, N, K, "planes", seed=641 + 4 * OPS.index(opA) + OPS.index(opB))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_small_int_exact(layout):
    check("H", "N", M, N, K, layout, seed=661, kind="int",
          alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0.0, -1.0, 0.0]))


def test_beta_zero_does_not_read_c():
    A, B, C = make_case("N", "T", M, N, K, "interleaved", 671)
    C[...] = np.nan
    zero = np.zeros(4)
    ref = oracle_full("N", "T", M, N, K, ALPHA, A, B, zero, np.zeros_like(C), "interleaved")
    got = gpu_run("N", "T", M, N, K, ALPHA, A, B, zero, C, "interleaved")
    g, r = qsynth.components(got, M, "interleaved"), qsynth.components(ref, M, "interleaved")
    assert np.all(np.isfinite(g)), "C was read although beta = 0"
    assert rel_fro(g, r) <= 1e-12
