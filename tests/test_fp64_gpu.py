"""FP64 path (DMMA) against the FP64 oracle, through the C ABI.

Bar: small-integer inputs bit-exact; N(0,1) inputs within 1e-12 relative
Frobenius error; padding rows (NaN guard) untouched."""
import ctypes

import numpy as np
import pytest
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import _abi, ops
from tests.gpu_util import gpu_run, make_case, oracle_full, padding, rel_fro, to_dev

pytestmark = pytest.mark.gpu

OPS = ("N", "T", "C", "H")
TOL = 1e-12
ALPHA = np.array([0.5, -1.0, 2.0, 0.25])   # non-commuting scalars
BETA = np.array([-1.0, 0.5, 0.0, 1.5])


def check(opA, opB, m, n, k, layout, seed, kind="normal", alpha=ALPHA, beta=BETA):
    A, B, C = make_case(opA, opB, m, n, k, layout, seed, kind)
    ref = oracle_full(opA, opB, m, n, k, alpha, A, B, beta, C, layout)
    got = gpu_run(opA, opB, m, n, k, alpha, A, B, beta, C, layout)
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    if kind == "int":
        assert np.array_equal(g, r), "small-integer result not bit-exact"
    else:
        err = rel_fro(g, r)
        assert err <= TOL, "relative Frobenius error %.3e" % err
    assert np.all(np.isnan(padding(got, m, layout))), "padding rows written"


def test_fp64_256_cubed_parity():
    """FP64, op N,N, m=n=k=256, alpha=1, beta=0, N(0,1), interleaved."""
    m = n = k = 256
    A = qsynth.normal(m, k, 1903)
    B = qsynth.normal(k, n, 1904)
    C = qsynth.empty(m, n)
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    ref = oracle_full("N", "N", m, n, k, one, A, B, zero, C, "interleaved")
    got = gpu_run("N", "N", m, n, k, one, A, B, zero, C, "interleaved")
    err = rel_fro(got, ref)
    print("256^3 rel_fro = %.3e" % err)
    assert err <= TOL


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("opA", OPS)
@pytest.mark.parametrize("opB", OPS)
def test_op_pairs_ragged(opA, opB, layout):
    """Every op pair and layout on a ragged shape spanning several tiles."""
    check(opA, opB, 70, 45, 37, layout, seed=11 + 4 * OPS.index(opA) + OPS.index(opB))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("opA", OPS)
@pytest.mark.parametrize("opB", OPS)
def test_op_pairs_small_int_exact(opA, opB, layout):
    check(opA, opB, 40, 33, 50, layout, seed=200 + 4 * OPS.index(opA) + OPS.index(opB),
          kind="int", alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0, 1.0, -1.0]))


@pytest.mark.parametrize("mnk", [(1, 1, 1), (7, 9, 8), (8, 8, 8), (9, 7, 1), (63, 65, 17),
                                 (65, 1, 63), (1, 40, 255), (33, 100, 2)])
@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_edge_sizes(mnk, layout):
    m, n, k = mnk
    for opA, opB in (("N", "N"), ("T", "H"), ("H", "C")):
        check(opA, opB, m, n, k, layout, seed=m * 1000 + n * 10 + k)


def test_beta_zero_does_not_read_c():
    m, n, k = 50, 40, 30
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 5)
    C[:] = np.nan
    got = gpu_run("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), C, "interleaved")
    assert not np.any(np.isnan(qsynth.components(got, m, "interleaved")))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_k_zero_and_alpha_zero_scale_c(layout):
    m, n, k = 21, 13, 9
    A, B, C = make_case("N", "N", m, n, k, layout, 6)
    for kk, al in ((0, ALPHA), (k, np.zeros(4))):
        ref = oracle_full("N", "N", m, n, kk, al, A, B, BETA, C, layout)
        got = gpu_run("N", "N", m, n, kk, al, A, B, BETA, C, layout)
        assert rel_fro(qsynth.components(got, m, layout), qsynth.components(ref, m, layout)) <= TOL


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_unaligned_operands_use_plain_loads(layout):
    """Operands whose base is 8 bytes off a 16-byte boundary (and odd ld for
    planes) cannot use TMA; the plain-load path must give the same result."""
    m, n, k = 37, 29, 41
    opA, opB = "T", "N"
    A, B, C = make_case(opA, opB, m, n, k, layout, 9, pad=(0, 1, 2))
    ref = oracle_full(opA, opB, m, n, k, ALPHA, A, B, BETA, C, layout)

    def shifted(X):
        buf = torch.zeros(X.size + 1, dtype=torch.float64, device="cuda")
        view = buf[1:].view(*X.shape)
        view.copy_(torch.from_numpy(X))
        return buf, view

    (_, dA), (_, dB) = shifted(A), shifted(B)
    dC = to_dev(C)
    assert dA.data_ptr() % 16 == 8
    ops.qgemm(opA, opB, m, n, k, ALPHA, dA, dB, BETA, dC, layout=layout)
    got = dC.cpu().numpy()
    assert rel_fro(qsynth.components(got, m, layout), qsynth.components(ref, m, layout)) <= TOL


def test_guard_band_around_c():
    """C inside a larger NaN buffer: nothing outside the m x n window changes."""
    m, n, k, ldc = 33, 17, 20, 40
    A, B, _ = make_case("N", "H", m, n, k, "interleaved", 12)
    buf = torch.full((n + 2, ldc, 4), float("nan"), dtype=torch.float64, device="cuda")
    C0 = qsynth.normal(m, n, 99, ld=ldc)
    buf[1:n + 1].copy_(torch.from_numpy(C0))
    ref = oracle_full("N", "H", m, n, k, ALPHA, A, B, BETA, C0, "interleaved")
    dA, dB = to_dev(A), to_dev(B)
    view = buf[1:n + 1]
    rc = _abi.lib().qgemm(0, 3, m, n, k, _abi.q4(ALPHA), dA.data_ptr(), A.shape[1], 0,
                          dB.data_ptr(), B.shape[1], 0, _abi.q4(BETA), view.data_ptr(), ldc, 0,
                          0, 0, None, 0, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    out = buf.cpu().numpy()
    assert np.all(np.isnan(out[0])) and np.all(np.isnan(out[n + 1]))
    assert np.all(np.isnan(out[1:n + 1, m:, :]))
    assert rel_fro(qsynth.components(out[1:n + 1], m, "interleaved"),
                   qsynth.components(ref, m, "interleaved")) <= TOL


def test_bounded_wait_reports_timeout_and_context_survives():
    L = _abi.lib()
    assert L.qgemm_get_last_device_error() == 0
    assert L.qgemm_debug_unsatisfied_wait(20_000_000, None) == 0   # 20 ms limit
    assert L.qgemm_get_last_device_error() == _abi.ERR_TIMEOUT
    assert L.qgemm_get_last_device_error() == 0                     # read clears it
    check("N", "N", 16, 16, 16, "interleaved", 77)                  # still usable


@pytest.mark.parametrize("stage", [0, 2])
def test_gemm_abort_path_reports_timeout_and_context_survives(stage):
    """A fault armed in the FP64 GEMM: the TMA producer of the first CTA
    leaves out the copies of one ring stage, so the consumers' bounded wait
    (20 ms) gives up.  The CTA drains its own copies in flight and stops; the
    launch reports QGEMM_ERR_TIMEOUT through the device status word and the
    next call on the same context computes the right product."""
    L = _abi.lib()
    assert L.qgemm_get_last_device_error() == 0
    m, n, k = 32, 32, 64                      # one CTA, four k-blocks
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 81)
    assert L.qgemm_debug_arm_fault(0, stage, 20_000_000) == 0
    gpu_run("N", "N", m, n, k, ALPHA, A, B, BETA, C, "interleaved")  # launch succeeds
    assert L.qgemm_get_last_device_error() == _abi.ERR_TIMEOUT
    assert L.qgemm_get_last_device_error() == 0
    check("N", "N", m, n, k, "interleaved", 81)


def _sampled_check(opA, opB, n, layout, seed, nrand=384):
    """m = n = k = n: sampled entries (2 full rows, 2 full columns, random
    entries) by exact oracle dot products, plus 2 Freivalds probes."""
    m = k = n
    alpha, beta = qsynth.unit_quaternion(seed), qsynth.unit_quaternion(seed + 1)
    A, B, C = make_case(opA, opB, m, n, k, layout, seed, pad=(0, 0, 0))
    got = gpu_run(opA, opB, m, n, k, alpha, A, B, beta, C, layout)
    g = qsynth.rng(seed + 5)
    rows = np.concatenate([np.repeat(g.integers(0, m, 2), n), np.tile(np.arange(m), 2),
                           g.integers(0, m, nrand)])
    cols = np.concatenate([np.tile(np.arange(n), 2), np.repeat(g.integers(0, n, 2), m),
                           g.integers(0, n, nrand)])
    ref = orc.qgemm_entries(opA, opB, m, n, k, alpha, A, B, beta, C, rows, cols, layout=layout)
    G = qsynth.components(got, m, layout)
    err = rel_fro(G[rows, cols], ref)
    assert err <= TOL, "sampled relative error %.3e" % err
    # Freivalds: C_out v == alpha op(A) (op(B) v) + beta C_in v, v random quaternion vectors
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    for p in range(2):
        v = qsynth.normal(n, 1, seed + 10 + p, layout)
        Bv = oracle_full(opB, "N", k, 1, n, one, B, v, zero, qsynth.empty(k, 1, layout), layout)
        ABv = oracle_full(opA, "N", m, 1, k, alpha, A, Bv, zero, qsynth.empty(m, 1, layout), layout)
        Cv = oracle_full("N", "N", m, 1, n, beta, C, v, one, ABv, layout)
        Gv = oracle_full("N", "N", m, 1, n, one, got, v, zero, qsynth.empty(m, 1, layout), layout)
        assert rel_fro(qsynth.components(Gv, m, layout), qsynth.components(Cv, m, layout)) <= 1e-11
    return err


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_sampled_1024_all_ops(layout):
    for i, (opA, opB) in enumerate([(a, b) for a in OPS for b in OPS]):
        _sampled_check(opA, opB, 1024, layout, 3000 + i, nrand=128)


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_sampled_2048_all_ops(layout):
    """m = n = k = 2048, every op pair: sampled entries and Freivalds probes."""
    for i, (opA, opB) in enumerate([(a, b) for a in OPS for b in OPS]):
        _sampled_check(opA, opB, 2048, layout, 3100 + i, nrand=128)


def test_sampled_4096_planes():
    """m = n = k = 4096 in the split-plane layout (op N,N)."""
    err = _sampled_check("N", "N", 4096, "planes", 1915)
    print("4096 planes sampled rel err %.3e" % err)


@pytest.mark.parametrize("opA,opB", [("H", "T"), ("C", "N")])
def test_sampled_4096_other_ops(opA, opB):
    """m = n = k = 4096 with transposed and conjugated operands."""
    err = _sampled_check(opA, opB, 4096, "interleaved", 1917 + OPS.index(opA))
    print("4096 %s,%s sampled rel err %.3e" % (opA, opB, err))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_sampled_8192(layout):
    """m = n = k = 8192 (op N,N), the largest square of the sweep: sampled
    entries and Freivalds probes (about 16 s on the DMMA path)."""
    err = _sampled_check("N", "N", 8192, layout, 1921, nrand=256)
    print("8192 %s sampled rel err %.3e" % (layout, err))


def test_sampled_4096_bench_config():
    """The benchmarked launch: m=n=k=4096, op N,N, interleaved, unit alpha/beta."""
    err = _sampled_check("N", "N", 4096, "interleaved", 1905)
    print("4096 sampled rel err %.3e" % err)
