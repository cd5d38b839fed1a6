"""Split-BF16 path (tcgen05) against the FP64 oracle, through the C ABI.

Inputs are float32; the oracle computes in FP64 on the same float32 values.
Bar: relative Frobenius error <= 2e-6 for N(0,1) and for the wide-range
(2^(u_r + v_c)) inputs; small integers (exactly representable, partial sums
below 2^24) bit-exact; padding rows untouched."""
import numpy as np
import pytest
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import _abi, ops
from tests.gpu_util import gpu_run, make_case, oracle_full, padding, rel_fro, to_dev

pytestmark = pytest.mark.gpu

OPS = ("N", "T", "C", "H")
TOL = 2e-6
ALPHA = np.array([0.5, -1.0, 2.0, 0.25])
BETA = np.array([-1.0, 0.5, 0.0, 1.5])


def check(opA, opB, m, n, k, layout, seed, kind="normal", alpha=ALPHA, beta=BETA, tol=TOL):
    A, B, C = make_case(opA, opB, m, n, k, layout, seed, kind, dtype=np.float32)
    ref = oracle_full(opA, opB, m, n, k, alpha, A, B, beta, C, layout)
    got = gpu_run(opA, opB, m, n, k, alpha, A, B, beta, C, layout, dtype=torch.float32)
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    if kind == "int":
        bad = np.argwhere(g != r)
        assert bad.size == 0, "not bit-exact at %d entries, first %s: got %s want %s" % (
            len(bad), bad[:4].tolist(), g[tuple(bad[0])], r[tuple(bad[0])])
        err = 0.0
    else:
        err = rel_fro(g, r)
        assert err <= tol, "relative Frobenius error %.3e" % err
    assert np.all(np.isnan(padding(got, m, layout))), "padding rows written"
    return err


def test_small_int_exact_one_tile():
    check("N", "N", 128, 64, 8, "interleaved", 1, kind="int",
          alpha=np.array([1.0, 0, 0, 0]), beta=np.zeros(4))


def test_normal_one_tile():
    check("N", "N", 128, 64, 40, "interleaved", 2)


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("opA", OPS)
@pytest.mark.parametrize("opB", OPS)
def test_op_pairs_ragged(opA, opB, layout):
    check(opA, opB, 150, 70, 45, layout, seed=31 + 4 * OPS.index(opA) + OPS.index(opB))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("T", "H"), ("C", "T"), ("H", "C")])
def test_small_int_exact(opA, opB, layout):
    check(opA, opB, 200, 90, 77, layout, seed=400 + OPS.index(opA), kind="int",
          alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0, 1.0, -1.0]))


@pytest.mark.parametrize("mnk", [(1, 1, 1), (7, 9, 8), (129, 65, 9), (1, 100, 300), (257, 3, 17)])
def test_edge_sizes(mnk):
    m, n, k = mnk
    for layout in qsynth.LAYOUTS:
        check("N", "H", m, n, k, layout, seed=m + 7 * n + 13 * k)


def test_beta_zero_does_not_read_c():
    m, n, k = 130, 66, 30
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 5, dtype=np.float32)
    C[:] = np.nan
    got = gpu_run("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), C, "interleaved",
                  dtype=torch.float32)
    assert not np.any(np.isnan(qsynth.components(got, m, "interleaved")))


def test_wide_range_inputs():
    """Components N(0,1) * 2^(u_r + v_c), u, v in [-20, 20] per row and column."""
    err = check("N", "N", 256, 128, 256, "interleaved", 8, kind="scaled")
    print("wide-range rel err %.3e" % err)


def test_workspace_checks():
    L = _abi.lib()
    m = n = k = 64
    need = L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 1)
    assert need > 0
    A = torch.zeros((k, m, 4), dtype=torch.float32, device="cuda")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    rc = L.qgemm(0, 0, m, n, k, _abi.q4([1, 0, 0, 0]), A.data_ptr(), m, 0, A.data_ptr(), k, 0,
                 _abi.q4([0, 0, 0, 0]), A.data_ptr(), m, 0, 0, 1, ws.data_ptr(), need - 1, None)
    assert rc == -20


def _sampled(n, kind, seed, layout="interleaved", opA="N", opB="N"):
    m = k = n
    alpha, beta = qsynth.unit_quaternion(seed), qsynth.unit_quaternion(seed + 1)
    A, B, C = make_case(opA, opB, m, n, k, layout, seed, kind, pad=(0, 0, 0), dtype=np.float32)
    got = gpu_run(opA, opB, m, n, k, alpha, A, B, beta, C, layout, dtype=torch.float32)
    g = qsynth.rng(seed + 3)
    rows = np.concatenate([np.repeat(g.integers(0, m, 2), n), g.integers(0, m, 2048)])
    cols = np.concatenate([np.tile(np.arange(n), 2), g.integers(0, n, 2048)])
    ref = orc.qgemm_entries(opA, opB, m, n, k, alpha, A, B, beta, C, rows, cols, layout=layout)
    return rel_fro(qsynth.components(got, m, layout)[rows, cols], ref)


@pytest.mark.parametrize("kind", ["normal", "scaled"])
def test_sampled_2048(kind):
    err = _sampled(2048, kind, 2100)
    print("2048 %s sampled rel err %.3e" % (kind, err))
    assert err <= TOL


@pytest.mark.parametrize("kind", ["normal", "scaled"])
def test_sampled_8192(kind):
    err = _sampled(8192, kind, 8200)
    print("8192 %s sampled rel err %.3e" % (kind, err))
    assert err <= TOL


SCALARS = {
    "one": np.array([1.0, 0.0, 0.0, 0.0]),
    "real": np.array([-1.75, 0.0, 0.0, 0.0]),
    "complex": np.array([0.5, -1.25, 0.0, 0.0]),
    "quaternion": np.array([0.5, -1.0, 2.0, 0.25]),
    "zero": np.zeros(4),
}


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("alpha", ["one", "real", "complex", "quaternion"])
@pytest.mark.parametrize("beta", ["zero", "real", "quaternion"])
def test_scalar_kinds(alpha, beta, layout):
    """alpha is applied to op(A) by the pre-pass (not at all when it is 1,
    componentwise when real, as a left Hamilton product otherwise) and beta
    C by the epilogue (skipped, real or quaternion): every combination on a
    ragged shape with conjugated operands against the oracle."""
    check("C", "T", 150, 70, 45, layout, seed=1200 + len(alpha) + 7 * len(beta),
          alpha=SCALARS[alpha], beta=SCALARS[beta])


@pytest.mark.parametrize("ncols", [1, 15, 16, 17, 33, 48, 63, 64, 65, 80])
def test_column_tile_widths(ncols):
    """The MMA width follows the last column tile (16-column granules up to
    64): every width on both sides of a granule edge."""
    check("N", "N", 130, ncols, 40, "interleaved", seed=1300 + ncols)


# ---------------------------------------------------------------- K split ---
def split_shares(m, n, k, sms):
    """Shares the split-BF16 path splits a single product into (tiles of 128
    x 64 quaternions, one CTA per SM, >= 32 stages of 16 quaternion k)."""
    tiles = -(-m // 128) * -(-n // 64)
    if tiles >= 8 * sms:
        return 1
    num_kb = -(-k // 16)

    def busy(s):
        return tiles * s / (-(-tiles * s // sms) * sms)
    if busy(1) > 0.5:                # at most half of the SMs busy unsplit
        return 1
    shares = range(2, min(256, num_kb // 32) + 1)
    top = max([busy(1)] + [busy(s) for s in shares])
    if top < busy(1) + 0.05:
        return 1
    return min(s for s in shares if busy(s) >= top - 0.02)


SPLIT_SHAPES = [(64, 64, 20000), (37, 29, 8000), (200, 130, 6000), (1, 1, 10000)]


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("shape", SPLIT_SHAPES)
@pytest.mark.parametrize("ops_", [("N", "N"), ("H", "N"), ("T", "C")])
def test_split_k_parity(ops_, shape, layout):
    """Few tiles of C, long k: K shares' FP32 products summed in FP64 by a
    second kernel, then alpha and beta; 2e-6 as unsplit."""
    m, n, k = shape
    assert split_shares(m, n, k, torch.cuda.get_device_properties(0).multi_processor_count) > 1
    check(ops_[0], ops_[1], m, n, k, layout, seed=m + n + k % 991)


def test_split_k_small_int_exact():
    check("N", "H", 37, 29, 8000, "interleaved", seed=8100, kind="int",
          alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0, 1.0, -1.0]))


def test_split_k_beta_zero_does_not_read_c():
    m, n, k = 64, 64, 20000
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 8200, dtype=np.float32)
    ref = oracle_full("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), C, "interleaved")
    C[:, :m] = np.nan
    got = gpu_run("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), C, "interleaved",
                  dtype=torch.float32)
    assert rel_fro(got[:, :m], ref[:, :m]) <= TOL


def test_split_k_optional_part_and_speed():
    """The minimum workspace runs K unsplit, the reported one splits it: both
    results within 2e-6 of the oracle, and the split run much faster (one
    tile of C leaves 151 SMs idle unsplit)."""
    m, n, k = 64, 64, 65536
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ks = split_shares(m, n, k, sms)
    assert ks > 1
    L = _abi.lib()
    full = L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 1)
    need_min = full - ks * m * n * 16
    gen = torch.Generator(device="cuda")
    gen.manual_seed(83)
    A = torch.randn((k, m, 4), dtype=torch.float32, device="cuda", generator=gen)
    B = torch.randn((n, k, 4), dtype=torch.float32, device="cuda", generator=gen)
    ws = torch.empty(full, dtype=torch.uint8, device="cuda")
    one, zero = _abi.q4([1, 0, 0, 0]), _abi.q4([0, 0, 0, 0])
    stream = torch.cuda.current_stream().cuda_stream
    outs, times = [], []
    for wb in (full, need_min):
        C = torch.zeros((n, m, 4), dtype=torch.float32, device="cuda")

        def call():
            _abi.check(L.qgemm(0, 0, m, n, k, one, A.data_ptr(), m, 0, B.data_ptr(), k, 0,
                               zero, C.data_ptr(), m, 0, 0, 1, ws.data_ptr(), wb, stream))
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        outs.append(C.double().cpu().numpy())
    print("split %.2f ms, unsplit %.2f ms" % tuple(times))
    ref = qsynth.empty(m, n, pad=0.0)
    orc.qgemm("N", "N", m, n, k, np.array([1.0, 0, 0, 0]), A.double().cpu().numpy(),
              B.double().cpu().numpy(), np.zeros(4), ref)
    for out in outs:                 # each within the bar of the exact product
        assert rel_fro(out, ref) <= TOL
    assert times[0] * 3 < times[1]


def test_two_unordered_streams_use_separate_workspaces():
    """Two qgemm calls on two streams with no ordering between them: each
    stream gets its own cached workspace, so both results equal the same
    products computed one after the other on one stream."""
    m, n, k = 300, 200, 700
    gen = torch.Generator(device="cuda")
    gen.manual_seed(91)
    A = [torch.randn((k, m, 4), dtype=torch.float32, device="cuda", generator=gen)
         for _ in range(2)]
    B = [torch.randn((n, k, 4), dtype=torch.float32, device="cuda", generator=gen)
         for _ in range(2)]
    C0 = torch.randn((n, m, 4), dtype=torch.float32, device="cuda", generator=gen)
    ref = [C0.clone() for _ in range(2)]
    for i in range(2):
        ops.qgemm("N", "N", m, n, k, ALPHA, A[i], B[i], BETA, ref[i])
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    out = [C0.clone() for _ in range(2)]
    torch.cuda.synchronize()
    for rep in range(3):
        for i in range(2):
            out[i].copy_(C0)
        torch.cuda.synchronize()
        for i in range(2):
            with torch.cuda.stream(streams[i]):
                ops.qgemm("N", "N", m, n, k, ALPHA, A[i], B[i], BETA, out[i])
        torch.cuda.synchronize()
        for i in range(2):
            assert torch.equal(out[i], ref[i]), "stream %d, repetition %d" % (i, rep)


@pytest.mark.parametrize("stage", [0, 3])
def test_gemm_abort_path_reports_timeout_and_context_survives(stage):
    """A fault armed in the split-BF16 GEMM: its TMA warp leaves out the
    copies of one ring stage, so the MMA warp's bounded wait (20 ms) gives
    up.  Every role of the CTA stops (the abort flag ends the other waits),
    the copies in flight land, all issued MMAs complete, tensor memory is
    released, and the launch reports QGEMM_ERR_TIMEOUT; the next call on the
    same context computes the right product."""
    L = _abi.lib()
    assert L.qgemm_get_last_device_error() == 0
    m, n, k = 100, 40, 80                      # one tile, five 16-kappa stages
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 82, dtype=np.float32)
    assert L.qgemm_debug_arm_fault(1, stage, 20_000_000) == 0
    gpu_run("N", "N", m, n, k, ALPHA, A, B, BETA, C, "interleaved", dtype=torch.float32)
    assert L.qgemm_get_last_device_error() == _abi.ERR_TIMEOUT
    assert L.qgemm_get_last_device_error() == 0
    check("N", "N", m, n, k, "interleaved", 82)


def test_arm_fault_argument_checks():
    L = _abi.lib()
    assert L.qgemm_debug_arm_fault(2, 0, 20_000_000) == -1
    assert L.qgemm_debug_arm_fault(1, -1, 20_000_000) == -2
    assert L.qgemm_debug_arm_fault(1, 0, 10) == -3
