"""FP64 path with K split across CTAs (products whose C is too small to fill
the GPU and whose k is long), against the FP64 oracle through the C ABI.

Bar as for the unsplit path: small-integer inputs bit-exact (every partial
sum is an integer below 2^53, so any summation order is exact), N(0,1)
inputs within 1e-12 relative Frobenius error, padding rows untouched, C not
read when beta == 0.  The split is deterministic: the partial products are
summed in a fixed order."""
import numpy as np
import pytest
import torch

import qsynth
from paper_1903_05575_gb300 import _abi, ops
from tests.gpu_util import make_case, oracle_full, padding, rel_fro, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-12
ALPHA = np.array([0.5, -1.0, 2.0, 0.25])   # non-commuting scalars
BETA = np.array([-1.0, 0.5, 0.0, 1.5])
SHAPES = [(64, 64, 20000), (37, 29, 3000), (130, 70, 4000), (1, 1, 10000), (16, 8, 5000)]
OP_PAIRS = [("N", "N"), ("H", "N"), ("T", "C"), ("C", "H")]


def run_abi(opA, opB, m, n, k, alpha, dA, dB, beta, dC, layout, ws_bytes):
    """qgemm through the C ABI with a workspace of ws_bytes (None: NULL)."""
    L = _abi.lib()
    lda, psA, _ = ops.geometry(dA, layout)
    ldb, psB, _ = ops.geometry(dB, layout)
    ldc, psC, _ = ops.geometry(dC, layout)
    ws = None
    if ws_bytes:
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dC.device)
    rc = L.qgemm(_abi.OP[opA], _abi.OP[opB], m, n, k, _abi.q4(alpha), dA.data_ptr(), lda, psA,
                 dB.data_ptr(), ldb, psB, _abi.q4(beta), dC.data_ptr(), ldc, psC,
                 _abi.LAYOUT[layout], _abi.PRECISION["fp64"],
                 ws.data_ptr() if ws is not None else None, ws_bytes or 0,
                 torch.cuda.current_stream().cuda_stream)
    _abi.check(rc, "qgemm")
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def workspace_for(opA, opB, m, n, k, layout):
    return _abi.lib().qgemm_workspace_bytes(_abi.OP[opA], _abi.OP[opB], m, n, k,
                                            _abi.LAYOUT[layout], _abi.PRECISION["fp64"])


def check(opA, opB, m, n, k, layout, seed, kind="normal", alpha=ALPHA, beta=BETA, ws_scale=1.0):
    A, B, C = make_case(opA, opB, m, n, k, layout, seed, kind)
    ref = oracle_full(opA, opB, m, n, k, alpha, A, B, beta, C, layout)
    need = workspace_for(opA, opB, m, n, k, layout)
    assert need > 0, "this shape should split K"
    got = run_abi(opA, opB, m, n, k, alpha, to_dev(A), to_dev(B), beta, to_dev(C), layout,
                  int(need * ws_scale))
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    if kind == "int":
        assert np.array_equal(g, r), "small-integer result not bit-exact"
    else:
        err = rel_fro(g, r)
        assert err <= TOL, "relative Frobenius error %.3e" % err
    assert np.all(np.isnan(padding(got, m, layout))), "padding rows written"
    return got


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("ops_", OP_PAIRS)
def test_splitk_parity(ops_, shape, layout):
    m, n, k = shape
    check(ops_[0], ops_[1], m, n, k, layout, seed=m + 7 * n + k % 1000)


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("ops_", OP_PAIRS)
def test_splitk_small_int_exact(ops_, layout):
    check(ops_[0], ops_[1], 37, 29, 3000, layout, seed=5100, kind="int",
          alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0, 1.0, -1.0]))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_splitk_beta_zero_does_not_read_c(layout):
    m, n, k = 64, 64, 20000
    A, B, _ = make_case("N", "N", m, n, k, layout, 5200)
    C = qsynth.empty(m, n, layout, ld=m + 3)            # NaN everywhere
    ref = oracle_full("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), qsynth.empty(m, n, layout,
                      ld=m + 3, pad=0.0), layout)
    got = run_abi("N", "N", m, n, k, ALPHA, to_dev(A), to_dev(B), np.zeros(4), to_dev(C),
                  layout, workspace_for("N", "N", m, n, k, layout))
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    assert np.all(np.isfinite(g))
    assert rel_fro(g, r) <= TOL


@pytest.mark.parametrize("ws_scale", [0.0, 0.5])
def test_unsplit_or_fewer_shares_with_smaller_workspace(ws_scale):
    """No workspace runs K unsplit; half the workspace runs fewer shares."""
    check("H", "N", 64, 64, 20000, "interleaved", seed=5300, ws_scale=ws_scale)


def test_splitk_deterministic():
    m, n, k = 37, 29, 3000
    A, B, C = make_case("N", "H", m, n, k, "interleaved", 5400)
    need = workspace_for("N", "H", m, n, k, "interleaved")
    dA, dB = to_dev(A), to_dev(B)
    r1 = run_abi("N", "H", m, n, k, ALPHA, dA, dB, BETA, to_dev(C), "interleaved", need)
    r2 = run_abi("N", "H", m, n, k, ALPHA, dA, dB, BETA, to_dev(C), "interleaved", need)
    assert np.array_equal(r1, r2, equal_nan=True)


def test_splitk_through_python_api():
    """ops.qgemm asks for the workspace and passes it: the split runs there."""
    m, n, k = 130, 70, 4000
    A, B, C = make_case("N", "N", m, n, k, "planes", 5500)
    ref = oracle_full("N", "N", m, n, k, ALPHA, A, B, BETA, C, "planes")
    dC = to_dev(C)
    ops.qgemm("N", "N", m, n, k, ALPHA, to_dev(A), to_dev(B), BETA, dC, layout="planes")
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    assert rel_fro(qsynth.components(got, m, "planes"),
                   qsynth.components(ref, m, "planes")) <= TOL


def test_split_runs_faster_than_unsplit():
    """The split really runs: C of 4 x 4 tiles and k = 65536 leaves 16 CTAs
    busy unsplit; with the workspace the shares fill the GPU (measured about
    10x faster; the bar here is 3x)."""
    m, n, k = 64, 64, 65536
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)
    A = torch.randn((k, m, 4), dtype=torch.float64, device="cuda", generator=gen)
    B = torch.randn((n, k, 4), dtype=torch.float64, device="cuda", generator=gen)
    C = torch.zeros((n, m, 4), dtype=torch.float64, device="cuda")
    need = workspace_for("N", "N", m, n, k, "interleaved")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    L = _abi.lib()
    one, zero = _abi.q4([1, 0, 0, 0]), _abi.q4([0, 0, 0, 0])
    stream = torch.cuda.current_stream().cuda_stream

    def timed(w, wb):
        for _ in range(2):
            _abi.check(L.qgemm(0, 0, m, n, k, one, A.data_ptr(), m, 0, B.data_ptr(), k, 0, zero,
                               C.data_ptr(), m, 0, 0, 0, w, wb, stream))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _abi.check(L.qgemm(0, 0, m, n, k, one, A.data_ptr(), m, 0, B.data_ptr(), k, 0, zero,
                           C.data_ptr(), m, 0, 0, 0, w, wb, stream))
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    t_split, t_plain = timed(ws.data_ptr(), need), timed(None, 0)
    print("split %.2f ms, unsplit %.2f ms" % (t_split, t_plain))
    assert t_split * 3 < t_plain


def test_backward_dw_long_batch_splits():
    """dW = X^H dY of a linear layer with a long batch (mb = 20000) and a
    small weight (40 x 24): qgemm_backward's workspace lets the FP64 product
    split its k = mb; dX = dY W^H (20000 x 40) fills the GPU unsplit."""
    mb, k, n = 20000, 40, 24
    L = _abi.lib()
    assert L.qgemm_backward_workspace_bytes(mb, k, n, 0, 0) >= workspace_for("H", "N", k, n, mb,
                                                                             "interleaved") > 0
    Xs = qsynth.normal(mb, k, 5600, pad=0.0)
    Ws = qsynth.normal(k, n, 5601, pad=0.0)
    dYs = qsynth.normal(mb, n, 5602, pad=0.0)
    X, W, dY = to_dev(Xs), to_dev(Ws), to_dev(dYs)
    dX, dW = torch.empty_like(X), torch.empty_like(W)
    ops.qgemm_backward(X, W, dY, mb, k, n, dX=dX, dW=dW)
    torch.cuda.synchronize()
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    refW = qsynth.empty(k, n)
    from oracle import oracle as orc
    orc.qgemm("H", "N", k, n, mb, one, Xs, dYs, zero, refW)
    refX = qsynth.empty(mb, k)
    orc.qgemm("N", "H", mb, k, n, one, dYs, Ws, zero, refX)
    assert rel_fro(dW.cpu().numpy(), refW) <= TOL
    assert rel_fro(dX.cpu().numpy(), refX) <= TOL
