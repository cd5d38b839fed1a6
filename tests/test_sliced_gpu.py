"""Digit-sliced FP64 path (precision "fp64_sliced": FP64 data, products on the
BF16 tensor cores with exact integer digit sums) against the FP64 oracle,
through the C ABI.

Bar: N(0,1) inputs within the FP64 target, 1e-12 relative Frobenius error;
small-integer inputs bit-exact; every entry within the path's stated bound
    |error| <= |alpha|_1 * 4k * 2^(e_i + e_n) * 2^-44 + (beta part, FP64)
with e_i, e_n the exponents of the largest component of row i of op(A) and
column n of op(B) (max < 2^e); rows or columns holding Inf or NaN give NaN."""
import numpy as np
import pytest
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import ops
from tests.gpu_util import make_case, oracle_full, padding, rel_fro, to_dev

pytestmark = pytest.mark.gpu

OPS = ("N", "T", "C", "H")
TOL = 1e-12
ALPHA = qsynth.unit_quaternion(51)
BETA = qsynth.unit_quaternion(52)


def run(opA, opB, m, n, k, alpha, A, B, beta, C, layout):
    dA, dB, dC = to_dev(A), to_dev(B), to_dev(C)
    ops.qgemm(opA, opB, m, n, k, alpha, dA, dB, beta, dC, layout=layout, precision="fp64_sliced")
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def op_abs(op, X, m_op, k_op, layout):
    """|components| of the op-matrix (m_op x k_op x 4) whose stored form is X."""
    rows, cols = qsynth.stored_shape(op, m_op, k_op)
    comp = np.abs(qsynth.components(X, rows, layout)[:, :cols])
    return comp.transpose(1, 0, 2) if op in ("T", "H") else comp


def frexp_exp(x):
    """e with 2^(e-1) <= |x| < 2^e; a very negative number for zero."""
    e = np.frexp(x)[1].astype(np.int64)
    return np.where(x > 0, e, -(1 << 40))


def entry_bound(opA, opB, m, n, k, alpha, A, B, layout):
    """The path's per-entry error bound with its kappa balancing: kappa gets
    t = floor((ka - kb) / 2) from the largest exponents ka of op(A)'s column
    kappa and kb of op(B)'s row kappa (0 when either is zero); row i of op(A)
    then has exponent e_i = max over kappa of e(a_ik) - t_k and column n of
    op(B) e_n = max of e(b_kn) + t_k."""
    a = frexp_exp(op_abs(opA, A, m, k, layout).max(axis=2))        # m x k
    b = frexp_exp(op_abs(opB, B, k, n, layout).max(axis=2))        # k x n
    ka, kb = a.max(axis=0), b.max(axis=1)
    live = (ka > -(1 << 39)) & (kb > -(1 << 39))
    t = np.where(live, np.floor_divide(ka - kb, 2), 0)
    ea = np.where(a > -(1 << 39), a - t[None, :], -(1 << 40)).max(axis=1)
    eb = np.where(b > -(1 << 39), b + t[:, None], -(1 << 40)).max(axis=0)
    ea, eb = np.maximum(ea, -1100), np.maximum(eb, -1100)   # zero rows: any small scale
    scale = np.ldexp(1.0, (ea[:, None] + eb[None, :]).astype(int))
    return np.abs(alpha).sum() * 4 * k * scale * 2.0 ** -44


def check(opA, opB, m, n, k, layout, seed, kind="normal", alpha=ALPHA, beta=BETA, tol=TOL):
    A, B, C = make_case(opA, opB, m, n, k, layout, seed, kind)
    ref = oracle_full(opA, opB, m, n, k, alpha, A, B, beta, C, layout)
    got = run(opA, opB, m, n, k, alpha, A, B, beta, C, layout)
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    if kind == "int":
        assert np.array_equal(g, r), "small-integer result not bit-exact"
    else:
        bound = entry_bound(opA, opB, m, n, k, alpha, A, B, layout)
        c_in = np.abs(qsynth.components(C, m, layout)).sum(axis=2)
        slack = bound + 1e-15 * (np.abs(r).sum(axis=2) + np.abs(beta).sum() * c_in)
        worst = (np.abs(g - r).max(axis=2) / slack).max()
        assert worst <= 1.0, "entry error above the stated bound (x%.2f)" % worst
        if tol is not None:
            err = rel_fro(g, r)
            assert err <= tol, "relative Frobenius error %.3e" % err
    assert np.all(np.isnan(padding(got, m, layout))), "padding rows written"
    return g, r


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("opA", OPS)
@pytest.mark.parametrize("opB", OPS)
def test_op_pairs_ragged(opA, opB, layout):
    """Every op pair and layout: 2 row tiles, 3 column tiles, 4.7 exact
    chunks of 256 real k, all ragged."""
    check(opA, opB, 200, 37, 300, layout, seed=700 + 4 * OPS.index(opA) + OPS.index(opB))


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("ops_pair", [("N", "N"), ("H", "T"), ("C", "H"), ("T", "C")])
def test_small_int_exact(ops_pair, layout):
    opA, opB = ops_pair
    check(opA, opB, 150, 40, 333, layout, seed=800 + OPS.index(opA), kind="int",
          alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0, 1.0, -1.0]))


@pytest.mark.parametrize("mnk", [(1, 1, 1), (7, 9, 8), (16, 16, 8), (17, 15, 9), (129, 17, 64),
                                 (128, 16, 65), (1, 40, 255), (33, 100, 2)])
@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_edge_sizes(mnk, layout):
    m, n, k = mnk
    for opA, opB in (("N", "N"), ("T", "H"), ("H", "C")):
        check(opA, opB, m, n, k, layout, seed=m * 1000 + n * 10 + k)


def test_extreme_digits_long_k():
    """Every component +-(1 - 2^-9) (digits 128 and -64), signs arranged so
    that the real component of every product adds up: the level-0 sums reach
    their largest possible value, 2^22 per 256-k chunk.  The inputs are
    represented exactly, so the result is exact."""
    m, n, k = 130, 20, 2048
    c = 1.0 - 2.0 ** -9
    A = qsynth.empty(m, k)
    B = qsynth.empty(k, n)
    A[:, :m, :] = c
    B[:, :k, :] = c
    A[:, :m, 1:] = -c          # a = c(1, -1, -1, -1): products add up, no cancellation
    C = qsynth.normal(m, n, 9)
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    ref = oracle_full("N", "N", m, n, k, one, A, B, zero, C, "interleaved")
    got = run("N", "N", m, n, k, one, A, B, zero, C, "interleaved")
    err = rel_fro(got[:, :m], ref[:, :m])
    print("extreme digits rel err %.3e" % err)
    assert err <= 1e-15


def componentwise_error(opA, opB, m, n, k, alpha, A, B, beta, C, got, ref, layout):
    """Largest error of an entry relative to the magnitudes that form it,
    |alpha| sum_kappa |a_ik| |b_kn| + |beta| |c_in| (quaternion norms): the
    accuracy of the FP64 product whatever the scales of the rows, columns
    and kappa."""
    na = np.sqrt((op_abs(opA, A, m, k, layout) ** 2).sum(axis=2))
    nb = np.sqrt((op_abs(opB, B, k, n, layout) ** 2).sum(axis=2))
    nc = np.sqrt((qsynth.components(C, m, layout) ** 2).sum(axis=2))
    scale = np.linalg.norm(alpha) * (na @ nb) + np.linalg.norm(beta) * nc
    g, r = qsynth.components(got, m, layout), qsynth.components(ref, m, layout)
    err = np.sqrt(((g - r) ** 2).sum(axis=2))
    return float((err / np.maximum(scale, 1e-300)).max())


def test_wide_range_rows_and_columns():
    """Rows of op(A) and columns of op(B) scaled by 2^u, u in [-40, 40]: the
    per-row and per-column exponents absorb the range; every entry within
    the bound and within 1e-12 of the magnitudes that form it."""
    m, n, k = 140, 50, 400
    g = qsynth.rng(31)
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 33)
    A[:, :m, :] *= np.ldexp(1.0, g.integers(-40, 41, m))[None, :, None]
    B[:, :k, :] *= np.ldexp(1.0, g.integers(-40, 41, n))[:, None, None]
    ref = oracle_full("N", "N", m, n, k, ALPHA, A, B, BETA, C, "interleaved")
    got = run("N", "N", m, n, k, ALPHA, A, B, BETA, C, "interleaved")
    bound = entry_bound("N", "N", m, n, k, ALPHA, A, B, "interleaved")
    gc, rc = qsynth.components(got, m, "interleaved"), qsynth.components(ref, m, "interleaved")
    assert (np.abs(gc - rc).max(axis=2) <= bound + 1e-15 * np.abs(rc).sum(axis=2) + 1e-300).all()
    worst = componentwise_error("N", "N", m, n, k, ALPHA, A, B, BETA, C, got, ref, "interleaved")
    print("wide range: worst componentwise error %.3e" % worst)
    assert worst <= 1e-12


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("opA,opB", [("N", "H"), ("T", "N")])
def test_range_along_k(opA, opB, layout):
    """Components scaled by 2^(u_r + v_c) along both stored indices (the
    scaled inputs of the split-BF16 tests), so the scales vary along kappa
    too: the kappa balancing keeps each row's and column's largest scales
    together, and the result meets the FP64 target, 1e-12 relative
    Frobenius, with every entry within 1e-12 of the magnitudes that form it."""
    m, n, k = 96, 30, 200
    A, B, C = make_case(opA, opB, m, n, k, layout, 61, "scaled")
    g, r = check(opA, opB, m, n, k, layout, seed=61, kind="scaled", tol=TOL)
    got = run(opA, opB, m, n, k, ALPHA, A, B, BETA, C, layout)
    ref = oracle_full(opA, opB, m, n, k, ALPHA, A, B, BETA, C, layout)
    worst = componentwise_error(opA, opB, m, n, k, ALPHA, A, B, BETA, C, got, ref, layout)
    print("range along k: Frobenius %.3e, worst componentwise %.3e" % (rel_fro(g, r), worst))
    assert worst <= 1e-12


def test_kappa_scales_apart():
    """The case the balancing exists for: column kappa of op(A) scaled by 2^s
    and row kappa of op(B) by 2^-s with s in [-60, 60], so each product
    a b keeps its size while the row maxima of op(A) and the column maxima
    of op(B) sit at different kappa; without balancing the small scales
    would lose all their digits."""
    m, n, k = 64, 40, 256
    g = qsynth.rng(71)
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 72)
    s = g.integers(-60, 61, k)
    A[:k, :m, :] *= np.ldexp(1.0, s)[:, None, None]
    B[:n, :k, :] *= np.ldexp(1.0, -s)[None, :, None]
    ref = oracle_full("N", "N", m, n, k, ALPHA, A, B, BETA, C, "interleaved")
    got = run("N", "N", m, n, k, ALPHA, A, B, BETA, C, "interleaved")
    gc, rc = qsynth.components(got, m, "interleaved"), qsynth.components(ref, m, "interleaved")
    err = rel_fro(gc, rc)
    worst = componentwise_error("N", "N", m, n, k, ALPHA, A, B, BETA, C, got, ref, "interleaved")
    print("kappa scales apart: Frobenius %.3e, worst componentwise %.3e" % (err, worst))
    assert err <= TOL and worst <= 1e-12


def test_beta_zero_does_not_read_c():
    m, n, k = 50, 40, 30
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 5)
    ref = oracle_full("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), C, "interleaved")
    C[:, :m] = np.nan
    got = run("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), C, "interleaved")
    assert rel_fro(got[:, :m], ref[:, :m]) <= TOL


def test_non_finite_rows_and_columns():
    """NaN in row 3 of A and Inf in column 5 of B: that row and that column of
    C are NaN, every other entry matches the oracle."""
    m, n, k = 40, 24, 50
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 71)
    A[7, 3, 2] = np.nan       # stored (row 3, col 7), component 2
    B[5, 11, 0] = np.inf      # stored (row 11, col 5)
    got = run("N", "N", m, n, k, ALPHA, A, B, BETA, C, "interleaved")
    g = qsynth.components(got, m, "interleaved")
    assert np.isnan(g[3, :, :]).all()
    assert np.isnan(g[:, 5, :]).all()
    A2, B2 = A.copy(), B.copy()
    A2[7, 3, 2] = 0.0
    B2[5, 11, 0] = 0.0
    ref = qsynth.components(oracle_full("N", "N", m, n, k, ALPHA, A2, B2, BETA, C,
                                        "interleaved"), m, "interleaved")
    mask = np.ones((m, n), bool)
    mask[3, :] = False
    mask[:, 5] = False
    assert rel_fro(g[mask], ref[mask]) <= TOL


def test_alpha_zero_and_k_zero_scale_c():
    m, n, k = 33, 20, 10
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 81)
    for kk, al in ((k, np.zeros(4)), (0, ALPHA)):
        ref = oracle_full("N", "N", m, n, kk, al, A, B, BETA, C, "interleaved")
        got = run("N", "N", m, n, kk, al, A, B, BETA, C, "interleaved")
        assert rel_fro(got[:, :m], ref[:, :m]) <= 1e-15


@pytest.mark.parametrize("uplo", ("L", "U"))
@pytest.mark.parametrize("trans", ("N", "H"))
def test_herk(uplo, trans):
    n, k = 150, 90
    A = qsynth.normal(n if trans == "N" else k, k if trans == "N" else n, 91, ld=None)
    C = qsynth.normal(n, n, 92)
    ref = C.copy()
    orc.qherk(uplo, trans, n, k, 0.75, A, -0.5, ref)
    dA, dC = to_dev(A), to_dev(C)
    ops.qherk(uplo, trans, n, k, 0.75, dA, -0.5, dC, precision="fp64_sliced")
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    assert rel_fro(got, ref) <= TOL


def test_backward():
    """dX = dY W^H and dW = X^H dY through qgemm_backward on the sliced path."""
    mb, k, n = 96, 40, 56
    X = qsynth.normal(mb, k, 101)
    W = qsynth.normal(k, n, 102)
    dY = qsynth.normal(mb, n, 103)
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    rX = oracle_full("N", "H", mb, k, n, one, dY, W, zero, qsynth.empty(mb, k), "interleaved")
    rW = oracle_full("H", "N", k, n, mb, one, X, dY, zero, qsynth.empty(k, n), "interleaved")
    dXt = torch.zeros((k, mb, 4), dtype=torch.float64, device="cuda")
    dWt = torch.zeros((n, k, 4), dtype=torch.float64, device="cuda")
    ops.qgemm_backward(to_dev(X), to_dev(W), to_dev(dY), mb, k, n, dX=dXt, dW=dWt,
                       precision="fp64_sliced")
    torch.cuda.synchronize()
    assert rel_fro(dXt.cpu().numpy(), rX) <= TOL
    assert rel_fro(dWt.cpu().numpy(), rW) <= TOL


def test_2048_sampled_and_status():
    """m = n = k = 2048, op N,N: 256 sampled entries against the oracle."""
    n = 2048
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2048)
    A = torch.randn((n, n, 4), dtype=torch.float64, device="cuda", generator=gen)
    B = torch.randn((n, n, 4), dtype=torch.float64, device="cuda", generator=gen)
    C0 = torch.randn((n, n, 4), dtype=torch.float64, device="cuda", generator=gen)
    C = C0.clone()
    ops.qgemm("N", "N", n, n, n, ALPHA, A, B, BETA, C, precision="fp64_sliced")
    torch.cuda.synchronize()
    g = np.random.default_rng(3)
    rows, cols = g.integers(0, n, 256), g.integers(0, n, 256)
    ref = orc.qgemm_entries("N", "N", n, n, n, ALPHA, A.cpu().numpy(), B.cpu().numpy(), BETA,
                            C0.cpu().numpy(), rows, cols)
    got = qsynth.components(C.cpu().numpy(), n, "interleaved")[rows, cols]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print("2048 sliced sampled rel err %.3e" % err)
    assert err <= TOL
    assert ops.last_device_error() == 0


@pytest.mark.parametrize("scalars", [((2.0, 0, 0, 0), (-0.5, 0, 0, 0)),
                                     ((1.0, 0, 0, 0), (0.25, 1.0, 0, 0)),
                                     ((0.5, 0.5, -0.5, 0.5), (3.0, 0, 0, 0))])
def test_real_and_quaternion_scalars(scalars):
    """Real alpha or beta take the 4-product epilogue, quaternion ones the
    16-product Hamilton form; both against the oracle."""
    al, be = (np.array(x) for x in scalars)
    check("N", "H", 140, 33, 90, "interleaved", seed=901, alpha=al, beta=be)


# ---------------------------------------------------------------- K split ---
def sliced_split_shares(m, n, k, sms):
    """Shares the digit-sliced path splits a single product into (tiles of
    128 x 16 quaternions, one CTA per SM, >= 32 k-blocks of 32 reals each)."""
    tiles = -(-m // 128) * -(-n // 16)
    if tiles >= 8 * sms:
        return 1
    num_kb = -(-4 * k // 32)

    def busy(s):
        return tiles * s / (-(-tiles * s // sms) * sms)
    if busy(1) > 0.5:                # at most half of the SMs busy unsplit
        return 1
    shares = range(2, min(256, num_kb // 32) + 1)
    top = max([busy(1)] + [busy(s) for s in shares])
    if top < busy(1) + 0.05:
        return 1
    return min(s for s in shares if busy(s) >= top - 0.02)


SPLIT_SHAPES = [(64, 64, 20000), (37, 29, 3000), (130, 70, 4000), (1, 1, 10000)]


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
@pytest.mark.parametrize("shape", SPLIT_SHAPES)
@pytest.mark.parametrize("ops_pair", [("N", "N"), ("H", "N"), ("T", "C")])
def test_split_k_parity(ops_pair, shape, layout):
    """Few tiles of C, long k: the K shares' partial products are summed by a
    second kernel; every entry stays within the bound, the Frobenius error
    within 1e-12."""
    m, n, k = shape
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert sliced_split_shares(m, n, k, sms) > 1
    check(ops_pair[0], ops_pair[1], m, n, k, layout, seed=m + n + k % 997)


def test_split_k_small_int_exact():
    check("N", "H", 37, 29, 3000, "interleaved", seed=7100, kind="int",
          alpha=np.array([1.0, -2.0, 0.0, 1.0]), beta=np.array([2.0, 0, 1.0, -1.0]))


def test_split_k_beta_zero_and_non_finite():
    """beta = 0 with NaN in C (not read), a NaN row of A and an Inf column of
    B: that row and column of C are NaN after the shares are summed."""
    m, n, k = 40, 24, 5000
    A, B, C = make_case("N", "N", m, n, k, "interleaved", 7200)
    A2, B2 = A.copy(), B.copy()
    A[7, 3, 2] = np.nan
    B[5, 11, 0] = np.inf
    ref = qsynth.components(oracle_full("N", "N", m, n, k, ALPHA, A2, B2, np.zeros(4), C,
                                        "interleaved"), m, "interleaved")
    C[:, :m] = np.nan
    got = run("N", "N", m, n, k, ALPHA, A, B, np.zeros(4), C, "interleaved")
    g = qsynth.components(got, m, "interleaved")
    assert np.isnan(g[3, :, :]).all() and np.isnan(g[:, 5, :]).all()
    mask = np.ones((m, n), bool)
    mask[3, :] = False
    mask[:, 5] = False
    assert rel_fro(g[mask], ref[mask]) <= TOL


def test_split_k_optional_part_and_speed():
    """The minimum workspace runs K unsplit, the reported one splits it: same
    results within the bound, and the split run much faster (4 tiles of C
    leave 148 SMs idle unsplit)."""
    from paper_1903_05575_gb300 import _abi
    m, n, k = 64, 64, 32768
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ks = sliced_split_shares(m, n, k, sms)
    assert ks > 1
    L = _abi.lib()
    full = L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 2)
    need_min = full - ks * m * n * 32
    gen = torch.Generator(device="cuda")
    gen.manual_seed(73)
    A = torch.randn((k, m, 4), dtype=torch.float64, device="cuda", generator=gen)
    B = torch.randn((n, k, 4), dtype=torch.float64, device="cuda", generator=gen)
    ws = torch.empty(full, dtype=torch.uint8, device="cuda")
    one, zero = _abi.q4([1, 0, 0, 0]), _abi.q4([0, 0, 0, 0])
    stream = torch.cuda.current_stream().cuda_stream
    outs, times = [], []
    for wb in (full, need_min):
        C = torch.zeros((n, m, 4), dtype=torch.float64, device="cuda")

        def call():
            _abi.check(L.qgemm(0, 0, m, n, k, one, A.data_ptr(), m, 0, B.data_ptr(), k, 0,
                               zero, C.data_ptr(), m, 0, 0, 2, ws.data_ptr(), wb, stream))
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        outs.append(C.cpu().numpy())
    assert L.qgemm(0, 0, m, n, k, one, A.data_ptr(), m, 0, B.data_ptr(), k, 0, zero,
                   C.data_ptr(), m, 0, 0, 2, ws.data_ptr(), need_min - 1, stream) == -20
    print("split %.2f ms, unsplit %.2f ms" % tuple(times))
    assert rel_fro(outs[0], outs[1]) <= 1e-13
    assert times[0] * 3 < times[1]
