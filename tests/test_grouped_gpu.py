"""Grouped batches through the C ABI (qgemm_batched_grouped via
GroupedBatch), each problem checked against the FP64 oracle; CUDA-graph
capture and replay of the launch; tile-table handling."""
import ctypes

import numpy as np
import pytest
import torch

import qsynth
from oracle import oracle as orc
from paper_1903_05575_gb300 import GroupedBatch, _abi, ops, set_tile_table
from tests.gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu
OPS = ("N", "T", "C", "H")


def make_batch(specs, layout, dtype=np.float64, seed=0, pad=1):
    """specs: list of (opA, opB, m, n, k).  Returns host problems and device tensors."""
    host, dev = [], []
    for i, (opA, opB, m, n, k) in enumerate(specs):
        s = seed + 7 * i
        ra, ca = qsynth.stored_shape(opA, m, k)
        rb, cb = qsynth.stored_shape(opB, k, n)
        A = qsynth.normal(ra, ca, s, layout, ld=ra + pad)
        B = qsynth.normal(rb, cb, s + 1, layout, ld=rb)
        C = qsynth.normal(m, n, s + 2, layout, ld=m + pad)
        al, be = qsynth.unit_quaternion(s + 3), qsynth.unit_quaternion(s + 4)
        host.append(dict(opA=opA, opB=opB, m=m, n=n, k=k, alpha=al, beta=be, A=A, B=B, C=C))
        tdt = torch.float64 if dtype == np.float64 else torch.float32
        dev.append(dict(opA=opA, opB=opB, m=m, n=n, k=k, alpha=al, beta=be,
                        A=to_dev(A, tdt), B=to_dev(B, tdt), C=to_dev(C, tdt)))
    return host, dev


def check_batch(host, dev, layout, tol, full=True):
    worst = 0.0
    for h, d in zip(host, dev):
        got = d["C"].double().cpu().numpy()
        m, n = h["m"], h["n"]
        if full:
            ref = h["C"].copy()
            orc.qgemm(h["opA"], h["opB"], m, n, h["k"], h["alpha"], h["A"], h["B"], h["beta"],
                      ref, layout=layout)
            err = rel_fro(qsynth.components(got, m, layout), qsynth.components(ref, m, layout))
            pad = got[:, m:, :] if layout == "interleaved" else got[:, :, m:]
            assert np.all(np.isnan(pad))
        else:
            g = qsynth.rng(m * 31 + n)
            rows, cols = g.integers(0, m, 6), g.integers(0, n, 6)
            ref = orc.qgemm_entries(h["opA"], h["opB"], m, n, h["k"], h["alpha"], h["A"], h["B"],
                                    h["beta"], h["C"], rows, cols, layout=layout)
            err = rel_fro(qsynth.components(got, m, layout)[rows, cols], ref)
        worst = max(worst, err)
        assert err <= tol, (h["opA"], h["opB"], m, n, h["k"], err)
    return worst


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_mixed_batch_fp64(layout):
    g = qsynth.rng(5)
    specs = []
    for i in range(60):
        m, n, k = (int(x) for x in g.integers(1, 90, size=3))
        specs.append((OPS[i % 4], OPS[(i // 4) % 4], m, n, k))
    host, dev = make_batch(specs, layout, seed=100)
    b = GroupedBatch(dev, layout=layout)
    b.launch()
    torch.cuda.synchronize()
    check_batch(host, dev, layout, 1e-12)
    assert _abi.lib().qgemm_get_last_device_error() == 0


@pytest.mark.parametrize("table", [[0] * 25, [3] * 25, [1] * 25, [2] * 25])
def test_every_tile_shape(table):
    set_tile_table(table)
    try:
        specs = [("N", "H", 40, 37, 20), ("H", "N", 17, 70, 33), ("T", "C", 64, 16, 5)]
        host, dev = make_batch(specs, "interleaved", seed=200)
        b = GroupedBatch(dev)
        b.launch()
        torch.cuda.synchronize()
        check_batch(host, dev, "interleaved", 1e-12)
    finally:
        set_tile_table(None)


def test_zero_sized_and_scale_only_problems():
    specs = [("N", "N", 20, 30, 0), ("N", "N", 16, 16, 16)]
    host, dev = make_batch(specs, "interleaved", seed=300)
    host[1]["alpha"] = np.zeros(4)
    dev[1]["alpha"] = np.zeros(4)
    b = GroupedBatch(dev)
    b.launch()
    torch.cuda.synchronize()
    check_batch(host, dev, "interleaved", 1e-12)


def test_invalid_problem_reports_index_and_argument():
    specs = [("N", "N", 8, 8, 8), ("N", "N", 8, 8, 8)]
    _, dev = make_batch(specs, "interleaved", seed=400)
    arr = (_abi.QgemmProblem * 2)()
    for i, p in enumerate(dev):
        q = arr[i]
        q.opA = q.opB = 0
        q.m = q.n = q.k = 8
        q.alpha[0] = 1.0
        q.A, q.B, q.C = p["A"].data_ptr(), p["B"].data_ptr(), p["C"].data_ptr()
        q.lda, q.ldb, q.ldc = 9, 8, 9
    arr[1].ldb = 3  # argument 11 of problem 1
    plan = _abi.QgemmGroupedPlan()
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    rc = _abi.lib().qgemm_grouped_prepare(arr, 2, 0, 0, ws.data_ptr(), ws.numel(), None,
                                          ctypes.byref(plan))
    assert rc == -(1000 * 2 + 11)


def test_batch_4096_problems_fp64_sampled():
    """4096 problems, m, n, k iid uniform in [8, 256], ops iid in {N, H}."""
    probs = qsynth.grouped_problems(4096, 1907)
    specs = [(p["opA"], p["opB"], p["m"], p["n"], p["k"]) for p in probs]
    host, dev = make_batch(specs, "interleaved", seed=500, pad=0)
    b = GroupedBatch(dev)
    b.launch()
    torch.cuda.synchronize()
    worst = check_batch(host, dev, "interleaved", 1e-12, full=False)
    print("4096-problem batch fp64 worst sampled rel err %.3e" % worst)


def test_graph_capture_and_replay():
    specs = [("N", "H", 50, 40, 30), ("H", "N", 20, 64, 48), ("N", "N", 33, 33, 33)]
    host, dev = make_batch(specs, "interleaved", seed=600)
    b = GroupedBatch(dev)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    C0 = [d["C"].clone() for d in dev]
    with torch.cuda.graph(g, stream=stream):
        b.launch()
    for rep in range(2):
        # new contents of A and C each replay; pointers are the captured ones
        for i, (h, d) in enumerate(zip(host, dev)):
            h["A"] = h["A"] * (rep + 2.0)
            d["A"].copy_(torch.from_numpy(h["A"]))
            d["C"].copy_(C0[i])
        g.replay()
        torch.cuda.synchronize()
        check_batch(host, dev, "interleaved", 1e-12)


# ------------------------------------------------------ split-BF16 path ---

@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_mixed_batch_split(layout):
    g = qsynth.rng(15)
    specs = []
    for i in range(40):
        m, n, k = (int(x) for x in g.integers(1, 200, size=3))
        specs.append((OPS[i % 4], OPS[(i // 4) % 4], m, n, k))
    host, dev = make_batch(specs, layout, dtype=np.float32, seed=700)
    for h in host:  # the oracle sees exactly the float32 values
        for name in ("A", "B", "C"):
            h[name] = h[name].astype(np.float32).astype(np.float64)
    b = GroupedBatch(dev, layout=layout)
    b.launch()
    torch.cuda.synchronize()
    check_batch(host, dev, layout, 2e-6)
    assert _abi.lib().qgemm_get_last_device_error() == 0


def test_batch_4096_problems_split_sampled_and_graph():
    probs = qsynth.grouped_problems(4096, 1908)
    specs = [(p["opA"], p["opB"], p["m"], p["n"], p["k"]) for p in probs]
    host, dev = make_batch(specs, "interleaved", dtype=np.float32, seed=800, pad=0)
    for h in host:
        for name in ("A", "B", "C"):
            h[name] = h[name].astype(np.float32).astype(np.float64)
    b = GroupedBatch(dev)
    C0 = [d["C"].clone() for d in dev]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, stream=stream):
        b.launch()
    for d, c in zip(dev, C0):
        d["C"].copy_(c)
    gr.replay()
    torch.cuda.synchronize()
    worst = check_batch(host, dev, "interleaved", 2e-6, full=False)
    print("4096-problem batch split worst sampled rel err %.3e" % worst)


def test_split_batch_ragged_all_ops():
    """A split batch of ragged problems over every op pair (some computed
    turned around, some with k below one 16-kappa stage) gives oracle-equal
    results."""
    g = qsynth.rng(25)
    specs = []
    for i in range(24):
        m, n, k = (int(x) for x in g.integers(1, 300, size=3))
        specs.append((OPS[i % 4], OPS[(i // 4) % 4], m, n, k))
    host, dev = make_batch(specs, "interleaved", dtype=np.float32, seed=900)
    for h in host:
        for name in ("A", "B", "C"):
            h[name] = h[name].astype(np.float32).astype(np.float64)
    b = GroupedBatch(dev)
    b.launch()
    torch.cuda.synchronize()
    check_batch(host, dev, "interleaved", 2e-6)


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_split_batch_transposed_orientation(layout):
    """Wide problems (m << n) are computed as (op(B)^H op(A)^H) and written
    back conjugate-transposed; every op pair, against the oracle."""
    specs = [(a, b, 20 + 3 * i, 200 + 5 * i, 30 + i) for i, (a, b) in
             enumerate([(x, y) for x in OPS for y in OPS])]
    host, dev = make_batch(specs, layout, dtype=np.float32, seed=1000)
    for h in host:
        for name in ("A", "B", "C"):
            h[name] = h[name].astype(np.float32).astype(np.float64)
    b = GroupedBatch(dev, layout=layout)
    b.launch()
    torch.cuda.synchronize()
    check_batch(host, dev, layout, 2e-6)


def test_fp64_batch_mixing_tma_and_plain_load_problems():
    """Problems whose operands TMA cannot address (odd leading dimensions in
    the planes layout: plain loads) interleaved with TMA problems in the same
    persistent CTAs: ring slots and barrier phases must stay in step."""
    set_tile_table([3] * 25)
    try:
        host, dev = [], []
        for i in range(40):
            m, n, k = 40 + i, 36 + 2 * i, 20 + 3 * i
            pad_a = 1 if i % 2 else 2   # lda = m + 1 (odd when m even) or m + 2
            layout = "planes"
            A = qsynth.normal(m, k, 1300 + i, layout, ld=m + pad_a + (m % 2 if i % 2 else 0))
            B = qsynth.normal(k, n, 1400 + i, layout, ld=k + (1 - k % 2 if i % 2 else k % 2))
            C = qsynth.normal(m, n, 1500 + i, layout, ld=m + 1)
            al, be = qsynth.unit_quaternion(i), qsynth.unit_quaternion(i + 77)
            host.append(dict(opA="N", opB="N", m=m, n=n, k=k, alpha=al, beta=be, A=A, B=B, C=C))
            dev.append(dict(opA="N", opB="N", m=m, n=n, k=k, alpha=al, beta=be, A=to_dev(A),
                            B=to_dev(B), C=to_dev(C)))
        b = GroupedBatch(dev, layout="planes")
        b.launch()
        torch.cuda.synchronize()
        check_batch(host, dev, "planes", 1e-12)
    finally:
        set_tile_table(None)


# ------------------------------------------------ digit-sliced FP64 batches
@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_sliced_mixed_batch(layout):
    """Every op pair, ragged sizes (row tiles of 128, column tiles of 16,
    several 256-k chunks), both orientations of the (AB)^H = B^H A^H swap."""
    g = qsynth.rng(15)
    specs = []
    for i in range(48):
        m, n, k = (int(x) for x in g.integers(1, 200, size=3))
        if i % 3 == 0:
            m, n = n // 8 + 1, m      # wide problems: computed transposed
        specs.append((OPS[i % 4], OPS[(i // 4) % 4], m, n, k))
    host, dev = make_batch(specs, layout, seed=1100)
    b = GroupedBatch(dev, layout=layout, precision="fp64_sliced")
    b.launch()
    torch.cuda.synchronize()
    worst = check_batch(host, dev, layout, 1e-12)
    print("sliced mixed batch worst rel err %.3e" % worst)
    assert _abi.lib().qgemm_get_last_device_error() == 0


def test_sliced_zero_sized_and_scale_only_problems():
    specs = [("N", "N", 20, 30, 0), ("N", "N", 16, 16, 16), ("H", "N", 0, 5, 7),
             ("N", "H", 33, 17, 300)]
    host, dev = make_batch(specs, "interleaved", seed=1300)
    host[1]["alpha"] = np.zeros(4)
    dev[1]["alpha"] = np.zeros(4)
    b = GroupedBatch(dev, precision="fp64_sliced")
    b.launch()
    torch.cuda.synchronize()
    check_batch(host, dev, "interleaved", 1e-12)


def test_sliced_graph_replay():
    specs = [("N", "H", 150, 40, 300), ("H", "N", 20, 64, 48), ("N", "N", 33, 133, 33)]
    host, dev = make_batch(specs, "interleaved", seed=1600)
    b = GroupedBatch(dev, precision="fp64_sliced")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    C0 = [d["C"].clone() for d in dev]
    with torch.cuda.graph(g, stream=stream):
        b.launch(stream=stream)
    for _ in range(2):
        for d, c0 in zip(dev, C0):
            d["C"].copy_(c0)
        g.replay()
        torch.cuda.synchronize()
        check_batch(host, dev, "interleaved", 1e-12)


def test_batch_4096_problems_sliced_sampled():
    """4096 problems, m, n, k iid uniform in [8, 256], ops iid in {N, H},
    FP64 data on the digit-sliced path."""
    probs = qsynth.grouped_problems(4096, 1907)
    specs = [(p["opA"], p["opB"], p["m"], p["n"], p["k"]) for p in probs]
    host, dev = make_batch(specs, "interleaved", seed=500, pad=0)
    b = GroupedBatch(dev, precision="fp64_sliced")
    b.launch()
    torch.cuda.synchronize()
    worst = check_batch(host, dev, "interleaved", 1e-12, full=False)
    print("4096-problem batch sliced worst sampled rel err %.3e" % worst)
    assert _abi.lib().qgemm_get_last_device_error() == 0
