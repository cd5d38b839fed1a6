"""Square-size sweeps of the quaternion GEMM (the paper measures square
N x N products, Sec. 5), printing one JSON line per case:

  fp64:  m = n = k in --sizes, every (opA, opB) in --ops, both layouts;
         effective TFLOP/s (32 m n k / t), fraction of the measured DMMA
         peak, relative error on sampled entries against an FP64 reference.
  split: m = n = k in --split-sizes, inputs N(0,1) and N(0,1) 2^(u_r + v_c)
         (u, v integers in [-20, 20] per row and column), op N,N; TFLOP/s,
         error, speedup over the FP64 rate at the same size.
  sliced: the digit-sliced FP64 path (FP64 data on the BF16 tensor cores),
         m = n = k in --sliced-sizes, the --ops pairs, both layouts.
  trmm:  qtrmm (left, lower, op N) at --trmm sizes on every precision, with
         its time relative to the GEMM of the same size.
  mixed: qgemm_mixed with complex / real factors at --mixed sizes on the
         tensor-core precisions.
  splitk: FP64 products with a small C and a long k (--splitk m x n x k
         shapes), with and without the workspace that lets K split.

Timing: CUDA events on the launching stream around `reps` calls after
warm-up; inputs of every case are larger than L2 except the smallest FP64
sizes, where the call is run `reps` times on the same data (stated in the
line).  Errors are on sampled entries against bench.sampled_reference, an
FP64 numpy computation of those entries.

  python sweep.py [--sizes 1024,2048,4096] [--ops all|NN]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from bench import sampled_reference  # noqa: E402


def _timed(fn, reps, warm=1):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _sampled_error(opA, opB, n, alpha, beta, A, B, C0, C, layout, count=256, seed=1):
    import qsynth
    g = np.random.default_rng(seed)
    rows, cols = g.integers(0, n, count), g.integers(0, n, count)
    ref = sampled_reference(opA, opB, n, n, n, alpha, A.double().cpu().numpy(),
                            B.double().cpu().numpy(), beta, C0.double().cpu().numpy(), rows, cols,
                            layout=layout)
    got = qsynth.components(C.double().cpu().numpy(), n, layout)[rows, cols]
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def fp64_case(n, opA, opB, layout, peak, reps, precision="fp64"):
    import torch

    import qsynth
    from paper_1903_05575_gb300 import ops
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(n + 17 * "NTCH".index(opA) + "NTCH".index(opB))
    shape = (n, n, 4) if layout == "interleaved" else (4, n, n)
    A = torch.randn(shape, dtype=torch.float64, device=dev, generator=gen)
    B = torch.randn(shape, dtype=torch.float64, device=dev, generator=gen)
    C0 = torch.randn(shape, dtype=torch.float64, device=dev, generator=gen)
    C = C0.clone()
    alpha, beta = qsynth.unit_quaternion(n + 1), qsynth.unit_quaternion(n + 2)
    ms = _timed(lambda: ops.qgemm(opA, opB, n, n, n, alpha, A, B, beta, C, layout=layout,
                                  precision=precision), reps)
    C.copy_(C0)
    ops.qgemm(opA, opB, n, n, n, alpha, A, B, beta, C, layout=layout, precision=precision)
    torch.cuda.synchronize()
    err = _sampled_error(opA, opB, n, alpha, beta, A, B, C0, C, layout)
    tf = 32.0 * n ** 3 / (ms * 1e-3) / 1e12
    return {"path": precision, "n": n, "op": opA + opB, "layout": layout, "ms": ms, "tflops": tf,
            "frac_of_dmma_peak": tf / peak, "rel_err_sampled": err, "tolerance": 1e-12,
            "l2": "inputs %.2f GiB" % (3 * n * n * 32 / 2 ** 30)}


def split_case(n, kind, fp64_tflops, reps):
    import torch

    import qsynth
    from paper_1903_05575_gb300 import ops
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(3 * n + (kind == "scaled"))
    shape = (n, n, 4)

    def scaled(X):
        if kind != "scaled":
            return X
        u = torch.randint(-20, 21, (n,), device=dev, generator=gen).double()
        v = torch.randint(-20, 21, (n,), device=dev, generator=gen).double()
        # interleaved (cols, rows, 4): entry (r, c) scaled by 2^(u_r + v_c)
        return X * torch.pow(2.0, u[None, :, None] + v[:, None, None]).float()
    A = scaled(torch.randn(shape, dtype=torch.float32, device=dev, generator=gen))
    B = scaled(torch.randn(shape, dtype=torch.float32, device=dev, generator=gen))
    C0 = torch.randn(shape, dtype=torch.float32, device=dev, generator=gen)
    C = C0.clone()
    alpha, beta = qsynth.unit_quaternion(n + 3), qsynth.unit_quaternion(n + 4)
    ms = _timed(lambda: ops.qgemm("N", "N", n, n, n, alpha, A, B, beta, C), reps)
    C.copy_(C0)
    ops.qgemm("N", "N", n, n, n, alpha, A, B, beta, C)
    torch.cuda.synchronize()
    err = _sampled_error("N", "N", n, alpha, beta, A, B, C0, C, "interleaved", count=512)
    tf = 32.0 * n ** 3 / (ms * 1e-3) / 1e12
    return {"path": "split_bf16", "n": n, "inputs": kind, "op": "NN", "layout": "interleaved",
            "ms": ms, "tflops": tf, "issued_bf16_tflops": 6 * tf, "rel_err_sampled": err,
            "tolerance": 2e-6, "speedup_vs_fp64": tf / fp64_tflops}


def trmm_case(n, precision, reps):
    """qtrmm side L, lower, op N, m = n: effective TFLOP/s on the triangular
    product's own work (16 n^3: half the GEMM's), its time relative to the
    GEMM of the same size and precision, sampled error against the triangular
    product computed as a GEMM with tri(A) written out."""
    import torch

    import qsynth
    from paper_1903_05575_gb300 import ops
    dev = torch.device("cuda", torch.cuda.current_device())
    dt = torch.float32 if precision == "split_bf16" else torch.float64
    gen = torch.Generator(device=dev)
    gen.manual_seed(5 * n)
    A = torch.randn((n, n, 4), dtype=dt, device=dev, generator=gen)
    B = torch.randn((n, n, 4), dtype=dt, device=dev, generator=gen)
    C = torch.empty((n, n, 4), dtype=dt, device=dev)
    al = qsynth.unit_quaternion(n + 5)
    p = None if precision == "split_bf16" else precision
    tr = _timed(lambda: ops.qtrmm("L", "L", "N", "N", n, n, al, A, B, C, precision=p), reps)
    gm = _timed(lambda: ops.qgemm("N", "N", n, n, n, al, A, B, (0, 0, 0, 0), C, precision=p),
                reps)
    ops.qtrmm("L", "L", "N", "N", n, n, al, A, B, C, precision=p)
    torch.cuda.synchronize()
    g = np.random.default_rng(4)
    rows, cols = g.integers(0, n, 128), g.integers(0, n, 128)
    Ah = A.double().cpu().numpy().copy()
    idx = np.arange(n)
    Ah[idx[:, None] > idx[None, :]] = 0.0  # stored (column, row): keep row >= column
    ref = sampled_reference("N", "N", n, n, n, al, Ah, B.double().cpu().numpy(), np.zeros(4),
                            np.zeros_like(Ah), rows, cols)
    got = qsynth.components(C.double().cpu().numpy(), n, "interleaved")[rows, cols]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"path": "trmm_" + precision, "n": n, "side": "L", "uplo": "L", "op": "N",
            "ms": tr, "gemm_ms": gm, "trmm_over_gemm_time": tr / gm,
            "tflops_trmm_work": 16.0 * n ** 3 / (tr * 1e-3) / 1e12, "rel_err_sampled": err}


def mixed_case(n, precision, types, reps):
    """qgemm_mixed at m = n = k = n, op N,N, alpha = 1, beta = 0: time of the
    mixed product and of the quaternion product on the same precision."""
    import torch

    from paper_1903_05575_gb300 import ops
    dev = torch.device("cuda", torch.cuda.current_device())
    dt = torch.float32 if precision == "split_bf16" else torch.float64
    width = {"H": 4, "C": 2, "R": 1}
    gen = torch.Generator(device=dev)
    gen.manual_seed(7 * n)
    A = torch.randn((n, n, width[types[0]]), dtype=dt, device=dev, generator=gen)
    B = torch.randn((n, n, width[types[1]]), dtype=dt, device=dev, generator=gen)
    C = torch.zeros((n, n, 4), dtype=dt, device=dev)
    p = None if precision == "split_bf16" else precision
    one, zero = (1.0, 0, 0, 0), (0.0, 0, 0, 0)
    ms = _timed(lambda: ops.qgemm_mixed(types[0], types[1], "N", "N", n, n, n, one, A, B, zero,
                                        C, precision=p), reps)
    return {"path": "mixed_" + precision, "types": types, "n": n, "ms": ms,
            "real_flops": {"HH": 32, "HC": 16, "CH": 16, "HR": 8, "RH": 8}.get(types, 0) * n ** 3}


def complex_comparison(n, reps, qgemm_ms=None):
    """The paper's experiment (Sec. 5, Fig. 4) on this GPU: the same product
    through cuBLAS ZGEMM on the 2n x 2n complex representation (Eq. qmat_complex,
    Tab. hc_mat_flops: twice the real work of the quaternion product) and cuBLAS
    DGEMM on the real form
    (4n x 4n) x (4n x n), against this library's FP64 QGEMM.  cuBLAS is only
    the comparison system here."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(n)
    Z1 = torch.randn((2 * n, 2 * n), dtype=torch.complex128, device=dev, generator=gen)
    Z2 = torch.randn((2 * n, 2 * n), dtype=torch.complex128, device=dev, generator=gen)
    Z3 = torch.empty_like(Z1)
    zms = _timed(lambda: torch.matmul(Z1, Z2, out=Z3), reps)
    del Z1, Z2, Z3
    R1 = torch.randn((4 * n, 4 * n), dtype=torch.float64, device=dev, generator=gen)
    R2 = torch.randn((4 * n, n), dtype=torch.float64, device=dev, generator=gen)
    R3 = torch.empty((4 * n, n), dtype=torch.float64, device=dev)
    dms = _timed(lambda: torch.matmul(R1, R2, out=R3), reps)
    del R1, R2, R3
    if qgemm_ms is None:
        from paper_1903_05575_gb300 import ops
        A = torch.randn((n, n, 4), dtype=torch.float64, device=dev, generator=gen)
        B = torch.randn((n, n, 4), dtype=torch.float64, device=dev, generator=gen)
        C = torch.empty((n, n, 4), dtype=torch.float64, device=dev)
        one, zero = (1.0, 0, 0, 0), (0.0, 0, 0, 0)
        qgemm_ms = _timed(lambda: ops.qgemm("N", "N", n, n, n, one, A, B, zero, C), reps)
    q = 32.0 * n ** 3
    return {"path": "comparison", "n": n, "qgemm_fp64_ms": qgemm_ms,
            "zgemm_2n_ms": zms, "dgemm_real_form_ms": dms,
            "qgemm_tflops": q / (qgemm_ms * 1e-3) / 1e12,
            "zgemm_tflops_same_product": q / (zms * 1e-3) / 1e12,
            "dgemm_tflops_same_product": q / (dms * 1e-3) / 1e12,
            "zgemm_over_qgemm_time": zms / qgemm_ms, "dgemm_over_qgemm_time": dms / qgemm_ms,
            "note": "rates count 32 n^3 flops (the quaternion product) for all three"}


def splitk_case(m, n, k, peak, reps):
    """FP64 product with a small C and a long k, run with the workspace that
    lets it split K and without one (unsplit); N(0,1) data, op N,N,
    interleaved, unit-quaternion alpha and beta; error of the split result on
    sampled entries against an FP64 reference."""
    import torch

    import qsynth
    from paper_1903_05575_gb300 import _abi, ops
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(m + 3 * n + k)
    A = torch.randn((k, m, 4), dtype=torch.float64, device=dev, generator=gen)
    B = torch.randn((n, k, 4), dtype=torch.float64, device=dev, generator=gen)
    C0 = torch.randn((n, m, 4), dtype=torch.float64, device=dev, generator=gen)
    C = C0.clone()
    alpha, beta = qsynth.unit_quaternion(m + 5), qsynth.unit_quaternion(n + 6)
    L = _abi.lib()
    need = L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 0)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    def call(w, wb):
        rc = L.qgemm(0, 0, m, n, k, _abi.q4(alpha), A.data_ptr(), m, 0, B.data_ptr(), k, 0,
                     _abi.q4(beta), C.data_ptr(), m, 0, 0, 0, w, wb, stream)
        _abi.check(rc, "qgemm")
    t_split = _timed(lambda: call(ws.data_ptr(), need), reps)
    t_plain = _timed(lambda: call(None, 0), reps)
    C.copy_(C0)
    call(ws.data_ptr(), need)
    torch.cuda.synchronize()
    g = np.random.default_rng(3)
    rows, cols = g.integers(0, m, 128), g.integers(0, n, 128)
    ref = sampled_reference("N", "N", m, n, k, alpha, A.cpu().numpy(), B.cpu().numpy(), beta,
                            C0.cpu().numpy(), rows, cols)
    got = qsynth.components(C.cpu().numpy(), m, "interleaved")[rows, cols]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    flops = 32.0 * m * n * k
    return {"path": "fp64 split K", "m": m, "n": n, "k": k, "op": "NN", "layout": "interleaved",
            "workspace_bytes": need, "ms_split": t_split, "ms_unsplit": t_plain,
            "tflops_split": flops / (t_split * 1e-3) / 1e12,
            "tflops_unsplit": flops / (t_plain * 1e-3) / 1e12,
            "frac_of_dmma_peak_split": flops / (t_split * 1e-3) / 1e12 / peak,
            "speedup": t_plain / t_split, "rel_err_sampled": err, "tolerance": 1e-12}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="1024,2048,4096")
    ap.add_argument("--ops", default="all")
    ap.add_argument("--layouts", default="interleaved,planes")
    ap.add_argument("--split-sizes", default="2048,8192")
    ap.add_argument("--sliced-sizes", default="")
    ap.add_argument("--trmm", default="", help="sizes for the triangular product")
    ap.add_argument("--mixed", default="", help="sizes for the mixed-type products")
    ap.add_argument("--mixed-fp64", default="", help="sizes for the FP64 mixed-type products")
    ap.add_argument("--splitk", default="",
                    help="m x n x k shapes (e.g. 64x64x65536,256x256x65536) for the FP64 K split")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--compare", default="", help="sizes for the cuBLAS ZGEMM/DGEMM comparison")
    a = ap.parse_args()
    from paper_1903_05575_gb300 import ops
    peak = ops.probe_peak(0, 0.4)
    pairs = ([x + y for x in "NTCH" for y in "NTCH"] if a.ops == "all" else a.ops.split(","))
    fp64_rate = {}
    for n in [int(x) for x in a.sizes.split(",") if x]:
        for layout in a.layouts.split(","):
            for op in pairs:
                t0 = time.time()
                rec = fp64_case(n, op[0], op[1], layout, peak, a.reps)
                rec["wall_s"] = time.time() - t0
                fp64_rate[n] = rec["tflops"]
                print(json.dumps(rec), flush=True)
    for n in [int(x) for x in a.sliced_sizes.split(",") if x]:
        for layout in a.layouts.split(","):
            for op in pairs:
                rec = fp64_case(n, op[0], op[1], layout, peak, max(a.reps, 3), "fp64_sliced")
                rec.pop("frac_of_dmma_peak")
                rec["issued_bf16_tflops"] = 21.0 * rec["tflops"]
                rec["speedup_vs_dmma_path"] = rec["tflops"] / fp64_rate.get(n, peak)
                print(json.dumps(rec), flush=True)
    for n in [int(x) for x in a.split_sizes.split(",") if x]:
        base = fp64_rate.get(n, peak)
        for kind in ("normal", "scaled"):
            print(json.dumps(split_case(n, kind, base, max(a.reps, 3))), flush=True)
    for n in [int(x) for x in a.trmm.split(",") if x]:
        for prec in ("fp64", "fp64_sliced", "split_bf16"):
            print(json.dumps(trmm_case(n, prec, 2 if prec == "fp64" else 5)), flush=True)
    for n in [int(x) for x in a.mixed.split(",") if x]:
        for prec in ("fp64_sliced", "split_bf16"):
            for types in ("HH", "HC", "CH", "HR", "RH"):
                print(json.dumps(mixed_case(n, prec, types, 5)), flush=True)
    for n in [int(x) for x in a.mixed_fp64.split(",") if x]:
        for types in ("HH", "HC", "CH", "HR", "RH"):
            print(json.dumps(mixed_case(n, "fp64", types, 2)), flush=True)
    for shape in [x for x in a.splitk.split(",") if x]:
        m, n, k = (int(v) for v in shape.split("x"))
        print(json.dumps(splitk_case(m, n, k, peak, max(a.reps, 3))), flush=True)
    for n in [int(x) for x in a.compare.split(",") if x]:
        print(json.dumps(complex_comparison(n, a.reps)), flush=True)


if __name__ == "__main__":
    main()
