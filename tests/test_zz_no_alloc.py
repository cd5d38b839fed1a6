"""The fixed-scratch split-BF16 entry point, qgemm_split_noalloc.

It exists for callers that cannot allocate device memory at the call: code
whose device memory all belongs to another allocator (a framework's pool, a
fixed arena), or a plain C caller that has no allocator of its own.  It must give the same result as qgemm() with
a caller workspace.  This file sorts last so that a run stopping at the first
failure has run everything else; it also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

import qsynth
from paper_1903_05575_gb300 import _abi, ops
from tests.gpu_util import make_case, rel_fro, to_dev

pytestmark = pytest.mark.gpu
TOL = 2e-6   # the split-BF16 tolerance of the other tests


def _noalloc(opA, opB, m, n, k, alpha, A, B, beta, C, layout):
    lda, psA, _ = ops.geometry(A, layout)
    ldb, psB, _ = ops.geometry(B, layout)
    ldc, psC, _ = ops.geometry(C, layout)
    return _abi.lib().qgemm_split_noalloc(
        _abi.OP[opA], _abi.OP[opB], m, n, k, _abi.q4(alpha), A.data_ptr(), lda, psA,
        B.data_ptr(), ldb, psB, _abi.q4(beta), C.data_ptr(), ldc, psC, _abi.LAYOUT[layout],
        torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("layout", qsynth.LAYOUTS)
def test_noalloc_matches_workspace_entry_point_twice(layout):
    """Two calls in a row (different shapes, so stale scratch contents from the
    first call would show in the second), each against qgemm()."""
    cases = [("N", "H", 300, 260, 200, 11), ("T", "N", 130, 70, 45, 12),
             # one tile of C, long k: K shares whose partial products sit in
             # the scratch after the split operands
             ("N", "N", 64, 64, 8192, 13)]
    for opA, opB, m, n, k, seed in cases:
        alpha, beta = qsynth.unit_quaternion(seed), qsynth.unit_quaternion(seed + 1)
        A, B, C = make_case(opA, opB, m, n, k, layout, seed, dtype=np.float32)
        dA, dB = to_dev(A, torch.float32), to_dev(B, torch.float32)
        ref = to_dev(C, torch.float32)
        ops.qgemm(opA, opB, m, n, k, alpha, dA, dB, beta, ref, layout=layout)
        got = to_dev(C, torch.float32)
        assert _noalloc(opA, opB, m, n, k, alpha, dA, dB, beta, got, layout) == 0
        torch.cuda.synchronize()
        g = qsynth.components(got.double().cpu().numpy(), m, layout)
        r = qsynth.components(ref.double().cpu().numpy(), m, layout)
        assert rel_fro(g, r) <= TOL
    assert _abi.lib().qgemm_get_last_device_error() == 0


def test_noalloc_rejects_problems_beyond_the_scratch():
    L = _abi.lib()
    n = 1181  # smallest square size whose split operands exceed the scratch
    assert L.qgemm_workspace_bytes(0, 0, n, n, n, 0, 1) > _abi.NOALLOC_SCRATCH_BYTES
    X = torch.zeros((n, n, 4), dtype=torch.float32, device="cuda")
    before = X.clone()
    rc = _noalloc("N", "N", n, n, n, [1, 0, 0, 0], X, X, [0, 0, 0, 0], X, "interleaved")
    assert rc == _abi.ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.equal(X, before)
