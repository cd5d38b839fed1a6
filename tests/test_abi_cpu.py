"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every entry point declared in include/qgemm.h, and rejects invalid
arguments with LAPACK-style -i codes before touching a device."""
import os
import re

import pytest

from paper_1903_05575_gb300 import _abi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "qgemm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|size_t|const char \*)\s*(qgemm\w*)\s*\(", src,
                                 flags=re.M)))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("qgemm", "qgemm_batched_grouped", "qgemm_backward"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = _abi.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert missing == []
    assert set(declared_functions()) <= set(_abi.SIGNATURES)


def test_plain_c_program_links_and_calls(tmp_path):
    """The boundary is a C ABI: a C99 program that includes qgemm.h (with
    -Wall -Wextra -Werror -pedantic), takes the address of every declared
    entry point, links against the library and calls the ones that need no
    device (version, workspace sizes, argument checks, quick returns)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    lib = _abi.lib_path()
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "qgemm.h"', "",
           "int main(void) {",
           "  void (*fns[])(void) = {"]
    src += ["    (void (*)(void))%s," % n for n in names]
    src += ["  };",
            "  const double one[4] = {1.0, 0.0, 0.0, 0.0};",
            "  double c = 0.0;",
            "  size_t i, live = 0;",
            "  for (i = 0; i < sizeof fns / sizeof fns[0]; ++i) live += fns[i] != NULL;",
            "  /* m = 0: returns before any device call */",
            "  int rc0 = qgemm(QGEMM_OP_N, QGEMM_OP_N, 0, 4, 4, one, NULL, 1, 0, NULL, 4, 0, one,",
            "                  &c, 1, 0, QGEMM_INTERLEAVED, QGEMM_FP64, NULL, 0, NULL);",
            "  /* opA = 7: argument 1 invalid */",
            "  int rc1 = qgemm(7, QGEMM_OP_N, 4, 4, 4, one, NULL, 4, 0, NULL, 4, 0, one,",
            "                  &c, 4, 0, QGEMM_INTERLEAVED, QGEMM_FP64, NULL, 0, NULL);",
            "  size_t ws = qgemm_workspace_bytes(QGEMM_OP_N, QGEMM_OP_N, 64, 64, 64,",
            "                                    QGEMM_INTERLEAVED, QGEMM_FP32_SPLIT_BF16);",
            '  printf("%zu %d %d %zu %s\\n", live, rc0, rc1, ws, qgemm_version());',
            "  return 0;",
            "}"]
    (tmp_path / "abi.c").write_text("\n".join(src) + "\n")
    exe = tmp_path / "abi"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-Wno-cast-function-type", "-I", os.path.dirname(HEADER), str(tmp_path / "abi.c"),
           "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    live, rc0, rc1, ws, version = out.stdout.split(maxsplit=4)
    assert int(live) == len(names)
    assert int(rc0) == 0 and int(rc1) == -1
    assert int(ws) == _abi.lib().qgemm_workspace_bytes(0, 0, 64, 64, 64, 0, 1) > 0
    assert version.strip() == _abi.lib().qgemm_version().decode()


def _call(**kw):
    a = dict(opA=0, opB=0, m=4, n=4, k=4, alpha=_abi.q4([1, 0, 0, 0]), A=64, lda=4, psA=0,
             B=64, ldb=4, psB=0, beta=_abi.q4([0, 0, 0, 0]), C=64, ldc=4, psC=0, layout=0,
             precision=0, ws=None, wsb=0, stream=None)
    a.update(kw)
    return _abi.lib().qgemm(a["opA"], a["opB"], a["m"], a["n"], a["k"], a["alpha"], a["A"],
                            a["lda"], a["psA"], a["B"], a["ldb"], a["psB"], a["beta"], a["C"],
                            a["ldc"], a["psC"], a["layout"], a["precision"], a["ws"], a["wsb"],
                            a["stream"])


@pytest.mark.parametrize("kw,code", [
    (dict(opA=4), -1), (dict(opB=-1), -2), (dict(m=-1), -3), (dict(n=-2), -4), (dict(k=-1), -5),
    (dict(alpha=None), -6), (dict(A=None), -7), (dict(lda=3), -8), (dict(B=None), -10),
    (dict(ldb=0), -11), (dict(beta=None), -13), (dict(C=None), -14), (dict(ldc=2), -15),
    (dict(layout=2), -17), (dict(precision=7), -18),
    (dict(layout=1, psA=15, psB=16, psC=16), -9), (dict(layout=1, psA=16, psB=3, psC=16), -12),
    (dict(layout=1, psA=16, psB=16, psC=0), -16),
    (dict(A=68), -7),              # FP64 element misaligned
    (dict(opA=1, m=6, lda=4, ldc=6), 0),  # op T: stored A is k x m, lda >= k = 4 is fine ...
    (dict(opA=0, m=6, lda=4, ldc=6), -8),  # ... op N: lda >= m = 6 is not
])
def test_argument_checks(kw, code):
    rc = _call(**kw)
    if code == 0:
        assert rc in (0, _abi.ERR_NO_DEVICE)
    else:
        assert rc == code


def test_quick_returns_need_no_device():
    assert _call(m=0, A=None, B=None, C=None) == 0
    assert _call(n=0, A=None, B=None, C=None) == 0


def test_alpha_zero_does_not_reference_operands():
    # alpha == 0: A and B are not read, so NULL is accepted (C <- beta C)
    rc = _call(alpha=_abi.q4([0, 0, 0, 0]), A=None, B=None)
    assert rc in (0, _abi.ERR_NO_DEVICE)


def test_split_precision_needs_workspace():
    L = _abi.lib()
    need = L.qgemm_workspace_bytes(0, 0, 64, 64, 64, 0, 1)
    if need == 0:
        pytest.skip("split path needs no workspace")
    assert _call(precision=1, m=64, n=64, k=64, lda=64, ldb=64, ldc=64) == -19
    assert _call(precision=1, m=64, n=64, k=64, lda=64, ldb=64, ldc=64, ws=256,
                 wsb=need - 1) == -20


def test_fp64_split_k_workspace():
    """FP64 needs no workspace, but reports the one that lets it split K: for
    C of fewer than 8 waves of 16 x 16 quaternion tiles (2 CTAs per SM, 152
    SMs without a device), the fewest shares s in [2, min(256, k-blocks / 8)]
    whose busy fraction (CTAs over whole waves) is within 2 % of the best, if
    the best gains 5 % over s = 1; s partial products of 32 bytes per
    quaternion; 0 when nothing is split.  The Hermitian update counts only
    the tiles that meet its triangle."""
    L = _abi.lib()

    def expect(m, n, k, sms=152, tri=False):
        tiles = -(-m // 16) * -(-n // 16)
        if tri:                      # tiles meeting the triangle of a square C
            t = -(-n // 16)
            tiles = t * (t + 1) // 2
        slots = 2 * sms
        if tiles >= 8 * slots:
            return 0

        def busy(s):
            return tiles * s / (-(-tiles * s // slots) * slots)
        shares = range(2, min(256, (-(-k // 16)) // 8) + 1)
        top = max([busy(1)] + [busy(s) for s in shares])
        if top < busy(1) + 0.05:
            return 0
        return min(s for s in shares if busy(s) >= top - 0.02) * m * n * 32
    for (m, n, k) in ((64, 64, 20000), (37, 29, 3000), (300, 300, 4096), (16, 16, 100),
                      (4096, 4096, 4096), (1, 1, 10000), (400, 390, 50000), (256, 256, 65536),
                      (128, 128, 131072)):
        assert L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 0) == expect(m, n, k), (m, n, k)
    assert L.qgemm_workspace_bytes(0, 0, 64, 64, 20000, 0, 0) > 0
    assert L.qgemm_workspace_bytes(0, 0, 256, 256, 65536, 0, 0) > 0
    for (n, k) in ((64, 20000), (200, 50000), (1000, 4096), (30, 100)):
        for uplo in (0, 1):
            assert L.qherk_workspace_bytes(uplo, 0, n, k, 0, 0) == expect(n, n, k, tri=True)
    assert L.qherk_workspace_bytes(0, 0, 64, 20000, 0, 0) > 0
    # the FP64 call itself never asks for it: no -19 / -20 without a workspace
    assert _call(m=64, n=64, k=20000, lda=64, ldb=20000, ldc=64, A=64, B=64,
                 C=64) in (0, _abi.ERR_NO_DEVICE)


def _tc_shares(m, n, k, bm, bnq, min_kb, sms=152, kb_quat=8):
    """K shares of a tensor-core path: tiles of bm x bnq quaternions, one
    CTA per SM, k-blocks of kb_quat quaternion k (8: 32 reals), at least
    min_kb per share; split only when at most half the SMs are busy
    unsplit."""
    tiles = -(-m // bm) * -(-n // bnq)
    if tiles >= 8 * sms:
        return 1

    def busy(s):
        return tiles * s / (-(-tiles * s // sms) * sms)
    if busy(1) > 0.5:
        return 1
    shares = range(2, min(256, (-(-k // kb_quat)) // min_kb) + 1)
    top = max([busy(1)] + [busy(s) for s in shares])
    if top < busy(1) + 0.05:
        return 1
    return min(s for s in shares if busy(s) >= top - 0.02)


def test_tensor_core_split_k_workspace():
    """Split-BF16 and digit-sliced paths: beyond the required operand
    workspace, qgemm_workspace_bytes reports s partial products (16 bytes
    per quaternion for the FP32 split path after the required part rounded
    to 256 bytes, 32 bytes for the FP64 digit-sliced path).  The split path's
    operands are 3 BF16 terms x 4 component planes of each factor, kappa
    pitch rounded up to 8; its shares count stages of 16 quaternion k, at
    least 32 per share."""
    L = _abi.lib()
    for (m, n, k) in ((64, 64, 65536), (37, 29, 8000), (200, 130, 6000), (1024, 1024, 8192)):
        kp = -(-k // 8) * 8
        a_bytes = 3 * 4 * m * kp * 2
        req = -(-a_bytes // 1024) * 1024 + 3 * 4 * n * kp * 2
        ks = _tc_shares(m, n, k, 128, 64, 32, kb_quat=16)
        want = req if ks == 1 else -(-req // 256) * 256 + ks * m * n * 16
        assert L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 1) == want, (m, n, k)
    for (m, n, k) in ((64, 64, 20000), (37, 29, 3000), (130, 70, 4000), (1024, 1024, 4096)):
        kp = -(-4 * k // 32) * 32
        slices = 6 * 2 * kp * (m + 4 * n)
        got = L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 2)
        ks = _tc_shares(m, n, k, 128, 16, 32)
        extra = ks * m * n * 32 if ks > 1 else 0
        assert slices <= got - extra <= slices + 8 * (m + n) + 8 * k + 8 * 1024, (m, n, k)
    assert _tc_shares(1024, 1024, 8192, 128, 64, 32, kb_quat=16) == 1   # 128 tiles: not split
    assert _tc_shares(64, 64, 65536, 128, 64, 32, kb_quat=16) > 1


def test_sliced_precision_workspace():
    """FP64 digit-sliced path: six BF16 slices of A' (m x 4k) and of the
    expanded B' (4n x 4k), K padded to 32 reals, plus per-row, per-column and
    per-kappa exponent maxima and the exponents used; it needs a workspace,
    and precision 3 is invalid."""
    L = _abi.lib()
    m, n, k = 100, 30, 50
    need = L.qgemm_workspace_bytes(0, 0, m, n, k, 0, 2)
    kp = (4 * k + 31) // 32 * 32
    slices = 6 * 2 * kp * (m + 4 * n)
    assert slices <= need <= slices + 8 * (m + n) + 8 * k + 8 * 1024
    assert L.qgemm_workspace_bytes(0, 0, m, n, 0, 0, 2) == 0
    assert _call(precision=2, m=m, n=n, k=k, lda=m, ldb=k, ldc=m, A=64, B=64, C=64) == -19
    assert _call(precision=2, m=m, n=n, k=k, lda=m, ldb=k, ldc=m, A=64, B=64, C=64, ws=256,
                 wsb=need - 1) == -20
    assert _call(precision=3) == -18


def test_backward_argument_numbers():
    L = _abi.lib()
    rc = L.qgemm_backward(-1, 4, 4, 64, 4, 0, 64, 4, 0, 64, 4, 0, 64, 4, 0, 64, 4, 0, 0, 0, 0,
                          None, 0, None)
    assert rc == -1
    # dX = dY W^H with a bad ldw (W is k x n, ldw >= k): argument 8
    rc = L.qgemm_backward(4, 6, 5, 64, 4, 0, 64, 5, 0, 64, 4, 0, 64, 4, 0, None, 6, 0, 0, 0, 0,
                          None, 0, None)
    assert rc == -8
    # dW = X^H dY with dW's ld too small (dW is k x n, lddw >= k = 6): argument 17
    rc = L.qgemm_backward(4, 6, 5, 64, 4, 0, 64, 6, 0, 64, 4, 0, None, 4, 0, 64, 5, 0, 0, 0, 0,
                          None, 0, None)
    assert rc == -17


def test_status_strings():
    L = _abi.lib()
    for rc in (0, 1, 2, 3, 4, 5, -3):
        assert len(L.qgemm_status_string(rc)) > 0


def test_grouped_workspace_by_precision():
    """Host-side grouped schedule sizes: the digit-sliced batch needs the
    six-slice operands (A' 6 x m x kp and B' 6 x 4n x kp BF16) on top of its
    descriptors; an unknown precision gives 0 (invalid)."""
    L = _abi.lib()
    arr = (_abi.QgemmProblem * 2)()
    for i, (m, n, k) in enumerate(((100, 30, 50), (20, 200, 7))):
        q = arr[i]
        q.opA = q.opB = 0
        q.m, q.n, q.k = m, n, k
        q.alpha[0] = 1.0
        q.A = q.B = q.C = 64
        q.lda, q.ldb, q.ldc = m, k, m
    sizes = {p: L.qgemm_grouped_workspace_bytes(arr, 2, 0, p) for p in (0, 1, 2, 3)}
    slices = 0
    for (m, n, k) in ((100, 30, 50), (20, 200, 7)):
        kp = (4 * k + 31) // 32 * 32

        def padded(r, c):   # tiles of 128 rows x 16 quaternion columns
            return -(-r // 128) * 128 * (-(-c // 16) * 16)
        if padded(n, m) < padded(m, n):   # computed as (AB)^H = B^H A^H
            m, n = n, m
        slices += 6 * 2 * kp * (m + 4 * n)
    assert sizes[2] >= slices
    assert sizes[0] > 0 and sizes[1] > 0
    assert sizes[3] == 0
