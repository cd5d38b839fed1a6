"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each pin is independent of the oracle's own code: the basis table and worked
products come from the paper (tests/golden), the complex 2x2 representation
is computed with numpy's complex matmul, and the matrix identities are exact
on small integers.  ``test_pins_catch_planted_mistakes`` compiles copies of
the oracle with a mistake planted in the C source and checks that at least
one pin fails for each.
"""
import os
import shutil
import tempfile

import numpy as np
import pytest

import qsynth
from oracle import oracle as orc
from tests import qref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OPS = ("N", "T", "C", "H")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def _basis(i):
    e = np.zeros(4)
    e[i] = 1.0
    return e


# ----------------------------------------------------------------- pins ---

def pin_basis_table(lib):
    """Eq. quaternion_alg: all 16 basis products, e1 e2 e3 = -e0, e_i e_j = -e_j e_i."""
    for i, j, s, k in _golden("hamilton_table.txt"):
        r = orc.hamilton(_basis(int(i)), _basis(int(j)), lib=lib)
        if not np.array_equal(r, s * _basis(int(k))):
            return False
    e123 = orc.hamilton(orc.hamilton(_basis(1), _basis(2), lib=lib), _basis(3), lib=lib)
    if not np.array_equal(e123, -_basis(0)):
        return False
    for i in (1, 2, 3):
        for j in (1, 2, 3):
            if i != j and not np.array_equal(orc.hamilton(_basis(i), _basis(j), lib=lib),
                                             -orc.hamilton(_basis(j), _basis(i), lib=lib)):
                return False
    return True


def pin_worked_products(lib):
    """Hand-expanded products of Eq. quaternion_prod (tests/golden)."""
    for row in _golden("worked_products.txt"):
        if not np.array_equal(orc.hamilton(row[0:4], row[4:8], lib=lib), row[8:12]):
            return False
    return True


def pin_norm_multiplicative(lib):
    """|pq| = |p||q| (H is a normed division algebra, Eq. quaternion_da)."""
    g = qsynth.rng(11)
    for _ in range(200):
        p, q = g.standard_normal(4), g.standard_normal(4)
        lhs = np.linalg.norm(orc.hamilton(p, q, lib=lib))
        rhs = np.linalg.norm(p) * np.linalg.norm(q)
        if abs(lhs - rhs) > 8e-16 * rhs:
            return False
    return True


def pin_complex_subalgebra(lib):
    """q^2 = q^3 = 0 gives exactly complex multiplication (Eq. h_c_iso)."""
    g = qsynth.rng(12)
    for _ in range(50):
        a, b = g.integers(-9, 10, size=2), g.integers(-9, 10, size=2)
        r = orc.hamilton([a[0], a[1], 0, 0], [b[0], b[1], 0, 0], lib=lib)
        z = complex(a[0], a[1]) * complex(b[0], b[1])
        if not np.array_equal(r, [z.real, z.imag, 0.0, 0.0]):
            return False
    return True


def pin_scalar_complex_rep(lib):
    """(pq)_C = p_C q_C for the 2x2 representation (Eq. h_matrep, Eq. hc_mult)."""
    g = qsynth.rng(13)
    for _ in range(100):
        p, q = g.standard_normal(4), g.standard_normal(4)
        lhs = qref.scalar_complex(orc.hamilton(p, q, lib=lib))
        rhs = qref.scalar_complex(p) @ qref.scalar_complex(q)
        if np.max(np.abs(lhs - rhs)) > 1e-14:
            return False
    return True


def _oracle_run(lib, opA, opB, m, n, k, alpha, A, B, beta, C, layout):
    Cw = C.copy()
    orc.qgemm(opA, opB, m, n, k, alpha, A, B, beta, Cw, layout=layout, lib=lib)
    return Cw


def pin_gemm_vs_complex(lib, exact_only=False):
    """Oracle GEMM == complex-representation GEMM for every op pair and both
    layouts, with non-commuting alpha, beta and ld > rows.  Small integers must
    agree exactly; N(0,1) data to 1e-13 relative Frobenius error."""
    m, n, k = 5, 4, 6
    alpha = np.array([1.0, 2.0, -1.0, 3.0])
    beta = np.array([-2.0, 1.0, 1.0, -1.0])
    seed = 100
    for layout in qsynth.LAYOUTS:
        for opA in OPS:
            for opB in OPS:
                for kind in (("int",) if exact_only else ("int", "normal")):
                    seed += 1
                    ra, ca = qsynth.stored_shape(opA, m, k)
                    rb, cb = qsynth.stored_shape(opB, k, n)
                    make = qsynth.small_int if kind == "int" else qsynth.normal
                    A = make(ra, ca, seed, layout, ld=ra + 2)
                    B = make(rb, cb, seed + 7, layout, ld=rb + 1)
                    C = make(m, n, seed + 13, layout, ld=m + 3)
                    got = _oracle_run(lib, opA, opB, m, n, k, alpha, A, B, beta, C, layout)
                    ref = qref.qgemm_complex(opA, opB, alpha,
                                             qsynth.components(A, ra, layout),
                                             qsynth.components(B, rb, layout), beta,
                                             qsynth.components(C, m, layout))
                    val = qsynth.components(got, m, layout)
                    if kind == "int":
                        if not np.array_equal(val, ref):
                            return False
                    elif qref.rel_fro(val, ref) > 1e-13:
                        return False
                    # padding rows untouched
                    pad = got[:, m:, :] if layout == "interleaved" else got[:, :, m:]
                    if not np.all(np.isnan(pad)):
                        return False
    return True


def pin_conj_transpose_identity(lib):
    """(AB)^H = B^H A^H exactly on small integers; (AB)^T != B^T A^T in general."""
    m, n, k = 4, 3, 5
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    A = qsynth.small_int(m, k, 21)
    B = qsynth.small_int(k, n, 22)
    AB = _oracle_run(lib, "N", "N", m, n, k, one, A, B, zero, qsynth.empty(m, n), "interleaved")
    BhAh = _oracle_run(lib, "H", "H", n, m, k, one, B, A, zero, qsynth.empty(n, m),
                       "interleaved")
    if not np.array_equal(qref.apply_op(qsynth.components(AB, m, "interleaved"), "H"),
                          qsynth.components(BhAh, n, "interleaved")):
        return False
    BtAt = _oracle_run(lib, "T", "T", n, m, k, one, B, A, zero, qsynth.empty(n, m),
                       "interleaved")
    if np.array_equal(qref.apply_op(qsynth.components(AB, m, "interleaved"), "T"),
                      qsynth.components(BtAt, n, "interleaved")):
        return False  # negative control: H is not commutative
    return True


def pin_associative(lib):
    """(AB)C = A(BC) exactly on small integers (H is associative, Sec. 2.1)."""
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    A, B, C = qsynth.small_int(3, 4, 31), qsynth.small_int(4, 2, 32), qsynth.small_int(2, 5, 33)
    AB = _oracle_run(lib, "N", "N", 3, 2, 4, one, A, B, zero, qsynth.empty(3, 2), "interleaved")
    ABC = _oracle_run(lib, "N", "N", 3, 5, 2, one, AB, C, zero, qsynth.empty(3, 5), "interleaved")
    BC = _oracle_run(lib, "N", "N", 4, 5, 2, one, B, C, zero, qsynth.empty(4, 5), "interleaved")
    ABC2 = _oracle_run(lib, "N", "N", 3, 5, 4, one, A, BC, zero, qsynth.empty(3, 5), "interleaved")
    return np.array_equal(ABC, ABC2)


def pin_scalar_side(lib):
    """alpha multiplies from the left: alpha(AB) = (alpha A)B, and differs from
    (AB)alpha for a non-real alpha (Sec. 2.2, Eq. no_scalar_comm_mat)."""
    m, n, k = 3, 3, 4
    alpha = np.array([0.0, 1.0, 2.0, -1.0])
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    A, B = qsynth.small_int(m, k, 41), qsynth.small_int(k, n, 42)
    got = qsynth.components(_oracle_run(lib, "N", "N", m, n, k, alpha, A, B, zero,
                                        qsynth.empty(m, n), "interleaved"), m, "interleaved")
    AB = qsynth.components(_oracle_run(lib, "N", "N", m, n, k, one, A, B, zero,
                                       qsynth.empty(m, n), "interleaved"), m, "interleaved")
    left = np.array([[orc.hamilton(alpha, AB[i, j], lib=lib) for j in range(n)]
                     for i in range(m)])
    right = np.array([[orc.hamilton(AB[i, j], alpha, lib=lib) for j in range(n)]
                      for i in range(m)])
    return np.array_equal(got, left) and not np.array_equal(got, right)


def pin_blas_conventions(lib):
    """beta = 0 never reads C (NaN ignored); k = 0 gives C = beta C;
    m = 0 or n = 0 leaves C untouched (BLAS conventions, paper silent)."""
    alpha = np.array([1.0, -1.0, 2.0, 0.5])
    A, B = qsynth.small_int(3, 2, 51), qsynth.small_int(2, 4, 52)
    Cnan = qsynth.empty(3, 4)  # all NaN
    got = _oracle_run(lib, "N", "N", 3, 4, 2, alpha, A, B, np.zeros(4), Cnan, "interleaved")
    if np.any(np.isnan(qsynth.components(got, 3, "interleaved"))):
        return False
    beta = np.array([0.0, 2.0, 0.0, 1.0])
    C = qsynth.small_int(3, 4, 53)
    got = _oracle_run(lib, "N", "N", 3, 4, 0, alpha, A, B, beta, C, "interleaved")
    Cc = qsynth.components(C, 3, "interleaved")
    want = np.array([[orc.hamilton(beta, Cc[i, j], lib=lib) for j in range(4)]
                     for i in range(3)])
    if not np.array_equal(qsynth.components(got, 3, "interleaved"), want):
        return False
    for (mm, nn) in ((0, 4), (3, 0)):
        got = _oracle_run(lib, "N", "N", mm, nn, 2, alpha, A, B, beta, C, "interleaved")
        if not np.array_equal(got, C):
            return False
    return True


def pin_entries_match_full(lib):
    """The sampled-entry routine equals the full GEMM entry by entry (exact)."""
    m, n, k = 7, 6, 5
    alpha, beta = np.array([1.0, 1, -2, 0]), np.array([0.0, -1, 1, 3])
    for layout in qsynth.LAYOUTS:
        for opA, opB in (("N", "N"), ("T", "H"), ("C", "T")):
            ra, ca = qsynth.stored_shape(opA, m, k)
            rb, cb = qsynth.stored_shape(opB, k, n)
            A = qsynth.small_int(ra, ca, 61, layout, ld=ra + 1)
            B = qsynth.small_int(rb, cb, 62, layout)
            C = qsynth.small_int(m, n, 63, layout, ld=m + 2)
            full = qsynth.components(_oracle_run(lib, opA, opB, m, n, k, alpha, A, B, beta,
                                                 C, layout), m, layout)
            rows, cols = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
            ent = orc.qgemm_entries(opA, opB, m, n, k, alpha, A, B, beta, C, rows.ravel(),
                                    cols.ravel(), layout=layout, lib=lib)
            if not np.array_equal(ent.reshape(m, n, 4), full):
                return False
    return True


def _hermitian_full(T, uplo):
    """Full Hermitian matrix from the uplo triangle of T (n, n, 4) components,
    diagonal vector parts zeroed."""
    n = T.shape[0]
    F = np.zeros_like(T)
    for i in range(n):
        for j in range(n):
            src = (i, j) if (i >= j) == (uplo == "L") or i == j else (j, i)
            v = T[src].copy()
            if src != (i, j):
                v[1:] = -v[1:]
            F[i, j] = v
    for i in range(n):
        F[i, i, 1:] = 0.0
    return F


def pin_herk_vs_complex(lib):
    """Hermitian rank-k update (Sec. 2.2 Hermiticity; rank-k updates of Sec. 3):
    the triangle equals alpha op(A) op(A)^H + beta C computed through the
    complex representation (numpy), exactly on small integers; the other
    triangle is untouched and the diagonal is real."""
    n, k = 5, 4
    for layout in qsynth.LAYOUTS:
        for uplo in ("L", "U"):
            for trans in ("N", "H"):
                ra, ca = (n, k) if trans == "N" else (k, n)
                A = qsynth.small_int(ra, ca, 91, layout, ld=ra + 1)
                C = qsynth.small_int(n, n, 92, layout, ld=n + 2)
                alpha, beta = 3.0, -2.0
                got = C.copy()
                orc.qherk(uplo, trans, n, k, alpha, A, beta, got, layout=layout, lib=lib)
                Ac = qsynth.components(A, ra, layout)
                Cc = qsynth.components(C, n, layout)
                Ao = qref.apply_op(Ac, trans)
                Cf = _hermitian_full(Cc, uplo)
                want = qref.from_complex(alpha * (qref.to_complex(Ao) @ qref.to_complex(Ao).conj().T)
                                         + beta * qref.to_complex(Cf), n, n)
                G = qsynth.components(got, n, layout)
                for i in range(n):
                    for j in range(n):
                        in_tri = (i >= j) if uplo == "L" else (i <= j)
                        if in_tri and not np.array_equal(G[i, j], want[i, j]):
                            return False
                        if not in_tri and not np.array_equal(G[i, j], Cc[i, j]):
                            return False
                    if np.any(G[i, i, 1:] != 0.0):
                        return False
    return True


def _tri_components(Ac, uplo, diag):
    """tri(A) on a (K, K, 4) component array: the uplo triangle, zeros
    elsewhere, the quaternion 1 on the diagonal when diag is "U"."""
    K = Ac.shape[0]
    mask = np.tril(np.ones((K, K), bool)) if uplo == "L" else np.triu(np.ones((K, K), bool))
    T = Ac * mask[:, :, None]
    if diag == "U":
        T[np.arange(K), np.arange(K)] = np.array([1.0, 0.0, 0.0, 0.0])
    return T


def pin_trmm_vs_complex(lib):
    """Triangular product (the BLAS-3 XTRMM built on GEMM, Sec. 3): C equals
    alpha op(tri(A)) B (left) or alpha B op(tri(A)) (right) computed through
    the complex representation (numpy), exactly on small integers, for every
    side, triangle, op and diagonal kind."""
    m, n = 4, 3
    alpha = np.array([2.0, -1.0, 1.0, 3.0])
    for layout in qsynth.LAYOUTS:
        for side in ("L", "R"):
            K = m if side == "L" else n
            A = qsynth.small_int(K, K, 93, layout, ld=K + 1)
            B = qsynth.small_int(m, n, 94, layout, ld=m + 2)
            Ac = qsynth.components(A, K, layout)
            Bc = qsynth.components(B, m, layout)
            for uplo in ("L", "U"):
                for trans in "NTCH":
                    for diag in ("N", "U"):
                        got = qsynth.empty(m, n, layout, ld=m + 1)
                        orc.qtrmm(side, uplo, trans, diag, m, n, alpha, A, B, got,
                                  layout=layout, lib=lib)
                        T = qref.apply_op(_tri_components(Ac, uplo, diag), trans)
                        P = (qref.to_complex(T) @ qref.to_complex(Bc) if side == "L"
                             else qref.to_complex(Bc) @ qref.to_complex(T))
                        want = qref.from_complex(np.kron(qref.scalar_complex(alpha), np.eye(m)) @ P,
                                                 m, n)
                        if not np.array_equal(qsynth.components(got, m, layout), want):
                            return False
    return True


def pin_trmm_transpose_duality(lib):
    """op(tri(A)) with op T is tri of the transposed matrix in the other
    triangle: qtrmm(uplo, T, A) = qtrmm(other uplo, N, A^T stored), and with
    op H the same on the conjugate transpose; a unit triangle of zeros gives
    C = alpha B."""
    m, n = 5, 4
    alpha = np.array([1.0, 2.0, 0.0, -1.0])
    A = qsynth.small_int(m, m, 95)
    B = qsynth.small_int(m, n, 96)
    Ac = qsynth.components(A, m, "interleaved")
    for uplo, other in (("L", "U"), ("U", "L")):
        for trans, flip in (("T", np.array([1.0, 1.0, 1.0, 1.0])),
                            ("H", np.array([1.0, -1.0, -1.0, -1.0]))):
            At = qsynth.empty(m, m)
            At[:, :m, :] = np.transpose(np.transpose(Ac, (1, 0, 2)) * flip, (1, 0, 2))
            x = orc.qtrmm("L", uplo, trans, "N", m, n, alpha, A, B, qsynth.empty(m, n), lib=lib)
            y = orc.qtrmm("L", other, "N", "N", m, n, alpha, At, B, qsynth.empty(m, n), lib=lib)
            if not np.array_equal(x, y):
                return False
    Z = qsynth.empty(m, m, pad=0.0)
    got = orc.qtrmm("L", "L", "N", "U", m, n, alpha, Z, B, qsynth.empty(m, n), lib=lib)
    Bc = qsynth.components(B, m, "interleaved")
    want = np.array([[orc.hamilton(alpha, Bc[i, j], lib=lib) for j in range(n)] for i in range(m)])
    return np.array_equal(qsynth.components(got, m, "interleaved"), want)


def _mixed_case(typeA, typeB, opA, opB, m, n, k, layout, seed, alpha, beta, lib):
    ra, ca = qsynth.stored_shape(opA, m, k)
    rb, cb = qsynth.stored_shape(opB, k, n)
    A = qsynth.typed(ra, ca, seed, typeA, layout, ld=ra + 1, kind="int")
    B = qsynth.typed(rb, cb, seed + 1, typeB, layout, ld=rb + 2, kind="int")
    C = qsynth.small_int(m, n, seed + 2, layout, ld=m + 1)
    got = C.copy()
    orc.qgemm_mixed(typeA, typeB, opA, opB, m, n, k, alpha, A, B, beta, got, layout=layout,
                    lib=lib)
    Ao = qref.apply_op(qsynth.typed_components(A, ra, typeA, layout), opA)
    Bo = qref.apply_op(qsynth.typed_components(B, rb, typeB, layout), opB)
    return Ao, Bo, qsynth.components(C, m, layout), qsynth.components(got, m, layout)


def pin_mixed_cayley_dickson(lib):
    """Mixed-type products (quaternion-complex and quaternion-real, Sec. 5)
    through a route that never forms a Hamilton product: with
    q = z1 + z2 e2 (z1 = q^0 + q^1 e1, z2 = q^2 + q^3 e1) and w complex,
    q w = z1 w + z2 conj(w) e2 and w q = w z1 + w z2 e2 (numpy complex
    matmuls); a real factor scales every component.  Exact on small integers,
    alpha = 1, beta = 0, every op, both layouts."""
    one, zero = np.array([1.0, 0, 0, 0]), np.zeros(4)
    m, n, k = 3, 4, 5

    def cd(Q):
        return Q[..., 0] + 1j * Q[..., 1], Q[..., 2] + 1j * Q[..., 3]

    for layout in qsynth.LAYOUTS:
        for opA in "NTCH":
            for opB in "NTCH":
                for tA, tB in (("H", "C"), ("C", "H"), ("C", "C"), ("H", "R"), ("R", "H"),
                               ("R", "C")):
                    Ao, Bo, _, G = _mixed_case(tA, tB, opA, opB, m, n, k, layout, 97, one, zero,
                                               lib)
                    z1, z2 = cd(Ao)
                    w1, w2 = cd(Bo)
                    want = np.zeros((m, n, 4))
                    if tB != "H":          # right factor complex (or real): q w
                        p1, p2 = z1 @ w1, z2 @ np.conj(w1)
                    else:                  # left factor complex (or real): w q
                        p1, p2 = z1 @ w1, z1 @ w2
                    want[..., 0], want[..., 1] = p1.real, p1.imag
                    want[..., 2], want[..., 3] = p2.real, p2.imag
                    if not np.array_equal(G, want):
                        return False
    return True


def pin_mixed_scalars(lib):
    """alpha, beta on the left of a mixed product: equal to the complex
    2x2 representation of alpha (op(A) op(B)) + beta C, exactly."""
    alpha, beta = np.array([1.0, -2.0, 1.0, 3.0]), np.array([2.0, 0.0, -1.0, 1.0])
    for tA, tB in (("H", "C"), ("R", "H")):
        Ao, Bo, Cc, G = _mixed_case(tA, tB, "H", "N", 4, 3, 5, "planes", 98, alpha, beta, lib)
        m, n = 4, 3
        P = qref.to_complex(Ao) @ qref.to_complex(Bo)
        want = qref.from_complex(np.kron(qref.scalar_complex(alpha), np.eye(m)) @ P
                                 + np.kron(qref.scalar_complex(beta), np.eye(m))
                                 @ qref.to_complex(Cc), m, n)
        if not np.array_equal(G, want):
            return False
    return True


PINS = [pin_basis_table, pin_worked_products, pin_norm_multiplicative, pin_complex_subalgebra,
        pin_scalar_complex_rep, pin_gemm_vs_complex, pin_conj_transpose_identity,
        pin_associative, pin_scalar_side, pin_blas_conventions, pin_entries_match_full,
        pin_herk_vs_complex, pin_trmm_vs_complex, pin_trmm_transpose_duality,
        pin_mixed_cayley_dickson, pin_mixed_scalars]


def failing_pins(lib, pins=PINS):
    bad = []
    for p in pins:
        try:
            ok = p(lib)
        except Exception:
            ok = False
        if not ok:
            bad.append(p.__name__)
    return bad


# ---------------------------------------------------------------- tests ---

@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    assert pin(orc._load()), pin.__doc__


def test_gemm_vs_complex_larger():
    """A larger case spanning several of the GPU's tile sizes, N(0,1) data."""
    m, n, k = 70, 33, 65
    alpha, beta = qsynth.unit_quaternion(1), qsynth.unit_quaternion(2)
    for opA, opB in (("N", "N"), ("H", "T")):
        ra, ca = qsynth.stored_shape(opA, m, k)
        rb, cb = qsynth.stored_shape(opB, k, n)
        A, B = qsynth.normal(ra, ca, 71), qsynth.normal(rb, cb, 72)
        C = qsynth.normal(m, n, 73)
        got = C.copy()
        orc.qgemm(opA, opB, m, n, k, alpha, A, B, beta, got)
        ref = qref.qgemm_complex(opA, opB, alpha, qsynth.components(A, ra, "interleaved"),
                                 qsynth.components(B, rb, "interleaved"), beta,
                                 qsynth.components(C, m, "interleaved"))
        assert qref.rel_fro(qsynth.components(got, m, "interleaved"), ref) < 1e-14


# Plausible mistakes, planted textually in a copy of the oracle's C source.
MUTATIONS = {
    "levi_civita_sign": ("return 1;\n    return -1;", "return -1;\n    return 1;"),
    "scalar_part_sign": ("s -= p[i] * q[i];", "s += p[i] * q[i];"),
    "dropped_cross_term": ("if (e) v += (double)e * p[i] * q[j];", "if (e > 0) v += p[i] * q[j];"),
    "no_conjugate": ("    q[1] = -q[1];\n    q[2] = -q[2];\n    q[3] = -q[3];", "    (void)q;"),
    "transpose_ignored": ("if (op == ORACLE_OP_T || op == ORACLE_OP_H)\n        load_stored(X, ld, ps, layout, c, r, q);",
                          "if (op == ORACLE_OP_H)\n        load_stored(X, ld, ps, layout, c, r, q);"),
    "alpha_on_right": ("oracle_hamilton(alpha, P, aP);", "oracle_hamilton(P, alpha, aP);"),
    "operands_swapped": ("oracle_hamilton(a, b, ab);\n                    double *p",
                         "oracle_hamilton(b, a, ab);\n                    double *p"),
    "beta_read_when_zero": ("const int read_c = !is_zero(beta);\n#ifdef _OPENMP\n    if (nthreads > 0) omp_set_num_threads(nthreads);\n#else\n    (void)nthreads;\n#endif\n    int status",
                            "const int read_c = 1;\n#ifdef _OPENMP\n    if (nthreads > 0) omp_set_num_threads(nthreads);\n#else\n    (void)nthreads;\n#endif\n    int status"),
    "herk_no_conjugate": ("conjugate(b);\n                oracle_hamilton(a, b, ab);",
                          "oracle_hamilton(a, b, ab);"),
    "herk_diag_not_real": ("if (i == j) out[1] = out[2] = out[3] = 0.0;", "(void)0;"),
    "herk_operands_swapped": ("load_op(A, lda, psA, layout, trans, i, kap, a);\n                load_op(A, lda, psA, layout, trans, j, kap, b);",
                              "load_op(A, lda, psA, layout, trans, j, kap, a);\n                load_op(A, lda, psA, layout, trans, i, kap, b);"),
    "trmm_triangle_flipped": ("const int in_triangle = uplo == 0 ? r >= c : r <= c;",
                              "const int in_triangle = uplo == 0 ? r <= c : r >= c;"),
    "trmm_unit_diag_ignored": ("    if (diag && r == c) {\n        q[0] = 1.0;",
                               "    if (0 && r == c) {\n        q[0] = 1.0;"),
    "trmm_transpose_before_mask": ("        load_tri(A, lda, psA, layout, uplo, diag, c, r, q);",
                                   "        load_stored(A, lda, psA, layout, c, r, q);"),
    "trmm_right_side_order": ("                    load_stored(B, ldb, psB, layout, i, kap, a);\n                    load_op_tri(A, lda, psA, layout, uplo, diag, trans, kap, j, b);",
                              "                    load_stored(B, ldb, psB, layout, i, kap, b);\n                    load_op_tri(A, lda, psA, layout, uplo, diag, trans, kap, j, a);"),
    "mixed_complex_width": ("const int w = type == 0 ? 4 : (type == 1 ? 2 : 1);",
                            "const int w = type == 0 ? 4 : (type == 1 ? 1 : 1);"),
    "mixed_no_conjugate": ("        load_typed(X, ld, ps, layout, type, r, c, q);\n    if (op == ORACLE_OP_C || op == ORACLE_OP_H) conjugate(q);",
                           "        load_typed(X, ld, ps, layout, type, r, c, q);\n    if (op == ORACLE_OP_C) conjugate(q);"),
    "mixed_planes_interleaved": ("X[w * (r + c * ld) + s] : X[s * ps + r + c * ld]",
                                 "X[4 * (r + c * ld) + s] : X[s * ps + r + c * ld]"),
    "plane_stride_wrong": ("q[0] = e[0]; q[1] = e[ps]; q[2] = e[2 * ps]; q[3] = e[3 * ps];",
                           "q[0] = e[0]; q[1] = e[ps]; q[2] = e[3 * ps]; q[3] = e[2 * ps];"),
}


def test_pins_catch_planted_mistakes():
    src = open(orc._SRC).read()
    assert failing_pins(orc._load()) == []
    tmp = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        for name, (old, new) in MUTATIONS.items():
            assert src.count(old) == 1, name
            path = os.path.join(tmp, name + ".c")
            with open(path, "w") as f:
                f.write(src.replace(old, new))
            lib = orc.load_variant(orc.build(force=True, src=path,
                                             out=os.path.join(tmp, name + ".so")))
            assert failing_pins(lib), "planted mistake %r not caught by any pin" % name
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
