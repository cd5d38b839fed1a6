"""Independent checks used to pin the oracle (test helpers, no GPU).

The complex 2x2 representation of Sec. 2.1 (Eq. h_matrep) and Sec. 2.2
(Eq. qmat_complex) maps a quaternion matrix Q (M x N) to the complex matrix
    Q_C = [[ Q^0 + i Q^1,   Q^2 + i Q^3 ],
           [ -Q^2 + i Q^3,  Q^0 - i Q^1 ]]      (2M x 2N)
and products to products (Eq. hc_mat_mult).  A scalar q acting from the left
is kron(q_C, I_M).  numpy's complex matmul is a different code path from the
oracle's Hamilton loop, so agreement pins the oracle's sign table, operand
order and scalar side.
"""
import numpy as np


def to_complex(Q):
    """(rows, cols, 4) components -> 2rows x 2cols complex representation."""
    Z0 = Q[..., 0] + 1j * Q[..., 1]
    Z1 = Q[..., 2] + 1j * Q[..., 3]
    return np.block([[Z0, Z1], [-np.conj(Z1), np.conj(Z0)]])


def from_complex(Zc, rows, cols):
    Z0 = Zc[:rows, :cols]
    Z1 = Zc[:rows, cols:]
    out = np.empty((rows, cols, 4))
    out[..., 0] = Z0.real
    out[..., 1] = Z0.imag
    out[..., 2] = Z1.real
    out[..., 3] = Z1.imag
    return out


def scalar_complex(q):
    q = np.asarray(q, dtype=np.float64)
    return np.array([[q[0] + 1j * q[1], q[2] + 1j * q[3]],
                     [-q[2] + 1j * q[3], q[0] - 1j * q[1]]])


def apply_op(Q, op):
    """op on a (rows, cols, 4) component array: N, T, C (conjugate) or H."""
    R = Q
    if op in ("T", "H"):
        R = np.transpose(R, (1, 0, 2))
    if op in ("C", "H"):
        R = R * np.array([1.0, -1.0, -1.0, -1.0])
    return np.ascontiguousarray(R)


def qgemm_complex(opA, opB, alpha, A, B, beta, C):
    """alpha op(A) op(B) + beta C through the complex representation.
    A, B, C are STORED component arrays (rows, cols, 4); C may be None."""
    Ao, Bo = apply_op(A, opA), apply_op(B, opB)
    m, n = Ao.shape[0], Bo.shape[1]
    P = to_complex(Ao) @ to_complex(Bo)
    out = np.kron(scalar_complex(alpha), np.eye(m)) @ P
    if C is not None:
        out = out + np.kron(scalar_complex(beta), np.eye(m)) @ to_complex(C)
    return from_complex(out, m, n)


def rel_fro(X, Ref):
    d = np.linalg.norm((X - Ref).ravel())
    r = np.linalg.norm(Ref.ravel())
    return d / r if r > 0 else d
