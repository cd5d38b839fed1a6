/*
 * Plain FP64 CPU oracle for quaternion GEMM.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library never calls it, and it shares no code, header or table with the
 * CUDA path.
 *
 * What it computes (the plain definition, no blocking, no reordering):
 *
 *   C <- alpha * op(A) * op(B) + beta * C                (Sec. 3.1, Eq. general_gemm)
 *
 * over the quaternions H, where
 *   - a quaternion is q = q^0 e0 + q^1 e1 + q^2 e2 + q^3 e3   (Sec. 2.1, Eq. quaternion_def)
 *   - the product is the Hamilton product                     (Sec. 2.1, Eq. quaternion_prod)
 *       (pq)^0 = p^0 q^0 - sum_i p^i q^i
 *       (pq)^k = p^0 q^k + p^k q^0 + sum_{i,j} eps_ijk p^i q^j
 *     with eps the Levi-Civita symbol, which is what the basis algebra
 *     e_i e_j = -delta_ij e0 + sum_k eps_ijk e_k gives   (Sec. 2.1, Eq. quaternion_alg)
 *   - conj(q) = q^0 e0 - q^1 e1 - q^2 e2 - q^3 e3          (Sec. 2.1, Eq. quaternion_conj)
 *   - op(X) is X, X^T, conj(X) or X^H = conj(X)^T          (Sec. 2.2, conj / conj-transpose)
 *   - alpha and beta multiply from the LEFT: the product of a scalar and a
 *     matrix is taken as (qQ)_{mu nu} = q Q_{mu nu} and the GEMM scaling as
 *     (qPQ)_{mu nu} = q sum_kappa P_{mu kappa} Q_{kappa nu}  (Sec. 2.2); the
 *     layered algorithm folds alpha into the packed A block, i.e. on the left
 *     of the product (Sec. 3.1, Algorithm 2 and the remark after it that
 *     moving it to B is only legal for commutative rings).
 *   - storage is column-major (Sec. 3.1): element (r, c) of a stored matrix
 *     with leading dimension ld sits at r + c*ld.  Two layouts:
 *       interleaved: the four components of one element are contiguous,
 *                    [q^0; q^1; q^2; q^3] (Sec. 4), component s of (r, c) at
 *                    4*(r + c*ld) + s;
 *       split planes: Q = Q^0 e0 + ... + Q^3 e3 with real planes Q^s
 *                    (Sec. 2.2, Eq. quaternion_mat_def), component s of (r, c)
 *                    at s*plane_stride + r + c*ld.
 *
 * The loop order follows the reference algorithm of Sec. 3.1 (Algorithm 1):
 * for each column nu of C, accumulate the column sum over kappa of
 * op(A)(:, kappa) op(B)(kappa, nu), then apply alpha and beta.  The sum over
 * kappa is taken in increasing kappa order in FP64.
 *
 * Readings where the paper is silent (BLAS convention):
 *   m == 0 or n == 0: nothing is done;  k == 0: the product term is zero;
 *   beta == 0: C is not read (NaN in C is ignored).
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORACLE_OP_N = 0, ORACLE_OP_T = 1, ORACLE_OP_C = 2, ORACLE_OP_H = 3 };
enum { ORACLE_INTERLEAVED = 0, ORACLE_SPLIT_PLANES = 1 };

/* Levi-Civita symbol eps_ijk for i, j, k in {1, 2, 3}. */
static int levi_civita(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0;
    /* even permutations of (1,2,3) give +1 */
    if ((i == 1 && j == 2 && k == 3) || (i == 2 && j == 3 && k == 1) ||
        (i == 3 && j == 1 && k == 2))
        return 1;
    return -1;
}

/* Hamilton product r = p q, Eq. quaternion_prod, term by term. */
void oracle_hamilton(const double p[4], const double q[4], double r[4])
{
    double s = p[0] * q[0];
    for (int i = 1; i <= 3; ++i) s -= p[i] * q[i];
    r[0] = s;
    for (int k = 1; k <= 3; ++k) {
        double v = p[0] * q[k] + p[k] * q[0];
        for (int i = 1; i <= 3; ++i)
            for (int j = 1; j <= 3; ++j) {
                int e = levi_civita(i, j, k);
                if (e) v += (double)e * p[i] * q[j];
            }
        r[k] = v;
    }
}

/* Quaternion conjugate, Eq. quaternion_conj. */
static void conjugate(double q[4])
{
    q[1] = -q[1];
    q[2] = -q[2];
    q[3] = -q[3];
}

/* Read element (r, c) of a stored matrix. */
static void load_stored(const double *X, int64_t ld, int64_t ps, int layout,
                        int64_t r, int64_t c, double q[4])
{
    if (layout == ORACLE_INTERLEAVED) {
        const double *e = X + 4 * (r + c * ld);
        q[0] = e[0]; q[1] = e[1]; q[2] = e[2]; q[3] = e[3];
    } else {
        const double *e = X + r + c * ld;
        q[0] = e[0]; q[1] = e[ps]; q[2] = e[2 * ps]; q[3] = e[3 * ps];
    }
}

static void store_stored(double *X, int64_t ld, int64_t ps, int layout,
                         int64_t r, int64_t c, const double q[4])
{
    if (layout == ORACLE_INTERLEAVED) {
        double *e = X + 4 * (r + c * ld);
        e[0] = q[0]; e[1] = q[1]; e[2] = q[2]; e[3] = q[3];
    } else {
        double *e = X + r + c * ld;
        e[0] = q[0]; e[ps] = q[1]; e[2 * ps] = q[2]; e[3 * ps] = q[3];
    }
}

/* Element (r, c) of op(X), from the definitions of Sec. 2.2:
 * (conj X)_{rc} = conj(X_{rc}),  (X^H)_{rc} = conj(X_{cr}),  (X^T)_{rc} = X_{cr}. */
static void load_op(const double *X, int64_t ld, int64_t ps, int layout, int op,
                    int64_t r, int64_t c, double q[4])
{
    if (op == ORACLE_OP_T || op == ORACLE_OP_H)
        load_stored(X, ld, ps, layout, c, r, q);
    else
        load_stored(X, ld, ps, layout, r, c, q);
    if (op == ORACLE_OP_C || op == ORACLE_OP_H) conjugate(q);
}

static int is_zero(const double q[4])
{
    return q[0] == 0.0 && q[1] == 0.0 && q[2] == 0.0 && q[3] == 0.0;
}

/* One output element: alpha * P + beta * Cin, left scalar products. */
static void finish(const double alpha[4], const double P[4], const double beta[4],
                   const double *Cin, double out[4])
{
    double aP[4];
    oracle_hamilton(alpha, P, aP);
    if (Cin) {
        double bC[4];
        oracle_hamilton(beta, Cin, bC);
        for (int s = 0; s < 4; ++s) out[s] = aP[s] + bC[s];
    } else {
        for (int s = 0; s < 4; ++s) out[s] = aP[s];
    }
}

/*
 * Full oracle GEMM, in place on C.  Returns 0, or -1 on an argument that
 * makes the call meaningless (negative size, bad enum).
 * nthreads <= 0 uses the OpenMP default.
 */
int oracle_qgemm(int opA, int opB, int64_t m, int64_t n, int64_t k,
                 const double alpha[4],
                 const double *A, int64_t lda, int64_t psA,
                 const double *B, int64_t ldb, int64_t psB,
                 const double beta[4],
                 double *C, int64_t ldc, int64_t psC,
                 int layout, int nthreads)
{
    if (m < 0 || n < 0 || k < 0) return -1;
    if (opA < 0 || opA > 3 || opB < 0 || opB > 3) return -1;
    if (layout != ORACLE_INTERLEAVED && layout != ORACLE_SPLIT_PLANES) return -1;
    if (m == 0 || n == 0) return 0;
    const int read_c = !is_zero(beta);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int status = 0;
#pragma omp parallel
    {
        double *col = (double *)malloc(sizeof(double) * 4 * (size_t)m);
        if (!col) {
#pragma omp atomic write
            status = -2;
        }
#pragma omp for schedule(static)
        for (int64_t nu = 0; nu < n; ++nu) {
            if (!col) continue;
            /* column accumulator P(:, nu), Algorithm 1 order */
            memset(col, 0, sizeof(double) * 4 * (size_t)m);
            for (int64_t kap = 0; kap < k; ++kap) {
                double b[4];
                load_op(B, ldb, psB, layout, opB, kap, nu, b);
                for (int64_t mu = 0; mu < m; ++mu) {
                    double a[4], ab[4];
                    load_op(A, lda, psA, layout, opA, mu, kap, a);
                    oracle_hamilton(a, b, ab);
                    double *p = col + 4 * mu;
                    p[0] += ab[0]; p[1] += ab[1]; p[2] += ab[2]; p[3] += ab[3];
                }
            }
            for (int64_t mu = 0; mu < m; ++mu) {
                double cin[4], out[4];
                if (read_c) load_stored(C, ldc, psC, layout, mu, nu, cin);
                finish(alpha, col + 4 * mu, beta, read_c ? cin : NULL, out);
                store_stored(C, ldc, psC, layout, mu, nu, out);
            }
        }
        free(col);
    }
    return status;
}

/*
 * Selected entries of alpha * op(A) op(B) + beta * C, without touching C.
 * For each e < count: out[4e .. 4e+3] = entry (rows[e], cols[e]).  Used to
 * check large problems on a sample of outputs.
 */
int oracle_qgemm_entries(int opA, int opB, int64_t m, int64_t n, int64_t k,
                         const double alpha[4],
                         const double *A, int64_t lda, int64_t psA,
                         const double *B, int64_t ldb, int64_t psB,
                         const double beta[4],
                         const double *C, int64_t ldc, int64_t psC,
                         int layout, const int64_t *rows, const int64_t *cols,
                         int64_t count, double *out, int nthreads)
{
    if (m < 0 || n < 0 || k < 0 || count < 0) return -1;
    if (opA < 0 || opA > 3 || opB < 0 || opB > 3) return -1;
    if (layout != ORACLE_INTERLEAVED && layout != ORACLE_SPLIT_PLANES) return -1;
    for (int64_t e = 0; e < count; ++e)
        if (rows[e] < 0 || rows[e] >= m || cols[e] < 0 || cols[e] >= n) return -1;
    const int read_c = !is_zero(beta);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < count; ++e) {
        double P[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t kap = 0; kap < k; ++kap) {
            double a[4], b[4], ab[4];
            load_op(A, lda, psA, layout, opA, rows[e], kap, a);
            load_op(B, ldb, psB, layout, opB, kap, cols[e], b);
            oracle_hamilton(a, b, ab);
            P[0] += ab[0]; P[1] += ab[1]; P[2] += ab[2]; P[3] += ab[3];
        }
        double cin[4];
        if (read_c) load_stored(C, ldc, psC, layout, rows[e], cols[e], cin);
        finish(alpha, P, beta, read_c ? cin : NULL, out + 4 * e);
    }
    return 0;
}

/*
 * Hermitian rank-k update, the quaternion analogue of BLAS xHERK: the kernels
 * of Sec. 3 serve rank-k updates as well as GEMM (Sec. 3, opening remarks),
 * and Hermiticity Q = Q^H is defined in Sec. 2.2.
 *
 *   trans = N:  C <- alpha A A^H + beta C      (A is n x k)
 *   trans = H:  C <- alpha A^H A + beta C      (A is k x n)
 *
 * alpha and beta are real.  Only the triangle uplo (0 lower: row >= column,
 * 1 upper: row <= column) of C is read and written; the vector parts of the
 * diagonal of C are taken as zero on input and set to zero on output (the
 * diagonal of a Hermitian matrix is real).  Each entry is the plain sum over
 * kappa of op(A)_{i kappa} conj(op(A)_{j kappa}), in increasing kappa order.
 */
int oracle_qherk(int uplo, int trans, int64_t n, int64_t k, double alpha,
                 const double *A, int64_t lda, int64_t psA, double beta,
                 double *C, int64_t ldc, int64_t psC, int layout, int nthreads)
{
    if (n < 0 || k < 0) return -1;
    if (uplo != 0 && uplo != 1) return -1;
    if (trans != ORACLE_OP_N && trans != ORACLE_OP_H) return -1;
    if (layout != ORACLE_INTERLEAVED && layout != ORACLE_SPLIT_PLANES) return -1;
    const int read_c = beta != 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        const int64_t i_lo = uplo == 0 ? j : 0, i_hi = uplo == 0 ? n : j + 1;
        for (int64_t i = i_lo; i < i_hi; ++i) {
            double P[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t kap = 0; kap < k; ++kap) {
                double a[4], b[4], ab[4];
                /* op(A)_{i kappa} and conj(op(A)_{j kappa}) = (op(A)^H)_{kappa j} */
                load_op(A, lda, psA, layout, trans, i, kap, a);
                load_op(A, lda, psA, layout, trans, j, kap, b);
                conjugate(b);
                oracle_hamilton(a, b, ab);
                P[0] += ab[0]; P[1] += ab[1]; P[2] += ab[2]; P[3] += ab[3];
            }
            double cin[4] = {0.0, 0.0, 0.0, 0.0}, out[4];
            if (read_c) load_stored(C, ldc, psC, layout, i, j, cin);
            for (int s = 0; s < 4; ++s) out[s] = alpha * P[s] + beta * cin[s];
            /* diagonal: the vector parts of C are taken as zero and written as zero */
            if (i == j) out[1] = out[2] = out[3] = 0.0;
            store_stored(C, ldc, psC, layout, i, j, out);
        }
    }
    return 0;
}

/*
 * Triangular matrix product, out of place (the XTRMM of the BLAS-3 set that
 * Sec. 3 builds on the GEMM kernels):
 *   side 0 (left):  C <- alpha op(T) B,   T = tri(A), m x m,  B and C m x n
 *   side 1 (right): C <- alpha B op(T),   T = tri(A), n x n
 * tri(A) is the stored triangle of A (uplo 0: lower, r >= c; 1: upper,
 * r <= c) with zeros elsewhere; diag 1 (unit) takes the diagonal as the
 * quaternion 1 and does not read it.  op as in oracle_qgemm; alpha
 * multiplies from the left.  C is written, not read.
 */
static void load_tri(const double *A, int64_t lda, int64_t psA, int layout, int uplo, int diag,
                     int64_t r, int64_t c, double q[4])
{
    if (diag && r == c) {
        q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
        return;
    }
    const int in_triangle = uplo == 0 ? r >= c : r <= c;
    if (!in_triangle) {
        q[0] = q[1] = q[2] = q[3] = 0.0;
        return;
    }
    load_stored(A, lda, psA, layout, r, c, q);
}

/* op(T)_{r c} for T = tri(A). */
static void load_op_tri(const double *A, int64_t lda, int64_t psA, int layout, int uplo,
                        int diag, int op, int64_t r, int64_t c, double q[4])
{
    if (op == ORACLE_OP_T || op == ORACLE_OP_H)
        load_tri(A, lda, psA, layout, uplo, diag, c, r, q);
    else
        load_tri(A, lda, psA, layout, uplo, diag, r, c, q);
    if (op == ORACLE_OP_C || op == ORACLE_OP_H) conjugate(q);
}

int oracle_qtrmm(int side, int uplo, int trans, int diag, int64_t m, int64_t n,
                 const double alpha[4], const double *A, int64_t lda, int64_t psA,
                 const double *B, int64_t ldb, int64_t psB, double *C, int64_t ldc, int64_t psC,
                 int layout, int nthreads)
{
    if (m < 0 || n < 0) return -1;
    if ((side != 0 && side != 1) || (uplo != 0 && uplo != 1) || (diag != 0 && diag != 1))
        return -1;
    if (trans < ORACLE_OP_N || trans > ORACLE_OP_H) return -1;
    if (layout != ORACLE_INTERLEAVED && layout != ORACLE_SPLIT_PLANES) return -1;
    const int64_t kdim = side == 0 ? m : n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double P[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t kap = 0; kap < kdim; ++kap) {
                double a[4], b[4], ab[4];
                if (side == 0) {
                    load_op_tri(A, lda, psA, layout, uplo, diag, trans, i, kap, a);
                    load_stored(B, ldb, psB, layout, kap, j, b);
                } else {
                    load_stored(B, ldb, psB, layout, i, kap, a);
                    load_op_tri(A, lda, psA, layout, uplo, diag, trans, kap, j, b);
                }
                oracle_hamilton(a, b, ab);
                P[0] += ab[0]; P[1] += ab[1]; P[2] += ab[2]; P[3] += ab[3];
            }
            double out[4];
            oracle_hamilton(alpha, P, out);
            store_stored(C, ldc, psC, layout, i, j, out);
        }
    }
    return 0;
}

/*
 * Mixed-type GEMM (the quaternion-complex and quaternion-real arithmetic the
 * paper's library provides next to HGEMM, Sec. 5):
 *   C <- alpha op(A) op(B) + beta C,   C quaternion,
 * with A and B each quaternion (type 0), complex (type 1: z = z^0 e0 + z^1 e1,
 * the complex subalgebra of H, Sec. 2.1) or real (type 2: x e0).  The
 * plain definition: every operand entry is the quaternion it is (missing
 * components zero) and the product is the quaternion GEMM above.
 * Storage: interleaved, 4 / 2 / 1 reals per element (component s of (r, c)
 * at w*(r + c*ld) + s, w the width); split planes, 4 / 2 / 1 planes at the
 * plane stride.
 */
static void load_typed(const double *X, int64_t ld, int64_t ps, int layout, int type,
                       int64_t r, int64_t c, double q[4])
{
    const int w = type == 0 ? 4 : (type == 1 ? 2 : 1);
    q[0] = q[1] = q[2] = q[3] = 0.0;
    for (int s = 0; s < w; ++s)
        q[s] = layout == ORACLE_INTERLEAVED ? X[w * (r + c * ld) + s] : X[s * ps + r + c * ld];
}

static void load_op_typed(const double *X, int64_t ld, int64_t ps, int layout, int type, int op,
                          int64_t r, int64_t c, double q[4])
{
    if (op == ORACLE_OP_T || op == ORACLE_OP_H)
        load_typed(X, ld, ps, layout, type, c, r, q);
    else
        load_typed(X, ld, ps, layout, type, r, c, q);
    if (op == ORACLE_OP_C || op == ORACLE_OP_H) conjugate(q);
}

int oracle_qgemm_mixed(int typeA, int typeB, int opA, int opB, int64_t m, int64_t n, int64_t k,
                       const double alpha[4], const double *A, int64_t lda, int64_t psA,
                       const double *B, int64_t ldb, int64_t psB, const double beta[4],
                       double *C, int64_t ldc, int64_t psC, int layout, int nthreads)
{
    if (m < 0 || n < 0 || k < 0) return -1;
    if (typeA < 0 || typeA > 2 || typeB < 0 || typeB > 2) return -1;
    if (opA < 0 || opA > 3 || opB < 0 || opB > 3) return -1;
    if (layout != ORACLE_INTERLEAVED && layout != ORACLE_SPLIT_PLANES) return -1;
    const int read_c = !is_zero(beta);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double P[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t kap = 0; kap < k; ++kap) {
                double a[4], b[4], ab[4];
                load_op_typed(A, lda, psA, layout, typeA, opA, i, kap, a);
                load_op_typed(B, ldb, psB, layout, typeB, opB, kap, j, b);
                oracle_hamilton(a, b, ab);
                P[0] += ab[0]; P[1] += ab[1]; P[2] += ab[2]; P[3] += ab[3];
            }
            double cin[4], out[4];
            if (read_c) load_stored(C, ldc, psC, layout, i, j, cin);
            finish(alpha, P, beta, read_c ? cin : NULL, out);
            store_stored(C, ldc, psC, layout, i, j, out);
        }
    }
    return 0;
}

/* Number of OpenMP threads the oracle would use by default. */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
