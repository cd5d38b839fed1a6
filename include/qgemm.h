/*
 * qgemm.h -- C ABI of the GB300 quaternion GEMM library.
 *
 * The operation (Sec. 3.1, Eq. general_gemm, over the quaternions H):
 *
 *     C <- alpha * op(A) * op(B) + beta * C
 *
 *   - A quaternion is q = q^0 e0 + q^1 e1 + q^2 e2 + q^3 e3 (Sec. 2.1,
 *     Eq. quaternion_def); products are Hamilton products (Eq. quaternion_prod),
 *     taken in the order A_{i kappa} B_{kappa j}.
 *   - op(X) is X (N), X^T (T), conj(X) (C) or X^H = conj(X)^T (H), with the
 *     element-wise conjugate and conjugate transpose of Sec. 2.2.
 *   - alpha and beta multiply from the LEFT, (alpha P)_{ij} = alpha P_{ij}
 *     (Sec. 2.2, Eq. no_scalar_comm_mat; Sec. 3.1, Algorithm 2 folds alpha into
 *     the packed A block).  Quaternions do not commute, so this is observable.
 *   - op(A) is m x k, op(B) is k x n, C is m x n.  The STORED A is m x k for N/C
 *     and k x m for T/H (likewise B).
 *
 * Storage (column-major, Sec. 3.1): element (r, c) of a stored matrix with
 * leading dimension ld (in quaternion elements) sits at r + c*ld.
 *   QGEMM_INTERLEAVED:  the four components of an element are contiguous,
 *       [q^0, q^1, q^2, q^3] (Sec. 4): component s at 4*(r + c*ld) + s reals.
 *   QGEMM_SPLIT_PLANES: four real column-major planes Q^s (Sec. 2.2,
 *       Eq. quaternion_mat_def): component s at s*plane_stride + r + c*ld reals.
 *       plane_stride must be >= ld * (stored columns); it is ignored for the
 *       interleaved layout.
 *
 * Precision:
 *   QGEMM_FP64:            double data; FP64 products, accumulation and
 *                          epilogue: a product whose 32 x 32-quaternion tiles
 *                          fill the GPU runs on the FP64 FMA pipe (the faster
 *                          FP64 pipe of GB300), the others on the FP64 tensor
 *                          cores (DMMA).  Needs no
 *                          workspace; given one of qgemm_workspace_bytes()
 *                          bytes, a product whose C is too small to fill the
 *                          GPU (fewer than 8 waves of 16 x 16 quaternion
 *                          tiles, the last one part-empty) and whose k is long
 *                          splits K across CTAs so that the waves fill:
 *                          each share's partial product goes to the workspace
 *                          and a second kernel sums the shares in a fixed
 *                          order (deterministic) before the epilogue.
 *   QGEMM_FP32_SPLIT_BF16: float data; each operand is split into three BF16
 *                          terms (hi, mid, lo), the six leading term products
 *                          run on the BF16 tensor cores (tcgen05) with FP32
 *                          accumulation in tensor memory, added every 16
 *                          kappa to a register sum by compensated (TwoSum)
 *                          addition; alpha scales op(A) in double-float before
 *                          the split and beta C (FP32 products) is the sum's
 *                          starting value; one final rounding to float.
 *                          Needs a workspace (qgemm_workspace_bytes;
 *                          beyond its minimum, the size reported lets a
 *                          product with few tiles of C and a long k split K
 *                          across CTAs, as QGEMM_FP64).
 *   QGEMM_FP64_SLICED_BF16: double data; FP64-class result on the BF16 tensor
 *                          cores (no paper counterpart; the paper is FP64
 *                          throughout, and GB300's FP64 pipe is narrow).  Each
 *                          quaternion row of op(A) and column of op(B) is
 *                          scaled by a power of two 2^e (e from its largest
 *                          component) and written as six integer digits of 8
 *                          bits (an error-free splitting after Ozaki et al.);
 *                          the 21 digit-pair products whose scale is >= 2^-40
 *                          run on tcgen05 with exact integer sums.  Error per
 *                          entry of op(A) op(B) <= 4k * 2^(e_i + e_n) * 2^-44,
 *                          i.e.
 *                          relative to max|row i of op(A)| * max|column n of
 *                          op(B)| rather than to |C_in| (inputs whose rows or
 *                          columns span many binades along k lose digits of
 *                          their small entries).  A row or column holding Inf
 *                          or NaN gives NaN in the matching row or column of
 *                          the product.  Needs a workspace; k <= 2^21
 *                          (QGEMM_ERR_UNSUPPORTED above).  The size that
 *                          qgemm_workspace_bytes() reports may exceed the
 *                          minimum: the rest lets a product with few tiles
 *                          of C and a long k split K across CTAs (as
 *                          QGEMM_FP64; without it the call runs unsplit).
 *
 * Memory and streams: every matrix pointer is a DEVICE pointer owned by the
 * caller; alpha and beta are HOST arrays of 4 doubles, read during the call
 * (so a captured CUDA graph freezes their values).  Calls are asynchronous on
 * `stream` (a cudaStream_t; NULL is the legacy default stream): buffers must
 * stay valid until the stream reaches the call.  The library never allocates
 * device memory in these calls; scratch space is the caller's workspace.
 * Elements must be aligned to their type (8 bytes FP64, 4 bytes FP32); tiles
 * are fetched with the tensor memory accelerator when base and strides are
 * 16-byte aligned, and with plain loads otherwise.
 *
 * Return values: 0 on success; -i when argument i (1-based) is invalid, in
 * the manner of LAPACK's INFO; a positive QGEMM_ERR_* code otherwise.
 * Argument checks happen before anything is launched.  A kernel that gives up
 * on a bounded wait records QGEMM_ERR_TIMEOUT in a device status word that
 * qgemm_get_last_device_error() reads.  The library never aborts, never
 * prints, and has no CPU fallback: without a usable sm_103 device the calls
 * return QGEMM_ERR_NO_DEVICE.
 *
 * BLAS conventions where the paper is silent: m == 0 or n == 0 returns at
 * once; k == 0 or alpha == 0 gives C <- beta * C; beta == 0 means C is not
 * read (it may hold NaN).
 */
#ifndef QGEMM_H
#define QGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QGEMM_OP_N 0
#define QGEMM_OP_T 1
#define QGEMM_OP_C 2
#define QGEMM_OP_H 3

#define QGEMM_INTERLEAVED 0
#define QGEMM_SPLIT_PLANES 1

#define QGEMM_LOWER 0
#define QGEMM_UPPER 1

#define QGEMM_LEFT 0
#define QGEMM_RIGHT 1

#define QGEMM_NON_UNIT 0
#define QGEMM_UNIT 1

#define QGEMM_TYPE_QUATERNION 0
#define QGEMM_TYPE_COMPLEX 1
#define QGEMM_TYPE_REAL 2

#define QGEMM_FP64 0
#define QGEMM_FP32_SPLIT_BF16 1
#define QGEMM_FP64_SLICED_BF16 2

#define QGEMM_SUCCESS 0
#define QGEMM_ERR_UNSUPPORTED 1 /* valid arguments, combination not implemented   */
#define QGEMM_ERR_CUDA 2        /* a CUDA runtime call or launch failed            */
#define QGEMM_ERR_TIMEOUT 3     /* a device-side bounded wait gave up              */
#define QGEMM_ERR_NO_DEVICE 4   /* no usable sm_103 device / driver entry point    */
#define QGEMM_ERR_WORKSPACE 5   /* workspace missing, too small or misaligned      */

/*
 * qgemm: C <- alpha op(A) op(B) + beta C   (Sec. 3.1, Eq. general_gemm).
 *
 *   1 opA, 2 opB         QGEMM_OP_{N,T,C,H}
 *   3 m, 4 n, 5 k        sizes in quaternions, >= 0
 *   6 alpha              host double[4], left scalar
 *   7 A, 8 lda, 9 psA    device pointer, leading dim (>= max(1, stored rows)),
 *                        plane stride (split planes only)
 *  10 B, 11 ldb, 12 psB  likewise
 *  13 beta               host double[4], left scalar
 *  14 C, 15 ldc, 16 psC  device pointer (read unless beta == 0, then written)
 *  17 layout             QGEMM_INTERLEAVED or QGEMM_SPLIT_PLANES (all three
 *                        matrices share it)
 *  18 precision          QGEMM_FP64, QGEMM_FP32_SPLIT_BF16 or
 *                        QGEMM_FP64_SLICED_BF16
 *  19 workspace          device scratch, 256-byte aligned, or NULL if
 *  20 workspace_bytes    qgemm_workspace_bytes() is 0 (optional for
 *                        QGEMM_FP64: NULL or a smaller one runs K unsplit)
 *  21 stream             cudaStream_t
 */
int qgemm(int opA, int opB, int64_t m, int64_t n, int64_t k,
          const double alpha[4],
          const void *A, int64_t lda, int64_t psA,
          const void *B, int64_t ldb, int64_t psB,
          const double beta[4],
          void *C, int64_t ldc, int64_t psC,
          int layout, int precision,
          void *workspace, size_t workspace_bytes,
          void *stream);

/* Workspace qgemm() needs for these arguments; for QGEMM_FP64 the workspace
 * that lets it split K (0 when the product would not be split; the SM count
 * of the current device decides, 152 when there is none).  Returns 0 for
 * invalid arguments as well; qgemm() itself reports those. */
size_t qgemm_workspace_bytes(int opA, int opB, int64_t m, int64_t n, int64_t k,
                             int layout, int precision);

/*
 * qgemm_split_noalloc: the split-BF16 qgemm() for callers that cannot
 * allocate device memory -- for example code whose device memory all belongs
 * to another allocator (a framework's pool, a fixed arena), or a plain C
 * caller with no allocator of its own.  It takes no workspace: the split
 * operands (and, for few tiles of C with a long k, the K shares' partial
 * products) go to a scratch array of QGEMM_NOALLOC_SCRATCH_BYTES that the
 * library keeps in device memory (every device that loads the library holds
 * it until the process exits).  The paper has no counterpart; it is an
 * interface convenience.
 *
 * Arguments 1-17 and 18 (stream) as in qgemm() with precision
 * QGEMM_FP32_SPLIT_BF16 (float data).  Returns QGEMM_ERR_WORKSPACE, before
 * launching anything, when the problem's split operands need more than
 * QGEMM_NOALLOC_SCRATCH_BYTES (qgemm_workspace_bytes() gives the need; for
 * square problems the largest that fits is m = n = k = 1180).
 * It calls no allocator.  The first call on a device looks up the scratch
 * array's device address once for that device, so make it before any stream
 * capture; the address is kept for the life of the process, so the library
 * must not be used across a cudaDeviceReset() of that device.  All calls
 * share the one array: calls that can overlap on the GPU (different streams
 * without ordering between them) race and give wrong results.  Each call
 * rewrites every scratch byte its kernels read, so nothing has to be cleared
 * between calls.
 */
#define QGEMM_NOALLOC_SCRATCH_BYTES (64u << 20)
int qgemm_split_noalloc(int opA, int opB, int64_t m, int64_t n, int64_t k,
                        const double alpha[4],
                        const void *A, int64_t lda, int64_t psA,
                        const void *B, int64_t ldb, int64_t psB,
                        const double beta[4],
                        void *C, int64_t ldc, int64_t psC,
                        int layout, void *stream);


/*
 * One problem of a grouped batch (host struct).  Same meaning as the qgemm()
 * arguments of the same names; ops are QGEMM_OP_* values.
 */
typedef struct qgemm_problem {
    int32_t opA, opB;
    int64_t m, n, k;
    double alpha[4], beta[4];
    const void *A; int64_t lda, psA;
    const void *B; int64_t ldb, psB;
    void *C; int64_t ldc, psC;
} qgemm_problem;

/*
 * Plan of a grouped batch, filled by qgemm_grouped_prepare() (host struct,
 * owned by the caller; it only describes what the prepare call wrote into
 * the workspace, so it can be copied freely).
 */
typedef struct qgemm_grouped_plan {
    void *workspace;          /* device schedule written by prepare           */
    size_t workspace_bytes;   /* bytes of it in use                           */
    int32_t layout, precision;
    int64_t count;            /* problems                                     */
    int64_t tiles;            /* output tiles in the schedule                 */
    int32_t grid;             /* persistent CTAs launched                     */
    int32_t reserved0;
    int64_t desc_offset;      /* byte offsets of the schedule's sections      */
    int64_t tile_offset;
    int64_t data_offset;
    int64_t reserved[4];
} qgemm_grouped_plan;

/*
 * qgemm_batched_grouped: `count` independent problems C_p <- alpha_p op(A_p)
 * op(B_p) + beta_p C_p (each as in qgemm()) in one persistent launch: the
 * batching of many uneven products; the tile shape of each problem comes
 * from a per-size-bucket table (qgemm_grouped_set_tile_table), the GPU
 * analogue of the paper's per-machine choice of blocking parameters
 * (Sec. 3.2, Sec. 5).  `problems` is a HOST array.  Equivalent to
 * qgemm_grouped_prepare() followed by qgemm_grouped_launch().
 * Return codes: -1 problems, -2 count, -3 layout, -4 precision, -5 workspace,
 * -6 workspace_bytes, -8 plan; -(1000*(p+1) + i) when argument i (numbered as
 * in qgemm()) of problem p is invalid; positive QGEMM_ERR_* otherwise.
 */
int qgemm_batched_grouped(const qgemm_problem *problems, int64_t count,
                          int layout, int precision,
                          void *workspace, size_t workspace_bytes,
                          void *stream);

/* Workspace for a grouped batch with these problems (0 if they are invalid). */
size_t qgemm_grouped_workspace_bytes(const qgemm_problem *problems, int64_t count,
                                     int layout, int precision);

/*
 * Split form for CUDA-graph capture.  qgemm_grouped_prepare() validates the
 * problems, encodes their tensor maps and tile schedule on the host and
 * copies them into `workspace` with cudaMemcpyAsync on `stream` (from
 * pageable host memory: do not call it during stream capture); it fills
 * *plan.  qgemm_grouped_launch() only resets the schedule's tile counter
 * (cudaMemsetAsync) and launches the persistent kernel, so it can be captured
 * and replayed.  Matrix pointers, sizes and scalars are frozen at prepare
 * time; the matrices' contents are read at launch time.  The workspace must
 * not be modified between the two, and launches sharing one workspace must
 * not overlap on the GPU.
 */
int qgemm_grouped_prepare(const qgemm_problem *problems, int64_t count,
                          int layout, int precision,
                          void *workspace, size_t workspace_bytes, void *stream,
                          qgemm_grouped_plan *plan);
int qgemm_grouped_launch(const qgemm_grouped_plan *plan, void *stream);

/*
 * Tile-shape table of the grouped path (the autotuner's output).  Problems
 * fall into 25 buckets, index 5*rm + rn, where rm (rn) is the range of m (n)
 * among (<=16, <=32, <=64, <=128, >128).  table[b] is a shape index (see
 * qgemm_grouped_tile_info).  table == NULL restores the built-in choice
 * (per dimension the shape with least padding).  FP64 only.
 */
int qgemm_grouped_set_tile_table(int precision, const int32_t *table, int32_t entries);

/* Shapes and buckets of the grouped path: number of shapes, their quaternion
 * rows / columns (arrays of at least 8), number of buckets, the 4 range edges. */
int qgemm_grouped_tile_info(int32_t *num_shapes, int32_t *shape_m, int32_t *shape_n,
                            int32_t *num_buckets, int32_t *edges);

/*
 * qherk: Hermitian rank-k update on one triangle of C (the quaternion xHERK;
 * the paper notes its GEMM kernels also serve rank-k updates, Sec. 3, and
 * defines Hermiticity Q = Q^H in Sec. 2.2):
 *     trans = QGEMM_OP_N:  C <- alpha A A^H + beta C     (A is n x k)
 *     trans = QGEMM_OP_H:  C <- alpha A^H A + beta C     (A is k x n)
 * alpha and beta are REAL.  Only the triangle `uplo` (QGEMM_LOWER: row >=
 * column; QGEMM_UPPER: row <= column) of C is read and written; the vector
 * parts of C's diagonal are taken as zero and written as zero.  It runs the
 * same kernels as qgemm() with op(B) = op(A)^H read from A itself, skipping
 * tiles outside the triangle.  Arguments, in order for the -i return:
 *   1 uplo, 2 trans, 3 n, 4 k, 5 alpha, 6 A, 7 lda, 8 psA, 9 beta, 10 C,
 *   11 ldc, 12 psC, 13 layout, 14 precision, 15 workspace, 16 workspace_bytes,
 *   17 stream; layouts, precisions and workspace as in qgemm().
 */
int qherk(int uplo, int trans, int64_t n, int64_t k, double alpha,
          const void *A, int64_t lda, int64_t psA, double beta,
          void *C, int64_t ldc, int64_t psC, int layout, int precision,
          void *workspace, size_t workspace_bytes, void *stream);

/* Workspace qherk() needs; for QGEMM_FP64 the optional one that lets an
 * update with few tiles in its triangle and a long k split K (as qgemm). */
size_t qherk_workspace_bytes(int uplo, int trans, int64_t n, int64_t k,
                             int layout, int precision);

/*
 * qtrmm: triangular matrix product, out of place (the quaternion xTRMM; the
 * paper notes its GEMM kernels also serve triangular products, Sec. 3):
 *     side = QGEMM_LEFT:   C <- alpha op(T) B     (T m x m, B and C m x n)
 *     side = QGEMM_RIGHT:  C <- alpha B op(T)     (T n x n)
 * T = tri(A): the triangle `uplo` of the stored A (QGEMM_LOWER: row >=
 * column; QGEMM_UPPER: row <= column), zeros elsewhere; diag QGEMM_UNIT takes
 * the diagonal as the quaternion 1 without reading it.  op(T) as in qgemm();
 * alpha multiplies from the left.  C is written, not read, and must not
 * overlap B (C == B is rejected).  The triangle is copied densely into the
 * workspace and the product runs on the qgemm() kernels of the chosen
 * precision, each output tile summing only over the k-range where op(T) can
 * be nonzero.  Arguments, in order for the -i return:
 *   1 side, 2 uplo, 3 transA, 4 diag, 5 m, 6 n, 7 alpha (host double[4]),
 *   8 A, 9 lda (>= max(1, m or n)), 10 psA, 11 B, 12 ldb, 13 psB, 14 C,
 *   15 ldc, 16 psC, 17 layout, 18 precision, 19 workspace, 20 workspace_bytes,
 *   21 stream.  A workspace is always needed (qtrmm_workspace_bytes()).
 */
int qtrmm(int side, int uplo, int transA, int diag, int64_t m, int64_t n,
          const double alpha[4],
          const void *A, int64_t lda, int64_t psA,
          const void *B, int64_t ldb, int64_t psB,
          void *C, int64_t ldc, int64_t psC,
          int layout, int precision,
          void *workspace, size_t workspace_bytes, void *stream);

/* Workspace qtrmm() needs (0 for invalid arguments or an empty C). */
size_t qtrmm_workspace_bytes(int side, int uplo, int transA, int diag, int64_t m, int64_t n,
                             int layout, int precision);

/*
 * qgemm_mixed: mixed-type product (the quaternion-complex and
 * quaternion-real arithmetic of the paper's library, Sec. 5):
 *     C <- alpha op(A) op(B) + beta C,   C quaternion,
 * with A and B each QGEMM_TYPE_QUATERNION, QGEMM_TYPE_COMPLEX (z = z^0 e0 +
 * z^1 e1, the complex numbers inside H) or QGEMM_TYPE_REAL (x e0).  A complex
 * element stores 2 reals, a real one 1: interleaved [z^0, z^1] (component s
 * of (r, c) at w*(r + c*ld) + s, w = 2 or 1), split planes 2 or 1 planes at
 * the plane stride.  op conjugates as in H (conj(z) = z^0 - z^1 e1).
 * Arguments: 1 typeA, 2 typeB, then the arguments of qgemm() as 3..23
 * (opA = 3 ... stream = 23) for the -i return.  A complex (real) factor
 * halves (quarters) the tensor-core or DMMA work of the quaternion product
 * (when both factors are narrow, the FP64 path copies the left one as a
 * quaternion matrix).  Workspace from qgemm_mixed_workspace_bytes().
 */
int qgemm_mixed(int typeA, int typeB, int opA, int opB, int64_t m, int64_t n, int64_t k,
                const double alpha[4],
                const void *A, int64_t lda, int64_t psA,
                const void *B, int64_t ldb, int64_t psB,
                const double beta[4],
                void *C, int64_t ldc, int64_t psC,
                int layout, int precision,
                void *workspace, size_t workspace_bytes, void *stream);

size_t qgemm_mixed_workspace_bytes(int typeA, int typeB, int opA, int opB, int64_t m,
                                   int64_t n, int64_t k, int layout, int precision);

/*
 * qgemm_backward: gradients of a quaternion linear map Y = X W, with
 * X (mb x k), W (k x n), Y (mb x n) stored untransposed.  With the real inner
 * product <P, Q> = Re tr(P^H Q) = sum of component products, and
 * Re tr(PQ) = Re tr(QP) on H, a real loss L with componentwise gradient
 * dY = dL/dY has
 *     dX = dY W^H   (mb x k)      dW = X^H dY   (k x n)
 * (conjugate transpose of Sec. 2.2, read directly by the tile loads; no
 * transposed copy is made).  dX or dW may be NULL to skip that gradient.
 * accumulate != 0 adds into dX / dW (beta = 1), else overwrites (beta = 0).
 * Arguments are numbered 1..24 for the -i return in the order below.
 */
int qgemm_backward(int64_t mb, int64_t k, int64_t n,
                   const void *X, int64_t ldx, int64_t psx,
                   const void *W, int64_t ldw, int64_t psw,
                   const void *dY, int64_t lddy, int64_t psdy,
                   void *dX, int64_t lddx, int64_t psdx,
                   void *dW, int64_t lddw, int64_t psdw,
                   int accumulate, int layout, int precision,
                   void *workspace, size_t workspace_bytes, void *stream);

/* Workspace qgemm_backward() needs (the larger of its two products; for
 * QGEMM_FP64 the optional one that lets a product split K, as qgemm). */
size_t qgemm_backward_workspace_bytes(int64_t mb, int64_t k, int64_t n,
                                      int layout, int precision);

/* Reads and clears the device status word (synchronises the device).
 * Returns QGEMM_SUCCESS or QGEMM_ERR_TIMEOUT. */
int qgemm_get_last_device_error(void);

/* Name of the CUDA error behind the most recent QGEMM_ERR_CUDA returned by a
 * launch in this process ("no error" if none); a diagnostic aid. */
const char *qgemm_last_cuda_error(void);

/* Static description of a status code. */
const char *qgemm_status_string(int status);

/*
 * Test hook for the bounded waits: launches one kernel that waits on a
 * barrier nothing ever arrives on, with the given limit in nanoseconds.  The
 * wait gives up, the kernel records QGEMM_ERR_TIMEOUT and returns, so the
 * context stays usable.  Returns the launch status.
 */
int qgemm_debug_unsatisfied_wait(uint64_t limit_ns, void *stream);

/*
 * Test hook for the abort paths of the GEMM kernels (no paper counterpart;
 * the failure detection of the library's own waits).  Arms a one-shot fault
 * for the next qgemm() launch of precision `path` (QGEMM_FP64 or
 * QGEMM_FP32_SPLIT_BF16): the kernel's TMA producer leaves out the copies of
 * its ring stage number `stage` (counted from 0 over the launch; for FP64 in
 * the first CTA), and that launch waits at most limit_ns (1 ms .. 10 s) per
 * wait.  The consumer's wait gives up, every role of the CTA stops, copies in
 * flight land, tensor memory is released, and qgemm_get_last_device_error()
 * then reports QGEMM_ERR_TIMEOUT; the context stays usable.  The launch's C
 * is undefined.  Returns 0, or -i for an invalid argument i.
 */
int qgemm_debug_arm_fault(int path, int stage, uint64_t limit_ns);

/*
 * Throughput microbenchmarks of the device's arithmetic pipes (no paper
 * counterpart; they supply the roofline denominators).  which:
 *   0 FP64 tensor (DMMA m16n8k4)   1 FP64 FMA (DFMA)   2 FP32 FMA (FFMA)
 *   3 BF16 tensor (tcgen05.mma kind::f16, 128x256x16, FP32 accumulate),
 *     zero operands
 *   4, 5, 6 the same instruction at N = 256, 128, 64 on operands holding
 *     integers in [-127, 127]
 *   7 DMMA and DFMA together (alternate warps): whether the two FP64 pipes add
 *   8 N = 64, four MMAs per A tile (four B tiles) with the A operand held in
 *     the tensor core's collector; 9 the same without the collector;
 *     10 N = 32 as 8; 11 N = 128, two MMAs per A tile, collector;
 *     12 N = 64, twelve MMAs per A tile, collector
 * Runs for roughly `seconds` and writes the achieved TFLOP/s (2 per FMA).
 */
int qgemm_probe_peak(int which, double seconds, double *tflops, void *stream);

/* Library version string. */
const char *qgemm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QGEMM_H */
