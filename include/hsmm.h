/*
 * hsmm.h -- C ABI of the hsmm library: dense matrix products on one NVIDIA GB300
 * (sm_103a), after Lippert, Petkov, Palazzari and Schilling, "Hyper-Systolic
 * Matrix Multiplication".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Storage is column-major (BLAS): element (i, j) of a matrix with leading
 *    dimension ld sits at index i + j*ld.  op(X) is X for HSMM_OP_N and X^T for
 *    HSMM_OP_T.  C is m x n, op(A) is m x k, op(B) is k x n.
 *  - A, B, C, x, y, workspace: DEVICE pointers owned by the caller.  The library
 *    keeps no reference to them after the call returns.  alpha and beta are HOST
 *    pointers to one scalar of the compute type (double for FP64 computation,
 *    float for FP32/BF16/TF32, int32_t for INT8).
 *  - stream: a cudaStream_t (NULL = the legacy default stream).  Every call is
 *    asynchronous with respect to the host and enqueues its kernels on stream.
 *  - Errors are returned, never raised: no call exits or aborts.  Argument errors
 *    are detected on the host before anything is enqueued.  An error inside a
 *    kernel (a bounded wait that ran out) sets a device status word that
 *    hsmm_sync_status() reports as HSMM_STATUS_TIMEOUT.
 *  - BLAS early-outs: m == 0 or n == 0 returns at once; k == 0 or *alpha == 0
 *    gives C = beta*C without reading A or B; beta == 0 never reads C (NaNs in
 *    C are not propagated).
 *  - No entry point allocates device memory, except the grouped plan, which
 *    allocates once in hsmm_grouped_plan_create and frees in
 *    hsmm_grouped_plan_destroy.  Scratch needed by a product (the slices of the
 *    FP64-accurate form, the descriptors of a grouped launch) comes from
 *    hsmm_config_t.workspace, sized by hsmm_workspace_size() and its siblings.
 *  - There is no CPU fallback: without a GB300 the calls return
 *    HSMM_STATUS_CUDA_ERROR.
 */
#ifndef HSMM_H
#define HSMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HSMM_STATUS_SUCCESS = 0,
    HSMM_STATUS_INVALID_VALUE = 1,          /* bad size, leading dimension, increment or pointer */
    HSMM_STATUS_NOT_SUPPORTED = 2,          /* dtype/compute combination, or TMA alignment not met */
    HSMM_STATUS_WORKSPACE_TOO_SMALL = 3,
    HSMM_STATUS_CUDA_ERROR = 4,             /* see hsmm_last_cuda_error() */
    HSMM_STATUS_TIMEOUT = 5                 /* a bounded device-side wait ran out */
} hsmm_status_t;

/* op(M): M, its transpose, or its conjugate transpose (complex matrices; for real ones C = T) */
typedef enum { HSMM_OP_N = 'N', HSMM_OP_T = 'T', HSMM_OP_C = 'C' } hsmm_op_t;

typedef enum {
    HSMM_R_64F = 0,
    HSMM_R_32F = 1,
    HSMM_R_16BF = 2,
    HSMM_R_8I = 3,
    HSMM_R_32I = 4,
    HSMM_C_64F = 5                  /* complex FP64: interleaved (re, im) doubles, 16 bytes */
} hsmm_dtype_t;

typedef enum {
    HSMM_COMPUTE_DEFAULT = 0,       /* BF16 in: FP32 accumulate on tcgen05; FP64 in: native FP64 */
    HSMM_COMPUTE_32F_FAST_TF32 = 1, /* FP32 in: TF32 products, FP32 accumulate on tcgen05 */
    HSMM_COMPUTE_64F_NATIVE = 2,    /* FP64 in: FP64 FMA pipe */
    HSMM_COMPUTE_64F_OZAKI = 3,     /* FP64 in: FP64-accurate product from BF16 slices on tcgen05 */
    HSMM_COMPUTE_64F_RING = 4       /* FP64 in: the paper's Algorithm 2 on p CTAs (hsmm_ring_gemm) */
} hsmm_compute_t;

typedef struct {
    hsmm_dtype_t a, b, c;           /* storage types of A, B and C */
    hsmm_compute_t compute;
    int ozaki_slices;               /* slices per operand, 0 = default (7) */
    int ozaki_bits;                 /* bits per slice (5, 6 or 7), 0 = default (7) */
    void* workspace;                /* device scratch, caller-owned */
    size_t workspace_bytes;
    int tile_n;                     /* 0 = autotuned; 64, 128 or 256 columns per tile */
    int ring_p;                     /* 0: persistent tile order.  2, 4, 8 or 16: the ring order of
                                       Algorithm 2 (Section 5.2.2) on thread-block clusters of ring_p
                                       CTAs; (16BF, 16BF, 32F, DEFAULT) only */
    int ring_k;                     /* auxiliary accumulators of the ring order: 1, 2 or 4, dividing
                                       ring_p; 0 = the largest power of two <= sqrt(ring_p) */
    int reserved[5];                /* must be zero */
} hsmm_config_t;

/*
 * hsmm_gemm: C <- alpha*op(A)*op(B) + beta*C.
 * The dense product of Eq. PRODUCT (Section 3.1), c_ij = sum_k a_ik b_kj, and its
 * transposed forms A^T*B, A*B^T (Section 8: "carried out on the same footing";
 * here by the major-ness of the operand tiles, without copies).
 *  cfg == NULL: a = b = c = HSMM_R_64F with HSMM_COMPUTE_DEFAULT.
 *  Supported (a, b, c, compute):
 *    (16BF, 16BF, 32F or 16BF, DEFAULT)  tcgen05 BF16, FP32 accumulation
 *    (32F, 32F, 32F, FAST_TF32)          tcgen05 TF32, FP32 accumulation, all four op forms
 *                                        (MN-major operands staged in the tensor core's
 *                                        128-byte swizzle of 32-byte units)
 *    (64F, 64F, 64F, DEFAULT or NATIVE)  FP64 FMA
 *    (64F, 64F, 64F, OZAKI)              error-free BF16 slices; needs workspace
 *    (C64F, C64F, C64F, DEFAULT or NATIVE)  complex product on the FP64 pipe (Section 7
 *                                        measures the method on complex data); op = N, T, C
 *    (C64F, C64F, C64F, OZAKI)           FP64-accurate complex product: the real product
 *                                        A' B'' of A' = [Re op(A), Im op(A)] (m x 2k) and
 *                                        B'' = [[Re op(B), Im op(B)], [-Im op(B), Re op(B)]]
 *                                        (2k x 2n), whose columns j and n + j are Re and Im
 *                                        of column j of op(A) op(B), by the FP64-accurate
 *                                        form below with n -> 2n, k -> 2k (one exponent per
 *                                        complex row / column); needs workspace
 *  Scalars: alpha and beta point to the compute type: double for 64F, two doubles
 *  (re, im) for C64F, float for BF16/TF32 products.
 *  Tensor-core paths need 16-byte aligned A, B and lda*size, ldb*size multiples of
 *  16 bytes (TMA); otherwise HSMM_STATUS_NOT_SUPPORTED.
 *  Ring order (ring_p != 0): a cluster of p = ring_p CTAs is the ring of p processors of
 *  Algorithm 2 and computes a 128 x 128p panel of C, CTA i block column i.  The
 *  contraction runs in rounds of p k-blocks of 64; A blocks move between the CTAs
 *  (A <- cshift-row^K(A), one 16 KiB shared-memory copy per step, K~ - 1 = p/K - 1 per
 *  round), each CTA keeps K = ring_k auxiliary 128 x 128 FP32 accumulators C^l in tensor
 *  memory, and the final back-shift C^(l-1) += cshift-row^1(C^l) moves K - 1 blocks of C
 *  per CTA.  Same result as the persistent order up to FP32 summation order; meant to
 *  compare the two schedules.  p = 16 needs a non-portable cluster size; if the GPU cannot
 *  hold such a cluster the call returns HSMM_STATUS_NOT_SUPPORTED.
 *  FP64-accurate form (OZAKI): s = ozaki_slices, b = ozaki_bits, kq = k rounded up
 *  to a multiple of 8.  cfg->workspace (256-byte aligned, hsmm_workspace_size()
 *  bytes) is carved, each piece starting on a 256-byte boundary, into
 *    QA  s planes of m x kq BF16   slices of op(A), [t][i][k] (as hsmm_ozaki_split, by rows)
 *    QB  s planes of n x kq BF16   slices of op(B), [u][j][k] (by columns)
 *    EA  m INT32, EB n INT32       exponents of rows / columns
 *    SD  s planes of m x n INT32   S_d = sum_{t+u=d} QA_t QB_u^T, d = 2..s+1, [d-2][j][i]
 *  where a plane of E elements of size z bytes has the pitch (round_up(E z, 256) + 1024) / z
 *  elements (the planes one thread touches are then not a power of two apart).
 *  and C = alpha 2^(EA_i + EB_j) sum_d 2^(-b d) S_d + beta C.  Every S_d is exact
 *  (FP32 tensor-core sums of at most 2^24 / (2^b - 1)^2 products, drained to INT32);
 *  requires s k (2^b - 1)^2 < 2^31, else HSMM_STATUS_NOT_SUPPORTED.
 *  lda >= max(1, rows of stored A) (m if transA == N else k); same for B; ldc >= max(1, m).
 *  Only the m x n elements of C are read (beta != 0) and written: rows m..ldc-1 of every
 *  column are left as they are.
 */
hsmm_status_t hsmm_gemm(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB,
                        int64_t m, int64_t n, int64_t k, const void* alpha,
                        const void* A, int64_t lda, const void* B, int64_t ldb,
                        const void* beta, void* C, int64_t ldc, void* stream);

/*
 * hsmm_gemm_host: hsmm_gemm with A, B and C in HOST memory (the operation of Eq. PRODUCT,
 * Section 3.1, and its complex and transposed forms as in hsmm_gemm; same cfg, ops,
 * scalars and leading dimensions, here of the host arrays).  C is computed in blocks:
 * row panels of op(A) (two once m >= 4096, four once m >= 8192) times column panels of
 * op(B) (two once n >= 4096).  The first panel of each operand is copied first, the later panels while
 * the first blocks are computed, and every finished block of C returns to the host while
 * the next one is computed.  The FP64-accurate forms split each panel of op(A) and of
 * op(B) once (the result equals that of hsmm_gemm on the same data).  Copies run on two
 * copy streams (one per direction) the library creates once per device; `stream` waits
 * for all of them, so C is complete once the caller's stream is.  Host arrays must stay valid until then; page-locked host memory lets the copies
 * run asynchronously, pageable memory works but serialises them.
 * cfg->workspace (256-byte aligned, hsmm_gemm_host_workspace_size() bytes) holds the
 * device copies of A, B and C (leading dimensions rounded up to 16 elements) and the
 * workspace of the compute form; nothing is allocated.  Calls on one device are
 * serialised by the library while they enqueue work.
 */
hsmm_status_t hsmm_gemm_host(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB,
                             int64_t m, int64_t n, int64_t k, const void* alpha,
                             const void* A, int64_t lda, const void* B, int64_t ldb,
                             const void* beta, void* C, int64_t ldc, void* stream);
hsmm_status_t hsmm_gemm_host_workspace_size(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB,
                                            int64_t m, int64_t n, int64_t k, size_t* bytes);

/*
 * hsmm_gemv: y <- alpha*op(A)*x + beta*y, A m x n.
 * The matrix-vector form named beside the product (Sections 1 and 8; no
 * algorithm is given there, so this is the BLAS definition).
 *  (a, c) = (32F, 32F): FP32 data, FP32 accumulation, deterministic order.
 *  (a, c) = (8I, 32I):  INT8 A and x, exact INT32 accumulation (alpha, beta int32).
 *  incx, incy > 0 (0 or negative: INVALID_VALUE / NOT_SUPPORTED).  lda >= max(1, m).
 *  Scratch: op = N splits the columns over CTAs and needs
 *  hsmm_gemv_workspace_size() bytes of cfg->workspace for the partial sums of the
 *  splits (added in a fixed order, so results are deterministic); op = T needs none.
 */
hsmm_status_t hsmm_gemv(const hsmm_config_t* cfg, hsmm_op_t trans, int64_t m, int64_t n,
                        const void* alpha, const void* A, int64_t lda, const void* x, int64_t incx,
                        const void* beta, void* y, int64_t incy, void* stream);

/*
 * hsmm_gemv_n_noalloc: y <- alpha*A*x + beta*y (op = N only) for callers that cannot
 * allocate or keep a workspace -- for example code running inside an application
 * that owns every byte of device memory through its own arena, or a latency-bound
 * loop that must not risk the device synchronisation an allocation can cause.
 * The paper has no counterpart; this is a service entry point of the library.
 *  a = HSMM_R_32F (FP32 A, x, y; alpha, beta float) or HSMM_R_8I (INT8 A and x,
 *  INT32 y; alpha, beta int32).  It runs hsmm_gemv's own op = N kernels, so its
 *  results are bit-identical to hsmm_gemv's on the same arguments (FP32: the same
 *  deterministic order; INT8: exact), including the early-outs (alpha == 0 or n == 0
 *  gives y = beta*y without reading A or x).
 *  The split partial sums go to one fixed 16 MiB array inside the library (per GPU,
 *  held until the process exits) instead of caller memory; nothing is allocated.
 *  m > 2^21 rows (or a split count that does not fit the array) returns
 *  HSMM_STATUS_WORKSPACE_TOO_SMALL without launching anything.  All calls on a GPU
 *  share that array, so calls whose work overlaps on the GPU (other streams, other
 *  threads) race and must be serialised by the caller.  Every partial sum is written
 *  before it is read within a call, so no state carries over between calls.  The
 *  first call on each device looks up the array's address (cudaGetSymbolAddress);
 *  make that call before any stream capture.  incx, incy > 0; lda >= max(1, m).
 */
hsmm_status_t hsmm_gemv_n_noalloc(hsmm_dtype_t a, int64_t m, int64_t n, const void* alpha, const void* A,
                                  int64_t lda, const void* x, int64_t incx, const void* beta, void* y,
                                  int64_t incy, void* stream);

/* One problem of a grouped launch. A, B, C are device pointers. */
typedef struct {
    hsmm_op_t transA, transB;
    int64_t m, n, k;
    const void* A;
    const void* B;
    void* C;
    int64_t lda, ldb, ldc;
} hsmm_gemm_desc_t;

/*
 * hsmm_gemm_grouped: count independent products C_g <- alpha*op(A_g)*op(B_g) + beta*C_g
 * (alpha, beta shared) in ONE persistent launch.  Each problem is the product of
 * Eq. PRODUCT (Section 3.1); the paper's cyclic mapping (Section 6.2) runs many
 * independent systolic processes side by side, which is the same batching idea.
 * descs is a HOST array; cfg types as for hsmm_gemm (BF16, or TF32 with FAST_TF32).
 * Nothing is allocated: the per-problem TMA descriptors, problem records and tile table
 * are built on the host and written into cfg->workspace (256-byte aligned, at least
 * hsmm_gemm_grouped_workspace_size() bytes; else WORKSPACE_TOO_SMALL / NOT_SUPPORTED) by
 * kernels on `stream` whose parameters carry them (at most 32704 bytes per launch), then
 * the grouped kernel runs.  The descriptors' data travel with those launches, so the host
 * array need not outlive the call and the whole call can be captured into a CUDA graph;
 * the workspace must stay untouched until the stream has run the launch.  Problems with
 * m == 0 or n == 0 are skipped; k == 0 with m, n > 0 returns NOT_SUPPORTED (use hsmm_gemm).
 * As for hsmm_gemm, only the m x n elements of each C are touched.
 * For repeated launches of the same problems the plan API below keeps the tables on the
 * device instead.
 */
hsmm_status_t hsmm_gemm_grouped(const hsmm_config_t* cfg, int64_t count, const hsmm_gemm_desc_t* descs,
                                const void* alpha, const void* beta, void* stream);
/* Bytes of cfg->workspace hsmm_gemm_grouped needs for these problems (same checks). */
hsmm_status_t hsmm_gemm_grouped_workspace_size(const hsmm_config_t* cfg, int64_t count,
                                               const hsmm_gemm_desc_t* descs, size_t* bytes);

typedef struct hsmm_grouped_plan_s* hsmm_grouped_plan_t;

/* Validates every problem, encodes per-problem TMA descriptors and the tile
 * schedule on the host, and copies them to device memory allocated here (the one
 * allocating call of the library).  Synchronous.  The plan may be launched many
 * times and captured into CUDA graphs; the descs' pointers must stay valid. */
hsmm_status_t hsmm_grouped_plan_create(const hsmm_config_t* cfg, int64_t count,
                                       const hsmm_gemm_desc_t* descs, hsmm_grouped_plan_t* plan);
/* As hsmm_grouped_plan_create, with the choices an autotuner makes: tile width per
 * problem (tile_n_per_problem[i] = 0 for automatic, NULL = all automatic; cfg->tile_n != 0
 * overrides all) and the schedule (0: problems in the given order, 1: longest k first, so
 * that the longest tiles start in the first wave).  Widths: 128 or 256 columns; on CTA
 * pairs (the default kernel) a problem with a K-major B (transB == N) takes any multiple of
 * 32 up to 256, else INVALID_VALUE.  Automatic: such problems cut n into ceil(n / 256)
 * equal tiles rounded up to 32 columns, the others take 256 when n > 192, else 128. */
hsmm_status_t hsmm_grouped_plan_create_ex(const hsmm_config_t* cfg, int64_t count, const hsmm_gemm_desc_t* descs,
                                          const int* tile_n_per_problem, int schedule, hsmm_grouped_plan_t* plan);
/* One kernel launch on stream; allocates nothing, so it is safe inside stream capture. */
hsmm_status_t hsmm_grouped_plan_launch(hsmm_grouped_plan_t plan, const void* alpha, const void* beta,
                                       void* stream);
/* Number of tiles and the tile width chosen per problem (host array of count ints, may be NULL). */
hsmm_status_t hsmm_grouped_plan_info(hsmm_grouped_plan_t plan, int64_t* tiles, int* tile_n_per_problem);
hsmm_status_t hsmm_grouped_plan_destroy(hsmm_grouped_plan_t plan);

/*
 * hsmm_nbody: the two-array n^2 problem of Section 4, F_i = sum_j f(x_i, z_j) for i < nx,
 * j < nz, with the gravitational interaction Section 2 names as the prototype application,
 *     f(x, z) = m_z (r_z - r_x) / (|r_z - r_x|^2 + eps2)^(3/2)    (0 for r = 0, eps2 = 0).
 * x: nx bodies, z: nz bodies, each 4 floats (px, py, pz, m; the mass of x is not used),
 * out: nx x 4 floats (ax, ay, az, 0); device pointers, 16-byte aligned, caller-owned.  FP32
 * arithmetic with the hardware reciprocal square root.  x and z may be the same array.
 *  ring_p = 0: tiled schedule (z streamed through shared memory by every CTA).
 *  ring_p = 2, 4, 8 or 16: the hyper-systolic recipe of Section 4.1 with the regular bases of
 *    Definition REGULARBASE2 on clusters of ring_p CTAs: K = ring_k replicas of x (1, 2 or 4,
 *    dividing ring_p; 0 = the largest power of two <= sqrt(ring_p)), z moving K~-1 times by K
 *    cells per round of ring_p blocks of 128 bodies, back-shift of the intermediate results;
 *    T = 2K + K~ - 3 shift events per round (Theorem GAIN2).  Same result up to FP32
 *    summation order.
 * Errors: INVALID_VALUE for negative sizes, eps2 < 0, null pointers with nonzero sizes or a
 * bad ring_p / ring_k; NOT_SUPPORTED for pointers not 16-byte aligned.  Allocates nothing.
 */
hsmm_status_t hsmm_nbody(int64_t nx, int64_t nz, const float* x, const float* z, float eps2, float* out,
                         int ring_p, int ring_k, void* stream);

/*
 * hsmm_ring_gemm: C = A*B for n x n FP64 matrices by Algorithm 2 (Section 5.2.2)
 * with the block mapping of Section 6.1: p virtual processors on a ring (the p
 * CTAs of one thread-block cluster), blocks of b = n/p, K*(p/K) = p.  B is
 * pre-shifted with strides MOD(1-j, K); between the p/K blocks of K steps, A moves
 * by cshift-row^K (Eq. CSHIFT1) from CTA to CTA through distributed shared memory;
 * the K auxiliary arrays C^1..C^K are back-shifted (cshift-row^1) and summed.
 * Requirements: 1 <= p <= 16, K | p, p | n, b = n/p a multiple of 8 and <= 32,
 * lda, ldb, ldc >= n.  C^2..C^K live in workspace: (K-1) n^2 doubles
 * (hsmm_ring_workspace_size); C^1 is accumulated in C.  Allocates nothing.
 */
hsmm_status_t hsmm_ring_gemm(int p, int K, int64_t n, const double* A, int64_t lda, const double* B,
                             int64_t ldb, double* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                             void* stream);
hsmm_status_t hsmm_ring_workspace_size(int p, int K, int64_t n, size_t* bytes);

/*
 * hsmm_ozaki_split: the splitting step of the FP64-accurate form, exposed for
 * checking and for staged use.  For op(M) viewed as rows x cols (by_rows = 1: one
 * exponent per row, the treatment of A; by_rows = 0: one per column, the treatment
 * of B):
 *   e_v = smallest integer with |m| < 2^e_v over the row/column (0 if all zero),
 *   x = m 2^-e_v;  for t = 1..s: y = x 2^bits, q_t = trunc(y), x = y - q_t.
 * Outputs: expo[v] (int32, device), slices as BF16 (exact integers |q| < 2^bits),
 * laid out [t][v][w] with w (the contraction index) contiguous, a row pitch of ldq
 * elements (ldq >= len, multiple of 8; columns len..ldq-1 are written as 0) and a
 * slice pitch of `plane` elements (0: lines * ldq; else >= lines * ldq, multiple of 8).
 * M is FP64, column-major rows x cols with leading dimension ld.
 * (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012; integer-slice form.)
 */
hsmm_status_t hsmm_ozaki_split(int64_t rows, int64_t cols, const double* M, int64_t ld, int by_rows,
                               int bits, int slices, int32_t* expo, void* q, int64_t ldq, int64_t plane,
                               void* stream);

/*
 * hsmm_ozaki_slice_products: the product stage of the FP64-accurate form on its
 * own.  qa: s slices of op(A) ([t][i][k], row pitch ldq, slice pitch qa_plane),
 * qb: s slices of op(B) ([u][j][k], pitch ldq, qb_plane).  Writes, for
 * d = 2..s+1, S_d = sum_{t+u=d} QA_t QB_u^T exactly as INT32 into sd
 * ([d-2][j][i], plane pitch sd_plane).  A pitch of 0 means contiguous planes.
 * Same requirements as hsmm_gemm's OZAKI mode.
 */
hsmm_status_t hsmm_ozaki_slice_products(int64_t m, int64_t n, int64_t k, int slices, int bits, const void* qa,
                                        int64_t qa_plane, const void* qb, int64_t qb_plane, int64_t ldq,
                                        int32_t* sd, int64_t sd_plane, void* stream);

/*
 * hsmm_ozaki_recombine: C = alpha 2^(ea_i + eb_j) sum_{d=2}^{s+1} 2^(-bits d) S_d + beta C
 * (FP64; beta == 0 does not read C).  sd as written by hsmm_ozaki_slice_products
 * (plane pitch sd_plane, 0 = m*n).  Consecutive anti-diagonals are combined
 * exactly in 64-bit integers first, so each element takes one FP64 rounding per
 * group of 1 + 21/bits anti-diagonals.  alpha, beta: host doubles.
 */
hsmm_status_t hsmm_ozaki_recombine(int64_t m, int64_t n, int slices, int bits, const int32_t* sd,
                                   int64_t sd_plane, const int32_t* ea, const int32_t* eb,
                                   const double* alpha, const double* beta, double* C, int64_t ldc,
                                   void* stream);

/* Bytes of workspace hsmm_gemm / hsmm_gemv need for this configuration; 0 when none. */
hsmm_status_t hsmm_workspace_size(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB,
                                  int64_t m, int64_t n, int64_t k, size_t* bytes);
hsmm_status_t hsmm_gemv_workspace_size(const hsmm_config_t* cfg, hsmm_op_t trans, int64_t m, int64_t n,
                                       size_t* bytes);

/* Synchronizes stream, then reports (and clears) the device status word:
 * HSMM_STATUS_TIMEOUT if a bounded wait ran out since the last check,
 * HSMM_STATUS_CUDA_ERROR if the stream reported an error. */
hsmm_status_t hsmm_sync_status(void* stream);

/* Limit of every device-side wait, in nanoseconds (default 4e9).  Applies to launches made after the call. */
hsmm_status_t hsmm_set_wait_timeout_ns(uint64_t ns);

/* Failure-detection self-test: one CTA waits on an mbarrier that nothing
 * arrives on, with a limit of timeout_ns; the wait gives up, the kernel records
 * the timeout and returns.  Returns the status of hsmm_sync_status afterwards
 * (HSMM_STATUS_TIMEOUT expected). */
hsmm_status_t hsmm_selftest_timeout(uint64_t timeout_ns, void* stream);

const char* hsmm_status_string(hsmm_status_t status);
/* The last CUDA error code seen by the library on this thread (cudaError_t value). */
int hsmm_last_cuda_error(void);
/* A one-line reason for the last failing status returned on this host thread
 * (which check failed, with the offending values); "" if none yet. */
const char* hsmm_last_error_detail(void);
/* Library version as 10000*major + 100*minor + patch. */
int hsmm_version(void);
/* Number of kernels launched by the library since the last reset (host counter). */
int64_t hsmm_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif /* HSMM_H */
