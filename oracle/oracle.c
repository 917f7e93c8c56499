/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct CPU implementations of what the hsmm hot path
 * computes, written from the paper (Lippert, Petkov, Palazzari, Schilling,
 * "Hyper-Systolic Matrix Multiplication") and, for the precision form, from the
 * published error-free splitting of Ozaki, Ogita, Oishi and Rump.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load this
 * library.  It shares no code, header or constant with the CUDA path.
 *
 * Conventions: column-major storage (BLAS), 0-based indices in code; the paper's
 * 1-based formulas are restated beside each use.  All floating point is FP64;
 * the library is compiled with -ffp-contract=off so that a*b+c is two roundings
 * on every host (the only fused operation is the explicit fma() of TwoProduct).
 *
 * Parity status of each function (see the tests that pin it):
 *   ora_gemm_f64 / ora_gemm_rows_f64 ... pinned (brute force on integers, A*I, transpose identity)
 *   ora_gemm_i64 ......................... pinned (Python big-int brute force)
 *   ora_dot2_rows ........................ pinned (exact rational arithmetic, Dot2 error bound)
 *   ora_gemv_f64 / ora_gemv_i8 ........... pinned (brute force, exact integers)
 *   ora_ring_systolic / ora_ring_hsmm .... pinned (bit-exact vs brute force on integers for all p<=16,
 *                                          K|p; visit counts; shift counts of Theorem GAIN3)
 *   ora_regular_base ..................... pinned (h-range theorem, by brute-force coverage)
 *   ora_ozaki_split / ora_ozaki_gemm ..... pinned (exact reconstruction with rationals; exact product
 *                                          for integer inputs; truncation error bound vs Dot2)
 *   ora_zgemm ............................ pinned (Python big-int brute force of the complex product for
 *                                          every op pair; real special case bitwise; (AB)^H = B^H A^H
 *                                          bitwise; rational error bound)
 *   ora_nbody_direct ..................... pinned (exact integer interaction vs Python brute force; two-body
 *                                          closed form; momentum conservation sum_i m_i a_i = 0)
 *   ora_nbody_hsys ....................... pinned (every block pair met exactly once; shift counts of
 *                                          Theorem GAIN2; exact integer interaction equals the direct sum;
 *                                          a planted non-covering stride fails)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CM(M, i, j, ld) ((M)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)])

int ora_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int is_n(char t) { return t == 'N' || t == 'n'; }

/* element (i,j) of op(M), op = identity ('N') or transpose ('T') */
static double op_f64(const double* M, int64_t ld, char t, int64_t i, int64_t j) {
    return is_n(t) ? CM(M, i, j, ld) : CM(M, j, i, ld);
}

/* ---------------------------------------------------------------------------
 * Eq. PRODUCT (Section 3.1): c_ij = sum_k a_ik b_kj.  The sum runs in the
 * natural order k = 0, 1, ..., K-1, one product and one addition per step.
 * BLAS semantics around it: C <- alpha*op(A)*op(B) + beta*C; beta == 0 means C
 * is not read; alpha == 0 or k == 0 means op(A), op(B) are not read.
 * ------------------------------------------------------------------------- */
void ora_gemm_f64(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb,
                  double beta, double* C, int64_t ldc) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            if (alpha != 0.0)
                for (int64_t p = 0; p < k; ++p) s += op_f64(A, lda, ta, i, p) * op_f64(B, ldb, tb, p, j);
            double c = (alpha != 0.0) ? alpha * s : 0.0;
            if (beta != 0.0) c += beta * CM(C, i, j, ldc);
            CM(C, i, j, ldc) = c;
        }
    }
}

/* ---------------------------------------------------------------------------
 * The complex product (Section 7 measures the method on real and on complex
 * data): c_ij = sum_k a_ik b_kj over complex numbers, with
 *   (x + iy)(u + iv) = (xu - yv) + i(xv + yu),
 * each product formed in that order and both sums running k = 0, 1, ..., K-1.
 * Storage: interleaved (re, im) doubles, column-major, ld in complex elements.
 * op: 'N' identity, 'T' transpose, 'C' conjugate transpose.
 * C <- alpha op(A) op(B) + beta C with complex alpha = (alpha[0], alpha[1]) and
 * beta; beta == 0 (both parts) means C is not read.
 * ------------------------------------------------------------------------- */
static void op_z(const double* M, int64_t ld, char t, int64_t i, int64_t j, double* re, double* im) {
    const double* e = is_n(t) ? &M[2 * (i + j * ld)] : &M[2 * (j + i * ld)];
    *re = e[0];
    *im = (t == 'C' || t == 'c') ? -e[1] : e[1];
}

void ora_zgemm(char ta, char tb, int64_t m, int64_t n, int64_t k, const double* alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb,
               const double* beta, double* C, int64_t ldc) {
    const int read_c = beta[0] != 0.0 || beta[1] != 0.0;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double sr = 0.0, si = 0.0;
            for (int64_t p = 0; p < k; ++p) {
                double ar, ai, br, bi;
                op_z(A, lda, ta, i, p, &ar, &ai);
                op_z(B, ldb, tb, p, j, &br, &bi);
                const double pr = ar * br - ai * bi;
                const double pi = ar * bi + ai * br;
                sr += pr;
                si += pi;
            }
            double vr = alpha[0] * sr - alpha[1] * si;
            double vi = alpha[0] * si + alpha[1] * sr;
            double* c = &C[2 * (i + j * ldc)];
            if (read_c) {
                const double cr = beta[0] * c[0] - beta[1] * c[1];
                const double ci = beta[0] * c[1] + beta[1] * c[0];
                vr += cr;
                vi += ci;
            }
            c[0] = vr;
            c[1] = vi;
        }
    }
}

/* Exact integer form of Eq. PRODUCT: C = op(A) op(B) in int64 (callers keep the
 * inputs small enough that no partial sum leaves int64). */
void ora_gemm_i64(char ta, char tb, int64_t m, int64_t n, int64_t k,
                  const int64_t* A, int64_t lda, const int64_t* B, int64_t ldb,
                  int64_t* C, int64_t ldc) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            int64_t s = 0;
            for (int64_t p = 0; p < k; ++p) {
                int64_t a = is_n(ta) ? CM(A, i, p, lda) : CM(A, p, i, lda);
                int64_t b = is_n(tb) ? CM(B, p, j, ldb) : CM(B, j, p, ldb);
                s += a * b;
            }
            CM(C, i, j, ldc) = s;
        }
    }
}

/* Selected rows of op(A)*op(B), Eq. PRODUCT with the same sequential k order as
 * ora_gemm_f64 (the operands are only gathered into contiguous buffers first; the
 * arithmetic is unchanged).  out is nrows x n, row-major. */
void ora_gemm_rows_f64(char ta, char tb, int64_t m, int64_t n, int64_t k,
                       const double* A, int64_t lda, const double* B, int64_t ldb,
                       int64_t nrows, const int64_t* rows, double* out) {
    (void)m;
    double* ar = (double*)malloc(sizeof(double) * (size_t)(nrows * k > 0 ? nrows * k : 1));
    for (int64_t r = 0; r < nrows; ++r)
        for (int64_t p = 0; p < k; ++p) ar[r * k + p] = op_f64(A, lda, ta, rows[r], p);
    #pragma omp parallel
    {
        double* bc = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        #pragma omp for schedule(dynamic, 8)
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t p = 0; p < k; ++p) bc[p] = op_f64(B, ldb, tb, p, j);
            for (int64_t r = 0; r < nrows; ++r) {
                const double* a = ar + r * k;
                double s = 0.0;
                for (int64_t p = 0; p < k; ++p) s += a[p] * bc[p];
                out[r * n + j] = s;
            }
        }
        free(bc);
    }
    free(ar);
}

/* ---------------------------------------------------------------------------
 * Accurate reference dot products: Dot2 of Ogita, Rump and Oishi ("Accurate sum
 * and dot product", SIAM J. Sci. Comput. 26(6), 2005, Algorithm 5.3), i.e. the
 * dot product computed as if in twice the working precision:
 *   |dot2 - x'y| <= u |x'y| + gamma_n^2 |x|'|y|.
 * TwoProduct uses fma; TwoSum is Knuth's branch-free form.
 * ------------------------------------------------------------------------- */
static void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static double dot2(const double* x, const double* y, int64_t n) {
    if (n <= 0) return 0.0;
    double p = x[0] * y[0];
    double s = fma(x[0], y[0], -p);
    for (int64_t i = 1; i < n; ++i) {
        double h = x[i] * y[i];
        double r = fma(x[i], y[i], -h);
        double q;
        two_sum(p, h, &p, &q);
        s = s + (q + r);
    }
    return p + s;
}

void ora_dot2_rows(char ta, char tb, int64_t m, int64_t n, int64_t k,
                   const double* A, int64_t lda, const double* B, int64_t ldb,
                   int64_t nrows, const int64_t* rows, double* out) {
    (void)m;
    double* ar = (double*)malloc(sizeof(double) * (size_t)(nrows * k > 0 ? nrows * k : 1));
    for (int64_t r = 0; r < nrows; ++r)
        for (int64_t p = 0; p < k; ++p) ar[r * k + p] = op_f64(A, lda, ta, rows[r], p);
    #pragma omp parallel
    {
        double* bc = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        #pragma omp for schedule(dynamic, 8)
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t p = 0; p < k; ++p) bc[p] = op_f64(B, ldb, tb, p, j);
            for (int64_t r = 0; r < nrows; ++r) out[r * n + j] = dot2(ar + r * k, bc, k);
        }
        free(bc);
    }
    free(ar);
}

/* Plain vector dot2, exposed for its own pin. */
double ora_dot2(const double* x, const double* y, int64_t n) { return dot2(x, y, n); }

/* ---------------------------------------------------------------------------
 * Matrix-vector form (the paper names it as a capability of the same alignment,
 * Section 8; no algorithm is printed, so this is the definition):
 *   y <- alpha*op(A)*x + beta*y,  op(A) = A (m x n) or A^T.
 * Increments must be positive.
 * ------------------------------------------------------------------------- */
void ora_gemv_f64(char t, int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                  const double* x, int64_t incx, double beta, double* y, int64_t incy) {
    int64_t leny = is_n(t) ? m : n, lenx = is_n(t) ? n : m;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < leny; ++i) {
        double s = 0.0;
        if (alpha != 0.0)
            for (int64_t j = 0; j < lenx; ++j) s += op_f64(A, lda, t, i, j) * x[j * incx];
        double v = (alpha != 0.0) ? alpha * s : 0.0;
        if (beta != 0.0) v += beta * y[i * incy];
        y[i * incy] = v;
    }
}

/* Exact integer matrix-vector product for INT8 data; the result is returned in
 * int64 so that the caller can check that it fits the INT32 of the GPU path. */
void ora_gemv_i8(char t, int64_t m, int64_t n, int64_t alpha, const int8_t* A, int64_t lda,
                 const int8_t* x, int64_t incx, int64_t beta, const int32_t* y_in, int64_t incy,
                 int64_t* y_out) {
    int64_t leny = is_n(t) ? m : n, lenx = is_n(t) ? n : m;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < leny; ++i) {
        int64_t s = 0;
        for (int64_t j = 0; j < lenx; ++j) {
            int64_t a = is_n(t) ? (int64_t)CM(A, i, j, lda) : (int64_t)CM(A, j, i, lda);
            s += a * (int64_t)x[j * incx];
        }
        int64_t v = alpha * s;
        if (beta != 0) v += beta * (int64_t)y_in[i * incy];
        y_out[i] = v;
    }
}

/* ===========================================================================
 * The paper's ring algorithms, simulated over p virtual processors.
 *
 * Block mapping (Section 6.1): the n x n matrices (n = p*b) are cut into p x p
 * blocks of b x b; a "matrix element" of the algorithms is one such block and
 * the product of two elements is the local block product (x), here a plain
 * triple loop.  Elementary blocks stay in normal order; only the p x p block
 * system is skewed (Section 7).
 *
 * Skew order (Section 3.2.1 / 3.3.1, reading c1): processor i (1..p) holds
 * column i, rotated so that slot l holds element ((l+i-2) mod p)+1 of that
 * column; slot 1 of processor i holds the diagonal element (i,i).  0-based:
 *   st[i][l] = M[(l+i) mod p][i].
 *
 * cshift-row (Eq. CSHIFT1): cshift-row^k(a_{j,i}) = a_{j,(i+k-1+n) mod n + 1},
 * i.e. processor i receives from processor i+k: 0-based dst[i] = src[(i+k) mod p].
 * This is the only operation that moves data between processors.
 * cshift-col: cshift-col^k(a_{j,i}) = a_{(j+k-1+n) mod n + 1, i}, an in-cell
 * re-addressing: 0-based slot l reads slot (l+k) mod p.
 * ========================================================================= */

typedef struct {
    int p, b;
    double* data;   /* p processors x p slots x b*b doubles */
    int* tag_r;     /* origin block row of each stored element (-1 = none)    */
    int* tag_c;     /* origin block column                                    */
} ring_arr;

static size_t blk_sz(const ring_arr* x) { return (size_t)x->b * (size_t)x->b; }
static double* blk(ring_arr* x, int i, int l) { return x->data + ((size_t)i * x->p + l) * blk_sz(x); }
static int ti(const ring_arr* x, int i, int l) { return i * x->p + l; }

static void ring_alloc(ring_arr* x, int p, int b) {
    x->p = p; x->b = b;
    x->data = (double*)calloc((size_t)p * p * b * b, sizeof(double));
    x->tag_r = (int*)malloc(sizeof(int) * p * p);
    x->tag_c = (int*)malloc(sizeof(int) * p * p);
    for (int q = 0; q < p * p; ++q) { x->tag_r[q] = -1; x->tag_c[q] = -1; }
}

static void ring_free(ring_arr* x) { free(x->data); free(x->tag_r); free(x->tag_c); }

static int pmod(int a, int p) { int r = a % p; return r < 0 ? r + p : r; }

/* Skew order: the block row held by processor i (0-based) in slot l. */
int ora_skew_row(int p, int i, int l) { return pmod(l + i, p); }

/* load an n x n column-major matrix into skew order, tagging every block */
static void ring_skew_load(ring_arr* x, const double* M, int64_t ldm) {
    int p = x->p, b = x->b;
    for (int i = 0; i < p; ++i)
        for (int l = 0; l < p; ++l) {
            int R = ora_skew_row(p, i, l), Q = i;
            double* d = blk(x, i, l);
            for (int c = 0; c < b; ++c)
                for (int r = 0; r < b; ++r) d[r + (size_t)c * b] = CM(M, (int64_t)R * b + r, (int64_t)Q * b + c, ldm);
            x->tag_r[ti(x, i, l)] = R; x->tag_c[ti(x, i, l)] = Q;
        }
}

/* store from skew order back to normal order */
static void ring_skew_store(const ring_arr* x, double* M, int64_t ldm) {
    int p = x->p, b = x->b;
    for (int i = 0; i < p; ++i)
        for (int l = 0; l < p; ++l) {
            int R = ora_skew_row(p, i, l), Q = i;
            const double* d = x->data + ((size_t)i * p + l) * blk_sz(x);
            for (int c = 0; c < b; ++c)
                for (int r = 0; r < b; ++r) CM(M, (int64_t)R * b + r, (int64_t)Q * b + c, ldm) = d[r + (size_t)c * b];
        }
}

/* cshift-row^k applied to whole slot rows: dst[i][l] = src[(i+k) mod p][l]
 * for the slots listed (all slots when only_slot < 0). Returns blocks moved. */
static int64_t cshift_row(ring_arr* x, int k, int only_slot) {
    int p = x->p;
    if (pmod(k, p) == 0) return 0;
    ring_arr t; ring_alloc(&t, p, x->b);
    memcpy(t.data, x->data, sizeof(double) * (size_t)p * p * blk_sz(x));
    memcpy(t.tag_r, x->tag_r, sizeof(int) * p * p);
    memcpy(t.tag_c, x->tag_c, sizeof(int) * p * p);
    int64_t moved = 0;
    for (int i = 0; i < p; ++i)
        for (int l = 0; l < p; ++l) {
            if (only_slot >= 0 && l != only_slot) continue;
            int src = pmod(i + k, p);
            memcpy(blk(x, i, l), blk(&t, src, l), sizeof(double) * blk_sz(x));
            x->tag_r[ti(x, i, l)] = t.tag_r[ti(&t, src, l)];
            x->tag_c[ti(x, i, l)] = t.tag_c[ti(&t, src, l)];
            ++moved;
        }
    ring_free(&t);
    return moved;
}

/* cshift-col^k as an address: slot l of a processor reads slot (l+k) mod p */
static int cshift_col_slot(int l, int k, int p) { return pmod(l + k, p); }

/* local block product (x): c += a * b on b x b blocks, sequential inner index */
static void block_mac(double* c, const double* a, const double* bb, int b) {
    for (int col = 0; col < b; ++col)
        for (int row = 0; row < b; ++row) {
            double s = c[row + (size_t)col * b];
            for (int q = 0; q < b; ++q) s += a[row + (size_t)q * b] * bb[q + (size_t)col * b];
            c[row + (size_t)col * b] = s;
        }
}

/* One accumulation c^l[i][n] += A-element (x) B-element with bookkeeping:
 * the A element's column must equal the B element's row (same summation index),
 * the aux-C slot keeps one destination (row of A, column of B), and the visit
 * count of (C row, C column, summation index) is incremented. */
static void ring_mac(ring_arr* C, int i, int n, ring_arr* A, int ia, int la, ring_arr* B, int ib, int lb,
                     int* cnt, int64_t* tag_errors) {
    int p = C->p;
    int ar = A->tag_r[ti(A, ia, la)], ac = A->tag_c[ti(A, ia, la)];
    int br = B->tag_r[ti(B, ib, lb)], bc = B->tag_c[ti(B, ib, lb)];
    if (ac != br) ++*tag_errors;
    int* cr = &C->tag_r[ti(C, i, n)];
    int* cc = &C->tag_c[ti(C, i, n)];
    if (*cr < 0) { *cr = ar; *cc = bc; }
    else if (*cr != ar || *cc != bc) ++*tag_errors;
    if (cnt && ar >= 0 && bc >= 0 && ac >= 0) cnt[((size_t)ar * p + bc) * p + ac] += 1;
    block_mac(blk(C, i, n), blk(A, ia, la), blk(B, ib, lb), C->b);
}

/* c_dst += cshift-row^1(c_src) with destination-tag check; returns blocks moved */
static int64_t ring_backshift_add(ring_arr* dst, ring_arr* src, int64_t* tag_errors) {
    int p = dst->p;
    int64_t moved = cshift_row(src, 1, -1);
    for (int i = 0; i < p; ++i)
        for (int l = 0; l < p; ++l) {
            int sr = src->tag_r[ti(src, i, l)], sc = src->tag_c[ti(src, i, l)];
            int* dr = &dst->tag_r[ti(dst, i, l)];
            int* dc = &dst->tag_c[ti(dst, i, l)];
            if (sr >= 0) {
                if (*dr < 0) { *dr = sr; *dc = sc; }
                else if (*dr != sr || *dc != sc) ++*tag_errors;
            }
            double* d = blk(dst, i, l);
            const double* s = blk(src, i, l);
            for (size_t e = 0; e < blk_sz(dst); ++e) d[e] += s[e];
        }
    return moved;
}

/* every stored C element must end in the skew slot of the block it belongs to */
static int64_t ring_check_home(const ring_arr* c) {
    int p = c->p;
    int64_t bad = 0;
    for (int i = 0; i < p; ++i)
        for (int l = 0; l < p; ++l)
            if (c->tag_r[ti(c, i, l)] != pmod(l + i, p) || c->tag_c[ti(c, i, l)] != i) ++bad;
    return bad;
}

/* stats layout (int64[8]):
 *  [0] B rows moved by the pre-shift          [1] A shift events (cshift-row of all of A)
 *  [2] C back-shift events                     [3] blocks moved between processors in total
 *  [4] bookkeeping errors (wrong pairing)      [5] 1 if A ended where the paper says it ends
 *  [6] B pre-shift events (1 if any row moved) [7] shift events in total (T)              */

/* Algorithm 1 (SYSTOLIC): p steps; in step j every processor i accumulates
 *   c_{l,i} += cshift-col^{1-j}(a_{l,i}) b_{j,i}   for all slots l,
 * then A moves one processor to the left (cshift-row^1).  C = A*B for n = p*b. */
int ora_ring_systolic(int p, int b, const double* A, const double* B, double* C, int64_t* stats, int* cnt) {
    if (p <= 0 || b <= 0) return -1;
    int64_t n = (int64_t)p * b;
    ring_arr a, bb, c;
    ring_alloc(&a, p, b); ring_alloc(&bb, p, b); ring_alloc(&c, p, b);
    ring_skew_load(&a, A, n); ring_skew_load(&bb, B, n);
    int64_t st[8] = {0};
    if (cnt) memset(cnt, 0, sizeof(int) * (size_t)p * p * p);
    ring_arr a0; ring_alloc(&a0, p, b); ring_skew_load(&a0, A, n);
    for (int j = 1; j <= p; ++j) {
        for (int i = 0; i < p; ++i)
            for (int l = 1; l <= p; ++l) {
                int src = cshift_col_slot(l - 1, 1 - j, p);
                ring_mac(&c, i, l - 1, &a, i, src, &bb, i, j - 1, cnt, &st[4]);
            }
        st[3] += cshift_row(&a, 1, -1);
        st[1] += 1;
    }
    /* after p unit shifts A is back where it started */
    st[5] = memcmp(a.data, a0.data, sizeof(double) * (size_t)p * p * b * b) == 0;
    st[7] = st[1];
    st[4] += ring_check_home(&c);
    ring_skew_store(&c, C, n);
    if (stats) memcpy(stats, st, sizeof(st));
    ring_free(&a); ring_free(&bb); ring_free(&c); ring_free(&a0);
    return 0;
}

/* Fortran MOD: the remainder takes the sign of the dividend (reading c2). */
static int fortran_mod(int a, int k) { return a - k * (a / k); }

/* Stride of the pre-shift of row j (1-based) of B in Algorithm 2: MOD(1-j, K).
 * planted != 0 gives the non-negative modulus instead (a deliberate mistake,
 * used only by a negative test). */
int ora_preshift_stride(int j, int K, int planted) {
    return planted ? pmod(1 - j, K) : fortran_mod(1 - j, K);
}

/* Algorithm 2 (HYPER-SYSTOLIC) with K*Kt = p:
 *  1. pre-shift of B: row j (1-based) of every processor column moves with
 *     stride MOD(1-j, K);
 *  2. Kt blocks of K steps: in step l of block jb (g = (jb-1)K + l)
 *       c^l_{n,i} += cshift-col^{1-g}(a_{n,i}) b_{g,i}   for every slot n,
 *     and after every block but the last, A <- cshift-row^K(A);
 *  3. back-shift: for j = 1..K-1, c^{K-j} += cshift-row^1(c^{K-j+1}).
 * The result is c^1 in skew order.  flags bit 0 plants the non-negative
 * reading of the pre-shift modulus (used only by a negative test). */
int ora_ring_hsmm(int p, int K, int b, const double* A, const double* B, double* C,
                  int64_t* stats, int* cnt, int flags) {
    if (p <= 0 || b <= 0 || K <= 0 || p % K != 0) return -1;
    int Kt = p / K;
    int64_t n = (int64_t)p * b;
    ring_arr a, bb, a0;
    ring_alloc(&a, p, b); ring_alloc(&bb, p, b); ring_alloc(&a0, p, b);
    ring_skew_load(&a, A, n); ring_skew_load(&bb, B, n); ring_skew_load(&a0, A, n);
    ring_arr* c = (ring_arr*)malloc(sizeof(ring_arr) * (size_t)K);
    for (int l = 0; l < K; ++l) ring_alloc(&c[l], p, b);
    int64_t st[8] = {0};
    if (cnt) memset(cnt, 0, sizeof(int) * (size_t)p * p * p);

    /* 1. pre-shift of B */
    for (int j = 1; j <= p; ++j) {
        int sigma = ora_preshift_stride(j, K, flags & 1);
        int64_t mv = cshift_row(&bb, sigma, j - 1);
        if (mv) { st[0] += 1; st[3] += mv; }
    }
    st[6] = st[0] > 0;

    /* 2. multiplication, with shifts of A by K between blocks */
    for (int jb = 1; jb <= Kt; ++jb) {
        for (int l = 1; l <= K; ++l) {
            int g = (jb - 1) * K + l;
            for (int i = 0; i < p; ++i)
                for (int nn = 1; nn <= p; ++nn) {
                    int src = cshift_col_slot(nn - 1, 1 - g, p);
                    ring_mac(&c[l - 1], i, nn - 1, &a, i, src, &bb, i, g - 1, cnt, &st[4]);
                }
        }
        if (jb < Kt) { st[3] += cshift_row(&a, K, -1); st[1] += 1; }
    }

    /* 3. back-shift and accumulation */
    for (int j = 1; j <= K - 1; ++j) {
        st[3] += ring_backshift_add(&c[K - j - 1], &c[K - j], &st[4]);
        st[2] += 1;
    }

    /* A ends shifted by (Kt-1)*K = p-K positions (reading c6) */
    ring_arr ae; ring_alloc(&ae, p, b); ring_skew_load(&ae, A, n);
    cshift_row(&ae, p - K, -1);
    st[5] = memcmp(a.data, ae.data, sizeof(double) * (size_t)p * p * b * b) == 0;
    ring_free(&ae);
    st[7] = st[6] + st[1] + st[2];
    st[4] += ring_check_home(&c[0]);

    ring_skew_store(&c[0], C, n);
    if (stats) memcpy(stats, st, sizeof(st));
    for (int l = 0; l < K; ++l) ring_free(&c[l]);
    free(c);
    ring_free(&a); ring_free(&bb); ring_free(&a0);
    return 0;
}

/* Regular bases of Section 5.2.1 (three-base form used by Algorithm 2):
 *   A_{Kt-1} = (0, K, ..., K)   (Kt entries)
 *   B_{K-1}  = (0, -1, ..., -1) (K entries)
 *   C_{K-1}  = (0, 1, ..., 1)   (K entries)
 * and the two-array regular bases of Definition REGULARBASE2 (Section 4.4):
 *   A2_{K-1} = (0, 1, ..., 1) (K entries), B2_{Kt-1} = (0, K, ..., K) (Kt entries). */
int ora_regular_base(int p, int K, int* a, int* bstr, int* c, int* a2, int* b2) {
    if (p <= 0 || K <= 0 || p % K != 0) return -1;
    int Kt = p / K;
    for (int t = 0; t < Kt; ++t) a[t] = t == 0 ? 0 : K;
    for (int t = 0; t < K; ++t) bstr[t] = t == 0 ? 0 : -1;
    for (int t = 0; t < K; ++t) c[t] = t == 0 ? 0 : 1;
    for (int t = 0; t < K; ++t) a2[t] = t == 0 ? 0 : 1;
    for (int t = 0; t < Kt; ++t) b2[t] = t == 0 ? 0 : K;
    return 0;
}

/* ===========================================================================
 * The two-array n^2 problem (Section 4): F_i = sum_j f(x_i, z_j), with the
 * gravitational n-body interaction that Section 2 cites as the prototype:
 *   f(x, z) = m_z (r_z - r_x) / (|r_z - r_x|^2 + eps2)^(3/2),
 * bodies stored as 4 doubles (px, py, pz, m; the mass of x is not used), results
 * as 3 doubles; a pair at distance 0 with eps2 = 0 (a body with itself) contributes 0.
 * kind 1 is the integer-valued interaction f(x, z) = m_z (r_z - r_x)
 * (exact in FP64 for small integers) that shows whether every pair was met once.
 * ========================================================================= */
static void pair_f(int kind, const double* x, const double* z, double eps2, double* f) {
    const double dx = z[0] - x[0], dy = z[1] - x[1], dz = z[2] - x[2];
    if (kind == 1) {
        f[0] = z[3] * dx;
        f[1] = z[3] * dy;
        f[2] = z[3] * dz;
        return;
    }
    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
    const double s = r2 > 0.0 ? z[3] / (r2 * sqrt(r2)) : 0.0;   /* coincident bodies (eps2 = 0): no force */
    f[0] = s * dx;
    f[1] = s * dy;
    f[2] = s * dz;
}

/* direct sum, j = 0, 1, ... in order */
void ora_nbody_direct(int kind, int64_t nx, int64_t nz, const double* x, const double* z, double eps2, double* F) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nx; ++i) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, f[3];
        for (int64_t j = 0; j < nz; ++j) {
            pair_f(kind, &x[4 * i], &z[4 * j], eps2, f);
            a0 += f[0];
            a1 += f[1];
            a2 += f[2];
        }
        F[3 * i] = a0;
        F[3 * i + 1] = a1;
        F[3 * i + 2] = a2;
    }
}

/* cshift on p cells of block indices: cell c receives the entry of cell c + k (Eq. CSHIFT1) */
static void cshift_idx(int p, const int* in, int k, int* out) {
    for (int c = 0; c < p; ++c) out[c] = in[((c + k) % p + p) % p];
}

/* The hyper-systolic recipe (Section 4.1) on p cells with the regular bases of Definition
 * REGULARBASE2, A = (0, 1, ..., 1) (K-1 strides 1) and B = (0, K, ..., K) (K~-1 strides K),
 * K K~ = p, block mapping (cell c holds block c of n/p bodies of x and of z):
 *   replicas    x^_t = cshift^1(x^_(t-1)), t = 1..K-1: cell c then holds block c+t of x;
 *   z phase     z^_s = cshift^K(z^_(s-1)), s = 1..K~-1; at every z^_s (s = 0 included) each
 *               cell adds f over its blocks of x^_t and z^_s into y^_t, t = 0..K-1;
 *   back-shift  the collector y starts as y^_(K-1); K-1 times it moves one cell against the
 *               replica shifts (cshift^-1) and adds y^_t, t = K-2..0; cell c then holds F of
 *               block c.
 * zstride != 0 replaces the z stride K (a planted non-covering base for the tests).
 * cnt[xb * p + zb] counts the block pairs met; shifts = {replica, z, back} shift events.
 * Returns -1 for an invalid p, K or n. */
int ora_nbody_hsys(int kind, int p, int K, int zstride, int64_t n, const double* x, const double* z, double eps2,
                   double* F, int* cnt, int* shifts) {
    if (p <= 0 || K <= 0 || p % K != 0 || n % p != 0) return -1;
    const int Kt = p / K, zs = zstride ? zstride : K;
    const int64_t nb = n / p;
    int* xidx = malloc(sizeof(int) * (size_t)K * (size_t)p);
    int* zidx = malloc(sizeof(int) * (size_t)p);
    int* tmp = malloc(sizeof(int) * (size_t)p);
    double* yhat = calloc((size_t)K * (size_t)n * 3, sizeof(double));   /* [t][cell][element][3] */
    double* y = malloc(sizeof(double) * (size_t)n * 3);
    double* ys = malloc(sizeof(double) * (size_t)n * 3);
    if (!xidx || !zidx || !tmp || !yhat || !y || !ys) return -2;
    memset(cnt, 0, sizeof(int) * (size_t)p * (size_t)p);
    shifts[0] = shifts[1] = shifts[2] = 0;
    for (int c = 0; c < p; ++c) xidx[c] = c;
    for (int t = 1; t < K; ++t) {
        cshift_idx(p, &xidx[(t - 1) * p], 1, &xidx[t * p]);
        ++shifts[0];
    }
    for (int c = 0; c < p; ++c) zidx[c] = c;
    for (int sz = 0; sz < Kt; ++sz) {
        if (sz > 0) {
            cshift_idx(p, zidx, zs, tmp);
            memcpy(zidx, tmp, sizeof(int) * (size_t)p);
            ++shifts[1];
        }
        for (int t = 0; t < K; ++t)
            for (int c = 0; c < p; ++c) {
                const int xb = xidx[t * p + c], zb = zidx[c];
                ++cnt[xb * p + zb];
                for (int64_t e = 0; e < nb; ++e) {
                    double* acc = &yhat[(((size_t)t * p + c) * nb + e) * 3];
                    const double* xe = &x[4 * ((int64_t)xb * nb + e)];
                    for (int64_t j = 0; j < nb; ++j) {
                        double f[3];
                        pair_f(kind, xe, &z[4 * ((int64_t)zb * nb + j)], eps2, f);
                        acc[0] += f[0];
                        acc[1] += f[1];
                        acc[2] += f[2];
                    }
                }
            }
    }
    /* back-shift phase: y <- y^_(K-1); then y <- cshift^-1(y) + y^_t for t = K-2..0 */
    memcpy(y, &yhat[(size_t)(K - 1) * n * 3], sizeof(double) * (size_t)n * 3);
    for (int t = K - 2; t >= 0; --t) {
        for (int c = 0; c < p; ++c) {
            const int from = ((c - 1) % p + p) % p;
            memcpy(&ys[(size_t)c * nb * 3], &y[(size_t)from * nb * 3], sizeof(double) * (size_t)nb * 3);
        }
        ++shifts[2];
        for (int64_t q = 0; q < n * 3; ++q) y[q] = ys[q] + yhat[(size_t)t * n * 3 + q];
    }
    /* cell c holds block c: write back in body order */
    memcpy(F, y, sizeof(double) * (size_t)n * 3);
    free(xidx); free(zidx); free(tmp); free(yhat); free(y); free(ys);
    return 0;
}

/* ===========================================================================
 * Precision form: error-free splitting (Ozaki, Ogita, Oishi, Rump, "Error-free
 * transformations of matrix multiplication by using fast routines of matrix
 * multiplication and its applications", Numer. Algorithms 59, 2012), in the
 * fixed-point integer form (every slice is an integer matrix scaled by a power
 * of two per row of A / per column of B).
 *
 *   e_r = smallest integer with |m_{r,j}| < 2^{e_r} for all j (0 for a zero row)
 *   x = m * 2^{-e_r}  (exact, |x| < 1)
 *   for t = 1..s:  y = x * 2^beta;  q_t = trunc(y);  x = y - q_t   (all exact)
 *   m = 2^{e_r} ( sum_t q_t 2^{-beta t} + x_s 2^{-beta s} ),  |q_t| <= 2^beta - 1.
 * ========================================================================= */
static int row_exponent(double mx) {
    if (mx == 0.0) return 0;
    int e;
    frexp(mx, &e);          /* mx = f 2^e, f in [0.5, 1): mx < 2^e */
    return e;
}

/* by_rows = 1: one exponent per row r (the splitting of A);
 * by_rows = 0: one exponent per column (the splitting of B).
 * slices: s blocks of rows x cols, column-major with ld = rows. */
void ora_ozaki_split(int64_t rows, int64_t cols, const double* M, int64_t ld, int by_rows,
                     int beta, int s, int32_t* expo, double* slices) {
    int64_t nvec = by_rows ? rows : cols, len = by_rows ? cols : rows;
    for (int64_t v = 0; v < nvec; ++v) {
        double mx = 0.0;
        for (int64_t w = 0; w < len; ++w) {
            double val = by_rows ? CM(M, v, w, ld) : CM(M, w, v, ld);
            if (fabs(val) > mx) mx = fabs(val);
        }
        int e = row_exponent(mx);
        expo[v] = e;
        for (int64_t w = 0; w < len; ++w) {
            int64_t r = by_rows ? v : w, c = by_rows ? w : v;
            double x = ldexp(CM(M, r, c, ld), -e);
            for (int t = 0; t < s; ++t) {
                double y = ldexp(x, beta);
                double q = trunc(y);
                x = y - q;
                slices[(int64_t)t * rows * cols + r + c * rows] = q;
            }
        }
    }
}

/* Exact anti-diagonal sums of the slice products, S_d = sum_{t+u=d} Q^A_t Q^B_u
 * for d = 2..s+1, as int64, layout [d-2][j][i] (column-major per d); the inputs
 * are already split (qa: s x m x k, [t] col-major m x k; qb: s x k x n). */
void ora_ozaki_diagonals(int64_t m, int64_t n, int64_t k, int s, const double* qa, const double* qb, int64_t* sd) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j)
        for (int d = 2; d <= s + 1; ++d)
            for (int64_t i = 0; i < m; ++i) {
                int64_t acc = 0;
                for (int t = 1; t <= s; ++t) {
                    int u = d - t;
                    if (u < 1 || u > s) continue;
                    const double* xa = qa + (int64_t)(t - 1) * m * k;
                    const double* xb = qb + (int64_t)(u - 1) * k * n;
                    for (int64_t p2 = 0; p2 < k; ++p2) acc += (int64_t)xa[i + p2 * m] * (int64_t)xb[p2 + j * k];
                }
                sd[(int64_t)(d - 2) * m * n + i + j * m] = acc;
            }
}

/* Full emulation of the FP64-accurate product:
 *   S_d = sum over slice pairs (t,u), t+u = d, 2 <= d <= s+1, of Q^A_t Q^B_u
 *         (exact integer products in int64);
 *   c_ij = 2^{e_i + f_j} * sum_{d = s+1 down to 2} 2^{-beta d} S_d(i,j)   (FP64, smallest terms first)
 *   C <- alpha*c + beta*C.
 * Operands follow op(A) (m x k) and op(B) (k x n). */
void ora_ozaki_gemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                    int64_t ldc, int beta_bits, int s) {
    /* explicit op(A), op(B) copies (column-major, exact) */
    double* Ao = (double*)malloc(sizeof(double) * (size_t)(m * k > 0 ? m * k : 1));
    double* Bo = (double*)malloc(sizeof(double) * (size_t)(k * n > 0 ? k * n : 1));
    for (int64_t p2 = 0; p2 < k; ++p2)
        for (int64_t i = 0; i < m; ++i) Ao[i + p2 * m] = op_f64(A, lda, ta, i, p2);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t p2 = 0; p2 < k; ++p2) Bo[p2 + j * k] = op_f64(B, ldb, tb, p2, j);
    int32_t* ea = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t* eb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double* qa = (double*)malloc(sizeof(double) * (size_t)(s * m * k > 0 ? s * m * k : 1));
    double* qb = (double*)malloc(sizeof(double) * (size_t)(s * k * n > 0 ? s * k * n : 1));
    ora_ozaki_split(m, k, Ao, m, 1, beta_bits, s, ea, qa);
    ora_ozaki_split(k, n, Bo, k, 0, beta_bits, s, eb, qb);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < m; ++i) {
            double acc = 0.0;
            for (int d = s + 1; d >= 2; --d) {
                int64_t Sd = 0;
                for (int t = 1; t <= s; ++t) {
                    int u = d - t;
                    if (u < 1 || u > s) continue;
                    const double* xa = qa + (int64_t)(t - 1) * m * k;
                    const double* xb = qb + (int64_t)(u - 1) * k * n;
                    for (int64_t p2 = 0; p2 < k; ++p2)
                        Sd += (int64_t)xa[i + p2 * m] * (int64_t)xb[p2 + j * k];
                }
                acc += ldexp((double)Sd, -beta_bits * d);
            }
            double c = (alpha != 0.0) ? alpha * ldexp(acc, ea[i] + eb[j]) : 0.0;
            if (beta != 0.0) c += beta * CM(C, i, j, ldc);
            CM(C, i, j, ldc) = c;
        }
    }
    free(Ao); free(Bo); free(ea); free(eb); free(qa); free(qb);
}
