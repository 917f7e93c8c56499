// api.cu -- the extern "C" boundary of libhsmm: argument checks, BLAS early-outs,
// dispatch to the kernels, status words and the failure-detection self-test.
#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#include <mutex>

#include <cuda_runtime.h>

#include "common.cuh"
#include "hsmm.h"
#include "internal.h"

namespace hsmm {

static std::atomic<uint64_t> g_timeout_ns{4000000000ull};
static std::atomic<int64_t> g_launches{0};
static thread_local int g_last_cuda = 0;

uint64_t wait_timeout_ns() { return g_timeout_ns.load(); }
void count_launches(int64_t n) { g_launches.fetch_add(n); }

// SM count of the current device (looked up once per device)
int num_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    if (dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

static thread_local char g_detail[256] = "";

hsmm_status_t record_cuda(cudaError_t e) {
    if (e == cudaSuccess) return HSMM_STATUS_SUCCESS;
    g_last_cuda = int(e);
    std::snprintf(g_detail, sizeof(g_detail), "CUDA error %d: %s", int(e), cudaGetErrorString(e));
    return HSMM_STATUS_CUDA_ERROR;
}

hsmm_status_t fail(hsmm_status_t st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
    return st;
}

const char* last_detail() { return g_detail; }

// ---------------------------------------------------------------------------
// failure-detection self-test: an mbarrier nothing arrives on
// ---------------------------------------------------------------------------
static __device__ uint32_t g_status_selftest;

uint32_t status_take_selftest() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_selftest, sizeof(v));
    cudaMemcpyToSymbol(g_status_selftest, &z, sizeof(z));
    return v;
}

__global__ void selftest_timeout_kernel(uint64_t timeout_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // phase 0 never completes: the wait must give up and record the timeout
        mbar_wait(&bar, 0, timeout_ns, &g_status_selftest, &abort);
    }
    __syncthreads();
}

hsmm_status_t selftest_timeout_launch(uint64_t timeout_ns, cudaStream_t st) {
    selftest_timeout_kernel<<<1, 32, 0, st>>>(timeout_ns);
    count_launches(1);
    return check_launch();
}


OzakiLayout ozaki_layout(int64_t m, int64_t n, int64_t k, int slices) {
    OzakiLayout L{};
    L.ldq = ozaki_ldq(k);
    L.qa_plane = ozaki_plane_pitch(m * L.ldq, 2);
    L.qb_plane = ozaki_plane_pitch(n * L.ldq, 2);
    L.sd_plane = ozaki_plane_pitch(m * n, 4);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t off = 0;
    L.qa = off; off = up(off + size_t(slices) * size_t(L.qa_plane) * 2);
    L.qb = off; off = up(off + size_t(slices) * size_t(L.qb_plane) * 2);
    L.ea = off; off = up(off + size_t(m) * 4);
    L.eb = off; off = up(off + size_t(n) * 4);
    L.sd = off; off = up(off + size_t(slices) * size_t(L.sd_plane) * 4);
    L.total = off;
    return L;
}

hsmm_status_t ozaki_split_op_a(bool cplx, hsmm_op_t ta, int64_t m, int64_t k, const void* A, int64_t lda, int bits,
                               int s, int32_t* ea, void* qa, int64_t ldq, int64_t plane, cudaStream_t st) {
    if (cplx) return ozaki_zsplit(m, k, A, lda, ta == HSMM_OP_N, ta == HSMM_OP_C, false, bits, s, ea, qa, ldq, plane, st);
    if (ta == HSMM_OP_N)
        return ozaki_split(m, k, static_cast<const double*>(A), lda, true, bits, s, ea, qa, ldq, plane, st);
    return ozaki_split(k, m, static_cast<const double*>(A), lda, false, bits, s, ea, qa, ldq, plane, st);
}

hsmm_status_t ozaki_split_op_b(bool cplx, hsmm_op_t tb, int64_t k, int64_t n, const void* B, int64_t ldb, int bits,
                               int s, int32_t* eb, void* qb, int64_t ldq, int64_t plane, cudaStream_t st) {
    if (cplx) return ozaki_zsplit(n, k, B, ldb, tb != HSMM_OP_N, tb == HSMM_OP_C, true, bits, s, eb, qb, ldq, plane, st);
    if (tb == HSMM_OP_N)
        return ozaki_split(k, n, static_cast<const double*>(B), ldb, false, bits, s, eb, qb, ldq, plane, st);
    return ozaki_split(n, k, static_cast<const double*>(B), ldb, true, bits, s, eb, qb, ldq, plane, st);
}

int default_slices(const hsmm_config_t* c) { return c->ozaki_slices > 0 ? c->ozaki_slices : 7; }
int default_bits(const hsmm_config_t* c) { return c->ozaki_bits > 0 ? c->ozaki_bits : 7; }

}  // namespace hsmm

using namespace hsmm;

namespace {

bool is_op(hsmm_op_t t) { return t == HSMM_OP_N || t == HSMM_OP_T || t == HSMM_OP_C; }

hsmm_config_t default_cfg_f64() {
    hsmm_config_t c;
    std::memset(&c, 0, sizeof(c));
    c.a = c.b = c.c = HSMM_R_64F;
    c.compute = HSMM_COMPUTE_DEFAULT;
    return c;
}

bool alpha_is_zero(hsmm_dtype_t ct, const void* alpha, bool f64) {
    if (f64) return *static_cast<const double*>(alpha) == 0.0;
    if (ct == HSMM_R_32I) return *static_cast<const int32_t*>(alpha) == 0;
    return *static_cast<const float*>(alpha) == 0.0f;
}


}  // namespace

extern "C" {

const char* hsmm_status_string(hsmm_status_t s) {
    switch (s) {
        case HSMM_STATUS_SUCCESS: return "HSMM_STATUS_SUCCESS";
        case HSMM_STATUS_INVALID_VALUE: return "HSMM_STATUS_INVALID_VALUE";
        case HSMM_STATUS_NOT_SUPPORTED: return "HSMM_STATUS_NOT_SUPPORTED";
        case HSMM_STATUS_WORKSPACE_TOO_SMALL: return "HSMM_STATUS_WORKSPACE_TOO_SMALL";
        case HSMM_STATUS_CUDA_ERROR: return "HSMM_STATUS_CUDA_ERROR";
        case HSMM_STATUS_TIMEOUT: return "HSMM_STATUS_TIMEOUT";
    }
    return "HSMM_STATUS_UNKNOWN";
}

int hsmm_last_cuda_error(void) { return g_last_cuda; }
const char* hsmm_last_error_detail(void) { return hsmm::last_detail(); }
int hsmm_version(void) { return 100; }

int64_t hsmm_launch_count(int reset) {
    return reset ? g_launches.exchange(0) : g_launches.load();
}

hsmm_status_t hsmm_set_wait_timeout_ns(uint64_t ns) {
    if (ns == 0) return HSMM_STATUS_INVALID_VALUE;
    g_timeout_ns.store(ns);
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_sync_status(void* stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return record_cuda(e);
    uint32_t s = status_take_gemv() | status_take_gemm_tc() | status_take_grouped() | status_take_ozaki_tc() |
                 status_take_gemm_f64() | status_take_ozaki() | status_take_ring() | status_take_ring_tc() |
                 status_take_selftest();
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda(e);
    if (s & DEV_TIMEOUT) return HSMM_STATUS_TIMEOUT;
    if (s & DEV_BADARG) return HSMM_STATUS_INVALID_VALUE;
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_selftest_timeout(uint64_t timeout_ns, void* stream) {
    if (timeout_ns == 0) return HSMM_STATUS_INVALID_VALUE;
    hsmm_status_t s = selftest_timeout_launch(timeout_ns, static_cast<cudaStream_t>(stream));
    if (s != HSMM_STATUS_SUCCESS) return s;
    return hsmm_sync_status(stream);
}

hsmm_status_t hsmm_workspace_size(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB, int64_t m,
                                  int64_t n, int64_t k, size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || k < 0 || !is_op(transA) || !is_op(transB)) return HSMM_STATUS_INVALID_VALUE;
    hsmm_config_t c = cfg ? *cfg : default_cfg_f64();
    *bytes = 0;
    if (c.a == HSMM_R_64F && c.compute == HSMM_COMPUTE_64F_OZAKI) {
        const int s = default_slices(&c);
        *bytes = ozaki_layout(m, n, k, s).total;
    }
    if (c.a == HSMM_C_64F && c.compute == HSMM_COMPUTE_64F_OZAKI) {
        const int s = default_slices(&c);
        *bytes = ozaki_layout(m, 2 * n, 2 * k, s).total;   // the real form: m x 2n x 2k
    }
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_gemv_workspace_size(const hsmm_config_t* cfg, hsmm_op_t trans, int64_t m, int64_t n,
                                       size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || !is_op(trans)) return HSMM_STATUS_INVALID_VALUE;
    const hsmm_dtype_t a = cfg ? cfg->a : HSMM_R_32F;
    *bytes = gemv_workspace_bytes(a, trans, m, n);
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_gemm(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB, int64_t m, int64_t n,
                        int64_t k, const void* alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                        const void* beta, void* C, int64_t ldc, void* stream) {
    hsmm_config_t c = cfg ? *cfg : default_cfg_f64();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!is_op(transA) || !is_op(transB)) return HSMM_STATUS_INVALID_VALUE;
    if (m < 0 || n < 0 || k < 0) return HSMM_STATUS_INVALID_VALUE;
    if (!alpha || !beta) return HSMM_STATUS_INVALID_VALUE;
    const int64_t rowsA = (transA == HSMM_OP_N) ? m : k;
    const int64_t rowsB = (transB == HSMM_OP_N) ? k : n;
    if (lda < (rowsA > 1 ? rowsA : 1) || ldb < (rowsB > 1 ? rowsB : 1) || ldc < (m > 1 ? m : 1))
        return HSMM_STATUS_INVALID_VALUE;
    for (int i = 0; i < 5; ++i)
        if (c.reserved[i] != 0) return HSMM_STATUS_INVALID_VALUE;
    if (c.ring_p < 0 || c.ring_k < 0) return HSMM_STATUS_INVALID_VALUE;

    // complex FP64 (interleaved re, im): native FP64 pipe or the FP64-accurate real form
    if (c.a == HSMM_C_64F || c.b == HSMM_C_64F || c.c == HSMM_C_64F) {
        if (!(c.a == HSMM_C_64F && c.b == HSMM_C_64F && c.c == HSMM_C_64F)) return HSMM_STATUS_NOT_SUPPORTED;
        if (c.ring_p != 0) return fail(HSMM_STATUS_NOT_SUPPORTED, "ring order: BF16 inputs and FP32 output only");
        const bool native = c.compute == HSMM_COMPUTE_DEFAULT || c.compute == HSMM_COMPUTE_64F_NATIVE;
        if (!native && c.compute != HSMM_COMPUTE_64F_OZAKI) return HSMM_STATUS_NOT_SUPPORTED;
        if (m == 0 || n == 0) return HSMM_STATUS_SUCCESS;
        if (!C) return HSMM_STATUS_INVALID_VALUE;
        const double* al = static_cast<const double*>(alpha);
        const double* be = static_cast<const double*>(beta);
        if (k == 0 || (al[0] == 0.0 && al[1] == 0.0)) return scale_matrix(HSMM_C_64F, m, n, beta, C, ldc, st);
        if (!A || !B) return HSMM_STATUS_INVALID_VALUE;
        if (native) return gemm_z64_native(transA, transB, m, n, k, al, A, lda, B, ldb, be, C, ldc, st);
        const int s = default_slices(&c), bits = default_bits(&c);
        if (bits < 2 || bits > 7 || s < 1 || s > 16) return HSMM_STATUS_INVALID_VALUE;
        if (2 * m > INT32_MAX || 2 * n > INT32_MAX || 2 * k > INT32_MAX) return HSMM_STATUS_NOT_SUPPORTED;
        const OzakiLayout L = ozaki_layout(m, 2 * n, 2 * k, s);
        if (!c.workspace || c.workspace_bytes < L.total) return HSMM_STATUS_WORKSPACE_TOO_SMALL;
        if (reinterpret_cast<uintptr_t>(c.workspace) % 256 != 0)
            return fail(HSMM_STATUS_NOT_SUPPORTED, "gemm: workspace must be 256-byte aligned");
        uint8_t* ws = static_cast<uint8_t*>(c.workspace);
        int32_t* ea = reinterpret_cast<int32_t*>(ws + L.ea);
        int32_t* eb = reinterpret_cast<int32_t*>(ws + L.eb);
        int32_t* sd = reinterpret_cast<int32_t*>(ws + L.sd);
        hsmm_status_t r = ozaki_split_op_a(true, transA, m, k, A, lda, bits, s, ea, ws + L.qa, L.ldq, L.qa_plane, st);
        if (r == HSMM_STATUS_SUCCESS)
            r = ozaki_split_op_b(true, transB, k, n, B, ldb, bits, s, eb, ws + L.qb, L.ldq, L.qb_plane, st);
        if (r == HSMM_STATUS_SUCCESS)
            r = gemm_ozaki_slices(m, 2 * n, 2 * k, L.ldq, s, bits, ws + L.qa, L.qa_plane, ws + L.qb, L.qb_plane, sd,
                                  L.sd_plane, st);
        if (r != HSMM_STATUS_SUCCESS) return r;
        return ozaki_zrecombine(m, n, s, bits, sd, L.sd_plane, ea, eb, al, be, C, ldc, st);
    }
    // real types: op = C is op = T
    if (transA == HSMM_OP_C) transA = HSMM_OP_T;
    if (transB == HSMM_OP_C) transB = HSMM_OP_T;

    // dtype / compute combinations
    const bool f64 = (c.a == HSMM_R_64F && c.b == HSMM_R_64F && c.c == HSMM_R_64F);
    const bool bf16 = (c.a == HSMM_R_16BF && c.b == HSMM_R_16BF && (c.c == HSMM_R_32F || c.c == HSMM_R_16BF) &&
                       c.compute == HSMM_COMPUTE_DEFAULT);
    const bool tf32 = (c.a == HSMM_R_32F && c.b == HSMM_R_32F && c.c == HSMM_R_32F &&
                       c.compute == HSMM_COMPUTE_32F_FAST_TF32);
    const bool f64_native = f64 && (c.compute == HSMM_COMPUTE_DEFAULT || c.compute == HSMM_COMPUTE_64F_NATIVE);
    const bool f64_ozaki = f64 && c.compute == HSMM_COMPUTE_64F_OZAKI;
    if (!(bf16 || tf32 || f64_native || f64_ozaki)) return HSMM_STATUS_NOT_SUPPORTED;
    if (c.tile_n != 0 && c.tile_n != 128 && c.tile_n != 256) return HSMM_STATUS_INVALID_VALUE;

    if (m == 0 || n == 0) return HSMM_STATUS_SUCCESS;
    if (!C) return HSMM_STATUS_INVALID_VALUE;
    if (k == 0 || alpha_is_zero(c.c, alpha, f64)) return scale_matrix(c.c, m, n, beta, C, ldc, st);
    if (!A || !B) return HSMM_STATUS_INVALID_VALUE;

    if (c.ring_p != 0) {
        if (!bf16 || c.c != HSMM_R_32F)
            return fail(HSMM_STATUS_NOT_SUPPORTED, "ring order: BF16 inputs and FP32 output only");
        int K = c.ring_k;
        if (K == 0)
            for (K = 1; 4 * K * K <= c.ring_p && 2 * K <= 4; K *= 2) {}
        return gemm_tc_ring(transA, transB, m, n, k, *static_cast<const float*>(alpha), A, lda, B, ldb,
                            *static_cast<const float*>(beta), static_cast<float*>(C), ldc, c.ring_p, K, st);
    }
    if (bf16 || tf32)
        return gemm_tc(c.a, c.c, transA, transB, m, n, k, *static_cast<const float*>(alpha), A, lda, B, ldb,
                       *static_cast<const float*>(beta), C, ldc, c.tile_n, st);
    const double al = *static_cast<const double*>(alpha), be = *static_cast<const double*>(beta);
    if (f64_native)
        return gemm_f64_native(transA, transB, m, n, k, al, static_cast<const double*>(A), lda,
                               static_cast<const double*>(B), ldb, be, static_cast<double*>(C), ldc, st);
    // FP64-accurate form: split op(A) by rows and op(B) by columns, then slice products.
    const int s = default_slices(&c), bits = default_bits(&c);
    if (bits < 2 || bits > 7 || s < 1 || s > 16) return HSMM_STATUS_INVALID_VALUE;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return HSMM_STATUS_NOT_SUPPORTED;
    const OzakiLayout L = ozaki_layout(m, n, k, s);
    if (!c.workspace || c.workspace_bytes < L.total) return HSMM_STATUS_WORKSPACE_TOO_SMALL;
    if (reinterpret_cast<uintptr_t>(c.workspace) % 256 != 0) return HSMM_STATUS_NOT_SUPPORTED;
    uint8_t* ws = static_cast<uint8_t*>(c.workspace);
    int32_t* ea = reinterpret_cast<int32_t*>(ws + L.ea);
    int32_t* eb = reinterpret_cast<int32_t*>(ws + L.eb);
    hsmm_status_t r = ozaki_split_op_a(false, transA, m, k, A, lda, bits, s, ea, ws + L.qa, L.ldq, L.qa_plane, st);
    if (r != HSMM_STATUS_SUCCESS) return r;
    r = ozaki_split_op_b(false, transB, k, n, B, ldb, bits, s, eb, ws + L.qb, L.ldq, L.qb_plane, st);
    if (r != HSMM_STATUS_SUCCESS) return r;
    int32_t* sd = reinterpret_cast<int32_t*>(ws + L.sd);
    r = gemm_ozaki_slices(m, n, k, L.ldq, s, bits, ws + L.qa, L.qa_plane, ws + L.qb, L.qb_plane, sd, L.sd_plane, st);
    if (r != HSMM_STATUS_SUCCESS) return r;
    return ozaki_recombine(m, n, s, bits, sd, L.sd_plane, ea, eb, al, be, static_cast<double*>(C), ldc, st);
}

hsmm_status_t hsmm_gemv(const hsmm_config_t* cfg, hsmm_op_t trans, int64_t m, int64_t n, const void* alpha,
                        const void* A, int64_t lda, const void* x, int64_t incx, const void* beta, void* y,
                        int64_t incy, void* stream) {
    hsmm_config_t c;
    if (cfg) c = *cfg;
    else { std::memset(&c, 0, sizeof(c)); c.a = c.b = c.c = HSMM_R_32F; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!is_op(trans) || m < 0 || n < 0 || !alpha || !beta) return HSMM_STATUS_INVALID_VALUE;
    if (lda < (m > 1 ? m : 1)) return HSMM_STATUS_INVALID_VALUE;
    if (incx == 0 || incy == 0) return HSMM_STATUS_INVALID_VALUE;
    if (incx < 0 || incy < 0) return HSMM_STATUS_NOT_SUPPORTED;
    const bool f32 = (c.a == HSMM_R_32F && c.c == HSMM_R_32F);
    const bool i8 = (c.a == HSMM_R_8I && c.c == HSMM_R_32I);
    if (!f32 && !i8) return HSMM_STATUS_NOT_SUPPORTED;
    const int64_t leny = (trans == HSMM_OP_N) ? m : n;
    const int64_t lenx = (trans == HSMM_OP_N) ? n : m;
    if (leny == 0) return HSMM_STATUS_SUCCESS;
    if (!y) return HSMM_STATUS_INVALID_VALUE;
    const bool azero = f32 ? (*static_cast<const float*>(alpha) == 0.f) : (*static_cast<const int32_t*>(alpha) == 0);
    if (lenx == 0 || azero) {
        // y = beta*y as a leny x 1 matrix with stride incy (ld irrelevant for one column)
        if (incy != 1) {
            // strided y: treat as a 1 x leny matrix with leading dimension incy
            return scale_matrix(c.c, 1, leny, beta, y, incy, st);
        }
        return scale_matrix(c.c, leny, 1, beta, y, leny, st);
    }
    if (!A || !x) return HSMM_STATUS_INVALID_VALUE;
    if (f32)
        return gemv_f32(trans, m, n, *static_cast<const float*>(alpha), static_cast<const float*>(A), lda,
                        static_cast<const float*>(x), incx, *static_cast<const float*>(beta), static_cast<float*>(y),
                        incy, c.workspace, c.workspace_bytes, st);
    return gemv_i8(trans, m, n, *static_cast<const int32_t*>(alpha), static_cast<const int8_t*>(A), lda,
                   static_cast<const int8_t*>(x), incx, *static_cast<const int32_t*>(beta), static_cast<int32_t*>(y),
                   incy, c.workspace, c.workspace_bytes, st);
}

hsmm_status_t hsmm_ozaki_split(int64_t rows, int64_t cols, const double* M, int64_t ld, int by_rows, int bits,
                               int slices, int32_t* expo, void* q, int64_t ldq, int64_t plane, void* stream) {
    if (rows < 0 || cols < 0 || ld < (rows > 1 ? rows : 1) || bits < 2 || bits > 7 || slices < 1 || slices > 16)
        return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_split: bad size, ld, bits or slices");
    const int64_t len = by_rows ? cols : rows;
    const int64_t nv = by_rows ? rows : cols;
    if (ldq < len || ldq % 8 != 0) return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_split: ldq < line length or not a multiple of 8");
    if (plane == 0) plane = nv * ldq;
    if (plane < nv * ldq || plane % 8 != 0) return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_split: bad slice pitch");
    if (rows == 0 || cols == 0) return HSMM_STATUS_SUCCESS;
    if (!M || !expo || !q) return HSMM_STATUS_INVALID_VALUE;
    return ozaki_split(rows, cols, M, ld, by_rows != 0, bits, slices, expo, q, ldq, plane,
                       static_cast<cudaStream_t>(stream));
}

hsmm_status_t hsmm_ozaki_slice_products(int64_t m, int64_t n, int64_t k, int slices, int bits, const void* qa,
                                        int64_t qa_plane, const void* qb, int64_t qb_plane, int64_t ldq,
                                        int32_t* sd, int64_t sd_plane, void* stream) {
    if (m < 0 || n < 0 || k < 0 || bits < 2 || bits > 7 || slices < 1 || slices > 16)
        return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_slice_products: bad size, bits or slices");
    if (ldq < k || ldq % 8 != 0) return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_slice_products: bad ldq");
    if (qa_plane == 0) qa_plane = m * ldq;
    if (qb_plane == 0) qb_plane = n * ldq;
    if (sd_plane == 0) sd_plane = m * n;
    if (qa_plane < m * ldq || qb_plane < n * ldq || qa_plane % 8 || qb_plane % 8 || sd_plane < m * n)
        return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_slice_products: bad plane pitch");
    if (m == 0 || n == 0) return HSMM_STATUS_SUCCESS;
    if (!qa || !qb || !sd) return HSMM_STATUS_INVALID_VALUE;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return HSMM_STATUS_NOT_SUPPORTED;
    if (reinterpret_cast<uintptr_t>(qa) % 16 || reinterpret_cast<uintptr_t>(qb) % 16)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "ozaki_slice_products: slices must be 16-byte aligned");
    if (k == 0) {
        for (int d = 0; d < slices; ++d) {
            cudaError_t e = cudaMemsetAsync(sd + int64_t(d) * sd_plane, 0, size_t(m) * size_t(n) * 4,
                                            static_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) return record_cuda(e);
        }
        return HSMM_STATUS_SUCCESS;
    }
    return gemm_ozaki_slices(m, n, k, ldq, slices, bits, qa, qa_plane, qb, qb_plane, sd, sd_plane,
                             static_cast<cudaStream_t>(stream));
}

hsmm_status_t hsmm_ozaki_recombine(int64_t m, int64_t n, int slices, int bits, const int32_t* sd, int64_t sd_plane,
                                   const int32_t* ea, const int32_t* eb, const double* alpha, const double* beta,
                                   double* C, int64_t ldc, void* stream) {
    if (m < 0 || n < 0 || bits < 2 || bits > 7 || slices < 1 || slices > 16 || !alpha || !beta)
        return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_recombine: bad size, bits, slices or scalars");
    if (ldc < (m > 1 ? m : 1)) return HSMM_STATUS_INVALID_VALUE;
    if (sd_plane == 0) sd_plane = m * n;
    if (sd_plane < m * n) return fail(HSMM_STATUS_INVALID_VALUE, "ozaki_recombine: bad plane pitch");
    if (m == 0 || n == 0) return HSMM_STATUS_SUCCESS;
    if (!sd || !ea || !eb || !C) return HSMM_STATUS_INVALID_VALUE;
    return ozaki_recombine(m, n, slices, bits, sd, sd_plane, ea, eb, *alpha, *beta, C, ldc,
                           static_cast<cudaStream_t>(stream));
}

hsmm_status_t hsmm_nbody(int64_t nx, int64_t nz, const float* x, const float* z, float eps2, float* out, int ring_p,
                         int ring_k, void* stream) {
    if (nx < 0 || nz < 0 || !(eps2 >= 0.f)) return HSMM_STATUS_INVALID_VALUE;
    if (ring_p != 0 && ring_p != 2 && ring_p != 4 && ring_p != 8 && ring_p != 16)
        return fail(HSMM_STATUS_INVALID_VALUE, "nbody: ring_p = %d (0, 2, 4, 8 or 16)", ring_p);
    int K = ring_k;
    if (ring_p != 0 && K == 0)
        for (K = 1; 4 * K * K <= ring_p && 2 * K <= 4; K *= 2) {}
    if (ring_p != 0 && ((K != 1 && K != 2 && K != 4) || ring_p % K != 0))
        return fail(HSMM_STATUS_INVALID_VALUE, "nbody: ring_k = %d (1, 2 or 4, dividing ring_p = %d)", ring_k, ring_p);
    if (nx == 0) return HSMM_STATUS_SUCCESS;
    if (!x || !out || (nz > 0 && !z)) return HSMM_STATUS_INVALID_VALUE;
    if (!aligned_to(x, 16) || !aligned_to(out, 16) || (nz > 0 && !aligned_to(z, 16)))
        return fail(HSMM_STATUS_NOT_SUPPORTED, "nbody: bodies must be 16-byte aligned float4");
    return nbody_forces(nx, nz, x, z, eps2, out, ring_p, K, static_cast<cudaStream_t>(stream));
}

hsmm_status_t hsmm_ring_workspace_size(int p, int K, int64_t n, size_t* bytes) {
    if (!bytes || p < 1 || K < 1 || p % K != 0 || n < 0) return HSMM_STATUS_INVALID_VALUE;
    *bytes = ring_workspace_bytes(p, K, n);
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_ring_gemm(int p, int K, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                             double* C, int64_t ldc, void* workspace, size_t workspace_bytes, void* stream) {
    if (p < 1 || p > 16 || K < 1 || p % K != 0 || n < 1 || n % p != 0) return HSMM_STATUS_INVALID_VALUE;
    const int64_t b = n / p;
    if (b % 8 != 0 || b > 32) return HSMM_STATUS_NOT_SUPPORTED;
    if (lda < n || ldb < n || ldc < n || !A || !B || !C) return HSMM_STATUS_INVALID_VALUE;
    return ring_gemm_f64(p, K, n, A, lda, B, ldb, C, ldc, workspace, workspace_bytes,
                         static_cast<cudaStream_t>(stream));
}

struct hsmm_grouped_plan_s {
    GroupedPlan* impl;
};

// Argument checks shared by the grouped entry points; on success `norm` holds the
// problems with op = C read as op = T (real operands).
static hsmm_status_t grouped_validate(const hsmm_config_t* cfg, int64_t count, const hsmm_gemm_desc_t* descs,
                                      const int* tile_n_per_problem, std::vector<hsmm_gemm_desc_t>* norm) {
    if (!cfg || count < 0 || (count > 0 && !descs)) return HSMM_STATUS_INVALID_VALUE;
    const bool bf16 = (cfg->a == HSMM_R_16BF && cfg->b == HSMM_R_16BF &&
                       (cfg->c == HSMM_R_32F || cfg->c == HSMM_R_16BF) && cfg->compute == HSMM_COMPUTE_DEFAULT);
    const bool tf32 = (cfg->a == HSMM_R_32F && cfg->b == HSMM_R_32F && cfg->c == HSMM_R_32F &&
                       cfg->compute == HSMM_COMPUTE_32F_FAST_TF32);
    if (!bf16 && !tf32) return HSMM_STATUS_NOT_SUPPORTED;
    if (cfg->tile_n != 0 && cfg->tile_n != 128 && cfg->tile_n != 256) return HSMM_STATUS_INVALID_VALUE;
    for (int64_t i = 0; i < count; ++i) {
        const hsmm_gemm_desc_t& d = descs[i];
        if (!is_op(d.transA) || !is_op(d.transB) || d.m < 0 || d.n < 0 || d.k < 0) return HSMM_STATUS_INVALID_VALUE;
        const int64_t rowsA = (d.transA == HSMM_OP_N) ? d.m : d.k;
        const int64_t rowsB = (d.transB == HSMM_OP_N) ? d.k : d.n;
        if (d.lda < (rowsA > 1 ? rowsA : 1) || d.ldb < (rowsB > 1 ? rowsB : 1) || d.ldc < (d.m > 1 ? d.m : 1))
            return HSMM_STATUS_INVALID_VALUE;
        if (d.m > 0 && d.n > 0 && !d.C) return HSMM_STATUS_INVALID_VALUE;
        if (d.m > 0 && d.n > 0 && d.k > 0 && (!d.A || !d.B)) return HSMM_STATUS_INVALID_VALUE;
        if (d.m > 0 && d.n > 0 && d.k == 0) return HSMM_STATUS_NOT_SUPPORTED;   // C = beta*C: use hsmm_gemm
        // widths: 0 (automatic) or a multiple of 32 up to 256; the image builder refuses widths
        // other than 128 and 256 where they need CTA pairs and a K-major B
        if (tile_n_per_problem && (tile_n_per_problem[i] < 0 || tile_n_per_problem[i] > 256 ||
                                   tile_n_per_problem[i] % 32 != 0))
            return HSMM_STATUS_INVALID_VALUE;
    }
    norm->assign(descs, descs + count);
    for (auto& d : *norm) {
        if (d.transA == HSMM_OP_C) d.transA = HSMM_OP_T;
        if (d.transB == HSMM_OP_C) d.transB = HSMM_OP_T;
    }
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_grouped_plan_create_ex(const hsmm_config_t* cfg, int64_t count, const hsmm_gemm_desc_t* descs,
                                          const int* tile_n_per_problem, int schedule, hsmm_grouped_plan_t* plan) {
    if (!plan) return HSMM_STATUS_INVALID_VALUE;
    if (schedule != 0 && schedule != 1) return HSMM_STATUS_INVALID_VALUE;
    std::vector<hsmm_gemm_desc_t> norm;
    hsmm_status_t s = grouped_validate(cfg, count, descs, tile_n_per_problem, &norm);
    if (s != HSMM_STATUS_SUCCESS) return s;
    GroupedPlan* impl = nullptr;
    s = grouped_plan_create_ex(cfg->a, cfg->c, count, norm.data(), cfg->tile_n, tile_n_per_problem, schedule, &impl);
    if (s != HSMM_STATUS_SUCCESS) return s;
    *plan = new hsmm_grouped_plan_s{impl};
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_grouped_plan_create(const hsmm_config_t* cfg, int64_t count, const hsmm_gemm_desc_t* descs,
                                       hsmm_grouped_plan_t* plan) {
    return hsmm_grouped_plan_create_ex(cfg, count, descs, nullptr, 1, plan);
}

hsmm_status_t hsmm_grouped_plan_launch(hsmm_grouped_plan_t plan, const void* alpha, const void* beta, void* stream) {
    if (!plan || !alpha || !beta) return HSMM_STATUS_INVALID_VALUE;
    return grouped_plan_launch(plan->impl, *static_cast<const float*>(alpha), *static_cast<const float*>(beta),
                               static_cast<cudaStream_t>(stream));
}

hsmm_status_t hsmm_grouped_plan_info(hsmm_grouped_plan_t plan, int64_t* tiles, int* tile_n_per_problem) {
    if (!plan) return HSMM_STATUS_INVALID_VALUE;
    return grouped_plan_info(plan->impl, tiles, tile_n_per_problem);
}

hsmm_status_t hsmm_grouped_plan_destroy(hsmm_grouped_plan_t plan) {
    if (!plan) return HSMM_STATUS_INVALID_VALUE;
    grouped_plan_destroy(plan->impl);
    delete plan;
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t hsmm_gemm_grouped_workspace_size(const hsmm_config_t* cfg, int64_t count, const hsmm_gemm_desc_t* descs,
                                               size_t* bytes) {
    if (!bytes) return HSMM_STATUS_INVALID_VALUE;
    std::vector<hsmm_gemm_desc_t> norm;
    hsmm_status_t s = grouped_validate(cfg, count, descs, nullptr, &norm);
    if (s != HSMM_STATUS_SUCCESS) return s;
    *bytes = grouped_workspace_bytes(cfg->a, cfg->c, count, norm.data(), cfg->tile_n, &s);
    return s;
}

hsmm_status_t hsmm_gemm_grouped(const hsmm_config_t* cfg, int64_t count, const hsmm_gemm_desc_t* descs,
                                const void* alpha, const void* beta, void* stream) {
    if (!alpha || !beta) return HSMM_STATUS_INVALID_VALUE;
    std::vector<hsmm_gemm_desc_t> norm;
    hsmm_status_t s = grouped_validate(cfg, count, descs, nullptr, &norm);
    if (s != HSMM_STATUS_SUCCESS) return s;
    return grouped_run_in_workspace(cfg->a, cfg->c, count, norm.data(), cfg->tile_n, cfg->workspace,
                                    cfg->workspace_bytes, *static_cast<const float*>(alpha),
                                    *static_cast<const float*>(beta), static_cast<cudaStream_t>(stream));
}

}  // extern "C"
