// gemv_noalloc.cu -- y <- alpha*A*x + beta*y (op = N) without any caller workspace.
//
// hsmm_gemv splits the columns of A over many CTAs and needs a workspace for the
// partial sums of the splits.  Some callers cannot provide one: code that runs
// inside a host application which owns all device memory through its own arena
// and forbids outside allocations, latency-critical loops in which the device-wide
// synchronisation that cudaMalloc/cudaFree can cause is not acceptable, or
// plug-ins that have no place to keep a buffer between calls.  For them this file
// keeps the partial sums in a fixed array that lives in the library's own device
// memory (a file-scope __device__ array, present on every GPU that loads the
// library until the process exits), so a call allocates nothing.
//
// The call runs hsmm_gemv's own op = N kernels (column splits, then the fixed-order
// reduction) with this array as their workspace, so its results are bit-identical to
// hsmm_gemv's, and it takes hsmm_gemv's early-outs (alpha == 0 or n == 0: y = beta*y
// without reading A or x).
//
// Limits and rules:
//  * the array holds GEMV_STATIC_SCRATCH_BYTES = 16 MiB, i.e. 2^22 four-byte partial
//    sums.  Rows are limited to m <= 2^21: on a 152-SM GB300 hsmm_gemv's splits then
//    need at most 8 MiB (FP32) or 16 MiB (INT8, 16 rows per thread).  Larger m, or a
//    split count that would not fit (another GPU), is rejected with
//    HSMM_STATUS_WORKSPACE_TOO_SMALL before anything is launched;
//  * every call on a device shares the array: calls whose kernels overlap on the
//    GPU (different streams, different host threads) race on it and must be
//    serialised by the caller;
//  * every partial sum the reduction reads is written by the same call first, so
//    nothing in the array has to start at zero; the array simply keeps the last
//    call's partial sums;
//  * the first call on a device looks up the array's device address once
//    (cudaGetSymbolAddress, with that device current) and caches it per device;
//    make that first call before any stream capture.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "common.cuh"
#include "hsmm.h"
#include "internal.h"

namespace hsmm {
namespace {

constexpr size_t GEMV_STATIC_SCRATCH_BYTES = size_t(16) << 20;
constexpr int64_t kMaxRows = int64_t(1) << 21;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_gemv_scratch[GEMV_STATIC_SCRATCH_BYTES / 4];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_gemv_scratch on the current device (looked up once per device).
hsmm_status_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e);
    if (dev < 0 || dev >= kMaxDevices) return HSMM_STATUS_NOT_SUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gemv_scratch);
        if (e != cudaSuccess) return record_cuda(e);
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return HSMM_STATUS_SUCCESS;
}

}  // namespace
}  // namespace hsmm

using namespace hsmm;

extern "C" hsmm_status_t hsmm_gemv_n_noalloc(hsmm_dtype_t a, int64_t m, int64_t n, const void* alpha, const void* A,
                                             int64_t lda, const void* x, int64_t incx, const void* beta, void* y,
                                             int64_t incy, void* stream) {
    if (m < 0 || n < 0 || !alpha || !beta) return HSMM_STATUS_INVALID_VALUE;
    if (a != HSMM_R_32F && a != HSMM_R_8I) return HSMM_STATUS_NOT_SUPPORTED;
    if (lda < (m > 1 ? m : 1) || incx == 0 || incy == 0) return HSMM_STATUS_INVALID_VALUE;
    if (incx < 0 || incy < 0) return HSMM_STATUS_NOT_SUPPORTED;
    if (m > kMaxRows) return HSMM_STATUS_WORKSPACE_TOO_SMALL;
    if (m == 0) return HSMM_STATUS_SUCCESS;
    if (!y) return HSMM_STATUS_INVALID_VALUE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const hsmm_dtype_t c = (a == HSMM_R_32F) ? HSMM_R_32F : HSMM_R_32I;
    const bool azero = (a == HSMM_R_32F) ? (*static_cast<const float*>(alpha) == 0.f)
                                         : (*static_cast<const int32_t*>(alpha) == 0);
    if (n == 0 || azero) {
        // BLAS early-out, as hsmm_gemv: y = beta*y without reading A or x (beta == 0 writes zeros)
        if (incy != 1) return scale_matrix(c, 1, m, beta, y, incy, st);
        return scale_matrix(c, m, 1, beta, y, m, st);
    }
    if (!A || !x) return HSMM_STATUS_INVALID_VALUE;
    void* scratch = nullptr;
    hsmm_status_t s = scratch_address(&scratch);
    if (s != HSMM_STATUS_SUCCESS) return s;
    // the op = N kernels of hsmm_gemv, with the library's array as their workspace: the same
    // splits, kernels and summation order, hence the same bits as hsmm_gemv
    if (gemv_workspace_bytes(a, HSMM_OP_N, m, n) > GEMV_STATIC_SCRATCH_BYTES)
        return HSMM_STATUS_WORKSPACE_TOO_SMALL;
    if (a == HSMM_R_32F)
        return gemv_f32(HSMM_OP_N, m, n, *static_cast<const float*>(alpha), static_cast<const float*>(A), lda,
                        static_cast<const float*>(x), incx, *static_cast<const float*>(beta), static_cast<float*>(y),
                        incy, scratch, GEMV_STATIC_SCRATCH_BYTES, st);
    return gemv_i8(HSMM_OP_N, m, n, *static_cast<const int32_t*>(alpha), static_cast<const int8_t*>(A), lda,
                   static_cast<const int8_t*>(x), incx, *static_cast<const int32_t*>(beta), static_cast<int32_t*>(y),
                   incy, scratch, GEMV_STATIC_SCRATCH_BYTES, st);
}
