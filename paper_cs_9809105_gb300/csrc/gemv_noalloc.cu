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
// Limits and rules:
//  * the array holds GEMV_STATIC_SCRATCH_BYTES = 8 MiB, i.e. 2^21 four-byte partial
//    sums; the column split is reduced until splits * m fits, and m > 2^21 rows is
//    rejected with HSMM_STATUS_WORKSPACE_TOO_SMALL before anything is launched;
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

constexpr size_t GEMV_STATIC_SCRATCH_BYTES = size_t(8) << 20;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

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

// Column-split partial sums, FP32: thread per row, sequential over its columns.
__global__ void __launch_bounds__(kThreads) nsplit_f32(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda,
                                                       const float* __restrict__ x, int64_t incx,
                                                       float* __restrict__ part, int64_t cols_per_split) {
    const int64_t r = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t j0 = int64_t(blockIdx.y) * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (r >= m) return;
    float acc = 0.f;
    int64_t j = j0;
    for (; j + 4 <= j1; j += 4) {
        const float a0 = __ldcs(A + r + (j + 0) * lda), a1 = __ldcs(A + r + (j + 1) * lda);
        const float a2 = __ldcs(A + r + (j + 2) * lda), a3 = __ldcs(A + r + (j + 3) * lda);
        acc = fmaf(a0, __ldg(x + (j + 0) * incx), acc);
        acc = fmaf(a1, __ldg(x + (j + 1) * incx), acc);
        acc = fmaf(a2, __ldg(x + (j + 2) * incx), acc);
        acc = fmaf(a3, __ldg(x + (j + 3) * incx), acc);
    }
    for (; j < j1; ++j) acc = fmaf(__ldcs(A + r + j * lda), __ldg(x + j * incx), acc);
    part[int64_t(blockIdx.y) * m + r] = acc;
}

__global__ void __launch_bounds__(kThreads) nsplit_i8(int64_t m, int64_t n, const int8_t* __restrict__ A, int64_t lda,
                                                      const int8_t* __restrict__ x, int64_t incx,
                                                      int32_t* __restrict__ part, int64_t cols_per_split) {
    const int64_t r = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t j0 = int64_t(blockIdx.y) * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (r >= m) return;
    int acc = 0;
    for (int64_t j = j0; j < j1; ++j) acc += int(__ldcs(A + r + j * lda)) * int(__ldg(x + j * incx));
    part[int64_t(blockIdx.y) * m + r] = acc;
}

// y_i = alpha * sum_s part[s][i] + beta*y_i, splits in the fixed order s = 0, 1, ...
__global__ void __launch_bounds__(kThreads) reduce_f32(int64_t m, int nsplit, const float* __restrict__ part,
                                                       float alpha, float beta, float* __restrict__ y, int64_t incy) {
    const int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (i >= m) return;
    float s = 0.f;
    for (int q = 0; q < nsplit; ++q) s += part[int64_t(q) * m + i];
    float v = alpha * s;
    if (beta != 0.f) v = fmaf(beta, y[i * incy], v);
    y[i * incy] = v;
}

__global__ void __launch_bounds__(kThreads) reduce_i32(int64_t m, int nsplit, const int32_t* __restrict__ part,
                                                       int32_t alpha, int32_t beta, int32_t* __restrict__ y,
                                                       int64_t incy) {
    const int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (i >= m) return;
    uint32_t s = 0;
    for (int q = 0; q < nsplit; ++q) s += uint32_t(part[int64_t(q) * m + i]);
    uint32_t v = uint32_t(alpha) * s;
    if (beta != 0) v += uint32_t(beta) * uint32_t(y[i * incy]);
    y[i * incy] = int32_t(v);
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
    const int64_t cap = int64_t(GEMV_STATIC_SCRATCH_BYTES / 4);   // partial sums that fit
    if (m > cap) return HSMM_STATUS_WORKSPACE_TOO_SMALL;
    if (m == 0) return HSMM_STATUS_SUCCESS;
    if (!A || !x || !y) return HSMM_STATUS_INVALID_VALUE;
    void* scratch = nullptr;
    hsmm_status_t s = scratch_address(&scratch);
    if (s != HSMM_STATUS_SUCCESS) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t ns = gemv_splits(m, n > 0 ? n : 1);
    if (ns * m > cap) ns = cap / m;
    if (ns < 1) ns = 1;
    const int64_t cps = n > 0 ? (n + ns - 1) / ns : 0;
    const dim3 grid(unsigned((m + kThreads - 1) / kThreads), unsigned(ns));
    const unsigned rgrid = unsigned((m + kThreads - 1) / kThreads);
    if (a == HSMM_R_32F) {
        float* part = static_cast<float*>(scratch);
        nsplit_f32<<<grid, kThreads, 0, st>>>(m, n, static_cast<const float*>(A), lda, static_cast<const float*>(x),
                                              incx, part, cps);
        reduce_f32<<<rgrid, kThreads, 0, st>>>(m, int(ns), part, *static_cast<const float*>(alpha),
                                               *static_cast<const float*>(beta), static_cast<float*>(y), incy);
    } else {
        int32_t* part = static_cast<int32_t*>(scratch);
        nsplit_i8<<<grid, kThreads, 0, st>>>(m, n, static_cast<const int8_t*>(A), lda, static_cast<const int8_t*>(x),
                                             incx, part, cps);
        reduce_i32<<<rgrid, kThreads, 0, st>>>(m, int(ns), part, *static_cast<const int32_t*>(alpha),
                                               *static_cast<const int32_t*>(beta), static_cast<int32_t*>(y), incy);
    }
    count_launches(2);
    return check_launch();
}
