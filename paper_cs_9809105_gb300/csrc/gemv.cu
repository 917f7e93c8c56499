// gemv.cu -- matrix-vector products y <- alpha*op(A)*x + beta*y (column-major A).
//
// The paper names the matrix-vector form as a capability of the same alignment
// (Sections 1 and 8) without printing an algorithm; these kernels compute the
// BLAS definition and are bound by HBM bandwidth (one pass over A).
//
//  op = N: y_i = sum_j A(i,j) x_j.  Rows are contiguous, so each thread owns a
//          few consecutive rows and streams down the columns with 128-bit loads.
//          The columns are split over CTAs to put enough bytes in flight; every
//          split writes its partial sums to the workspace and a second kernel,
//          launched as a programmatic dependent (it starts while the splits finish),
//          adds the splits in a fixed order (deterministic results).
//  op = T: y_j = sum_i A(i,j) x_i.  Column j is contiguous: one warp per column,
//          128-bit loads, a fixed shuffle tree for the reduction.
//  INT8:   exact INT32 accumulation with dp4a; for op = N the 16-row x 4-column
//          byte tiles are transposed in registers (byte permutes) so that dp4a
//          multiplies four columns of one row by four packed entries of x.
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace hsmm {

static __device__ uint32_t g_status_gemv;

uint32_t status_take_gemv() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_gemv, sizeof(v));
    cudaMemcpyToSymbol(g_status_gemv, &z, sizeof(z));
    return v;
}

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// FP32, op = N
// ---------------------------------------------------------------------------
// Vector path: 4 rows per thread (float4), grid (row blocks, column splits).
__global__ void __launch_bounds__(kThreads) gemv_f32_n_vec(int64_t m, int64_t n, const float* __restrict__ A,
                                                           int64_t lda, const float* __restrict__ x, int64_t incx,
                                                           float* __restrict__ part, int64_t cols_per_split) {
    pdl_trigger();   // the reduction may be scheduled; it waits for this grid to finish
    const int64_t r0 = (int64_t(blockIdx.x) * kThreads + threadIdx.x) * 4;
    const int64_t j0 = int64_t(blockIdx.y) * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (r0 >= m) return;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const float* a = A + r0;
    int64_t j = j0;
    // 8 columns in flight per thread
    for (; j + 8 <= j1; j += 8) {
        float4 v[8];
        float xs[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcs(reinterpret_cast<const float4*>(a + (j + u) * lda));
#pragma unroll
        for (int u = 0; u < 8; ++u) xs[u] = __ldg(x + (j + u) * incx);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            acc.x = fmaf(v[u].x, xs[u], acc.x);
            acc.y = fmaf(v[u].y, xs[u], acc.y);
            acc.z = fmaf(v[u].z, xs[u], acc.z);
            acc.w = fmaf(v[u].w, xs[u], acc.w);
        }
    }
    for (; j < j1; ++j) {
        float4 v = __ldcs(reinterpret_cast<const float4*>(a + j * lda));
        float xv = __ldg(x + j * incx);
        acc.x = fmaf(v.x, xv, acc.x);
        acc.y = fmaf(v.y, xv, acc.y);
        acc.z = fmaf(v.z, xv, acc.z);
        acc.w = fmaf(v.w, xv, acc.w);
    }
    float* p = part + int64_t(blockIdx.y) * m + r0;
    *reinterpret_cast<float4*>(p) = acc;
}

// Scalar path (unaligned A or odd sizes): 1 row per thread.
__global__ void __launch_bounds__(kThreads) gemv_f32_n_scalar(int64_t m, int64_t n, const float* __restrict__ A,
                                                              int64_t lda, const float* __restrict__ x,
                                                              int64_t incx, float* __restrict__ part,
                                                              int64_t cols_per_split) {
    pdl_trigger();   // the reduction may be scheduled; it waits for this grid to finish
    const int64_t r = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t j0 = int64_t(blockIdx.y) * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (r >= m) return;
    float acc = 0.f;
    for (int64_t j = j0; j < j1; ++j) acc = fmaf(A[r + j * lda], __ldg(x + j * incx), acc);
    part[int64_t(blockIdx.y) * m + r] = acc;
}

// y_i = alpha * sum_s part[s][i] + beta*y_i.  A CTA takes 32 rows; its 8 warps add the
// splits s = g, g + 8, ... (warp g) and the 8 sums are added in the order g = 0..7: a fixed
// order, so the result is deterministic.  Launched as a programmatic dependent of the split
// kernel: the CTAs start while the splits finish and wait for them on the device.
template <typename T, typename Acc>
__global__ void __launch_bounds__(kThreads) gemv_reduce(int64_t m, int nsplit, const T* __restrict__ part, T alpha,
                                                        T beta, T* __restrict__ y, int64_t incy) {
    pdl_wait();
    const int r = int(lane_id()), g = int(warp_id());
    const int64_t i = int64_t(blockIdx.x) * 32 + r;
    Acc sum = Acc(0);
    if (i < m)
        for (int q = g; q < nsplit; q += kThreads / 32) sum += Acc(part[int64_t(q) * m + i]);
    __shared__ Acc red[kThreads / 32][32];
    red[g][r] = sum;
    __syncthreads();
    if (g != 0 || i >= m) return;
    Acc t = red[0][r];
#pragma unroll
    for (int k = 1; k < kThreads / 32; ++k) t += red[k][r];
    if constexpr (sizeof(Acc) == 4 && Acc(-1) > Acc(0)) {
        // INT32 BLAS arithmetic: two's-complement wrap-around
        uint32_t v = uint32_t(alpha) * t;
        if (beta != 0) v += uint32_t(beta) * uint32_t(y[i * incy]);
        y[i * incy] = T(v);
    } else {
        T v = alpha * t;
        if (beta != T(0)) v = fmaf(beta, y[i * incy], v);
        y[i * incy] = v;
    }
}

// launch the reduction as a programmatic dependent of the kernel just launched on st
template <typename T, typename Acc>
cudaError_t launch_reduce(int64_t m, int nsplit, const T* part, T alpha, T beta, T* y, int64_t incy,
                          cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned((m + 31) / 32), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gemv_reduce<T, Acc>, m, nsplit, part, alpha, beta, y, incy);
}

// ---------------------------------------------------------------------------
// FP32, op = T: one warp per column
// ---------------------------------------------------------------------------
template <bool kVec>
__global__ void __launch_bounds__(kThreads) gemv_f32_t(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda,
                                                       const float* __restrict__ x, int64_t incx, float alpha,
                                                       float beta, float* __restrict__ y, int64_t incy) {
    const int64_t col = int64_t(blockIdx.x) * (kThreads / 32) + warp_id();
    if (col >= n) return;
    const float* a = A + col * lda;
    const int lane = lane_id();
    float acc = 0.f;
    if (kVec) {
        // m % 4 == 0, a and x 16-byte aligned, incx == 1
        const int64_t m4 = m / 4;
        const float4* a4 = reinterpret_cast<const float4*>(a);
        const float4* x4 = reinterpret_cast<const float4*>(x);
        int64_t i = lane;
        for (; i + 96 < m4; i += 128) {
            float4 v0 = __ldcs(a4 + i), v1 = __ldcs(a4 + i + 32), v2 = __ldcs(a4 + i + 64), v3 = __ldcs(a4 + i + 96);
            float4 w0 = __ldg(x4 + i), w1 = __ldg(x4 + i + 32), w2 = __ldg(x4 + i + 64), w3 = __ldg(x4 + i + 96);
            acc = fmaf(v0.x, w0.x, acc); acc = fmaf(v0.y, w0.y, acc); acc = fmaf(v0.z, w0.z, acc); acc = fmaf(v0.w, w0.w, acc);
            acc = fmaf(v1.x, w1.x, acc); acc = fmaf(v1.y, w1.y, acc); acc = fmaf(v1.z, w1.z, acc); acc = fmaf(v1.w, w1.w, acc);
            acc = fmaf(v2.x, w2.x, acc); acc = fmaf(v2.y, w2.y, acc); acc = fmaf(v2.z, w2.z, acc); acc = fmaf(v2.w, w2.w, acc);
            acc = fmaf(v3.x, w3.x, acc); acc = fmaf(v3.y, w3.y, acc); acc = fmaf(v3.z, w3.z, acc); acc = fmaf(v3.w, w3.w, acc);
        }
        for (; i < m4; i += 32) {
            float4 v = __ldcs(a4 + i);
            float4 w = __ldg(x4 + i);
            acc = fmaf(v.x, w.x, acc); acc = fmaf(v.y, w.y, acc); acc = fmaf(v.z, w.z, acc); acc = fmaf(v.w, w.w, acc);
        }
    } else {
        for (int64_t i = lane; i < m; i += 32) acc = fmaf(a[i], __ldg(x + i * incx), acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        float v = alpha * acc;
        if (beta != 0.f) v = fmaf(beta, y[col * incy], v);
        y[col * incy] = v;
    }
}

// ---------------------------------------------------------------------------
// INT8, op = N: 16 rows per thread, 4 columns per dp4a group
// ---------------------------------------------------------------------------
__device__ __forceinline__ void transpose4x4_bytes(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t& t0,
                                                   uint32_t& t1, uint32_t& t2, uint32_t& t3) {
    // w_c holds rows r..r+3 of column c; t_r holds columns c0..c3 of row r
    const uint32_t u0 = __byte_perm(w0, w1, 0x5140);
    const uint32_t u1 = __byte_perm(w0, w1, 0x7362);
    const uint32_t u2 = __byte_perm(w2, w3, 0x5140);
    const uint32_t u3 = __byte_perm(w2, w3, 0x7362);
    t0 = __byte_perm(u0, u2, 0x5410);
    t1 = __byte_perm(u0, u2, 0x7632);
    t2 = __byte_perm(u1, u3, 0x5410);
    t3 = __byte_perm(u1, u3, 0x7632);
}

__device__ __forceinline__ uint32_t pack_x4(const int8_t* x, int64_t j, int64_t incx) {
    const uint32_t b0 = uint8_t(__ldg(x + (j + 0) * incx));
    const uint32_t b1 = uint8_t(__ldg(x + (j + 1) * incx));
    const uint32_t b2 = uint8_t(__ldg(x + (j + 2) * incx));
    const uint32_t b3 = uint8_t(__ldg(x + (j + 3) * incx));
    return b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
}

__global__ void __launch_bounds__(kThreads) gemv_i8_n_vec(int64_t m, int64_t n, const int8_t* __restrict__ A,
                                                          int64_t lda, const int8_t* __restrict__ x, int64_t incx,
                                                          int32_t* __restrict__ part, int64_t cols_per_split) {
    pdl_trigger();   // the reduction may be scheduled; it waits for this grid to finish
    const int64_t r0 = (int64_t(blockIdx.x) * kThreads + threadIdx.x) * 16;
    const int64_t j0 = int64_t(blockIdx.y) * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (r0 >= m) return;
    int acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0;
    const int8_t* a = A + r0;
    int64_t j = j0;
    // two groups of four columns (eight 16-byte loads) in flight per thread
    for (; j + 8 <= j1; j += 8) {
        uint4 c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) c[u] = __ldcs(reinterpret_cast<const uint4*>(a + (j + u) * lda));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int xp = int(pack_x4(x, j + 4 * h, incx));
            const uint4* cc = c + 4 * h;
            uint32_t t[4];
            transpose4x4_bytes(cc[0].x, cc[1].x, cc[2].x, cc[3].x, t[0], t[1], t[2], t[3]);
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r] = __dp4a(int(t[r]), xp, acc[r]);
            transpose4x4_bytes(cc[0].y, cc[1].y, cc[2].y, cc[3].y, t[0], t[1], t[2], t[3]);
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[4 + r] = __dp4a(int(t[r]), xp, acc[4 + r]);
            transpose4x4_bytes(cc[0].z, cc[1].z, cc[2].z, cc[3].z, t[0], t[1], t[2], t[3]);
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[8 + r] = __dp4a(int(t[r]), xp, acc[8 + r]);
            transpose4x4_bytes(cc[0].w, cc[1].w, cc[2].w, cc[3].w, t[0], t[1], t[2], t[3]);
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[12 + r] = __dp4a(int(t[r]), xp, acc[12 + r]);
        }
    }
    for (; j + 4 <= j1; j += 4) {
        uint4 c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = __ldcs(reinterpret_cast<const uint4*>(a + (j + u) * lda));
        const int xp = int(pack_x4(x, j, incx));
        uint32_t t[4];
        transpose4x4_bytes(c[0].x, c[1].x, c[2].x, c[3].x, t[0], t[1], t[2], t[3]);
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = __dp4a(int(t[r]), xp, acc[r]);
        transpose4x4_bytes(c[0].y, c[1].y, c[2].y, c[3].y, t[0], t[1], t[2], t[3]);
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[4 + r] = __dp4a(int(t[r]), xp, acc[4 + r]);
        transpose4x4_bytes(c[0].z, c[1].z, c[2].z, c[3].z, t[0], t[1], t[2], t[3]);
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[8 + r] = __dp4a(int(t[r]), xp, acc[8 + r]);
        transpose4x4_bytes(c[0].w, c[1].w, c[2].w, c[3].w, t[0], t[1], t[2], t[3]);
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[12 + r] = __dp4a(int(t[r]), xp, acc[12 + r]);
    }
    for (; j < j1; ++j) {
        const uint4 c = __ldcs(reinterpret_cast<const uint4*>(a + j * lda));
        const int xv = int(__ldg(x + j * incx));
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[4 * q + b] += int(int8_t((w[q] >> (8 * b)) & 0xffu)) * xv;
    }
    int32_t* p = part + int64_t(blockIdx.y) * m + r0;
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<int4*>(p)[q] = make_int4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
}

__global__ void __launch_bounds__(kThreads) gemv_i8_n_scalar(int64_t m, int64_t n, const int8_t* __restrict__ A,
                                                             int64_t lda, const int8_t* __restrict__ x, int64_t incx,
                                                             int32_t* __restrict__ part, int64_t cols_per_split) {
    pdl_trigger();   // the reduction may be scheduled; it waits for this grid to finish
    const int64_t r = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const int64_t j0 = int64_t(blockIdx.y) * cols_per_split;
    const int64_t j1 = min(n, j0 + cols_per_split);
    if (r >= m) return;
    int acc = 0;
    for (int64_t j = j0; j < j1; ++j) acc += int(A[r + j * lda]) * int(__ldg(x + j * incx));
    part[int64_t(blockIdx.y) * m + r] = acc;
}

// INT8, op = T: one warp per column, 16 bytes per lane per step, dp4a against packed x.
template <bool kVec>
__global__ void __launch_bounds__(kThreads) gemv_i8_t(int64_t m, int64_t n, const int8_t* __restrict__ A, int64_t lda,
                                                      const int8_t* __restrict__ x, int64_t incx, int32_t alpha,
                                                      int32_t beta, int32_t* __restrict__ y, int64_t incy) {
    const int64_t col = int64_t(blockIdx.x) * (kThreads / 32) + warp_id();
    if (col >= n) return;
    const int8_t* a = A + col * lda;
    const int lane = lane_id();
    int acc = 0;
    if (kVec) {
        // m % 16 == 0, 16-byte aligned column and x, incx == 1
        const int64_t m16 = m / 16;
        const int4* a16 = reinterpret_cast<const int4*>(a);
        const int4* x16 = reinterpret_cast<const int4*>(x);
        int64_t i = lane;
        // four 16-byte loads of A in flight per lane
        for (; i + 96 < m16; i += 128) {
            int4 v[4], w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcs(a16 + i + 32 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = __ldg(x16 + i + 32 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc = __dp4a(v[u].x, w[u].x, acc); acc = __dp4a(v[u].y, w[u].y, acc);
                acc = __dp4a(v[u].z, w[u].z, acc); acc = __dp4a(v[u].w, w[u].w, acc);
            }
        }
        for (; i < m16; i += 32) {
            const int4 v = __ldcs(a16 + i);
            const int4 w = __ldg(x16 + i);
            acc = __dp4a(v.x, w.x, acc); acc = __dp4a(v.y, w.y, acc);
            acc = __dp4a(v.z, w.z, acc); acc = __dp4a(v.w, w.w, acc);
        }
    } else {
        for (int64_t i = lane; i < m; i += 32) acc += int(a[i]) * int(__ldg(x + i * incx));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        uint32_t v = uint32_t(alpha) * uint32_t(acc);
        if (beta != 0) v += uint32_t(beta) * uint32_t(y[col * incy]);
        y[col * incy] = int32_t(v);
    }
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// Column splits for op = N: enough CTAs for about 4 waves of 256-thread blocks on every SM
// (CTAs of 256 threads with rows_per_thread rows each).
int gemv_splits_rows(int64_t m, int64_t n, int rows_per_thread) {
    const int64_t rows_per_cta = int64_t(kThreads) * rows_per_thread;
    const int64_t rb = (m + rows_per_cta - 1) / rows_per_cta;
    int64_t target = int64_t(num_sms()) * 4;
    int64_t s = (target + rb - 1) / rb;
    if (s < 1) s = 1;
    if (s > 256) s = 256;
    const int64_t min_cols = 64;
    if (n / s < min_cols) s = (n + min_cols - 1) / min_cols;
    if (s < 1) s = 1;
    return int(s);
}

int gemv_splits(int64_t m, int64_t n) { return gemv_splits_rows(m, n, 4); }

// rows per thread of the op = N kernels: 4 (FP32, float4) or 16 (INT8, 16-byte loads)
static int rows_per_thread(hsmm_dtype_t a) { return a == HSMM_R_8I ? 16 : 4; }

size_t gemv_workspace_bytes(hsmm_dtype_t a, hsmm_op_t trans, int64_t m, int64_t n) {
    if (trans != HSMM_OP_N) return 0;
    return size_t(gemv_splits_rows(m, n, rows_per_thread(a))) * size_t(m) * 4u;
}

hsmm_status_t gemv_f32(hsmm_op_t trans, int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
                       const float* x, int64_t incx, float beta, float* y, int64_t incy, void* ws, size_t ws_bytes,
                       cudaStream_t st) {
    if (trans == HSMM_OP_N) {
        const int ns = gemv_splits(m, n);
        if (ws_bytes < size_t(ns) * size_t(m) * 4u || ws == nullptr) return HSMM_STATUS_WORKSPACE_TOO_SMALL;
        const int64_t cps = (n + ns - 1) / ns;
        float* part = static_cast<float*>(ws);
        const bool vec = (m % 4 == 0) && (lda % 4 == 0) && aligned16(A) && aligned16(ws);
        if (vec) {
            dim3 grid(unsigned((m / 4 + kThreads - 1) / kThreads), unsigned(ns));
            gemv_f32_n_vec<<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, part, cps);
        } else {
            dim3 grid(unsigned((m + kThreads - 1) / kThreads), unsigned(ns));
            gemv_f32_n_scalar<<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, part, cps);
        }
        const cudaError_t e = launch_reduce<float, float>(m, ns, part, alpha, beta, y, incy, st);
        count_launches(2);
        if (e != cudaSuccess) return record_cuda(e);
    } else {
        const bool vec = (m % 4 == 0) && (lda % 4 == 0) && aligned16(A) && aligned16(x) && incx == 1;
        const unsigned grid = unsigned((n + kThreads / 32 - 1) / (kThreads / 32));
        if (vec)
            gemv_f32_t<true><<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, alpha, beta, y, incy);
        else
            gemv_f32_t<false><<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, alpha, beta, y, incy);
        count_launches(1);
    }
    return check_launch();
}

hsmm_status_t gemv_i8(hsmm_op_t trans, int64_t m, int64_t n, int32_t alpha, const int8_t* A, int64_t lda,
                      const int8_t* x, int64_t incx, int32_t beta, int32_t* y, int64_t incy, void* ws,
                      size_t ws_bytes, cudaStream_t st) {
    if (trans == HSMM_OP_N) {
        const int ns = gemv_splits_rows(m, n, rows_per_thread(HSMM_R_8I));
        if (ws_bytes < size_t(ns) * size_t(m) * 4u || ws == nullptr) return HSMM_STATUS_WORKSPACE_TOO_SMALL;
        const int64_t cps = (n + ns - 1) / ns;
        int32_t* part = static_cast<int32_t*>(ws);
        const bool vec = (m % 16 == 0) && (lda % 16 == 0) && aligned16(A) && aligned16(ws);
        if (vec) {
            dim3 grid(unsigned((m / 16 + kThreads - 1) / kThreads), unsigned(ns));
            gemv_i8_n_vec<<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, part, cps);
        } else {
            dim3 grid(unsigned((m + kThreads - 1) / kThreads), unsigned(ns));
            gemv_i8_n_scalar<<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, part, cps);
        }
        const cudaError_t e = launch_reduce<int32_t, uint32_t>(m, ns, part, alpha, beta, y, incy, st);
        count_launches(2);
        if (e != cudaSuccess) return record_cuda(e);
    } else {
        const bool vec = (m % 16 == 0) && (lda % 16 == 0) && aligned16(A) && aligned16(x) && incx == 1;
        const unsigned grid = unsigned((n + kThreads / 32 - 1) / (kThreads / 32));
        if (vec)
            gemv_i8_t<true><<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, alpha, beta, y, incy);
        else
            gemv_i8_t<false><<<grid, kThreads, 0, st>>>(m, n, A, lda, x, incx, alpha, beta, y, incy);
        count_launches(1);
    }
    return check_launch();
}

}  // namespace hsmm
