// gemm_f64.cu -- native FP64 product C <- alpha*op(A)*op(B) + beta*C on the FP64 pipe.
//
// Eq. PRODUCT (Section 3.1) computed with FP64 fused multiply-adds.  This is the
// baseline the FP64-accurate slice form is measured against.  The FP64 pipe of a
// GB300 is narrow, so the kernel only has to keep it busy: a 64 x 64 tile per
// CTA, k-slabs of 16 staged through shared memory (loads follow whichever index
// is contiguous for op = N / T), and a 4 x 4 register block per thread.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace hsmm {

static __device__ uint32_t g_status_gemm_f64;

uint32_t status_take_gemm_f64() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_gemm_f64, sizeof(v));
    cudaMemcpyToSymbol(g_status_gemm_f64, &z, sizeof(z));
    return v;
}

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// Load the BM x BK tile of op(M) at (r0, k0) into s[k][r] (zero outside).
template <int ROWS>
__device__ __forceinline__ void load_tile(double (*s)[ROWS + 1], const double* __restrict__ M, int64_t ld, bool trans,
                                          int64_t rows, int64_t kdim, int64_t r0, int64_t k0) {
    const int t = threadIdx.x;
    if (!trans) {
        // op(M)(r, kk) = M[r + kk*ld]: r contiguous
#pragma unroll
        for (int q = 0; q < (ROWS * BK) / NT; ++q) {
            const int idx = t + q * NT;
            const int r = idx % ROWS, kk = idx / ROWS;
            const int64_t gr = r0 + r, gk = k0 + kk;
            s[kk][r] = (gr < rows && gk < kdim) ? M[gr + gk * ld] : 0.0;
        }
    } else {
        // op(M)(r, kk) = M[kk + r*ld]: kk contiguous
#pragma unroll
        for (int q = 0; q < (ROWS * BK) / NT; ++q) {
            const int idx = t + q * NT;
            const int kk = idx % BK, r = idx / BK;
            const int64_t gr = r0 + r, gk = k0 + kk;
            s[kk][r] = (gr < rows && gk < kdim) ? M[gk + gr * ld] : 0.0;
        }
    }
}

__global__ void __launch_bounds__(NT) gemm_f64_kernel(int64_t m, int64_t n, int64_t k, double alpha,
                                                     const double* __restrict__ A, int64_t lda, bool ta,
                                                     const double* __restrict__ B, int64_t ldb, bool tb, double beta,
                                                     double* __restrict__ C, int64_t ldc) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int64_t m0 = int64_t(blockIdx.x) * BM, n0 = int64_t(blockIdx.y) * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int64_t k0 = 0; k0 < k; k0 += BK) {
        load_tile<BM>(As, A, lda, ta, m, k, m0, k0);
        // op(B) is k x n; tile (k0.., n0..): stored as Bs[kk][c]
        {
            const int t = threadIdx.x;
            if (!tb) {
                // op(B)(kk, c) = B[kk + c*ldb]: kk contiguous
#pragma unroll
                for (int q = 0; q < (BN * BK) / NT; ++q) {
                    const int idx = t + q * NT;
                    const int kk = idx % BK, c = idx / BK;
                    const int64_t gk = k0 + kk, gc = n0 + c;
                    Bs[kk][c] = (gk < k && gc < n) ? B[gk + gc * ldb] : 0.0;
                }
            } else {
                // op(B)(kk, c) = B[c + kk*ldb]: c contiguous
#pragma unroll
                for (int q = 0; q < (BN * BK) / NT; ++q) {
                    const int idx = t + q * NT;
                    const int c = idx % BN, kk = idx / BN;
                    const int64_t gk = k0 + kk, gc = n0 + c;
                    Bs[kk][c] = (gk < k && gc < n) ? B[gc + gk * ldb] : 0.0;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t c = n0 + tx + 16 * j;
        if (c >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t r = m0 + ty + 16 * i;
            if (r >= m) continue;
            double v = alpha * acc[i][j];
            if (beta != 0.0) v = fma(beta, C[r + c * ldc], v);
            C[r + c * ldc] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Complex product (Section 7: the method measured on complex data) on the FP64
// pipe: interleaved (re, im) doubles, op = N, T or C (conjugate transpose).  A
// 32 x 32 complex tile per CTA, k-slabs of 16, a 2 x 2 complex register block per
// thread; each complex multiply-add is four FP64 FMAs.
// ---------------------------------------------------------------------------
constexpr int ZB = 32, ZK = 16;

template <int ROWS>
__device__ __forceinline__ void load_ztile(double2 (*s)[ROWS + 1], const double2* __restrict__ M, int64_t ld, char t,
                                           int64_t rows, int64_t kdim, int64_t r0, int64_t k0) {
    const int tid = threadIdx.x;
    const bool conj = (t == 'C');
#pragma unroll
    for (int q = 0; q < (ROWS * ZK) / NT; ++q) {
        const int idx = tid + q * NT;
        int r, kk;
        if (t == 'N') { r = idx % ROWS; kk = idx / ROWS; }     // op(M)(r, kk) = M[r + kk*ld]
        else { kk = idx % ZK; r = idx / ZK; }                  // op(M)(r, kk) = M[kk + r*ld] (conjugated for C)
        const int64_t gr = r0 + r, gk = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (gr < rows && gk < kdim) {
            v = (t == 'N') ? M[gr + gk * ld] : M[gk + gr * ld];
            if (conj) v.y = -v.y;
        }
        s[kk][r] = v;
    }
}

__global__ void __launch_bounds__(NT) gemm_z64_kernel(int64_t m, int64_t n, int64_t k, double2 alpha,
                                                     const double2* __restrict__ A, int64_t lda, char ta,
                                                     const double2* __restrict__ B, int64_t ldb, char tb,
                                                     double2 beta, double2* __restrict__ C, int64_t ldc) {
    __shared__ double2 As[ZK][ZB + 1];
    __shared__ double2 Bs[ZK][ZB + 1];     // Bs[kk][c] = op(B)(k0 + kk, n0 + c)
    const int64_t m0 = int64_t(blockIdx.x) * ZB, n0 = int64_t(blockIdx.y) * ZB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double accr[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, acci[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int64_t k0 = 0; k0 < k; k0 += ZK) {
        load_ztile<ZB>(As, A, lda, ta, m, k, m0, k0);
        {
            // Bs[kk][c] = op(B)(k0+kk, n0+c): N -> B[kk + c*ldb]; T -> B[c + kk*ldb]; C -> conj(B[c + kk*ldb])
            const int tid = threadIdx.x;
#pragma unroll
            for (int q = 0; q < (ZB * ZK) / NT; ++q) {
                const int idx = tid + q * NT;
                int c, kk;
                if (tb == 'N') { kk = idx % ZK; c = idx / ZK; }      // kk contiguous
                else { c = idx % ZB; kk = idx / ZB; }               // c contiguous
                const int64_t gk = k0 + kk, gc = n0 + c;
                double2 v = make_double2(0.0, 0.0);
                if (gk < k && gc < n) {
                    v = (tb == 'N') ? B[gk + gc * ldb] : B[gc + gk * ldb];
                    if (tb == 'C') v.y = -v.y;
                }
                Bs[kk][c] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < ZK; ++kk) {
            double2 a[2], b[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 2; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    accr[i][j] = fma(a[i].x, b[j].x, accr[i][j]);
                    accr[i][j] = fma(-a[i].y, b[j].y, accr[i][j]);
                    acci[i][j] = fma(a[i].x, b[j].y, acci[i][j]);
                    acci[i][j] = fma(a[i].y, b[j].x, acci[i][j]);
                }
        }
        __syncthreads();
    }
    const bool read_c = beta.x != 0.0 || beta.y != 0.0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int64_t c = n0 + tx + 16 * j;
        if (c >= n) continue;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int64_t r = m0 + ty + 16 * i;
            if (r >= m) continue;
            double vr = alpha.x * accr[i][j] - alpha.y * acci[i][j];
            double vi = alpha.x * acci[i][j] + alpha.y * accr[i][j];
            if (read_c) {
                const double2 c0 = C[r + c * ldc];
                vr = fma(beta.x, c0.x, fma(-beta.y, c0.y, vr));
                vi = fma(beta.x, c0.y, fma(beta.y, c0.x, vi));
            }
            C[r + c * ldc] = make_double2(vr, vi);
        }
    }
}

__global__ void scale_z64_kernel(int64_t m, int64_t n, double2 beta, double2* __restrict__ C, int64_t ldc) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t jj = blockIdx.y; jj < n; jj += gridDim.y) {
        if (i >= m) continue;
        double2 v = make_double2(0.0, 0.0);
        if (beta.x != 0.0 || beta.y != 0.0) {
            const double2 c = C[i + jj * ldc];
            v = make_double2(beta.x * c.x - beta.y * c.y, beta.x * c.y + beta.y * c.x);
        }
        C[i + jj * ldc] = v;
    }
}

template <typename T>
__global__ void scale_kernel(int64_t m, int64_t n, T beta, T* __restrict__ C, int64_t ldc) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y;
    for (int64_t jj = j; jj < n; jj += gridDim.y) {
        if (i < m) C[i + jj * ldc] = (beta == T(0)) ? T(0) : T(beta * C[i + jj * ldc]);
    }
}

__global__ void scale_bf16_kernel(int64_t m, int64_t n, float beta, __nv_bfloat16* __restrict__ C, int64_t ldc) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t jj = blockIdx.y; jj < n; jj += gridDim.y) {
        if (i < m)
            C[i + jj * ldc] = (beta == 0.f) ? __float2bfloat16_rn(0.f)
                                            : __float2bfloat16_rn(beta * __bfloat162float(C[i + jj * ldc]));
    }
}

}  // namespace

hsmm_status_t gemm_f64_native(hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k, double alpha,
                              const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                              int64_t ldc, cudaStream_t st) {
    dim3 grid(unsigned((m + BM - 1) / BM), unsigned((n + BN - 1) / BN));
    if (grid.y > 65535u) return HSMM_STATUS_NOT_SUPPORTED;
    gemm_f64_kernel<<<grid, NT, 0, st>>>(m, n, k, alpha, A, lda, ta == HSMM_OP_T, B, ldb, tb == HSMM_OP_T, beta, C,
                                         ldc);
    count_launches(1);
    return check_launch();
}

hsmm_status_t gemm_z64_native(hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k, const double* alpha,
                              const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                              int64_t ldc, cudaStream_t st) {
    dim3 grid(unsigned((m + ZB - 1) / ZB), unsigned((n + ZB - 1) / ZB));
    if (grid.y > 65535u) return HSMM_STATUS_NOT_SUPPORTED;
    gemm_z64_kernel<<<grid, NT, 0, st>>>(m, n, k, make_double2(alpha[0], alpha[1]), static_cast<const double2*>(A),
                                         lda, char(ta), static_cast<const double2*>(B), ldb, char(tb),
                                         make_double2(beta[0], beta[1]), static_cast<double2*>(C), ldc);
    count_launches(1);
    return check_launch();
}

hsmm_status_t scale_matrix(hsmm_dtype_t c, int64_t m, int64_t n, const void* beta, void* C, int64_t ldc,
                           cudaStream_t st) {
    dim3 grid(unsigned((m + 255) / 256), unsigned(n < 65535 ? n : 65535));
    switch (c) {
        case HSMM_R_64F:
            scale_kernel<double><<<grid, 256, 0, st>>>(m, n, *static_cast<const double*>(beta),
                                                       static_cast<double*>(C), ldc);
            break;
        case HSMM_R_32F:
            scale_kernel<float><<<grid, 256, 0, st>>>(m, n, *static_cast<const float*>(beta), static_cast<float*>(C),
                                                      ldc);
            break;
        case HSMM_R_32I:
            scale_kernel<int32_t><<<grid, 256, 0, st>>>(m, n, *static_cast<const int32_t*>(beta),
                                                        static_cast<int32_t*>(C), ldc);
            break;
        case HSMM_C_64F: {
            const double* b = static_cast<const double*>(beta);
            scale_z64_kernel<<<grid, 256, 0, st>>>(m, n, make_double2(b[0], b[1]), static_cast<double2*>(C), ldc);
            break;
        }
        case HSMM_R_16BF:
            scale_bf16_kernel<<<grid, 256, 0, st>>>(m, n, *static_cast<const float*>(beta),
                                                    static_cast<__nv_bfloat16*>(C), ldc);
            break;
        default:
            return HSMM_STATUS_NOT_SUPPORTED;
    }
    count_launches(1);
    return check_launch();
}

}  // namespace hsmm
