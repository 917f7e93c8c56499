// internal.h -- host-side declarations shared by the translation units of libhsmm.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "hsmm.h"

namespace hsmm {

// ---- library state (api.cu) ----
uint64_t wait_timeout_ns();
void count_launches(int64_t n);
int num_sms();
hsmm_status_t record_cuda(cudaError_t e);           // SUCCESS or CUDA_ERROR (remembers the code)
// Remember a human-readable reason for a failing status (per host thread) and return the status.
hsmm_status_t fail(hsmm_status_t st, const char* fmt, ...);
const char* last_detail();
inline hsmm_status_t check_launch() { return record_cuda(cudaGetLastError()); }
inline bool aligned_to(const void* p, uintptr_t bytes) { return reinterpret_cast<uintptr_t>(p) % bytes == 0; }

// Kernel function attributes (dynamic shared memory, non-portable cluster sizes) apply per
// device: `set` runs once for each device the calling thread uses (one bit per device in
// `done`; two threads may both run it, which is harmless).
template <typename F>
inline hsmm_status_t attrs_once_per_device(std::atomic<uint64_t>& done, F&& set) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e);
    const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return HSMM_STATUS_SUCCESS;
    e = set();
    if (e != cudaSuccess) return record_cuda(e);
    if (bit) done.fetch_or(bit, std::memory_order_release);
    return HSMM_STATUS_SUCCESS;
}

// ---- per translation unit device status words (read and cleared) ----
uint32_t status_take_gemv();
uint32_t status_take_gemm_tc();
uint32_t status_take_grouped();
uint32_t status_take_ozaki_tc();
uint32_t status_take_gemm_f64();
uint32_t status_take_ozaki();
uint32_t status_take_ring();
uint32_t status_take_selftest();

// ---- gemv.cu ----
int gemv_splits(int64_t m, int64_t n);
int gemv_splits_rows(int64_t m, int64_t n, int rows_per_thread);
size_t gemv_workspace_bytes(hsmm_dtype_t a, hsmm_op_t trans, int64_t m, int64_t n);
hsmm_status_t gemv_f32(hsmm_op_t trans, int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
                       const float* x, int64_t incx, float beta, float* y, int64_t incy, void* ws, size_t ws_bytes,
                       cudaStream_t st);
hsmm_status_t gemv_i8(hsmm_op_t trans, int64_t m, int64_t n, int32_t alpha, const int8_t* A, int64_t lda,
                      const int8_t* x, int64_t incx, int32_t beta, int32_t* y, int64_t incy, void* ws,
                      size_t ws_bytes, cudaStream_t st);

// ---- gemm_f64.cu ----
hsmm_status_t gemm_f64_native(hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k, double alpha,
                              const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                              int64_t ldc, cudaStream_t st);
// complex FP64 product on the FP64 pipe; A, B, C interleaved (re, im), alpha and beta (re, im)
hsmm_status_t gemm_z64_native(hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k, const double* alpha,
                              const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                              int64_t ldc, cudaStream_t st);
// C = beta*C (beta == 0 writes zeros), for the BLAS early-outs; element type by size (4 or 8) or bf16 (2)
hsmm_status_t scale_matrix(hsmm_dtype_t c, int64_t m, int64_t n, const void* beta, void* C, int64_t ldc,
                           cudaStream_t st);

// ---- gemm_tc.cu ----
struct TcOperand {
    const void* ptr;
    int64_t ld;
    bool mn_major;   // true: the M (or N) index is contiguous in memory
};
hsmm_status_t gemm_tc(hsmm_dtype_t ab, hsmm_dtype_t c, hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k,
                      float alpha, const void* A, int64_t lda, const void* B, int64_t ldb, float beta, void* C,
                      int64_t ldc, int tile_n, cudaStream_t st);
bool tma_operand_ok(const void* p, int64_t ld, size_t esize);
// 2D (or 3D with a batch dimension) TMA map with 128-byte swizzle; false if encoding failed
// (last_encode_result() then holds the CUresult)
bool encode_map(CUtensorMap* map, CUtensorMapDataType dt, int esize, const void* base, uint64_t inner, uint64_t outer,
                uint64_t ld, uint32_t box_inner, uint32_t box_outer, uint64_t batch = 0,
                uint64_t batch_stride_elems = 0, CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B,
                uint32_t box_batch = 1);
int last_encode_result();

// ---- gemm_ozaki_tc.cu ----
// Slice products of the FP64-accurate form: S_d = sum_{t+u=d} Q^A_t (Q^B_u)^T, d = 2..s+1, exact INT32,
// stored as [d-2][n][m].
hsmm_status_t gemm_ozaki_slices(int64_t m, int64_t n, int64_t k, int64_t ldq, int slices, int bits, const void* qa,
                                int64_t qa_plane, const void* qb, int64_t qb_plane, int32_t* sd, int64_t sd_plane,
                                cudaStream_t st);

// ---- ozaki.cu ----
// slices written as [t][v][w]: row pitch ldq, slice (plane) pitch `plane` elements (>= lines * ldq)
hsmm_status_t ozaki_split(int64_t rows, int64_t cols, const double* M, int64_t ld, bool by_rows, int bits,
                          int slices, int32_t* expo, void* q, int64_t ldq, int64_t plane, cudaStream_t st);
// C = alpha 2^(ea_i + eb_j) sum_d 2^(-bits d) S_d + beta C
hsmm_status_t ozaki_recombine(int64_t m, int64_t n, int slices, int bits, const int32_t* sd, int64_t sd_plane,
                              const int32_t* ea, const int32_t* eb, double alpha, double beta, double* C, int64_t ldc,
                              cudaStream_t st);
// Complex operands into the real form of the complex product (A' = [Re, Im] rows of op(A) for
// role_b = false; B'' = [[Re, Im], [-Im, Re]] columns of op(B) for role_b = true, 2 nv lines)
hsmm_status_t ozaki_zsplit(int64_t nv, int64_t nw, const void* M, int64_t ld, bool v_contig, bool conj, bool role_b,
                           int bits, int slices, int32_t* expo, void* q, int64_t ldq, int64_t plane, cudaStream_t st);
// C = alpha (Re + i Im) + beta C from the real form's S_d (m x 2n), complex alpha, beta (re, im)
hsmm_status_t ozaki_zrecombine(int64_t m, int64_t n, int slices, int bits, const int32_t* sd, int64_t sd_plane,
                               const int32_t* ea, const int32_t* eb, const double* alpha, const double* beta, void* C,
                               int64_t ldc, cudaStream_t st);
// The workspace carve-up of the FP64-accurate form (documented in hsmm.h)
struct OzakiLayout {
    int64_t ldq, qa_plane, qb_plane, sd_plane;   // pitches in elements
    size_t qa, qb, ea, eb, sd, total;            // byte offsets
};
OzakiLayout ozaki_layout(int64_t m, int64_t n, int64_t k, int slices);
int default_slices(const hsmm_config_t* c);   // cfg->ozaki_slices, or 7
int default_bits(const hsmm_config_t* c);     // cfg->ozaki_bits, or 7
// Rows of op(A) (m x k) / columns of op(B) (k x n) into slices; cplx: complex operands into the
// real form (A' = [Re, Im]; B'' = [[Re, Im], [-Im, Re]], 2n lines)
hsmm_status_t ozaki_split_op_a(bool cplx, hsmm_op_t ta, int64_t m, int64_t k, const void* A, int64_t lda, int bits,
                               int s, int32_t* ea, void* qa, int64_t ldq, int64_t plane, cudaStream_t st);
hsmm_status_t ozaki_split_op_b(bool cplx, hsmm_op_t tb, int64_t k, int64_t n, const void* B, int64_t ldb, int bits,
                               int s, int32_t* eb, void* qb, int64_t ldq, int64_t plane, cudaStream_t st);
// Plane pitch (elements) of the workspace planes of hsmm_gemm's FP64-accurate form: the
// plane size rounded up to 256 bytes plus 1 KiB, so that the s planes one thread touches
// are not a power of two apart (such strides land on the same DRAM channels).
int64_t ozaki_plane_pitch(int64_t elems, int64_t elem_bytes);
int64_t ozaki_ldq(int64_t k);

// ---- gemm_ring_tc.cu ----
// C = alpha op(A) op(B) + beta C (BF16 in, FP32 out) in the ring order of Algorithm 2 on
// clusters of p CTAs with K auxiliary accumulators
hsmm_status_t gemm_tc_ring(hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k, float alpha, const void* A,
                           int64_t lda, const void* B, int64_t ldb, float beta, float* C, int64_t ldc, int p, int K,
                           cudaStream_t st);
uint32_t status_take_ring_tc();

// ---- nbody.cu ----
// F_i = sum_j f(x_i, z_j) (gravitational f), float4 bodies; ring_p = 0: tiled, else the
// hyper-systolic recipe on clusters of ring_p CTAs with ring_k replicas
hsmm_status_t nbody_forces(int64_t nx, int64_t nz, const float* x, const float* z, float eps2, float* out,
                           int ring_p, int ring_k, cudaStream_t st);

// ---- ring.cu ----
size_t ring_workspace_bytes(int p, int K, int64_t n);
hsmm_status_t ring_gemm_f64(int p, int K, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                            double* C, int64_t ldc, void* workspace, size_t workspace_bytes, cudaStream_t st);

// ---- grouped (gemm_tc.cu) ----
struct GroupedPlan;
hsmm_status_t grouped_plan_create(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                                  int tile_n, GroupedPlan** out);
// tile_n_per_problem: per problem 128/256 or 0 = automatic (NULL: all automatic);
// schedule 0: problems in the given order, 1: longest k first
hsmm_status_t grouped_plan_create_ex(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                                     int tile_n, const int* tile_n_per_problem, int schedule, GroupedPlan** out);
hsmm_status_t grouped_plan_launch(GroupedPlan* plan, float alpha, float beta, cudaStream_t st);
hsmm_status_t grouped_plan_info(GroupedPlan* plan, int64_t* tiles, int* tile_n);
void grouped_plan_destroy(GroupedPlan* plan);
// Without a plan: bytes of workspace the launch of these problems needs (0 and *st set on an
// error), and the launch itself with its descriptors and tile table written into the
// workspace by kernels on the stream (nothing allocated; capturable)
size_t grouped_workspace_bytes(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                               int tile_n, hsmm_status_t* st);
hsmm_status_t grouped_run_in_workspace(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                                       int tile_n, void* ws, size_t ws_bytes, float alpha, float beta,
                                       cudaStream_t st);

// ---- selftest (api.cu) ----
hsmm_status_t selftest_timeout_launch(uint64_t timeout_ns, cudaStream_t st);

}  // namespace hsmm
