// host_gemm.cu -- the product with A, B and C in host memory, copies overlapped with the
// computation.
//
// hsmm_gemm_host computes C in blocks: row panels of op(A) times column panels of op(B).
// The host-to-device copies (the first row panel of op(A) and the first column panel of
// op(B) ahead of everything else) run on an internal copy stream, the blocks are computed on
// the caller's stream as soon as their panels are on the device, and every finished block of
// C returns to the host on a second internal stream while the next block is computed.  The
// host link moves ~210 GB/s one way (~170 GB/s each way when both directions run), one copy
// stream or several alike, so the exposed time is the first two panels' copy and the last
// block's return; the blocks keep both short.  For the FP64-accurate forms each row panel of
// op(A) and each column panel of op(B) is split once (the slices of a row of op(A) or a
// column of op(B) depend on that line alone, so the result is the same as one hsmm_gemm on
// the whole matrices).  Device copies of A, B, C and the compute workspace are carved from
// cfg->workspace (hsmm_gemm_host_workspace_size bytes); the call allocates nothing.  The
// copy streams and their events are created once per device, on the first call.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "hsmm.h"
#include "internal.h"

namespace hsmm {
namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxPanels = 8;      // column panels of op(B)
constexpr int kMaxRowPanels = 4;   // row panels of op(A)
constexpr int kEvents = 2 + kMaxRowPanels + kMaxPanels + kMaxRowPanels * kMaxPanels;

struct CopyEngine {
    std::mutex mu;
    cudaStream_t stream = nullptr;   // host to device
    cudaStream_t back = nullptr;     // device to host
    cudaEvent_t ev[kEvents] = {};
    bool ready = false;
};
CopyEngine g_engine[kMaxDevices];

// the engine of the current device, created on first use (its mutex must be held)
hsmm_status_t engine_ready(CopyEngine* E) {
    if (E->ready) return HSMM_STATUS_SUCCESS;
    cudaError_t e = cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&E->back, cudaStreamNonBlocking);
    for (int i = 0; i < kEvents && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&E->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return record_cuda(e);
    E->ready = true;
    return HSMM_STATUS_SUCCESS;
}

size_t elem_bytes(hsmm_dtype_t t) {
    switch (t) {
        case HSMM_R_64F: return 8;
        case HSMM_R_32F: return 4;
        case HSMM_R_16BF: return 2;
        case HSMM_R_8I: return 1;
        case HSMM_R_32I: return 4;
        case HSMM_C_64F: return 16;
    }
    return 0;
}

// device leading dimensions: 16 elements, so that every tensor-core operand row is 16-byte aligned
int64_t pad16(int64_t rows) { return ((rows > 1 ? rows : 1) + 15) / 16 * 16; }
size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct HostPlan {
    int64_t rowsA, colsA, rowsB, colsB, ldA, ldB, ldC;
    size_t ea, eb, ec;
    size_t offA, offB, offC, offW, total;
    int panels, rpanels;   // column panels of op(B) (nj columns), row panels of op(A) (mi rows)
    int64_t nj, mi;
    bool ozaki, cplx;
    int slices, bits;
    OzakiLayout L;
};

HostPlan host_plan(const hsmm_config_t& c, hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k) {
    HostPlan P{};
    P.rowsA = (ta == HSMM_OP_N) ? m : k;
    P.colsA = (ta == HSMM_OP_N) ? k : m;
    P.rowsB = (tb == HSMM_OP_N) ? k : n;
    P.colsB = (tb == HSMM_OP_N) ? n : k;
    P.ldA = pad16(P.rowsA);
    P.ldB = pad16(P.rowsB);
    P.ldC = pad16(m);
    P.ea = elem_bytes(c.a);
    P.eb = elem_bytes(c.b);
    P.ec = elem_bytes(c.c);
    P.cplx = (c.a == HSMM_C_64F);
    P.ozaki = (c.compute == HSMM_COMPUTE_64F_OZAKI);
    // two panels once each holds at least 2048 columns (whole 256-column tiles)
    P.panels = n >= 4096 ? 2 : 1;
    P.nj = P.panels == 1 ? n : ((n + P.panels - 1) / P.panels + 255) / 256 * 256;
    P.panels = int((n + P.nj - 1) / P.nj);
    // and two or four row panels once each holds at least 2048 rows (whole 256-row pair
    // tiles).  A block of 2048 x 4096 is 128 pair tiles, 96% of whole waves of the product
    // kernel (as for 4096 x 4096); four column panels as well would leave 64 tiles a block,
    // cut into 256 quarter-tile items for 76 pairs, 84% busy.
    P.rpanels = m >= 8192 ? 4 : (m >= 4096 ? 2 : 1);
    P.mi = P.rpanels == 1 ? m : ((m + P.rpanels - 1) / P.rpanels + 255) / 256 * 256;
    P.rpanels = int((m + P.mi - 1) / P.mi);
    size_t off = 0;
    P.offA = off; off += up256(size_t(P.ldA) * size_t(P.colsA) * P.ea);
    P.offB = off; off += up256(size_t(P.ldB) * size_t(P.colsB) * P.eb);
    P.offC = off; off += up256(size_t(P.ldC) * size_t(n) * P.ec);
    P.offW = off;
    P.slices = default_slices(&c);
    P.bits = default_bits(&c);
    if (P.ozaki) {
        P.L = P.cplx ? ozaki_layout(m, 2 * P.nj, 2 * k, P.slices) : ozaki_layout(m, P.nj, k, P.slices);
        off += P.L.total;
    }
    P.total = off;
    return P;
}

bool is_zero_scalar(hsmm_dtype_t c, const void* v) {
    switch (c) {
        case HSMM_R_64F: return *static_cast<const double*>(v) == 0.0;
        case HSMM_C_64F: return static_cast<const double*>(v)[0] == 0.0 && static_cast<const double*>(v)[1] == 0.0;
        case HSMM_R_32I: return *static_cast<const int32_t*>(v) == 0;
        default: return *static_cast<const float*>(v) == 0.0f;
    }
}

bool valid_op(hsmm_op_t t) { return t == HSMM_OP_N || t == HSMM_OP_T || t == HSMM_OP_C; }

}  // namespace
}  // namespace hsmm

using namespace hsmm;

extern "C" hsmm_status_t hsmm_gemm_host_workspace_size(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB,
                                                       int64_t m, int64_t n, int64_t k, size_t* bytes) {
    if (!cfg || !bytes || m < 0 || n < 0 || k < 0 || !valid_op(transA) || !valid_op(transB))
        return HSMM_STATUS_INVALID_VALUE;
    if (elem_bytes(cfg->a) == 0 || elem_bytes(cfg->b) == 0 || elem_bytes(cfg->c) == 0) return HSMM_STATUS_NOT_SUPPORTED;
    *bytes = host_plan(*cfg, transA, transB, m, n, k).total;
    return HSMM_STATUS_SUCCESS;
}

extern "C" hsmm_status_t hsmm_gemm_host(const hsmm_config_t* cfg, hsmm_op_t transA, hsmm_op_t transB, int64_t m,
                                        int64_t n, int64_t k, const void* alpha, const void* A, int64_t lda,
                                        const void* B, int64_t ldb, const void* beta, void* C, int64_t ldc,
                                        void* stream) {
    if (!cfg || !alpha || !beta || !valid_op(transA) || !valid_op(transB) || m < 0 || n < 0 || k < 0)
        return HSMM_STATUS_INVALID_VALUE;
    hsmm_config_t c = *cfg;
    if (elem_bytes(c.a) == 0 || elem_bytes(c.b) == 0 || elem_bytes(c.c) == 0) return HSMM_STATUS_NOT_SUPPORTED;
    const int64_t rowsA = (transA == HSMM_OP_N) ? m : k;
    const int64_t rowsB = (transB == HSMM_OP_N) ? k : n;
    if (lda < (rowsA > 1 ? rowsA : 1) || ldb < (rowsB > 1 ? rowsB : 1) || ldc < (m > 1 ? m : 1))
        return HSMM_STATUS_INVALID_VALUE;
    if (m == 0 || n == 0) return HSMM_STATUS_SUCCESS;
    if (!C || (k > 0 && (!A || !B))) return HSMM_STATUS_INVALID_VALUE;
    const HostPlan P = host_plan(c, transA, transB, m, n, k);
    if (P.panels > kMaxPanels || P.rpanels > kMaxRowPanels) return HSMM_STATUS_NOT_SUPPORTED;
    if (!c.workspace || c.workspace_bytes < P.total) return HSMM_STATUS_WORKSPACE_TOO_SMALL;
    if (reinterpret_cast<uintptr_t>(c.workspace) % 256 != 0)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "gemm_host: workspace must be 256-byte aligned");
    if (P.ozaki && (P.bits < 2 || P.bits > 7 || P.slices < 1 || P.slices > 16)) return HSMM_STATUS_INVALID_VALUE;
    if (P.ozaki && !(c.a == c.b && c.b == c.c && (c.a == HSMM_R_64F || c.a == HSMM_C_64F)))
        return HSMM_STATUS_NOT_SUPPORTED;

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return record_cuda(ce);
    if (dev < 0 || dev >= kMaxDevices) return HSMM_STATUS_NOT_SUPPORTED;
    CopyEngine* E = &g_engine[dev];
    std::lock_guard<std::mutex> lock(E->mu);
    hsmm_status_t r = engine_ready(E);
    if (r != HSMM_STATUS_SUCCESS) return r;

    cudaStream_t S = static_cast<cudaStream_t>(stream), X = E->stream, Y = E->back;
    uint8_t* ws = static_cast<uint8_t*>(c.workspace);
    uint8_t* dA = ws + P.offA;
    uint8_t* dB = ws + P.offB;
    uint8_t* dC = ws + P.offC;
    uint8_t* W = ws + P.offW;
    const bool read_c = !is_zero_scalar(c.c, beta);
    cudaEvent_t evStart = E->ev[0], evDone = E->ev[1];
    cudaEvent_t* evA = E->ev + 2;                                  // row panel I of op(A) on the device
    cudaEvent_t* evB = E->ev + 2 + kMaxRowPanels;                  // column panel J of op(B) (and of C)
    cudaEvent_t* evR = E->ev + 2 + kMaxRowPanels + kMaxPanels;     // block (I, J) of C computed
    auto panel_w = [&](int p) { const int64_t j0 = p * P.nj; return (n - j0) < P.nj ? (n - j0) : P.nj; };
    auto panel_h = [&](int p) { const int64_t i0 = p * P.mi; return (m - i0) < P.mi ? (m - i0) : P.mi; };
    // offset of row i0 of op(A) in A (host, ld lda) or its device copy (ld P.ldA)
    auto a_row = [&](int64_t i0, int64_t ld) { return transA == HSMM_OP_N ? i0 * int64_t(P.ea) : i0 * ld * int64_t(P.ea); };

    auto copy_a = [&](int I) {   // rows i0.. of op(A)
        const int64_t i0 = I * P.mi, h = panel_h(I);
        if (transA == HSMM_OP_N)   // rows i0.. of A (m x k): h elements of each of k columns
            return cudaMemcpy2DAsync(dA + a_row(i0, P.ldA), P.ldA * P.ea, static_cast<const uint8_t*>(A) + a_row(i0, lda),
                                     lda * P.ea, h * P.ea, k, cudaMemcpyHostToDevice, X);
        // columns i0.. of A (k x m)
        return cudaMemcpy2DAsync(dA + a_row(i0, P.ldA), P.ldA * P.ea, static_cast<const uint8_t*>(A) + a_row(i0, lda),
                                 lda * P.ea, k * P.ea, h, cudaMemcpyHostToDevice, X);
    };
    auto copy_b = [&](int J) {   // columns j0.. of op(B), and of C when it is read
        const int64_t j0 = J * P.nj, w = panel_w(J);
        cudaError_t e = cudaSuccess;
        if (k > 0 && transB == HSMM_OP_N)   // columns j0.. of B (k x n)
            e = cudaMemcpy2DAsync(dB + j0 * P.ldB * P.eb, P.ldB * P.eb, static_cast<const uint8_t*>(B) + j0 * ldb * P.eb,
                                  ldb * P.eb, k * P.eb, w, cudaMemcpyHostToDevice, X);
        else if (k > 0)                     // rows j0.. of B (n x k)
            e = cudaMemcpy2DAsync(dB + j0 * P.eb, P.ldB * P.eb, static_cast<const uint8_t*>(B) + j0 * P.eb, ldb * P.eb,
                                  w * P.eb, k, cudaMemcpyHostToDevice, X);
        if (e == cudaSuccess && read_c)
            e = cudaMemcpy2DAsync(dC + j0 * P.ldC * P.ec, P.ldC * P.ec, static_cast<const uint8_t*>(C) + j0 * ldc * P.ec,
                                  ldc * P.ec, m * P.ec, w, cudaMemcpyHostToDevice, X);
        return e;
    };

    // copies into the device buffers wait for the caller's earlier work on them; the first
    // row panel of op(A) and the first column panel of op(B) go first
    ce = cudaEventRecord(evStart, S);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(X, evStart, 0);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(Y, evStart, 0);
    for (int I = 0; I < P.rpanels && ce == cudaSuccess; ++I) {
        if (k > 0) ce = copy_a(I);
        if (ce == cudaSuccess) ce = cudaEventRecord(evA[I], X);
        if (ce == cudaSuccess && I == 0) {
            ce = copy_b(0);
            if (ce == cudaSuccess) ce = cudaEventRecord(evB[0], X);
        }
    }
    for (int J = 1; J < P.panels && ce == cudaSuccess; ++J) {
        ce = copy_b(J);
        if (ce == cudaSuccess) ce = cudaEventRecord(evB[J], X);
    }
    if (ce != cudaSuccess) {
        cudaStreamSynchronize(X);
        return record_cuda(ce);
    }

    // computation on the caller's stream, block by block; every finished block returns on Y
    hsmm_config_t cp = c;
    cp.workspace = nullptr;
    cp.workspace_bytes = 0;
    r = HSMM_STATUS_SUCCESS;
    int32_t* ea = reinterpret_cast<int32_t*>(W + P.L.ea);
    int32_t* eb = reinterpret_cast<int32_t*>(W + P.L.eb);
    int32_t* sd = reinterpret_cast<int32_t*>(W + P.L.sd);
    uint8_t* qa = W + P.L.qa;
    const bool ozaki_run = P.ozaki && k > 0 && !is_zero_scalar(c.c, alpha);
    // the first row panel of op(A) arrives first: its split runs while op(B)'s first panel is copied
    auto split_a = [&](int I) {
        const int64_t i0 = I * P.mi, h = panel_h(I);
        hsmm_status_t q = record_cuda(cudaStreamWaitEvent(S, evA[I], 0));
        if (q == HSMM_STATUS_SUCCESS && ozaki_run)
            q = ozaki_split_op_a(P.cplx, transA, h, k, dA + a_row(i0, P.ldA), P.ldA, P.bits, P.slices, ea + i0,
                                 qa + i0 * P.L.ldq * 2, P.L.ldq, P.L.qa_plane, S);
        return q;
    };
    r = split_a(0);
    for (int J = 0; J < P.panels && r == HSMM_STATUS_SUCCESS; ++J) {
        const int64_t j0 = J * P.nj, w = panel_w(J);
        r = record_cuda(cudaStreamWaitEvent(S, evB[J], 0));
        const uint8_t* dBp = (transB == HSMM_OP_N) ? dB + j0 * P.ldB * P.eb : dB + j0 * P.eb;
        if (r == HSMM_STATUS_SUCCESS && ozaki_run)
            r = ozaki_split_op_b(P.cplx, transB, k, w, dBp, P.ldB, P.bits, P.slices, eb, W + P.L.qb, P.L.ldq,
                                 P.L.qb_plane, S);
        for (int I = 0; I < P.rpanels && r == HSMM_STATUS_SUCCESS; ++I) {
            const int64_t i0 = I * P.mi, h = panel_h(I);
            const uint8_t* dAp = dA + a_row(i0, P.ldA);
            uint8_t* dCp = dC + (i0 + j0 * P.ldC) * P.ec;
            if (J == 0 && I > 0) r = split_a(I);
            if (r != HSMM_STATUS_SUCCESS) break;
            if (ozaki_run) {
                r = gemm_ozaki_slices(h, P.cplx ? 2 * w : w, P.cplx ? 2 * k : k, P.L.ldq, P.slices, P.bits,
                                      qa + i0 * P.L.ldq * 2, P.L.qa_plane, W + P.L.qb, P.L.qb_plane, sd, P.L.sd_plane, S);
                if (r == HSMM_STATUS_SUCCESS) {
                    if (P.cplx)
                        r = ozaki_zrecombine(h, w, P.slices, P.bits, sd, P.L.sd_plane, ea + i0, eb,
                                             static_cast<const double*>(alpha), static_cast<const double*>(beta), dCp,
                                             P.ldC, S);
                    else
                        r = ozaki_recombine(h, w, P.slices, P.bits, sd, P.L.sd_plane, ea + i0, eb,
                                            *static_cast<const double*>(alpha), *static_cast<const double*>(beta),
                                            reinterpret_cast<double*>(dCp), P.ldC, S);
                }
            } else {
                cp.compute = P.ozaki ? HSMM_COMPUTE_64F_NATIVE : c.compute;   // k == 0 or alpha == 0: only beta C
                r = hsmm_gemm(&cp, transA, transB, h, w, k, alpha, dAp, P.ldA, dBp, P.ldB, beta, dCp, P.ldC, S);
            }
            cudaEvent_t done = evR[I * kMaxPanels + J];
            if (r == HSMM_STATUS_SUCCESS) r = record_cuda(cudaEventRecord(done, S));
            if (r == HSMM_STATUS_SUCCESS) r = record_cuda(cudaStreamWaitEvent(Y, done, 0));
            if (r == HSMM_STATUS_SUCCESS)
                r = record_cuda(cudaMemcpy2DAsync(static_cast<uint8_t*>(C) + (i0 + j0 * ldc) * P.ec, ldc * P.ec, dCp,
                                                  P.ldC * P.ec, h * P.ec, w, cudaMemcpyDeviceToHost, Y));
        }
    }
    // the caller's stream ends after the last block is back (and the copy stream is idle)
    cudaError_t ce2 = cudaEventRecord(evDone, Y);
    if (ce2 == cudaSuccess) ce2 = cudaStreamWaitEvent(S, evDone, 0);
    if (ce2 == cudaSuccess) ce2 = cudaEventRecord(evDone, X);
    if (ce2 == cudaSuccess) ce2 = cudaStreamWaitEvent(S, evDone, 0);
    if (r != HSMM_STATUS_SUCCESS || ce2 != cudaSuccess) {
        cudaStreamSynchronize(X);   // host buffers must not be released while copies are in flight
        cudaStreamSynchronize(Y);
        return r != HSMM_STATUS_SUCCESS ? r : record_cuda(ce2);
    }
    return HSMM_STATUS_SUCCESS;
}
