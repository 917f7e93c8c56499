// host_gemm.cu -- the product with A, B and C in host memory, copies overlapped with the
// computation.
//
// hsmm_gemm_host copies op(A) to the device once, then walks the columns of C in panels:
// the copy of the next panel of B runs on an internal copy stream while the current panel
// is computed on the caller's stream, and every finished panel of C returns to the host
// while the next one is computed.  For the FP64-accurate forms op(A) is split once and
// only the panels of B are split per panel (the slices of a column of op(B) depend on
// that column alone, so the result is the same as one hsmm_gemm on the whole matrices).
// Device copies of A, B, C and the compute workspace are carved from cfg->workspace
// (hsmm_gemm_host_workspace_size bytes); the call allocates nothing.  The copy stream and
// its events are created once per device, on the first call.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "hsmm.h"
#include "internal.h"

namespace hsmm {
namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxPanels = 8;
constexpr int kEvents = 2 * kMaxPanels + 3;

struct CopyEngine {
    std::mutex mu;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev[kEvents] = {};
    bool ready = false;
};
CopyEngine g_engine[kMaxDevices];

// the engine of the current device, created on first use (its mutex must be held)
hsmm_status_t engine_ready(CopyEngine* E) {
    if (E->ready) return HSMM_STATUS_SUCCESS;
    cudaError_t e = cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking);
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
    int panels;
    int64_t nj;
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
    if (P.panels > kMaxPanels) return HSMM_STATUS_NOT_SUPPORTED;
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

    cudaStream_t S = static_cast<cudaStream_t>(stream), X = E->stream;
    uint8_t* ws = static_cast<uint8_t*>(c.workspace);
    uint8_t* dA = ws + P.offA;
    uint8_t* dB = ws + P.offB;
    uint8_t* dC = ws + P.offC;
    uint8_t* W = ws + P.offW;
    const bool read_c = !is_zero_scalar(c.c, beta);
    cudaEvent_t evStart = E->ev[0], evA = E->ev[1], evDone = E->ev[2];
    cudaEvent_t* evB = E->ev + 3;
    cudaEvent_t* evR = E->ev + 3 + kMaxPanels;
    auto panel_w = [&](int p) { const int64_t j0 = p * P.nj; return (n - j0) < P.nj ? (n - j0) : P.nj; };

    // copies into the device buffers wait for the caller's earlier work on them
    ce = cudaEventRecord(evStart, S);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(X, evStart, 0);
    if (ce == cudaSuccess && k > 0)
        ce = cudaMemcpy2DAsync(dA, P.ldA * P.ea, A, lda * P.ea, P.rowsA * P.ea, P.colsA, cudaMemcpyHostToDevice, X);
    if (ce == cudaSuccess) ce = cudaEventRecord(evA, X);
    for (int p = 0; p < P.panels && ce == cudaSuccess; ++p) {
        const int64_t j0 = p * P.nj, w = panel_w(p);
        if (k > 0) {
            if (transB == HSMM_OP_N)   // columns j0.. of B (k x n)
                ce = cudaMemcpy2DAsync(dB + j0 * P.ldB * P.eb, P.ldB * P.eb, static_cast<const uint8_t*>(B) + j0 * ldb * P.eb,
                                       ldb * P.eb, k * P.eb, w, cudaMemcpyHostToDevice, X);
            else                       // rows j0.. of B (n x k)
                ce = cudaMemcpy2DAsync(dB + j0 * P.eb, P.ldB * P.eb, static_cast<const uint8_t*>(B) + j0 * P.eb,
                                       ldb * P.eb, w * P.eb, k, cudaMemcpyHostToDevice, X);
        }
        if (ce == cudaSuccess && read_c)
            ce = cudaMemcpy2DAsync(dC + j0 * P.ldC * P.ec, P.ldC * P.ec, static_cast<const uint8_t*>(C) + j0 * ldc * P.ec,
                                   ldc * P.ec, m * P.ec, w, cudaMemcpyHostToDevice, X);
        if (ce == cudaSuccess) ce = cudaEventRecord(evB[p], X);
    }
    if (ce != cudaSuccess) {
        cudaStreamSynchronize(X);
        return record_cuda(ce);
    }

    // computation on the caller's stream, panel by panel
    hsmm_config_t cp = c;
    cp.workspace = nullptr;
    cp.workspace_bytes = 0;
    ce = cudaStreamWaitEvent(S, evA, 0);
    r = record_cuda(ce);
    int32_t* ea = reinterpret_cast<int32_t*>(W + P.L.ea);
    int32_t* eb = reinterpret_cast<int32_t*>(W + P.L.eb);
    int32_t* sd = reinterpret_cast<int32_t*>(W + P.L.sd);
    const bool ozaki_run = P.ozaki && k > 0 && !is_zero_scalar(c.c, alpha);
    if (r == HSMM_STATUS_SUCCESS && ozaki_run)
        r = ozaki_split_op_a(P.cplx, transA, m, k, dA, P.ldA, P.bits, P.slices, ea, W + P.L.qa, P.L.ldq, P.L.qa_plane,
                             S);
    int recorded = 0;
    for (int p = 0; p < P.panels && r == HSMM_STATUS_SUCCESS; ++p) {
        const int64_t j0 = p * P.nj, w = panel_w(p);
        r = record_cuda(cudaStreamWaitEvent(S, evB[p], 0));
        if (r != HSMM_STATUS_SUCCESS) break;
        const uint8_t* dBp = (transB == HSMM_OP_N) ? dB + j0 * P.ldB * P.eb : dB + j0 * P.eb;
        uint8_t* dCp = dC + j0 * P.ldC * P.ec;
        if (ozaki_run) {
            r = ozaki_split_op_b(P.cplx, transB, k, w, dBp, P.ldB, P.bits, P.slices, eb, W + P.L.qb, P.L.ldq,
                                 P.L.qb_plane, S);
            if (r == HSMM_STATUS_SUCCESS)
                r = gemm_ozaki_slices(m, P.cplx ? 2 * w : w, P.cplx ? 2 * k : k, P.L.ldq, P.slices, P.bits, W + P.L.qa,
                                      P.L.qa_plane, W + P.L.qb, P.L.qb_plane, sd, P.L.sd_plane, S);
            if (r == HSMM_STATUS_SUCCESS) {
                if (P.cplx)
                    r = ozaki_zrecombine(m, w, P.slices, P.bits, sd, P.L.sd_plane, ea, eb,
                                         static_cast<const double*>(alpha), static_cast<const double*>(beta), dCp,
                                         P.ldC, S);
                else
                    r = ozaki_recombine(m, w, P.slices, P.bits, sd, P.L.sd_plane, ea, eb,
                                        *static_cast<const double*>(alpha), *static_cast<const double*>(beta),
                                        reinterpret_cast<double*>(dCp), P.ldC, S);
            }
        } else {
            cp.compute = P.ozaki ? HSMM_COMPUTE_64F_NATIVE : c.compute;   // k == 0 or alpha == 0: only beta C
            r = hsmm_gemm(&cp, transA, transB, m, w, k, alpha, dA, P.ldA, dBp, P.ldB, beta, dCp, P.ldC, S);
        }
        if (r == HSMM_STATUS_SUCCESS) r = record_cuda(cudaEventRecord(evR[p], S));
        if (r == HSMM_STATUS_SUCCESS) ++recorded;
    }
    // finished panels of C go back on the copy stream; the caller's stream then waits for them
    for (int p = 0; p < recorded && r == HSMM_STATUS_SUCCESS; ++p) {
        const int64_t j0 = p * P.nj, w = panel_w(p);
        ce = cudaStreamWaitEvent(X, evR[p], 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpy2DAsync(static_cast<uint8_t*>(C) + j0 * ldc * P.ec, ldc * P.ec, dC + j0 * P.ldC * P.ec,
                                   P.ldC * P.ec, m * P.ec, w, cudaMemcpyDeviceToHost, X);
        r = record_cuda(ce);
    }
    cudaError_t ce2 = cudaEventRecord(evDone, X);
    if (ce2 == cudaSuccess) ce2 = cudaStreamWaitEvent(S, evDone, 0);
    if (r != HSMM_STATUS_SUCCESS || ce2 != cudaSuccess) {
        cudaStreamSynchronize(X);   // host buffers must not be released while copies are in flight
        return r != HSMM_STATUS_SUCCESS ? r : record_cuda(ce2);
    }
    return HSMM_STATUS_SUCCESS;
}
