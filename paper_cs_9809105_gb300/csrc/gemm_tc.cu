// gemm_tc.cu -- tensor-core products on sm_103a: TMA -> shared memory -> tcgen05.mma -> TMEM.
//
// The local block product (x) of the block mapping (Section 6.1), which holds all
// the flops of the paper's method, is here a 128 x BN output tile of one CTA:
//
//   warp 0 (one lane)   TMA producer: k-slabs of op(A) and op(B) into a ring of
//                       STAGES shared-memory stages (128-byte swizzle), mbarrier
//                       full/empty handshake;
//   warp 1 (one lane)   MMA issuer: tcgen05.mma (M = 128, N = BN, K = 32 bytes per
//                       instruction) into one of two TMEM accumulators, commits
//                       free the stages and hand finished accumulators over;
//   warps 2..5          epilogue: tcgen05.ld of their 32 TMEM lanes, alpha/beta,
//                       coalesced stores of column-major C.
//
// The kernel is persistent (one CTA per SM, tiles strided by the grid) and the
// two TMEM accumulators let the epilogue of tile t overlap the main loop of
// tile t+1.  The transposed forms A^T B, A B^T (Section 8: "on the same footing")
// cost nothing extra: an operand whose M/N index is contiguous is loaded as
// 64-element MN chunks and described to the MMA as MN-major, one whose K index is
// contiguous as K-major rows.  Ragged edges come from TMA out-of-bounds zero fill.
//
// The same main loop, fed with a different k-schedule and epilogue, computes the
// slice products of the FP64-accurate form (gemm_ozaki_slices below) and the
// grouped launch (many problems, one persistent grid).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace hsmm {

static __device__ uint32_t g_status_gemm_tc;

uint32_t status_take_gemm_tc() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_gemm_tc, sizeof(v));
    cudaMemcpyToSymbol(g_status_gemm_tc, &z, sizeof(z));
    return v;
}

// ---------------------------------------------------------------------------
// TMA descriptor encoding (driver entry point fetched through the runtime)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool tma_operand_ok(const void* p, int64_t ld, size_t esize) {
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((uint64_t(ld) * esize) % 16 == 0);
}

// 2D (or 3D with a batch dimension) tiled map with 128-byte swizzle.
static bool encode_map(CUtensorMap* map, CUtensorMapDataType dt, int esize, const void* base, uint64_t inner,
                       uint64_t outer, uint64_t ld, uint32_t box_inner, uint32_t box_outer, uint64_t batch = 0,
                       uint64_t batch_stride_elems = 0) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {inner, outer, batch};
    cuuint64_t strides[2] = {ld * uint64_t(esize), batch_stride_elems * uint64_t(esize)};
    cuuint32_t box[3] = {box_inner, box_outer, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t rank = batch ? 3 : 2;
    CUresult r = fn(map, dt, rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

constexpr int BM = 128;
constexpr int kNumThreads = 192;   // 6 warps: producer, MMA, 4 x epilogue

template <int BN_, bool TF32_>
struct Cfg {
    static constexpr int BN = BN_;
    static constexpr bool TF32 = TF32_;
    static constexpr int ESIZE = TF32 ? 4 : 2;
    static constexpr int BK = 128 / ESIZE;            // one 128-byte swizzle row of K
    static constexpr int UMMA_K = 32 / ESIZE;         // K per tcgen05.mma (32 bytes)
    static constexpr int KSTEPS = BK / UMMA_K;        // 4
    static constexpr int MN_CHUNK = 128 / ESIZE;      // MN elements per 128-byte row (MN-major operands)
    static constexpr int A_BYTES = BM * 128;
    static constexpr int B_BYTES = BN * 128;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = (BN >= 256) ? 4 : 6;
    static constexpr int TMEM_COLS = 2 * BN;          // two accumulators
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};

struct Bars {
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t mma_done;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Tile index -> (tile row, tile column): groups of 16 tile rows sweep the columns,
// so that the A panels of a group and the B panels they meet stay in L2.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
    constexpr int G = 16;
    const int group_size = G * tiles_n;
    const int g = t / group_size;
    const int first = g * G;
    const int rows_in_group = min(G, tiles_m - first);
    const int r = t - g * group_size;
    tm = first + r % rows_in_group;
    tn = r / rows_in_group;
}

template <typename C_>
__device__ __forceinline__ uint64_t operand_desc(uint32_t base, int ks, bool mn_major) {
    if (mn_major) {
        // MN-major: 64-element MN chunks of BK rows each; LBO = chunk bytes, SBO = 8 rows.
        return smem_desc_sw128(base + uint32_t(ks) * uint32_t(C_::UMMA_K) * 128u, uint32_t(C_::BK) * 128u, 1024u);
    }
    // K-major: rows of 128 bytes; the K step moves 32 bytes inside the swizzled row.
    return smem_desc_sw128(base + uint32_t(ks) * 32u, 16u, 1024u);
}

// Issue the TMA loads of one operand k-slab (rows r0.. of the MN dimension, k-block kb).
template <typename C_, int ROWS>
__device__ __forceinline__ void load_operand(uint8_t* dst, const void* map, uint64_t* bar, bool mn_major, int r0,
                                             int kb, int batch, bool batched) {
    if (!mn_major) {
        if (batched)
            tma_load_3d(dst, map, bar, kb * C_::BK, r0, batch);
        else
            tma_load_2d(dst, map, bar, kb * C_::BK, r0);
    } else {
#pragma unroll
        for (int c = 0; c < ROWS / C_::MN_CHUNK; ++c)
            tma_load_2d(dst + c * C_::BK * 128, map, bar, r0 + c * C_::MN_CHUNK, kb * C_::BK);
    }
}

struct GemmArgs {
    int M, N, K;
    int a_mn, b_mn;
    float alpha, beta;
    void* C;
    int64_t ldc;
    uint64_t timeout_ns;
};

// ---------------------------------------------------------------------------
// Plain product kernel
// ---------------------------------------------------------------------------
template <int BN, bool TF32, bool OUT_BF16>
__global__ void __launch_bounds__(kNumThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
    using C_ = Cfg<BN, TF32>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    Bars* bars = reinterpret_cast<Bars*>(smem + C_::STAGES * C_::STAGE_BYTES);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_gemm_tc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C_::STAGES; ++s) {
            mbar_init(&bars->full[s], 1);
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], 4);
        }
        mbar_init(&bars->mma_done, 1);
        bars->abort = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 1) {
        tmem_alloc(&bars->tmem_base, C_::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;

    const int tiles_m = (g.M + BM - 1) / BM;
    const int tiles_n = (g.N + BN - 1) / BN;
    const int ntiles = tiles_m * tiles_n;
    const int nkb = (g.K + C_::BK - 1) / C_::BK;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[8];
            for (int s = 0; s < 8; ++s) last_parity[s] = -1;
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                int tm, tn;
                tile_coords(t, tiles_m, tiles_n, tm, tn);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&bars->empty[stage], phase ^ 1u, g.timeout_ns, status, abort)) break;
                    uint8_t* a_dst = smem + stage * C_::STAGE_BYTES;
                    uint8_t* b_dst = a_dst + C_::A_BYTES;
                    mbar_arrive_expect_tx(&bars->full[stage], C_::STAGE_BYTES);
                    load_operand<C_, BM>(a_dst, &tmA, &bars->full[stage], g.a_mn, tm * BM, kb, 0, false);
                    load_operand<C_, BN>(b_dst, &tmB, &bars->full[stage], g.b_mn, tn * BN, kb, 0, false);
                    last_parity[stage] = int(phase);
                    if (++stage == C_::STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            // make sure no bulk copy is still landing in shared memory
            for (int s = 0; s < C_::STAGES; ++s)
                if (last_parity[s] >= 0) mbar_wait(&bars->full[s], uint32_t(last_parity[s]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int abuf = 0;
            uint32_t aphase = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                if (!mbar_wait(&bars->acc_empty[abuf], aphase ^ 1u, g.timeout_ns, status, abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + uint32_t(abuf * BN);
                uint32_t idesc = make_idesc(TF32 ? 2u : 1u, g.a_mn != 0, g.b_mn != 0, BM, BN);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&bars->full[stage], phase, g.timeout_ns, status, abort)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(smem + stage * C_::STAGE_BYTES);
                    const uint32_t b_base = a_base + C_::A_BYTES;
#pragma unroll
                    for (int ks = 0; ks < C_::KSTEPS; ++ks) {
                        const uint64_t ad = operand_desc<C_>(a_base, ks, g.a_mn != 0);
                        const uint64_t bd = operand_desc<C_>(b_base, ks, g.b_mn != 0);
                        if (TF32)
                            umma_tf32(d_tmem, ad, bd, idesc, (kb | ks) != 0);
                        else
                            umma_f16(d_tmem, ad, bd, idesc, (kb | ks) != 0);
                    }
                    umma_commit(&bars->empty[stage]);
                    if (++stage == C_::STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit(&bars->acc_full[abuf]);
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1u;
            }
            // all issued MMAs complete before TMEM is released
            umma_commit(&bars->mma_done);
            mbar_wait(&bars->mma_done, 0, g.timeout_ns, status, abort);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31
        const int q = warp & 3;
        int abuf = 0;
        uint32_t aphase = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int done = 0;
            if (lane == 0) done = mbar_wait(&bars->acc_full[abuf], aphase, g.timeout_ns, status, abort) ? 1 : 0;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) break;
            tc_fence_after();
            int tm, tn;
            tile_coords(t, tiles_m, tiles_n, tm, tn);
            const int64_t row = int64_t(tm) * BM + q * 32 + lane;
            const uint32_t t_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(abuf * BN);
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(t_base + uint32_t(c0), r);
                tmem_ld_wait();
                const int64_t col0 = int64_t(tn) * BN + c0;
                if (row < g.M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t col = col0 + j;
                        if (col < g.N) {
                            float v = g.alpha * __uint_as_float(r[j]);
                            if (OUT_BF16) {
                                __nv_bfloat16* Cp = static_cast<__nv_bfloat16*>(g.C) + row + col * g.ldc;
                                if (g.beta != 0.f) v = fmaf(g.beta, __bfloat162float(*Cp), v);
                                *Cp = __float2bfloat16_rn(v);
                            } else {
                                float* Cp = static_cast<float*>(g.C) + row + col * g.ldc;
                                if (g.beta != 0.f) v = fmaf(g.beta, *Cp, v);
                                *Cp = v;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->acc_empty[abuf]);
            abuf ^= 1;
            if (abuf == 0) aphase ^= 1u;
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, C_::TMEM_COLS);
}

template <int BN, bool TF32, bool OUT_BF16>
hsmm_status_t launch_plain(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, cudaStream_t st) {
    using C_ = Cfg<BN, TF32>;
    auto kern = gemm_tc_kernel<BN, TF32, OUT_BF16>;
    static bool attr_done = false;
    if (!attr_done) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C_::SMEM_BYTES) != cudaSuccess)
            return record_cuda(cudaGetLastError());
        attr_done = true;
    }
    const int tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    const int grid = std::min(tiles, num_sms());
    kern<<<grid, kNumThreads, C_::SMEM_BYTES, st>>>(ta, tb, g);
    count_launches(1);
    return check_launch();
}

}  // namespace

hsmm_status_t gemm_tc(hsmm_dtype_t ab, hsmm_dtype_t c, hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k,
                      float alpha, const void* A, int64_t lda, const void* B, int64_t ldb, float beta, void* C,
                      int64_t ldc, int tile_n, cudaStream_t st) {
    const bool tf32 = (ab == HSMM_R_32F);
    const int esize = tf32 ? 4 : 2;
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return HSMM_STATUS_NOT_SUPPORTED;
    if (!tma_operand_ok(A, lda, esize) || !tma_operand_ok(B, ldb, esize)) return HSMM_STATUS_NOT_SUPPORTED;
    const int BN = (tile_n == 128) ? 128 : 256;
    const int BK = 128 / esize, MN_CHUNK = 128 / esize;
    GemmArgs g{};
    g.M = int(m); g.N = int(n); g.K = int(k);
    g.a_mn = (ta == HSMM_OP_N);   // A stored m x k: M contiguous
    g.b_mn = (tb == HSMM_OP_T);   // B stored n x k: N contiguous
    g.alpha = alpha; g.beta = beta; g.C = C; g.ldc = ldc;
    g.timeout_ns = wait_timeout_ns();
    CUtensorMap mA, mB;
    bool ok = g.a_mn ? encode_map(&mA, dt, esize, A, uint64_t(m), uint64_t(k), uint64_t(lda), MN_CHUNK, BK)
                     : encode_map(&mA, dt, esize, A, uint64_t(k), uint64_t(m), uint64_t(lda), BK, BM);
    ok = ok && (g.b_mn ? encode_map(&mB, dt, esize, B, uint64_t(n), uint64_t(k), uint64_t(ldb), MN_CHUNK, BK)
                       : encode_map(&mB, dt, esize, B, uint64_t(k), uint64_t(n), uint64_t(ldb), BK, uint32_t(BN)));
    if (!ok) return HSMM_STATUS_NOT_SUPPORTED;
    const bool out_bf16 = (c == HSMM_R_16BF);
    if (tf32) {
        if (out_bf16) return HSMM_STATUS_NOT_SUPPORTED;
        return BN == 128 ? launch_plain<128, true, false>(mA, mB, g, st) : launch_plain<256, true, false>(mA, mB, g, st);
    }
    if (out_bf16)
        return BN == 128 ? launch_plain<128, false, true>(mA, mB, g, st) : launch_plain<256, false, true>(mA, mB, g, st);
    return BN == 128 ? launch_plain<128, false, false>(mA, mB, g, st) : launch_plain<256, false, false>(mA, mB, g, st);
}

}  // namespace hsmm
