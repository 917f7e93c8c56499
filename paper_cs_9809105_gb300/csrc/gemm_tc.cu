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
//                       coalesced stores of column-major C (the CTA-pair kernel
//                       below stages 32 x 32 blocks in shared memory and writes
//                       them by TMA stores when beta == 0).
//
// The kernel is persistent (one CTA per SM, tiles strided by the grid) and the
// two TMEM accumulators let the epilogue of tile t overlap the main loop of
// tile t+1.  The transposed forms A^T B, A B^T (Section 8: "on the same footing")
// cost nothing extra: an operand whose M/N index is contiguous is loaded as
// MN chunks of one 128-byte row (64 BF16 or 32 TF32 elements) and described to the
// MMA as MN-major, one whose K index is contiguous as K-major rows.  Ragged edges come from TMA out-of-bounds zero fill.
//
// The same main loop, fed with a different tile schedule and epilogue, runs the
// grouped launch (many problems, one persistent grid; gemm_grouped.cu) and, with a
// k-schedule over slice pairs, the slice products of the FP64-accurate form
// (gemm_ozaki_tc.cu).
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc_tile.cuh"
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

static thread_local int g_last_encode_result = 0;

int last_encode_result() { return g_last_encode_result; }

// The last few encoded maps of this host thread, keyed by every argument of encode_map: a
// repeated product (the same operands, as in every step of a training loop) reuses them
// instead of encoding again.  A map depends on nothing but these arguments.
namespace {
struct MapKey {
    uint64_t base, inner, outer, ld, batch, batch_stride;
    uint32_t box_inner, box_outer, box_batch;
    int32_t dt, esize, swizzle;
};
struct MapCacheEntry {
    CUtensorMap map;
    MapKey key;
    bool valid;
};
constexpr int kMapCache = 16;
thread_local MapCacheEntry t_map_cache[kMapCache];
thread_local int t_map_next = 0;
}  // namespace

// 2D (or 3D with a batch dimension) tiled map with 128-byte swizzle.
bool encode_map(CUtensorMap* map, CUtensorMapDataType dt, int esize, const void* base, uint64_t inner, uint64_t outer,
                uint64_t ld, uint32_t box_inner, uint32_t box_outer, uint64_t batch, uint64_t batch_stride_elems,
                CUtensorMapSwizzle swizzle, uint32_t box_batch) {
    MapKey key;
    std::memset(&key, 0, sizeof(key));
    key.base = reinterpret_cast<uintptr_t>(base); key.inner = inner; key.outer = outer; key.ld = ld;
    key.batch = batch; key.batch_stride = batch_stride_elems;
    key.box_inner = box_inner; key.box_outer = box_outer; key.box_batch = box_batch;
    key.dt = int32_t(dt); key.esize = esize; key.swizzle = int32_t(swizzle);
    for (int i = 0; i < kMapCache; ++i)
        if (t_map_cache[i].valid && std::memcmp(&t_map_cache[i].key, &key, sizeof(key)) == 0) {
            *map = t_map_cache[i].map;
            g_last_encode_result = 0;
            return true;
        }
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {inner, outer, batch};
    cuuint64_t strides[2] = {ld * uint64_t(esize), batch_stride_elems * uint64_t(esize)};
    cuuint32_t box[3] = {box_inner, box_outer, box_batch};
    cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t rank = batch ? 3 : 2;
    CUresult r = fn(map, dt, rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        // a host thread that has not touched the runtime yet may have no current context:
        // make the current device's primary context current and encode once more
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess)
            r = fn(map, dt, rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    g_last_encode_result = int(r);
    if (r != CUDA_SUCCESS) return false;
    MapCacheEntry& e = t_map_cache[t_map_next];
    t_map_next = (t_map_next + 1) % kMapCache;
    e.map = *map;
    e.key = key;
    e.valid = true;
    return true;
}

namespace {

using namespace tc;

constexpr int kNumThreads = 192;   // 6 warps: producer, MMA, 4 x epilogue

struct GemmArgs {
    int M, N, K;
    int a_mn, b_mn;
    int a_mn3, b_mn3;       // MN-major operand loaded as one 3D box of MN chunks (see gemm_tc)
    float alpha, beta;
    void* C;
    int64_t ldc;
    uint64_t timeout_ns;
    int c_tma;              // pair kernel: beta == 0 and C written by TMA stores through tmC
    int m_tma;              // rows of C that tmC covers: M rounded down to whole 16-byte units
};

// ---------------------------------------------------------------------------
// Plain product kernel
// ---------------------------------------------------------------------------
// Stages of the one-CTA plain kernel: what fits beside four epilogue warps' two 32 x 32 FP32
// staging buffers (C leaves by TMA stores, as in the pair kernel below).
constexpr int S1_STAGE_C = 4 * 2 * 32 * 32 * 4;
template <class C_>
struct OneCta {
    static constexpr int FIT = (227 * 1024 - 2048 - S1_STAGE_C) / C_::STAGE_BYTES;
    static constexpr int STAGES = FIT > 8 ? 8 : FIT;
    static constexpr int SMEM = STAGES * C_::STAGE_BYTES + S1_STAGE_C + 1024 + 256;
    static_assert(STAGES >= 3 && SMEM <= 227 * 1024, "one-CTA plain kernel shared memory");
};

template <int BN, bool TF32, bool OUT_BF16>
__global__ void __launch_bounds__(kNumThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, GemmArgs g) {
    using C_ = Cfg<BN, TF32>;
    constexpr int STAGES = OneCta<C_>::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint8_t* stage_c = smem + STAGES * C_::STAGE_BYTES;
    Bars* bars = reinterpret_cast<Bars*>(stage_c + S1_STAGE_C);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_gemm_tc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
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
        if (g.c_tma) tma_prefetch_desc(&tmC);
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
    // launched as a programmatic dependent: the setup above overlapped the previous kernel;
    // the producer and the epilogue wait for it before touching global memory
    pdl_trigger();

    const int tiles_m = (g.M + BM - 1) / BM;
    const int tiles_n = (g.N + BN - 1) / BN;
    const int ntiles = tiles_m * tiles_n;
    const int nkb = (g.K + C_::BK - 1) / C_::BK;

    if (warp == 0) {
        if (lane == 0) {
            pdl_wait();   // A and B may be written by the previous kernel
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
                    load_operand<C_, BM>(a_dst, &tmA, &bars->full[stage], g.a_mn, tm * BM, kb, 0, false, g.a_mn3);
                    load_operand<C_, BN>(b_dst, &tmB, &bars->full[stage], g.b_mn, tn * BN, kb, 0, false, g.b_mn3);
                    last_parity[stage] = int(phase);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            // make sure no bulk copy is still landing in shared memory
            for (int s = 0; s < STAGES; ++s)
                if (last_parity[s] >= 0) mbar_wait(&bars->full[s], uint32_t(last_parity[s]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int abuf = 0;
            uint32_t aphase = 0;
            const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, g.a_mn != 0, g.b_mn != 0, BM, BN);
            const uint64_t a0 = operand_desc<C_>(smem_u32(smem), 0, g.a_mn != 0);
            const uint64_t b0 = operand_desc<C_>(smem_u32(smem) + C_::A_BYTES, 0, g.b_mn != 0);
            const uint64_t aks = ks_step<C_>(g.a_mn != 0), bks = ks_step<C_>(g.b_mn != 0);
            const uint64_t sstep = uint64_t(C_::STAGE_BYTES / 16);
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                if (!mbar_wait(&bars->acc_empty[abuf], aphase ^ 1u, g.timeout_ns, status, abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + uint32_t(abuf * BN);
                bool ok = true;
                // lean issue loop: descriptors from the stage index, four k-blocks per unrolled iteration
#pragma unroll 4
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&bars->full[stage], phase, g.timeout_ns, status, abort)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t ad = a0 + uint64_t(stage) * sstep, bd = b0 + uint64_t(stage) * sstep;
#pragma unroll
                    for (int ks = 0; ks < C_::KSTEPS; ++ks) {
                        const uint32_t acc = ks == 0 ? uint32_t(kb) : 1u;
                        if (TF32)
                            umma_tf32(d_tmem, ad + ks * aks, bd + ks * bks, idesc, acc);
                        else
                            umma_f16(d_tmem, ad + ks * aks, bd + ks * bks, idesc, acc);
                    }
                    umma_commit(&bars->empty[stage]);
                    stage = (stage + 1 == STAGES) ? 0 : stage + 1;
                    phase ^= (stage == 0) ? 1u : 0u;
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
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31; with beta == 0 and a TMA-able C,
        // 32 x 32 blocks go out through two shared-memory buffers per warp by TMA stores (the
        // map covers the rows up to the last whole 16-byte unit; the lanes of the rows after it
        // store directly), else element by element
        const int q = warp & 3;
        float* stage_w = reinterpret_cast<float*>(stage_c) + (warp - 2) * 2 * 32 * 32;
        int abuf = 0;
        uint32_t aphase = 0;
        uint32_t cbuf = 0;
        pdl_wait();   // C may be read or written by the previous kernel
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int done = 0;
            if (lane == 0) done = mbar_wait(&bars->acc_full[abuf], aphase, g.timeout_ns, status, abort) ? 1 : 0;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) break;
            tc_fence_after();
            int tm, tn;
            tile_coords(t, tiles_m, tiles_n, tm, tn);
            const int row0 = tm * BM + q * 32;
            const int64_t row = int64_t(row0) + lane;
            const uint32_t t_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(abuf * BN);
            if (g.c_tma && row0 < g.M) {
                const int cols = min(BN, g.N - tn * BN);
                const bool tail_lane = row >= g.m_tma && row < g.M;
#pragma unroll 1
                for (int c0 = 0; c0 < cols; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(t_base + uint32_t(c0), r);
                    tmem_ld_wait();
                    if (row0 < g.m_tma) {
                        float* sb = stage_w + (cbuf & 1u) * 32 * 32;
                        if (lane == 0) bulk_wait_group_read<1>();   // the store that last used this buffer has read it
                        __syncwarp();
                        if (OUT_BF16) {
                            __nv_bfloat16* sh = reinterpret_cast<__nv_bfloat16*>(sb);
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                sh[j * 32 + lane] = __float2bfloat16_rn(g.alpha * __uint_as_float(r[j]));
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j) sb[j * 32 + lane] = g.alpha * __uint_as_float(r[j]);
                        }
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_2d(&tmC, sb, row0, tn * BN + c0);
                            bulk_commit_group();
                        }
                        ++cbuf;
                    }
                    if (tail_lane) {
                        const int64_t col0 = int64_t(tn) * BN + c0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (col0 + j < g.N) {
                                const float v = g.alpha * __uint_as_float(r[j]);
                                if (OUT_BF16)
                                    static_cast<__nv_bfloat16*>(g.C)[row + (col0 + j) * g.ldc] = __float2bfloat16_rn(v);
                                else
                                    static_cast<float*>(g.C)[row + (col0 + j) * g.ldc] = v;
                            }
                        }
                    }
                }
            } else if (!g.c_tma) {
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
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->acc_empty[abuf]);
            abuf ^= 1;
            if (abuf == 0) aphase ^= 1u;
        }
        if (lane == 0) bulk_wait_group<0>();   // every bulk store complete before the CTA leaves
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, C_::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Plain product on a CTA pair: 256 x 256 tile, cta_group::2
// ---------------------------------------------------------------------------
// As gemm_tc_kernel, but two CTAs of a cluster share one 256 x 256 tile: the even
// CTA stages A rows 0-127 and B columns 0-127 of each k-slab, the odd CTA rows
// 128-255 and columns 128-255; the even CTA issues tcgen05.mma.cta_group::2
// (M = 256, N = 256), which writes each CTA's 128 x 256 accumulator into its own
// TMEM.  32 KiB per stage and CTA instead of 48 KiB.  Both CTAs' copies complete on
// the even CTA's `full` barrier; the commits that free a stage or publish an
// accumulator are multicast to both.
//
// The epilogue of a tile must end within the next tile's main loop (the accumulator
// is double-buffered), and with k = 2048 that loop is only 32 k-blocks (~16K cycles).
// Element-wise global stores (a 64-bit address and a 2- or 4-byte store per element)
// took about as long; so with beta == 0 and a TMA-able C each warp stages 32 x 32
// blocks in shared memory and writes them with one TMA store each (clipped at the
// matrix edge by the TMA unit), which leaves room for six stages.
#ifndef PP_STAGES_CFG
#define PP_STAGES_CFG 6
#define PP_EPI_CFG 4
#define PP_CBUF_CFG 2
#endif
constexpr int PP_STAGES = PP_STAGES_CFG;
constexpr int PP_EPI_WARPS = PP_EPI_CFG;                   // 4: one per TMEM lane quarter; 8: two, half the columns each
constexpr int PP_CBUF = PP_CBUF_CFG;                       // staging buffers per epilogue warp
constexpr int PP_THREADS = 64 + 32 * PP_EPI_WARPS;         // producer, MMA issuer, epilogue
constexpr int PP_STAGE_C = PP_EPI_WARPS * PP_CBUF * 32 * 32 * 4;
constexpr int PP_SMEM = PP_STAGES * PAIR_STAGE_BYTES + PP_STAGE_C + 1024 + 256;
static_assert(PP_SMEM <= 227 * 1024, "plain pair kernel shared memory");
static_assert(PP_STAGES <= 8 && (PP_EPI_WARPS == 4 || PP_EPI_WARPS == 8) && (PP_CBUF == 1 || PP_CBUF == 2),
              "plain pair kernel configuration");

template <bool TF32, bool OUT_BF16>
__global__ void __launch_bounds__(PP_THREADS, 1)
    gemm_tc_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, GemmArgs g) {
    using C_ = Cfg<256, TF32>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint8_t* stage_c = smem + PP_STAGES * PAIR_STAGE_BYTES;
    Bars* bars = reinterpret_cast<Bars*>(stage_c + PP_STAGE_C);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_gemm_tc;
    const uint32_t rank = cluster_ctarank() & 1u;
    const bool leader = (rank == 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < PP_STAGES; ++s) {
            mbar_init(&bars->full[s], 1);
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], 2 * PP_EPI_WARPS);
        }
        mbar_init(&bars->mma_done, 1);
        bars->abort = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
        if (g.c_tma) tma_prefetch_desc(&tmC);
    }
    if (warp == 1) {
        tmem_alloc_pair(&bars->tmem_base, 512);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;
    // launched as a programmatic dependent: everything above overlapped the previous kernel of
    // the stream; the roles that touch global memory (operand loads, C) wait for it below, and
    // the next kernel may be scheduled as soon as every CTA of this one has got here
    pdl_trigger();

    const int tiles_m = (g.M + 2 * BM - 1) / (2 * BM);
    const int tiles_n = (g.N + PAIR_BN - 1) / PAIR_BN;
    const int ntiles = tiles_m * tiles_n;
    const int pair = int(blockIdx.x >> 1), npairs = int(gridDim.x >> 1);
    const int nkb = (g.K + C_::BK - 1) / C_::BK;

    if (warp == 0) {
        if (lane == 0) {
            pdl_wait();   // A and B may be written by the previous kernel
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[8];
            for (int i = 0; i < 8; ++i) last_parity[i] = -1;
            bool ok = true;
            for (int t = pair; t < ntiles && ok && !*abort; t += npairs) {
                int tm, tn;
                tile_coords(t, tiles_m, tiles_n, tm, tn);
                const int arow = tm * 2 * BM + int(rank) * BM;
                const int brow = tn * PAIR_BN + int(rank) * BM;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&bars->empty[stage], phase ^ 1u, g.timeout_ns, status, abort)) { ok = false; break; }
                    uint8_t* a_dst = smem + stage * PAIR_STAGE_BYTES;
                    uint8_t* b_dst = a_dst + BM * 128;
                    const uint32_t full_leader = mapa_shared(smem_u32(&bars->full[stage]), 0);
                    if (leader) mbar_arrive_expect_tx(&bars->full[stage], 2 * PAIR_STAGE_BYTES);
                    if (!g.a_mn) {
                        tma_load_2d_pair(a_dst, &tmA, full_leader, kb * C_::BK, arow);
                    } else if (g.a_mn3) {
                        tma_load_3d_pair(a_dst, &tmA, full_leader, 0, kb * C_::BK, arow / C_::MN_CHUNK);
                    } else {
#pragma unroll
                        for (int c = 0; c < BM / C_::MN_CHUNK; ++c)
                            tma_load_2d_pair(a_dst + c * C_::BK * 128, &tmA, full_leader, arow + c * C_::MN_CHUNK,
                                             kb * C_::BK);
                    }
                    if (!g.b_mn) {
                        tma_load_2d_pair(b_dst, &tmB, full_leader, kb * C_::BK, brow);
                    } else if (g.b_mn3) {
                        tma_load_3d_pair(b_dst, &tmB, full_leader, 0, kb * C_::BK, brow / C_::MN_CHUNK);
                    } else {
#pragma unroll
                        for (int c = 0; c < BM / C_::MN_CHUNK; ++c)
                            tma_load_2d_pair(b_dst + c * C_::BK * 128, &tmB, full_leader, brow + c * C_::MN_CHUNK,
                                             kb * C_::BK);
                    }
                    last_parity[stage] = int(phase);
                    if (++stage == PP_STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            for (int i = 0; i < PP_STAGES; ++i)
                if (last_parity[i] >= 0) mbar_wait(&bars->empty[i], uint32_t(last_parity[i]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, g.a_mn != 0, g.b_mn != 0, 2 * BM, PAIR_BN);
            const uint64_t a0 = operand_desc<C_>(smem_u32(smem), 0, g.a_mn != 0);
            const uint64_t b0 = operand_desc<C_>(smem_u32(smem) + BM * 128, 0, g.b_mn != 0);
            const uint64_t aks = ks_step<C_>(g.a_mn != 0), bks = ks_step<C_>(g.b_mn != 0);
            const uint64_t sstep = uint64_t(PAIR_STAGE_BYTES / 16);
            int stage = 0;
            uint32_t phase = 0;
            int abuf = 0;
            uint32_t aphase = 0;
            bool ok = true;
            for (int t = pair; t < ntiles && ok && !*abort; t += npairs) {
                if (!mbar_wait(&bars->acc_empty[abuf], aphase ^ 1u, g.timeout_ns, status, abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + uint32_t(abuf * PAIR_BN);
                // lean issue loop (the single issuing thread must keep up with the tensor pipe):
                // descriptors from the stage index, four k-blocks per unrolled iteration
#pragma unroll 4
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&bars->full[stage], phase, g.timeout_ns, status, abort)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t ad = a0 + uint64_t(stage) * sstep, bd = b0 + uint64_t(stage) * sstep;
#pragma unroll
                    for (int ks = 0; ks < C_::KSTEPS; ++ks) {
                        const uint32_t acc = ks == 0 ? uint32_t(kb) : 1u;
                        if (TF32)
                            umma_tf32_pair(d_tmem, ad + ks * aks, bd + ks * bks, idesc, acc);
                        else
                            umma_f16_pair(d_tmem, ad + ks * aks, bd + ks * bks, idesc, acc);
                    }
                    umma_commit_pair(&bars->empty[stage], 0x3);
                    stage = (stage + 1 == PP_STAGES) ? 0 : stage + 1;
                    phase ^= (stage == 0) ? 1u : 0u;
                }
                if (!ok) break;
                umma_commit_pair(&bars->acc_full[abuf], 0x3);
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1u;
            }
            umma_commit_pair(&bars->mma_done, 0x1);
            mbar_wait(&bars->mma_done, 0, g.timeout_ns, status, abort);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. of this CTA's 128 rows and, with eight
        // epilogue warps, the column half (w-2)/4 of them
        const int q = warp & 3;
        const int half = PP_EPI_WARPS == 8 ? (warp - 2) >> 2 : 0;
        const int cbeg = PP_EPI_WARPS == 8 ? half * (PAIR_BN / 2) : 0;
        const int cend = PP_EPI_WARPS == 8 ? cbeg + PAIR_BN / 2 : PAIR_BN;
        float* stage_w = reinterpret_cast<float*>(stage_c) + (warp - 2) * PP_CBUF * 32 * 32;
        const uint32_t acc_empty_leader0 = mapa_shared(smem_u32(&bars->acc_empty[0]), 0);
        const uint32_t acc_empty_leader1 = mapa_shared(smem_u32(&bars->acc_empty[1]), 0);
        int abuf = 0;
        uint32_t aphase = 0;
        uint32_t cbuf = 0;
        pdl_wait();   // C may be read or written by the previous kernel
        for (int t = pair; t < ntiles; t += npairs) {
            int done = 0;
            if (lane == 0) done = mbar_wait(&bars->acc_full[abuf], aphase, g.timeout_ns, status, abort) ? 1 : 0;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) break;
            tc_fence_after();
            int tm, tn;
            tile_coords(t, tiles_m, tiles_n, tm, tn);
            const int row0 = tm * 2 * BM + int(rank) * BM + q * 32;   // first row of this warp
            const uint32_t t_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(abuf * PAIR_BN);
            if (g.c_tma && row0 < g.M) {
                // a TMA store clips the row (inner) dimension only to whole 16-byte units, so tmC
                // covers the first m_tma rows; the (at most 7) rows after them are stored by their lanes
                const int cols = min(cend, g.N - tn * PAIR_BN);
                const int64_t row = int64_t(row0) + lane;
                const bool tail_lane = row >= g.m_tma && row < g.M;
#pragma unroll 1
                for (int c0 = cbeg; c0 < cols; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(t_base + uint32_t(c0), r);
                    tmem_ld_wait();
                    if (row0 < g.m_tma) {
                        float* sb = stage_w + (cbuf % PP_CBUF) * 32 * 32;
                        if (lane == 0) {    // the store that last used this buffer has read it
                            if (PP_CBUF == 2) bulk_wait_group_read<1>();
                            else bulk_wait_group_read<0>();
                        }
                        __syncwarp();
                        if (OUT_BF16) {
                            __nv_bfloat16* sh = reinterpret_cast<__nv_bfloat16*>(sb);
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                sh[j * 32 + lane] = __float2bfloat16_rn(g.alpha * __uint_as_float(r[j]));
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j) sb[j * 32 + lane] = g.alpha * __uint_as_float(r[j]);
                        }
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_2d(&tmC, sb, row0, tn * PAIR_BN + c0);
                            bulk_commit_group();
                        }
                        ++cbuf;
                    }
                    if (tail_lane) {
                        const int64_t col0 = int64_t(tn) * PAIR_BN + c0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (col0 + j < g.N) {
                                const float v = g.alpha * __uint_as_float(r[j]);
                                if (OUT_BF16)
                                    static_cast<__nv_bfloat16*>(g.C)[row + (col0 + j) * g.ldc] = __float2bfloat16_rn(v);
                                else
                                    static_cast<float*>(g.C)[row + (col0 + j) * g.ldc] = v;
                            }
                        }
                    }
                }
            } else if (!g.c_tma) {
                const int64_t row = int64_t(row0) + lane;
#pragma unroll 1
                for (int c0 = cbeg; c0 < cend; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(t_base + uint32_t(c0), r);
                    tmem_ld_wait();
                    const int64_t col0 = int64_t(tn) * PAIR_BN + c0;
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
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (leader) mbar_arrive(&bars->acc_empty[abuf]);
                else mbar_arrive_remote(abuf ? acc_empty_leader1 : acc_empty_leader0);
            }
            abuf ^= 1;
            if (abuf == 0) aphase ^= 1u;
        }
        if (lane == 0) bulk_wait_group<0>();   // every bulk store complete before the CTA leaves
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync_all();
    tc_fence_after();
    if (warp == 1) tmem_dealloc_pair(tmem, 512);
}

template <bool TF32, bool OUT_BF16>
hsmm_status_t launch_pair(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc_, const GemmArgs& g,
                          cudaStream_t st) {
    auto kern = gemm_tc_pair_kernel<TF32, OUT_BF16>;
    static std::atomic<uint64_t> attrs{0};
    const hsmm_status_t as = attrs_once_per_device(
        attrs, [kern] { return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, PP_SMEM); });
    if (as != HSMM_STATUS_SUCCESS) return as;
    const int ptiles = ((g.M + 2 * BM - 1) / (2 * BM)) * ((g.N + PAIR_BN - 1) / PAIR_BN);
    const int pairs = std::max(1, std::min(ptiles, num_sms() / 2));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(unsigned(2 * pairs), 1, 1);
    lc.blockDim = dim3(PP_THREADS, 1, 1);
    lc.dynamicSmemBytes = PP_SMEM;
    lc.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // see pdl_wait in the kernel
    at[1].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 2;
    cudaError_t e = cudaLaunchKernelEx(&lc, kern, ta, tb, tc_, g);
    count_launches(1);
    if (e != cudaSuccess) return record_cuda(e);
    return check_launch();
}

template <int BN, bool TF32, bool OUT_BF16>
hsmm_status_t launch_plain(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tc_, const GemmArgs& g,
                           cudaStream_t st) {
    using C_ = Cfg<BN, TF32>;
    constexpr int smem = OneCta<C_>::SMEM;
    auto kern = gemm_tc_kernel<BN, TF32, OUT_BF16>;
    static std::atomic<uint64_t> attrs{0};
    const hsmm_status_t as = attrs_once_per_device(
        attrs, [kern] { return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); });
    if (as != HSMM_STATUS_SUCCESS) return as;
    const int tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(unsigned(std::min(tiles, num_sms())), 1, 1);
    lc.blockDim = dim3(kNumThreads, 1, 1);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // see pdl_wait in the kernel
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&lc, kern, ta, tb, tc_, g);
    count_launches(1);
    if (e != cudaSuccess) return record_cuda(e);
    return check_launch();
}

}  // namespace

// Plain 256-wide tiles run on CTA pairs unless HSMM_GEMM_KERNEL=single selects one CTA per tile.
static bool gemm_pair_enabled() {
    const char* v = std::getenv("HSMM_GEMM_KERNEL");
    return !(v && std::strcmp(v, "single") == 0);
}

hsmm_status_t gemm_tc(hsmm_dtype_t ab, hsmm_dtype_t c, hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k,
                      float alpha, const void* A, int64_t lda, const void* B, int64_t ldb, float beta, void* C,
                      int64_t ldc, int tile_n, cudaStream_t st) {
    const bool tf32 = (ab == HSMM_R_32F);
    const int esize = tf32 ? 4 : 2;
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "gemm: a dimension exceeds 2^31-1");
    if (!tma_operand_ok(A, lda, esize) || !tma_operand_ok(B, ldb, esize))
        return fail(HSMM_STATUS_NOT_SUPPORTED,
                    "gemm: TMA needs 16-byte aligned A, B and ld*size multiples of 16 (A %% 16 = %d, lda = %lld, "
                    "B %% 16 = %d, ldb = %lld)",
                    int(reinterpret_cast<uintptr_t>(A) % 16), (long long)lda, int(reinterpret_cast<uintptr_t>(B) % 16),
                    (long long)ldb);
    // MN-major TF32 operands are staged with 128-byte swizzling of 32-byte units
    const CUtensorMapSwizzle mn_sw = tf32 ? CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B : CU_TENSOR_MAP_SWIZZLE_128B;
    const int BN = (tile_n == 128) ? 128 : 256;
    const int BK = 128 / esize, MN_CHUNK = 128 / esize;
    GemmArgs g{};
    g.M = int(m); g.N = int(n); g.K = int(k);
    g.a_mn = (ta == HSMM_OP_N);   // A stored m x k: M contiguous
    g.b_mn = (tb == HSMM_OP_T);   // B stored n x k: N contiguous
    g.alpha = alpha; g.beta = beta; g.C = C; g.ldc = ldc;
    g.timeout_ns = wait_timeout_ns();
    // An MN-major operand whose MN extent is a whole number of chunks is described as a 3D
    // tensor {chunk, K, extent / chunk}, so that the rows of one stage (two or four chunks) come
    // in ONE TMA load instead of one per chunk: the producer thread issues half or a quarter of
    // the instructions (the box then never reaches past the last row, so nothing outside the
    // operand is read).
    g.a_mn3 = g.a_mn && (m % MN_CHUNK == 0);
    g.b_mn3 = g.b_mn && (n % MN_CHUNK == 0);
    auto enc_mn3 = [&](CUtensorMap* map, const void* base, int64_t ext, int64_t ld, int rows) {
        return encode_map(map, dt, esize, base, uint64_t(MN_CHUNK), uint64_t(k), uint64_t(ld), MN_CHUNK, BK,
                          uint64_t(ext / MN_CHUNK), uint64_t(MN_CHUNK), mn_sw, uint32_t(rows / MN_CHUNK));
    };
    const bool out_bf16 = (c == HSMM_R_16BF);
    // C through TMA stores of 32 x 32 blocks when beta == 0 and C is TMA-able; the map covers
    // the rows up to the last whole 16-byte unit (a store clips rows only to such units)
    CUtensorMap pC;
    std::memset(&pC, 0, sizeof(pC));
    const int esc = out_bf16 ? 2 : 4;
    g.m_tma = int(m - m % (16 / esc));
    g.c_tma = (beta == 0.f && g.m_tma > 0 && tma_operand_ok(C, ldc, size_t(esc)) &&
               encode_map(&pC, out_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, esc, C,
                          uint64_t(g.m_tma), uint64_t(n), uint64_t(ldc), 32, 32, 0, 0, CU_TENSOR_MAP_SWIZZLE_NONE))
                  ? 1 : 0;
    // CTA pairs for 256-wide tiles whenever M fills more than one 128-row half
    if (BN == 256 && m > BM && gemm_pair_enabled()) {
        CUtensorMap pA, pB;
        bool okp = g.a_mn ? (g.a_mn3 ? enc_mn3(&pA, A, m, lda, BM)
                                     : encode_map(&pA, dt, esize, A, uint64_t(m), uint64_t(k), uint64_t(lda), MN_CHUNK,
                                                  BK, 0, 0, mn_sw))
                          : encode_map(&pA, dt, esize, A, uint64_t(k), uint64_t(m), uint64_t(lda), BK, BM);
        okp = okp && (g.b_mn ? (g.b_mn3 ? enc_mn3(&pB, B, n, ldb, BM)
                                        : encode_map(&pB, dt, esize, B, uint64_t(n), uint64_t(k), uint64_t(ldb),
                                                     MN_CHUNK, BK, 0, 0, mn_sw))
                             : encode_map(&pB, dt, esize, B, uint64_t(k), uint64_t(n), uint64_t(ldb), BK, BM));
        if (!okp) return fail(HSMM_STATUS_NOT_SUPPORTED, "gemm: TMA descriptor encoding failed (CUresult %d)",
                              g_last_encode_result);
        if (tf32) {
            if (out_bf16) return HSMM_STATUS_NOT_SUPPORTED;
            return launch_pair<true, false>(pA, pB, pC, g, st);
        }
        return out_bf16 ? launch_pair<false, true>(pA, pB, pC, g, st) : launch_pair<false, false>(pA, pB, pC, g, st);
    }
    // one CTA per tile
    CUtensorMap mA, mB;
    bool ok = g.a_mn ? (g.a_mn3 ? enc_mn3(&mA, A, m, lda, BM)
                                : encode_map(&mA, dt, esize, A, uint64_t(m), uint64_t(k), uint64_t(lda), MN_CHUNK, BK, 0,
                                             0, mn_sw))
                     : encode_map(&mA, dt, esize, A, uint64_t(k), uint64_t(m), uint64_t(lda), BK, BM);
    ok = ok && (g.b_mn ? (g.b_mn3 ? enc_mn3(&mB, B, n, ldb, BN)
                                  : encode_map(&mB, dt, esize, B, uint64_t(n), uint64_t(k), uint64_t(ldb), MN_CHUNK, BK,
                                               0, 0, mn_sw))
                       : encode_map(&mB, dt, esize, B, uint64_t(k), uint64_t(n), uint64_t(ldb), BK, uint32_t(BN)));
    if (!ok)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "gemm: TMA descriptor encoding failed (m %lld n %lld k %lld lda %lld "
                    "ldb %lld, A %s-major, B %s-major, CUresult %d)", (long long)m, (long long)n, (long long)k,
                    (long long)lda, (long long)ldb, g.a_mn ? "MN" : "K", g.b_mn ? "MN" : "K",
                    g_last_encode_result);
    if (tf32) {
        if (out_bf16) return HSMM_STATUS_NOT_SUPPORTED;
        return BN == 128 ? launch_plain<128, true, false>(mA, mB, pC, g, st)
                         : launch_plain<256, true, false>(mA, mB, pC, g, st);
    }
    if (out_bf16)
        return BN == 128 ? launch_plain<128, false, true>(mA, mB, pC, g, st)
                         : launch_plain<256, false, true>(mA, mB, pC, g, st);
    return BN == 128 ? launch_plain<128, false, false>(mA, mB, pC, g, st)
                     : launch_plain<256, false, false>(mA, mB, pC, g, st);
}

}  // namespace hsmm
