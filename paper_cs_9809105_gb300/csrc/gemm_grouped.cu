// gemm_grouped.cu -- grouped products on sm_103a: many independent problems
// C_g <- alpha op(A_g) op(B_g) + beta C_g (alpha, beta shared) in one persistent launch.
//
// Each problem is the block product of Eq. PRODUCT (Section 3.1); the paper's cyclic
// mapping (Section 6.2) runs many independent systolic processes side by side, which is the
// same batching idea.  The host flattens every problem into output tiles, one 16-byte
// record per tile, and writes per-problem TMA descriptors, problem records and the tile
// table as one image into device memory (a plan's allocation, or caller workspace through
// kernels whose parameter block carries the image, so that the call allocates nothing and
// can be captured).  The kernels walk the table with the main loop of the plain products
// (gemm_tc.cu): TMA into a ring of shared-memory stages, tcgen05.mma into two TMEM
// accumulators, an epilogue that stores C by TMA in 32 x 32 blocks.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc_tile.cuh"
#include "internal.h"

namespace hsmm {

static __device__ uint32_t g_status_grouped;

uint32_t status_take_grouped() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_grouped, sizeof(v));
    cudaMemcpyToSymbol(g_status_grouped, &z, sizeof(z));
    return v;
}

namespace {

using namespace tc;

constexpr int kNumThreads = 192;   // one-CTA grouped kernel: producer, MMA, 4 x epilogue

// ---------------------------------------------------------------------------
// Grouped products: many independent problems in one persistent launch
// ---------------------------------------------------------------------------
// The host plan flattens every problem into tiles (128 rows on one CTA, 256 on a CTA
// pair; BN_p columns chosen per problem), orders the problems (as given, or longest k
// first so that the long tiles start early), and stores per problem its TMA
// descriptors (A, B, C) and a small record in device memory.  Persistent CTAs walk the
// flattened tile list with a stride of the grid; a host-built table gives each tile's
// problem, coordinates, k-blocks and widths in one 16-byte load, and the producer
// prefetches the next tile's record and descriptors while the current tile streams.
struct GroupedProblem {
    int M, N, K;
    int a_mn, b_mn;
    int bn;                 // tile columns: 128 or 256, or on CTA pairs with K-major B any multiple of 32 to 256
    int tiles_m, tiles_n;
    int64_t tile_start;     // first flattened tile of this problem
    void* C;
    int64_t ldc;
};

struct GroupedArgs {
    const CUtensorMap* maps;          // 3 per problem (A, B, C), 64-byte aligned
    const GroupedProblem* probs;
    const uint4* tiles;               // per flattened tile, see GroupedTile
    int count;
    int64_t total_tiles;
    float alpha, beta;
    uint64_t timeout_ns;
};

// Flattened tile record (16 bytes, one load): x problem, y tile row | tile column << 16,
// z k-blocks, w tile width / 128 (bits 0-1) | A MN-major (2) | B MN-major (3) | C by TMA
// stores (4) | valid rows (8-16, 1..256) | valid columns (17-25, 1..256).  A tile row is
// 128 rows for the one-CTA kernel and 256 for the CTA-pair kernel.
__device__ __forceinline__ int rec_bn(const uint4& r) { return int((r.w >> 26) & 7u) * 32 + 32; }

// A TMA store clips the row (inner) dimension of C only to whole 16-byte units, so a grouped
// problem's C map covers its rows rounded down to such units, and the lanes of the (at most 7)
// rows after them store their 32 values of a column block directly.
struct TailC {
    void* C;
    int64_t ldc;
    int N;
};
template <bool OUT_BF16>
__device__ __forceinline__ void store_tail_row(const TailC& T, int64_t row, int64_t col0, const uint32_t* r, float alpha) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (col0 + j < T.N) {
            const float v = alpha * __uint_as_float(r[j]);
            if (OUT_BF16)
                static_cast<__nv_bfloat16*>(T.C)[row + (col0 + j) * T.ldc] = __float2bfloat16_rn(v);
            else
                static_cast<float*>(T.C)[row + (col0 + j) * T.ldc] = v;
        }
    }
}
__host__ __device__ constexpr int c_rows_unit(bool out_bf16) { return out_bf16 ? 8 : 4; }   // rows per 16-byte unit of C
__device__ __forceinline__ bool rec_amn(const uint4& r) { return (r.w >> 2) & 1u; }
__device__ __forceinline__ bool rec_bmn(const uint4& r) { return (r.w >> 3) & 1u; }
__device__ __forceinline__ bool rec_ctma(const uint4& r) { return (r.w >> 4) & 1u; }
__device__ __forceinline__ int rec_rows(const uint4& r) { return int((r.w >> 8) & 0x1FFu); }
__device__ __forceinline__ int rec_cols(const uint4& r) { return int((r.w >> 17) & 0x1FFu); }

constexpr int GROUPED_STAGE_C = 4 * 2 * 32 * 32 * 4;   // 4 epilogue warps x 2 buffers x 32 x 32 FP32

template <bool TF32, bool OUT_BF16>
__global__ void __launch_bounds__(kNumThreads, 1) gemm_grouped_kernel(GroupedArgs g) {
    using C_ = Cfg<256, TF32>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint8_t* stage_c = smem + C_::STAGES * C_::STAGE_BYTES;
    Bars* bars = reinterpret_cast<Bars*>(stage_c + GROUPED_STAGE_C);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_grouped;

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

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[8];
            for (int i = 0; i < 8; ++i) last_parity[i] = -1;
            bool ok = true;
            uint4 rec = g.tiles[blockIdx.x];
            for (int64_t t = blockIdx.x; t < g.total_tiles && ok && !*abort; t += gridDim.x) {
                const int64_t tnext = t + gridDim.x;
                const uint4 rec_next = tnext < g.total_tiles ? g.tiles[tnext] : rec;
                const int pi = int(rec.x);
                const int tm = int(rec.y & 0xFFFFu), tn = int(rec.y >> 16);
                const int bn = rec_bn(rec), nkb = int(rec.z);
                const bool a_mn = rec_amn(rec), b_mn = rec_bmn(rec);
                const CUtensorMap* mA = g.maps + 3 * pi;
                const CUtensorMap* mB = mA + 1;
                if (tnext < g.total_tiles && rec_next.x != rec.x) {
                    tma_prefetch_desc(g.maps + 3 * rec_next.x);
                    tma_prefetch_desc(g.maps + 3 * rec_next.x + 1);
                }
                const uint32_t bytes = uint32_t(BM + bn) * 128u;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&bars->empty[stage], phase ^ 1u, g.timeout_ns, status, abort)) { ok = false; break; }
                    uint8_t* a_dst = smem + stage * C_::STAGE_BYTES;
                    uint8_t* b_dst = a_dst + C_::A_BYTES;
                    mbar_arrive_expect_tx(&bars->full[stage], bytes);
                    if (!a_mn) {
                        tma_load_2d(a_dst, mA, &bars->full[stage], kb * C_::BK, tm * BM);
                    } else {
                        for (int c = 0; c < BM / C_::MN_CHUNK; ++c)
                            tma_load_2d(a_dst + c * C_::BK * 128, mA, &bars->full[stage], tm * BM + c * C_::MN_CHUNK,
                                        kb * C_::BK);
                    }
                    if (!b_mn) {
                        tma_load_2d(b_dst, mB, &bars->full[stage], kb * C_::BK, tn * bn);
                    } else {
                        for (int c = 0; c < bn / C_::MN_CHUNK; ++c)
                            tma_load_2d(b_dst + c * C_::BK * 128, mB, &bars->full[stage], tn * bn + c * C_::MN_CHUNK,
                                        kb * C_::BK);
                    }
                    last_parity[stage] = int(phase);
                    if (++stage == C_::STAGES) { stage = 0; phase ^= 1u; }
                }
                rec = rec_next;
            }
            for (int i = 0; i < C_::STAGES; ++i)
                if (last_parity[i] >= 0) mbar_wait(&bars->full[i], uint32_t(last_parity[i]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int abuf = 0;
            uint32_t aphase = 0;
            bool ok = true;
            // the next tile's record is loaded while this tile's MMAs are issued
            uint4 rec = g.tiles[blockIdx.x];
            for (int64_t t = blockIdx.x; t < g.total_tiles && ok && !*abort; t += gridDim.x) {
                const int64_t tnext = t + gridDim.x;
                const uint4 rec_next = tnext < g.total_tiles ? g.tiles[tnext] : rec;
                const int nkb = int(rec.z), bn = rec_bn(rec);
                const bool a_mn = rec_amn(rec), b_mn = rec_bmn(rec);
                if (!mbar_wait(&bars->acc_empty[abuf], aphase ^ 1u, g.timeout_ns, status, abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + uint32_t(abuf * 256);
                const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, a_mn, b_mn, BM, uint32_t(bn));
                const uint64_t a0 = operand_desc<C_>(smem_u32(smem), 0, a_mn);
                const uint64_t b0 = operand_desc<C_>(smem_u32(smem) + C_::A_BYTES, 0, b_mn);
                const uint64_t aks = ks_step<C_>(a_mn), bks = ks_step<C_>(b_mn);
                const uint64_t sstep = uint64_t(C_::STAGE_BYTES / 16);
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
                    stage = (stage + 1 == C_::STAGES) ? 0 : stage + 1;
                    phase ^= (stage == 0) ? 1u : 0u;
                }
                if (!ok) break;
                umma_commit(&bars->acc_full[abuf]);
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1u;
                rec = rec_next;
            }
            umma_commit(&bars->mma_done);
            mbar_wait(&bars->mma_done, 0, g.timeout_ns, status, abort);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32*(w%4) ..; with beta == 0 and a TMA-able C each
        // 32 x 32 block goes out through a shared-memory staging buffer as one bulk store
        // (clipped at the matrix edge by the TMA unit), else element by element
        const int q = warp & 3;
        float* stage_w = reinterpret_cast<float*>(stage_c) + q * 2 * 32 * 32;
        int abuf = 0;
        uint32_t aphase = 0;
        uint32_t cbuf = 0;
        uint4 rec = g.tiles[blockIdx.x];
        for (int64_t t = blockIdx.x; t < g.total_tiles; t += gridDim.x) {
            const int64_t tnext = t + gridDim.x;
            const uint4 rec_next = tnext < g.total_tiles ? g.tiles[tnext] : rec;
            int done = 0;
            if (lane == 0) done = mbar_wait(&bars->acc_full[abuf], aphase, g.timeout_ns, status, abort) ? 1 : 0;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) break;
            tc_fence_after();
            const int tm = int(rec.y & 0xFFFFu), tn = int(rec.y >> 16);
            const int bn = rec_bn(rec);
            const uint32_t t_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(abuf * 256);
            if (lane == 0 && tnext < g.total_tiles && rec_next.x != rec.x) tma_prefetch_desc(g.maps + 3 * rec_next.x + 2);
            const bool c_tma = rec_ctma(rec) && g.beta == 0.f;
            if (c_tma && q * 32 < rec_rows(rec)) {
                const int cols = rec_cols(rec);
                const CUtensorMap* mC = g.maps + 3 * rec.x + 2;
                const int rows_tma = rec_rows(rec) & ~(c_rows_unit(OUT_BF16) - 1);
                const bool tail_lane = q * 32 + lane >= rows_tma && q * 32 + lane < rec_rows(rec);
                TailC tc_{nullptr, 0, 0};
                if (q * 32 + 32 > rows_tma) {   // this warp holds rows past the map: read the problem once
                    const GroupedProblem& P = g.probs[rec.x];
                    tc_ = TailC{P.C, P.ldc, P.N};
                }
#pragma unroll 1
                for (int c0 = 0; c0 < cols; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(t_base + uint32_t(c0), r);
                    tmem_ld_wait();
                    if (q * 32 < rows_tma) {
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
                            tma_store_2d(mC, sb, tm * BM + q * 32, tn * bn + c0);
                            bulk_commit_group();
                        }
                        ++cbuf;
                    }
                    if (tail_lane)
                        store_tail_row<OUT_BF16>(tc_, int64_t(tm) * BM + q * 32 + lane, int64_t(tn) * bn + c0, r, g.alpha);
                }
            } else if (!c_tma) {
                const GroupedProblem P = g.probs[rec.x];
                const int64_t row = int64_t(tm) * BM + q * 32 + lane;
#pragma unroll 1
                for (int c0 = 0; c0 < bn; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(t_base + uint32_t(c0), r);
                    tmem_ld_wait();
                    const int64_t col0 = int64_t(tn) * bn + c0;
                    if (row < P.M) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int64_t col = col0 + j;
                            if (col < P.N) {
                                float v = g.alpha * __uint_as_float(r[j]);
                                if (OUT_BF16) {
                                    __nv_bfloat16* Cp = static_cast<__nv_bfloat16*>(P.C) + row + col * P.ldc;
                                    if (g.beta != 0.f) v = fmaf(g.beta, __bfloat162float(*Cp), v);
                                    *Cp = __float2bfloat16_rn(v);
                                } else {
                                    float* Cp = static_cast<float*>(P.C) + row + col * P.ldc;
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
            rec = rec_next;
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
// Grouped products on CTA pairs: 256-row tiles, cta_group::2
// ---------------------------------------------------------------------------
// The grouped launch with the tile of gemm_tc_pair_kernel: each cluster of two CTAs takes
// 256 x BN_p tiles (BN_p per problem, see auto_tile_n) from the flattened table; the even CTA
// stages A rows 0-127 and B columns 0..BN_p/2-1 of each k-slab, the odd CTA the other
// halves, and the even CTA issues M = 256, N = BN_p MMAs that write each CTA's 128 rows
// into its own TMEM.  Per tile and SM that stages (128 + BN_p/2) instead of 128 + BN_p
// rows of operands per k-block: the one-CTA kernel is bound by the bytes its SMs can
// stage, not by the MMAs.  Six 32 KiB stages leave room for the C staging buffers
// (eight epilogue warps with one 4 KiB buffer each).
#ifndef GP_STAGES_CFG
#define GP_STAGES_CFG 6
#define GP_EPI_CFG 8
#define GP_CBUF_CFG 1
#define GP_PRODUCERS_CFG 2
#endif
constexpr int GP_STAGES = GP_STAGES_CFG;
constexpr int GP_EPI_WARPS = GP_EPI_CFG;                   // 4, 8 or 16: 1, 2 or 4 per TMEM lane quarter
constexpr int GP_EPI_PARTS = GP_EPI_WARPS / 4;              // column parts of a tile, one per warp of a quarter
constexpr int GP_CBUF = GP_CBUF_CFG;
constexpr int GP_PRODUCERS = GP_PRODUCERS_CFG;             // warps 0 and (with two) 2
constexpr int GP_THREADS = 96 + 32 * GP_EPI_WARPS;         // producer, MMA issuer, producer or idle, epilogue
constexpr int GP_STAGE_C = GP_EPI_WARPS * GP_CBUF * 32 * 32 * 4;  // 32 x 32 FP32 staging buffers per epilogue warp
constexpr int GP_SMEM = GP_STAGES * PAIR_STAGE_BYTES + GP_STAGE_C + 1024 + 256;
static_assert(GP_SMEM <= 227 * 1024, "grouped pair kernel shared memory");
// The two producers take alternate k-blocks, so with an even stage count each stage always
// belongs to the same producer; with an odd one both would refill it, and a producer's final
// wait for its last use of a stage could name a phase that has already been passed twice.
static_assert(GP_PRODUCERS == 1 || GP_STAGES % 2 == 0, "grouped pair kernel: two producers need an even number of stages");
static_assert(GP_EPI_WARPS == 4 || GP_EPI_WARPS == 8 || GP_EPI_WARPS == 16, "grouped pair kernel: epilogue warps");

// Tile records are read two tiles ahead, so that no role waits on a global load at a tile
// boundary (the producer needs the next record at once, to prefetch its descriptors).
struct RecPipe {
    uint4 cur, next, next2;
};
__device__ __forceinline__ uint4 rec_at(const GroupedArgs& g, int64_t t, const uint4& fallback) {
    return t < g.total_tiles ? g.tiles[t] : fallback;
}

template <bool TF32, bool OUT_BF16>
__global__ void __launch_bounds__(GP_THREADS, 1) gemm_grouped_pair_kernel(GroupedArgs g) {
    using C_ = Cfg<256, TF32>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint8_t* stage_c = smem + GP_STAGES * PAIR_STAGE_BYTES;
    Bars* bars = reinterpret_cast<Bars*>(stage_c + GP_STAGE_C);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_grouped;
    const uint32_t rank = cluster_ctarank() & 1u;
    const bool leader = (rank == 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < GP_STAGES; ++s) {
            mbar_init(&bars->full[s], 1);
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], 2 * GP_EPI_WARPS);
        }
        mbar_init(&bars->mma_done, 1);
        bars->abort = 0;
        fence_mbar_init();
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
    const int64_t pair = int64_t(blockIdx.x >> 1), npairs = int64_t(gridDim.x >> 1);

    if (warp == 0 || (warp == 2 && GP_PRODUCERS == 2)) {
        // two producers (warps 0 and 2), each for every other k-block of the CTA's stream: the
        // TMA loads of a grouped launch name descriptors in global memory, and one issuing
        // thread cannot keep the MMAs fed with them
        if (lane == 0) {
            const int pid = warp == 0 ? 0 : 1;
            int64_t gk = 0;                  // k-blocks of this CTA so far (both producers count all)
            int last_parity[8];
            for (int i = 0; i < 8; ++i) last_parity[i] = -1;
            bool ok = true;
            RecPipe rp;
            rp.cur = g.tiles[pair];
            rp.next = rec_at(g, pair + npairs, rp.cur);
            for (int64_t t = pair; t < g.total_tiles && ok && !*abort; t += npairs) {
                const int64_t tnext = t + npairs;
                rp.next2 = rec_at(g, tnext + npairs, rp.next);
                const uint4 rec = rp.cur, rec_next = rp.next;
                const int pi = int(rec.x);
                const int tm = int(rec.y & 0xFFFFu), tn = int(rec.y >> 16);
                const int bn = rec_bn(rec), nkb = int(rec.z);
                const bool a_mn = rec_amn(rec), b_mn = rec_bmn(rec);
                const CUtensorMap* mA = g.maps + 3 * pi;
                const CUtensorMap* mB = mA + 1;
                if (tnext < g.total_tiles && rec_next.x != rec.x) {
                    tma_prefetch_desc(g.maps + 3 * rec_next.x);
                    tma_prefetch_desc(g.maps + 3 * rec_next.x + 1);
                }
                const int arow = tm * 2 * BM + int(rank) * BM;
                const int bhalf = bn / 2;
                const int brow = tn * bn + int(rank) * bhalf;
                const uint32_t bytes = 2u * uint32_t(BM + bhalf) * 128u;   // both CTAs' copies
                for (int kb = 0; kb < nkb; ++kb, ++gk) {
                    if (GP_PRODUCERS == 2 && int(gk & 1) != pid) continue;
                    const int stage = int(gk % GP_STAGES);
                    const uint32_t phase = uint32_t((gk / GP_STAGES) & 1);
                    if (!mbar_wait(&bars->empty[stage], phase ^ 1u, g.timeout_ns, status, abort)) { ok = false; break; }
                    uint8_t* a_dst = smem + stage * PAIR_STAGE_BYTES;
                    uint8_t* b_dst = a_dst + BM * 128;
                    const uint32_t full_leader = mapa_shared(smem_u32(&bars->full[stage]), 0);
                    if (leader) mbar_arrive_expect_tx(&bars->full[stage], bytes);
                    if (!a_mn) {
                        tma_load_2d_pair(a_dst, mA, full_leader, kb * C_::BK, arow);
                    } else {
                        for (int c = 0; c < BM / C_::MN_CHUNK; ++c)
                            tma_load_2d_pair(a_dst + c * C_::BK * 128, mA, full_leader, arow + c * C_::MN_CHUNK,
                                             kb * C_::BK);
                    }
                    if (!b_mn) {
                        tma_load_2d_pair(b_dst, mB, full_leader, kb * C_::BK, brow);
                    } else {
                        for (int c = 0; c < bhalf / C_::MN_CHUNK; ++c)
                            tma_load_2d_pair(b_dst + c * C_::BK * 128, mB, full_leader, brow + c * C_::MN_CHUNK,
                                             kb * C_::BK);
                    }
                    last_parity[stage] = int(phase);
                }
                rp.cur = rp.next;
                rp.next = rp.next2;
            }
            // the leader's MMAs read both CTAs' stages: a stage is free only once they completed
            for (int i = 0; i < GP_STAGES; ++i)
                if (last_parity[i] >= 0) mbar_wait(&bars->empty[i], uint32_t(last_parity[i]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            int stage = 0;
            uint32_t phase = 0;
            int abuf = 0;
            uint32_t aphase = 0;
            bool ok = true;
            const uint64_t sstep = uint64_t(PAIR_STAGE_BYTES / 16);
            RecPipe rp;
            rp.cur = g.tiles[pair];
            rp.next = rec_at(g, pair + npairs, rp.cur);
            for (int64_t t = pair; t < g.total_tiles && ok && !*abort; t += npairs) {
                rp.next2 = rec_at(g, t + 2 * npairs, rp.next);
                const uint4 rec = rp.cur;
                const int nkb = int(rec.z), bn = rec_bn(rec);
                const bool a_mn = rec_amn(rec), b_mn = rec_bmn(rec);
                if (!mbar_wait(&bars->acc_empty[abuf], aphase ^ 1u, g.timeout_ns, status, abort)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + uint32_t(abuf * 256);
                const uint32_t idesc = make_idesc(TF32 ? 2u : 1u, a_mn, b_mn, 2 * BM, uint32_t(bn));
                const uint64_t a0 = operand_desc<C_>(smem_u32(smem), 0, a_mn);
                const uint64_t b0 = operand_desc<C_>(smem_u32(smem) + BM * 128, 0, b_mn);
                const uint64_t aks = ks_step<C_>(a_mn), bks = ks_step<C_>(b_mn);
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
                    stage = (stage + 1 == GP_STAGES) ? 0 : stage + 1;
                    phase ^= (stage == 0) ? 1u : 0u;
                }
                if (!ok) break;
                umma_commit_pair(&bars->acc_full[abuf], 0x3);
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1u;
                rp.cur = rp.next;
                rp.next = rp.next2;
            }
            umma_commit_pair(&bars->mma_done, 0x1);
            mbar_wait(&bars->mma_done, 0, g.timeout_ns, status, abort);
        }
    } else if (warp >= 3) {
        // epilogue: warp w reads TMEM lanes 32*(w%4) .. of this CTA's 128 rows of the tile and
        // the column part (w-3)/4 of them
        const int q = warp & 3;
        const int part = (warp - 3) >> 2;
        float* stage_w = reinterpret_cast<float*>(stage_c) + (warp - 3) * GP_CBUF * 32 * 32;
        const uint32_t acc_empty_leader0 = mapa_shared(smem_u32(&bars->acc_empty[0]), 0);
        const uint32_t acc_empty_leader1 = mapa_shared(smem_u32(&bars->acc_empty[1]), 0);
        int abuf = 0;
        uint32_t aphase = 0;
        uint32_t cbuf = 0;
        RecPipe rp;
        rp.cur = g.tiles[pair];
        rp.next = rec_at(g, pair + npairs, rp.cur);
        for (int64_t t = pair; t < g.total_tiles; t += npairs) {
            const int64_t tnext = t + npairs;
            rp.next2 = rec_at(g, tnext + npairs, rp.next);
            const uint4 rec = rp.cur, rec_next = rp.next;
            int done = 0;
            if (lane == 0) done = mbar_wait(&bars->acc_full[abuf], aphase, g.timeout_ns, status, abort) ? 1 : 0;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) break;
            tc_fence_after();
            const int tm = int(rec.y & 0xFFFFu), tn = int(rec.y >> 16);
            const int bn = rec_bn(rec);
            const int row_base = int(rank) * BM + q * 32;      // first row of this warp within the tile
            const uint32_t t_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(abuf * 256);
            if (lane == 0 && tnext < g.total_tiles && rec_next.x != rec.x) tma_prefetch_desc(g.maps + 3 * rec_next.x + 2);
            // the column parts of the epilogue warps of one lane quarter, cut at multiples of 32
            const int pcut = (bn / GP_EPI_PARTS + 31) / 32 * 32;
            const int cbeg = min(bn, part * pcut), cend = part + 1 == GP_EPI_PARTS ? bn : min(bn, (part + 1) * pcut);
            const bool c_tma = rec_ctma(rec) && g.beta == 0.f;
            const int rows = rec_rows(rec);
            if (c_tma && row_base < rows) {
                const int cols = min(rec_cols(rec), cend);
                const CUtensorMap* mC = g.maps + 3 * rec.x + 2;
                const int rows_tma = rows & ~(c_rows_unit(OUT_BF16) - 1);
                const bool tail_lane = row_base + lane >= rows_tma && row_base + lane < rows;
                TailC tc_{nullptr, 0, 0};
                if (row_base + 32 > rows_tma) {   // this warp holds rows past the map: read the problem once
                    const GroupedProblem& P = g.probs[rec.x];
                    tc_ = TailC{P.C, P.ldc, P.N};
                }
#pragma unroll 1
                for (int c0 = cbeg; c0 < cols; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(t_base + uint32_t(c0), r);
                    tmem_ld_wait();
                    if (row_base < rows_tma) {
                        float* sb = stage_w + (cbuf % GP_CBUF) * 32 * 32;
                        if (lane == 0) {    // the store that last used this buffer has read it
                            if (GP_CBUF == 2) bulk_wait_group_read<1>();
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
                            tma_store_2d(mC, sb, tm * 2 * BM + row_base, tn * bn + c0);
                            bulk_commit_group();
                        }
                        ++cbuf;
                    }
                    if (tail_lane)
                        store_tail_row<OUT_BF16>(tc_, int64_t(tm) * 2 * BM + row_base + lane, int64_t(tn) * bn + c0, r,
                                                 g.alpha);
                }
            } else if (!c_tma) {
                const GroupedProblem P = g.probs[rec.x];
                const int64_t row = int64_t(tm) * 2 * BM + row_base + lane;
#pragma unroll 1
                for (int c0 = cbeg; c0 < cend; c0 += 32) {
                    uint32_t r[32];
                    tmem_ld32(t_base + uint32_t(c0), r);
                    tmem_ld_wait();
                    const int64_t col0 = int64_t(tn) * bn + c0;
                    if (row < P.M) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int64_t col = col0 + j;
                            if (col < P.N) {
                                float v = g.alpha * __uint_as_float(r[j]);
                                if (OUT_BF16) {
                                    __nv_bfloat16* Cp = static_cast<__nv_bfloat16*>(P.C) + row + col * P.ldc;
                                    if (g.beta != 0.f) v = fmaf(g.beta, __bfloat162float(*Cp), v);
                                    *Cp = __float2bfloat16_rn(v);
                                } else {
                                    float* Cp = static_cast<float*>(P.C) + row + col * P.ldc;
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
            rp.cur = rp.next;
            rp.next = rp.next2;
        }
        if (lane == 0) bulk_wait_group<0>();   // every bulk store complete before the CTA leaves
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync_all();            // the leader's MMAs and the peer's remote arrivals are done before TMEM goes
    tc_fence_after();
    if (warp == 1) tmem_dealloc_pair(tmem, 512);
}

}  // namespace

// ---------------------------------------------------------------------------
// grouped plan (host)
// ---------------------------------------------------------------------------
// Everything one grouped launch reads from device memory, built on the host: the TMA
// descriptors (64-byte aligned), the problem records and the flattened tile table, laid out
// as one byte image that goes to the device in one piece (a plan's own allocation, or the
// caller's workspace).
struct GroupedImage {
    bool tf32 = false, out_bf16 = false;
    bool pairs = true;                   // 256-row tiles on CTA pairs, else 128-row tiles on one CTA
    int count = 0;                       // problems with work
    int64_t total_tiles = 0;
    std::vector<int> bn_per_problem;     // in the caller's order
    std::vector<uint8_t> bytes;          // maps | problem records | tile table
    size_t probs_off = 0, tiles_off = 0;
};

struct GroupedPlan {
    GroupedImage img;
    void* dev = nullptr;                 // device copy of img.bytes
};

// Per-problem tile width.  Tiles on CTA pairs with a K-major B take any multiple of 32 up to
// 256 (each CTA stages bn/2 rows of B; the MMA's N is bn): the columns are cut into
// ceil(n / 256) equal tiles, rounded up to 32, so that little of the tensor work is padding
// (1.33 instead of 1.44 times the flops on log-uniform sizes in [64, 2048]).  Otherwise (one-CTA
// kernel, or B in 64-element MN-major chunks): 256 when the problem fills it, else 128.
static int auto_tile_n(int64_t m, int64_t n, int64_t k, bool flex) {
    (void)m; (void)k;
    if (flex) {
        const int64_t t = (n + 255) / 256;
        return int(((n + t - 1) / t + 31) / 32 * 32);
    }
    return n > 192 ? 256 : 128;
}

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The grouped launch runs on CTA pairs; HSMM_GROUPED_KERNEL = single selects the one-CTA
// kernel (kept for comparison; both give the same results up to FP32 summation order).
static bool grouped_pairs_enabled() {
    const char* v = std::getenv("HSMM_GROUPED_KERNEL");
    return !(v && std::strcmp(v, "single") == 0);
}

static hsmm_status_t grouped_build_image(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                                         int tile_n, const int* tile_n_per_problem, int schedule, GroupedImage* img) {
    const bool tf32 = (ab == HSMM_R_32F);
    const int esize = tf32 ? 4 : 2;
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const int BK = 128 / esize, MN_CHUNK = 128 / esize;
    const CUtensorMapSwizzle mn_sw = tf32 ? CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B : CU_TENSOR_MAP_SWIZZLE_128B;
    img->tf32 = tf32;
    img->out_bf16 = (c == HSMM_R_16BF);
    img->pairs = grouped_pairs_enabled();
    const int TM = img->pairs ? 2 * BM : BM;   // rows of a tile
    img->bn_per_problem.assign(size_t(count), 0);
    // problem order
    std::vector<int64_t> order;
    for (int64_t i = 0; i < count; ++i)
        if (descs[i].m > 0 && descs[i].n > 0 && descs[i].k > 0) order.push_back(i);
    if (schedule == 1)
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return descs[a].k > descs[b].k; });
    std::vector<CUtensorMap> maps(order.size() * 3);
    std::vector<uint8_t> c_tma(order.size(), 0);
    const int esc = img->out_bf16 ? 2 : 4;
    const CUtensorMapDataType dtc = img->out_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    std::vector<GroupedProblem> probs(order.size());
    int64_t tiles = 0;
    for (size_t q = 0; q < order.size(); ++q) {
        const hsmm_gemm_desc_t& d = descs[order[q]];
        if (d.m > INT32_MAX || d.n > INT32_MAX || d.k > INT32_MAX) return HSMM_STATUS_NOT_SUPPORTED;
        if (!tma_operand_ok(d.A, d.lda, esize) || !tma_operand_ok(d.B, d.ldb, esize)) return HSMM_STATUS_NOT_SUPPORTED;
        const bool flex = img->pairs && d.transB != HSMM_OP_T;   // CTA pairs, K-major B
        int bn = tile_n ? tile_n : (tile_n_per_problem ? tile_n_per_problem[order[q]] : 0);
        if (bn == 0) bn = auto_tile_n(d.m, d.n, d.k, flex);
        if (flex ? (bn < 32 || bn > 256 || bn % 32 != 0) : (bn != 128 && bn != 256)) return HSMM_STATUS_INVALID_VALUE;
        img->bn_per_problem[size_t(order[q])] = bn;
        GroupedProblem& P = probs[q];
        P.M = int(d.m); P.N = int(d.n); P.K = int(d.k);
        P.a_mn = (d.transA == HSMM_OP_N);
        P.b_mn = (d.transB == HSMM_OP_T);
        P.bn = bn;
        P.tiles_m = int((d.m + TM - 1) / TM);
        P.tiles_n = int((d.n + bn - 1) / bn);
        P.tile_start = tiles;
        P.C = d.C;
        P.ldc = d.ldc;
        tiles += int64_t(P.tiles_m) * P.tiles_n;
        bool ok = P.a_mn ? encode_map(&maps[3 * q], dt, esize, d.A, uint64_t(d.m), uint64_t(d.k), uint64_t(d.lda),
                                      MN_CHUNK, BK, 0, 0, mn_sw)
                         : encode_map(&maps[3 * q], dt, esize, d.A, uint64_t(d.k), uint64_t(d.m), uint64_t(d.lda), BK,
                                      BM);
        ok = ok && (P.b_mn ? encode_map(&maps[3 * q + 1], dt, esize, d.B, uint64_t(d.n), uint64_t(d.k),
                                        uint64_t(d.ldb), MN_CHUNK, BK, 0, 0, mn_sw)
                           : encode_map(&maps[3 * q + 1], dt, esize, d.B, uint64_t(d.k), uint64_t(d.n),
                                        uint64_t(d.ldb), BK, uint32_t(img->pairs ? bn / 2 : bn)));
        if (!ok) return HSMM_STATUS_NOT_SUPPORTED;
        // C by TMA stores of 32 x 32 blocks when its base and columns are 16-byte aligned; the map
        // covers the rows up to the last whole 16-byte unit (a store clips to such units), the
        // epilogue stores the rows after them directly
        std::memset(&maps[3 * q + 2], 0, sizeof(CUtensorMap));
        const int64_t m_tma = d.m - d.m % (16 / esc);
        if (m_tma > 0 && tma_operand_ok(d.C, d.ldc, size_t(esc)) &&
            encode_map(&maps[3 * q + 2], dtc, esc, d.C, uint64_t(m_tma), uint64_t(d.n), uint64_t(d.ldc), 32, 32, 0, 0,
                       CU_TENSOR_MAP_SWIZZLE_NONE))
            c_tma[q] = 1;
    }
    img->count = int(order.size());
    img->total_tiles = tiles;
    // flattened tile table (problem-major order), one 16-byte record per tile: problem,
    // (tile row, tile column), k-blocks, and width / majorness / C path / valid rows and columns
    std::vector<uint4> tile_tab(static_cast<size_t>(tiles));
    for (size_t q = 0; q < probs.size(); ++q) {
        const GroupedProblem& P = probs[q];
        if (P.tiles_m > 65535 || P.tiles_n > 65535) return HSMM_STATUS_NOT_SUPPORTED;
        const uint32_t nkb = uint32_t((int64_t(P.K) + BK - 1) / BK);
        for (int tn = 0; tn < P.tiles_n; ++tn)
            for (int tm = 0; tm < P.tiles_m; ++tm) {
                const uint32_t rows = uint32_t(std::min<int64_t>(TM, int64_t(P.M) - int64_t(tm) * TM));
                const uint32_t cols = uint32_t(std::min<int64_t>(P.bn, int64_t(P.N) - int64_t(tn) * P.bn));
                const uint32_t w = (uint32_t(P.bn / 32 - 1) << 26) | (uint32_t(P.a_mn) << 2) | (uint32_t(P.b_mn) << 3) |
                                   (uint32_t(c_tma[q]) << 4) | (rows << 8) | (cols << 17);
                tile_tab[size_t(P.tile_start + int64_t(tn) * P.tiles_m + tm)] =
                    make_uint4(uint32_t(q), uint32_t(tm) | (uint32_t(tn) << 16), nkb, w);
            }
    }
    const size_t maps_bytes = maps.size() * sizeof(CUtensorMap);
    img->probs_off = round_up(maps_bytes, 64);
    img->tiles_off = round_up(img->probs_off + probs.size() * sizeof(GroupedProblem), 64);
    img->bytes.assign(round_up(img->tiles_off + tile_tab.size() * sizeof(uint4), 64), 0);
    if (maps_bytes) std::memcpy(img->bytes.data(), maps.data(), maps_bytes);
    if (!probs.empty())
        std::memcpy(img->bytes.data() + img->probs_off, probs.data(), probs.size() * sizeof(GroupedProblem));
    if (!tile_tab.empty())
        std::memcpy(img->bytes.data() + img->tiles_off, tile_tab.data(), tile_tab.size() * sizeof(uint4));
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t grouped_plan_create_ex(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                                     int tile_n, const int* tile_n_per_problem, int schedule, GroupedPlan** out) {
    auto* plan = new GroupedPlan();
    hsmm_status_t s = grouped_build_image(ab, c, count, descs, tile_n, tile_n_per_problem, schedule, &plan->img);
    if (s != HSMM_STATUS_SUCCESS) { delete plan; return s; }
    if (plan->img.total_tiles > 0) {
        cudaError_t e = cudaMalloc(&plan->dev, plan->img.bytes.size());
        if (e != cudaSuccess) { delete plan; return record_cuda(e); }
        e = cudaMemcpy(plan->dev, plan->img.bytes.data(), plan->img.bytes.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(plan->dev); delete plan; return record_cuda(e); }
    }
    *out = plan;
    return HSMM_STATUS_SUCCESS;
}

hsmm_status_t grouped_plan_create(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                                  int tile_n, GroupedPlan** out) {
    return grouped_plan_create_ex(ab, c, count, descs, tile_n, nullptr, 1, out);
}

template <bool TF32, bool OUT_BF16>
static hsmm_status_t launch_grouped(const GroupedArgs& a, cudaStream_t st) {
    using C_ = Cfg<256, TF32>;
    constexpr int smem = C_::STAGES * C_::STAGE_BYTES + GROUPED_STAGE_C + 1024 + 256;
    static_assert(smem <= 227 * 1024, "grouped kernel shared memory");
    auto kern = gemm_grouped_kernel<TF32, OUT_BF16>;
    static std::atomic<uint64_t> attrs{0};
    const hsmm_status_t as = attrs_once_per_device(
        attrs, [kern] { return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); });
    if (as != HSMM_STATUS_SUCCESS) return as;
    const int64_t grid = std::min<int64_t>(a.total_tiles, num_sms());
    kern<<<unsigned(grid), kNumThreads, smem, st>>>(a);
    count_launches(1);
    return check_launch();
}

template <bool TF32, bool OUT_BF16>
static hsmm_status_t launch_grouped_pair(const GroupedArgs& a, cudaStream_t st) {
    auto kern = gemm_grouped_pair_kernel<TF32, OUT_BF16>;
    static std::atomic<uint64_t> attrs{0};
    const hsmm_status_t as = attrs_once_per_device(
        attrs, [kern] { return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, GP_SMEM); });
    if (as != HSMM_STATUS_SUCCESS) return as;
    const int64_t pairs = std::max<int64_t>(1, std::min<int64_t>(a.total_tiles, num_sms() / 2));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(unsigned(2 * pairs), 1, 1);
    lc.blockDim = dim3(GP_THREADS, 1, 1);
    lc.dynamicSmemBytes = GP_SMEM;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&lc, kern, a);
    count_launches(1);
    if (e != cudaSuccess) return record_cuda(e);
    return check_launch();
}

// The launch of an image already on the device at `dev`.
static hsmm_status_t grouped_launch_image(const GroupedImage& img, const void* dev, float alpha, float beta,
                                          cudaStream_t st) {
    if (img.total_tiles == 0) return HSMM_STATUS_SUCCESS;
    const uint8_t* base = static_cast<const uint8_t*>(dev);
    GroupedArgs a{};
    a.maps = reinterpret_cast<const CUtensorMap*>(base);
    a.probs = reinterpret_cast<const GroupedProblem*>(base + img.probs_off);
    a.tiles = reinterpret_cast<const uint4*>(base + img.tiles_off);
    a.count = img.count;
    a.total_tiles = img.total_tiles;
    a.alpha = alpha;
    a.beta = beta;
    a.timeout_ns = wait_timeout_ns();
    if (img.tf32) {
        if (img.out_bf16) return HSMM_STATUS_NOT_SUPPORTED;
        return img.pairs ? launch_grouped_pair<true, false>(a, st) : launch_grouped<true, false>(a, st);
    }
    if (img.pairs)
        return img.out_bf16 ? launch_grouped_pair<false, true>(a, st) : launch_grouped_pair<false, false>(a, st);
    return img.out_bf16 ? launch_grouped<false, true>(a, st) : launch_grouped<false, false>(a, st);
}

hsmm_status_t grouped_plan_launch(GroupedPlan* plan, float alpha, float beta, cudaStream_t st) {
    return grouped_launch_image(plan->img, plan->dev, alpha, beta, st);
}

hsmm_status_t grouped_plan_info(GroupedPlan* plan, int64_t* tiles, int* tile_n) {
    if (tiles) *tiles = plan->img.total_tiles;
    if (tile_n)
        for (size_t i = 0; i < plan->img.bn_per_problem.size(); ++i) tile_n[i] = plan->img.bn_per_problem[i];
    return HSMM_STATUS_SUCCESS;
}

void grouped_plan_destroy(GroupedPlan* plan) {
    if (!plan) return;
    if (plan->dev) cudaFree(plan->dev);
    delete plan;
}

// ---------------------------------------------------------------------------
// the grouped launch without a plan: the image goes into the caller's workspace
// ---------------------------------------------------------------------------
// The image is written by kernels whose parameter block carries it, up to kFillChunk bytes
// per launch, on the caller's stream: the data travel with the launches, so nothing is
// allocated, no host buffer has to outlive the call, and a stream capture records the
// data into the graph's kernel nodes.
constexpr uint32_t kFillChunk = 32704;   // a multiple of 16; parameter block <= 32764 bytes

struct FillArgs {
    uint8_t* dst;
    uint32_t nbytes;                     // a multiple of 16
    uint32_t pad;
    alignas(16) uint8_t data[kFillChunk];
};

__global__ void __launch_bounds__(256) fill_from_params(const __grid_constant__ FillArgs a) {
    const uint32_t n16 = a.nbytes / 16;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += gridDim.x * blockDim.x)
        reinterpret_cast<uint4*>(a.dst)[i] = reinterpret_cast<const uint4*>(a.data)[i];
}

size_t grouped_workspace_bytes(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                               int tile_n, hsmm_status_t* st) {
    GroupedImage img;
    *st = grouped_build_image(ab, c, count, descs, tile_n, nullptr, 1, &img);
    return *st == HSMM_STATUS_SUCCESS ? img.bytes.size() : 0;
}

hsmm_status_t grouped_run_in_workspace(hsmm_dtype_t ab, hsmm_dtype_t c, int64_t count, const hsmm_gemm_desc_t* descs,
                                       int tile_n, void* ws, size_t ws_bytes, float alpha, float beta,
                                       cudaStream_t st) {
    GroupedImage img;
    hsmm_status_t s = grouped_build_image(ab, c, count, descs, tile_n, nullptr, 1, &img);
    if (s != HSMM_STATUS_SUCCESS) return s;
    if (img.total_tiles == 0) return HSMM_STATUS_SUCCESS;
    if (!ws || ws_bytes < img.bytes.size())
        return fail(HSMM_STATUS_WORKSPACE_TOO_SMALL, "gemm_grouped: workspace of %zu bytes, %zu needed", ws_bytes,
                    img.bytes.size());
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "gemm_grouped: workspace not 256-byte aligned");
    FillArgs* fa = new FillArgs;
    for (size_t off = 0; off < img.bytes.size(); off += kFillChunk) {
        const size_t n = std::min<size_t>(kFillChunk, img.bytes.size() - off);   // image size is a multiple of 64
        fa->dst = static_cast<uint8_t*>(ws) + off;
        fa->nbytes = uint32_t(n);
        fa->pad = 0;
        std::memcpy(fa->data, img.bytes.data() + off, n);
        fill_from_params<<<8, 256, 0, st>>>(*fa);
        count_launches(1);
        const hsmm_status_t ls = check_launch();
        if (ls != HSMM_STATUS_SUCCESS) { delete fa; return ls; }
    }
    delete fa;
    return grouped_launch_image(img, ws, alpha, beta, st);
}

}  // namespace hsmm
