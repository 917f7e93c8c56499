// gemm_ozaki_tc.cu -- the slice products of the FP64-accurate form on the tcgen05 tensor cores.
//
// For split operands (BF16 slices of integer digits, see ozaki.cu) this computes the
// exact anti-diagonal sums S_d = sum_{t+u=d} Q^A_t (Q^B_u)^T, d = 2..s+1, as INT32 planes
// in the caller's workspace.  The main loop is that of the plain products (gemm_tc.cu):
// TMA -> shared memory -> tcgen05.mma -> TMEM, here with a k-schedule over the slice
// pairs and an epilogue that drains exact FP32 chunks into INT32 sums held in registers.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc_tile.cuh"
#include "internal.h"

namespace hsmm {

static __device__ uint32_t g_status_ozaki_tc;

uint32_t status_take_ozaki_tc() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_ozaki_tc, sizeof(v));
    cudaMemcpyToSymbol(g_status_ozaki_tc, &z, sizeof(z));
    return v;
}

namespace {

using namespace tc;

// ---------------------------------------------------------------------------
// Slice products of the FP64-accurate form
// ---------------------------------------------------------------------------
// Per 128 x 256 output tile the k-schedule runs over the anti-diagonals
// d = s+1 down to 2 of the slice pairs (t, u), t + u = d, and over k inside each
// pair.  Slice entries are integers with |q| <= 2^bits - 1, so an FP32 sum of
// kc products, kc (2^bits - 1)^2 <= 2^24, is exact; the MMA warp hands the
// accumulator over every kc_blocks k-blocks (and at the end of each d), the
// epilogue converts it to INT32 and adds it to S_d held in registers (exact:
// |S_d| <= s k (2^bits-1)^2 < 2^31 is checked on the host), and at the end of
// the anti-diagonal stores S_d.  No FP64 arithmetic runs in this kernel: the
// recombination (ozaki_recombine in ozaki.cu) reads the s INT32 planes once.
// Twelve warps: warpgroup 0 holds the TMA producer (warp 0) and the MMA issuer
// (warp 1) and lowers its register budget (setmaxnreg.dec to 152); warpgroups 1
// and 2 are eight epilogue warps that raise theirs (setmaxnreg.inc to 176).  The
// launch holds 384 x 168 = 64512 registers = 128 x 152 + 256 x 176; neither side
// spills (a tighter producer/MMA budget spilled inside the MMA issue loop and
// halved the tensor-pipe rate).  Epilogue warp w owns TMEM lanes 32*(w%4).. and
// the column half (w-4)/4 of the 256-column accumulator: 128 INT32 partial sums
// per thread, kept in registers.
struct OzakiArgs {
    int M, N, K;
    int slices, kc_blocks;
    int32_t* sd;        // S_d, d = 2..s+1, as [d-2][N][M] INT32 (column-major per anti-diagonal)
    int64_t sd_plane;   // elements between consecutive anti-diagonal planes
    uint64_t timeout_ns;
};

constexpr int OZ_BN = 256;
constexpr int OZ_HALF = OZ_BN / 2;
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 128 + 32 * OZ_EPI_WARPS;     // 384
constexpr uint32_t OZ_REGS_LAUNCH = 168, OZ_REGS_LOW = 152, OZ_REGS_HIGH = 176;
static_assert(OZ_THREADS * OZ_REGS_LAUNCH == 128 * OZ_REGS_LOW + 256 * OZ_REGS_HIGH, "register split must balance");

__host__ __device__ __forceinline__ int oz_tlo(int d, int s) { return d - s > 1 ? d - s : 1; }
__host__ __device__ __forceinline__ int oz_thi(int d, int s) { return d - 1 < s ? d - 1 : s; }

// Work of the CTA pairs of the slice-product kernel.  The tiles of the full waves are whole
// items (all anti-diagonals d = s+1 .. 2, tile t = pair + i npairs).  The tiles of the last,
// partial wave are cut into G = s/2 + 1 groups of anti-diagonals that hold (nearly) the same
// number of slice pairs: group 0 is d = s+1 (s pairs), group j >= 1 is d = s+1-j and d = j+1
// ((s-j) + j pairs; for even s the last group is d = s/2+1 alone).  The groups are dealt to
// the pairs in turn, so the last wave ends within one group of the mean instead of a tile.
struct OzItem {
    int t;        // tile
    int j;        // -1: whole tile; else the anti-diagonal group
};
__host__ __device__ __forceinline__ int oz_groups(int s) { return s / 2 + 1; }
__host__ __device__ __forceinline__ int oz_items(int ntiles, int npairs, int pair, int s) {
    const int full = ntiles / npairs;
    const int units = (ntiles - full * npairs) * oz_groups(s);
    return full + (units > pair ? (units - pair + npairs - 1) / npairs : 0);
}
__host__ __device__ __forceinline__ OzItem oz_item(int i, int ntiles, int npairs, int pair, int s) {
    const int full = ntiles / npairs;
    if (i < full) return OzItem{pair + i * npairs, -1};
    const int u = pair + (i - full) * npairs;
    return OzItem{full * npairs + u / oz_groups(s), u % oz_groups(s)};
}
// anti-diagonals of an item: count, and the di-th (descending within the item)
__host__ __device__ __forceinline__ int oz_item_nd(const OzItem& it, int s) {
    if (it.j < 0) return s;
    return (it.j >= 1 && it.j + 1 < s + 1 - it.j) ? 2 : 1;
}
__host__ __device__ __forceinline__ int oz_item_d(const OzItem& it, int di, int s) {
    if (it.j < 0) return s + 1 - di;
    return di == 0 ? s + 1 - it.j : it.j + 1;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    gemm_ozaki_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzakiArgs g) {
    using C_ = Cfg<OZ_BN, false>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    Bars* bars = reinterpret_cast<Bars*>(smem + C_::STAGES * C_::STAGE_BYTES);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_ozaki_tc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C_::STAGES; ++s) {
            mbar_init(&bars->full[s], 1);
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], OZ_EPI_WARPS);
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
    const int tiles_n = (g.N + OZ_BN - 1) / OZ_BN;
    const int ntiles = tiles_m * tiles_n;
    const int nkb = (g.K + C_::BK - 1) / C_::BK;
    const int s = g.slices;
    const int kcb = g.kc_blocks;

    if (warp < 4) regs_dec<OZ_REGS_LOW>();
    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[8];
            for (int i = 0; i < 8; ++i) last_parity[i] = -1;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
                int tm, tn;
                tile_coords(t, tiles_m, tiles_n, tm, tn);
                for (int d = s + 1; d >= 2 && ok; --d)
                    for (int ta = oz_tlo(d, s); ta <= oz_thi(d, s) && ok; ++ta) {
                        const int ub = d - ta;
                        for (int kb = 0; kb < nkb; ++kb) {
                            if (!mbar_wait(&bars->empty[stage], phase ^ 1u, g.timeout_ns, status, abort)) { ok = false; break; }
                            uint8_t* a_dst = smem + stage * C_::STAGE_BYTES;
                            uint8_t* b_dst = a_dst + C_::A_BYTES;
                            mbar_arrive_expect_tx(&bars->full[stage], C_::STAGE_BYTES);
                            tma_load_3d(a_dst, &tmA, &bars->full[stage], kb * C_::BK, tm * BM, ta - 1);
                            tma_load_3d(b_dst, &tmB, &bars->full[stage], kb * C_::BK, tn * OZ_BN, ub - 1);
                            last_parity[stage] = int(phase);
                            if (++stage == C_::STAGES) { stage = 0; phase ^= 1u; }
                        }
                    }
            }
            for (int i = 0; i < C_::STAGES; ++i)
                if (last_parity[i] >= 0) mbar_wait(&bars->full[i], uint32_t(last_parity[i]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc(1u, false, false, BM, OZ_BN);
            const uint64_t a0 = operand_desc<C_>(smem_u32(smem), 0, false);
            const uint64_t b0 = operand_desc<C_>(smem_u32(smem) + C_::A_BYTES, 0, false);
            const uint64_t kstep = ks_step<C_>(false);
            const uint64_t sstep = uint64_t(C_::STAGE_BYTES / 16);
            uint64_t acur = a0, bcur = b0;
            int stage = 0;
            uint32_t phase = 0;
            int abuf = 0;
            uint32_t aphase = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
                for (int d = s + 1; d >= 2 && ok; --d) {
                    int left_d = (oz_thi(d, s) - oz_tlo(d, s) + 1) * nkb;   // k-blocks left in this anti-diagonal
                    int left_c = 0;                                         // k-blocks left in this FP32 chunk
                    uint32_t d_tmem = tmem;
                    uint32_t acc_flag = 0;
                    while (left_d > 0) {
                        if (left_c == 0) {
                            if (!mbar_wait(&bars->acc_empty[abuf], aphase ^ 1u, g.timeout_ns, status, abort)) { ok = false; break; }
                            tc_fence_after();
                            left_c = kcb;
                            d_tmem = tmem + uint32_t(abuf * OZ_BN);
                            acc_flag = 0;
                        }
                        if (!mbar_wait(&bars->full[stage], phase, g.timeout_ns, status, abort)) { ok = false; break; }
                        tc_fence_after();
                        umma_f16(d_tmem, acur, bcur, idesc, acc_flag);
#pragma unroll
                        for (int ks = 1; ks < C_::KSTEPS; ++ks)
                            umma_f16(d_tmem, acur + ks * kstep, bcur + ks * kstep, idesc, 1u);
                        acc_flag = 1u;
                        umma_commit(&bars->empty[stage]);
                        if (++stage == C_::STAGES) { stage = 0; phase ^= 1u; acur = a0; bcur = b0; }
                        else { acur += sstep; bcur += sstep; }
                        --left_d;
                        if (--left_c == 0 || left_d == 0) {
                            umma_commit(&bars->acc_full[abuf]);
                            abuf ^= 1;
                            if (abuf == 0) aphase ^= 1u;
                            left_c = 0;
                        }
                    }
                }
            }
            umma_commit(&bars->mma_done);
            mbar_wait(&bars->mma_done, 0, g.timeout_ns, status, abort);
        }
    } else if (warp >= 4) {
        regs_inc<OZ_REGS_HIGH>();
        const int q = warp & 3;
        const int half = (warp - 4) >> 2;
        int abuf = 0;
        uint32_t aphase = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int tm, tn;
            tile_coords(t, tiles_m, tiles_n, tm, tn);
            const int64_t row = int64_t(tm) * BM + q * 32 + lane;
            const int64_t col0 = int64_t(tn) * OZ_BN + half * OZ_HALF;
            const bool row_ok = row < g.M;
            for (int d = s + 1; d >= 2 && ok; --d) {
                int S[OZ_HALF];
#pragma unroll
                for (int j = 0; j < OZ_HALF; ++j) S[j] = 0;
                const int total = (oz_thi(d, s) - oz_tlo(d, s) + 1) * nkb;
                const int nch = (total + kcb - 1) / kcb;
                for (int c = 0; c < nch; ++c) {
                    int okw = 0;
                    if (lane == 0) okw = mbar_wait(&bars->acc_full[abuf], aphase, g.timeout_ns, status, abort) ? 1 : 0;
                    okw = __shfl_sync(0xffffffffu, okw, 0);
                    if (!okw) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t t_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(abuf * OZ_BN + half * OZ_HALF);
#pragma unroll
                    for (int cc = 0; cc < OZ_HALF / 16; ++cc) {
                        uint32_t r[16];
                        tmem_ld16(t_base + uint32_t(cc * 16), r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) S[cc * 16 + j] += __float2int_rn(__uint_as_float(r[j]));
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bars->acc_empty[abuf]);
                    abuf ^= 1;
                    if (abuf == 0) aphase ^= 1u;
                }
                if (!ok) break;
                // store S_d (INT32) for this row segment: lanes are consecutive rows, so
                // each column is one 128-byte coalesced store per warp
                if (!row_ok) continue;
                const int64_t rem = int64_t(g.N) - col0;
                const int jmax = rem < OZ_HALF ? int(rem) : OZ_HALF;
                int32_t* Sp = g.sd + int64_t(d - 2) * g.sd_plane + row + col0 * int64_t(g.M);
#pragma unroll
                for (int j = 0; j < OZ_HALF; ++j)
                    if (j < jmax) Sp[int64_t(j) * g.M] = S[j];
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, C_::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Slice products on a CTA pair (cta_group::2): one 256 x 256 tile per pair
// ---------------------------------------------------------------------------
// The same k-schedule, chunking and epilogue as gemm_ozaki_kernel, with the MMA
// spread over two SMs: the even CTA holds A rows 0-127 and B rows 0-127 of the
// tile, the odd CTA rows 128-255 of each; one tcgen05.mma.cta_group::2 (M = 256,
// N = 256) issued by the even CTA reads both CTAs' shared memory and writes the
// 128 x 256 accumulator of each CTA into that CTA's TMEM.  Each CTA stages only
// 32 KiB per k-block (7 stages instead of 4), half the L2 traffic per tile row.
// Both CTAs' TMA copies complete on the even CTA's `full` barrier; the MMA
// commits are multicast to both CTAs (stage release, accumulator ready); both
// CTAs' epilogue warps release an accumulator on the even CTA's `acc_empty`.

__global__ void __launch_bounds__(OZ_THREADS, 1)
    gemm_ozaki_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                           OzakiArgs g) {
    using C_ = Cfg<OZ_BN, false>;                  // BK, KSTEPS, descriptors (K-major, 128-byte rows)
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    Bars* bars = reinterpret_cast<Bars*>(smem + PAIR_STAGES * PAIR_STAGE_BYTES);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_ozaki_tc;
    const uint32_t rank = cluster_ctarank() & 1u;  // role in the pair
    const bool leader = (rank == 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < PAIR_STAGES; ++s) {
            mbar_init(&bars->full[s], 1);
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], 2 * OZ_EPI_WARPS);
        }
        mbar_init(&bars->mma_done, 1);
        bars->abort = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 1) {
        tmem_alloc_pair(&bars->tmem_base, 512);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync_all();            // barriers of every CTA initialised before anyone signals them
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;

    const int tiles_m = (g.M + 2 * BM - 1) / (2 * BM);
    const int tiles_n = (g.N + PAIR_BN - 1) / PAIR_BN;
    const int ntiles = tiles_m * tiles_n;
    const int pair = int(blockIdx.x >> 1), npairs = int(gridDim.x >> 1);
    const int nkb = (g.K + C_::BK - 1) / C_::BK;
    const int s = g.slices;
    const int kcb = g.kc_blocks;
    const int nitems = oz_items(ntiles, npairs, pair, s);

    if (warp < 4) regs_dec<OZ_REGS_LOW>();
    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_parity[8];
            for (int i = 0; i < 8; ++i) last_parity[i] = -1;
            bool ok = true;
            for (int i = 0; i < nitems && ok && !*abort; ++i) {
                const OzItem it = oz_item(i, ntiles, npairs, pair, s);
                int tm, tn;
                tile_coords(it.t, tiles_m, tiles_n, tm, tn);
                const int arow = tm * 2 * BM + int(rank) * BM;
                const int brow = tn * PAIR_BN + int(rank) * BM;
                for (int di = 0; di < oz_item_nd(it, s) && ok; ++di) {
                    const int d = oz_item_d(it, di, s);
                    for (int ta = oz_tlo(d, s); ta <= oz_thi(d, s) && ok; ++ta) {
                        const int ub = d - ta;
                        for (int kb = 0; kb < nkb; ++kb) {
                            if (!mbar_wait(&bars->empty[stage], phase ^ 1u, g.timeout_ns, status, abort)) { ok = false; break; }
                            uint8_t* a_dst = smem + stage * PAIR_STAGE_BYTES;
                            uint8_t* b_dst = a_dst + BM * 128;
                            const uint32_t full_leader = mapa_shared(smem_u32(&bars->full[stage]), 0);
                            if (leader) mbar_arrive_expect_tx(&bars->full[stage], 2 * PAIR_STAGE_BYTES);
                            tma_load_3d_pair(a_dst, &tmA, full_leader, kb * C_::BK, arow, ta - 1);
                            tma_load_3d_pair(b_dst, &tmB, full_leader, kb * C_::BK, brow, ub - 1);
                            last_parity[stage] = int(phase);
                            if (++stage == PAIR_STAGES) { stage = 0; phase ^= 1u; }
                        }
                    }
                }
            }
            // every issued stage is released (empty) only after its copies landed and were consumed
            for (int i = 0; i < PAIR_STAGES; ++i)
                if (last_parity[i] >= 0) mbar_wait(&bars->empty[i], uint32_t(last_parity[i]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            const uint32_t idesc = make_idesc(1u, false, false, 2 * BM, PAIR_BN);
            const uint64_t a0 = operand_desc<C_>(smem_u32(smem), 0, false);
            const uint64_t b0 = operand_desc<C_>(smem_u32(smem) + BM * 128, 0, false);
            const uint64_t kstep = ks_step<C_>(false);
            const uint64_t sstep = uint64_t(PAIR_STAGE_BYTES / 16);
            int stage = 0;
            uint32_t phase = 0;
            int abuf = 0;
            uint32_t aphase = 0;
            bool ok = true;
            // One thread issues every MMA of the pair, so its own instruction time per k-block
            // (one wait, four MMAs, one commit) has to stay below the 512 tensor-pipe cycles
            // the k-block takes.  The loop is kept lean for that: one counter per FP32 chunk,
            // descriptors formed from the stage index (no state carried between k-blocks
            // but the stage and its phase), and four k-blocks per unrolled iteration.
            for (int i = 0; i < nitems && ok && !*abort; ++i) {
                const OzItem it = oz_item(i, ntiles, npairs, pair, s);
                for (int di = 0; di < oz_item_nd(it, s) && ok; ++di) {
                    const int d = oz_item_d(it, di, s);
                    int left_d = (oz_thi(d, s) - oz_tlo(d, s) + 1) * nkb;
                    while (left_d > 0 && ok) {
                        if (!mbar_wait(&bars->acc_empty[abuf], aphase ^ 1u, g.timeout_ns, status, abort)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t d_tmem = tmem + uint32_t(abuf * PAIR_BN);
                        const int nk = min(kcb, left_d);     // k-blocks of this exact FP32 chunk
#pragma unroll 4
                        for (int j = 0; j < nk; ++j) {
                            if (!mbar_wait(&bars->full[stage], phase, g.timeout_ns, status, abort)) { ok = false; break; }
                            tc_fence_after();
                            const uint64_t ad = a0 + uint64_t(stage) * sstep, bd = b0 + uint64_t(stage) * sstep;
                            umma_f16_pair(d_tmem, ad, bd, idesc, uint32_t(j));    // j == 0 starts the chunk
#pragma unroll
                            for (int ks = 1; ks < C_::KSTEPS; ++ks)
                                umma_f16_pair(d_tmem, ad + ks * kstep, bd + ks * kstep, idesc, 1u);
                            umma_commit_pair(&bars->empty[stage], 0x3);
                            stage = (stage + 1 == PAIR_STAGES) ? 0 : stage + 1;
                            phase ^= (stage == 0) ? 1u : 0u;
                        }
                        if (!ok) break;
                        umma_commit_pair(&bars->acc_full[abuf], 0x3);
                        abuf ^= 1;
                        if (abuf == 0) aphase ^= 1u;
                        left_d -= nk;
                    }
                }
            }
            umma_commit_pair(&bars->mma_done, 0x1);
            mbar_wait(&bars->mma_done, 0, g.timeout_ns, status, abort);
        }
    } else if (warp >= 4) {
        regs_inc<OZ_REGS_HIGH>();
        const int q = warp & 3;
        const int half = (warp - 4) >> 2;
        const uint32_t acc_empty_leader0 = mapa_shared(smem_u32(&bars->acc_empty[0]), 0);
        const uint32_t acc_empty_leader1 = mapa_shared(smem_u32(&bars->acc_empty[1]), 0);
        int abuf = 0;
        uint32_t aphase = 0;
        bool ok = true;
        for (int i = 0; i < nitems && ok; ++i) {
            const OzItem it = oz_item(i, ntiles, npairs, pair, s);
            int tm, tn;
            tile_coords(it.t, tiles_m, tiles_n, tm, tn);
            const int64_t row = int64_t(tm) * 2 * BM + int64_t(rank) * BM + q * 32 + lane;
            const int64_t col0 = int64_t(tn) * PAIR_BN + half * OZ_HALF;
            const bool row_ok = row < g.M;
            for (int di = 0; di < oz_item_nd(it, s) && ok; ++di) {
                const int d = oz_item_d(it, di, s);
                int S[OZ_HALF];
#pragma unroll
                for (int j = 0; j < OZ_HALF; ++j) S[j] = 0;
                const int total = (oz_thi(d, s) - oz_tlo(d, s) + 1) * nkb;
                const int nch = (total + kcb - 1) / kcb;
                for (int c = 0; c < nch; ++c) {
                    int okw = 0;
                    if (lane == 0) okw = mbar_wait(&bars->acc_full[abuf], aphase, g.timeout_ns, status, abort) ? 1 : 0;
                    okw = __shfl_sync(0xffffffffu, okw, 0);
                    if (!okw) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t t_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(abuf * PAIR_BN + half * OZ_HALF);
#pragma unroll
                    for (int cc = 0; cc < OZ_HALF / 16; ++cc) {
                        uint32_t r[16];
                        tmem_ld16(t_base + uint32_t(cc * 16), r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; ++j) S[cc * 16 + j] += __float2int_rn(__uint_as_float(r[j]));
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
                if (!ok) break;
                if (!row_ok) continue;
                const int64_t rem = int64_t(g.N) - col0;
                const int jmax = rem < OZ_HALF ? int(rem) : OZ_HALF;
                int32_t* Sp = g.sd + int64_t(d - 2) * g.sd_plane + row + col0 * int64_t(g.M);
#pragma unroll
                for (int j = 0; j < OZ_HALF; ++j)
                    if (j < jmax) Sp[int64_t(j) * g.M] = S[j];
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync_all();            // the peers' MMAs and remote arrivals are done before TMEM goes
    tc_fence_after();
    if (warp == 1) tmem_dealloc_pair(tmem, 512);
}
}  // namespace

// The slice products run on CTA pairs; HSMM_OZAKI_KERNEL = single selects the one-CTA kernel
// (kept for comparison; both produce the same exact S_d).
static bool ozaki_pairs_enabled() {
    const char* v = std::getenv("HSMM_OZAKI_KERNEL");
    return !(v && std::strcmp(v, "single") == 0);
}

static hsmm_status_t launch_ozaki_pairs(const CUtensorMap& mA, const CUtensorMap& mB, const OzakiArgs& g, int slices,
                                        cudaStream_t st) {
    static std::atomic<uint64_t> attrs{0};
    hsmm_status_t as = attrs_once_per_device(attrs, [] {
        return cudaFuncSetAttribute(gemm_ozaki_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR_SMEM);
    });
    if (as != HSMM_STATUS_SUCCESS) return as;
    const int max_pairs = num_sms() / 2;
    const int tiles = ((g.M + 2 * BM - 1) / (2 * BM)) * ((g.N + PAIR_BN - 1) / PAIR_BN);
    // whole tiles while they fill every pair; fewer tiles than pairs are cut into anti-diagonal groups
    const int pairs = std::max(1, tiles >= max_pairs ? max_pairs : std::min(max_pairs, tiles * oz_groups(slices)));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(unsigned(2 * pairs), 1, 1);
    lc.blockDim = dim3(OZ_THREADS, 1, 1);
    lc.dynamicSmemBytes = PAIR_SMEM;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&lc, gemm_ozaki_pair_kernel, mA, mB, g);
    count_launches(1);
    if (e != cudaSuccess) return record_cuda(e);
    return check_launch();
}

hsmm_status_t gemm_ozaki_slices(int64_t m, int64_t n, int64_t k, int64_t ldq, int slices, int bits, const void* qa,
                                int64_t qa_plane, const void* qb, int64_t qb_plane, int32_t* sd, int64_t sd_plane,
                                cudaStream_t st) {
    using C_ = Cfg<OZ_BN, false>;
    // exactness of the FP32 chunks and of the INT32 anti-diagonal sums
    const double qmax = double((1 << bits) - 1);
    const int64_t kc = int64_t(16777216.0 / (qmax * qmax));
    const int kc_blocks = int(kc / C_::BK);
    if (kc_blocks < 1) return fail(HSMM_STATUS_NOT_SUPPORTED, "ozaki: slice width leaves no exact FP32 chunk");
    if (double(slices) * double(k) * qmax * qmax >= 2147483648.0)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "ozaki: s k (2^bits-1)^2 >= 2^31, the INT32 sums would not be exact");
    OzakiArgs g{};
    g.M = int(m); g.N = int(n); g.K = int(k);
    g.slices = slices; g.kc_blocks = kc_blocks;
    g.sd = sd;
    g.sd_plane = sd_plane;
    g.timeout_ns = wait_timeout_ns();
    if (ozaki_pairs_enabled()) {
        // pair kernel: boxes of 128 rows (each CTA stages its half of the 256 x 256 tile's A and B)
        CUtensorMap mA2, mB2;
        if (!encode_map(&mA2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, qa, uint64_t(k), uint64_t(m), uint64_t(ldq), C_::BK,
                        BM, uint64_t(slices), uint64_t(qa_plane)) ||
            !encode_map(&mB2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, qb, uint64_t(k), uint64_t(n), uint64_t(ldq), C_::BK,
                        BM, uint64_t(slices), uint64_t(qb_plane)))
            return HSMM_STATUS_NOT_SUPPORTED;
        return launch_ozaki_pairs(mA2, mB2, g, slices, st);
    }
    CUtensorMap mA, mB;
    bool ok = encode_map(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, qa, uint64_t(k), uint64_t(m), uint64_t(ldq), C_::BK,
                         BM, uint64_t(slices), uint64_t(qa_plane));
    ok = ok && encode_map(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, qb, uint64_t(k), uint64_t(n), uint64_t(ldq), C_::BK,
                          OZ_BN, uint64_t(slices), uint64_t(qb_plane));
    if (!ok) return HSMM_STATUS_NOT_SUPPORTED;
    static std::atomic<uint64_t> attrs{0};
    hsmm_status_t as = attrs_once_per_device(attrs, [] {
        return cudaFuncSetAttribute(gemm_ozaki_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, C_::SMEM_BYTES);
    });
    if (as != HSMM_STATUS_SUCCESS) return as;
    const int tiles = ((g.M + BM - 1) / BM) * ((g.N + OZ_BN - 1) / OZ_BN);
    const int grid = std::min(tiles, num_sms());
    gemm_ozaki_kernel<<<grid, OZ_THREADS, C_::SMEM_BYTES, st>>>(mA, mB, g);
    count_launches(1);
    return check_launch();
}

}  // namespace hsmm
