// tc_tile.cuh -- the operand tile of the tcgen05 kernels: a 128-row (M) by BN (N)
// output tile fed by k-slabs of one 128-byte swizzle row of K per stage.
//
// Shared by the persistent kernels (gemm_tc.cu), the slice products of the FP64-accurate
// form (gemm_ozaki_tc.cu) and the cluster ring order (gemm_ring_tc.cu): stage geometry,
// the CTA-pair tile, the barrier block and tile order of the persistent kernels, UMMA
// shared-memory descriptors for K-major and MN-major operands, and the TMA loads of one
// operand k-slab.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace hsmm {
namespace tc {

constexpr int BM = 128;

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
    static constexpr int STAGES_FIT = (227 * 1024 - 2048) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
    static constexpr int TMEM_COLS = (2 * BN <= 256) ? 256 : 512;   // two accumulators, power of two
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};

// CTA-pair tiles (cta_group::2): 256 x 256 per pair, each CTA stages A and B halves of 128 rows
constexpr int PAIR_BN = 256;                       // N of the pair tile
constexpr int PAIR_STAGE_BYTES = 2 * BM * 128;     // A half (128 rows) + B half (128 rows)
constexpr int PAIR_STAGES = 7;
constexpr int PAIR_SMEM = PAIR_STAGES * PAIR_STAGE_BYTES + 1024 + 256;

struct Bars {
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t mma_done;
    uint32_t tmem_base;
    int abort;
};

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

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

template <typename C_>
__device__ __forceinline__ uint64_t operand_desc(uint32_t base, int ks, bool mn_major) {
    if (mn_major) {
        // MN-major: chunks of one 128-byte row of MN (64 BF16 / 32 TF32 elements) by BK rows of
        // K each; LBO = chunk bytes.  A k-step is UMMA_K rows.  BF16: 128-byte swizzle, the
        // tensor core reads K in groups of 8 rows (SBO = 1024 bytes).  TF32: 128-byte swizzle
        // of 32-byte units (the TMA map uses the matching 128B_ATOM_32B pattern) and K in
        // groups of 4 rows (SBO = 512 bytes).  Both found on the GPU with an operand whose
        // entries encode their own row and column (C = A I and C = I B, every element checked).
        return smem_desc_sw128(base + uint32_t(ks) * uint32_t(C_::UMMA_K) * 128u, uint32_t(C_::BK) * 128u,
                               C_::TF32 ? 512u : 1024u, C_::TF32 ? SW128_ATOM32 : SW128);
    }
    // K-major: rows of 128 bytes; the K step moves 32 bytes inside the swizzled row.
    return smem_desc_sw128(base + uint32_t(ks) * 32u, 16u, 1024u);
}

// Start-address increment (16-byte units of the descriptor's 14-bit address field) of
// one MMA k-step.  Shared-memory addresses stay below 2^18, so stepping a descriptor by a
// k-step or a whole stage is a plain 64-bit add with no carry out of the field; the MMA
// thread precomputes its stage-0 descriptors once and only adds in its loop (a single
// issuing thread pays full dependent latency for every instruction it executes).
template <typename C_>
__device__ __forceinline__ uint64_t ks_step(bool mn_major) {
    return mn_major ? uint64_t(C_::UMMA_K * 128 / 16) : uint64_t(32 / 16);
}

// Issue the TMA loads of one operand k-slab (rows r0.. of the MN dimension, k-block kb).  An
// MN-major operand comes as ROWS / MN_CHUNK boxes of one chunk each, or (mn3) as one 3D box
// {MN_CHUNK, BK, ROWS / MN_CHUNK} of a map that views the operand as {chunk, K, chunks}.
template <typename C_, int ROWS>
__device__ __forceinline__ void load_operand(uint8_t* dst, const void* map, uint64_t* bar, bool mn_major, int r0,
                                             int kb, int batch, bool batched, bool mn3 = false) {
    if (!mn_major) {
        if (batched)
            tma_load_3d(dst, map, bar, kb * C_::BK, r0, batch);
        else
            tma_load_2d(dst, map, bar, kb * C_::BK, r0);
    } else if (mn3) {
        tma_load_3d(dst, map, bar, 0, kb * C_::BK, r0 / C_::MN_CHUNK);
    } else {
#pragma unroll
        for (int c = 0; c < ROWS / C_::MN_CHUNK; ++c)
            tma_load_2d(dst + c * C_::BK * 128, map, bar, r0 + c * C_::MN_CHUNK, kb * C_::BK);
    }
}

}  // namespace tc
}  // namespace hsmm
