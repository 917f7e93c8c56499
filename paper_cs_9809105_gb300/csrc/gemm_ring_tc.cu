// gemm_ring_tc.cu -- the hyper-systolic ring order (Algorithm 2, Section 5.2.2) on one
// thread-block cluster, with the local block product (x) on the tensor cores.
//
// Mapping.  The p processors of the ring are the p CTAs of a cluster.  A cluster
// computes a 128 x (p * 128) panel of C; CTA i owns block column i of the panel (the
// block-column distribution of Section 6.1).  The contraction index runs in rounds of
// p k-blocks of 64 elements; in a round, k-block j of the round starts on CTA j (A is
// distributed by block columns as well).  With K auxiliary accumulators and
// K~ = p / K:
//   main phase  K~ steps per round.  At step jb, CTA i holds the A block that started
//               on CTA (i + jb K) mod p and meets K blocks of B in the accumulators
//                   C^l += A_blk (x) B[k-block, block column (i - l) mod p],  l = 0..K-1;
//               the pre-shifted B of the paper is an address here (each CTA loads the
//               B blocks it needs from global memory by TMA).  Between steps
//               A <- cshift-row^K(A): CTA i forwards its block to CTA (i - K) mod p with
//               one 16 KiB DSMEM bulk copy, counted on the receiver's mbarrier;
//   back-shift  C^(l-1) += cshift-row^1(C^l) for l = K-1 .. 1: CTA i sends its C^l to
//               CTA i-1 (DSMEM stores); at the end C^0 of CTA i is block column i.
// Every (A block, output column) pair meets exactly once: the block that started on CTA
// x visits the CTAs x - jb K and feeds the columns x - jb K - l, and jb K + l runs over
// 0..p-1.  The K accumulators (128 x 128 FP32 each) live in TMEM, K * 128 <= 512 columns,
// so K <= 4: the TMEM capacity takes the place of the paper's memory for the K copies of C.
//
// Eight warps: 0 TMA loads of B; 1 MMA issue; 2 arms the A slots (TMA load at the start
// of a round, else a credit to the CTA that forwards into the slot); 3 forwards A blocks;
// 4-7 back-shift and epilogue.  A slot is free again after two arrivals: the commit of the
// MMAs that read it, and the completion of its forward copy (the receiver's MMA thread
// arrives remotely once the copy has landed; with no forward the forwarding warp arrives
// itself).  Every wait is bounded; the cluster barriers run the same number of times in
// every CTA whatever happens, so an abort in one CTA cannot strand the others.
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "tc_tile.cuh"

namespace hsmm {

static __device__ uint32_t g_status_ring_tc;

uint32_t status_take_ring_tc() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_ring_tc, sizeof(v));
    cudaMemcpyToSymbol(g_status_ring_tc, &z, sizeof(z));
    return v;
}

namespace {

using namespace tc;

using RC = Cfg<128, false>;                  // BF16: BK = 64, UMMA_K = 16, 4 k-steps per block
constexpr int RING_BN = 128;                 // block width (columns of one accumulator)
constexpr int NSLOT = 12;                    // 16 KiB slots, split between A slots and B stages
constexpr int SLOT = BM * 128;               // 16 KiB: 128 rows x 64 BF16 (A block or B block)
static_assert(RING_BN * 128 == SLOT, "A and B blocks have the same size");
constexpr int RING_THREADS = 256;
constexpr int RECV_BYTES = BM * RING_BN * 4;  // one 128 x 128 FP32 block of C
static_assert(2 * RECV_BYTES <= NSLOT * SLOT, "the receive buffers alias the stage memory");
constexpr int GROUP_ROWS = 16;                // row blocks per group of the cluster order

struct RingBars {
    uint64_t a_full[NSLOT];
    uint64_t a_free[NSLOT];
    uint64_t credit[NSLOT];
    uint64_t b_full[NSLOT];
    uint64_t b_empty[NSLOT];
    uint64_t acc_full;
    uint64_t mma_done;
    uint32_t tmem_base;
    int abort;
};
constexpr int RING_SMEM = NSLOT * SLOT + 1024 + int(sizeof(RingBars));

struct RingTcArgs {
    int M, N, K;
    int a_mn, b_mn;
    int P, KA;
    int ra;                 // A slots (the other NSLOT - ra slots are B stages)
    int tiles_m, panels;
    float alpha, beta;
    float* C;
    int64_t ldc;
    uint64_t timeout_ns;
};

// Back-shift receive buffer: 128 rows of 32 16-byte chunks; chunk c of row r sits at
// position c XOR (r mod 32), so the 32 rows a warp writes at one column fall on all banks.
__device__ __forceinline__ uint32_t recv_offset(int row, int chunk) {
    return uint32_t(row) * 512u + uint32_t((chunk ^ (row & 31)) * 16);
}

__global__ void __launch_bounds__(RING_THREADS, 1)
    gemm_tc_ring_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        RingTcArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint8_t* a_slots = smem;
    const int RA = g.ra, RB = NSLOT - g.ra;
    uint8_t* b_stages = smem + RA * SLOT;
    RingBars* bars = reinterpret_cast<RingBars*>(smem + NSLOT * SLOT);
    const int warp = int(warp_id()), lane = int(lane_id());
    uint32_t* status = &g_status_ring_tc;
    const int P = g.P, KA = g.KA, KT = P / KA;
    const int ci = int(cluster_ctarank());
    const uint32_t up = uint32_t((ci + KA) % P);        // A blocks arrive from here
    const uint32_t down = uint32_t((ci - KA + P) % P);  // and leave to here
    // cluster -> (row block tm, column panel cx): groups of GROUP_ROWS row blocks sweep the
    // panels, so that the B panels the running clusters read are shared by many row blocks in L2
    int tm, cx;
    {
        const int c = int(blockIdx.x) / P;
        const int gsz = GROUP_ROWS * g.panels;
        const int first = (c / gsz) * GROUP_ROWS;
        const int rows = min(GROUP_ROWS, g.tiles_m - first);
        const int r = c - (c / gsz) * gsz;
        tm = first + r % rows;
        cx = r / rows;
    }
    const int nkb = (g.K + RC::BK - 1) / RC::BK;
    const int rounds = (nkb + P - 1) / P;
    const int F = rounds * KT;                          // A blocks that pass through this CTA
    const uint32_t tmem_cols = uint32_t(KA * RING_BN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < RA; ++s) {
            mbar_init(&bars->a_full[s], 1);
            mbar_init(&bars->a_free[s], 2);
            mbar_init(&bars->credit[s], 1);
        }
        for (int s = 0; s < RB; ++s) {
            mbar_init(&bars->b_full[s], 1);
            mbar_init(&bars->b_empty[s], 1);
        }
        mbar_init(&bars->acc_full, 1);
        mbar_init(&bars->mma_done, 1);
        bars->abort = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 1) {
        tmem_alloc(&bars->tmem_base, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    cluster_sync_all();   // every CTA's barriers exist before a peer arrives on them or copies into it
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile int* abort = &bars->abort;

    // fill f (0-based): round f / KT, step jb = f % KT, the k-block that started on CTA (ci + jb K) mod P
    auto kblock = [&](int f) { return (f / KT) * P + (ci + (f % KT) * KA) % P; };
    // first column of accumulator l: block column (ci - l) mod P of the panel
    auto acc_col = [&](int l) { return (cx * P + (ci - l + P) % P) * RING_BN; };

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last[NSLOT];
            for (int s = 0; s < RB; ++s) last[s] = -1;
            bool ok = true;
            for (int f = 0; f < F && ok; ++f) {
                const int kb = kblock(f);
                for (int l = 0; l < KA; ++l) {
                    if (!mbar_wait(&bars->b_empty[stage], phase ^ 1u, g.timeout_ns, status, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&bars->b_full[stage], SLOT);
                    load_operand<RC, RING_BN>(b_stages + stage * SLOT, &tmB, &bars->b_full[stage], g.b_mn != 0,
                                              acc_col(l), kb, 0, false);
                    last[stage] = int(phase);
                    if (++stage == RB) { stage = 0; phase ^= 1u; }
                }
            }
            for (int s = 0; s < RB; ++s)
                if (last[s] >= 0) mbar_wait(&bars->b_full[s], uint32_t(last[s]), g.timeout_ns, status, abort);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc(1u, g.a_mn != 0, g.b_mn != 0, BM, RING_BN);
            const uint64_t a0 = operand_desc<RC>(smem_u32(a_slots), 0, g.a_mn != 0);
            const uint64_t b0 = operand_desc<RC>(smem_u32(b_stages), 0, g.b_mn != 0);
            const uint64_t aks = ks_step<RC>(g.a_mn != 0), bks = ks_step<RC>(g.b_mn != 0);
            const uint64_t sstep = uint64_t(SLOT / 16);
            int bstage = 0;
            uint32_t bphase = 0;
            uint64_t bcur = b0;
            bool ok = true;
            for (int f = 0; f < F && ok; ++f) {
                const int s = f % RA;
                if (!mbar_wait(&bars->a_full[s], uint32_t(f / RA) & 1u, g.timeout_ns, status, abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // a forwarded block has landed: the sender's copy of its fill f-1 is complete
                if (f % KT != 0) mbar_arrive_remote(mapa_shared(smem_u32(&bars->a_free[(f - 1) % RA]), up));
                const uint64_t acur = a0 + uint64_t(s) * sstep;
                for (int l = 0; l < KA; ++l) {
                    if (!mbar_wait(&bars->b_full[bstage], bphase, g.timeout_ns, status, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + uint32_t(l * RING_BN);
#pragma unroll
                    for (int ks = 0; ks < RC::KSTEPS; ++ks)
                        umma_f16(d, acur + ks * aks, bcur + ks * bks, idesc, (f | ks) != 0);
                    umma_commit(&bars->b_empty[bstage]);
                    if (++bstage == RB) { bstage = 0; bphase ^= 1u; bcur = b0; }
                    else bcur += sstep;
                }
                if (ok) umma_commit(&bars->a_free[s]);
            }
            umma_commit(&bars->acc_full);
            umma_commit(&bars->mma_done);
            mbar_wait(&bars->mma_done, 0, g.timeout_ns, status, abort);
        }
    } else if (warp == 2) {
        if (lane == 0) {
            int armed[NSLOT];
            for (int s = 0; s < RA; ++s) armed[s] = -1;
            for (int f = 0; f < F; ++f) {
                const int s = f % RA;
                const uint32_t u = uint32_t(f / RA);
                if (!mbar_wait(&bars->a_free[s], (u & 1u) ^ 1u, g.timeout_ns, status, abort)) break;
                mbar_arrive_expect_tx(&bars->a_full[s], SLOT);
                armed[s] = int(u & 1u);
                if (f % KT == 0)
                    load_operand<RC, BM>(a_slots + s * SLOT, &tmA, &bars->a_full[s], g.a_mn != 0, tm * BM,
                                         kblock(f), 0, false);
                // a forwarded fill: the CTA that sends it may now write slot s (credit of its fill f-1).
                // Only forwarded fills get credits: the next credit of a slot then needs this
                // copy to have landed, so a credit barrier never runs two phases ahead of its waiter.
                if (f % KT != 0) mbar_arrive_remote(mapa_shared(smem_u32(&bars->credit[(f - 1) % RA]), up));
            }
            // no copy may still be landing in this CTA's shared memory when the stage memory is reused
            for (int s = 0; s < RA; ++s)
                if (armed[s] >= 0) mbar_wait(&bars->a_full[s], uint32_t(armed[s]), g.timeout_ns, status, abort);
        }
    } else if (warp == 3) {
        if (lane == 0) {
            uint32_t credit_phase = 0;   // bit s: parity of the next credit phase of slot s
            for (int f = 0; f < F; ++f) {
                const int s = f % RA;
                const uint32_t u = uint32_t(f / RA);
                if (!mbar_wait(&bars->a_full[s], u & 1u, g.timeout_ns, status, abort)) break;
                if (f % KT != KT - 1) {
                    // the receiver has armed its slot for its fill f+1
                    if (!mbar_wait(&bars->credit[s], (credit_phase >> s) & 1u, g.timeout_ns, status, abort)) break;
                    credit_phase ^= 1u << s;
                    const int s1 = (f + 1) % RA;
                    bulk_copy_to_peer(mapa_shared(smem_u32(a_slots + s1 * SLOT), down), a_slots + s * SLOT, SLOT,
                                      mapa_shared(smem_u32(&bars->a_full[s1]), down));
                } else {
                    mbar_arrive(&bars->a_free[s]);   // last step of a round: nothing to forward
                }
            }
        }
    }

    // ---- back-shift and epilogue (every warp takes part in the cluster barriers) ----
    bool have_acc = false;
    if (warp >= 4) {
        int done = 0;
        if (lane == 0) done = mbar_wait(&bars->acc_full, 0, g.timeout_ns, status, abort) ? 1 : 0;
        done = __shfl_sync(0xffffffffu, done, 0);
        have_acc = done != 0 && *abort == 0;
        tc_fence_after();
    }
    __syncwarp();
    fence_proxy_async_smem();
    tc_fence_before();
    cluster_sync_all();   // every CTA's main loop is over: its stage memory becomes the receive buffers
    tc_fence_after();

    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t trow = tmem + (uint32_t(q * 32) << 16);
    const uint32_t left = uint32_t((ci - 1 + P) % P);
    for (int l = KA - 1; l >= 1; --l) {
        if (warp >= 4 && have_acc) {
            // X = C^l + (what CTA i+1 sent at step l+1); X goes to CTA i-1 for its C^(l-1)
            const uint32_t dst = mapa_shared(smem_u32(smem + ((l - 1) & 1) * RECV_BYTES), left);
            const uint8_t* mine = smem + (l & 1) * RECV_BYTES;
#pragma unroll 1
            for (int c0 = 0; c0 < RING_BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(trow + uint32_t(l * RING_BN + c0), r);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int chunk = c0 / 4 + c;
                    float v0 = __uint_as_float(r[4 * c]), v1 = __uint_as_float(r[4 * c + 1]);
                    float v2 = __uint_as_float(r[4 * c + 2]), v3 = __uint_as_float(r[4 * c + 3]);
                    if (l < KA - 1) {
                        const float4 a = *reinterpret_cast<const float4*>(mine + recv_offset(row, chunk));
                        v0 += a.x; v1 += a.y; v2 += a.z; v3 += a.w;
                    }
                    st_peer_v4(dst + recv_offset(row, chunk), v0, v1, v2, v3);
                }
            }
        }
        __syncwarp();
        cluster_sync_all();   // this step's blocks are visible; the other buffer is free again
    }

    if (warp >= 4 && have_acc) {
        const int64_t grow = int64_t(tm) * BM + row;
        const int64_t gcol0 = int64_t(cx * P + ci) * RING_BN;
#pragma unroll 1
        for (int c0 = 0; c0 < RING_BN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(trow + uint32_t(c0), r);
            tmem_ld_wait();
            float v[32];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                if (KA > 1) a = *reinterpret_cast<const float4*>(smem + recv_offset(row, c0 / 4 + c));
                v[4 * c] = __uint_as_float(r[4 * c]) + a.x;
                v[4 * c + 1] = __uint_as_float(r[4 * c + 1]) + a.y;
                v[4 * c + 2] = __uint_as_float(r[4 * c + 2]) + a.z;
                v[4 * c + 3] = __uint_as_float(r[4 * c + 3]) + a.w;
            }
            if (grow < g.M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t col = gcol0 + c0 + j;
                    if (col < g.N) {
                        float* Cp = g.C + grow + col * g.ldc;
                        float o = g.alpha * v[j];
                        if (g.beta != 0.f) o = fmaf(g.beta, *Cp, o);
                        *Cp = o;
                    }
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync_all();   // no CTA leaves while a peer may still address its shared memory
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, tmem_cols);
}

}  // namespace

hsmm_status_t gemm_tc_ring(hsmm_op_t ta, hsmm_op_t tb, int64_t m, int64_t n, int64_t k, float alpha, const void* A,
                           int64_t lda, const void* B, int64_t ldb, float beta, float* C, int64_t ldc, int p, int K,
                           cudaStream_t st) {
    if (p != 2 && p != 4 && p != 8 && p != 16)
        return fail(HSMM_STATUS_INVALID_VALUE, "ring order: p = %d (cluster of 2, 4, 8 or 16 CTAs)", p);
    if (K < 1 || K > 4 || p % K != 0)
        return fail(HSMM_STATUS_INVALID_VALUE, "ring order: K = %d (1..4, dividing p = %d)", K, p);
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "ring order: a dimension exceeds 2^31-1");
    if (!tma_operand_ok(A, lda, 2) || !tma_operand_ok(B, ldb, 2))
        return fail(HSMM_STATUS_NOT_SUPPORTED, "ring order: TMA needs 16-byte aligned A, B and ld*2 multiples of 16");
    const int64_t tiles_m = (m + BM - 1) / BM;
    const int64_t panels = (n + int64_t(p) * RING_BN - 1) / (int64_t(p) * RING_BN);
    if (tiles_m * panels * p > INT32_MAX) return fail(HSMM_STATUS_NOT_SUPPORTED, "ring order: grid too large");
    RingTcArgs g{};
    g.M = int(m); g.N = int(n); g.K = int(k);
    g.a_mn = (ta == HSMM_OP_N);
    g.b_mn = (tb == HSMM_OP_T);
    g.P = p; g.KA = K;
    // deeper A chains when A moves often (small K), more B stages when each A block meets many
    g.ra = K == 1 ? 8 : (K == 2 ? 6 : 4);
    g.tiles_m = int(tiles_m);
    g.panels = int(panels);
    g.alpha = alpha; g.beta = beta; g.C = C; g.ldc = ldc;
    g.timeout_ns = wait_timeout_ns();
    const CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUtensorMap mA, mB;
    bool ok = g.a_mn ? encode_map(&mA, dt, 2, A, uint64_t(m), uint64_t(k), uint64_t(lda), RC::MN_CHUNK, RC::BK)
                     : encode_map(&mA, dt, 2, A, uint64_t(k), uint64_t(m), uint64_t(lda), RC::BK, BM);
    ok = ok && (g.b_mn ? encode_map(&mB, dt, 2, B, uint64_t(n), uint64_t(k), uint64_t(ldb), RC::MN_CHUNK, RC::BK)
                       : encode_map(&mB, dt, 2, B, uint64_t(k), uint64_t(n), uint64_t(ldb), RC::BK, RING_BN));
    if (!ok) return fail(HSMM_STATUS_NOT_SUPPORTED, "ring order: TMA descriptor encoding failed (CUresult %d)",
                         last_encode_result());
    static std::atomic<uint64_t> attrs{0};
    const hsmm_status_t as = attrs_once_per_device(attrs, [] {
        cudaError_t e = cudaFuncSetAttribute(gemm_tc_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, RING_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(gemm_tc_ring_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return e;
    });
    if (as != HSMM_STATUS_SUCCESS) return as;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(tiles_m * panels * p), 1, 1);
    cfg.blockDim = dim3(RING_THREADS, 1, 1);
    cfg.dynamicSmemBytes = RING_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(p);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, gemm_tc_ring_kernel, &cfg);
    if (e != cudaSuccess) return record_cuda(e);
    if (clusters < 1)
        return fail(HSMM_STATUS_NOT_SUPPORTED, "ring order: a cluster of %d CTAs with %d bytes of shared memory each "
                    "does not fit on this GPU", p, RING_SMEM);
    e = cudaLaunchKernelEx(&cfg, gemm_tc_ring_kernel, mA, mB, g);
    count_launches(1);
    if (e != cudaSuccess) return record_cuda(e);
    return check_launch();
}

}  // namespace hsmm
