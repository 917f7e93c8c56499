// nbody.cu -- the two-array n^2 problem of Section 4, F_i = sum_j f(x_i, z_j), with the
// gravitational interaction Section 2 cites as the prototype hyper-systolic application:
//   f(x, z) = m_z (r_z - r_x) / (|r_z - r_x|^2 + eps2)^(3/2)   (0 for coincident bodies).
// Bodies are float4 (px, py, pz, m), results float4 (ax, ay, az, 0); FP32 arithmetic with the
// hardware reciprocal square root.  With eps2 > 0 the kernels work on pairs of x bodies with
// the packed FP32 instructions of this GPU (sub/mul/fma .f32x2: two interactions per
// instruction, the reciprocal square root per half).
//
// Two schedules:
//  * tiled: each thread owns x bodies; the z array streams through shared memory in tiles
//    that every CTA reads from L2 (the GPU's own way to share one array among all cells);
//  * hyper-systolic (Section 4.1 with the regular bases of Definition REGULARBASE2): a
//    cluster of p CTAs is the ring of p cells, each owning a block of x; the K replicas of
//    x (A = (0, 1, ..., 1)) are the blocks of the K-1 right-hand neighbours, read once
//    through distributed shared memory; z passes through the cluster in rounds of p blocks,
//    each block moving K~-1 times by K cells (B = (0, K, ..., K)), and every cell adds the
//    interactions of its K replicas with the z block it holds into K intermediate results;
//    the collector then moves K-1 times by one cell against the replica shifts, adding the
//    intermediate results (back-shift phase).  Every (x block, z block) pair meets once per
//    round because the distances s K - t, 0 <= t < K, 0 <= s < K~, cover 0..p-1.
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace hsmm {
namespace {

constexpr int NB_TILE = 256;    // threads and z tile of the tiled kernel
constexpr int ILP = 2;          // x bodies per thread (tiled, scalar)
constexpr int NB_RING = 128;    // bodies per cell and threads per CTA (hyper-systolic)

// a += f(x, z): m_z d / (|d|^2 + eps2)^(3/2), d = r_z - r_x
__device__ __forceinline__ void interact(const float4& x, const float4& z, float eps2, float3& a) {
    const float dx = z.x - x.x, dy = z.y - x.y, dz = z.z - x.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float inv = rsqrtf(r2);
    const float s = r2 > 0.f ? z.w * (inv * inv * inv) : 0.f;
    a.x = fmaf(s, dx, a.x);
    a.y = fmaf(s, dy, a.y);
    a.z = fmaf(s, dz, a.z);
}

// ---- packed FP32 pairs (f32x2): two x bodies against one z body per instruction ----
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float rsqrt_approx(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// two x bodies (packed coordinates X, Y, Z) against z (coordinates and mass broadcast to both
// halves); eps2 > 0, so r^2 > 0 and no pair needs the r = 0 case
struct XPair {
    uint64_t X, Y, Z, ax, ay, az;
};
__device__ __forceinline__ void interact2(XPair& p, uint64_t zx, uint64_t zy, uint64_t zz, uint64_t zm,
                                          uint64_t eps2x2) {
    const uint64_t dx = sub2(zx, p.X), dy = sub2(zy, p.Y), dz = sub2(zz, p.Z);
    const uint64_t r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, eps2x2)));
    float lo, hi;
    upk2(r2, lo, hi);
    const uint64_t inv = pk2(rsqrt_approx(lo), rsqrt_approx(hi));
    const uint64_t s = mul2(zm, mul2(mul2(inv, inv), inv));
    p.ax = fma2(s, dx, p.ax);
    p.ay = fma2(s, dy, p.ay);
    p.az = fma2(s, dz, p.az);
}

__device__ __forceinline__ XPair make_pair(const float4& a, const float4& b) {
    return XPair{pk2(a.x, b.x), pk2(a.y, b.y), pk2(a.z, b.z), pk2(0.f, 0.f), pk2(0.f, 0.f), pk2(0.f, 0.f)};
}

// 16-byte load from the shared memory of another CTA of the cluster
__device__ __forceinline__ float4 ld_peer_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

// PACKED (eps2 > 0): ILP x bodies per thread as ILP/2 packed pairs; else one body at a time
// with the r = 0 case handled.  The z array is split over the CTAs of a cluster (4 to 8, the
// host picks the count that spreads the CTAs evenly over the SMs) that share the same x bodies;
// their partial sums are added in the fixed order of the cluster ranks through distributed
// shared memory (deterministic, no workspace).
template <bool PACKED, int ILPN>
__global__ void __launch_bounds__(NB_TILE) nbody_tiled(int64_t nx, int64_t nz, const float4* __restrict__ x,
                                                       const float4* __restrict__ z, float eps2,
                                                       float4* __restrict__ out) {
    __shared__ float4 tile[NB_TILE];
    __shared__ float4 part[ILPN][NB_TILE];
    const int zs = int(cluster_ctarank());
    const int ZS = int(cluster_nctarank());
    const int64_t i0 = int64_t(blockIdx.x / ZS) * NB_TILE * ILPN + threadIdx.x;
    const int64_t zchunk = ((nz + ZS - 1) / ZS + NB_TILE - 1) / NB_TILE * NB_TILE;
    const int64_t zbeg = int64_t(zs) * zchunk;
    const int64_t zend = min(nz, zbeg + zchunk);
    float4 xi[ILPN];
#pragma unroll
    for (int k = 0; k < ILPN; ++k) {
        const int64_t i = i0 + k * NB_TILE;
        xi[k] = i < nx ? x[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float3 a[PACKED ? 1 : ILPN];
    XPair pr[PACKED ? ILPN / 2 : 1];
    if constexpr (PACKED) {
#pragma unroll
        for (int k = 0; k < ILPN / 2; ++k) pr[k] = make_pair(xi[2 * k], xi[2 * k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < ILPN; ++k) a[k] = make_float3(0.f, 0.f, 0.f);
    }
    const uint64_t e2 = pk2(eps2, eps2);
    for (int64_t j0 = zbeg; j0 < zend; j0 += NB_TILE) {
        const int64_t j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < zend ? z[j] : make_float4(0.f, 0.f, 0.f, 0.f);   // padding: zero mass
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < NB_TILE; ++q) {
            const float4 zj = tile[q];
            if constexpr (PACKED) {
                const uint64_t zx = pk2(zj.x, zj.x), zy = pk2(zj.y, zj.y), zz = pk2(zj.z, zj.z),
                               zm = pk2(zj.w, zj.w);
#pragma unroll
                for (int k = 0; k < ILPN / 2; ++k) interact2(pr[k], zx, zy, zz, zm, e2);
            } else {
#pragma unroll
                for (int k = 0; k < ILPN; ++k) interact(xi[k], zj, eps2, a[k]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < ILPN; ++k) {
        float3 r;
        if constexpr (PACKED) {
            float l0, h0, l1, h1, l2, h2;
            upk2(pr[k / 2].ax, l0, h0);
            upk2(pr[k / 2].ay, l1, h1);
            upk2(pr[k / 2].az, l2, h2);
            r = (k & 1) ? make_float3(h0, h1, h2) : make_float3(l0, l1, l2);
        } else {
            r = a[k];
        }
        part[k][threadIdx.x] = make_float4(r.x, r.y, r.z, 0.f);
    }
    cluster_sync_all();
    if (zs == 0) {
#pragma unroll
        for (int k = 0; k < ILPN; ++k) {
            float4 sum = part[k][threadIdx.x];
            for (int q = 1; q < ZS; ++q) {
                const float4 v = ld_peer_f4(mapa_shared(smem_u32(&part[k][threadIdx.x]), uint32_t(q)));
                sum.x += v.x;
                sum.y += v.y;
                sum.z += v.z;
            }
            const int64_t i = i0 + k * NB_TILE;
            if (i < nx) out[i] = make_float4(sum.x, sum.y, sum.z, 0.f);
        }
    }
    __syncwarp();
    cluster_sync_all();   // the other ranks keep their partial sums until rank 0 has read them
}

template <int K, bool PACKED>
__global__ void __launch_bounds__(NB_RING) nbody_hsys(int64_t nx, int64_t nz, const float4* __restrict__ x,
                                                      const float4* __restrict__ z, float eps2,
                                                      float4* __restrict__ out, int P) {
    static_assert(!PACKED || K % 2 == 0, "packed replicas come in pairs");
    __shared__ float4 xs[NB_RING];          // this cell's block of x
    __shared__ float4 zb[2][NB_RING];       // the z block held in step s (buffer s % 2) and the next
    __shared__ float4 recv[2][NB_RING];     // back-shift: the collector arriving from the left
    const int c = int(cluster_ctarank());
    const int t = int(threadIdx.x);
    const int Kt = P / K;
    const int64_t cx = int64_t(blockIdx.x) / P;                  // cluster: x blocks cx*P .. cx*P + P-1
    const int64_t xi = (cx * P + c) * NB_RING + t;
    xs[t] = xi < nx ? x[xi] : make_float4(0.f, 0.f, 0.f, 0.f);
    cluster_sync_all();
    // replicas: x^_r at cell c is the block of cell c + r (r shifts of stride 1)
    float4 xr[K];
    float3 acc[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        xr[r] = ld_peer_f4(mapa_shared(smem_u32(&xs[t]), uint32_t((c + r) % P)));
        acc[r] = make_float3(0.f, 0.f, 0.f);
    }
    XPair pr[PACKED ? K / 2 : 1];
    if constexpr (PACKED) {
#pragma unroll
        for (int r = 0; r < K / 2; ++r) pr[r] = make_pair(xr[2 * r], xr[2 * r + 1]);
    }
    const uint64_t e2 = pk2(eps2, eps2);
    const int64_t rounds = (nz + int64_t(P) * NB_RING - 1) / (int64_t(P) * NB_RING);
    for (int64_t rd = 0; rd < rounds; ++rd) {
        __syncthreads();                                          // done with buffer 0 of the last round
        const int64_t zj = (rd * P + c) * NB_RING + t;
        zb[0][t] = zj < nz ? z[zj] : make_float4(0.f, 0.f, 0.f, 0.f);   // padding: zero mass
        cluster_sync_all();                                       // every cell holds its own z block
        for (int s = 0; s < Kt; ++s) {
            const float4* zc = zb[s & 1];
#pragma unroll 4
            for (int q = 0; q < NB_RING; ++q) {
                const float4 zq = zc[q];
                if constexpr (PACKED) {
                    const uint64_t zx = pk2(zq.x, zq.x), zy = pk2(zq.y, zq.y), zz = pk2(zq.z, zq.z),
                                   zm = pk2(zq.w, zq.w);
#pragma unroll
                    for (int r = 0; r < K / 2; ++r) interact2(pr[r], zx, zy, zz, zm, e2);
                } else {
#pragma unroll
                    for (int r = 0; r < K; ++r) interact(xr[r], zq, eps2, acc[r]);
                }
            }
            if (s + 1 < Kt) {
                // z <- cshift^K(z): this cell takes the block of cell c + K into its other buffer
                zb[(s + 1) & 1][t] = ld_peer_f4(mapa_shared(smem_u32(&zb[s & 1][t]), uint32_t((c + K) % P)));
                cluster_sync_all();
            }
        }
    }
    if constexpr (PACKED) {
#pragma unroll
        for (int r = 0; r < K / 2; ++r) {
            float l0, h0, l1, h1, l2, h2;
            upk2(pr[r].ax, l0, h0);
            upk2(pr[r].ay, l1, h1);
            upk2(pr[r].az, l2, h2);
            acc[2 * r] = make_float3(l0, l1, l2);
            acc[2 * r + 1] = make_float3(h0, h1, h2);
        }
    }
    // back-shift: the collector starts as acc[K-1] and moves one cell to the right K-1 times,
    // adding acc[r] (r = K-2 .. 0) at each arrival; it ends on the cell that owns its block
    float3 y = acc[K - 1];
    const uint32_t right = uint32_t((c + 1) % P);
#pragma unroll
    for (int u = 0; u < K - 1; ++u) {
        const uint32_t dst = mapa_shared(smem_u32(&recv[u & 1][t]), right);
        asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "f"(y.x), "f"(y.y), "f"(y.z),
                     "f"(0.f)
                     : "memory");
        cluster_sync_all();
        const float4 in = recv[u & 1][t];
        const int r = K - 2 - u;
        y = make_float3(in.x + acc[r].x, in.y + acc[r].y, in.z + acc[r].z);
    }
    if (xi < nx) out[xi] = make_float4(y.x, y.y, y.z, 0.f);
    __syncwarp();
    cluster_sync_all();                                           // no cell leaves while peers read it
}

}  // namespace

hsmm_status_t nbody_forces(int64_t nx, int64_t nz, const float* x, const float* z, float eps2, float* out,
                           int ring_p, int ring_k, cudaStream_t st) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* z4 = reinterpret_cast<const float4*>(z);
    float4* o4 = reinterpret_cast<float4*>(out);
    // eps2 > 0: r^2 > 0 for every pair, the packed FP32 pair kernels apply
    const bool packed = eps2 > 0.f;
    if (ring_p == 0) {
        const int ilp = packed ? 4 : ILP;
        // z split over zsplit CTAs: the count in 4..8 that spreads the CTAs most evenly over the SMs
        const int64_t xblocks = (nx + int64_t(NB_TILE) * ilp - 1) / (int64_t(NB_TILE) * ilp);
        const int sms = num_sms();
        int zsplit = 4;
        double best = -1.0;
        for (int c = 4; c <= 8; ++c) {
            const double per_sm = double(xblocks * c) / sms;
            const double eff = per_sm / double(int64_t(per_sm + 0.999999));
            if (eff > best + 1e-9) { best = eff; zsplit = c; }
        }
        const int64_t blocks = xblocks * zsplit;
        if (blocks > INT32_MAX) return HSMM_STATUS_NOT_SUPPORTED;
        cudaLaunchConfig_t tc = {};
        tc.gridDim = dim3(unsigned(blocks), 1, 1);
        tc.blockDim = dim3(NB_TILE, 1, 1);
        tc.stream = st;
        cudaLaunchAttribute ta[1];
        ta[0].id = cudaLaunchAttributeClusterDimension;
        ta[0].val.clusterDim.x = unsigned(zsplit);
        ta[0].val.clusterDim.y = 1;
        ta[0].val.clusterDim.z = 1;
        tc.attrs = ta;
        tc.numAttrs = 1;
        const cudaError_t te = packed ? cudaLaunchKernelEx(&tc, nbody_tiled<true, 4>, nx, nz, x4, z4, eps2, o4)
                                      : cudaLaunchKernelEx(&tc, nbody_tiled<false, ILP>, nx, nz, x4, z4, eps2, o4);
        count_launches(1);
        if (te != cudaSuccess) return record_cuda(te);
        return check_launch();
    }
    const int P = ring_p, K = ring_k;
    const int64_t clusters = (nx + int64_t(P) * NB_RING - 1) / (int64_t(P) * NB_RING);
    if (clusters * P > INT32_MAX) return HSMM_STATUS_NOT_SUPPORTED;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(clusters * P), 1, 1);
    cfg.blockDim = dim3(NB_RING, 1, 1);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = unsigned(P);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    static std::atomic<uint64_t> attrs{0};
    const hsmm_status_t as = attrs_once_per_device(attrs, [] {
        const void* kerns[5] = {reinterpret_cast<const void*>(nbody_hsys<1, false>),
                                reinterpret_cast<const void*>(nbody_hsys<2, false>),
                                reinterpret_cast<const void*>(nbody_hsys<4, false>),
                                reinterpret_cast<const void*>(nbody_hsys<2, true>),
                                reinterpret_cast<const void*>(nbody_hsys<4, true>)};
        cudaError_t r = cudaSuccess;
        for (int i = 0; i < 5 && r == cudaSuccess; ++i)
            r = cudaFuncSetAttribute(kerns[i], cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return r;
    });
    if (as != HSMM_STATUS_SUCCESS) return as;
    switch (K) {
        case 1: e = cudaLaunchKernelEx(&cfg, nbody_hsys<1, false>, nx, nz, x4, z4, eps2, o4, P); break;
        case 2:
            e = packed ? cudaLaunchKernelEx(&cfg, nbody_hsys<2, true>, nx, nz, x4, z4, eps2, o4, P)
                       : cudaLaunchKernelEx(&cfg, nbody_hsys<2, false>, nx, nz, x4, z4, eps2, o4, P);
            break;
        case 4:
            e = packed ? cudaLaunchKernelEx(&cfg, nbody_hsys<4, true>, nx, nz, x4, z4, eps2, o4, P)
                       : cudaLaunchKernelEx(&cfg, nbody_hsys<4, false>, nx, nz, x4, z4, eps2, o4, P);
            break;
        default: return HSMM_STATUS_INVALID_VALUE;
    }
    count_launches(1);
    if (e != cudaSuccess) return record_cuda(e);
    return check_launch();
}

}  // namespace hsmm
