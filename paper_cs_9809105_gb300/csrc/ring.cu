// ring.cu -- the paper's hyper-systolic matrix product (Algorithm 2) on one GPU.
//
// p virtual processors = the p CTAs of one thread-block cluster (p <= 16; 16 is a
// non-portable cluster size).  Block mapping (Section 6.1): the n x n matrices are
// p x p systems of b x b blocks (b = n/p), each CTA owns one block column, and the
// p x p system is held in skew order: CTA i, slot l holds block row (l+i) mod p of
// column i (Sections 3.2.1, 3.3.1; 0-based).
//
//   pre-shift of B   row g of every block column moves with stride MOD(1-g, K)
//                    (Fortran sign, i.e. -((g-1) mod K)); a one-time permutation,
//                    realised by reading the pre-shifted blocks of B from memory;
//   main phase       K~ = p/K blocks of K steps.  Step g = (jb-1)K + l:
//                      C^l[n] += A[slot (n-g) mod p] (x) B'[g]     for all slots n
//                    (cshift-col^(1-g) is an address, Eq. CSHIFT1's companion); between
//                    blocks A <- cshift-row^K(A): every CTA copies the A slab of CTA
//                    (i+K) mod p out of that CTA's shared memory (DSMEM), in chunks
//                    through a staging buffer, with cluster barriers between reads
//                    and writes;
//   back-shift       for j = 1..K-1: C^(K-j) += cshift-row^1(C^(K-j+1)).
//
// The A slab (p b^2 doubles, 128 KiB for p = 16, b = 32) lives in shared memory;
// C^1 is accumulated directly into C (normal order, skew addressing), the aux
// arrays C^2..C^K live in the caller's workspace.  The local block product (x) is
// a plain FP64 FMA loop: this workload is a correctness configuration of the
// paper's schedule, not a throughput path.
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace hsmm {

static __device__ uint32_t g_status_ring;

uint32_t status_take_ring() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_ring, sizeof(v));
    cudaMemcpyToSymbol(g_status_ring, &z, sizeof(z));
    return v;
}

namespace {

constexpr int RT = 256;          // threads per CTA (virtual processor)
constexpr int CHUNK_SLOTS = 4;   // slots moved per DSMEM staging round

struct RingArgs {
    int p, K, b;
    int64_t n;
    const double* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    double* C;
    int64_t ldc;
    double* aux;        // (K-1) arrays, each p processors x p slots x b*b, column-major blocks
};

__device__ __forceinline__ int pmod(int a, int p) {
    const int r = a % p;
    return r < 0 ? r + p : r;
}

// Fortran MOD(a, k): remainder with the sign of a
__device__ __forceinline__ int fmod_int(int a, int k) { return a - k * (a / k); }

__global__ void __launch_bounds__(RT, 1) ring_kernel(RingArgs g) {
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) double sm[];
    const int p = g.p, K = g.K, b = g.b, bb = b * b;
    const int i = int(cluster.block_rank());       // processor index (0-based)
    double* As = sm;                                 // p slots x b*b
    double* stage = As + size_t(p) * bb;             // CHUNK_SLOTS x b*b
    double* Bs = stage + size_t(CHUNK_SLOTS) * bb;   // one block of B'
    const int tid = threadIdx.x;

    // load the A slab of processor i in skew order: slot l = block row (l + i) mod p
    for (int l = 0; l < p; ++l) {
        const int R = pmod(l + i, p);
        for (int e = tid; e < bb; e += RT) {
            const int r = e % b, c = e / b;
            As[size_t(l) * bb + e] = g.A[int64_t(R) * b + r + (int64_t(i) * b + c) * g.lda];
        }
    }
    cluster.sync();

    const int Kt = p / K;
    for (int jb = 0; jb < Kt; ++jb) {
        for (int l = 0; l < K; ++l) {
            const int g1 = jb * K + l + 1;                 // step g, 1-based
            // B'[g] of processor i: pre-shift stride sigma = MOD(1-g, K) moves row g of the
            // skewed B so that processor i holds the slot-g block of processor i + sigma
            const int sigma = fmod_int(1 - g1, K);
            const int src = pmod(i + sigma, p);
            const int Rb = pmod((g1 - 1) + src, p);         // skew: slot g-1 of processor src
            __syncthreads();
            for (int e = tid; e < bb; e += RT) {
                const int r = e % b, c = e / b;
                Bs[e] = g.B[int64_t(Rb) * b + r + (int64_t(src) * b + c) * g.ldb];
            }
            __syncthreads();
            // C^l[n] += A[slot (n - g) mod p] (x) B'[g], all slots n
            for (int nslot = 0; nslot < p; ++nslot) {
                const double* Ab = As + size_t(pmod(nslot - (g1 - 1), p)) * bb;
                for (int e = tid; e < bb; e += RT) {
                    const int r = e % b, c = e / b;
                    double acc = 0.0;
                    for (int kk = 0; kk < b; ++kk) acc = fma(Ab[r + kk * b], Bs[kk + c * b], acc);
                    double* dst;
                    if (l == 0) {
                        // C^1 is stored in C: slot nslot of processor i is block row (nslot + i) mod p
                        const int R = pmod(nslot + i, p);
                        dst = g.C + int64_t(R) * b + r + (int64_t(i) * b + c) * g.ldc;
                    } else {
                        dst = g.aux + (size_t(l - 1) * p * p + size_t(i) * p + nslot) * bb + e;
                    }
                    *dst = (jb == 0) ? acc : *dst + acc;
                }
            }
        }
        if (jb + 1 < Kt) {
            // A <- cshift-row^K(A): processor i receives the slab of processor (i + K) mod p
            const int from = pmod(i + K, p);
            for (int s0 = 0; s0 < p; s0 += CHUNK_SLOTS) {
                const int ns = (p - s0) < CHUNK_SLOTS ? (p - s0) : CHUNK_SLOTS;
                cluster.sync();                               // all reads of these slots are done
                const double* remote = cluster.map_shared_rank(As, from) + size_t(s0) * bb;
                for (int e = tid; e < ns * bb; e += RT) stage[e] = remote[e];
                cluster.sync();                               // every CTA holds its incoming chunk
                for (int e = tid; e < ns * bb; e += RT) As[size_t(s0) * bb + e] = stage[e];
            }
            cluster.sync();
        }
    }
    // back-shift and accumulation: C^(K-j) += cshift-row^1(C^(K-j+1)), j = 1..K-1
    const int right = pmod(i + 1, p);
    for (int j = 1; j <= K - 1; ++j) {
        __threadfence();
        cluster.sync();                                        // C^(K-j+1) complete everywhere
        const int lsrc = K - j + 1, ldst = K - j;              // 1-based aux indices
        const double* srcslab = g.aux + (size_t(lsrc - 2) * p * p + size_t(right) * p) * bb;
        for (int nslot = 0; nslot < p; ++nslot) {
            for (int e = tid; e < bb; e += RT) {
                const double v = srcslab[size_t(nslot) * bb + e];
                if (ldst == 1) {
                    const int r = e % b, c = e / b;
                    const int R = pmod(nslot + i, p);
                    g.C[int64_t(R) * b + r + (int64_t(i) * b + c) * g.ldc] += v;
                } else {
                    g.aux[(size_t(ldst - 2) * p * p + size_t(i) * p + nslot) * bb + e] += v;
                }
            }
        }
    }
    cluster.sync();
}

}  // namespace

size_t ring_workspace_bytes(int p, int K, int64_t n) {
    (void)p;
    return size_t(K - 1) * size_t(n) * size_t(n) * sizeof(double);
}

hsmm_status_t ring_gemm_f64(int p, int K, int64_t n, const double* A, int64_t lda, const double* B, int64_t ldb,
                            double* C, int64_t ldc, void* workspace, size_t workspace_bytes, cudaStream_t st) {
    const int b = int(n / p);
    if (workspace_bytes < ring_workspace_bytes(p, K, n) || (K > 1 && !workspace))
        return HSMM_STATUS_WORKSPACE_TOO_SMALL;
    RingArgs g{p, K, b, n, A, lda, B, ldb, C, ldc, static_cast<double*>(workspace)};
    const size_t smem = (size_t(p) + CHUNK_SLOTS + 1) * size_t(b) * b * sizeof(double);
    static std::atomic<uint64_t> attrs{0};
    const hsmm_status_t as = attrs_once_per_device(attrs, [] {
        cudaError_t e = cudaFuncSetAttribute(ring_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return e;
    });
    if (as != HSMM_STATUS_SUCCESS) return as;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(p), 1, 1);
    cfg.blockDim = dim3(RT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(p);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, ring_kernel, g);
    count_launches(1);
    if (e != cudaSuccess) return record_cuda(e);
    return check_launch();
}

}  // namespace hsmm
