// ozaki.cu -- the splitting step of the FP64-accurate product.
//
// Error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59,
// 2012) in its fixed-point integer form: for every row of op(A) (every column of
// op(B)) with exponent e (the smallest integer with |m| < 2^e over that line),
//   x = m 2^-e,  for t = 1..s:  y = x 2^bits,  q_t = trunc(y),  x = y - q_t.
// The digits q_t are read from the IEEE-754 significand with integer shifts (the
// values the exact FP64 steps give); |q_t| <= 2^bits - 1 <= 127, so the slices are
// stored exactly as BF16.  Output layout [t][v][w]: v = row of op(A) (column of
// op(B)), w = the contraction index, contiguous, row pitch ldq (a multiple of 8 so
// that the TMA row stride is a multiple of 16 bytes).
//
// Kernels: (1) exponent init, (2) per-line maximum exponent with atomicMax,
// (3) slicing (transposing through shared memory when the input has v contiguous),
// (4) zero-line fix-up of the exponents.  All HBM-bound.
#include <climits>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace hsmm {

static __device__ uint32_t g_status_ozaki;

uint32_t status_take_ozaki() {
    uint32_t v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_status_ozaki, sizeof(v));
    cudaMemcpyToSymbol(g_status_ozaki, &z, sizeof(z));
    return v;
}

int64_t ozaki_ldq(int64_t k) { return (k + 7) / 8 * 8; }

int64_t ozaki_plane_pitch(int64_t elems, int64_t elem_bytes) {
    const int64_t bytes = (elems * elem_bytes + 255) / 256 * 256 + 1024;
    return bytes / elem_bytes;
}

namespace {

__global__ void expo_init(int64_t nvec, int32_t* expo) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < nvec) expo[i] = INT_MIN;
}

__global__ void expo_fix(int64_t nvec, int32_t* expo) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < nvec && expo[i] == INT_MIN) expo[i] = 0;
}

__device__ __forceinline__ int line_exponent(double mx) {
    if (mx == 0.0) return INT_MIN;
    int e;
    frexp(mx, &e);       // mx = f 2^e with f in [0.5, 1): mx < 2^e, and 2^(e-1) <= mx
    return e;
}

// |x| as its IEEE-754 bit pattern without the sign.  For finite values the unsigned order of
// these patterns is the order of the magnitudes.  A line's exponent needs only the largest
// high word (sign cleared) while any is non-zero, and the largest low word when all high
// words are zero (tiny subnormals), so the running "maximum" keeps the two 32-bit halves'
// maxima apart: 32-bit integer operations only (64-bit compares went to the narrow FP64 pipe).
__device__ __forceinline__ uint64_t mag_bits(double x) {
    return uint64_t(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ uint64_t mag_max(uint64_t a, uint64_t b) {
    const uint32_t hi = max(uint32_t(a >> 32), uint32_t(b >> 32)), lo = max(uint32_t(a), uint32_t(b));
    return (uint64_t(hi) << 32) | lo;
}
// exponent of a line from its halfwise maximum (INT_MIN for an all-zero line)
__device__ __forceinline__ int line_exponent_bits(uint64_t mb) {
    const uint64_t top = (mb >> 32) ? (mb & 0xFFFFFFFF00000000ull) : mb;   // the low word matters only alone
    return top == 0 ? INT_MIN : line_exponent(__longlong_as_double(int64_t(top)));
}

// v contiguous in memory (M(v, w) at v + w*ld): thread per v, w split over blockIdx.y;
// four independent maxima keep four loads in flight per thread
__global__ void __launch_bounds__(256) expo_vcontig(int64_t nv, int64_t nw, const double* __restrict__ M, int64_t ld,
                                                   int64_t w_per_split, int32_t* expo) {
    const int64_t v = int64_t(blockIdx.x) * 256 + threadIdx.x;
    if (v >= nv) return;
    const int64_t w0 = int64_t(blockIdx.y) * w_per_split;
    const int64_t w1 = min(nw, w0 + w_per_split);
    const double* p = M + v;
    uint64_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int64_t w = w0;
    for (; w + 4 <= w1; w += 4) {
        m0 = mag_max(m0, mag_bits(__ldcs(p + (w + 0) * ld)));
        m1 = mag_max(m1, mag_bits(__ldcs(p + (w + 1) * ld)));
        m2 = mag_max(m2, mag_bits(__ldcs(p + (w + 2) * ld)));
        m3 = mag_max(m3, mag_bits(__ldcs(p + (w + 3) * ld)));
    }
    for (; w < w1; ++w) m0 = mag_max(m0, mag_bits(__ldcs(p + w * ld)));
    const int e = line_exponent_bits(mag_max(mag_max(m0, m1), mag_max(m2, m3)));
    if (e != INT_MIN) atomicMax(&expo[v], e);
}

// The same with two lines per thread and 16-byte loads (nv even, ld even, M 16-byte aligned):
// half the load requests
__global__ void __launch_bounds__(256) expo_vcontig2(int64_t nv, int64_t nw, const double* __restrict__ M, int64_t ld,
                                                    int64_t w_per_split, int32_t* expo) {
    const int64_t v = (int64_t(blockIdx.x) * 256 + threadIdx.x) * 2;
    if (v >= nv) return;
    const int64_t w0 = int64_t(blockIdx.y) * w_per_split;
    const int64_t w1 = min(nw, w0 + w_per_split);
    const double2* p = reinterpret_cast<const double2*>(M + v);
    const int64_t ld2 = ld / 2;
    uint64_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    int64_t w = w0;
    for (; w + 2 <= w1; w += 2) {
        const double2 x0 = __ldcs(p + w * ld2), x1 = __ldcs(p + (w + 1) * ld2);
        a0 = mag_max(a0, mag_bits(x0.x));
        b0 = mag_max(b0, mag_bits(x0.y));
        a1 = mag_max(a1, mag_bits(x1.x));
        b1 = mag_max(b1, mag_bits(x1.y));
    }
    if (w < w1) {
        const double2 x0 = __ldcs(p + w * ld2);
        a0 = mag_max(a0, mag_bits(x0.x));
        b0 = mag_max(b0, mag_bits(x0.y));
    }
    const int ea = line_exponent_bits(mag_max(a0, a1)), eb = line_exponent_bits(mag_max(b0, b1));
    if (ea != INT_MIN) atomicMax(&expo[v], ea);
    if (eb != INT_MIN) atomicMax(&expo[v + 1], eb);
}

// w contiguous in memory (M(w, v) at w + v*ld): block per (v, w-chunk)
__global__ void __launch_bounds__(256) expo_wcontig(int64_t nv, int64_t nw, const double* __restrict__ M, int64_t ld,
                                                   int64_t w_per_split, int32_t* expo) {
    const int64_t v = blockIdx.x;
    const int64_t w0 = int64_t(blockIdx.y) * w_per_split;
    const int64_t w1 = min(nw, w0 + w_per_split);
    uint64_t mx = 0;
    const double* line = M + v * ld;
    if ((reinterpret_cast<uintptr_t>(line + w0) & 15u) == 0) {
        // 16-byte loads: two consecutive entries per thread and step (the line start is aligned)
        const double2* l2 = reinterpret_cast<const double2*>(line + w0);
        const int64_t n2 = (w1 - w0) / 2;
        for (int64_t i = threadIdx.x; i < n2; i += 256) {
            const double2 x = __ldcs(l2 + i);
            mx = mag_max(mx, mag_max(mag_bits(x.x), mag_bits(x.y)));
        }
        if (threadIdx.x == 0 && ((w1 - w0) & 1)) mx = mag_max(mx, mag_bits(__ldcs(line + w1 - 1)));
    } else {
        for (int64_t w = w0 + threadIdx.x; w < w1; w += 256) mx = mag_max(mx, mag_bits(__ldcs(line + w)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = mag_max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    __shared__ uint64_t red[8];
    if (lane_id() == 0) red[warp_id()] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t m2 = red[0];
        for (int i = 1; i < 8; ++i) m2 = mag_max(m2, red[i]);
        const int e = line_exponent_bits(m2);
        if (e != INT_MIN) atomicMax(&expo[v], e);
    }
    (void)nv;
}

// BF16 bit pattern of a small integer q (|q| <= 255: exact), from integer operations only
__device__ __forceinline__ uint16_t bf16_of_small_int(uint32_t mag, uint32_t neg) {
    if (mag == 0) return 0;
    const uint32_t top = 31u - uint32_t(__clz(mag));          // 0..7
    const uint32_t mant = (mag << (7u - top)) & 0x7Fu;
    return uint16_t((neg << 15) | ((127u + top) << 7) | mant);
}

// Slice one value into s digits of `bits` bits, truncating toward zero.  With
// |v| = M 2^(E-1075) (M the 53-bit significand), digit t of |v| 2^(-e) is
//   floor(M 2^(E - 1075 - e + bits t)) mod 2^bits,
// read from the significand with integer shifts: the same digits the FP64 steps
// y = x 2^bits, q = trunc(y), x = y - q produce, without FP64 arithmetic (the FP64
// pipe of this GPU is narrow).  Each digit carries the sign of v.
__device__ __forceinline__ void slice_value(double val, int e, int bits, int s, __nv_bfloat16* out,
                                            int64_t slice_stride) {
    const uint64_t u = uint64_t(__double_as_longlong(val));
    const uint32_t neg = uint32_t(u >> 63);
    int E = int((u >> 52) & 0x7FF);
    uint64_t M = u & ((uint64_t(1) << 52) - 1);
    if (E != 0) M |= uint64_t(1) << 52; else E = 1;           // subnormals: no implicit bit
    const uint32_t mask = (1u << bits) - 1u;
    uint16_t* o = reinterpret_cast<uint16_t*>(out);
    if (e == INT_MIN || M == 0) {
        for (int t = 0; t < s; ++t) o[int64_t(t) * slice_stride] = 0;
        return;
    }
    const int base = E - 1075 - e;                             // <= -53 because |v| < 2^e
    if (bits * s <= 63) {
        // all s digits at once: F = floor(|v| 2^(bits s - e)) fits in 63 bits
        const int sh = base + bits * s;
        const uint64_t F = sh >= 0 ? (M << sh) : (-sh >= 64 ? 0 : (M >> -sh));
        for (int t = 1; t <= s; ++t) {
            const uint32_t d = uint32_t(F >> (bits * (s - t))) & mask;
            o[int64_t(t - 1) * slice_stride] = bf16_of_small_int(d, neg);
        }
    } else {
        for (int t = 1; t <= s; ++t) {
            const int sh = base + bits * t;
            uint32_t d;
            if (sh < 0) d = (-sh >= 64) ? 0u : uint32_t(M >> -sh) & mask;
            else d = (sh >= bits) ? 0u : uint32_t(M << sh) & mask;
            o[int64_t(t - 1) * slice_stride] = bf16_of_small_int(d, neg);
        }
    }
}

// w contiguous: thread per (w, v) element, coalesced in and out
__global__ void __launch_bounds__(256) slice_wcontig(int64_t nv, int64_t nw, const double* __restrict__ M, int64_t ld,
                                                    const int32_t* __restrict__ expo, int bits, int s,
                                                    __nv_bfloat16* __restrict__ q, int64_t ldq, int64_t slice_stride) {
    const int64_t v = blockIdx.y;
    const int64_t w = int64_t(blockIdx.x) * 256 + threadIdx.x;
    if (w >= ldq) return;
    __nv_bfloat16* out = q + v * ldq + w;
    if (w >= nw) {
        for (int t = 0; t < s; ++t) out[int64_t(t) * slice_stride] = __float2bfloat16_rn(0.f);
        return;
    }
    slice_value(M[w + v * ld], expo[v], bits, s, out, slice_stride);
}

// v contiguous: 32 x 32 tiles transposed through shared memory
__global__ void __launch_bounds__(256) slice_vcontig(int64_t nv, int64_t nw, const double* __restrict__ M, int64_t ld,
                                                    const int32_t* __restrict__ expo, int bits, int s,
                                                    __nv_bfloat16* __restrict__ q, int64_t ldq, int64_t slice_stride) {
    __shared__ double tile[32][33];
    const int64_t v0 = int64_t(blockIdx.y) * 32, w0 = int64_t(blockIdx.x) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    // load: threads along v (contiguous)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int wl = ty + 8 * i;
        const int64_t v = v0 + tx, w = w0 + wl;
        tile[wl][tx] = (v < nv && w < nw) ? M[v + w * ld] : 0.0;
    }
    __syncthreads();
    // store: threads along w (contiguous in the output)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int vl = ty + 8 * i;
        const int64_t v = v0 + vl, w = w0 + tx;
        if (v >= nv || w >= ldq) continue;
        __nv_bfloat16* out = q + v * ldq + w;
        if (w >= nw) {
            for (int t = 0; t < s; ++t) out[int64_t(t) * slice_stride] = __float2bfloat16_rn(0.f);
            continue;
        }
        slice_value(tile[tx][vl], expo[v], bits, s, out, slice_stride);
    }
}

// One value prepared for digit extraction: |v| = mag 2^(base + e), so digit t of
// |v| 2^(-e) is floor(mag 2^(base + bits t)) mod 2^bits (see slice_value).
struct Digits {
    uint64_t mag;
    int base;
    uint32_t neg;
};

__device__ __forceinline__ Digits prepare_digits(double val, int e) {
    const uint64_t u = uint64_t(__double_as_longlong(val));
    Digits r;
    r.neg = uint32_t(u >> 63);
    int E = int((u >> 52) & 0x7FF);
    r.mag = u & ((uint64_t(1) << 52) - 1);
    if (E != 0) r.mag |= uint64_t(1) << 52; else E = 1;
    if (e == INT_MIN) r.mag = 0;
    r.base = E - 1075 - (e == INT_MIN ? 0 : e);
    return r;
}

__device__ __forceinline__ uint32_t digit_bits(const Digits& x, int bits, int t) {
    const uint32_t mask = (1u << bits) - 1u;
    const int sh = x.base + bits * t;
    if (sh < 0) return (-sh >= 64) ? 0u : uint32_t(x.mag >> -sh) & mask;
    return (sh >= bits) ? 0u : uint32_t(x.mag << sh) & mask;
}

// Four consecutive values of one line -> for each slice t one 8-byte store of four BF16 digits.
__device__ __forceinline__ void slice_store4(const double (&x)[4], int e, int bits, int s, uint16_t* out,
                                             int64_t slice_stride) {
    Digits dg[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) dg[c] = prepare_digits(x[c], e);
    for (int t = 1; t <= s; ++t) {
        uint32_t h[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) h[c] = bf16_of_small_int(digit_bits(dg[c], bits, t), dg[c].neg);
        uint2 pk;
        pk.x = h[0] | (h[1] << 16);
        pk.y = h[2] | (h[3] << 16);
        *reinterpret_cast<uint2*>(out + int64_t(t - 1) * slice_stride) = pk;
    }
}

// Fixed digit width and count known at compile time with BITS * S <= 63: the integer
// F = floor(|v| 2^(BITS S - e)) < 2^(BITS S) holds all S digits (digit t is bits
// BITS (S - t) .. BITS (S - t + 1) - 1 of F), the same digits as digit_bits gives.
template <int BITS, int S>
__device__ __forceinline__ uint64_t digits_word(double val, int e, uint32_t& neg) {
    static_assert(BITS * S <= 63, "all digits must fit one 64-bit word");
    const uint64_t u = uint64_t(__double_as_longlong(val));
    neg = uint32_t(u >> 63);
    int E = int((u >> 52) & 0x7FF);
    uint64_t mag = u & ((uint64_t(1) << 52) - 1);
    if (E != 0) mag |= uint64_t(1) << 52; else E = 1;
    if (e == INT_MIN) return 0;
    const int sh = E - 1075 - e + BITS * S;
    if (sh >= 0) return sh >= 64 ? 0 : (mag << sh);
    return -sh >= 64 ? 0 : (mag >> -sh);
}

// BF16 patterns of two digits d in [0, 255], each with the sign n of its value (none for d = 0):
// the FP32 number (-1)^n (2^23 + d) holds d in its low significand bits, and minus (-1)^n 2^23
// it is exactly (-1)^n d (+0 for d = 0); one packed subtraction makes both, and the upper halves
// of the two results, gathered by one byte permutation, are the two BF16 patterns (float(d)
// has at most 8 significant bits).  Full-rate FP32 and integer operations only.
__device__ __forceinline__ uint32_t bf16x2_of_digits(uint32_t d0, uint32_t d1, uint64_t signed_bias) {
    const uint64_t a = (uint64_t(uint32_t(signed_bias >> 32) | d1) << 32) | (uint32_t(signed_bias) | d0);
    uint64_t y;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(y) : "l"(a), "l"(signed_bias));
    return __byte_perm(uint32_t(y), uint32_t(y >> 32), 0x7632);
}

template <int BITS, int S>
__device__ __forceinline__ void slice_store4_fixed(const double (&x)[4], int e, uint16_t* out, int64_t slice_stride) {
    constexpr uint32_t MASK = (1u << BITS) - 1u;
    uint64_t F[4];
    uint32_t ng[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) F[c] = digits_word<BITS, S>(x[c], e, ng[c]);
    // (-1)^n 2^23 of each value, two per 64-bit word
    const uint64_t b01 = (uint64_t(0x4B000000u | (ng[1] << 31)) << 32) | (0x4B000000u | (ng[0] << 31));
    const uint64_t b23 = (uint64_t(0x4B000000u | (ng[3] << 31)) << 32) | (0x4B000000u | (ng[2] << 31));
#pragma unroll
    for (int t = 1; t <= S; ++t) {
        uint32_t d[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) d[c] = uint32_t(F[c] >> (BITS * (S - t))) & MASK;
        uint2 pk;
        pk.x = bf16x2_of_digits(d[0], d[1], b01);
        pk.y = bf16x2_of_digits(d[2], d[3], b23);
        *reinterpret_cast<uint2*>(out + int64_t(t - 1) * slice_stride) = pk;
    }
}

// BITS = 0: digit width and count from the arguments; else the compile-time form
template <int BITS, int S>
__device__ __forceinline__ void slice_store4_any(const double (&x)[4], int e, int bits, int s, uint16_t* out,
                                                 int64_t slice_stride) {
    if constexpr (BITS > 0) slice_store4_fixed<BITS, S>(x, e, out, slice_stride);
    else slice_store4(x, e, bits, s, out, slice_stride);
}

// w contiguous, four consecutive w per thread: 16-byte loads (ld even, M 16-byte aligned)
// and 8-byte stores (ldq and the slice pitch multiples of 4, q 8-byte aligned)
template <int BITS, int S>
__global__ void __launch_bounds__(256) slice_wcontig4(int64_t nv, int64_t nw, const double* __restrict__ M, int64_t ld,
                                                     const int32_t* __restrict__ expo, int bits, int s,
                                                     __nv_bfloat16* __restrict__ q, int64_t ldq, int64_t slice_stride) {
    const int64_t v = blockIdx.y;
    const int64_t w = (int64_t(blockIdx.x) * 256 + threadIdx.x) * 4;
    if (w >= ldq) return;
    const double* row = M + v * ld;
    double x[4];
    if (w + 4 <= nw) {
        const double2 p0 = __ldcs(reinterpret_cast<const double2*>(row + w));
        const double2 p1 = __ldcs(reinterpret_cast<const double2*>(row + w + 2));
        x[0] = p0.x; x[1] = p0.y; x[2] = p1.x; x[3] = p1.y;
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = (w + c < nw) ? row[w + c] : 0.0;
    }
    slice_store4_any<BITS, S>(x, expo[v], bits, s, reinterpret_cast<uint16_t*>(q) + v * ldq + w, slice_stride);
}

// v contiguous: 64 (w) x 32 (v) tiles transposed through shared memory; each thread then
// slices four consecutive w of two lines
template <int BITS, int S>
__global__ void __launch_bounds__(256) slice_vcontig4(int64_t nv, int64_t nw, const double* __restrict__ M, int64_t ld,
                                                     const int32_t* __restrict__ expo, int bits, int s,
                                                     __nv_bfloat16* __restrict__ q, int64_t ldq, int64_t slice_stride) {
    __shared__ double tile[64][33];
    const int64_t v0 = int64_t(blockIdx.y) * 32, w0 = int64_t(blockIdx.x) * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int wl = ty + 8 * i;
        const int64_t v = v0 + tx, w = w0 + wl;
        tile[wl][tx] = (v < nv && w < nw) ? __ldcs(M + v + w * ld) : 0.0;
    }
    __syncthreads();
    const int wq = threadIdx.x & 15, vh = threadIdx.x >> 4;   // 16 x 16
    const int64_t w = w0 + 4 * wq;
    if (w >= ldq) return;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int vl = vh + 16 * r;
        const int64_t v = v0 + vl;
        if (v >= nv) continue;
        double x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = tile[4 * wq + c][vl];   // zero beyond nw (loaded as 0)
        slice_store4_any<BITS, S>(x, expo[v], bits, s, reinterpret_cast<uint16_t*>(q) + v * ldq + w, slice_stride);
    }
}

// ---------------------------------------------------------------------------
// Complex operands (Section 7: the method on complex data).  The complex product
// op(A) op(B) is the real product A' B'' of
//   A'  = [Re op(A), Im op(A)]                              m x 2k
//   B'' = [[Re op(B), Im op(B)], [-Im op(B), Re op(B)]]     2k x 2n
// whose first n columns are Re(op(A) op(B)) and last n are Im(op(A) op(B)).  Each
// line (row of op(A), column of op(B)) gets one exponent from the largest real or
// imaginary part; each entry is sliced once and its digits are written to the
// two (A') or four (B'') places it occupies, negated where B'' has -Im.
// ---------------------------------------------------------------------------

// complex lines, v contiguous (M(v, w) at v + w*ld): thread per v
__global__ void __launch_bounds__(256) zexpo_vcontig(int64_t nv, int64_t nw, const double2* __restrict__ M, int64_t ld,
                                                    int64_t w_per_split, int32_t* expo) {
    const int64_t v = int64_t(blockIdx.x) * 256 + threadIdx.x;
    if (v >= nv) return;
    const int64_t w0 = int64_t(blockIdx.y) * w_per_split;
    const int64_t w1 = min(nw, w0 + w_per_split);
    uint64_t m0 = 0, m1 = 0;
    int64_t w = w0;
    for (; w + 2 <= w1; w += 2) {
        const double2 a = M[v + w * ld], b = M[v + (w + 1) * ld];
        m0 = mag_max(m0, mag_max(mag_bits(a.x), mag_bits(a.y)));
        m1 = mag_max(m1, mag_max(mag_bits(b.x), mag_bits(b.y)));
    }
    for (; w < w1; ++w) {
        const double2 a = M[v + w * ld];
        m0 = mag_max(m0, mag_max(mag_bits(a.x), mag_bits(a.y)));
    }
    const int e = line_exponent_bits(mag_max(m0, m1));
    if (e != INT_MIN) atomicMax(&expo[v], e);
}

// complex lines, w contiguous (M(w, v) at w + v*ld): block per (v, w-chunk)
__global__ void __launch_bounds__(256) zexpo_wcontig(int64_t nv, int64_t nw, const double2* __restrict__ M, int64_t ld,
                                                    int64_t w_per_split, int32_t* expo) {
    const int64_t v = blockIdx.x;
    const int64_t w0 = int64_t(blockIdx.y) * w_per_split;
    const int64_t w1 = min(nw, w0 + w_per_split);
    uint64_t mx = 0;
    for (int64_t w = w0 + threadIdx.x; w < w1; w += 256) {
        const double2 a = M[w + v * ld];
        mx = mag_max(mx, mag_max(mag_bits(a.x), mag_bits(a.y)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = mag_max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    __shared__ uint64_t red[8];
    if (lane_id() == 0) red[warp_id()] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t m2 = red[0];
        for (int i = 1; i < 8; ++i) m2 = mag_max(m2, red[i]);
        const int e = line_exponent_bits(m2);
        if (e != INT_MIN) atomicMax(&expo[v], e);
    }
    (void)nv;
}

// The s digits of `valid` (<= 4) consecutive entries of one output line, negated if
// flip; one 8-byte store per slice when vec (and all four present), else 2-byte stores.
__device__ __forceinline__ void emit4(const Digits (&dg)[4], int valid, uint32_t flip, int bits, int s, uint16_t* out,
                                      int64_t slice_stride, bool vec) {
    for (int t = 1; t <= s; ++t) {
        uint32_t h[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
            h[c] = c < valid ? bf16_of_small_int(digit_bits(dg[c], bits, t), dg[c].neg ^ flip) : 0u;
        uint16_t* o = out + int64_t(t - 1) * slice_stride;
        if (vec && valid == 4) {
            uint2 pk;
            pk.x = h[0] | (h[1] << 16);
            pk.y = h[2] | (h[3] << 16);
            *reinterpret_cast<uint2*>(o) = pk;
        } else {
            for (int c = 0; c < valid; ++c) o[c] = uint16_t(h[c]);
        }
    }
}

// The compile-time form of emit4 (digits from one 64-bit word per value, see digits_word)
template <int BITS, int S>
__device__ __forceinline__ void emit4_fixed(const uint64_t (&F)[4], const uint32_t (&ng)[4], int valid, uint32_t flip,
                                            uint16_t* out, int64_t slice_stride, bool vec) {
    constexpr uint32_t MASK = (1u << BITS) - 1u;
    uint32_t sg[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) sg[c] = c < valid ? ((ng[c] ^ flip) << 31) : 0u;
    const uint64_t b01 = (uint64_t(0x4B000000u | sg[1]) << 32) | (0x4B000000u | sg[0]);
    const uint64_t b23 = (uint64_t(0x4B000000u | sg[3]) << 32) | (0x4B000000u | sg[2]);
#pragma unroll
    for (int t = 1; t <= S; ++t) {
        uint32_t d[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) d[c] = c < valid ? uint32_t(F[c] >> (BITS * (S - t))) & MASK : 0u;
        const uint32_t w01 = bf16x2_of_digits(d[0], d[1], b01), w23 = bf16x2_of_digits(d[2], d[3], b23);
        uint16_t* o = out + int64_t(t - 1) * slice_stride;
        if (vec && valid == 4) {
            *reinterpret_cast<uint2*>(o) = make_uint2(w01, w23);
        } else {
            const uint32_t h[4] = {w01 & 0xFFFFu, w01 >> 16, w23 & 0xFFFFu, w23 >> 16};
            for (int c = 0; c < valid; ++c) o[c] = uint16_t(h[c]);
        }
    }
}

// Digits of entries w..w+valid-1 of line v (values x, conjugated if conj) into the real form.
// role_b = false: A' (line v: Re at w, Im at nw + w).  role_b = true: B'' (line v = j < n:
// Re at w, -Im at nw + w; line n + j: Im at w, Re at nw + w).
template <int BITS, int S>
__device__ __forceinline__ void zslice_emit(const double2 (&x)[4], int valid, int e, bool conj, bool role_b,
                                            int64_t v, int64_t nv, int64_t nw, int64_t w, int bits, int s,
                                            uint16_t* q, int64_t ldq, int64_t slice_stride, bool vec) {
    if constexpr (BITS > 0) {
        uint64_t Fr[4], Fi[4];
        uint32_t nr[4], ni[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Fr[c] = digits_word<BITS, S>(x[c].x, e, nr[c]);
            Fi[c] = digits_word<BITS, S>(conj ? -x[c].y : x[c].y, e, ni[c]);
        }
        uint16_t* row = q + v * ldq;
        emit4_fixed<BITS, S>(Fr, nr, valid, 0u, row + w, slice_stride, vec);
        emit4_fixed<BITS, S>(Fi, ni, valid, role_b ? 1u : 0u, row + nw + w, slice_stride, vec);
        if (role_b) {
            uint16_t* row2 = q + (nv + v) * ldq;
            emit4_fixed<BITS, S>(Fi, ni, valid, 0u, row2 + w, slice_stride, vec);
            emit4_fixed<BITS, S>(Fr, nr, valid, 0u, row2 + nw + w, slice_stride, vec);
        }
    } else {
        Digits dr[4], di[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            dr[c] = prepare_digits(x[c].x, e);
            di[c] = prepare_digits(conj ? -x[c].y : x[c].y, e);
        }
        uint16_t* row = q + v * ldq;
        emit4(dr, valid, 0u, bits, s, row + w, slice_stride, vec);
        emit4(di, valid, role_b ? 1u : 0u, bits, s, row + nw + w, slice_stride, vec);
        if (role_b) {
            uint16_t* row2 = q + (nv + v) * ldq;
            emit4(di, valid, 0u, bits, s, row2 + w, slice_stride, vec);
            emit4(dr, valid, 0u, bits, s, row2 + nw + w, slice_stride, vec);
        }
    }
}

// w contiguous: four consecutive w of one line per thread
template <int BITS, int S>
__global__ void __launch_bounds__(256) zslice_wcontig(int64_t nv, int64_t nw, const double2* __restrict__ M, int64_t ld,
                                                     const int32_t* __restrict__ expo, bool conj, bool role_b, int bits,
                                                     int s, __nv_bfloat16* __restrict__ q, int64_t ldq,
                                                     int64_t slice_stride, bool vec) {
    const int64_t v = blockIdx.y;
    const int64_t w = (int64_t(blockIdx.x) * 256 + threadIdx.x) * 4;
    if (w >= nw) return;
    const int valid = nw - w < 4 ? int(nw - w) : 4;
    double2 x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = c < valid ? M[w + c + v * ld] : make_double2(0.0, 0.0);
    zslice_emit<BITS, S>(x, valid, expo[v], conj, role_b, v, nv, nw, w, bits, s, reinterpret_cast<uint16_t*>(q),
                         ldq, slice_stride, vec);
}

// v contiguous: 64 (w) x 32 (v) complex tiles transposed through shared memory
template <int BITS, int S>
__global__ void __launch_bounds__(256) zslice_vcontig(int64_t nv, int64_t nw, const double2* __restrict__ M, int64_t ld,
                                                     const int32_t* __restrict__ expo, bool conj, bool role_b, int bits,
                                                     int s, __nv_bfloat16* __restrict__ q, int64_t ldq,
                                                     int64_t slice_stride, bool vec) {
    __shared__ double2 tile[64][33];
    const int64_t v0 = int64_t(blockIdx.y) * 32, w0 = int64_t(blockIdx.x) * 64;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int wl = ty + 8 * i;
        const int64_t v = v0 + tx, w = w0 + wl;
        tile[wl][tx] = (v < nv && w < nw) ? M[v + w * ld] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int wq = threadIdx.x & 15, vh = threadIdx.x >> 4;
    const int64_t w = w0 + 4 * wq;
    if (w >= nw) return;
    const int valid = nw - w < 4 ? int(nw - w) : 4;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int vl = vh + 16 * r;
        const int64_t v = v0 + vl;
        if (v >= nv) continue;
        double2 x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = tile[4 * wq + c][vl];
        zslice_emit<BITS, S>(x, valid, expo[v], conj, role_b, v, nv, nw, w, bits, s, reinterpret_cast<uint16_t*>(q),
                             ldq, slice_stride, vec);
    }
}

// zero the padding [from, ldq) of every line of every slice
__global__ void zpad_kernel(int64_t lines, int64_t from, int64_t ldq, int s, __nv_bfloat16* __restrict__ q,
                            int64_t slice_stride) {
    const int64_t line = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (line >= lines) return;
    uint16_t* o = reinterpret_cast<uint16_t*>(q) + line * ldq;
    for (int t = 0; t < s; ++t)
        for (int64_t w = from; w < ldq; ++w) o[int64_t(t) * slice_stride + w] = 0;
}

}  // namespace

namespace {

// G 2^P as a double for an integer |G| < 2^53 (so double(G) is exact), built from
// integer operations: the exponent field takes P directly, no FP64 arithmetic.
// Results outside the normal range go through ldexp (exact or correctly rounded).
__device__ __forceinline__ double scaled_int(int64_t G, int P) {
    if (G == 0) return 0.0;
    const uint64_t neg = G < 0 ? 1u : 0u;
    const uint64_t mag = uint64_t(G < 0 ? -G : G);
    const int top = 63 - __clzll(int64_t(mag));                       // 0..52
    const int ef = top + P + 1023;
    if (ef < 1 || ef > 2046) return ldexp(double(G), P);
    const uint64_t mant = (mag << (52 - top)) & ((uint64_t(1) << 52) - 1);
    return __longlong_as_double(int64_t((neg << 63) | (uint64_t(ef) << 52) | mant));
}

// C_ij = alpha 2^(e_i + f_j) sum_{d=2}^{s+1} 2^(-bits d) S_d(i,j) + beta C_ij.
// Consecutive anti-diagonals are first combined exactly in INT64,
//   G = sum_{d=dl}^{dh} S_d 2^(bits (dh - d)),  |G| < 2^(31 + bits (g-1) + 1) <= 2^53,
// so G 2^(e_i + f_j - bits dh) is an exact double and each group costs one FP64
// addition (smallest group first).
__global__ void __launch_bounds__(256) ozaki_recombine_kernel(int64_t m, int64_t n, int s, int bits, int gsize,
                                                             const int32_t* __restrict__ sd, int64_t plane,
                                                             const int32_t* __restrict__ ea,
                                                             const int32_t* __restrict__ eb, double alpha, double beta,
                                                             double* __restrict__ C, int64_t ldc) {
    const int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x;
    if (i >= m) return;
    const int ei = ea[i];
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const int32_t* p = sd + i + j * m;
        const int E0 = ei + eb[j];
        double acc = 0.0;
        for (int dh = s + 1; dh >= 2; dh -= gsize) {
            const int dl = dh - gsize + 1 > 2 ? dh - gsize + 1 : 2;
            int64_t G = 0;
            for (int d = dl; d <= dh; ++d) G = G * (int64_t(1) << bits) + int64_t(__ldcs(p + int64_t(d - 2) * plane));
            const double gv = scaled_int(G, E0 - bits * dh);
            acc = (dh == s + 1) ? gv : acc + gv;      // the first group needs no FP64 addition
        }
        double v = (alpha == 1.0) ? acc : alpha * acc;
        if (beta != 0.0) v = fma(beta, C[i + j * ldc], v);
        C[i + j * ldc] = v;
    }
}

// The same for four consecutive rows per thread: 16-byte loads of every S_d plane and
// 16-byte stores of C (m, the plane pitch and ldc suitably aligned; checked by the host).
// FIXED77: s = 7 slices of 7 bits (groups d = 5..8 and d = 2..4), all seven planes loaded
// before any arithmetic, the same operations in the same order as the general loop.
__device__ __forceinline__ int lane_of(const int4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
template <bool FIXED77>
__global__ void __launch_bounds__(256) ozaki_recombine4_kernel(int64_t m, int64_t n, int s, int bits, int gsize,
                                                              const int32_t* __restrict__ sd, int64_t plane,
                                                              const int32_t* __restrict__ ea,
                                                              const int32_t* __restrict__ eb, double alpha,
                                                              double beta, double* __restrict__ C, int64_t ldc) {
    const int64_t i = (int64_t(blockIdx.x) * 256 + threadIdx.x) * 4;
    if (i >= m) return;
    const int4 ei = *reinterpret_cast<const int4*>(ea + i);
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const int32_t* p = sd + i + j * m;
        const int fj = eb[j];
        const int E0[4] = {ei.x + fj, ei.y + fj, ei.z + fj, ei.w + fj};
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        if constexpr (FIXED77) {
            int4 v[7];
#pragma unroll
            for (int d = 2; d <= 8; ++d) v[d - 2] = __ldcs(reinterpret_cast<const int4*>(p + int64_t(d - 2) * plane));
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int64_t G1 = 0, G2 = 0;
#pragma unroll
                for (int d = 5; d <= 8; ++d) G1 = G1 * 128 + int64_t(lane_of(v[d - 2], c));
#pragma unroll
                for (int d = 2; d <= 4; ++d) G2 = G2 * 128 + int64_t(lane_of(v[d - 2], c));
                acc[c] = scaled_int(G1, E0[c] - 7 * 8) + scaled_int(G2, E0[c] - 7 * 4);
            }
        } else {
        for (int dh = s + 1; dh >= 2; dh -= gsize) {
            const int dl = dh - gsize + 1 > 2 ? dh - gsize + 1 : 2;
            int64_t G[4] = {0, 0, 0, 0};
            for (int d = dl; d <= dh; ++d) {
                const int4 v = __ldcs(reinterpret_cast<const int4*>(p + int64_t(d - 2) * plane));
                G[0] = G[0] * (int64_t(1) << bits) + int64_t(v.x);
                G[1] = G[1] * (int64_t(1) << bits) + int64_t(v.y);
                G[2] = G[2] * (int64_t(1) << bits) + int64_t(v.z);
                G[3] = G[3] * (int64_t(1) << bits) + int64_t(v.w);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double gv = scaled_int(G[c], E0[c] - bits * dh);
                acc[c] = (dh == s + 1) ? gv : acc[c] + gv;   // the first group needs no FP64 addition
            }
        }
        }
        double* cp = C + i + j * ldc;
        double v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (alpha == 1.0) ? acc[c] : alpha * acc[c];
        if (beta != 0.0) {
            const double2 c0 = reinterpret_cast<const double2*>(cp)[0], c1 = reinterpret_cast<const double2*>(cp)[1];
            v[0] = fma(beta, c0.x, v[0]); v[1] = fma(beta, c0.y, v[1]);
            v[2] = fma(beta, c1.x, v[2]); v[3] = fma(beta, c1.y, v[3]);
        }
        reinterpret_cast<double2*>(cp)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(cp)[1] = make_double2(v[2], v[3]);
    }
}

// Complex result: Re and Im of op(A) op(B) are columns j and n + j of the real form's
// S_d; C = alpha (Re + i Im) + beta C, alpha and beta complex.
__global__ void __launch_bounds__(256) ozaki_zrecombine_kernel(int64_t m, int64_t n, int s, int bits, int gsize,
                                                              const int32_t* __restrict__ sd, int64_t plane,
                                                              const int32_t* __restrict__ ea,
                                                              const int32_t* __restrict__ eb, double2 alpha,
                                                              double2 beta, double2* __restrict__ C, int64_t ldc) {
    const int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x;
    if (i >= m) return;
    const int ei = ea[i];
    const int64_t m2 = m;   // plane row pitch: S_d is [d-2][column of the real form][i]
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const int32_t* pr = sd + i + j * m2;
        const int32_t* pi = sd + i + (n + j) * m2;
        const int E0 = ei + eb[j];
        double re = 0.0, im = 0.0;
        for (int dh = s + 1; dh >= 2; dh -= gsize) {
            const int dl = dh - gsize + 1 > 2 ? dh - gsize + 1 : 2;
            int64_t Gr = 0, Gi = 0;
            for (int d = dl; d <= dh; ++d) {
                Gr = Gr * (int64_t(1) << bits) + int64_t(__ldcs(pr + int64_t(d - 2) * plane));
                Gi = Gi * (int64_t(1) << bits) + int64_t(__ldcs(pi + int64_t(d - 2) * plane));
            }
            const double gr = scaled_int(Gr, E0 - bits * dh), gi = scaled_int(Gi, E0 - bits * dh);
            re = (dh == s + 1) ? gr : re + gr;      // the first group needs no FP64 addition
            im = (dh == s + 1) ? gi : im + gi;
        }
        double vr = alpha.x * re - alpha.y * im;
        double vi = alpha.x * im + alpha.y * re;
        if (beta.x != 0.0 || beta.y != 0.0) {
            const double2 c = C[i + j * ldc];
            vr = fma(beta.x, c.x, fma(-beta.y, c.y, vr));
            vi = fma(beta.x, c.y, fma(beta.y, c.x, vi));
        }
        C[i + j * ldc] = make_double2(vr, vi);
    }
}

}  // namespace

hsmm_status_t ozaki_recombine(int64_t m, int64_t n, int slices, int bits, const int32_t* sd, int64_t sd_plane,
                              const int32_t* ea, const int32_t* eb, double alpha, double beta, double* C, int64_t ldc,
                              cudaStream_t st) {
    const int gsize = 1 + 21 / bits;
    const unsigned gy = unsigned(n < 65535 ? n : 65535);
    const bool vec4 = m % 4 == 0 && sd_plane % 4 == 0 && ldc % 2 == 0 && aligned_to(sd, 16) && aligned_to(ea, 16) &&
                      aligned_to(C, 16);
    if (vec4 && slices == 7 && bits == 7)
        ozaki_recombine4_kernel<true><<<dim3(unsigned((m / 4 + 255) / 256), gy), 256, 0, st>>>(
            m, n, slices, bits, gsize, sd, sd_plane, ea, eb, alpha, beta, C, ldc);
    else if (vec4)
        ozaki_recombine4_kernel<false><<<dim3(unsigned((m / 4 + 255) / 256), gy), 256, 0, st>>>(
            m, n, slices, bits, gsize, sd, sd_plane, ea, eb, alpha, beta, C, ldc);
    else
        ozaki_recombine_kernel<<<dim3(unsigned((m + 255) / 256), gy), 256, 0, st>>>(m, n, slices, bits, gsize, sd,
                                                                                   sd_plane, ea, eb, alpha, beta, C,
                                                                                   ldc);
    count_launches(1);
    return check_launch();
}

// rows x cols column-major M; by_rows: v = row (w = column), else v = column (w = row).
hsmm_status_t ozaki_split(int64_t rows, int64_t cols, const double* M, int64_t ld, bool by_rows, int bits,
                          int slices, int32_t* expo, void* qv, int64_t ldq, int64_t plane, cudaStream_t st) {
    const int64_t nv = by_rows ? rows : cols;
    const int64_t nw = by_rows ? cols : rows;
    __nv_bfloat16* q = static_cast<__nv_bfloat16*>(qv);
    if (nv > 65535 * 32LL && by_rows) return HSMM_STATUS_NOT_SUPPORTED;
    if (nv > 65535 && !by_rows) return HSMM_STATUS_NOT_SUPPORTED;
    expo_init<<<unsigned((nv + 255) / 256), 256, 0, st>>>(nv, expo);
    const int sms = num_sms();
    // four digits per 8-byte store when every slice row starts 8-byte aligned; the default
    // 7 slices of 7 bits with compile-time digit positions
    const bool q8 = ldq % 4 == 0 && plane % 4 == 0 && aligned_to(qv, 8);
    const bool fixed77 = bits == 7 && slices == 7;
    if (by_rows) {
        // v = row: contiguous
        const int64_t vb = (nv + 255) / 256;
        int64_t splits = (int64_t(sms) * 8 + vb - 1) / vb;
        splits = splits < 1 ? 1 : (splits > nw ? nw : splits);
        const int64_t wps = (nw + splits - 1) / splits;
        if (nv % 2 == 0 && ld % 2 == 0 && aligned_to(M, 16))
            expo_vcontig2<<<dim3(unsigned((nv / 2 + 255) / 256), unsigned((nw + wps - 1) / wps)), 256, 0, st>>>(
                nv, nw, M, ld, wps, expo);
        else
            expo_vcontig<<<dim3(unsigned(vb), unsigned((nw + wps - 1) / wps)), 256, 0, st>>>(nv, nw, M, ld, wps, expo);
        if (q8 && fixed77)
            slice_vcontig4<7, 7><<<dim3(unsigned((ldq + 63) / 64), unsigned((nv + 31) / 32)), 256, 0, st>>>(
                nv, nw, M, ld, expo, bits, slices, q, ldq, plane);
        else if (q8)
            slice_vcontig4<0, 0><<<dim3(unsigned((ldq + 63) / 64), unsigned((nv + 31) / 32)), 256, 0, st>>>(
                nv, nw, M, ld, expo, bits, slices, q, ldq, plane);
        else
            slice_vcontig<<<dim3(unsigned((ldq + 31) / 32), unsigned((nv + 31) / 32)), 256, 0, st>>>(
                nv, nw, M, ld, expo, bits, slices, q, ldq, plane);
    } else {
        int64_t splits = (int64_t(sms) * 8 + nv - 1) / nv;
        const int64_t maxs = (nw + 2047) / 2048;
        splits = splits < 1 ? 1 : (splits > maxs ? maxs : splits);
        const int64_t wps = (nw + splits - 1) / splits;
        expo_wcontig<<<dim3(unsigned(nv), unsigned((nw + wps - 1) / wps)), 256, 0, st>>>(nv, nw, M, ld, wps, expo);
        if (q8 && ld % 2 == 0 && aligned_to(M, 16) && fixed77)
            slice_wcontig4<7, 7><<<dim3(unsigned((ldq + 1023) / 1024), unsigned(nv)), 256, 0, st>>>(
                nv, nw, M, ld, expo, bits, slices, q, ldq, plane);
        else if (q8 && ld % 2 == 0 && aligned_to(M, 16))
            slice_wcontig4<0, 0><<<dim3(unsigned((ldq + 1023) / 1024), unsigned(nv)), 256, 0, st>>>(
                nv, nw, M, ld, expo, bits, slices, q, ldq, plane);
        else
            slice_wcontig<<<dim3(unsigned((ldq + 255) / 256), unsigned(nv)), 256, 0, st>>>(nv, nw, M, ld, expo, bits,
                                                                                           slices, q, ldq, plane);
    }
    expo_fix<<<unsigned((nv + 255) / 256), 256, 0, st>>>(nv, expo);
    count_launches(4);
    return check_launch();
}


hsmm_status_t ozaki_zrecombine(int64_t m, int64_t n, int slices, int bits, const int32_t* sd, int64_t sd_plane,
                               const int32_t* ea, const int32_t* eb, const double* alpha, const double* beta, void* C,
                               int64_t ldc, cudaStream_t st) {
    const int gsize = 1 + 21 / bits;
    const unsigned gy = unsigned(n < 65535 ? n : 65535);
    ozaki_zrecombine_kernel<<<dim3(unsigned((m + 255) / 256), gy), 256, 0, st>>>(
        m, n, slices, bits, gsize, sd, sd_plane, ea, eb, make_double2(alpha[0], alpha[1]),
        make_double2(beta[0], beta[1]), static_cast<double2*>(C), ldc);
    count_launches(1);
    return check_launch();
}

// Complex operand into the real form (A' for role_b = false, B'' for role_b = true).
// Lines v (rows of op(A) / columns of op(B)), nv of them, each of nw complex entries;
// v_contig: entry (v, w) at M[v + w*ld], else at M[w + v*ld]; conj: op = C.
hsmm_status_t ozaki_zsplit(int64_t nv, int64_t nw, const void* Mv, int64_t ld, bool v_contig, bool conj, bool role_b,
                           int bits, int slices, int32_t* expo, void* qv, int64_t ldq, int64_t plane, cudaStream_t st) {
    const double2* M = static_cast<const double2*>(Mv);
    __nv_bfloat16* q = static_cast<__nv_bfloat16*>(qv);
    if (v_contig && nv > 65535 * 32LL) return HSMM_STATUS_NOT_SUPPORTED;
    if (!v_contig && nv > 65535) return HSMM_STATUS_NOT_SUPPORTED;
    expo_init<<<unsigned((nv + 255) / 256), 256, 0, st>>>(nv, expo);
    const int sms = num_sms();
    const bool vec = ldq % 4 == 0 && plane % 4 == 0 && nw % 4 == 0 && aligned_to(qv, 8);
    const bool fixed77 = bits == 7 && slices == 7;
    if (v_contig) {
        const int64_t vb = (nv + 255) / 256;
        int64_t splits = (int64_t(sms) * 8 + vb - 1) / vb;
        splits = splits < 1 ? 1 : (splits > nw ? nw : splits);
        const int64_t wps = (nw + splits - 1) / splits;
        zexpo_vcontig<<<dim3(unsigned(vb), unsigned((nw + wps - 1) / wps)), 256, 0, st>>>(nv, nw, M, ld, wps, expo);
        const dim3 grid(unsigned((nw + 63) / 64), unsigned((nv + 31) / 32));
        if (fixed77)
            zslice_vcontig<7, 7><<<grid, 256, 0, st>>>(nv, nw, M, ld, expo, conj, role_b, bits, slices, q, ldq, plane,
                                                       vec);
        else
            zslice_vcontig<0, 0><<<grid, 256, 0, st>>>(nv, nw, M, ld, expo, conj, role_b, bits, slices, q, ldq, plane,
                                                       vec);
    } else {
        int64_t splits = (int64_t(sms) * 8 + nv - 1) / nv;
        const int64_t maxs = (nw + 2047) / 2048;
        splits = splits < 1 ? 1 : (splits > maxs ? maxs : splits);
        const int64_t wps = (nw + splits - 1) / splits;
        zexpo_wcontig<<<dim3(unsigned(nv), unsigned((nw + wps - 1) / wps)), 256, 0, st>>>(nv, nw, M, ld, wps, expo);
        const dim3 grid(unsigned((nw + 1023) / 1024), unsigned(nv));
        if (fixed77)
            zslice_wcontig<7, 7><<<grid, 256, 0, st>>>(nv, nw, M, ld, expo, conj, role_b, bits, slices, q, ldq, plane,
                                                       vec);
        else
            zslice_wcontig<0, 0><<<grid, 256, 0, st>>>(nv, nw, M, ld, expo, conj, role_b, bits, slices, q, ldq, plane,
                                                       vec);
    }
    const int64_t lines = role_b ? 2 * nv : nv;
    int launches = 4;
    if (2 * nw < ldq) {
        zpad_kernel<<<unsigned((lines + 255) / 256), 256, 0, st>>>(lines, 2 * nw, ldq, slices, q, plane);
        ++launches;
    }
    expo_fix<<<unsigned((nv + 255) / 256), 256, 0, st>>>(nv, expo);
    count_launches(launches);
    return check_launch();
}

}  // namespace hsmm
