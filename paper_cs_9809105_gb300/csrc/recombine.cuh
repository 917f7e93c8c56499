// recombine.cuh -- the recombination step of the FP64-accurate product for one entry of C,
// shared by the recombination kernels (ozaki.cu) and the slice-product kernel that folds
// it into its epilogue for whole tiles (gemm_tc.cu), so that both give the same bits.
//
// With per-row exponents e_i of op(A), per-column exponents f_j of op(B) and the exact
// anti-diagonal sums S_d (d = 2..s+1) of the b-bit slice products,
//   C_ij = alpha 2^(e_i + f_j) sum_d 2^(-b d) S_d(i,j) + beta C_ij
// (Ozaki et al., error-free transformation of the product: the split is a sum of exact
// slices, and every slice product is exact in integer arithmetic).
#pragma once

#include <cstdint>

namespace hsmm {

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

// sum_d 2^(E0 - 7d) S_d for the default form (s = 7 slices of b = 7 bits), v[d-2] = S_d,
// d = 2..8.  The anti-diagonals are combined exactly in INT64 in two groups,
//   G1 = S_5 2^21 + S_6 2^14 + S_7 2^7 + S_8,   G2 = S_2 2^14 + S_3 2^7 + S_4,
// |G| < 2^(31 + 21 + 1) = 2^53, so each G 2^(E0 - 7 dh) (dh the group's largest d) is an
// exact double, and the sum costs one FP64 addition, the smaller group first.
__device__ __forceinline__ double recombine77(const int32_t (&v)[7], int E0) {
    int64_t G1 = 0, G2 = 0;
#pragma unroll
    for (int d = 5; d <= 8; ++d) G1 = G1 * 128 + int64_t(v[d - 2]);
#pragma unroll
    for (int d = 2; d <= 4; ++d) G2 = G2 * 128 + int64_t(v[d - 2]);
    return scaled_int(G1, E0 - 7 * 8) + scaled_int(G2, E0 - 7 * 4);
}

// alpha acc + beta c (c not read when beta = 0, so a NaN in C does not propagate)
__device__ __forceinline__ double blas_update(double acc, double alpha, double beta, const double* c) {
    const double v = (alpha == 1.0) ? acc : alpha * acc;
    return beta != 0.0 ? fma(beta, *c, v) : v;
}

}  // namespace hsmm
