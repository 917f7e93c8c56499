"""Pins of the oracle's simulation of the paper's ring algorithms (CPU only).

Algorithm 1 (systolic) and Algorithm 2 (hyper-systolic) over p virtual
processors are checked bit for bit against brute force on integer matrices, and
their bookkeeping against the closed forms the paper states.
"""
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def divisors(p):
    return [K for K in range(1, p + 1) if p % K == 0]


def int_pair(n, seed, lo=-8, hi=8):
    return (W.integers((n, n), seed, lo, hi, np.float64), W.integers((n, n), seed + 1, lo, hi, np.float64))


@pytest.mark.parametrize("p", list(range(1, 17)))
def test_hsmm_bitexact_all_K(ora, p):
    b = 2
    A, B = int_pair(p * b, 100 + p)
    exact = ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
    for K in divisors(p):
        C, st, cnt = ora.ring_hsmm(A, B, p, K, with_counts=True)
        assert np.array_equal(C, exact), (p, K)
        assert st["pairing_errors"] == 0
        # every block product A_rk (x) B_kq lands in C_rq exactly once
        assert (cnt == 1).all(), (p, K)
        assert st["a_final_ok"] == 1


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 16])
def test_systolic_bitexact(ora, p):
    A, B = int_pair(p * 3, 200 + p)
    C, st, cnt = ora.ring_systolic(A, B, p, with_counts=True)
    assert np.array_equal(C, ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64))
    assert (cnt == 1).all() and st["pairing_errors"] == 0
    assert st["a_final_ok"] == 1          # p unit shifts bring A back


def test_workload_ring_integer_512(ora):
    # the n = 512, p = 16, 32 x 32 block workload, integer-valued: exact
    A, B = W.ring_inputs(integer=True)
    C, st = ora.ring_hsmm(A, B, 16, 4)
    assert np.array_equal(C, ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64))
    assert st["shift_events"] == 7


def test_workload_ring_fp64_gamma(ora):
    # FP64 uniform(-1,1), n = 512: the ring order differs from the triple loop only by
    # rounding, bounded elementwise by gamma_n (|A||B|)_ij
    A, B = W.ring_inputs(n=128)
    C, _ = ora.ring_hsmm(A, B, 16, 4)
    ref = ora.gemm(A, B)
    u = 2.0 ** -53
    n = 128
    gam = n * u / (1 - n * u)
    bound = 2 * gam * ora.gemm(np.abs(A), np.abs(B))
    assert (np.abs(C - ref) <= bound).all()


def test_k1_equals_systolic_bitwise(ora):
    # K = 1: no pre-shift, one aux array, no back-shift -> Algorithm 1, same sums in same order
    A, B = W.ring_inputs(n=64)
    C1, st1 = ora.ring_hsmm(A, B, 8, 1)
    C0, _ = ora.ring_systolic(A, B, 8)
    assert np.array_equal(C1, C0)
    assert st1["b_rows_shifted"] == 0 and st1["c_shifts"] == 0 and st1["a_shifts"] == 7


def test_planted_nonnegative_modulus_fails(ora):
    # the non-negative reading of MOD(1-j, K) gives a wrong product for 1 < K < p
    for p, K in [(4, 2), (16, 4), (16, 2), (12, 3), (16, 8)]:
        A, B = int_pair(p * 2, 300 + p + K)
        C, st = ora.ring_hsmm(A, B, p, K, planted_nonneg_mod=True)
        exact = ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
        assert not np.array_equal(C, exact)
        assert st["pairing_errors"] > 0


def test_shift_counts_closed_forms(ora):
    rows = [list(map(int, ln.split())) for ln in open(os.path.join(GOLDEN, "shift_complexity.txt"))
            if ln.strip() and not ln.startswith("#")]
    for p, K, t_hyper, t_sys, rnum, rden in rows:
        A, B = int_pair(p, 400 + p)
        _, st = ora.ring_hsmm(A, B, p, K)
        assert st["shift_events"] == t_hyper == K + p // K - 1
        assert st["b_preshift_events"] == 1 and st["a_shifts"] == p // K - 1 and st["c_shifts"] == K - 1
        _, s1 = ora.ring_hsmm(A, B, p, 1)
        assert s1["shift_events"] == t_sys == p - 1
        assert (p - 1) * rden == rnum * st["shift_events"]


def test_worked_example_p4(ora):
    facts = {}
    for ln in open(os.path.join(GOLDEN, "worked_example_p4.txt")):
        if ln.strip() and not ln.startswith("#"):
            key, *vals = ln.split()
            facts[key] = list(map(int, vals))
    p, K = 4, 2
    assert [abs(ora.preshift_stride(j, K)) for j in range(1, p + 1)] == facts["preshift_abs"]
    A, B = int_pair(p, 500)
    _, st = ora.ring_hsmm(A, B, p, K)
    assert st["a_shifts"] == facts["a_shift_events"][0]
    assert st["c_shifts"] == facts["c_shift_events"][0]
    base = ora.regular_base(p, K)
    assert base["A"][1:] == facts["a_shift_stride"] * (p // K - 1)
    assert base["C"][1:] == facts["c_shift_stride"] * (K - 1)
    assert len(base["C"]) == facts["aux_arrays"][0]
    assert [ora.skew_row(p, i, 0) + 1 for i in range(p)] == facts["slot1_rows"]


def test_preshift_volume(ora):
    # B moves (K-1)/K of its rows once (Section 5.2.2: blocks of K rows, strides 0..K-1)
    for p, K in [(16, 4), (12, 3), (8, 2)]:
        A, B = int_pair(p, 600 + p)
        _, st = ora.ring_hsmm(A, B, p, K)
        assert st["b_rows_shifted"] * K == p * (K - 1)
        assert [-ora.preshift_stride(j, K) for j in range(1, K + 1)] == list(range(K))


def covers(p, A, B):
    """h-range check of Definition OPTI2: every m in [0, p) as a partial sum of A plus one of B."""
    def partial_sums(base):
        out = {0}
        for i in range(len(base)):
            for j in range(i, len(base)):
                out.add(sum(base[i:j + 1]))
        return out
    sa, sb = partial_sums(A), partial_sums(B)
    return all(any((m - x) in sb for x in sa) for m in range(p))


@pytest.mark.parametrize("p", [4, 6, 9, 12, 16, 25, 36, 64])
def test_regular_base_h_range(ora, p):
    for K in divisors(p):
        base = ora.regular_base(p, K)
        # two-array regular bases (Definition REGULARBASE2): h-range = p (Theorem, Section 4.4)
        assert covers(p, base["A2"], base["B2"])
        # matrix-product bases (Section 5.2.1): the offsets l0 + jb*K that Algorithm 2 visits,
        # formed from partial sums of -B (within a block) and A (between blocks), hit every
        # ring distance in [0, p) exactly once
        offs = sorted(-sum(base["B"][:l + 1]) + sum(base["A"][:jb + 1]) for l in range(K) for jb in range(p // K))
        assert offs == list(range(p))


def test_optimal_regular_base_length():
    # Section 4.4: the length K + p/K - 1 is minimal at K = sqrt(p); T of Eq. COMPLEXR and the
    # lower bound 3(sqrt(n) - 1) of Theorem MINIMUM2 coincide there
    for p in [4, 16, 64, 256]:
        best = min(divisors(p), key=lambda K: K + p // K - 1)
        assert best == math.isqrt(p)
        K = math.isqrt(p)
        assert 2 * K + p // K - 3 == 3 * (K - 1)
