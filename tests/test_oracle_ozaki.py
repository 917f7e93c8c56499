"""Pins of the oracle's FP64-accurate product by error-free splitting (CPU only).

Checked against exact rational arithmetic (the splitting), the exact integer
product (integer inputs with enough slices), and the truncation error bound of
the splitting against the Dot2 reference.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("beta,s", [(5, 10), (6, 8), (7, 7)])
@pytest.mark.parametrize("by_rows", [True, False])
def test_split_exact_truncation(ora, beta, s, by_rows):
    M = W.scaled_f64((6, 9), 31)
    M[2, :] = 0.0                      # a zero row
    M[:, 3] = 0.0                      # a zero column
    expo, sl = ora.ozaki_split(M, by_rows, beta, s)
    for r in range(M.shape[0]):
        for c in range(M.shape[1]):
            v = (r if by_rows else c)
            e = int(expo[v])
            line = M[r, :] if by_rows else M[:, c]
            mx = max(abs(x) for x in line)
            if mx == 0:
                assert e == 0
            else:
                # e is the smallest integer with max |m| < 2^e
                assert mx < 2.0 ** e and mx >= 2.0 ** (e - 1)
            q = [sl[t, r, c] for t in range(s)]
            assert all(float(x).is_integer() and abs(x) <= 2 ** beta - 1 for x in q)
            x = Fraction(M[r, c]) / Fraction(2) ** e
            head = sum(Fraction(int(q[t])) / Fraction(2) ** (beta * (t + 1)) for t in range(s))
            rest = x - head
            # truncation toward zero: the rest is below one unit of the last slice, same sign as x
            assert abs(rest) < Fraction(1, 2 ** (beta * s))
            assert rest == 0 or (rest > 0) == (x > 0)


def test_split_exact_with_enough_slices(ora):
    # 53-bit significands within a row spanning 2^24: beta*s >= 24 + 53 + 1 bits reproduces them exactly
    M = W.scaled_f64((4, 16), 32)
    beta, s = 7, 12
    expo, sl = ora.ozaki_split(M, True, beta, s)
    for r in range(4):
        for c in range(16):
            rec = sum(Fraction(int(sl[t, r, c])) / Fraction(2) ** (beta * (t + 1)) for t in range(s))
            assert rec * Fraction(2) ** int(expo[r]) == Fraction(M[r, c])


def test_ozaki_integer_inputs_exact(ora):
    # integer inputs: with enough slices every product term is kept, so the result is the exact product
    g = W.rng(33)
    A = np.asfortranarray(g.integers(-1000, 1001, size=(9, 40)).astype(np.float64))
    B = np.asfortranarray(g.integers(-1000, 1001, size=(40, 7)).astype(np.float64))
    exact = ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64)
    got = ora.ozaki_gemm(A, B, beta_bits=6, s=4)      # 24 bits per operand > 11 bits used
    assert np.array_equal(got, exact)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_ozaki_transposed_forms(ora, ta, tb):
    A = W.scaled_f64((24, 32) if ta == "N" else (32, 24), 34)
    B = W.scaled_f64((32, 16) if tb == "N" else (16, 32), 35)
    Ao = A if ta == "N" else np.asfortranarray(A.T)
    Bo = B if tb == "N" else np.asfortranarray(B.T)
    assert np.array_equal(ora.ozaki_gemm(A, B, ta, tb), ora.ozaki_gemm(Ao, Bo))


@pytest.mark.parametrize("beta,s", [(5, 6), (6, 5), (7, 4), (7, 7), (6, 9)])
def test_ozaki_error_bound_vs_dot2(ora, beta, s):
    """Error of the truncated splitting, elementwise against the accurate product.

    With |q| < 2^beta per slice, the dropped remainder of each operand is below
    2^(e - beta*s) and the dropped pairs (t+u > s+1) sum to at most
    (s-1) 2^(-beta*s) (1 + 2^-beta)/(1 - 2^-beta) in the scaled units, so
      |C - AB|_ij <= 2^(e_i + f_j) k 2^(-beta*s) (s + 3)  (+ FP64 recombination)
    """
    m = n = 24
    k = 64
    A = W.scaled_f64((m, k), 36)
    B = W.scaled_f64((k, n), 37)
    got = ora.ozaki_gemm(A, B, beta_bits=beta, s=s)
    ref = ora.gemm_rows(A, B, list(range(m)), accurate=True)
    ea = np.array([math.frexp(np.abs(A[i]).max())[1] for i in range(m)])
    eb = np.array([math.frexp(np.abs(B[:, j]).max())[1] for j in range(n)])
    scale = np.ldexp(1.0, (ea[:, None] + eb[None, :]))
    bound = scale * k * 2.0 ** (-beta * s) * (s + 3) + 4 * s * 2.0 ** -53 * np.abs(ref)
    assert (np.abs(got - ref) <= bound).all()


def test_ozaki_more_slices_more_accurate(ora):
    A = W.scaled_f64((32, 128), 38)
    B = W.scaled_f64((128, 32), 39)
    ref = ora.gemm_rows(A, B, list(range(32)), accurate=True)
    errs = []
    for s in (3, 5, 7, 9):
        got = ora.ozaki_gemm(A, B, beta_bits=6, s=s)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] <= 1e-13


def test_ozaki_blas_semantics(ora):
    A = W.scaled_f64((8, 16), 40)
    B = W.scaled_f64((16, 8), 41)
    C = W.uniform_f64((8, 8), 42)
    base = ora.ozaki_gemm(A, B)
    got = ora.ozaki_gemm(A, B, alpha=2.0, beta=-1.0, C=C)
    assert np.array_equal(got, 2.0 * base - C)
    Cn = np.full((8, 8), np.nan, order="F")
    assert np.isfinite(ora.ozaki_gemm(A, B, beta=0.0, C=Cn)).all()
