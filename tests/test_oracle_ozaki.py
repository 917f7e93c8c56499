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


# ---------------------------------------------------------------------------------------------
# Pins of ora_ozaki_diagonals: the exact anti-diagonal sums S_d that every bit-exact GPU check
# of the slice products compares against (Ozaki et al. 2012, integer-slice form).
# ---------------------------------------------------------------------------------------------
def _ozaki_operands(m, n, k, ta, tb, seed):
    A = W.scaled_f64((m, k) if ta == "N" else (k, m), seed)
    B = W.scaled_f64((k, n) if tb == "N" else (n, k), seed + 1)
    # a row of A and a column of B at the largest magnitude of their line: digits of 2^beta - 1
    Ao = A if ta == "N" else A.T
    Bo = B if tb == "N" else B.T
    Ao[0, :] = np.where(Ao[0, :] < 0, -1.0, 1.0) * np.nextafter(1.0, 0.0)
    Bo[:, 0] = np.where(Bo[:, 0] < 0, -1.0, 1.0) * np.nextafter(1.0, 0.0)
    return A, B, np.asfortranarray(Ao), np.asfortranarray(Bo)


@pytest.mark.parametrize("s", [3, 7])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_diagonals_big_integer_brute_force(ora, s, ta, tb):
    """S_d for d = 2..s+1 equals the Python big-integer sum over the slice pairs t + u = d
    (1 <= t, u <= s) of the slices that ora_ozaki_split returns, element by element."""
    m, n, k, beta = 5, 4, 9, 7
    A, B, Ao, Bo = _ozaki_operands(m, n, k, ta, tb, 51 + s)
    ea, eb, sd = ora.ozaki_diagonals(A, B, ta, tb, beta_bits=beta, s=s)
    ea2, qa = ora.ozaki_split(Ao, True, beta, s)
    eb2, qb = ora.ozaki_split(Bo, False, beta, s)
    assert np.array_equal(ea, ea2) and np.array_equal(eb, eb2)
    assert sd.shape == (s, m, n)
    # the extreme line really reaches digits of magnitude 2^beta - 1
    assert np.abs(qa[:, 0, :]).max() == 2 ** beta - 1 and np.abs(qb[:, :, 0]).max() == 2 ** beta - 1
    qa_i = [[[int(qa[t, i, p]) for p in range(k)] for i in range(m)] for t in range(s)]
    qb_i = [[[int(qb[u, p, j]) for p in range(k)] for j in range(n)] for u in range(s)]
    for d in range(2, s + 2):
        for i in range(m):
            for j in range(n):
                want = 0
                for t in range(1, s + 1):
                    u = d - t
                    if 1 <= u <= s:
                        want += sum(a * b for a, b in zip(qa_i[t - 1][i], qb_i[u - 1][j]))
                assert int(sd[d - 2, i, j]) == want, (d, i, j)


def test_diagonals_raw_layout(ora):
    """The C routine writes S_d column-major per anti-diagonal: index (d-2) m n + i + j m."""
    import ctypes
    m, n, k, s, beta = 3, 5, 6, 4, 6
    A = W.scaled_f64((m, k), 61)
    B = W.scaled_f64((k, n), 62)
    _, qa = ora.ozaki_split(A, True, beta, s)
    _, qb = ora.ozaki_split(B, False, beta, s)
    qa_f = np.ascontiguousarray(np.stack([q.ravel(order="F") for q in qa]))
    qb_f = np.ascontiguousarray(np.stack([q.ravel(order="F") for q in qb]))
    raw = np.zeros(s * m * n, dtype=np.int64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ora.lib().ora_ozaki_diagonals(m, n, k, s, p(qa_f), p(qb_f), p(raw))
    for d in range(2, s + 2):
        for i in range(m):
            for j in range(n):
                want = sum(int(qa[t - 1, i, q]) * int(qb[d - t - 1, q, j])
                           for t in range(max(1, d - s), min(s, d - 1) + 1) for q in range(k))
                assert int(raw[(d - 2) * m * n + i + j * m]) == want


@pytest.mark.parametrize("s,beta", [(3, 7), (7, 7), (5, 6)])
def test_diagonals_complete_with_dropped_pairs(ora, s, beta):
    """Every slice pair is counted once: the kept anti-diagonals plus the dropped pairs
    (t + u > s + 1) give exactly the product of the truncated operands,
        sum_{d=2}^{s+1} 2^-(beta d) S_d + sum_{t+u>s+1} 2^-(beta(t+u)) QA_t QB_u = A~ B~,
    A~ = sum_t 2^(-beta t) QA_t, B~ = sum_u 2^(-beta u) QB_u (exact rationals).  A wrong range of
    d, a wrong pairing of t and u or a dropped term breaks the identity."""
    m, n, k = 4, 3, 7
    A = W.scaled_f64((m, k), 71 + s)
    B = W.scaled_f64((k, n), 72 + s)
    _, _, sd = ora.ozaki_diagonals(A, B, beta_bits=beta, s=s)
    _, qa = ora.ozaki_split(A, True, beta, s)
    _, qb = ora.ozaki_split(B, False, beta, s)
    two = Fraction(2)
    for i in range(m):
        for j in range(n):
            at = [sum(Fraction(int(qa[t, i, p])) / two ** (beta * (t + 1)) for t in range(s)) for p in range(k)]
            bt = [sum(Fraction(int(qb[u, p, j])) / two ** (beta * (u + 1)) for u in range(s)) for p in range(k)]
            full = sum(a * b for a, b in zip(at, bt))
            kept = sum(Fraction(int(sd[d - 2, i, j])) / two ** (beta * d) for d in range(2, s + 2))
            dropped = sum(Fraction(int(qa[t - 1, i, p]) * int(qb[u - 1, p, j])) / two ** (beta * (t + u))
                          for t in range(1, s + 1) for u in range(1, s + 1) if t + u > s + 1 for p in range(k))
            assert kept + dropped == full


def test_diagonals_recombine_to_ozaki_gemm(ora):
    """On integer inputs that the slices hold exactly, 2^(e_i + f_j) sum_d 2^(-beta d) S_d formed
    with rationals is the exact integer product and equals ora_ozaki_gemm bit for bit."""
    g = W.rng(81)
    A = np.asfortranarray(g.integers(-3000, 3001, size=(6, 11)).astype(np.float64))
    B = np.asfortranarray(g.integers(-3000, 3001, size=(11, 5)).astype(np.float64))
    beta, s = 7, 4                                     # 28 bits per operand > 12 bits used
    ea, eb, sd = ora.ozaki_diagonals(A, B, beta_bits=beta, s=s)
    got = ora.ozaki_gemm(A, B, beta_bits=beta, s=s)
    exact = ora.gemm_i64(A.astype(np.int64), B.astype(np.int64))
    two = Fraction(2)
    for i in range(6):
        for j in range(5):
            v = sum(Fraction(int(sd[d - 2, i, j])) / two ** (beta * d) for d in range(2, s + 2))
            v *= two ** (int(ea[i]) + int(eb[j]))
            assert v == int(exact[i, j])
            assert Fraction(got[i, j]) == v
