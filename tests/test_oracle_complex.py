"""Pins of the oracle's complex product (Section 7 measures the method on complex data).

ora_zgemm is the definition of the complex product summed in order; the pins below fix
it to things other than itself: exact big-integer brute force for every op pair (a
dropped term, a wrong sign, a missing conjugation or a transposed operand changes an
integer result), the real special case bit for bit, the identity (AB)^H = B^H A^H bit for
bit, and the floating-point error bound against exact rational arithmetic.  The real form
zembed used by the FP64-accurate complex product is pinned to the brute force as well.
"""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

OPS = ["N", "T", "C"]


def rand_int_complex(shape, seed, lo=-9, hi=9):
    r = W.rng(seed)
    return np.asfortranarray(r.integers(lo, hi + 1, size=shape) + 1j * r.integers(lo, hi + 1, size=shape))


def stored(rows, cols, t):
    return (rows, cols) if t == "N" else (cols, rows)


def brute(A, B, ta, tb, alpha=(1, 0), beta=(0, 0), C=None):
    """Python-integer brute force: complex numbers as pairs of ints."""
    def op(M, t, i, j):
        x = M[i, j] if t == "N" else M[j, i]
        re, im = int(x.real), int(x.imag)
        return (re, -im) if t == "C" else (re, im)
    m = A.shape[0] if ta == "N" else A.shape[1]
    k = A.shape[1] if ta == "N" else A.shape[0]
    n = B.shape[1] if tb == "N" else B.shape[0]
    out = np.zeros((m, n), np.complex128)
    for i in range(m):
        for j in range(n):
            sr = si = 0
            for p in range(k):
                ar, ai = op(A, ta, i, p)
                br, bi = op(B, tb, p, j)
                sr += ar * br - ai * bi
                si += ar * bi + ai * br
            vr = alpha[0] * sr - alpha[1] * si
            vi = alpha[0] * si + alpha[1] * sr
            if C is not None:
                cr, ci = int(C[i, j].real), int(C[i, j].imag)
                vr += beta[0] * cr - beta[1] * ci
                vi += beta[0] * ci + beta[1] * cr
            out[i, j] = complex(vr, vi)
    return out


@pytest.mark.parametrize("ta", OPS)
@pytest.mark.parametrize("tb", OPS)
def test_zgemm_integer_brute_force(ora, ta, tb):
    m, n, k = 5, 4, 7
    A = rand_int_complex(stored(m, k, ta), 31 + ord(ta))
    B = rand_int_complex(stored(k, n, tb), 37 + ord(tb))
    assert np.array_equal(ora.zgemm(A, B, ta, tb), brute(A, B, ta, tb))


def test_zgemm_alpha_beta_integer(ora):
    A = rand_int_complex((4, 6), 41)
    B = rand_int_complex((6, 3), 42)
    C = rand_int_complex((4, 3), 43)
    got = ora.zgemm(A, B, "N", "N", alpha=complex(2, -3), beta=complex(-1, 4), C=C)
    assert np.array_equal(got, brute(A, B, "N", "N", (2, -3), (-1, 4), C))
    # beta == 0: C is not read (NaNs stay out of the result)
    got = ora.zgemm(A, B, "N", "N", C=np.full((4, 3), np.nan + 0j))
    assert np.array_equal(got, brute(A, B, "N", "N"))


def test_zgemm_real_special_case_bitwise(ora):
    """Zero imaginary parts: the real parts are the real oracle's result bit for bit."""
    A = W.uniform_f64((9, 13), 44)
    B = W.uniform_f64((13, 8), 45)
    got = ora.zgemm(A.astype(np.complex128), B.astype(np.complex128))
    assert np.array_equal(got.real, ora.gemm(A, B)) and (got.imag == 0).all()


def test_zgemm_conjugate_transpose_identity(ora):
    """(A B)^H = B^H A^H bit for bit: the same products and sums in the same order."""
    A = np.asfortranarray(W.uniform_f64((7, 11), 46) + 1j * W.uniform_f64((7, 11), 47))
    B = np.asfortranarray(W.uniform_f64((11, 6), 48) + 1j * W.uniform_f64((11, 6), 49))
    AB = ora.zgemm(A, B)
    BhAh = ora.zgemm(B, A, "C", "C")
    assert np.array_equal(AB.conj().T, BhAh)
    # op = T of A^T and op = C of conj(A)^T are op = N of A
    assert np.array_equal(ora.zgemm(np.asfortranarray(A.T), B, "T", "N"), AB)
    assert np.array_equal(ora.zgemm(np.asfortranarray(A.conj().T), B, "C", "N"), AB)


def test_zgemm_error_bound_rational(ora):
    """|fl(c) - c| <= gamma_{k+2} sum_k (|Re a|+|Im a|)(|Re b|+|Im b|) per part, c exact."""
    m, n, k = 3, 3, 20
    A = np.asfortranarray(W.uniform_f64((m, k), 50) + 1j * W.uniform_f64((m, k), 51))
    B = np.asfortranarray(W.uniform_f64((k, n), 52) + 1j * W.uniform_f64((k, n), 53))
    got = ora.zgemm(A, B)
    u = 2.0 ** -53
    gam = (k + 2) * u / (1 - (k + 2) * u)
    for i in range(m):
        for j in range(n):
            er = sum(Fraction(A[i, p].real) * Fraction(B[p, j].real) - Fraction(A[i, p].imag) * Fraction(B[p, j].imag)
                     for p in range(k))
            ei = sum(Fraction(A[i, p].real) * Fraction(B[p, j].imag) + Fraction(A[i, p].imag) * Fraction(B[p, j].real)
                     for p in range(k))
            mag = sum((abs(A[i, p].real) + abs(A[i, p].imag)) * (abs(B[p, j].real) + abs(B[p, j].imag))
                      for p in range(k))
            assert abs(Fraction(got[i, j].real) - er) <= Fraction(gam * mag)
            assert abs(Fraction(got[i, j].imag) - ei) <= Fraction(gam * mag)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("C", "T"), ("T", "C")])
def test_zembed_is_the_complex_product(ora, ta, tb):
    """The real form A' B'' = [Re, Im] of the complex product, on integers exactly."""
    m, n, k = 6, 5, 9
    A = rand_int_complex(stored(m, k, ta), 60)
    B = rand_int_complex(stored(k, n, tb), 61)
    Ap, Bpp = ora.zembed(A, B, ta, tb)
    assert Ap.shape == (m, 2 * k) and Bpp.shape == (2 * k, 2 * n)
    P = ora.gemm_i64(Ap.astype(np.int64), Bpp.astype(np.int64))
    want = brute(A, B, ta, tb)
    assert np.array_equal(P[:, :n], want.real.astype(np.int64))
    assert np.array_equal(P[:, n:], want.imag.astype(np.int64))
    rows = [0, 3, 5]
    assert np.array_equal(ora.zgemm_rows(A, B, rows, ta, tb), want[rows])
