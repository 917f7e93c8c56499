"""Pins of the oracle's dense products (CPU only).

The oracle is checked against things other than itself: Python big-integer brute
force, identities of the product, exact rational arithmetic and the published
Dot2 error bound.
"""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


def brute(A, B, ta, tb):
    """Eq. PRODUCT with Python integers (exact)."""
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    m, k = opA.shape
    n = opB.shape[1]
    return [[sum(int(opA[i, p]) * int(opB[p, j]) for p in range(k)) for j in range(n)] for i in range(m)]


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 7), (17, 9, 13), (2, 3, 0)])
def test_gemm_bruteforce_integers(ora, ta, tb, m, n, k):
    g = W.rng(11 + m + 7 * n + 13 * k)
    A = np.asfortranarray(g.integers(-50, 51, size=(m, k) if ta == "N" else (k, m)).astype(np.float64))
    B = np.asfortranarray(g.integers(-50, 51, size=(k, n) if tb == "N" else (n, k)).astype(np.float64))
    exact = np.array(brute(A, B, ta, tb), dtype=np.float64).reshape(m, n)
    assert np.array_equal(ora.gemm(A, B, ta, tb), exact)
    assert np.array_equal(ora.gemm_i64(A.astype(np.int64), B.astype(np.int64), ta, tb), exact.astype(np.int64))
    C0 = np.asfortranarray(g.integers(-9, 10, size=(m, n)).astype(np.float64))
    got = ora.gemm(A, B, ta, tb, alpha=3.0, beta=-2.0, C=C0)
    assert np.array_equal(got, 3.0 * exact - 2.0 * C0)


def test_gemm_large_integers_exact(ora):
    # entries up to 2^20, k = 64: every partial sum < 2^47, so FP64 is exact
    g = W.rng(5)
    A = np.asfortranarray(g.integers(-2**20, 2**20, size=(9, 64)).astype(np.float64))
    B = np.asfortranarray(g.integers(-2**20, 2**20, size=(64, 6)).astype(np.float64))
    exact = np.array(brute(A, B, "N", "N"), dtype=object)
    got = ora.gemm(A, B)
    assert all(int(got[i, j]) == exact[i, j] for i in range(9) for j in range(6))


def test_gemm_identity(ora):
    A = W.uniform_f64((37, 29), 1)
    assert np.array_equal(ora.gemm(A, np.eye(29)), A)
    assert np.array_equal(ora.gemm(np.eye(37), A), A)


def test_gemm_transpose_identity(ora):
    # (A B)^T = B^T A^T, bit for bit: the same products are summed in the same order
    A = W.uniform_f64((23, 31), 2)
    B = W.uniform_f64((31, 19), 3)
    assert np.array_equal(ora.gemm(A, B).T, ora.gemm(B, A, "T", "T"))
    assert np.array_equal(ora.gemm(A.T.copy(order="F"), B, "T", "N"), ora.gemm(A, B))


def test_gemm_blas_edge_semantics(ora):
    A = W.uniform_f64((5, 4), 4)
    B = W.uniform_f64((4, 3), 5)
    C = np.full((5, 3), np.nan, order="F")
    out = ora.gemm(A, B, beta=0.0, C=C)               # beta == 0: C not read
    assert np.isfinite(out).all()
    An = A.copy(order="F"); An[0, 0] = np.nan
    C2 = W.uniform_f64((5, 3), 6)
    out = ora.gemm(An, B, alpha=0.0, beta=2.0, C=C2)  # alpha == 0: A, B not read
    assert np.array_equal(out, 2.0 * C2)
    out = ora.gemm(np.zeros((5, 0), order="F"), np.zeros((0, 3), order="F"), beta=1.0, C=C2)  # k == 0
    assert np.array_equal(out, C2)


def test_gemm_rows_match_full(ora):
    A = W.uniform_f64((40, 33), 7)
    B = W.uniform_f64((21, 33), 8)   # used transposed
    full = ora.gemm(A, B, "N", "T")
    rows = [0, 5, 39]
    assert np.array_equal(ora.gemm_rows(A, B, rows, "N", "T"), full[rows])


def test_fp64_error_within_gamma_bound(ora):
    # the sequential sum obeys |fl(x'y) - x'y| <= gamma_k |x|'|y| (Higham, Thm 3.1)
    A = W.uniform_f64((6, 200), 9)
    B = W.uniform_f64((200, 4), 10)
    got = ora.gemm(A, B)
    u = 2.0 ** -53
    gam = 200 * u / (1 - 200 * u)
    for i in range(6):
        for j in range(4):
            exact = sum(Fraction(A[i, p]) * Fraction(B[p, j]) for p in range(200))
            bound = gam * float(sum(abs(Fraction(A[i, p]) * Fraction(B[p, j])) for p in range(200)))
            assert abs(Fraction(got[i, j]) - exact) <= Fraction(bound)


def test_dot2_exact_cancellation(ora):
    # x'y = 1 exactly, with huge cancelling terms: plain summation returns 0
    x = np.array([1e16, 1.0, -1e16, 3.0, -3.0])
    y = np.array([1.0, 1.0, 1.0, 1.0, 1.0])
    assert ora.dot2(x, y) == 1.0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dot2_error_bound(ora, seed):
    # Ogita-Rump-Oishi: |dot2 - x'y| <= u |x'y| + gamma_n^2 |x|'|y|
    g = W.rng(seed)
    n = 300
    x = np.ldexp(g.uniform(-1, 1, n), g.integers(-30, 30, n))
    y = np.ldexp(g.uniform(-1, 1, n), g.integers(-30, 30, n))
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
    absdot = sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(x, y))
    u = Fraction(1, 2 ** 53)
    gam = n * u / (1 - n * u)
    got = Fraction(ora.dot2(x, y))
    assert abs(got - exact) <= u * abs(exact) + gam * gam * absdot


def test_dot2_rows_vs_exact(ora):
    A = W.scaled_f64((3, 64), 12)
    B = W.scaled_f64((64, 5), 13)
    got = ora.gemm_rows(A, B, [0, 2], accurate=True)
    for r, i in enumerate([0, 2]):
        for j in range(5):
            exact = sum(Fraction(A[i, p]) * Fraction(B[p, j]) for p in range(64))
            # within one rounding of the exact value plus the tiny Dot2 term
            assert abs(Fraction(got[r, j]) - exact) <= abs(exact) * Fraction(1, 2 ** 52)


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_bruteforce(ora, trans):
    g = W.rng(21)
    A = np.asfortranarray(g.integers(-9, 10, size=(13, 7)).astype(np.float64))
    lenx = 7 if trans == "N" else 13
    x = g.integers(-9, 10, size=lenx * 2).astype(np.float64)   # stride 2
    y0 = g.integers(-9, 10, size=(13 if trans == "N" else 7) * 3).astype(np.float64)
    got = ora.gemv(A, x, trans, alpha=2.0, beta=-1.0, y=y0, incx=2, incy=3)
    opA = A if trans == "N" else A.T
    want = y0.copy()
    for i in range(opA.shape[0]):
        want[3 * i] = 2.0 * sum(opA[i, j] * x[2 * j] for j in range(opA.shape[1])) - y0[3 * i]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_i8_exact(ora, trans):
    A = W.integers((33, 21), 22, -128, 127, np.int8)
    lenx = 21 if trans == "N" else 33
    x = W.integers((lenx,), 23, -128, 127, np.int8)
    y0 = W.integers((33 if trans == "N" else 21,), 24, -1000, 1000, np.int32)
    got = ora.gemv_i8(A, x, trans, alpha=-3, beta=5, y=y0)
    opA = A.astype(object) if trans == "N" else A.T.astype(object)
    for i in range(opA.shape[0]):
        assert got[i] == -3 * sum(int(opA[i, j]) * int(x[j]) for j in range(lenx)) + 5 * int(y0[i])


def test_gemv_i8_extreme_fits_int32(ora):
    # all entries -128: |sum| = n * 2^14, the largest magnitude of the 16384 workload
    n = 16384
    A = np.full((4, n), -128, dtype=np.int8, order="F")
    x = np.full(n, -128, dtype=np.int8)
    got = ora.gemv_i8(A, x, "N")
    assert (got == n * 128 * 128).all() and got.max() < 2 ** 31
