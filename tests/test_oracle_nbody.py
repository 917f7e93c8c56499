"""Pins of the oracle's two-array n^2 problem (Section 4) and its gravitational instance (Section 2).

ora_nbody_direct is the definition F_i = sum_j f(x_i, z_j); it is pinned by an integer
interaction against Python brute force, by Newton's law for two bodies, by exact scaling laws
(positions x2 and eps2 x4 quarter the accelerations; masses x2 double them: powers of two, so
bit for bit) and by momentum conservation.  ora_nbody_hsys, the recipe of Section 4.1 with the
regular bases, is pinned by its counters (every block pair met exactly once, the shift counts
of Theorem GAIN2), by the exact integer interaction against the direct sum, and by a planted
non-covering stride that must fail.
"""
import math

import numpy as np
import pytest

import workloads as W


def bodies(n, seed, integer=False):
    r = W.rng(seed)
    if integer:
        return np.c_[r.integers(-20, 21, size=(n, 3)), r.integers(1, 5, size=n)].astype(np.float64)
    return np.c_[r.uniform(-1, 1, size=(n, 3)), r.uniform(0.5, 1.5, size=n)]


def divisors(p):
    return [k for k in range(1, p + 1) if p % k == 0]


def test_direct_integer_brute_force(ora):
    x, z = bodies(9, 1, True), bodies(13, 2, True)
    F = ora.nbody_direct(x, z, 0.0, kind=1)
    for i in range(9):
        want = [sum(int(z[j, 3]) * (int(z[j, c]) - int(x[i, c])) for j in range(13)) for c in range(3)]
        assert F[i].tolist() == want


def test_direct_two_bodies_newton():
    """|a| = m / d^2 towards the other body (eps = 0): d = 2, m = 4 gives exactly 1."""
    import oracle as ora
    x = np.array([[0.0, 0.0, 0.0, 1.0], [2.0, 0.0, 0.0, 4.0]])
    F = ora.nbody_direct(x, x, 0.0)
    assert F[0].tolist() == [1.0, 0.0, 0.0]          # pulled towards +x
    assert F[1].tolist() == [-0.25, 0.0, 0.0]        # m = 1 at distance 2, towards -x
    x2 = np.array([[0.0, 0.0, 0.0, 1.0], [0.0, -3.0, 4.0, 25.0]])   # d = 5
    F2 = ora.nbody_direct(x2, x2, 0.0)
    assert np.allclose(F2[0], [0.0, -3.0 / 5.0, 4.0 / 5.0], rtol=0, atol=1e-15)


def test_direct_scaling_laws_bitwise(ora):
    x = bodies(40, 3)
    eps2 = 0.01
    F = ora.nbody_direct(x, x, eps2)
    xs = x.copy(); xs[:, :3] *= 2.0
    assert np.array_equal(ora.nbody_direct(xs, xs, 4.0 * eps2), F / 4.0)
    xm = x.copy(); xm[:, 3] *= 2.0
    assert np.array_equal(ora.nbody_direct(xm, xm, eps2), F * 2.0)


def test_direct_momentum_conservation(ora):
    """sum_i m_i a_i = 0 for a self-interacting system (f(x_i, x_j) m_i = -f(x_j, x_i) m_j)."""
    x = bodies(200, 4)
    F = ora.nbody_direct(x, x, 1e-3)
    total = (x[:, 3:4] * F).sum(axis=0)
    scale = (x[:, 3:4] * np.abs(F)).sum()
    assert np.all(np.abs(total) <= 1e-12 * scale)


@pytest.mark.parametrize("p", [1, 2, 4, 6, 8, 9, 12, 16])
def test_hsys_every_pair_once_and_shift_counts(ora, p):
    x = bodies(2 * p, 5, True)
    for K in divisors(p):
        F, cnt, sh = ora.nbody_hsys(x, x, p, K, 0.0, kind=1)
        assert (cnt == 1).all(), (p, K)
        Kt = p // K
        assert sh == (K - 1, Kt - 1, K - 1)
        assert sum(sh) == 2 * K + Kt - 3 if p > 1 else sum(sh) == 0      # T of Eq. COMPLEXR
        assert np.array_equal(F, ora.nbody_direct(x, x, 0.0, kind=1))


def test_hsys_gravity_matches_direct(ora):
    x = bodies(64, 6)
    want = ora.nbody_direct(x, x, 1e-2)
    for p, K in [(4, 2), (16, 4), (8, 2)]:
        F, cnt, _ = ora.nbody_hsys(x, x, p, K, 1e-2)
        assert (cnt == 1).all()
        assert np.allclose(F, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_hsys_two_arrays(ora):
    """x and z different arrays (the general form F_i = sum_j f(x_i, z_j))."""
    x, z = bodies(32, 7, True), bodies(32, 8, True)
    F, cnt, _ = ora.nbody_hsys(x, z, 8, 2, 0.0, kind=1)
    assert np.array_equal(F, ora.nbody_direct(x, z, 0.0, kind=1))


def test_hsys_planted_stride_fails(ora):
    """z moving by K + 1 instead of K misses some distances and repeats others."""
    x = bodies(16, 9, True)
    F, cnt, _ = ora.nbody_hsys(x, x, 16, 4, 0.0, kind=1, zstride=5)
    assert not (cnt == 1).all()
    assert not np.array_equal(F, ora.nbody_direct(x, x, 0.0, kind=1))
