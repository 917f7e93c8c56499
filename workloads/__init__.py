"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic.  Every generator is a NumPy ``Generator(PCG64(seed))``, so
the CUDA path and the oracle consume identical bytes.  Matrices are returned in
column-major (Fortran) order, the storage convention of the hsmm C-ABI.

Workloads (the shapes and distributions of the paper's dense products):
  ring     -- n = 512 FP64, uniform(-1, 1); block-mapped ring with p = 16 (blocks of 32)
  gemv     -- A 16384 x 16384 FP32 uniform(-1, 1), x of length 16384;
              INT8 variant with A, x uniform integers in [-128, 127]
  precise  -- m = n = k = 8192 FP64 entries s * 2^e, s ~ U(1, 2) with a fair random sign,
              e uniform integer in [-12, 12]
  autograd -- A 4096 x 2048, B 2048 x 8192 BF16 from N(0, 1/k); upstream gradient N(0, 1)
  grouped  -- 512 problems, m, n, k log-uniform in [64, 2048], BF16 uniform(-1, 1)
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20250
SEED_RING, SEED_GEMV, SEED_PRECISE, SEED_AUTOGRAD, SEED_GROUPED, SEED_ZPRECISE, SEED_NBODY = (
    SEED_BASE + i for i in range(1, 8))
NBODY_N = 131072
NBODY_EPS2 = 1e-4


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_f64(shape, seed, lo=-1.0, hi=1.0):
    return np.asfortranarray(rng(seed).uniform(lo, hi, size=shape))


def uniform_f32(shape, seed, lo=-1.0, hi=1.0):
    return np.asfortranarray(rng(seed).uniform(lo, hi, size=shape).astype(np.float32))


def integers(shape, seed, lo, hi, dtype):
    """Uniform integers in [lo, hi] (inclusive)."""
    return np.asfortranarray(rng(seed).integers(lo, hi + 1, size=shape, dtype=np.int64).astype(dtype))


def scaled_f64(shape, seed, emin=-12, emax=12):
    """Entries s * 2^e: s ~ U(1, 2), random sign, e uniform integer in [emin, emax]."""
    g = rng(seed)
    s = g.uniform(1.0, 2.0, size=shape)
    sign = np.where(g.integers(0, 2, size=shape) == 0, -1.0, 1.0)
    e = g.integers(emin, emax + 1, size=shape)
    return np.asfortranarray(np.ldexp(sign * s, e))


def bf16_bits_from_f32(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even) and return the 16-bit patterns."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    out = r.reshape(x.shape)
    return np.asfortranarray(out) if x.ndim == 2 and np.isfortran(x) else out


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """Exact widening of BF16 bit patterns to float64."""
    f = (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)
    out = f.astype(np.float64)
    return np.asfortranarray(out) if out.ndim == 2 else out


def normal_bf16(shape, seed, std=1.0):
    x = (rng(seed).standard_normal(size=shape) * std).astype(np.float32)
    return bf16_bits_from_f32(np.asfortranarray(x))


def uniform_bf16(shape, seed, lo=-1.0, hi=1.0):
    return bf16_bits_from_f32(uniform_f32(shape, seed, lo, hi))


# ---- named workloads ---------------------------------------------------------

def ring_inputs(n=512, seed=SEED_RING, integer=False):
    """n x n FP64 pair (uniform(-1, 1), or uniform integers in [-8, 8])."""
    if integer:
        return (integers((n, n), seed, -8, 8, np.float64), integers((n, n), seed + 1000, -8, 8, np.float64))
    return uniform_f64((n, n), seed), uniform_f64((n, n), seed + 1000)


def gemv_inputs(m=16384, n=16384, seed=SEED_GEMV):
    A = uniform_f32((m, n), seed)
    xs = uniform_f32((max(m, n),), seed + 1000)
    return A, xs


def gemv_i8_inputs(m=16384, n=16384, seed=SEED_GEMV):
    A = integers((m, n), seed + 2000, -128, 127, np.int8)
    xs = integers((max(m, n),), seed + 3000, -128, 127, np.int8)
    return A, xs


def precise_inputs(m=8192, n=8192, k=8192, seed=SEED_PRECISE):
    return scaled_f64((m, k), seed), scaled_f64((k, n), seed + 1000)


def scaled_c128(shape, seed, emin=-12, emax=12):
    """Complex entries whose real and imaginary parts are drawn independently as scaled_f64."""
    return np.asfortranarray(scaled_f64(shape, seed, emin, emax) + 1j * scaled_f64(shape, seed + 500, emin, emax))


def zprecise_inputs(m=4096, n=4096, k=4096, seed=SEED_ZPRECISE):
    """The complex precision workload: A (m x k), B (k x n) complex128."""
    return scaled_c128((m, k), seed), scaled_c128((k, n), seed + 1000)


def nbody_bodies(n=NBODY_N, seed=SEED_NBODY):
    """n bodies (px, py, pz, m): positions uniform in the unit ball, masses uniform in [0.5, 1.5] / n."""
    r = rng(seed)
    d = r.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pos = d * r.uniform(0, 1, size=(n, 1)) ** (1.0 / 3.0)
    return np.ascontiguousarray(np.c_[pos, r.uniform(0.5, 1.5, size=n) / n])


def autograd_inputs(m=4096, k=2048, n=8192, seed=SEED_AUTOGRAD):
    """Row-major (PyTorch) BF16 bit patterns: A (m,k), B (k,n), dC (m,n)."""
    std = 1.0 / np.sqrt(k)
    A = np.ascontiguousarray(normal_bf16((m, k), seed, std))
    B = np.ascontiguousarray(normal_bf16((k, n), seed + 1000, std))
    G = np.ascontiguousarray(normal_bf16((m, n), seed + 2000, 1.0))
    return A, B, G


def grouped_shapes(count=512, lo=64, hi=2048, seed=SEED_GROUPED):
    """(m, n, k) per problem, each log-uniform in [lo, hi], rounded to integers."""
    g = rng(seed)
    v = np.exp(g.uniform(np.log(lo), np.log(hi), size=(count, 3)))
    return np.clip(np.rint(v).astype(np.int64), lo, hi)


def pad_ld(rows: int, mult: int = 8) -> int:
    """Leading dimension padded to a multiple of `mult` elements (16 bytes for BF16)."""
    return max(mult, (rows + mult - 1) // mult * mult)
