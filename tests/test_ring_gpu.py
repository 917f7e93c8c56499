"""GPU parity of the paper's ring algorithm (Algorithm 2 on a cluster of p CTAs).

Integer-valued inputs: bit-exact against the oracle's literal ring simulation and
the exact product (every partial sum is an integer below 2^53).  FP64 uniform
inputs: within gamma_n (|A||B|)_ij of the oracle (the orders of summation differ).
"""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_colmajor, hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]
U = 2.0 ** -53


def run(A, B, p, K):
    h = hsmm()
    n = A.shape[0]
    dC = dev_colmajor(np.full((n, n), np.nan))
    h.ring_gemm(dev_colmajor(A), dev_colmajor(B), dC, p=p, K=K)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return dC.cpu().numpy()


@pytest.mark.parametrize("K", [1, 2, 4, 8, 16])
def test_ring_512_integer_bitexact(ora, K):
    A, B = W.ring_inputs(integer=True)
    got = run(A, B, 16, K)
    ref, st = ora.ring_hsmm(A, B, 16, K)
    assert np.array_equal(got, ref)
    assert np.array_equal(got, ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("p,K,b", [(4, 2, 8), (8, 2, 16), (12, 3, 8), (16, 4, 16), (2, 1, 32), (1, 1, 8)])
def test_ring_shapes_integer(ora, p, K, b):
    n = p * b
    A, B = W.ring_inputs(n=n, integer=True, seed=p * 100 + K)
    got = run(A, B, p, K)
    assert np.array_equal(got, ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64))


def test_ring_512_fp64(ora):
    """The n = 512, p = 16, K = 4 workload with FP64 uniform(-1, 1) entries."""
    A, B = W.ring_inputs()
    got = run(A, B, 16, 4)
    ref = ora.gemm(A, B)
    ring_ref, _ = ora.ring_hsmm(A, B, 16, 4)
    n = 512
    gam = n * U / (1 - n * U)
    mag = ora.gemm(np.abs(A), np.abs(B))
    assert (np.abs(got - ref) <= 2 * gam * mag).all()
    assert (np.abs(got - ring_ref) <= 2 * gam * mag).all()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-14
