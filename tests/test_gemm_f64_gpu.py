"""GPU parity of the native FP64 product against the oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_colmajor, host, hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]
U = 2.0 ** -53


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 16), (100, 70, 33), (257, 130, 129)])
def test_f64_native(ora, ta, tb, m, n, k):
    h = hsmm()
    sa = (m, k) if ta == "N" else (k, m)
    sb = (k, n) if tb == "N" else (n, k)
    A = W.uniform_f64(sa, 1 + m)
    B = W.uniform_f64(sb, 2 + n)
    C0 = W.uniform_f64((m, n), 3)
    dC = dev_colmajor(C0, ld=m + 1)
    h.gemm(dev_colmajor(A, ld=sa[0] + 2), dev_colmajor(B), dC, ta, tb, alpha=1.5, beta=-0.5)
    torch.cuda.synchronize()
    want = ora.gemm(A, B, ta, tb, 1.5, -0.5, C0)
    mag = ora.gemm(np.abs(A), np.abs(B), ta, tb, 1.5) + 0.5 * np.abs(C0)
    gam = (k + 2) * U / (1 - (k + 2) * U)
    assert (np.abs(host(dC) - want) <= 2 * gam * mag).all()


def test_f64_integer_exact(ora):
    h = hsmm()
    A = W.integers((130, 300), 7, -1000, 1000, np.float64)
    B = W.integers((300, 90), 8, -1000, 1000, np.float64)
    dC = dev_colmajor(np.zeros((130, 90)))
    h.gemm(dev_colmajor(A), dev_colmajor(B), dC)
    torch.cuda.synchronize()
    assert np.array_equal(host(dC), ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64))
