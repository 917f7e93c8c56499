"""hsmm_gemm_host: the product with A, B, C in host memory, copies overlapped with the computation.

The blocks of C (row panels of op(A) times column panels of op(B)) only change which entries
are computed together: every entry goes through the same arithmetic as hsmm_gemm on device
copies of the same data, so the results agree bit for bit (the FP64-accurate forms split each
row of op(A) and each column of op(B) from that line alone).  One case is also held against
the oracle directly.
"""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def host_colmajor(X, dtype, ld=None):
    """Page-locked column-major host tensor holding X."""
    rows, cols = X.shape
    ld = rows if ld is None else ld
    base = torch.zeros((max(cols, 1), max(ld, 1)), dtype=dtype).pin_memory()
    base[:cols, :rows] = torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to(dtype)
    return base.t()[:rows, :cols]


def dev_like(t):
    """Device copy with the same column-major layout."""
    rows, cols = t.shape
    base = torch.zeros((max(cols, 1), max(t.stride(1), rows, 1)), dtype=t.dtype, device="cuda")
    base[:cols, :rows] = t.t().cuda()
    return base.t()[:rows, :cols]


def both(A, B, C0, ta, tb, **kw):
    h = hsmm()
    hA, hB, hC = A, B, C0.clone()
    dA, dB, dC = dev_like(A), dev_like(B), dev_like(C0)
    h.gemm_host(hA, hB, hC, ta, tb, **kw)
    h.gemm(dA, dB, dC, ta, tb, **kw)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return hC, dC.cpu()


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("n", [300, 4500])
def test_fp64_accurate_same_as_device(ora, ta, tb, n):
    h = hsmm()
    m, k = 200, 150
    sa, sb = ((m, k) if ta == "N" else (k, m)), ((k, n) if tb == "N" else (n, k))
    A = host_colmajor(W.scaled_f64(sa, 1), torch.float64, ld=sa[0] + 1)
    B = host_colmajor(W.scaled_f64(sb, 2), torch.float64)
    C0 = host_colmajor(np.full((m, n), np.nan), torch.float64, ld=m + 3)
    got, want = both(A, B, C0, ta, tb, compute=h.COMPUTE_64F_OZAKI)
    assert torch.equal(got, want)
    if ta == "N" and tb == "N":
        ref = ora.ozaki_gemm(A.numpy(), B.numpy(), beta_bits=7, s=7)
        mag = ora.gemm(np.abs(A.numpy()), np.abs(B.numpy()))
        assert (np.abs(got.numpy() - ref) <= 16 * 2.0 ** -53 * mag).all()


def test_fp64_accurate_beta_two_panels():
    h = hsmm()
    m, n, k = 130, 4200, 96
    A = host_colmajor(W.scaled_f64((m, k), 3), torch.float64)
    B = host_colmajor(W.scaled_f64((k, n), 4), torch.float64)
    C0 = host_colmajor(W.uniform_f64((m, n), 5), torch.float64)
    got, want = both(A, B, C0, "N", "N", alpha=-1.5, beta=0.5, compute=h.COMPUTE_64F_OZAKI)
    assert torch.equal(got, want)


@pytest.mark.parametrize("tb", ["N", "T"])
def test_bf16_same_as_device(tb):
    m, n, k = 256, 4352, 192
    A = host_colmajor(W.bf16_bits_to_f64(W.uniform_bf16((m, k), 6)), torch.bfloat16)
    sb = (k, n) if tb == "N" else (n, k)
    B = host_colmajor(W.bf16_bits_to_f64(W.uniform_bf16(sb, 7)), torch.bfloat16)
    C0 = host_colmajor(np.zeros((m, n)), torch.float32)
    got, want = both(A, B, C0, "N", tb)
    assert torch.equal(got, want)


def test_complex_accurate_two_panels():
    h = hsmm()
    m, n, k = 64, 4100, 80
    A = host_colmajor(W.scaled_c128((k, m), 8), torch.complex128)
    B = host_colmajor(W.scaled_c128((k, n), 9), torch.complex128)
    C0 = host_colmajor(W.scaled_c128((m, n), 10), torch.complex128)
    got, want = both(A, B, C0, "C", "N", alpha=complex(0.5, -1), beta=complex(0, 2), compute=h.COMPUTE_64F_OZAKI)
    assert torch.equal(got, want)


def test_native_and_k_zero():
    h = hsmm()
    m, n, k = 70, 90, 33
    A = host_colmajor(W.uniform_f64((m, k), 11), torch.float64)
    B = host_colmajor(W.uniform_f64((k, n), 12), torch.float64)
    C0 = host_colmajor(W.uniform_f64((m, n), 13), torch.float64)
    got, want = both(A, B, C0, "N", "N", beta=2.0, compute=h.COMPUTE_64F_NATIVE)
    assert torch.equal(got, want)
    C1 = C0.clone()
    h.gemm_host(A[:, :0], B[:0, :], C1, beta=3.0, compute=h.COMPUTE_64F_OZAKI)
    torch.cuda.synchronize()
    assert torch.equal(C1, 3.0 * C0)


def test_errors():
    h = hsmm()
    A = host_colmajor(np.ones((8, 8)), torch.float64)
    C = host_colmajor(np.zeros((8, 8)), torch.float64)
    with pytest.raises(h.HsmmError) as e:
        h.gemm_host(A, A, C, compute=h.COMPUTE_64F_OZAKI,
                    workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert e.value.status == 3
    with pytest.raises(ValueError):
        h.gemm_host(A.cuda(), A, C)


@pytest.mark.parametrize("ta", ["N", "T"])
def test_row_and_column_panels_fp64_accurate(ta):
    """m >= 4096 and n >= 4096: 2 x 2 blocks, the row panels of op(A) copied and split apart."""
    h = hsmm()
    m, n, k = 4300, 4200, 40
    sa = (m, k) if ta == "N" else (k, m)
    A = host_colmajor(W.scaled_f64(sa, 21), torch.float64, ld=sa[0] + 5)
    B = host_colmajor(W.scaled_f64((k, n), 22), torch.float64)
    C0 = host_colmajor(W.uniform_f64((m, n), 23), torch.float64, ld=m + 1)
    got, want = both(A, B, C0, ta, "N", alpha=0.75, beta=-2.0, compute=h.COMPUTE_64F_OZAKI)
    assert torch.equal(got, want)


@pytest.mark.parametrize("ta", ["N", "T"])
def test_row_panels_bf16(ta):
    m, n, k = 4160, 320, 64
    sa = (m, k) if ta == "N" else (k, m)
    A = host_colmajor(W.bf16_bits_to_f64(W.uniform_bf16(sa, 24)), torch.bfloat16)
    B = host_colmajor(W.bf16_bits_to_f64(W.uniform_bf16((k, n), 25)), torch.bfloat16)
    C0 = host_colmajor(np.zeros((m, n)), torch.float32)
    got, want = both(A, B, C0, ta, "N")
    assert torch.equal(got, want)


def test_row_panels_complex_accurate():
    h = hsmm()
    m, n, k = 4100, 72, 24
    A = host_colmajor(W.scaled_c128((k, m), 26), torch.complex128)
    B = host_colmajor(W.scaled_c128((k, n), 27), torch.complex128)
    C0 = host_colmajor(np.zeros((m, n), dtype=np.complex128), torch.complex128)
    got, want = both(A, B, C0, "C", "N", compute=h.COMPUTE_64F_OZAKI)
    assert torch.equal(got, want)


@pytest.mark.parametrize("ta", ["N", "T"])
def test_four_row_panels_fp64_accurate(ta):
    """m >= 8192: four row panels of op(A) (the last one ragged), each split on its own."""
    h = hsmm()
    m, n, k = 8300, 4160, 24
    sa = (m, k) if ta == "N" else (k, m)
    A = host_colmajor(W.scaled_f64(sa, 28), torch.float64, ld=sa[0] + 3)
    B = host_colmajor(W.scaled_f64((k, n), 29), torch.float64)
    C0 = host_colmajor(W.uniform_f64((m, n), 30), torch.float64)
    got, want = both(A, B, C0, ta, "N", alpha=1.25, beta=0.5, compute=h.COMPUTE_64F_OZAKI)
    assert torch.equal(got, want)


def test_four_row_panels_bf16():
    m, n, k = 8200, 256, 32
    A = host_colmajor(W.bf16_bits_to_f64(W.uniform_bf16((m, k), 31)), torch.bfloat16)
    B = host_colmajor(W.bf16_bits_to_f64(W.uniform_bf16((n, k), 32)), torch.bfloat16)
    C0 = host_colmajor(np.zeros((m, n)), torch.float32)
    got, want = both(A, B, C0, "N", "T")
    assert torch.equal(got, want)
