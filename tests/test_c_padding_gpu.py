"""Every product form touches only the m x n elements of C: with C's storage NaN everywhere
(the padding rows m..ldc-1 of each column included), the padding must still be NaN after the
call and the m x n block must be finite.  Leading dimensions are whole 16-byte units, so the
TMA-store epilogues run (their row clipping works on 16-byte units, and the rows past the last
whole unit must be stored another way)."""
import pytest
import torch

import workloads as W
from _gpu import dev_bf16_colmajor, dev_colmajor, hsmm, padded, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

SHAPES = [(300, 170, 96), (129, 257, 65), (77, 40, 33), (517, 300, 200)]


def nan_c(m, n, dtype, beta_block=None):
    """Column-major m x n view into NaN-filled storage with ldc = m rounded up to 16 bytes plus 16 bytes."""
    esize = torch.empty((), dtype=dtype).element_size()
    unit = max(1, 16 // esize)
    ldc = (m + unit - 1) // unit * unit + unit
    base = torch.full((n, ldc), float("nan"), dtype=dtype, device="cuda")
    C = base[:, :m].t()
    if beta_block is not None:
        C.copy_(beta_block)
    return base, C


def check(base, C, m):
    torch.cuda.synchronize()
    h = hsmm()
    assert h.sync_status() == 0
    assert torch.isnan(base[:, m:]).all(), "a padding row of C was written"
    assert torch.isfinite(C).all(), "an element of C was not written"


@pytest.mark.parametrize("kernel", ["pair", "single"])
@pytest.mark.parametrize("out", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_bf16_products(m, n, k, out, kernel, monkeypatch):
    monkeypatch.setenv("HSMM_GEMM_KERNEL", kernel)
    h = hsmm()
    A = dev_bf16_colmajor(W.uniform_bf16((m, k), 31), ld=padded(m))
    B = dev_bf16_colmajor(W.uniform_bf16((k, n), 32), ld=padded(k))
    base, C = nan_c(m, n, out)
    h.gemm(A, B, C)
    check(base, C, m)
    # beta != 0 reads C: only the m x n block
    base, C = nan_c(m, n, out, beta_block=torch.ones((m, n), dtype=out, device="cuda"))
    h.gemm(A, B, C, alpha=0.5, beta=2.0)
    check(base, C, m)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_tf32_products(m, n, k):
    h = hsmm()
    A = dev_colmajor(W.uniform_f32((m, k), 33), ld=padded(m, 4))
    B = dev_colmajor(W.uniform_f32((k, n), 34), ld=padded(k, 4))
    base, C = nan_c(m, n, torch.float32)
    h.gemm(A, B, C, compute=h.COMPUTE_32F_FAST_TF32)
    check(base, C, m)


@pytest.mark.parametrize("compute", ["native", "ozaki"])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_fp64_products(m, n, k, compute):
    h = hsmm()
    cp = h.COMPUTE_64F_NATIVE if compute == "native" else h.COMPUTE_64F_OZAKI
    A = dev_colmajor(W.uniform_f64((m, k), 35))
    B = dev_colmajor(W.uniform_f64((k, n), 36))
    base, C = nan_c(m, n, torch.float64)
    h.gemm(A, B, C, compute=cp)
    check(base, C, m)
    base, C = nan_c(m, n, torch.float64, beta_block=torch.ones((m, n), dtype=torch.float64, device="cuda"))
    h.gemm(A, B, C, alpha=0.5, beta=-1.0, compute=cp)
    check(base, C, m)


@pytest.mark.parametrize("compute", ["native", "ozaki"])
@pytest.mark.parametrize("m,n,k", SHAPES[:2])
def test_complex_products(m, n, k, compute):
    h = hsmm()
    cp = h.COMPUTE_64F_NATIVE if compute == "native" else h.COMPUTE_64F_OZAKI
    A = dev_colmajor(W.scaled_c128((m, k), 37))
    B = dev_colmajor(W.scaled_c128((k, n), 38))
    base, C = nan_c(m, n, torch.complex128)
    h.gemm(A, B, C, compute=cp)
    check(base, C, m)
