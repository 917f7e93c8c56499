"""The allocation-free matrix-vector entry point (hsmm_gemv_n_noalloc).

It serves callers that cannot allocate device memory or hold a workspace (code
living inside another application's memory arena, or latency-bound loops that
must not risk an allocation's device synchronisation).  Its partial sums live in
a fixed array inside the library and it runs hsmm_gemv's own op = N kernels, so
this test checks, on two calls in a row (the second call reuses the array the
first one left behind):
  * the result against the oracle: FP32 within gamma_(n+2) (|A||x|) elementwise
    plus the beta*y term, INT8 bit for bit;
  * bit equality with the workspace-based hsmm_gemv on the same inputs;
  * the BLAS early-out alpha == 0 (y = beta*y without reading A: NaN in A stays out);
  * that an over-size request is refused before anything runs.
Collected last on purpose: a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from _gpu import dev_colmajor, hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]
U32 = 2.0 ** -24


def call_noalloc(h, A, x, y, dtype_code, alpha, beta):
    """Direct C-ABI call of hsmm_gemv_n_noalloc (no workspace argument exists)."""
    L = h.lib()
    if dtype_code == h.R_32F:
        al, be = ctypes.c_float(alpha), ctypes.c_float(beta)
    else:
        al, be = ctypes.c_int32(alpha), ctypes.c_int32(beta)
    m, n = A.shape
    st = L.hsmm_gemv_n_noalloc(dtype_code, m, n, ctypes.byref(al), A.data_ptr(), A.stride(1), x.data_ptr(), 1,
                               ctypes.byref(be), y.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
    assert st == 0, h.hsmm.status_string(st)


@pytest.mark.parametrize("m,n", [(16384, 16384), (1000, 777)])
def test_noalloc_f32_oracle_and_gemv_twice(m, n):
    h = hsmm()
    alpha, beta = 0.5, 2.0
    for call, seed in enumerate((31, 32)):
        A = W.uniform_f32((m, n), seed)
        x = W.uniform_f32((n,), seed + 100)
        y0 = W.uniform_f32((m,), seed + 200)
        dA = dev_colmajor(A)
        dx = torch.from_numpy(x).cuda()
        y_ref = torch.from_numpy(y0.copy()).cuda()
        y_new = torch.from_numpy(y0.copy()).cuda()
        h.gemv(dA, dx, y_ref, "N", alpha=alpha, beta=beta)
        call_noalloc(h, dA, dx, y_new, h.R_32F, alpha, beta)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        # the same kernels and order as hsmm_gemv: the same bits
        assert torch.equal(y_new, y_ref), call
        A64, x64, y64 = A.astype(np.float64), x.astype(np.float64), y0.astype(np.float64)
        want = oracle.gemv(A64, x64, "N", alpha=alpha, beta=beta, y=y64.copy())
        mag = alpha * (np.abs(A64) @ np.abs(x64)) + beta * np.abs(y64)
        gam = (n + 2) * U32 / (1 - (n + 2) * U32)
        got = y_new.cpu().numpy().astype(np.float64)
        assert (np.abs(got - want) <= gam * mag).all(), (call, float(np.max(np.abs(got - want) / (gam * mag))))


def test_noalloc_i8_oracle_exact_twice():
    h = hsmm()
    m, n = 4096, 3000
    for seed in (41, 42):
        A = W.integers((m, n), seed, -128, 127, np.int8)
        x = W.integers((n,), seed + 1, -128, 127, np.int8)
        y0 = W.integers((m,), seed + 2, -1000, 1000, np.int32)
        dA = dev_colmajor(A)
        dx = torch.from_numpy(x).cuda()
        y_ref = torch.from_numpy(y0.copy()).cuda()
        y_new = torch.from_numpy(y0.copy()).cuda()
        h.gemv(dA, dx, y_ref, "N", alpha=3, beta=-2)
        call_noalloc(h, dA, dx, y_new, h.R_8I, 3, -2)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        want = oracle.gemv_i8(A, x, "N", alpha=3, beta=-2, y=y0.copy())
        assert np.array_equal(y_new.cpu().numpy().astype(np.int64), np.asarray(want, dtype=np.int64))
        assert torch.equal(y_new, y_ref)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_noalloc_alpha_zero_reads_no_A(dtype):
    """alpha == 0: y = beta*y without reading A or x, so NaN in A never reaches y."""
    h = hsmm()
    m, n = 777, 513
    if dtype == "f32":
        A = W.uniform_f32((m, n), 51)
        A[3, 5] = np.nan
        x = W.uniform_f32((n,), 52)
        x[7] = np.inf
        y0 = W.uniform_f32((m,), 53)
        y = torch.from_numpy(y0.copy()).cuda()
        call_noalloc(h, dev_colmajor(A), torch.from_numpy(x).cuda(), y, h.R_32F, 0.0, 1.5)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.array_equal(got, (np.float32(1.5) * y0).astype(np.float32))
    else:
        A = W.integers((m, n), 54, -128, 127, np.int8)
        x = W.integers((n,), 55, -128, 127, np.int8)
        y0 = W.integers((m,), 56, -1000, 1000, np.int32)
        y = torch.from_numpy(y0.copy()).cuda()
        call_noalloc(h, dev_colmajor(A), torch.from_numpy(x).cuda(), y, h.R_8I, 0, -3)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), -3 * y0)
    assert h.sync_status() == 0


def test_noalloc_rejects_oversize_before_launch():
    h = hsmm()
    L = h.lib()
    al = ctypes.c_float(1.0)
    m = (1 << 21) + 1
    st = L.hsmm_gemv_n_noalloc(h.R_32F, m, 1, ctypes.byref(al), 16, m, 16, 1, ctypes.byref(al), 16, 1, None)
    assert st == h.hsmm.WORKSPACE_TOO_SMALL
