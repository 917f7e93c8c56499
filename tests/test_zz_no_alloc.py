"""The allocation-free matrix-vector entry point (hsmm_gemv_n_noalloc).

It serves callers that cannot allocate device memory or hold a workspace (code
living inside another application's memory arena, or latency-bound loops that
must not risk an allocation's device synchronisation).  Its partial sums live in
a fixed array inside the library, so this test checks that its results match the
workspace-based hsmm_gemv on the same inputs, twice in a row (the second call
reuses the array the first one left behind), and that an over-size request is
refused before anything runs.  Collected last on purpose: a failure here leaves
every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

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
def test_noalloc_f32_matches_gemv_twice(m, n):
    h = hsmm()
    for call, seed in enumerate((31, 32)):
        A = W.uniform_f32((m, n), seed)
        x = W.uniform_f32((n,), seed + 100)
        y0 = W.uniform_f32((m,), seed + 200)
        dA = dev_colmajor(A)
        dx = torch.from_numpy(x).cuda()
        y_ref = torch.from_numpy(y0.copy()).cuda()
        y_new = torch.from_numpy(y0.copy()).cuda()
        h.gemv(dA, dx, y_ref, "N", alpha=0.5, beta=2.0)
        call_noalloc(h, dA, dx, y_new, h.R_32F, 0.5, 2.0)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        a64 = np.abs(A.astype(np.float64))
        mag = 0.5 * (a64 @ np.abs(x.astype(np.float64))) + 2.0 * np.abs(y0.astype(np.float64))
        gam = (n + 2) * U32 / (1 - (n + 2) * U32)
        diff = np.abs(y_new.cpu().numpy().astype(np.float64) - y_ref.cpu().numpy().astype(np.float64))
        # both results lie within gamma_(n+2) |A||x| of the exact value, hence within twice that of each other
        assert (diff <= 2 * gam * mag).all(), (call, float(np.max(diff / (gam * mag))))


def test_noalloc_i8_matches_gemv_twice():
    h = hsmm()
    m, n = 4096, 3000
    for seed in (41, 42):
        A = W.integers((m, n), seed, -128, 127, np.int8)
        x = W.integers((n,), seed + 1, -128, 127, np.int8)
        dA = dev_colmajor(A)
        dx = torch.from_numpy(x).cuda()
        y_ref = torch.zeros(m, dtype=torch.int32, device="cuda")
        y_new = torch.full((m,), 7, dtype=torch.int32, device="cuda")
        h.gemv(dA, dx, y_ref, "N")
        call_noalloc(h, dA, dx, y_new, h.R_8I, 1, 0)
        torch.cuda.synchronize()
        assert torch.equal(y_new, y_ref)


def test_noalloc_rejects_oversize_before_launch():
    h = hsmm()
    L = h.lib()
    al = ctypes.c_float(1.0)
    m = (1 << 21) + 1
    st = L.hsmm_gemv_n_noalloc(h.R_32F, m, 1, ctypes.byref(al), 16, m, 16, 1, ctypes.byref(al), 16, 1, None)
    assert st == h.hsmm.WORKSPACE_TOO_SMALL
