"""GPU parity of the FP64-accurate product (BF16 slices on the tensor cores).

Three levels: (1) the exact anti-diagonal sums S_d that the kernel leaves in the
caller's workspace equal the oracle's INT64 products of its own slices, bit for
bit; (2) the FP64 result equals the oracle's emulation up to the rounding of the
recombination; (3) the normwise error against the accurate (Dot2) product is at
most 1e-13 on the precision workload's distribution.
"""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_colmajor, hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]
U = 2.0 ** -53


@pytest.fixture(params=["pair", "single"])
def slice_kernel(request, monkeypatch):
    """The slice-product kernels: CTA pairs (default) and one CTA per tile."""
    monkeypatch.setenv("HSMM_OZAKI_KERNEL", request.param)
    return request.param


def plane_pitch(elems, z):
    """Documented plane pitch (elements) of the workspace planes (include/hsmm.h)."""
    return ((elems * z + 255) // 256 * 256 + 1024) // z


def workspace_views(ws, m, n, k, s):
    """Views of the documented workspace carve-up (include/hsmm.h)."""
    up = lambda v: (v + 255) // 256 * 256
    kq = (k + 7) // 8 * 8
    pa, pb, ps = plane_pitch(m * kq, 2), plane_pitch(n * kq, 2), plane_pitch(m * n, 4)
    off = 0
    qa = off; off = up(off + s * pa * 2)
    qb = off; off = up(off + s * pb * 2)
    ea = off; off = up(off + m * 4)
    eb = off; off = up(off + n * 4)
    sd = off
    planes = ws[sd:sd + s * ps * 4].view(torch.int32).view(s, ps)[:, :m * n]
    sd_t = planes.reshape(s, n, m)                                           # [d-2][j][i]
    return sd_t, ws[ea:ea + 4 * m].view(torch.int32), ws[eb:eb + 4 * n].view(torch.int32)


def run(ora, m, n, k, ta="N", tb="N", alpha=1.0, beta=0.0, s=7, bits=7, seed=0, with_c=False, c_pad=1):
    h = hsmm()
    sa = (m, k) if ta == "N" else (k, m)
    sb = (k, n) if tb == "N" else (n, k)
    A = W.scaled_f64(sa, 1000 + seed)
    B = W.scaled_f64(sb, 2000 + seed)
    C0 = W.uniform_f64((m, n), 3000 + seed)
    # c_pad = 0 with m % 4 == 0 takes the recombination's 4-rows-per-thread path, else the scalar one
    dC = dev_colmajor(C0 if with_c else np.full((m, n), np.nan), ld=m + c_pad)
    cfg = h.hsmm.make_config(h.R_64F, h.R_64F, h.R_64F, h.COMPUTE_64F_OZAKI, s, bits)
    need = h.workspace_size(cfg, ta, tb, m, n, k)
    ws = torch.zeros(need, dtype=torch.uint8, device="cuda")
    h.gemm(dev_colmajor(A, ld=sa[0] + 3), dev_colmajor(B), dC, ta, tb, alpha=alpha, beta=beta,
           compute=h.COMPUTE_64F_OZAKI, slices=s, bits=bits, workspace=ws)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return A, B, C0, dC.cpu().numpy(), ws


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (200, 300, 150), (129, 257, 1030), (1, 1, 1), (64, 40, 8),
                                   (513, 600, 2100)])
def test_diagonal_sums_bitexact(ora, ta, tb, m, n, k, slice_kernel):
    A, B, C0, got, ws = run(ora, m, n, k, ta, tb, seed=m + n + k, c_pad=0 if m % 4 == 0 else 1)
    sd, ea, eb = workspace_views(ws, m, n, k, 7)
    e_a, e_b, sd_ref = ora.ozaki_diagonals(A, B, ta, tb, 7, 7)
    assert np.array_equal(ea.cpu().numpy(), e_a)
    assert np.array_equal(eb.cpu().numpy(), e_b)
    assert np.array_equal(sd.cpu().numpy().transpose(0, 2, 1).astype(np.int64), sd_ref)
    # the FP64 result matches the oracle's emulation up to recombination rounding
    want = ora.ozaki_gemm(A, B, ta, tb, beta_bits=7, s=7)
    mag = ora.gemm(np.abs(A), np.abs(B), ta, tb)
    assert (np.abs(got - want) <= 16 * U * mag).all()


@pytest.mark.parametrize("bits,s", [(7, 7), (7, 8), (6, 9), (5, 10)])
def test_normwise_error_vs_dot2(ora, bits, s):
    m, n, k = 256, 192, 2048
    A, B, _, got, _ = run(ora, m, n, k, bits=bits, s=s, seed=bits * 10 + s)
    ref = ora.gemm_rows(A, B, list(range(m)), accurate=True)
    nw = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert nw <= 1e-13, nw
    assert np.array_equal(got, ora.ozaki_gemm(A, B, beta_bits=bits, s=s)) or \
        (np.abs(got - ora.ozaki_gemm(A, B, beta_bits=bits, s=s)) <= 16 * U * ora.gemm(np.abs(A), np.abs(B))).all()


@pytest.mark.parametrize("m,c_pad", [(150, 1), (152, 0)])
def test_alpha_beta(ora, m, c_pad):
    A, B, C0, got, _ = run(ora, m, 100, 96, "T", "N", alpha=-2.5, beta=0.75, seed=7, with_c=True, c_pad=c_pad)
    want = ora.ozaki_gemm(A, B, "T", "N", alpha=-2.5, beta=0.75, C=C0)
    mag = 2.5 * ora.gemm(np.abs(A), np.abs(B), "T", "N") + 0.75 * np.abs(C0)
    assert (np.abs(got - want) <= 16 * U * mag).all()


def test_integer_inputs_exact(ora):
    """Integers of 11 bits need two 7-bit slices; with s = 3 every dropped pair (t + u > 4)
    involves the zero third slice, so the product is exact."""
    h = hsmm()
    m, n, k = 96, 80, 512
    A = W.integers((m, k), 9, -2047, 2047, np.float64)
    B = W.integers((k, n), 10, -2047, 2047, np.float64)
    dC = dev_colmajor(np.zeros((m, n)))
    h.gemm(dev_colmajor(A), dev_colmajor(B), dC, compute=h.COMPUTE_64F_OZAKI, slices=3, bits=7)
    torch.cuda.synchronize()
    assert np.array_equal(dC.cpu().numpy(), ora.gemm_i64(A.astype(np.int64), B.astype(np.int64)).astype(np.float64))


def test_zero_rows_and_columns(ora):
    h = hsmm()
    A = W.scaled_f64((70, 50), 11); A[3, :] = 0
    B = W.scaled_f64((50, 60), 12); B[:, 5] = 0
    dC = dev_colmajor(np.full((70, 60), np.nan))
    h.gemm(dev_colmajor(A), dev_colmajor(B), dC, compute=h.COMPUTE_64F_OZAKI)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    assert (got[3, :] == 0).all() and (got[:, 5] == 0).all()
    ref = ora.gemm_rows(A, B, list(range(70)), accurate=True)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-13


def test_workspace_too_small():
    h = hsmm()
    A = h.colmajor(64, 64, torch.float64); A.zero_()
    C = h.colmajor(64, 64, torch.float64)
    with pytest.raises(h.HsmmError) as e:
        h.gemm(A, A, C, compute=h.COMPUTE_64F_OZAKI, workspace=torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert e.value.status == 3


def test_full_size_precision_sampled(ora, slice_kernel):
    """m = n = k = 8192, the benchmark's configuration: sampled rows against Dot2."""
    h = hsmm()
    A, B = W.precise_inputs()
    dA, dB = dev_colmajor(A), dev_colmajor(B)
    dC = h.colmajor(8192, 8192, torch.float64)
    h.gemm(dA, dB, dC, compute=h.COMPUTE_64F_OZAKI)
    torch.cuda.synchronize()
    rows = W.rng(17).choice(8192, size=32, replace=False)
    ref = ora.gemm_rows(A, B, rows, accurate=True)
    got = dC[torch.from_numpy(rows).cuda()].cpu().numpy()
    nw = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert nw <= 1e-13, nw
