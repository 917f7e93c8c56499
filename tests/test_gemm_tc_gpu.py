"""GPU parity of the tcgen05 products (BF16 and TF32 inputs, FP32 accumulation) against the oracle.

Bar (BF16): |C - C*|_ij <= k 2^-8 (|A||B|)_ij with C* the FP64 product of the BF16
inputs; the test also holds the result to the much tighter FP32-accumulation
bound gamma_k(2^-24) (|A||B|)_ij that the tensor core should meet.
"""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_bf16_colmajor, dev_colmajor, host, hsmm, padded, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.fixture(params=["pair", "single"])
def gemm_kernel(request, monkeypatch):
    """256-wide tiles on CTA pairs (default) and on one CTA per tile."""
    monkeypatch.setenv("HSMM_GEMM_KERNEL", request.param)
    return request.param


def stored_shape(rows, cols, trans):
    return (rows, cols) if trans == "N" else (cols, rows)


def run_bf16(ora, m, n, k, ta, tb, alpha=1.0, beta=0.0, out=torch.float32, seed=0, tile_n=0, with_c0=False):
    h = hsmm()
    sa = stored_shape(m, k, ta)
    sb = stored_shape(k, n, tb)
    Ab = W.uniform_bf16(sa, 100 + seed)
    Bb = W.uniform_bf16(sb, 200 + seed)
    A64, B64 = W.bf16_bits_to_f64(Ab), W.bf16_bits_to_f64(Bb)
    dA = dev_bf16_colmajor(Ab, ld=padded(sa[0]))
    dB = dev_bf16_colmajor(Bb, ld=padded(sb[0]))
    C0 = W.uniform_f32((m, n), 300 + seed)
    if out == torch.bfloat16:
        C0 = W.bf16_bits_to_f64(W.bf16_bits_from_f32(C0)).astype(np.float32)
    dC = dev_colmajor(C0, dtype=out, ld=m + 3) if with_c0 else dev_colmajor(np.full((m, n), np.nan, np.float32), dtype=out, ld=m + 3)
    h.gemm(dA, dB, dC, ta, tb, alpha=alpha, beta=beta, tile_n=tile_n)
    torch.cuda.synchronize()
    got = host(dC)
    want = ora.gemm(A64, B64, ta, tb, alpha, beta, C0.astype(np.float64) if with_c0 else None)
    mag = ora.gemm(np.abs(A64), np.abs(B64), ta, tb, abs(alpha)) + (abs(beta) * np.abs(C0) if with_c0 else 0)
    return got, want, mag


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (256, 512, 256), (300, 500, 200), (129, 257, 65),
                                   (1, 1, 1), (17, 9, 8), (640, 384, 1000)])
def test_bf16_transposed_forms(ora, ta, tb, m, n, k, gemm_kernel):
    got, want, mag = run_bf16(ora, m, n, k, ta, tb, seed=m + n + k)
    err = np.abs(got - want)
    assert (err <= k * 2.0 ** -8 * mag + 1e-30).all()
    gam = k * 2.0 ** -24 / (1 - k * 2.0 ** -24)
    assert (err <= 2 * gam * mag + 1e-30).all(), float(np.max(err / (gam * mag + 1e-30)))


@pytest.mark.parametrize("out", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(300, 500, 200), (1500, 1300, 300), (129, 257, 65), (640, 384, 1000),
                                   (520, 72, 64), (32, 40, 16)])
def test_bf16_tma_store_epilogue(ora, ta, tb, m, n, k, out, gemm_kernel):
    """beta = 0 and a C whose leading dimension is a whole number of 16-byte units: the pair kernel
    writes C as 32 x 32 blocks through shared memory and TMA stores, clipped at the ragged edges.
    C's storage is NaN everywhere first, so a block skipped inside C or a write into the padding
    rows beyond m shows."""
    h = hsmm()
    sa = stored_shape(m, k, ta)
    sb = stored_shape(k, n, tb)
    Ab = W.uniform_bf16(sa, 400 + m + k)
    Bb = W.uniform_bf16(sb, 500 + n + k)
    A64, B64 = W.bf16_bits_to_f64(Ab), W.bf16_bits_to_f64(Bb)
    dA = dev_bf16_colmajor(Ab, ld=padded(sa[0]))
    dB = dev_bf16_colmajor(Bb, ld=padded(sb[0]))
    ldc = padded(m, 8 if out == torch.bfloat16 else 4) + (8 if out == torch.bfloat16 else 4)
    base = torch.full((n, ldc), float("nan"), dtype=out, device="cuda")
    dC = base[:, :m].t()
    h.gemm(dA, dB, dC, ta, tb)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    assert torch.isnan(base[:, m:].float()).all(), "the padding rows beyond m were written"
    got = dC.double().cpu().numpy()
    want = ora.gemm(A64, B64, ta, tb)
    mag = ora.gemm(np.abs(A64), np.abs(B64), ta, tb)
    err = np.abs(got - want)
    if out == torch.bfloat16:   # one BF16 rounding of the FP32 sum
        assert (err <= 2.0 ** -8 * np.abs(want) + 2 * k * 2.0 ** -24 * mag + 1e-30).all()
    else:
        assert (err <= 2 * k * 2.0 ** -24 * mag + 1e-30).all(), float(np.nanmax(err / (mag + 1e-30)))


@pytest.mark.parametrize("tile_n", [128, 256])
def test_bf16_tile_widths(ora, tile_n):
    got, want, mag = run_bf16(ora, 384, 640, 320, "N", "N", tile_n=tile_n, seed=tile_n)
    gam = 320 * 2.0 ** -24
    assert (np.abs(got - want) <= 2 * gam * mag).all()


def test_bf16_alpha_beta(ora, gemm_kernel):
    got, want, mag = run_bf16(ora, 200, 300, 128, "T", "N", alpha=-0.75, beta=1.25, with_c0=True, seed=5)
    gam = 130 * 2.0 ** -24
    assert (np.abs(got - want) <= 2 * gam * mag).all()


def test_bf16_out_bf16(ora, gemm_kernel):
    got, want, mag = run_bf16(ora, 256, 256, 256, "N", "T", out=torch.bfloat16, seed=6)
    # one BF16 rounding of the output on top of FP32 accumulation
    assert (np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 256 * 2.0 ** -23 * mag).all()


def test_bf16_integer_exact(ora):
    """Integer-valued BF16 inputs with all partial sums below 2^24: FP32 accumulation is exact."""
    h = hsmm()
    m, n, k = 256, 512, 1024
    A = W.integers((m, k), 41, -7, 7, np.float32)
    B = W.integers((k, n), 42, -7, 7, np.float32)
    dA = dev_colmajor(A, dtype=torch.bfloat16)
    dB = dev_colmajor(B, dtype=torch.bfloat16)
    dC = dev_colmajor(np.zeros((m, n), np.float32))
    h.gemm(dA, dB, dC)
    torch.cuda.synchronize()
    want = ora.gemm_i64(A.astype(np.int64), B.astype(np.int64))
    assert np.array_equal(host(dC).astype(np.int64), want)


def test_bf16_k_zero_and_alpha_zero(ora):
    h = hsmm()
    m, n = 64, 48
    C0 = W.uniform_f32((m, n), 50)
    dC = dev_colmajor(C0)
    dA = dev_colmajor(np.zeros((m, 8), np.float32), dtype=torch.bfloat16)
    dB = dev_colmajor(np.zeros((8, n), np.float32), dtype=torch.bfloat16)
    h.gemm(dA[:, :0], dB[:0, :], dC, beta=2.0)
    torch.cuda.synchronize()
    assert np.array_equal(host(dC), 2.0 * C0.astype(np.float64))
    h.gemm(dA, dB, dC, alpha=0.0, beta=0.0)
    torch.cuda.synchronize()
    assert (host(dC) == 0).all()


def test_bf16_unaligned_ld_not_supported():
    h = hsmm()
    A = torch.zeros((8, 15), dtype=torch.bfloat16, device="cuda").t()   # 15 x 8 with ld 15: 30 bytes
    B = h.colmajor(8, 16, torch.bfloat16)
    C = h.colmajor(15, 16, torch.float32)
    with pytest.raises(h.HsmmError) as e:
        h.gemm(A, B, C)
    assert e.value.status == 2


@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "N"), ("N", "T"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(300, 260, 192), (128, 256, 32), (129, 300, 1000), (64, 64, 8)])
def test_tf32_transposed_forms(ora, ta, tb, m, n, k, gemm_kernel):
    """TF32 products in all four operand forms: K-major operands (op(A) = A^T, op(B) = B) as
    128-byte rows of K, MN-major ones as chunks of 32 elements in the 32-byte-unit swizzle."""
    h = hsmm()
    sa = stored_shape(m, k, ta)
    sb = stored_shape(k, n, tb)
    A = W.uniform_f32(sa, 60 + m + (ta == "T"))
    B = W.uniform_f32(sb, 61 + n + (tb == "T"))
    dA = dev_colmajor(A, ld=padded(sa[0], 4))
    dB = dev_colmajor(B, ld=padded(sb[0], 4))
    dC = dev_colmajor(np.full((m, n), np.nan, np.float32))
    h.gemm(dA, dB, dC, ta, tb, compute=h.COMPUTE_32F_FAST_TF32)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    want = ora.gemm(A64, B64, ta, tb)
    mag = ora.gemm(np.abs(A64), np.abs(B64), ta, tb)
    # TF32 keeps 10 fraction bits of each input: |d(ab)| <= 2*2^-10 |a||b| (truncation), plus FP32 sums
    err = np.abs(host(dC) - want)
    assert (err <= (2.0 ** -9 + k * 2.0 ** -23) * mag).all(), float(np.max(err / (mag + 1e-30)))


def test_matmul_rowmajor_all_forms(ora):
    """Row-major entry (autograd path): C = op(a) op(b) through the column-major kernels."""
    h = hsmm()
    m, n, k = 192, 320, 136
    for ta in (False, True):
        for tb in (False, True):
            a_bits = W.uniform_bf16((k, m) if ta else (m, k), 70)
            b_bits = W.uniform_bf16((n, k) if tb else (k, n), 71)
            a = torch.from_numpy(np.ascontiguousarray(a_bits).view(np.int16)).cuda().view(torch.bfloat16)
            b = torch.from_numpy(np.ascontiguousarray(b_bits).view(np.int16)).cuda().view(torch.bfloat16)
            c = h.matmul(a, b, trans_a=ta, trans_b=tb)
            torch.cuda.synchronize()
            a64 = W.bf16_bits_to_f64(a_bits)
            b64 = W.bf16_bits_to_f64(b_bits)
            opa = a64.T if ta else a64
            opb = b64.T if tb else b64
            want = ora.gemm(np.asfortranarray(opa), np.asfortranarray(opb))
            mag = ora.gemm(np.abs(np.asfortranarray(opa)), np.abs(np.asfortranarray(opb)))
            assert (np.abs(c.double().cpu().numpy() - want) <= 2 * k * 2.0 ** -24 * mag).all(), (ta, tb)


def test_full_size_autograd_forward_sampled(ora, gemm_kernel):
    """The 4096 x 2048 x 8192 forward in the benchmark's launch configuration, sampled rows vs the oracle."""
    h = hsmm()
    A_bits, B_bits, _ = W.autograd_inputs()
    a = torch.from_numpy(A_bits.view(np.int16)).cuda().view(torch.bfloat16)
    b = torch.from_numpy(B_bits.view(np.int16)).cuda().view(torch.bfloat16)
    c = h.matmul(a, b)
    torch.cuda.synchronize()
    rows = W.rng(5).choice(4096, size=24, replace=False)
    A64 = np.asfortranarray(W.bf16_bits_to_f64(A_bits))
    B64 = np.asfortranarray(W.bf16_bits_to_f64(B_bits))
    want = ora.gemm_rows(A64, B64, rows)
    mag = ora.gemm_rows(np.abs(A64), np.abs(B64), rows)
    got = c[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert (np.abs(got - want) <= 2048 * 2.0 ** -8 * mag).all()
    assert (np.abs(got - want) <= 2 * 2048 * 2.0 ** -24 * mag).all()
