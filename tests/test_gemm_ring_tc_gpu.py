"""GPU parity of the ring order of Algorithm 2 on thread-block clusters (tensor-core products).

A cluster of p CTAs is the ring: A blocks move by cshift-row^K between the CTAs, each CTA
keeps K auxiliary accumulators, and the back-shift C^(l-1) += cshift-row^1(C^l) folds them.
(1) Integer-valued BF16 inputs whose partial sums stay below 2^24 make FP32 accumulation
exact, so the result equals the oracle's INT64 product bit for bit only if every block
product A_rk B_kq is accumulated exactly once into the right block of C (Section 5.2.2,
the coverage of the distances by the base).  (2) Random inputs meet the FP32-accumulation
bound against the FP64 oracle of the same BF16 inputs.
"""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_bf16_colmajor, dev_colmajor, host, hsmm, padded, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

PK = [(2, 1), (2, 2), (4, 1), (4, 2), (4, 4), (8, 1), (8, 2), (8, 4), (16, 1), (16, 2), (16, 4)]


def stored_shape(rows, cols, trans):
    return (rows, cols) if trans == "N" else (cols, rows)


def ring_gemm(A, B, C, ta, tb, p, K, **kw):
    h = hsmm()
    try:
        h.gemm(A, B, C, ta, tb, ring_p=p, ring_k=K, **kw)
    except h.HsmmError as e:
        if p == 16 and e.status == 2:
            pytest.skip("this GPU holds no cluster of 16 CTAs with the ring kernel's shared memory")
        raise
    torch.cuda.synchronize()
    assert h.sync_status() == 0


@pytest.mark.parametrize("p,K", PK)
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_integer_exact(ora, p, K, ta, tb):
    """Every block product exactly once: bit-exact against the INT64 product."""
    m, n, k = 200, 128 * p + 72, 64 * p * 2 + 40          # ragged in every dimension, > 1 round
    sa, sb = stored_shape(m, k, ta), stored_shape(k, n, tb)
    A = W.integers(sa, 500 + p + K, -15, 15, np.float32)
    B = W.integers(sb, 600 + p + K, -15, 15, np.float32)
    dA = dev_colmajor(A, dtype=torch.bfloat16, ld=padded(sa[0]))
    dB = dev_colmajor(B, dtype=torch.bfloat16, ld=padded(sb[0]))
    dC = dev_colmajor(np.full((m, n), np.nan, np.float32), ld=m + 1)
    ring_gemm(dA, dB, dC, ta, tb, p, K)
    want = ora.gemm_i64(A.astype(np.int64), B.astype(np.int64), ta, tb)
    assert np.array_equal(host(dC).astype(np.int64), want)


@pytest.mark.parametrize("p,K", [(4, 2), (8, 4), (16, 4), (2, 1)])
@pytest.mark.parametrize("m,n,k", [(128, 512, 64), (129, 1100, 1000), (1, 1, 1), (300, 700, 4096)])
def test_random_fp32_bound(ora, p, K, m, n, k):
    Ab, Bb = W.uniform_bf16((m, k), 700 + m), W.uniform_bf16((k, n), 800 + n)
    A64, B64 = W.bf16_bits_to_f64(Ab), W.bf16_bits_to_f64(Bb)
    dA, dB = dev_bf16_colmajor(Ab, ld=padded(m)), dev_bf16_colmajor(Bb, ld=padded(k))
    dC = dev_colmajor(np.full((m, n), np.nan, np.float32))
    ring_gemm(dA, dB, dC, "N", "N", p, K)
    want = ora.gemm(A64, B64)
    mag = ora.gemm(np.abs(A64), np.abs(B64))
    gam = (k + K) * 2.0 ** -24 / (1 - (k + K) * 2.0 ** -24)     # k products plus K - 1 back-shift additions
    assert (np.abs(host(dC) - want) <= 2 * gam * mag + 1e-30).all()


@pytest.mark.parametrize("p,K", [(4, 2), (8, 1)])
def test_alpha_beta(ora, p, K):
    m, n, k = 256, 600, 512
    Ab, Bb = W.uniform_bf16((k, m), 901), W.uniform_bf16((k, n), 902)
    A64, B64 = W.bf16_bits_to_f64(Ab), W.bf16_bits_to_f64(Bb)
    C0 = W.uniform_f32((m, n), 903)
    dA, dB = dev_bf16_colmajor(Ab), dev_bf16_colmajor(Bb)
    dC = dev_colmajor(C0, ld=m + 5)
    ring_gemm(dA, dB, dC, "T", "N", p, K, alpha=-1.5, beta=0.5)
    want = ora.gemm(A64, B64, "T", "N", -1.5, 0.5, C0.astype(np.float64))
    mag = 1.5 * ora.gemm(np.abs(A64), np.abs(B64), "T", "N") + 0.5 * np.abs(C0)
    gam = (k + 4) * 2.0 ** -24
    assert (np.abs(host(dC) - want) <= 2 * gam * mag).all()


def test_same_as_persistent_order_on_integers(ora):
    """Ring order and persistent order agree bit for bit where both are exact."""
    h = hsmm()
    m, n, k = 384, 1024, 2048
    A = W.integers((m, k), 910, -3, 3, np.float32)
    B = W.integers((k, n), 911, -3, 3, np.float32)
    dA, dB = dev_colmajor(A, dtype=torch.bfloat16), dev_colmajor(B, dtype=torch.bfloat16)
    c1 = dev_colmajor(np.zeros((m, n), np.float32))
    c2 = dev_colmajor(np.zeros((m, n), np.float32))
    h.gemm(dA, dB, c1)
    ring_gemm(dA, dB, c2, "N", "N", 8, 2)
    assert torch.equal(c1, c2)


def test_full_size_sampled(ora):
    """The 8192^3 BF16 product the ring-order comparison times, 16 sampled rows."""
    m = n = k = 8192
    Ab, Bb = W.uniform_bf16((m, k), 920), W.uniform_bf16((k, n), 921)
    dA, dB = dev_bf16_colmajor(Ab), dev_bf16_colmajor(Bb)
    dC = dev_colmajor(np.zeros((m, n), np.float32))
    ring_gemm(dA, dB, dC, "N", "N", 8, 2)
    rows = W.rng(922).choice(m, size=16, replace=False)
    A64 = W.bf16_bits_to_f64(Ab[rows])
    B64 = W.bf16_bits_to_f64(Bb)
    want = ora.gemm(np.asfortranarray(A64), B64)
    mag = ora.gemm(np.asfortranarray(np.abs(A64)), np.abs(B64))
    got = dC[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    gam = (k + 2) * 2.0 ** -24
    assert (np.abs(got - want) <= 2 * gam * mag).all()


def test_bad_arguments():
    h = hsmm()
    A = h.colmajor(128, 64, torch.bfloat16)
    B = h.colmajor(64, 128, torch.bfloat16)
    C = h.colmajor(128, 128, torch.float32)
    for p, K in ((3, 1), (4, 3), (2, 4), (32, 4), (8, 8)):
        with pytest.raises(h.HsmmError) as e:
            h.gemm(A, B, C, ring_p=p, ring_k=K)
        assert e.value.status == 1, (p, K)
    Cb = h.colmajor(128, 128, torch.bfloat16)
    with pytest.raises(h.HsmmError) as e:
        h.gemm(A, B, Cb, ring_p=4)
    assert e.value.status == 2
