"""Differentiation form: backward on the library's transposed-product kernels."""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_gradcheck_fp64_64():
    """torch.autograd.gradcheck (central finite differences, FP64) at m = n = k = 64."""
    from paper_cs_9809105_gb300.autograd import HsmmMatmul
    hsmm()
    g = torch.Generator().manual_seed(3)
    a = torch.rand(64, 64, dtype=torch.float64, generator=g).cuda().requires_grad_()
    b = torch.rand(64, 64, dtype=torch.float64, generator=g).cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda x, y: HsmmMatmul.apply(x, y), (a, b), eps=2.0 ** -10, atol=1e-10,
                                    rtol=1e-9)


def test_finite_differences_against_bilinear_form(ora):
    """L = <G, A B> is bilinear: its central differences are exact up to rounding, so the
    FP64 gradient must equal them (and the oracle's G B^T, A^T G) to ~1e-10."""
    from paper_cs_9809105_gb300.autograd import hsmm_matmul
    hsmm()
    m = n = k = 64
    A = W.uniform_f64((m, k), 1); B = W.uniform_f64((k, n), 2); G = W.uniform_f64((m, n), 3)
    a = torch.from_numpy(np.ascontiguousarray(A)).cuda().requires_grad_()
    b = torch.from_numpy(np.ascontiguousarray(B)).cuda().requires_grad_()
    c = hsmm_matmul(a, b)
    c.backward(torch.from_numpy(np.ascontiguousarray(G)).cuda())
    dA = a.grad.cpu().numpy(); dB = b.grad.cpu().numpy()
    assert np.allclose(dA, ora.gemm(G, B, "N", "T"), rtol=0, atol=1e-12)
    assert np.allclose(dB, ora.gemm(A, G, "T", "N"), rtol=0, atol=1e-12)
    h = 2.0 ** -10
    L = lambda X, Y: float(np.sum(G * ora.gemm(X, Y)))
    for (i, j) in [(0, 0), (5, 17), (63, 63)]:
        Ap = A.copy(order="F"); Am = A.copy(order="F")
        Ap[i, j] += h; Am[i, j] -= h
        fd = (L(Ap, B) - L(Am, B)) / (2 * h)
        assert abs(fd - dA[i, j]) <= 1e-10 * max(1.0, abs(fd))
        Bp = B.copy(order="F"); Bm = B.copy(order="F")
        Bp[i, j] += h; Bm[i, j] -= h
        fd = (L(A, Bp) - L(A, Bm)) / (2 * h)
        assert abs(fd - dB[i, j]) <= 1e-10 * max(1.0, abs(fd))


def test_bf16_full_size_gradients_sampled(ora):
    """A 4096 x 2048, B 2048 x 8192 BF16, dC N(0,1): forward and both gradients on sampled
    rows against the FP64 oracle of the same BF16 inputs, bar k 2^-8 (|X||Y|)_ij."""
    from paper_cs_9809105_gb300.autograd import hsmm_matmul
    hsmm()
    A_bits, B_bits, G_bits = W.autograd_inputs()
    t = lambda bits: torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    a = t(A_bits).requires_grad_()
    b = t(B_bits).requires_grad_()
    c = hsmm_matmul(a, b)
    assert c.dtype == torch.bfloat16
    c.backward(t(G_bits))
    torch.cuda.synchronize()
    A = W.bf16_bits_to_f64(A_bits); B = W.bf16_bits_to_f64(B_bits); G = W.bf16_bits_to_f64(G_bits)
    rng = W.rng(4)
    # forward rows
    rows = rng.choice(4096, 8, replace=False)
    want = ora.gemm_rows(A, B, rows); mag = ora.gemm_rows(np.abs(A), np.abs(B), rows)
    got = c.detach()[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert (np.abs(got - want) <= 2048 * 2.0 ** -8 * mag).all()
    # dA = G B^T: rows of dA
    want = ora.gemm_rows(G, B, rows, "N", "T"); mag = ora.gemm_rows(np.abs(G), np.abs(B), rows, "N", "T")
    got = a.grad[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert (np.abs(got - want) <= 8192 * 2.0 ** -8 * mag).all()
    assert (np.abs(got - want) <= (2.0 ** -8 + 8192 * 2.0 ** -23) * mag).all()
    # dB = A^T G: rows of dB
    rows = rng.choice(2048, 8, replace=False)
    want = ora.gemm_rows(A, G, rows, "T", "N"); mag = ora.gemm_rows(np.abs(A), np.abs(G), rows, "T", "N")
    got = b.grad[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert (np.abs(got - want) <= 4096 * 2.0 ** -8 * mag).all()
    assert (np.abs(got - want) <= (2.0 ** -8 + 4096 * 2.0 ** -23) * mag).all()


def test_backward_after_direct_products():
    """The benchmark's sequence: direct products first, then forward + backward through autograd."""
    import paper_cs_9809105_gb300 as hh
    from paper_cs_9809105_gb300.autograd import hsmm_matmul
    hsmm()
    A_bits, B_bits, G_bits = W.autograd_inputs(m=512, k=256, n=1024)
    t = lambda bits: torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    a, b, g = t(A_bits), t(B_bits), t(G_bits)
    hh.matmul(a, b, out_dtype=torch.bfloat16)
    hh.matmul(g, b, trans_b=True, out_dtype=torch.bfloat16)
    hh.matmul(a, g, trans_a=True, out_dtype=torch.bfloat16)
    ar = a.clone().requires_grad_()
    br = b.clone().requires_grad_()
    for _ in range(2):
        ar.grad = None
        br.grad = None
        hsmm_matmul(ar, br).backward(g)
    torch.cuda.synchronize()
    want = hh.matmul(g, b, trans_b=True, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    assert torch.equal(ar.grad, want)


def test_step_captured_in_cuda_graph(ora):
    """Forward and backward captured once in a CUDA graph (as the benchmark times it) and
    replayed on new inputs copied into the captured tensors: the same bits as eager steps, and
    the eager result within the BF16 bound of the oracle."""
    from paper_cs_9809105_gb300.autograd import hsmm_matmul
    h = hsmm()
    m, k, n = 640, 384, 512
    bits = [W.uniform_bf16(s, 90 + i) for i, s in enumerate(((m, k), (k, n), (m, n), (m, k), (k, n), (m, n)))]
    t = lambda b: torch.from_numpy(np.ascontiguousarray(b).view(np.int16)).cuda().view(torch.bfloat16)
    a = t(bits[0]).requires_grad_()
    b = t(bits[1]).requires_grad_()
    g = t(bits[2])

    def step():
        a.grad = None
        b.grad = None
        hsmm_matmul(a, b).backward(g)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    with torch.no_grad():   # new inputs into the captured tensors, then one replay
        a.copy_(t(bits[3])); b.copy_(t(bits[4])); g.copy_(t(bits[5]))
    graph.replay()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    da_g, db_g = a.grad.clone(), b.grad.clone()
    step()
    torch.cuda.synchronize()
    assert torch.equal(da_g, a.grad) and torch.equal(db_g, b.grad)
    A64, B64, G64 = (W.bf16_bits_to_f64(x) for x in bits[3:])
    for got, want, mag, kk in ((a.grad, ora.gemm(G64, B64, "N", "T"), ora.gemm(np.abs(G64), np.abs(B64), "N", "T"), n),
                               (b.grad, ora.gemm(A64, G64, "T", "N"), ora.gemm(np.abs(A64), np.abs(G64), "T", "N"), m)):
        err = np.abs(got.double().cpu().numpy() - want)
        assert (err <= (2.0 ** -8 + 2 * kk * 2.0 ** -24) * mag + 1e-30).all()
