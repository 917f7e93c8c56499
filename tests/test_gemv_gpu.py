"""GPU parity of hsmm_gemv against the oracle (FP32: gamma_n bound; INT8: bit-exact)."""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_colmajor, hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

U32 = 2.0 ** -24


def gamma(n, u=U32):
    return n * u / (1 - n * u)


def check_f32(ora, A, x, trans, alpha, beta, y0, got, incx=1, incy=1):
    want = ora.gemv(A.astype(np.float64), x.astype(np.float64), trans, alpha, beta,
                    None if y0 is None else y0.astype(np.float64), incx, incy)
    absA = np.abs(A.astype(np.float64))
    mag = ora.gemv(absA, np.abs(x.astype(np.float64)), trans, abs(alpha), 0.0, None, incx, 1)
    n = A.shape[1] if trans == "N" else A.shape[0]
    ys = got[::incy]
    ws = want[::incy]
    yb = 0 if y0 is None else np.abs(y0[::incy].astype(np.float64)) * abs(beta)
    bound = (gamma(n + 2)) * (mag + yb) + 1e-38
    assert (np.abs(ys - ws) <= bound).all(), float(np.max(np.abs(ys - ws) / bound))


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("m,n", [(1, 1), (7, 5), (64, 33), (1000, 777), (4096, 300), (129, 4100)])
def test_gemv_f32_shapes(ora, trans, m, n):
    h = hsmm()
    A = W.uniform_f32((m, n), 1 + m + n)
    lenx, leny = (n, m) if trans == "N" else (m, n)
    x = W.uniform_f32((lenx,), 2 + m)
    dA = dev_colmajor(A)
    dx = torch.from_numpy(x).cuda()
    dy = torch.zeros(leny, dtype=torch.float32, device="cuda")
    h.gemv(dA, dx, dy, trans)
    torch.cuda.synchronize()
    check_f32(ora, A, x, trans, 1.0, 0.0, None, dy.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_f32_alpha_beta_strides(ora, trans):
    h = hsmm()
    m, n = 300, 200
    A = W.uniform_f32((m, n), 7)
    lenx, leny = (n, m) if trans == "N" else (m, n)
    x = W.uniform_f32((lenx * 2,), 8)
    y0 = W.uniform_f32((leny * 3,), 9)
    dA = dev_colmajor(A, ld=m + 5)
    dx = torch.from_numpy(x).cuda()
    dy = torch.from_numpy(y0.copy()).cuda()
    h.gemv(dA, dx, dy, trans, alpha=-1.5, beta=0.5, incx=2, incy=3)
    torch.cuda.synchronize()
    got = dy.cpu().numpy().astype(np.float64)
    check_f32(ora, A, x, trans, -1.5, 0.5, y0, got, incx=2, incy=3)
    # elements between the strided outputs are untouched
    mask = np.ones(leny * 3, bool); mask[::3] = False
    assert np.array_equal(got[mask], y0[mask].astype(np.float64))


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_f32_beta_zero_ignores_nan(ora, trans):
    h = hsmm()
    A = W.uniform_f32((96, 80), 10)
    lenx, leny = (80, 96) if trans == "N" else (96, 80)
    x = W.uniform_f32((lenx,), 11)
    dy = torch.full((leny,), float("nan"), device="cuda")
    h.gemv(dev_colmajor(A), torch.from_numpy(x).cuda(), dy, trans, beta=0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(dy).all()


@pytest.mark.parametrize("trans", ["N", "T"])
@pytest.mark.parametrize("m,n", [(16, 4), (48, 7), (1024, 999), (4096, 2048), (33, 65), (1, 1)])
def test_gemv_i8_bitexact(ora, trans, m, n):
    h = hsmm()
    A = W.integers((m, n), 20 + m, -128, 127, np.int8)
    lenx, leny = (n, m) if trans == "N" else (m, n)
    x = W.integers((lenx,), 21 + n, -128, 127, np.int8)
    y0 = W.integers((leny,), 22, -100, 100, np.int32)
    dy = torch.from_numpy(y0.copy()).cuda()
    h.gemv(dev_colmajor(A), torch.from_numpy(x).cuda(), dy, trans, alpha=3, beta=-2)
    torch.cuda.synchronize()
    want = ora.gemv_i8(A, x, trans, 3, -2, y0)
    assert np.abs(want).max() < 2 ** 31
    assert np.array_equal(dy.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_full_size_f32(ora, trans):
    """The 16384 x 16384 FP32 workload, same launch configuration as the benchmark; all outputs checked."""
    h = hsmm()
    A, xs = W.gemv_inputs()
    x = xs[:16384]
    dA = dev_colmajor(A)
    dx = torch.from_numpy(x).cuda()
    dy = torch.zeros(16384, device="cuda")
    h.gemv(dA, dx, dy, trans)
    torch.cuda.synchronize()
    check_f32(ora, A, x, trans, 1.0, 0.0, None, dy.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("trans", ["N", "T"])
def test_gemv_full_size_i8(ora, trans):
    h = hsmm()
    A, xs = W.gemv_i8_inputs()
    x = xs[:16384]
    dy = torch.zeros(16384, dtype=torch.int32, device="cuda")
    h.gemv(dev_colmajor(A), torch.from_numpy(x).cuda(), dy, trans)
    torch.cuda.synchronize()
    assert np.array_equal(dy.cpu().numpy().astype(np.int64), ora.gemv_i8(A, x, trans))


def test_gemv_i8_extreme_values(ora):
    # every entry -128: the largest |sum| of the 16384 workload (2^28), exact in INT32
    h = hsmm()
    n = 16384
    A = np.full((64, n), -128, dtype=np.int8, order="F")
    x = np.full(n, -128, dtype=np.int8)
    for trans, leny in (("N", 64),):
        dy = torch.zeros(leny, dtype=torch.int32, device="cuda")
        h.gemv(dev_colmajor(A), torch.from_numpy(x).cuda(), dy, trans)
        torch.cuda.synchronize()
        assert (dy.cpu().numpy() == n * 128 * 128).all()
    At = np.full((n, 64), -128, dtype=np.int8, order="F")
    dy = torch.zeros(64, dtype=torch.int32, device="cuda")
    h.gemv(dev_colmajor(At), torch.from_numpy(x).cuda(), dy, "T")
    torch.cuda.synchronize()
    assert (dy.cpu().numpy() == n * 128 * 128).all()


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_gemv_n_deterministic_and_graph_capture(ora, dtype):
    """op = N adds the column splits in a fixed order: repeated calls agree bit for bit, and the
    split kernel with its programmatically dependent reduction replays from a CUDA graph."""
    h = hsmm()
    m, n = 4096, 3000
    if dtype == "f32":
        A = W.uniform_f32((m, n), 41)
        x = W.uniform_f32((n,), 42)
        dA, dx = dev_colmajor(A), torch.from_numpy(x).cuda()
        ydt = torch.float32
    else:
        A = W.integers((m, n), 43, -128, 127, np.int8)
        x = W.integers((n,), 44, -128, 127, np.int8)
        dA, dx = dev_colmajor(A, dtype=torch.int8), torch.from_numpy(x).cuda()
        ydt = torch.int32
    y1 = torch.zeros(m, dtype=ydt, device="cuda")
    y2 = torch.zeros(m, dtype=ydt, device="cuda")
    h.gemv(dA, dx, y1)
    h.gemv(dA, dx, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    y3 = torch.zeros(m, dtype=ydt, device="cuda")
    ws = torch.empty(h.hsmm.gemv_workspace_size(h.R_32F if dtype == "f32" else h.R_8I, "N", m, n),
                     dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        h.gemv(dA, dx, y3, workspace=ws)          # warm-up outside capture
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            h.gemv(dA, dx, y3, workspace=ws)
    y3.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y1, y3)
    if dtype == "i8":
        assert np.array_equal(y1.cpu().numpy().astype(np.int64), ora.gemv_i8(A, x, "N"))
