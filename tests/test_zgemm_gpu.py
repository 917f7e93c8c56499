"""GPU parity of the complex product (Section 7 measures the method on complex data).

Native form: the FP64 pipe, four FMAs per complex multiply-add; bit-exact on integer-valued
inputs, within gamma bounds otherwise.  FP64-accurate form: the real product A' B'' of the
real form (A' = [Re, Im] rows of op(A), B'' = [[Re, Im], [-Im, Re]] columns of op(B)) by the
slice kernels; the exact anti-diagonal sums S_d left in the workspace equal the oracle's
INT64 sums of its own splitting of the same real form bit for bit, and the result meets the
normwise 1e-13 bar against Dot2.
"""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]
U = 2.0 ** -53
OPS = ["N", "T", "C"]


def dev_z(X, ld=None):
    """Column-major complex128 device copy (optionally padded leading dimension)."""
    rows, cols = X.shape
    ld = rows if ld is None else ld
    base = torch.zeros((max(cols, 1), max(ld, 1)), dtype=torch.complex128, device="cuda")
    base[:cols, :rows] = torch.from_numpy(np.ascontiguousarray(np.asarray(X, np.complex128).T)).cuda()
    return base.t()[:rows, :cols]


def host_z(x):
    return np.asfortranarray(x.cpu().numpy())


def stored(rows, cols, t):
    return (rows, cols) if t == "N" else (cols, rows)


def absmag(ora, A, B, ta, tb):
    """sum_k (|Re a| + |Im a|)(|Re b| + |Im b|): the scale of each entry's rounding errors."""
    a, b = ora.zop(A, ta), ora.zop(B, tb)
    return ora.gemm(np.abs(a.real) + np.abs(a.imag), np.abs(b.real) + np.abs(b.imag))


def int_z(shape, seed, lo, hi):
    r = W.rng(seed)
    return np.asfortranarray(r.integers(lo, hi + 1, size=shape) + 1j * r.integers(lo, hi + 1, size=shape))


# ---- native complex product -------------------------------------------------------

@pytest.mark.parametrize("ta", OPS)
@pytest.mark.parametrize("tb", OPS)
def test_native_integer_exact(ora, ta, tb):
    h = hsmm()
    m, n, k = 70, 45, 133
    A = int_z(stored(m, k, ta), 10 + ord(ta), -50, 50)
    B = int_z(stored(k, n, tb), 20 + ord(tb), -50, 50)
    dC = dev_z(np.full((m, n), np.nan + 0j), ld=m + 2)
    h.gemm(dev_z(A, ld=A.shape[0] + 1), dev_z(B), dC, ta, tb, compute=h.COMPUTE_64F_NATIVE)
    torch.cuda.synchronize()
    assert np.array_equal(host_z(dC), ora.zgemm(A, B, ta, tb))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (33, 65, 17), (128, 96, 300)])
def test_native_alpha_beta_bound(ora, m, n, k):
    h = hsmm()
    A = W.scaled_c128((m, k), 30 + m, -3, 3)
    B = W.scaled_c128((k, n), 31 + n, -3, 3)
    C0 = W.scaled_c128((m, n), 32, -3, 3)
    al, be = complex(0.75, -1.25), complex(-0.5, 2.0)
    dC = dev_z(C0)
    h.gemm(dev_z(A), dev_z(B), dC, "N", "N", alpha=al, beta=be, compute=h.COMPUTE_64F_NATIVE)
    torch.cuda.synchronize()
    want = ora.zgemm(A, B, "N", "N", al, be, C0)
    mag = (abs(al.real) + abs(al.imag)) * absmag(ora, A, B, "N", "N") + \
          (abs(be.real) + abs(be.imag)) * (np.abs(C0.real) + np.abs(C0.imag))
    gam = (2 * k + 8) * U
    err = host_z(dC) - want
    assert (np.abs(err.real) <= 2 * gam * mag).all() and (np.abs(err.imag) <= 2 * gam * mag).all()


# ---- FP64-accurate complex product ---------------------------------------------------

def plane_pitch(elems, z):
    return ((elems * z + 255) // 256 * 256 + 1024) // z


def real_form_workspace(ws, m, n, k, s):
    """Views of the workspace of the complex form: the real layout with n -> 2n, k -> 2k."""
    n2, k2 = 2 * n, 2 * k
    up = lambda v: (v + 255) // 256 * 256
    kq = (k2 + 7) // 8 * 8
    pa, pb, ps = plane_pitch(m * kq, 2), plane_pitch(n2 * kq, 2), plane_pitch(m * n2, 4)
    off = 0
    qa = off; off = up(off + s * pa * 2)
    qb = off; off = up(off + s * pb * 2)
    ea = off; off = up(off + m * 4)
    eb = off; off = up(off + n2 * 4)
    sd = off
    planes = ws[sd:sd + s * ps * 4].view(torch.int32).view(s, ps)[:, :m * n2]
    return (planes.reshape(s, n2, m), ws[ea:ea + 4 * m].view(torch.int32), ws[eb:eb + 4 * n2].view(torch.int32))


def run_z(h, A, B, ta, tb, m, n, alpha=1.0, beta=0.0, C0=None, s=7, bits=7, c_pad=1):
    cfg = h.hsmm.make_config(h.C_64F, h.C_64F, h.C_64F, h.COMPUTE_64F_OZAKI, s, bits)
    k = A.shape[1] if ta == "N" else A.shape[0]
    ws = torch.zeros(h.workspace_size(cfg, ta, tb, m, n, k), dtype=torch.uint8, device="cuda")
    dC = dev_z(C0 if C0 is not None else np.full((m, n), np.nan + 0j), ld=m + c_pad)
    h.gemm(dev_z(A, ld=A.shape[0] + 1), dev_z(B), dC, ta, tb, alpha=alpha, beta=beta,
           compute=h.COMPUTE_64F_OZAKI, slices=s, bits=bits, workspace=ws)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return host_z(dC), ws


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("C", "N"), ("N", "C"), ("C", "T"),
                                   ("T", "C"), ("C", "C")])
@pytest.mark.parametrize("m,n,k", [(64, 48, 40), (129, 70, 301), (1, 1, 1)])
def test_accurate_diagonal_sums_bitexact(ora, ta, tb, m, n, k):
    h = hsmm()
    A = W.scaled_c128(stored(m, k, ta), 40 + m + k)
    B = W.scaled_c128(stored(k, n, tb), 41 + n + k)
    got, ws = run_z(h, A, B, ta, tb, m, n)
    sd, ea, eb = real_form_workspace(ws, m, n, k, 7)
    Ap, Bpp = ora.zembed(A, B, ta, tb)
    e_a, e_b, sd_ref = ora.ozaki_diagonals(Ap, Bpp, "N", "N", 7, 7)
    assert np.array_equal(ea.cpu().numpy(), e_a)
    assert np.array_equal(eb.cpu().numpy()[:n], e_b[:n])
    assert np.array_equal(sd.cpu().numpy().transpose(0, 2, 1).astype(np.int64), sd_ref)
    want = ora.ozaki_gemm(Ap, Bpp, beta_bits=7, s=7)
    want = want[:, :n] + 1j * want[:, n:]
    mag = absmag(ora, A, B, ta, tb)
    err = got - want
    assert (np.abs(err.real) <= 16 * U * mag).all() and (np.abs(err.imag) <= 16 * U * mag).all()


@pytest.mark.parametrize("bits,s", [(7, 7), (6, 9)])
def test_accurate_normwise_vs_dot2(ora, bits, s):
    h = hsmm()
    m, n, k = 160, 96, 1024
    A, B = W.scaled_c128((m, k), 50 + s), W.scaled_c128((k, n), 51 + s)
    got, _ = run_z(h, A, B, "N", "N", m, n, s=s, bits=bits, c_pad=0)
    ref = ora.zgemm_rows(A, B, list(range(m)))
    nw = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert nw <= 1e-13, nw


def test_accurate_alpha_beta(ora):
    h = hsmm()
    m, n, k = 96, 80, 200
    A, B = W.scaled_c128((k, m), 60), W.scaled_c128((k, n), 61)
    C0 = W.scaled_c128((m, n), 62)
    al, be = complex(-1.5, 0.25), complex(0.5, -0.75)
    got, ws = run_z(h, A, B, "C", "N", m, n, alpha=al, beta=be, C0=C0)
    Ap, Bpp = ora.zembed(A, B, "C", "N")
    P = ora.ozaki_gemm(Ap, Bpp, beta_bits=7, s=7)
    P = P[:, :n] + 1j * P[:, n:]
    want = al * P + be * C0
    mag = (abs(al.real) + abs(al.imag)) * absmag(ora, A, B, "C", "N") + \
          (abs(be.real) + abs(be.imag)) * (np.abs(C0.real) + np.abs(C0.imag))
    err = got - want
    assert (np.abs(err.real) <= 16 * U * mag).all() and (np.abs(err.imag) <= 16 * U * mag).all()


def test_accurate_integer_inputs_exact(ora):
    """Integer parts of up to 11 bits need two 7-bit slices; with s = 3 the product is exact."""
    h = hsmm()
    m, n, k = 72, 40, 256
    A, B = int_z((m, k), 70, -2047, 2047), int_z((k, n), 71, -2047, 2047)
    got, _ = run_z(h, A, B, "N", "N", m, n, s=3, c_pad=0)
    assert np.array_equal(got, ora.zgemm(A, B))


def test_accurate_workspace_and_early_outs(ora):
    h = hsmm()
    A = dev_z(W.scaled_c128((32, 16), 80))
    B = dev_z(W.scaled_c128((16, 24), 81))
    C0 = W.scaled_c128((32, 24), 82)
    dC = dev_z(C0)
    with pytest.raises(h.HsmmError) as e:
        h.gemm(A, B, dC, compute=h.COMPUTE_64F_OZAKI, workspace=torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert e.value.status == 3
    h.gemm(A, B, dC, alpha=0.0, beta=complex(0, 1), compute=h.COMPUTE_64F_OZAKI)   # C = i C
    torch.cuda.synchronize()
    assert np.array_equal(host_z(dC), 1j * C0)


def test_full_size_sampled(ora):
    """The 4096^3 complex precision workload, 8 sampled rows against Dot2."""
    h = hsmm()
    A, B = W.zprecise_inputs()
    m, n = A.shape[0], B.shape[1]
    got, _ = run_z(h, A, B, "N", "N", m, n, c_pad=0)
    rows = W.rng(83).choice(m, size=8, replace=False)
    ref = ora.zgemm_rows(A, B, rows)
    nw = np.linalg.norm(got[rows] - ref) / np.linalg.norm(ref)
    assert nw <= 1e-13, nw
