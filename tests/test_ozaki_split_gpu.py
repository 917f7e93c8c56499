"""GPU splitting step of the FP64-accurate form: bit-exact against the oracle's splitting."""
import numpy as np
import pytest
import torch

import workloads as W
from _gpu import dev_colmajor, hsmm, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.mark.parametrize("by_rows", [True, False])
@pytest.mark.parametrize("bits,s", [(7, 7), (6, 9), (5, 10)])
@pytest.mark.parametrize("rows,cols", [(33, 70), (256, 100), (5, 3000)])
@pytest.mark.parametrize("q_off", [0, 1])
def test_split_bitexact(ora, by_rows, bits, s, rows, cols, q_off):
    """q_off = 1 starts the slices 2 bytes past an 8-byte boundary: the one-digit-per-store
    kernels; q_off = 0 takes the four-digits-per-store kernels where the input allows."""
    h = hsmm()
    M = W.scaled_f64((rows, cols), rows + cols + bits)
    M[1, :] = 0.0
    M[:, 2] = 0.0
    nv, length = (rows, cols) if by_rows else (cols, rows)
    ldq = (length + 7) // 8 * 8
    buf = torch.empty(s * nv * ldq + q_off, dtype=torch.bfloat16, device="cuda")
    q = buf[q_off:].view(s, nv, ldq)
    expo, q = h.ozaki_split(dev_colmajor(M, ld=rows + 3), by_rows, bits, s, q=q)
    torch.cuda.synchronize()
    e_ref, q_ref = ora.ozaki_split(M, by_rows, bits, s)
    assert np.array_equal(expo.cpu().numpy(), e_ref)
    qd = q.float().cpu().numpy().astype(np.float64)      # [t][v][w]
    length = cols if by_rows else rows
    for t in range(s):
        ref_t = q_ref[t] if by_rows else q_ref[t].T          # -> [v][w]
        assert np.array_equal(qd[t, :, :length], ref_t)
        assert (qd[t, :, length:] == 0).all()


def test_split_full_size_sampled(ora):
    """The 8192 x 8192 precision workload (A by rows, B by columns), sampled lines, bit-exact."""
    h = hsmm()
    A, B = W.precise_inputs()
    ea, qa = h.ozaki_split(dev_colmajor(A), True, 7, 7)
    eb, qb = h.ozaki_split(dev_colmajor(B), False, 7, 7)
    torch.cuda.synchronize()
    lines = W.rng(3).choice(8192, size=16, replace=False)
    e_ref, q_ref = ora.ozaki_split(A[lines], True, 7, 7)
    assert np.array_equal(ea.cpu().numpy()[lines], e_ref)
    got = qa[:, torch.from_numpy(lines).cuda(), :8192].float().cpu().numpy()
    assert np.array_equal(got, q_ref)
    e_ref, q_ref = ora.ozaki_split(np.asfortranarray(B[:, lines]), False, 7, 7)
    assert np.array_equal(eb.cpu().numpy()[lines], e_ref)
    got = qb[:, torch.from_numpy(lines).cuda(), :8192].float().cpu().numpy()
    assert np.array_equal(got, np.transpose(q_ref, (0, 2, 1)))


@pytest.mark.parametrize("by_rows", [True, False])
@pytest.mark.parametrize("bits,s", [(7, 7), (6, 9)])
@pytest.mark.parametrize("q_off", [0, 1])
def test_split_extreme_lines(ora, by_rows, bits, s, q_off):
    """Lines whose largest entry is subnormal (digits then come from a left shift of the
    significand), lines mixing subnormal and normal entries, lines near the top of the FP64
    range, a zero line and negative zeros: bit-exact against the oracle's FP64 steps."""
    h = hsmm()
    rows, cols = 40, 72
    r = W.rng(77)
    M = np.asfortranarray(r.uniform(-1, 1, size=(rows, cols)) * 2.0 ** r.integers(-30, 30, size=(rows, cols)))
    tiny = 2.0 ** -1074
    if by_rows:
        M[0, :] = r.integers(-(2 ** 20), 2 ** 20, size=cols) * tiny            # all subnormal
        M[1, :] = r.integers(-3, 4, size=cols) * tiny                          # a few ulps of zero
        M[2, :] = M[2, :] * 2.0 ** -1000                                       # normal and subnormal mixed
        M[3, :] = r.uniform(-1, 1, size=cols) * 2.0 ** 1023                    # near the top of the range
        M[4, :] = 0.0
        M[5, ::2] = -0.0
    else:
        M[:, 0] = r.integers(-(2 ** 20), 2 ** 20, size=rows) * tiny
        M[:, 1] = r.integers(-3, 4, size=rows) * tiny
        M[:, 2] = M[:, 2] * 2.0 ** -1000
        M[:, 3] = r.uniform(-1, 1, size=rows) * 2.0 ** 1023
        M[:, 4] = 0.0
        M[::2, 5] = -0.0
    nv, length = (rows, cols) if by_rows else (cols, rows)
    ldq = (length + 7) // 8 * 8
    buf = torch.empty(s * nv * ldq + q_off, dtype=torch.bfloat16, device="cuda")
    q = buf[q_off:].view(s, nv, ldq)
    expo, q = h.ozaki_split(dev_colmajor(M), by_rows, bits, s, q=q)
    torch.cuda.synchronize()
    e_ref, q_ref = ora.ozaki_split(M, by_rows, bits, s)
    assert np.array_equal(expo.cpu().numpy(), e_ref)
    qd = q.float().cpu().numpy().astype(np.float64)
    for t in range(s):
        ref_t = q_ref[t] if by_rows else q_ref[t].T
        assert np.array_equal(qd[t, :, :length], ref_t)
