"""The synthetic-input recipe and the binding's host helpers (no GPU).

The inputs stand in for the paper's workloads; these tests pin their seeds, ranges and
distributions, and the BF16 rounding the tensor-core inputs go through."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_cs_9809105_gb300 import hsmm as H


def test_generators_are_deterministic_and_column_major():
    for gen in (lambda: W.uniform_f64((33, 17), 5), lambda: W.uniform_f32((33, 17), 5),
                lambda: W.scaled_f64((33, 17), 5), lambda: W.integers((33, 17), 5, -128, 127, np.int8)):
        a, b = gen(), gen()
        assert np.array_equal(a, b) and np.isfortran(a)
    assert not np.array_equal(W.uniform_f64((8, 8), 1), W.uniform_f64((8, 8), 2))


def test_scaled_entries_follow_the_precision_recipe():
    x = W.scaled_f64((256, 256), W.SEED_PRECISE)
    mant, e = np.frexp(np.abs(x))          # |x| = mant 2^e with mant in [0.5, 1): s 2^e' has e = e' + 1
    assert np.all((e - 1 >= -12) & (e - 1 <= 12))
    assert set(np.unique(e - 1)) == set(range(-12, 13))       # every exponent occurs
    assert 0.45 < np.mean(x > 0) < 0.55                       # fair signs


def test_integer_inputs_cover_the_int8_range():
    a = W.integers((512, 512), W.SEED_GEMV, -128, 127, np.int8)
    assert a.dtype == np.int8 and a.min() == -128 and a.max() == 127


def test_grouped_shapes_log_uniform():
    sh = W.grouped_shapes()
    assert sh.shape == (512, 3) and sh.min() >= 64 and sh.max() <= 2048
    logs = np.log(sh.astype(np.float64))
    # log-uniform on [log 64, log 2048]: mean at the midpoint, variance (range^2 / 12)
    mid, rng2 = (np.log(64) + np.log(2048)) / 2, (np.log(2048) - np.log(64)) ** 2 / 12
    assert abs(logs.mean() - mid) < 0.1 and abs(logs.var() - rng2) / rng2 < 0.15
    assert np.array_equal(sh, W.grouped_shapes())


def test_bf16_rounding_is_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 3.0e38, 1e-40], np.float32)
    back = W.bf16_bits_to_f64(W.bf16_bits_from_f32(vals))
    # halfway cases go to the even neighbour; everything else to the nearest BF16 value
    assert back[0] == 1.0 and back[1] == 1.0 and back[2] == 1.0 + 4 * 2 ** -8 and back[3] == 1.0
    assert back[4] == -2.5
    ref = torch.from_numpy(vals).to(torch.bfloat16).double().numpy()
    assert np.array_equal(back, ref)


def test_uniform_bf16_values_are_exact_bf16():
    bits = W.uniform_bf16((64, 64), 9)
    v = W.bf16_bits_to_f64(bits)
    assert np.all(np.abs(v) <= 1.0)
    assert np.array_equal(W.bf16_bits_from_f32(v.astype(np.float32)), bits)


def test_pad_ld():
    assert [W.pad_ld(r) for r in (1, 8, 9, 300)] == [8, 8, 16, 304]
    assert [W.pad_ld(r, 4) for r in (1, 4, 5)] == [4, 4, 8]


def test_binding_leading_dimension_and_ops():
    c = H.colmajor(5, 3, torch.float32, device="cpu", ld=8)
    assert c.shape == (5, 3) and c.stride() == (1, 8) and H._ld(c) == 8
    row = H.colmajor(1, 4, torch.float32, device="cpu")
    assert H._ld(row) == 1
    with pytest.raises(ValueError):
        H._ld(torch.empty(4, 5))                  # row-major: not column-major
    x = torch.arange(12.0).reshape(3, 4)
    y = H.to_colmajor(x.to("cpu"))
    assert torch.equal(y, x) and y.stride()[0] == 1
    assert (H._op("n"), H._op("T"), H._op("c")) == (ord("N"), ord("T"), ord("C"))
    with pytest.raises(ValueError):
        H._op("X")


def test_binding_scalar_cache_is_bounded():
    a = H._scalar_cached(1.0, H.R_32F)
    assert a is H._scalar_cached(1.0, H.R_32F) and a.value == 1.0
    for i in range(200):
        assert H._scalar_cached(float(i) + 0.5, H.R_64F).value == float(i) + 0.5
    assert len(H._SCALARS) <= 64
    z = H._scalar_cached(complex(1, -2), H.C_64F)
    assert (z[0], z[1]) == (1.0, -2.0)
