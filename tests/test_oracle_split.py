"""Pins of the split-BF16 encoding oracle (CPU only)."""
import numpy as np
import pytest
import torch

from oracle import split_oracle as SO


def test_bf16_rounding_matches_torch_conversion():
    rng = np.random.default_rng(14)
    v = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38, 1e-40, -2.5],
                                 dtype=np.float32)]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(SO.bf16_round_bits(v), ref)


def test_split_error_bound_and_scale():
    rng = np.random.default_rng(15)
    A = (rng.uniform(0.0, 1.0, (64, 16)) * 10.0 ** rng.uniform(-12, 0, (1, 16))).astype(np.float32)
    scale = np.array([SO.pow2_scale_at_least(float(m)) for m in A.max(axis=0)])
    for s_, m in zip(scale, A.max(axis=0)):
        assert m <= s_ < 2 * m and np.log2(s_) == np.round(np.log2(s_))
    hi, lo = SO.split_columns(A, scale)
    dec = SO.decode(hi, lo, scale)
    assert np.all(np.abs(dec - A.astype(np.float64)) <= 2.0 ** -17 * np.abs(A.astype(np.float64)))
    assert np.all(np.abs(SO.bf16_bits_to_float(hi)) <= 1.0)


@pytest.mark.parametrize("m", [1.0, 0.75, 3.0e-9, 2.0 ** -20])
def test_pow2_scale(m):
    s = SO.pow2_scale_at_least(m)
    assert m <= s < 2 * m


def test_bf16_hi_alone_error_bound_is_2_to_minus_8_and_attained():
    """BF16 storage keeps hi alone: |sigma hi - A| <= 2^-8 |A| (round to nearest with an 8-bit
    significand: half an ulp of 2^-7 relative spacing), and values near a rounding midpoint just
    above a power of two come within 2% of that bound, so a row dominated by one element can
    carry a bound-relative image error near 2^-8 (3.9e-3)."""
    rng = np.random.default_rng(16)
    A = (rng.uniform(0.0, 1.0, (4096, 8)) * 10.0 ** rng.uniform(-12, 0, (1, 8))).astype(np.float32)
    scale = np.array([SO.pow2_scale_at_least(float(m)) for m in A.max(axis=0)])
    hi, _ = SO.split_columns(A, scale)
    dec = SO.decode(hi, np.zeros_like(hi), scale)
    rel = np.abs(dec - A.astype(np.float64)) / np.abs(A.astype(np.float64))
    assert rel.max() <= 2.0 ** -8
    assert rel.max() >= 0.98 * 2.0 ** -8
