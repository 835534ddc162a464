"""Split-BF16 encoding of a matrix column by column (TEST INFRASTRUCTURE ONLY).

Storage form of A used by the batched tensor-core path (not in the paper, whose
A is FP64, Table 2): per column j a power-of-two scale sigma_j, then
hi = RN_bf16(A_ij / sigma_j), lo = RN_bf16(A_ij / sigma_j - hi), so that
A_ij ~= sigma_j (hi + lo).  RN_bf16 is round-to-nearest-even to 8 significant
bits, written here on the float32 bit pattern.  For float32 input the residual
A/sigma - hi is exact in float32, and |A/sigma - hi - lo| <= 2^-17 |A/sigma|.
"""
from __future__ import annotations

import numpy as np


def bf16_round_bits(v: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); returns uint16 bits."""
    u = np.ascontiguousarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    rounded = (u + 0x7FFF + lsb) >> 16
    nan = np.isnan(np.asarray(v, dtype=np.float32))
    out = (rounded & 0xFFFF).astype(np.uint16)
    out[nan] = 0x7FC0
    return out


def bf16_bits_to_float(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def pow2_scale_at_least(m: float) -> float:
    """Smallest power of two >= m (1.0 for m == 0)."""
    if m <= 0.0:
        return 1.0
    e = int(np.ceil(np.log2(m)))
    s = 2.0 ** e
    if s < m:
        s *= 2.0
    while s / 2.0 >= m:
        s /= 2.0
    return s


def split_columns(A32: np.ndarray, col_scale: np.ndarray):
    """(hi_bits, lo_bits) of float32 A scaled by 1/col_scale per column (exact powers of two)."""
    A32 = np.asarray(A32, dtype=np.float32)
    scaled = (A32 / np.asarray(col_scale, dtype=np.float32)[None, :]).astype(np.float32)
    hi = bf16_round_bits(scaled)
    resid = (scaled - bf16_bits_to_float(hi)).astype(np.float32)
    lo = bf16_round_bits(resid)
    return hi, lo


def decode(hi_bits, lo_bits, col_scale) -> np.ndarray:
    v = bf16_bits_to_float(hi_bits).astype(np.float64) + bf16_bits_to_float(lo_bits)
    return v * np.asarray(col_scale, dtype=np.float64)[None, :]
