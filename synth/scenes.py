"""Synthetic exozodiacal ring scenes with point planets (input preparation only).

Stands in for the ZODIPIC scenes of Sec. 2 (not available).  A scene is N x N
at S lambda0/D per pixel, flattened row-major (j = iy*N + ix), pixel centres at
((ix - (N-1)/2) S, (iy - (N-1)/2) S), masked beyond r_max (the paper masks its
scenes beyond the outer working angle, Sec. 2).

Ring brightness (optically thin, smooth in every parameter):
  disk-plane coordinates xd = x, yd = y / cos(i), rd = hypot(xd, yd);
  I = B * exp(-4 ln2 (rd - R)^2 / w^2) * HG_g(mu) / HG_g(0),  mu = sin(i) yd / rd,
  HG_g(mu) = (1 - g^2) / (4 pi (1 + g^2 - 2 g mu)^1.5)   (Henyey-Greenstein).
w is the full width at half maximum of the radial profile.
"""
from __future__ import annotations

import numpy as np


def pixel_centres(N: int, S: float) -> tuple[np.ndarray, np.ndarray]:
    c = (np.arange(N, dtype=np.float64) - (N - 1) / 2.0) * S
    X, Y = np.meshgrid(c, c, indexing="xy")
    return X, Y


def ring_image(N: int, S: float, R: float, w: float, inc: float, g: float, B: float,
               r_max: float) -> np.ndarray:
    """N x N ring brightness (float64); inc in radians."""
    X, Y = pixel_centres(N, S)
    xd = X
    yd = Y / np.cos(inc)
    rd = np.hypot(xd, yd)
    radial = np.exp(-4.0 * np.log(2.0) * (rd - R) ** 2 / (w * w))
    safe = np.where(rd > 0.0, rd, 1.0)
    mu = np.where(rd > 0.0, np.sin(inc) * yd / safe, 0.0)
    phase = ((1.0 + g * g) / (1.0 + g * g - 2.0 * g * mu)) ** 1.5
    img = B * radial * phase
    img[np.hypot(X, Y) > r_max] = 0.0
    return img


def add_planets(img: np.ndarray, S: float, rng: np.random.Generator, count: int,
                flux_lo: float, flux_hi: float, r_lo: float = 3.0, r_hi: float = 9.0,
                log_uniform: bool = True) -> list[tuple[int, int, float]]:
    """Add `count` single-pixel planets at seeded pixel centres with r_lo <= r <= r_hi."""
    N = img.shape[0]
    X, Y = pixel_centres(N, S)
    rr = np.hypot(X, Y)
    iy, ix = np.nonzero((rr >= r_lo) & (rr <= r_hi))
    placed = []
    for _ in range(count):
        t = int(rng.integers(len(iy)))
        if log_uniform:
            f = float(np.exp(rng.uniform(np.log(flux_lo), np.log(flux_hi))))
        else:
            f = float(rng.uniform(flux_lo, flux_hi))
        img[iy[t], ix[t]] += f
        placed.append((int(iy[t]), int(ix[t]), f))
    return placed
