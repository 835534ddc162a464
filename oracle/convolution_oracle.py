"""FP64 direct convolution: the oracle of the convolution comparator (Sec. 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Sec. 3 compares the
matrix method with a simulation that convolves the scene with one PSF, masked
to its core and shifted to the array centre.  Written here as the plain sum
that defines a linear convolution: every scene pixel adds a copy of the
kernel, scaled by its value and shifted so that the kernel's core lands on
that pixel.  No FFT.  Pinned by tests/test_oracle_convolution.py: a single
point source reproduces the (masked) kernel, the exact shift-invariant case
equals the method's A Z, and a random case equals a zero-padded FFT product.
"""
from __future__ import annotations

import numpy as np


def masked_kernel(kernel, cp: int, cq: int, mask_radius_px=None) -> np.ndarray:
    """The kernel with entries farther than mask_radius_px from (cp, cq) set to 0."""
    g = np.array(kernel, dtype=np.float64)
    if mask_radius_px is not None:
        n = g.shape[0]
        pp, qq = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        g[(pp - cp) ** 2 + (qq - cq) ** 2 > mask_radius_px ** 2] = 0.0
    return g


def direct_convolution(scene, kernel, iy_ref: int, ix_ref: int, mask_radius_px=None) -> np.ndarray:
    """out[p, q] = sum_{iy, ix} scene[iy, ix] * g[p - iy + iy_ref, q - ix + ix_ref] on the n x n
    image grid, g the (masked) n x n kernel, entries outside g counting 0.  The scene (N x N,
    n - N even) sits on the image grid at offset o = (n - N) / 2, and the kernel's core is its
    pixel (iy_ref + o, ix_ref + o), so a point at scene pixel (iy_ref, ix_ref) reproduces g."""
    scene = np.asarray(scene, dtype=np.float64)
    n, N = kernel.shape[0], scene.shape[0]
    o = (n - N) // 2
    cp, cq = iy_ref + o, ix_ref + o
    g = masked_kernel(kernel, cp, cq, mask_radius_px)
    out = np.zeros((n, n))
    for iy, ix in zip(*np.nonzero(scene)):
        # scene pixel (iy, ix) is image pixel (iy + o, ix + o); its copy of g is shifted by
        # (iy + o - cp, ix + o - cq)
        dp, dq = iy + o - cp, ix + o - cq
        p0, p1 = max(0, dp), min(n, n + dp)
        q0, q1 = max(0, dq), min(n, n + dq)
        if p0 < p1 and q0 < q1:
            out[p0:p1, q0:q1] += scene[iy, ix] * g[p0 - dp:p1 - dp, q0 - dq:q1 - dq]
    return out


def convolution_bound(scene, kernel, iy_ref: int, ix_ref: int, mask_radius_px=None) -> np.ndarray:
    """sum of |scene| |g| over the same terms (the scale of each output's rounding error)."""
    return direct_convolution(np.abs(scene), np.abs(np.asarray(kernel, dtype=np.float64)), iy_ref, ix_ref,
                              mask_radius_px)
