"""Convolution comparator (Sec. 3): a scene simulated by convolving it with one
off-axis PSF, masked to its core and shifted to the centre, instead of the
field-dependent matrix method.  It quantifies the field dependence the method
keeps; it is a comparison system, not a step of the method.

Linear convolution by zero-padded FFTs (cuFFT through torch.fft) on the
n x n image grid.
"""
from __future__ import annotations

import torch


def convolution_image(scene: torch.Tensor, kernel: torch.Tensor, iy_ref: int, ix_ref: int,
                      mask_radius_px: float | None = None) -> torch.Tensor:
    """scene (N x N) convolved with kernel (n x n) whose core sits at image pixel
    (iy_ref + o, ix_ref + o), o = (n - N) / 2 -- the image pixel of scene pixel (iy_ref, ix_ref):
        out[p, q] = sum_{iy, ix} scene[iy, ix] * kernel[p - iy + iy_ref, q - ix + ix_ref],
    kernel entries outside the array (or, with mask_radius_px, farther than that from the
    core) counting 0.  Needs s = S and n - N even (the scene grid then maps onto the image
    grid by the integer offset o)."""
    n, N = kernel.shape[0], scene.shape[0]
    if kernel.shape != (n, n) or scene.shape != (N, N) or (n - N) % 2 or n < N:
        raise ValueError("kernel must be n x n and scene N x N with n - N even and >= 0")
    o = (n - N) // 2
    cp, cq = iy_ref + o, ix_ref + o
    g = kernel
    if mask_radius_px is not None:
        pp = torch.arange(n, device=g.device).view(-1, 1)
        qq = torch.arange(n, device=g.device).view(1, -1)
        g = torch.where((pp - cp) ** 2 + (qq - cq) ** 2 <= mask_radius_px ** 2, g, torch.zeros_like(g))
    P = 2 * n
    xp = torch.zeros(P, P, device=g.device, dtype=torch.float32)
    xp[o:o + N, o:o + N] = scene
    kp = torch.roll(torch.nn.functional.pad(g, (0, P - n, 0, P - n)), shifts=(-cp, -cq), dims=(0, 1))
    out = torch.fft.irfft2(torch.fft.rfft2(xp) * torch.fft.rfft2(kp), s=(P, P))
    return out[:n, :n]
