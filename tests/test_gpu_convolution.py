"""The convolution comparator on the GPU (cuFFT through torch.fft): Sec. 3
simulates the same scene by convolving it with one off-axis PSF, masked and
shifted to the centre.  Checked element by element against the FP64 direct
convolution of the oracle on the benchmarked 128^2 workload.  The bench takes
the PSF from the method itself (the column of one scene pixel), so where the
library is shift-invariant and the field points sit on the axes at sampled
radii the two images agree to float32 rounding; elsewhere their difference is
the field dependence the method keeps (reported by bench.py).

Tolerance: an FFT's float32 rounding error is spread over the whole output, so
it is bounded relative to the largest output scale, not per pixel:
|y - y_ref| <= 1e-5 * max_i sum |x||g| (a 256^2 transform has 16 butterfly
levels, each adding a few 2^-24 relative to the transform's norm)."""
import numpy as np
import pytest
import torch

from oracle import convolution_oracle as CO
from synth import scenes, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _gauss(u, v, sig):
    return np.exp(-(u * u + v * v) / (2.0 * sig * sig))


def test_convolution_comparator_equals_method_for_shift_invariant_library():
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.convolution import convolution_image
    n, s, N, S = 31, 0.5, 9, 0.5
    radii = np.arange(0, 9) * 0.5
    c = (n - 1) / 2.0
    p, q = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    lib = np.stack([_gauss(q - c - r / s, p - c, 1.7) for r in radii]).astype(np.float32)
    plan = Plan(torch.from_numpy(lib).to(DEV), radii, s, N=N, S=S)
    ix, iy = np.meshgrid(np.arange(N), np.arange(N))
    on_axes = ((ix == N // 2) | (iy == N // 2)).ravel()
    rng = np.random.default_rng(5)
    scene = np.where(on_axes, rng.uniform(0.5, 1.5, N * N), 0.0).astype(np.float32)
    scene[N * N // 2] = 0.0                      # nothing at the centre (r = 0 is the on-axis PSF)
    y_method = plan.forward(torch.from_numpy(scene).to(DEV)).view(n, n)
    j_ref = (N // 2) * N + N // 2 + 2            # (+2 S, 0) on the +x axis
    one_hot = torch.zeros(N * N, device=DEV)
    one_hot[j_ref] = 1.0
    col = plan.forward(one_hot).view(n, n)
    y_conv = convolution_image(torch.from_numpy(scene).to(DEV).view(N, N), col, j_ref // N, j_ref % N)
    err = (y_conv - y_method).abs().max().item() / y_method.abs().max().item()
    assert err < 2e-6, err


def test_convolution_comparator_with_mask_keeps_only_the_core():
    from paper_2106_09122_gb300.convolution import convolution_image
    n = 32
    col = torch.rand(n, n, device=DEV)
    x = torch.zeros(n, n, device=DEV)
    x[10, 12] = 2.0                              # one point source
    img = convolution_image(x, col, 16, 20, mask_radius_px=3.0)
    # a single point reproduces the kernel, masked to a disk of 3 px around its core
    pp, qq = torch.meshgrid(torch.arange(n, device=DEV), torch.arange(n, device=DEV), indexing="ij")
    keep = ((pp - 16) ** 2 + (qq - 20) ** 2) <= 9.0
    want = torch.zeros(n, n, device=DEV)
    src = torch.where(keep, col, torch.zeros_like(col))
    for dp in range(-3, 4):
        for dq in range(-3, 4):
            if keep[16 + dp, 20 + dq]:
                want[10 + dp, 12 + dq] = 2.0 * src[16 + dp, 20 + dq]
    assert torch.allclose(img, want, rtol=1e-5, atol=1e-6)


def test_convolution_comparator_matches_fp64_direct_convolution_on_the_128_workload():
    """The bench's comparator shape: the 128^2 ring scene convolved with a 128^2 Lyot PSF of
    the workload's library (the one at 6 lambda/D-ish offset, core at its source pixel),
    with and without the 3 lambda/D core mask."""
    from paper_2106_09122_gb300.convolution import convolution_image
    w = workloads.adjoint_128()
    lib = w.library()
    k = int(np.argmin(np.abs(w.radii - 6.0)))
    c = (w.n - 1) / 2.0
    cp, cq = int(round(c)), int(round(c + w.radii[k] / w.s))   # the PSF's core pixel
    kernel = lib[k].astype(np.float32)
    ring = scenes.ring_image(w.N, w.S, 5.0, 1.0, np.deg2rad(60.0), 0.3, 1e-9, w.r_max).astype(np.float32)
    for mask in (None, 3.0 / w.s):
        y = convolution_image(torch.from_numpy(ring).to(DEV), torch.from_numpy(kernel).to(DEV), cp, cq,
                              mask_radius_px=mask).double().cpu().numpy()
        ref = CO.direct_convolution(ring.astype(np.float64), kernel.astype(np.float64), cp, cq, mask)
        bound = CO.convolution_bound(ring, kernel, cp, cq, mask)
        err = np.abs(y - ref)
        assert err.max() <= 1e-5 * bound.max(), (mask, err.max() / bound.max())
