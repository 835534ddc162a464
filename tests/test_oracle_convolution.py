"""Shift-invariant libraries: the method must reduce to convolution (CPU only).

Sec. 3 contrasts the matrix method with convolution by a single PSF: when every
library PSF is the same shape shifted to its offset, the interpolated and
rotated PSFs are that shape shifted to each field point, and A Z is the
convolution of the scene with it.  Exactly so on axis at sampled radii; to
second order in the pixel and radial spacing elsewhere.
"""
import numpy as np

from oracle import psfsim_oracle as O


def _gauss(u, v, sig):
    return np.exp(-(u * u + v * v) / (2.0 * sig * sig))


def _shifted_library(n, s, radii, sig_px):
    c = (n - 1) / 2.0
    p, q = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    return np.stack([_gauss(q - c - r / s, p - c, sig_px) for r in radii])


def test_exact_convolution_on_axes():
    n, s = 31, 0.5
    N, S = 9, 0.5                              # odd N: pixels on the axes at integer multiples of S
    radii = np.arange(0, 9) * 0.5
    sig = 1.7
    lib = _shifted_library(n, s, radii, sig)
    A = O.build_A(lib, radii, N, S)
    x, y = O.scene_offsets(N, S)
    rng = np.random.default_rng(11)
    scene = np.where((x == 0.0) | (y == 0.0), rng.uniform(0.5, 1.5, N * N), 0.0)
    scene[np.hypot(x, y) > radii[-1]] = 0.0
    c = (n - 1) / 2.0
    p, q = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    direct = np.zeros((n, n))
    for j in np.nonzero(scene)[0]:
        direct += scene[j] * _gauss(q - c - x[j] / s, p - c - y[j] / s, sig)
        np.testing.assert_array_equal(A[:, j].reshape(n, n),
                                      _gauss(q - c - x[j] / s, p - c - y[j] / s, sig))
    np.testing.assert_allclose(O.forward(A, scene).reshape(n, n), direct, rtol=1e-13, atol=1e-14)


def _method_error(s, dr):
    """Max column error of the method against the exactly shifted Gaussian."""
    half = 7.0
    n = int(round(2 * half / s)) + 1
    radii = np.arange(0.0, 3.0 + 1e-9, dr)
    sig_ld = 0.8
    lib = _shifted_library(n, s, radii, sig_ld / s)
    rng = np.random.default_rng(12)
    pts = rng.uniform(-2.0, 2.0, size=(24, 2))
    c = (n - 1) / 2.0
    p, q = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    err = 0.0
    for xj, yj in pts:
        col = O.psf_column(lib, radii, xj, yj).reshape(n, n)
        exact = _gauss(q - c - xj / s, p - c - yj / s, sig_ld / s)
        err = max(err, np.max(np.abs(col - exact)))
    return err


def test_second_order_convergence_to_convolution():
    e1 = _method_error(0.2, 0.2)
    e2 = _method_error(0.1, 0.1)
    assert e2 < e1
    assert 3.0 < e1 / e2 < 5.5


# ---- the direct-convolution oracle of the GPU comparator ----------------------------------

from oracle import convolution_oracle as CO  # noqa: E402


def test_point_source_reproduces_the_masked_kernel():
    rng = np.random.default_rng(31)
    n, N = 21, 15
    o = (n - N) // 2
    g = rng.uniform(0.0, 1.0, (n, n))
    scene = np.zeros((N, N))
    scene[4, 9] = 2.5
    iy_ref, ix_ref = 6, 8                      # kernel core at image pixel (9, 11)
    out = CO.direct_convolution(scene, g, iy_ref, ix_ref, mask_radius_px=4.0)
    cp, cq = iy_ref + o, ix_ref + o
    gm = CO.masked_kernel(g, cp, cq, 4.0)
    want = np.zeros((n, n))
    dp, dq = 4 + o - cp, 9 + o - cq           # shift of the copy
    for p in range(n):
        for q in range(n):
            if 0 <= p - dp < n and 0 <= q - dq < n:
                want[p, q] = 2.5 * gm[p - dp, q - dq]
    np.testing.assert_array_equal(out, want)
    # the core itself lands on the source pixel's image position
    assert out[4 + o, 9 + o] == 2.5 * g[cp, cq]
    # and nothing farther than the mask radius from it
    pp, qq = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    assert np.all(out[(pp - 4 - o) ** 2 + (qq - 9 - o) ** 2 > 16.0] == 0.0)


def test_direct_convolution_equals_the_method_for_the_exact_shift_invariant_case():
    """On the axes at sampled radii the method's columns are exactly shifted copies of one
    shape (test_exact_convolution_on_axes), so A Z equals the direct convolution of the scene
    with the column of any one of those pixels."""
    n, s = 31, 0.5
    N, S = 9, 0.5
    radii = np.arange(0, 9) * 0.5
    lib = _shifted_library(n, s, radii, 1.7)
    A = O.build_A(lib, radii, N, S)
    x, y = O.scene_offsets(N, S)
    rng = np.random.default_rng(13)
    scene = np.where((x == 0.0) | (y == 0.0), rng.uniform(0.5, 1.5, N * N), 0.0)
    scene[(x == 0.0) & (y == 0.0)] = 0.0
    j_ref = (N // 2) * N + N // 2 + 2         # (+2 S, 0)
    col = A[:, j_ref].reshape(n, n)
    conv = CO.direct_convolution(scene.reshape(N, N), col, j_ref // N, j_ref % N)
    np.testing.assert_allclose(conv, O.forward(A, scene).reshape(n, n), rtol=1e-13, atol=1e-13)


def test_direct_convolution_equals_a_zero_padded_fft_product():
    rng = np.random.default_rng(17)
    n, N = 24, 16
    g = rng.uniform(-1.0, 1.0, (n, n))
    scene = rng.uniform(0.0, 1.0, (N, N)) * (rng.uniform(size=(N, N)) < 0.3)
    iy_ref, ix_ref = 5, 11
    out = CO.direct_convolution(scene, g, iy_ref, ix_ref)
    o = (n - N) // 2
    P = 2 * n
    xp = np.zeros((P, P))
    xp[o:o + N, o:o + N] = scene
    kp = np.zeros((P, P))
    kp[:n, :n] = g
    kp = np.roll(kp, (-(iy_ref + o), -(ix_ref + o)), axis=(0, 1))
    fft = np.real(np.fft.ifft2(np.fft.fft2(xp) * np.fft.fft2(kp)))[:n, :n]
    np.testing.assert_allclose(out, fft, rtol=0, atol=1e-12)
