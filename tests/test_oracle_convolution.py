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
