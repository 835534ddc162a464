"""Pins of the oracle's ring model, its Jacobian and the fit gradient (CPU only)."""
import numpy as np
import pytest

from oracle import psfsim_oracle as O
from oracle import ring_oracle as RO


def test_hg_is_normalised_over_the_sphere():
    integrate = pytest.importorskip("scipy.integrate")
    for g in (0.0, 0.3, 0.6):
        val, _ = integrate.quad(lambda mu: 2.0 * np.pi * RO.hg(mu, g), -1.0, 1.0)
        assert val == pytest.approx(1.0, abs=1e-10)


def test_ring_phase_factor_is_hg_ratio():
    N, S = 16, 0.7
    theta = (3.0, 1.2, np.deg2rad(50.0), 0.45, 2.0)
    Z = RO.ring_scene(theta, N, S, 100.0)
    x, y = O.scene_offsets(N, S)
    yd = y / np.cos(theta[2])
    rd = np.hypot(x, yd)
    mu = np.sin(theta[2]) * yd / rd
    ref = theta[4] * np.exp(-4 * np.log(2) * (rd - theta[0]) ** 2 / theta[1] ** 2) \
        * RO.hg(mu, theta[3]) / RO.hg(0.0, theta[3])
    np.testing.assert_allclose(Z, ref, rtol=1e-12)


def test_face_on_ring_peak_and_fwhm():
    N, S = 20, 0.5
    x, y = O.scene_offsets(N, S)
    r = np.hypot(x, y)
    j = 57
    B, w = 3.0, 0.8
    Z = RO.ring_scene((r[j], w, 0.0, 0.0, B), N, S, 100.0)
    assert Z[j] == B
    Zh = RO.ring_scene((r[j] - w / 2, w, 0.0, 0.0, B), N, S, 100.0)
    assert Zh[j] == pytest.approx(B / 2, rel=1e-14)


def test_forward_scattering_side_and_mask():
    N, S = 24, 0.5
    Z = RO.ring_scene((4.0, 1.0, np.deg2rad(60.0), 0.5, 1.0), N, S, 5.0).reshape(N, N)
    assert Z[N // 2:].sum() > 2.0 * Z[: N // 2].sum()        # +y half is the forward side
    x, y = O.scene_offsets(N, S)
    assert not np.any(Z.ravel()[np.hypot(x, y) > 5.0])


def test_jacobian_matches_central_differences():
    N, S, rmax = 18, 0.6, 5.0
    theta = np.array([3.2, 0.9, np.deg2rad(55.0), 0.35, 1.5])
    _, J = RO.ring_scene_and_jacobian(theta, N, S, rmax)
    for m in range(5):
        h = 1e-6 * max(1.0, abs(theta[m]))
        tp, tm = theta.copy(), theta.copy()
        tp[m] += h
        tm[m] -= h
        fd = (RO.ring_scene(tp, N, S, rmax) - RO.ring_scene(tm, N, S, rmax)) / (2 * h)
        np.testing.assert_allclose(J[:, m], fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_fit_gradient_matches_central_differences_and_vanishes_at_truth():
    n, N, S = 14, 12, 0.5
    radii = np.linspace(0.0, 4.5, 10)
    rng = np.random.default_rng(13)
    lib = rng.uniform(0.0, 1.0, size=(10, n, n))
    A = O.build_A(lib, radii, N, S)
    truth = np.array([2.5, 1.0, np.deg2rad(40.0), 0.3, 1.0])
    d = O.forward(A, RO.ring_scene(truth, N, S, 4.0))
    loss0, g0 = RO.fit_loss_and_grad(A, truth, d, 0.1, N, S, 4.0)
    assert loss0 == 0.0 and not np.any(g0)
    theta = truth + np.array([0.2, -0.1, 0.05, 0.05, 0.1])
    loss, g = RO.fit_loss_and_grad(A, theta, d, 0.1, N, S, 4.0)
    assert loss == pytest.approx(RO.fit_loss(A, theta, d, 0.1, N, S, 4.0), rel=1e-14)
    for m in range(5):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[m] += h
        tm[m] -= h
        fd = (RO.fit_loss(A, tp, d, 0.1, N, S, 4.0) - RO.fit_loss(A, tm, d, 0.1, N, S, 4.0)) / (2 * h)
        assert g[m] == pytest.approx(fd, rel=1e-6)
