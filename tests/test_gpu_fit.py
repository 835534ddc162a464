"""GPU parity of the fit operators (ring model, loss, chain, full gradient)
against the FP64 oracle, and the gradient against central differences of the
oracle's loss (relative 1e-4)."""
import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O
from oracle import ring_oracle as RO
from synth import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _problem(lib32, radii, s, N, S, r_max, d32, sigma):
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.fit import RingProblem
    plan = Plan(torch.from_numpy(lib32).to(DEV), radii, s, N=N, S=S)
    return RingProblem(plan, N, S, r_max, torch.from_numpy(d32).to(DEV), sigma)


def _small_setup(seed=31):
    rng = np.random.default_rng(seed)
    n, N, S = 40, 40, 0.3
    radii = np.linspace(0.0, 6.0, 16)
    lib32 = rng.uniform(0.0, 1e-3, (16, n, n)).astype(np.float32)
    truth = np.array([3.0, 1.0, np.deg2rad(50.0), 0.3, 1e-9])
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    d = O.forward(A, RO.ring_scene(truth, N, S, 5.5)) + rng.standard_normal(n * n) * 1e-14
    d32 = d.astype(np.float32)
    return n, N, S, radii, lib32, truth, A, d32


def test_ring_scene_chain_and_loss_match_oracle():
    n, N, S, radii, lib32, truth, A, d32 = _small_setup()
    P = _problem(lib32, radii, 0.3, N, S, 5.5, d32, 1e-14)
    theta = truth * np.array([1.05, 0.9, 1.03, 1.2, 1.1])
    z = P.scene(theta).double().cpu().numpy()
    Zr, J = RO.ring_scene_and_jacobian(theta, N, S, 5.5)
    assert np.all(np.abs(z - Zr) <= 1e-5 * np.abs(Zr).max())
    rng = np.random.default_rng(32)
    gz = rng.standard_normal(N * N).astype(np.float32)
    dth = P.chain(theta, torch.from_numpy(gz).to(DEV)).cpu().numpy()
    ref = J.T @ gz.astype(np.float64)
    scale = np.abs(J).T @ np.abs(gz.astype(np.float64))
    assert np.all(np.abs(dth - ref) <= 1e-5 * scale)
    y = torch.from_numpy(rng.standard_normal(n * n).astype(np.float32) * 1e-12).to(DEV)
    loss = float(P.residual_loss(y, P.target, True).item())
    diff = y.double().cpu().numpy() - d32.astype(np.float64)
    assert loss == pytest.approx(0.5 * np.sum((diff / 1e-14) ** 2), rel=1e-6)
    np.testing.assert_allclose(P.r.double().cpu().numpy(), diff / 1e-28, rtol=1e-5)


def test_gradient_matches_oracle_and_finite_differences_small():
    n, N, S, radii, lib32, truth, A, d32 = _small_setup()
    P = _problem(lib32, radii, 0.3, N, S, 5.5, d32, 1e-14)
    theta = truth + np.array([0.2, -0.1, 0.05, 0.05, 1e-10])
    loss, g = P.loss_and_grad(theta)
    d64 = d32.astype(np.float64)
    loss_o, g_o = RO.fit_loss_and_grad(A, theta, d64, 1e-14, N, S, 5.5)
    assert loss == pytest.approx(loss_o, rel=1e-4)
    np.testing.assert_allclose(g, g_o, rtol=1e-4)
    for m in range(5):
        h = 1e-6 * (abs(theta[m]) if m == 4 else 1.0)
        tp, tm = theta.copy(), theta.copy()
        tp[m] += h
        tm[m] -= h
        fd = (RO.fit_loss(A, tp, d64, 1e-14, N, S, 5.5) - RO.fit_loss(A, tm, d64, 1e-14, N, S, 5.5)) / (2 * h)
        assert g[m] == pytest.approx(fd, rel=1e-4)


def test_autograd_function_backward_is_the_adjoint_chain():
    from paper_2106_09122_gb300.fit import RingImage
    n, N, S, radii, lib32, truth, A, d32 = _small_setup()
    P = _problem(lib32, radii, 0.3, N, S, 5.5, d32, 1e-14)
    theta = torch.tensor(truth * np.array([1.04, 1.1, 0.97, 0.8, 1.05]), dtype=torch.float64, requires_grad=True)
    y = RingImage.apply(theta, P)
    gy = torch.from_numpy(np.random.default_rng(33).standard_normal(n * n).astype(np.float32)).to(DEV)
    (y * gy).sum().backward()
    _, J = RO.ring_scene_and_jacobian(theta.detach().numpy(), N, S, 5.5)
    ref = J.T @ (A.T @ gy.double().cpu().numpy())
    scale = np.abs(J).T @ (np.abs(A).T @ np.abs(gy.double().cpu().numpy()))
    assert np.all(np.abs(theta.grad.numpy() - ref) <= 1e-5 * scale)


def test_adjoint_fit_workload_gradient_and_fit():
    """128^2 fit workload: gradient vs the oracle and its central differences, then 200 steps."""
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    truth = np.array(w.extra["truth"])
    sigma = w.extra["sigma"]
    A = O.build_A(lib32.astype(np.float64), w.radii, w.N, w.S)
    d = O.forward(A, RO.ring_scene(truth, w.N, w.S, w.r_max)) + workloads.fit_target_noise(w, w.M)
    d32 = d.astype(np.float32)
    d64 = d32.astype(np.float64)
    P = _problem(lib32, w.radii, w.s, w.N, w.S, w.r_max, d32, sigma)
    theta0 = workloads.fit_init(w)
    loss, g = P.loss_and_grad(theta0)
    loss_o, g_o = RO.fit_loss_and_grad(A, theta0, d64, sigma, w.N, w.S, w.r_max)
    assert loss == pytest.approx(loss_o, rel=1e-4)
    np.testing.assert_allclose(g, g_o, rtol=1e-4)
    for m in range(5):
        h = 1e-6 * (abs(theta0[m]) if m == 4 else 1.0)
        tp, tm = theta0.copy(), theta0.copy()
        tp[m] += h
        tm[m] -= h
        fd = (RO.fit_loss(A, tp, d64, sigma, w.N, w.S, w.r_max)
              - RO.fit_loss(A, tm, d64, sigma, w.N, w.S, w.r_max)) / (2 * h)
        assert g[m] == pytest.approx(fd, rel=1e-4)
    theta, hist = P.fit(theta0, steps=w.extra["steps"])
    assert np.all(np.diff(hist) <= 0.0)
    assert hist[-1] < 1e-3 * hist[0]
    assert np.all(np.abs(theta - truth) <= np.abs(theta0 - truth))


def test_fused_gradient_equals_separate_operators():
    """psfsim_ring_gradient (2 launches) against ring + forward + loss + adjoint + chain."""
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    truth = np.array(w.extra["truth"])
    rng = np.random.default_rng(35)
    d32 = (rng.uniform(0.5, 1.5, w.M) * 1e-10).astype(np.float32)
    P = _problem(lib32, w.radii, w.s, w.N, w.S, w.r_max, d32, w.extra["sigma"])
    assert P.fused
    theta = truth * np.array([1.03, 0.95, 1.02, 1.1, 1.2])
    loss_f, g_f = P.loss_and_grad(theta)
    y_f = P.y.clone()
    P.fused = False
    loss_s, g_s = P.loss_and_grad(theta)
    assert torch.allclose(P.y, y_f, rtol=1e-6, atol=0)
    assert loss_f == pytest.approx(loss_s, rel=1e-6)
    np.testing.assert_allclose(g_f, g_s, rtol=1e-5)


@pytest.mark.parametrize("n,N", [(21, 6), (48, 40), (33, 70)])
def test_fused_gradient_on_ragged_shapes_repeats_and_matches_separate(n, N):
    """Ragged row tiles (M = n^2 not a multiple of the 1024-row tile, odd M for the
    scalar adjoint path), fewer columns than the forward's splits (K = 36), and
    repeated calls: the arrival counters must be back at zero after every launch,
    so a second gradient, and the adjoint half called twice, give identical bits."""
    rng = np.random.default_rng(100 * n + N)
    S = 0.3
    radii = np.linspace(0.0, 6.0, 12)
    lib32 = rng.uniform(0.0, 1e-3, (12, n, n)).astype(np.float32)
    d32 = (rng.uniform(0.5, 1.5, n * n) * 1e-10).astype(np.float32)
    half = N * S / 2
    P = _problem(lib32, radii, S, N, S, 0.95 * half, d32, 1e-11)
    assert P.fused
    theta = np.array([half / 2, half / 3, np.deg2rad(50.0), 0.3, 1e-9])
    loss_f, g_f = P.loss_and_grad(theta)
    loss_f2, g_f2 = P.loss_and_grad(theta)
    assert loss_f2 == loss_f and np.array_equal(g_f2, g_f)
    y_f = P.y.clone()
    P.enqueue_adjoint_chain(theta)
    out_a = P.out6.cpu().numpy().copy()
    P.enqueue_adjoint_chain(theta)
    out_b = P.out6.cpu().numpy().copy()
    assert np.array_equal(out_a, out_b) and out_a[0] == loss_f and np.array_equal(out_a[1:], g_f)
    P.fused = False
    loss_s, g_s = P.loss_and_grad(theta)
    assert torch.allclose(P.y, y_f, rtol=1e-6, atol=0)
    assert loss_f == pytest.approx(loss_s, rel=1e-6)
    np.testing.assert_allclose(g_f, g_s, rtol=1e-5, atol=1e-6 * np.abs(g_s).max())


def test_gradient_reads_target_and_writes_result_in_pinned_host_memory():
    """psfsim_ring_gradient with the target and the result in pinned host memory (mapped into
    the device's address space): the same bits as with both in device memory."""
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    rng = np.random.default_rng(36)
    d32 = (rng.uniform(0.5, 1.5, w.M) * 1e-10).astype(np.float32)
    P = _problem(lib32, w.radii, w.s, w.N, w.S, w.r_max, d32, w.extra["sigma"])
    from paper_2106_09122_gb300.fit import RingProblem
    host_d = torch.from_numpy(d32).pin_memory()
    Q = RingProblem(P.plan, w.N, w.S, w.r_max, host_d, w.extra["sigma"])
    out = torch.zeros(6, dtype=torch.float64).pin_memory()
    Q.out6, Q.loss_d, Q.dtheta = out, out[:1], out[1:]
    theta = np.array(w.extra["truth"]) * np.array([1.02, 0.97, 1.01, 1.05, 1.1])
    l_dev, g_dev = P.loss_and_grad(theta)
    Q.enqueue_gradient(theta)
    torch.cuda.synchronize()
    assert out[0].item() == l_dev and np.array_equal(out[1:].numpy(), g_dev)
