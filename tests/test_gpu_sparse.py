"""GPU parity of the forward that skips zero scene pixels (psfsim_forward_sparse,
FP32 storage): against the FP64 oracle on sparse scenes (a few point sources),
against the dense forward on ring scenes that are zero beyond the outer working
angle (bitwise equal when no pixel is zero: the column list is then every column
and the split of it is the dense one), and on the degenerate batches."""
import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O
from synth import scenes, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _setup(seed, n, N, S):
    from paper_2106_09122_gb300 import Plan
    rng = np.random.default_rng(seed)
    radii = np.linspace(0.0, 5.0, 11)
    lib32 = rng.uniform(0.0, 1.0, (11, n, n)).astype(np.float32)
    plan = Plan(torch.from_numpy(lib32).to(DEV), radii, 0.5, N=N, S=S)
    return rng, radii, lib32, plan


def test_point_sources_match_oracle_and_dense():
    rng, radii, lib32, plan = _setup(80, 24, 37, 0.3)       # K = 1369: two ragged 1024-column chunks
    X = np.zeros((3, 37 * 37), dtype=np.float32)
    for b, npts in enumerate((1, 5, 40)):
        X[b, rng.choice(37 * 37, npts, replace=False)] = rng.uniform(0.5, 2.0, npts)
    x = torch.from_numpy(X).to(DEV)
    y = plan.forward(x, skip_zeros=True).double().cpu().numpy()
    y_dense = plan.forward(x).double().cpu().numpy()
    A = O.build_A(lib32.astype(np.float64), radii, 37, 0.3)
    for b in range(3):
        x64 = X[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], O.forward(A, x64), O.error_bound(A, x64), floor=O.FLT_MIN)
        assert rel.max() <= 1e-5, (b, rel.max())
    np.testing.assert_allclose(y, y_dense, rtol=1e-5, atol=1e-30)


def test_dense_scene_is_bitwise_the_dense_forward():
    rng, radii, lib32, plan = _setup(81, 20, 30, 0.3)
    x = torch.from_numpy(rng.uniform(0.1, 1.0, (2, 900)).astype(np.float32)).to(DEV)
    assert torch.equal(plan.forward(x, skip_zeros=True), plan.forward(x))


def test_ring_scene_beyond_owa_and_empty_batch():
    w = workloads.adjoint_128()
    from paper_2106_09122_gb300 import Plan
    plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(DEV), w.radii, w.s, N=w.N, S=w.S)
    ring = scenes.ring_image(w.N, w.S, 5.0, 1.0, np.deg2rad(60.0), 0.3, 1e-9, w.r_max).astype(np.float32)
    assert (ring == 0).mean() > 0.5                           # zero beyond 12 lambda/D
    x = torch.from_numpy(ring.ravel()).to(DEV)
    y = plan.forward(x, skip_zeros=True)
    y_dense = plan.forward(x)
    bound = (plan.A_fp32().abs() @ x.abs())
    assert torch.all((y - y_dense).abs() <= 2e-6 * bound + 1e-37)
    z = torch.zeros((2, w.K), device=DEV)
    yz = torch.full((2, w.M), float("nan"), device=DEV)
    plan.forward(z, out=yz, skip_zeros=True)
    assert torch.all(yz == 0)
