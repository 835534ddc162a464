"""GPU parity of FP32 storage compacted by the quarter-turn symmetry and the
zero columns (PSFSIM_FP32_SYM): forward and adjoint against the FP64 oracle
and against the dense FP32 path (same A elements, different sum order)."""
import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O
from synth import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _plan(lib32, radii, s, **kw):
    from paper_2106_09122_gb300 import Plan
    return Plan(torch.from_numpy(np.ascontiguousarray(lib32)).to(DEV), radii, s, **kw)


@pytest.mark.parametrize("n,N,S", [(20, 16, 0.35), (15, 10, 0.5), (24, 30, 0.2)])
def test_sym_forward_adjoint_match_oracle(n, N, S):
    rng = np.random.default_rng(n + N)
    radii = np.sort(rng.uniform(0.0, 3.5, 8))
    radii[0] = 0.0
    lib32 = rng.uniform(0.0, 1.0, (8, n, n)).astype(np.float32)
    plan = _plan(lib32, radii, 0.5, N=N, S=S, storage="fp32_sym")
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    x = rng.uniform(0.0, 1.0, (3, N * N)).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    for b in range(3):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], A @ x64, np.abs(A) @ np.abs(x64), floor=O.FLT_MIN)
        assert rel.max() <= 1e-5, rel.max()
    g = rng.standard_normal((2, n * n)).astype(np.float32)
    gx = plan.adjoint(torch.from_numpy(g).to(DEV)).double().cpu().numpy()
    ref = O.adjoint(A, g.astype(np.float64))
    bound = O.adjoint(np.abs(A), np.abs(g.astype(np.float64)))
    assert np.all(np.abs(gx - ref) <= 1e-5 * bound + 1e-30)
    assert plan.sync_status() == 0


def test_sym_equals_dense_on_the_fit_workload():
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    dense = _plan(lib32, w.radii, w.s, N=w.N, S=w.S)
    sym = _plan(lib32, w.radii, w.s, N=w.N, S=w.S, storage="fp32_sym")
    x = torch.from_numpy(workloads.scene_batch(w, 2).astype(np.float32)).to(DEV)
    Ad = dense.A_fp32()
    bound = (Ad.abs() @ x.abs().t()).t()
    yd, ys = dense.forward(x), sym.forward(x)
    assert torch.all((yd - ys).abs() <= 2e-6 * bound)
    g = torch.randn(2, w.M, device=DEV)
    gd, gs = dense.adjoint(g), sym.adjoint(g)
    gbound = (Ad.abs().t() @ g.abs().t()).t()
    assert torch.all((gd - gs).abs() <= 2e-6 * gbound + 1e-30)


@pytest.mark.parametrize("n,N", [(128, 128), (21, 20)])
def test_sym_fit_gradient_matches_separate_operators_and_dense(n, N):
    """psfsim_ring_gradient on FP32_SYM storage (three launches) against the same gradient
    from the separate operators on the same plan, and against the dense FP32 plan; twice in a
    row (counters back at zero, identical bits).  n = 21: odd image side (scalar adjoint path)."""
    from paper_2106_09122_gb300.fit import RingProblem
    S = 0.25
    rng = np.random.default_rng(90 + n)
    radii = np.linspace(0.0, 12.0 * N / 128.0 + 0.5, 12)
    lib32 = (rng.uniform(0.0, 1.0, (12, n, n)) * 1e-3).astype(np.float32)
    r_max = 0.95 * N * S / 2
    sym = _plan(lib32, radii, 0.25, N=N, S=S, storage="fp32_sym")
    dense = _plan(lib32, radii, 0.25, N=N, S=S)
    d = torch.from_numpy((rng.uniform(0.5, 1.5, n * n) * 1e-12).astype(np.float32)).to(DEV)
    theta = np.array([r_max / 2, r_max / 5, np.deg2rad(55.0), 0.3, 1e-9])
    ps = RingProblem(sym, N, S, r_max, d, 1e-13)
    pd = RingProblem(dense, N, S, r_max, d, 1e-13)
    assert ps.fused and pd.fused
    l1, g1 = ps.loss_and_grad(theta)
    y1, gz1 = ps.y.clone(), ps.gz.clone()
    l2, g2 = ps.loss_and_grad(theta)
    assert l1 == l2 and np.array_equal(g1, g2)
    ld, gd = pd.loss_and_grad(theta)
    assert l1 == pytest.approx(ld, rel=1e-6)
    np.testing.assert_allclose(g1, gd, rtol=1e-5, atol=1e-6 * np.abs(gd).max())
    assert torch.allclose(y1, pd.y, rtol=1e-5, atol=0)
    gzb = float(pd.gz.abs().max())
    assert torch.all((gz1 - pd.gz).abs() <= 1e-5 * gzb)
    ps.fused = False
    l3, g3 = ps.loss_and_grad(theta)
    assert l1 == pytest.approx(l3, rel=1e-6)
    np.testing.assert_allclose(g1, g3, rtol=1e-5, atol=1e-6 * np.abs(g3).max())


@pytest.mark.parametrize("n,N,S,B", [(20, 16, 0.35, 3), (24, 30, 0.2, 23), (15, 10, 0.5, 1)])
def test_split_sym_forward_adjoint_match_oracle(n, N, S, B):
    """SPLIT_BF16_SYM: the quadrant's split-BF16 columns; the four rotated scenes ride as a batch
    of 4B through the tcgen05 product (B = 23: 92 rotated scenes, two launches of the product)."""
    rng = np.random.default_rng(3 * n + N + B)
    radii = np.sort(rng.uniform(0.0, 3.5, 8))
    radii[0] = 0.0
    lib32 = rng.uniform(0.0, 1.0, (8, n, n)).astype(np.float32)
    plan = _plan(lib32, radii, 0.5, N=N, S=S, storage="split_bf16_sym")
    assert plan.info.K_stored < N * N // 4 + 1
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    x = rng.uniform(0.0, 1.0, (B, N * N)).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    assert plan.sync_status() == 0
    for b in range(B):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], A @ x64, np.abs(A) @ np.abs(x64), floor=O.FLT_MIN)
        assert rel.max() <= 1e-5, (b, rel.max())
    g = rng.standard_normal((2, n * n)).astype(np.float32)
    gx = plan.adjoint(torch.from_numpy(g).to(DEV)).double().cpu().numpy()
    ref = O.adjoint(A, g.astype(np.float64))
    bound = O.adjoint(np.abs(A), np.abs(g.astype(np.float64)))
    assert np.all(np.abs(gx - ref) <= 1e-5 * bound + 1e-30)
