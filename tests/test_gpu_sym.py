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
