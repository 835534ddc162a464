"""GPU parity of the FP32 build / forward / adjoint against the FP64 oracle.

The oracle gets the same float32-rounded library the GPU gets (promoted to
float64), so the comparison isolates the kernels' arithmetic.  Element bound:
|A_gpu - A| <= 1e-6 * T + 1e-9 * max|L|, with T the oracle's A built from |L|
(about 16 float32 roundings of the 8-tap lerp/bilinear sum, plus the fixed-point
coordinate difference).  Image bound: |y - y_ref| <= 1e-5 * sum_j |A_ij||x_j|.
"""
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


def _check_A(A_gpu, lib32, radii, build):
    lib64 = lib32.astype(np.float64)
    A = build(lib64)
    T = build(np.abs(lib64))
    tol = 1e-6 * T + 1e-9 * np.abs(lib64).max()
    err = np.abs(A_gpu - A)
    assert np.all(err <= tol), f"max excess {np.max(err - tol)} at {np.unravel_index(np.argmax(err - tol), err.shape)}"
    return A


def _check_image(y, A, x):
    rel = O.bound_relative_error(y, O.forward(A, x), O.error_bound(A, x), floor=O.FLT_MIN)
    assert rel.max() <= 1e-5, rel.max()
    return rel.max()


def test_plain_small_workload_full_A_and_image():
    w = workloads.plain_small()
    lib32 = w.library().astype(np.float32)
    plan = _plan(lib32, w.radii, w.s, N=w.N, S=w.S)
    A_gpu = plan.A_fp32().double().cpu().numpy()
    A = _check_A(A_gpu, lib32, w.radii, lambda L: O.build_A(L, w.radii, w.N, w.S))
    x = workloads.plain_small_scene(w).ravel().astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    _check_image(y, A, x.astype(np.float64))
    assert plan.sync_status() == 0


@pytest.mark.parametrize("n,N,s,S,interp", [(15, 9, 0.5, 0.7, "linear"), (16, 11, 0.3, 0.45, "nearest"),
                                           (12, 20, 0.5, 0.5, "linear"), (33, 7, 0.25, 1.1, "linear")])
def test_odd_and_ragged_shapes(n, N, s, S, interp):
    rng = np.random.default_rng(n * 100 + N)
    radii = np.sort(rng.uniform(0.0, 4.0, 7))
    radii[0] = 0.0
    lib32 = rng.uniform(-1.0, 1.0, (7, n, n)).astype(np.float32)
    plan = _plan(lib32, radii, s, N=N, S=S, interp=interp)
    A_gpu = plan.A_fp32().double().cpu().numpy()
    A = _check_A(A_gpu, lib32, radii, lambda L: O.build_A(L, radii, N, S, interp))
    x = rng.standard_normal((3, N * N)).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    for b in range(3):
        _check_image(y[b], A, x[b].astype(np.float64))
    g = rng.standard_normal((2, n * n)).astype(np.float32)
    gx = plan.adjoint(torch.from_numpy(g).to(DEV)).double().cpu().numpy()
    ref = O.adjoint(A, g.astype(np.float64))
    bound = O.adjoint(np.abs(A), np.abs(g.astype(np.float64)))
    assert np.all(np.abs(gx - ref) <= 1e-5 * bound + 1e-30)


def test_exact_invariants_through_points():
    """theta = 0 is the identity, quarter turns are exact permutations, lerp hits samples."""
    rng = np.random.default_rng(21)
    n = 24
    radii = np.array([0.0, 0.75, 1.5, 3.0, 4.0])
    lib32 = rng.uniform(0.0, 1.0, (5, n, n)).astype(np.float32)
    pts = []
    for r in radii[1:]:
        pts += [(r, 0.0), (0.0, r), (-r, 0.0), (0.0, -r)]
    pts.append((0.5 * (radii[1] + radii[2]), 0.0))
    pts.append((4.0001, 0.0))
    plan = _plan(lib32, radii, 0.5, points=np.array(pts))
    A = plan.A_fp32().cpu().numpy()
    for t, r in enumerate(radii[1:]):
        k = t + 1
        cols = [A[:, 4 * t + m].reshape(n, n) for m in range(4)]
        assert np.array_equal(cols[0], lib32[k])
        assert np.array_equal(cols[1], np.rot90(lib32[k], -1))
        assert np.array_equal(cols[2], np.rot90(lib32[k], 2))
        assert np.array_equal(cols[3], np.rot90(lib32[k], 1))
    mid = A[:, -2].reshape(n, n)
    assert np.array_equal(mid, (np.float32(0.5) * lib32[1] + np.float32(0.5) * lib32[2]))
    assert not np.any(A[:, -1])


def test_scene_grid_quarter_turn_is_bitwise():
    rng = np.random.default_rng(22)
    n, N, S = 20, 10, 0.55
    radii = np.linspace(0.0, 4.0, 9)
    lib32 = rng.uniform(0.0, 1.0, (9, n, n)).astype(np.float32)
    A = _plan(lib32, radii, 0.5, N=N, S=S).A_fp32().cpu().numpy()
    for iy in range(N):
        for ix in range(N):
            a = A[:, iy * N + ix].reshape(n, n)
            b = A[:, ix * N + (N - 1 - iy)].reshape(n, n)
            assert np.array_equal(b, np.rot90(a, -1))


# n = 32, 96, 128: the bracket pair staged in shared memory; n = 192: taps read through L1/L2
@pytest.mark.parametrize("n,N,S", [(32, 24, 0.3), (96, 20, 0.3), (128, 16, 0.5), (192, 12, 0.6)])
def test_symmetric_build_equals_direct_build_bit_for_bit(n, N, S):
    """An even grid with n % 32 == 0 is built from the x > 0, y > 0 quadrant's columns, each
    written in 32 x 32 pixel blocks to its four quarter-turned places; the same grid given as
    field points takes the direct build, column by column.  Both must store the same bits."""
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.plan import workspace_bytes
    rng = np.random.default_rng(n + 7 * N)
    radii = np.linspace(0.0, 0.55 * N * S, 9)  # the grid's corners lie beyond the last radius
    lib32 = rng.uniform(0.1, 1.0, (9, n, n)).astype(np.float32)
    lib = torch.from_numpy(lib32).to(DEV)
    iy, ix = np.divmod(np.arange(N * N), N)
    pts = np.stack([(ix - (N - 1) / 2) * S, (iy - (N - 1) / 2) * S], axis=1)
    direct = Plan(lib, radii, 0.5, points=pts)
    # the symmetric build's workspace comes from a block just filled with 0xFF, so a position
    # it failed to write would not read as a matching zero
    poison = torch.full((workspace_bytes(n, 9, N * N, "fp32"),), 0xFF, dtype=torch.uint8, device=DEV)
    del poison
    sym = Plan(lib, radii, 0.5, N=N, S=S)
    torch.cuda.synchronize()
    assert sym.sync_status() == 0 and direct.sync_status() == 0
    assert torch.equal(sym.A_fp32().view(torch.int32), direct.A_fp32().view(torch.int32))
    assert torch.count_nonzero(sym.A_fp32()).item() > 0


def test_forward_is_deterministic_and_linear_batch():
    w = workloads.plain_small()
    lib32 = w.library().astype(np.float32)
    plan = _plan(lib32, w.radii, w.s, N=w.N, S=w.S)
    xs = torch.from_numpy(workloads.scene_batch(w, 11).astype(np.float32)).to(DEV)
    y1 = plan.forward(xs)
    y2 = plan.forward(xs)
    assert torch.equal(y1, y2)
    for b in (0, 5, 10):
        yb = plan.forward(xs[b].contiguous())
        assert torch.allclose(yb, y1[b], rtol=1e-6, atol=0)


def test_adjoint_workload_sampled_rows():
    """Full 16384 x 16384 A (the fit workload) checked on seeded sampled rows."""
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    plan = _plan(lib32, w.radii, w.s, N=w.N, S=w.S)
    rng = np.random.default_rng(23)
    rows = np.sort(rng.choice(w.M, 192, replace=False))
    xs, ys = O.scene_offsets(w.N, w.S)
    lib64 = lib32.astype(np.float64)
    A_rows = O.A_rows(lib64, w.radii, xs, ys, rows)
    T_rows = O.A_rows(np.abs(lib64), w.radii, xs, ys, rows)
    A_gpu = plan.A_fp32()[torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
    assert np.all(np.abs(A_gpu - A_rows) <= 1e-6 * T_rows + 1e-9 * np.abs(lib64).max())
    x = workloads.random_ring_scene(w.N, w.S, w.r_max, 99).ravel().astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()[rows]
    x64 = x.astype(np.float64)
    rel = O.bound_relative_error(y, A_rows @ x64, np.abs(A_rows) @ np.abs(x64), floor=O.FLT_MIN)
    assert rel.max() <= 1e-5
    g = rng.standard_normal(w.M).astype(np.float32)
    gx = plan.adjoint(torch.from_numpy(g).to(DEV)).double().cpu().numpy()
    # dot-product test <A x, g> = <x, A^T g> on the full size
    yfull = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    lhs, rhs = yfull @ g.astype(np.float64), x64 @ gx
    scale = np.abs(yfull) @ np.abs(g.astype(np.float64))
    assert abs(lhs - rhs) <= 1e-5 * scale
