"""GPU parity of split-BF16 storage, the tcgen05 batched forward and the
split adjoint against the FP64 oracle.

Storage bound: sigma_j (hi + lo) carries <= 2^-17 relative error per element
on top of the FP32 element error (1e-6 of the tap magnitude T).  Images: the
bound-relative error of every pixel <= 1e-5 (the forward drops only the
lo * x3 product, < 2^-24 relative, and accumulates in FP32)."""
import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O
from oracle import split_oracle as SO
from synth import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _plan(lib32, radii, s, **kw):
    from paper_2106_09122_gb300 import Plan
    return Plan(torch.from_numpy(np.ascontiguousarray(lib32)).to(DEV), radii, s, storage="split_bf16", **kw)


def _decode(plan):
    hi, lo, sc = plan.A_split()
    dec = (hi.double() + lo.double()) * sc.double()[None, :]
    return dec[: plan.M, : plan.K].cpu().numpy(), sc.cpu().numpy()


@pytest.mark.parametrize("n,N,S", [(16, 8, 0.5), (20, 13, 0.35), (32, 24, 0.25)])
def test_split_storage_matches_oracle(n, N, S):
    rng = np.random.default_rng(n + N)
    radii = np.sort(rng.uniform(0.0, 3.5, 6))
    radii[0] = 0.0
    lib32 = (rng.uniform(0.0, 1.0, (6, n, n)) * 10.0 ** rng.uniform(-6, 0, (6, 1, 1))).astype(np.float32)
    plan = _plan(lib32, radii, 0.5, N=N, S=S)
    dec, sc = _decode(plan)
    lib64 = lib32.astype(np.float64)
    A = O.build_A(lib64, radii, N, S)
    T = O.build_A(np.abs(lib64), radii, N, S)
    tol = (2.0 ** -17 + 1e-6) * T + 1e-9 * np.abs(lib64).max()
    assert np.all(np.abs(dec - A) <= tol)
    # per-column power-of-two scale: bound over the radial bracket, 1 for zero columns
    x, y = O.scene_offsets(N, S)
    r, _, _ = O.polar(x, y)
    k, _, valid = O.radial_bracket(r, radii)
    m = np.abs(lib32).reshape(6, -1).max(axis=1)
    want = np.array([SO.pow2_scale_at_least(float(max(m[kk], m[kk + 1]))) if v else 1.0
                     for kk, v in zip(k, valid)])
    assert np.array_equal(sc[: N * N], want.astype(np.float32))


# N = 32, 64: whole 16 x 16 quadrant blocks; N = 48: whole blocks and an 8-wide edge block;
# N = 40 (N % 16 != 0): element-by-element copies.  M = n^2 is never a multiple of 32.
@pytest.mark.parametrize("n,N,S,storage", [(24, 32, 0.3, "split_bf16"), (20, 48, 0.2, "split_bf16"),
                                           (36, 64, 0.12, "bf16"), (17, 40, 0.25, "split_bf16")])
def test_symmetric_build_equals_direct_build_bit_for_bit(n, N, S, storage):
    """An even grid is built from the x > 0, y > 0 quadrant's columns, each written to its four
    quarter-turned positions; the same grid given as field points takes the direct build, column
    by column.  Both must store the same bits, padding included."""
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.plan import workspace_bytes
    rng = np.random.default_rng(n * 3 + N)
    radii = np.linspace(0.0, 0.55 * N * S, 9)  # the grid's corners lie beyond the last radius
    lib32 = rng.uniform(0.1, 1.0, (9, n, n)).astype(np.float32)
    lib = torch.from_numpy(lib32).to(DEV)
    iy, ix = np.divmod(np.arange(N * N), N)
    pts = np.stack([(ix - (N - 1) / 2) * S, (iy - (N - 1) / 2) * S], axis=1)
    direct = Plan(lib, radii, 0.5, points=pts, storage=storage)
    # the symmetric build's workspace comes from a block just filled with 0xFF, so a position
    # it failed to write would not read as a matching zero
    poison = torch.full((workspace_bytes(n, 9, N * N, storage),), 0xFF, dtype=torch.uint8, device=DEV)
    del poison
    sym = Plan(lib, radii, 0.5, N=N, S=S, storage=storage)
    torch.cuda.synchronize()
    assert sym.sync_status() == 0 and direct.sync_status() == 0
    for a, b in zip(sym.A_split(), direct.A_split()):
        if a is None:
            assert b is None
            continue
        bits = torch.int16 if a.dtype == torch.bfloat16 else torch.int32
        assert torch.equal(a.view(bits), b.view(bits))
    assert torch.count_nonzero(sym.A_split()[0][: n * n, : N * N]).item() > 0


@pytest.mark.parametrize("B", [1, 3, 16, 20, 85])
def test_tensor_core_forward_small(B):
    rng = np.random.default_rng(40 + B)
    n, N, S = 24, 22, 0.3
    radii = np.linspace(0.0, 4.0, 9)
    lib32 = rng.uniform(0.0, 1.0, (9, n, n)).astype(np.float32)
    plan = _plan(lib32, radii, 0.5, N=N, S=S)
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    x = (rng.uniform(0.0, 1.0, (B, N * N)) * 10.0 ** rng.uniform(-10, -7, (B, 1))).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    assert plan.sync_status() == 0
    for b in range(B):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], O.forward(A, x64), O.error_bound(A, x64), floor=O.FLT_MIN)
        assert rel.max() <= 1e-5, (b, rel.max())


def test_split_adjoint_small():
    rng = np.random.default_rng(50)
    n, N, S = 20, 17, 0.35
    radii = np.linspace(0.0, 4.0, 8)
    lib32 = rng.uniform(0.0, 1.0, (8, n, n)).astype(np.float32)
    plan = _plan(lib32, radii, 0.5, N=N, S=S)
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    g = rng.standard_normal((5, n * n)).astype(np.float32)
    gx = plan.adjoint(torch.from_numpy(g).to(DEV)).double().cpu().numpy()
    ref = O.adjoint(A, g.astype(np.float64))
    bound = O.adjoint(np.abs(A), np.abs(g.astype(np.float64)))
    assert np.all(np.abs(gx - ref) <= 1e-5 * bound + 1e-30)


def test_batched_256_workload_sampled_rows():
    """One wavelength of the 256^2 batched workload: 65536 x 65536 split-BF16 A, 64 scenes."""
    w = workloads.batched_256()
    lib32 = w.library(0).astype(np.float32)
    plan = _plan(lib32, w.radii, w.s, N=w.N, S=w.S)
    X = workloads.scene_batch(w, 64).astype(np.float32)
    Y = plan.forward(torch.from_numpy(X).to(DEV))
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    rng = np.random.default_rng(51)
    rows = np.sort(rng.choice(w.M, 48, replace=False))
    xs, ys = O.scene_offsets(w.N, w.S)
    A_r = O.A_rows(lib32.astype(np.float64), w.radii, xs, ys, rows)
    X64 = X.astype(np.float64)
    Yr = Y[:, torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
    rel = O.bound_relative_error(Yr, X64 @ A_r.T, np.abs(X64) @ np.abs(A_r).T, floor=O.FLT_MIN)
    assert rel.max() <= 1e-5, rel.max()
