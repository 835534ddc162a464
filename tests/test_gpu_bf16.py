"""GPU parity of plain BF16 storage (hi alone, per-column power-of-two scale):
the build, the tcgen05 forward and the CUDA-core adjoint against the FP64
oracle, and a multi-job launch mixing BF16 and split-BF16 plans.

Tolerance, from the arithmetic: each stored element is RN_bf16(A/sigma) sigma,
within 2^-8 |A| (8-bit significand); the forward multiplies it by the first
two bf16 parts of x (the dropped third part is below 2^-16 |x|); the FP32
element and the chunked FP32 accumulation add below 1e-5.  So a pixel's
bound-relative error is at most TOL = 2^-8 + 2.5e-5."""
import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O
from synth import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 2.0 ** -8 + 2.5e-5


def _plan(lib32, radii, s, storage="bf16", **kw):
    from paper_2106_09122_gb300 import Plan
    return Plan(torch.from_numpy(np.ascontiguousarray(lib32)).to(DEV), radii, s, storage=storage, **kw)


def _setup(seed, n, N, n_r=8):
    rng = np.random.default_rng(seed)
    radii = np.linspace(0.0, 4.0, n_r)
    lib32 = rng.uniform(0.0, 1.0, (n_r, n, n)).astype(np.float32)
    return rng, radii, lib32


def test_bf16_storage_is_the_split_hi_and_within_2_to_minus_8():
    rng, radii, lib32 = _setup(60, 20, 13)
    bf = _plan(lib32, radii, 0.5, N=13, S=0.35)
    sp = _plan(lib32, radii, 0.5, N=13, S=0.35, storage="split_bf16")
    hi_b, lo_b, sc_b = bf.A_split()
    hi_s, _, sc_s = sp.A_split()
    assert lo_b is None
    assert torch.equal(hi_b.view(torch.int16), hi_s.view(torch.int16))
    assert torch.equal(sc_b, sc_s)
    dec = (hi_b.double() * sc_b.double()[None, :])[: bf.M, : bf.K].cpu().numpy()
    lib64 = lib32.astype(np.float64)
    A = O.build_A(lib64, radii, 13, 0.35)
    T = O.build_A(np.abs(lib64), radii, 13, 0.35)
    assert np.all(np.abs(dec - A) <= 2.0 ** -8 * np.abs(A) + 1e-6 * T + 1e-12)


@pytest.mark.parametrize("B", [1, 16, 85])
def test_bf16_tensor_core_forward(B):
    rng, radii, lib32 = _setup(61 + B, 24, 22, 9)
    plan = _plan(lib32, radii, 0.5, N=22, S=0.3)
    A = O.build_A(lib32.astype(np.float64), radii, 22, 0.3)
    x = (rng.uniform(0.0, 1.0, (B, 22 * 22)) * 10.0 ** rng.uniform(-10, -7, (B, 1))).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    assert plan.sync_status() == 0
    worst = 0.0
    for b in range(B):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], O.forward(A, x64), O.error_bound(A, x64), floor=O.FLT_MIN)
        worst = max(worst, float(rel.max()))
    assert worst <= TOL, worst
    assert worst > 1e-5      # the 8-bit storage is visible: BF16 is not the split encoding


def test_bf16_adjoint_and_transpose():
    rng, radii, lib32 = _setup(62, 20, 17)
    plan = _plan(lib32, radii, 0.5, N=17, S=0.35)
    A = O.build_A(lib32.astype(np.float64), radii, 17, 0.35)
    g = rng.standard_normal((3, 400)).astype(np.float32)
    gx = plan.adjoint(torch.from_numpy(g).to(DEV)).double().cpu().numpy()
    g64 = g.astype(np.float64)
    ref = O.adjoint(A, g64)
    bound = O.adjoint(np.abs(A), np.abs(g64))
    assert np.all(np.abs(gx - ref) <= TOL * bound + 1e-30)
    # forward and adjoint use the same stored matrix: <A x, g> = <x, A^T g> to FP32 sums
    x = rng.uniform(0.0, 1.0, (1, 17 * 17)).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()[0]
    lhs, rhs = float(y @ g64[0]), float(x[0].astype(np.float64) @ gx[0])
    scale = float(np.abs(A).sum(axis=1) @ np.abs(g64[0])) * float(np.abs(x).max())
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_multi_job_mixes_bf16_and_split_plans():
    from paper_2106_09122_gb300.serve import MultiForward
    rng, radii, lib32 = _setup(63, 24, 16)
    lib = torch.from_numpy(lib32).to(DEV)
    from paper_2106_09122_gb300 import Plan
    specs = [(16, 0.3, "bf16"), (12, 0.5, "split_bf16"), (16, 0.5, "bf16")]
    plans = [Plan(lib, radii, 0.25, N=N, S=S, storage=st) for N, S, st in specs]
    mf = MultiForward(plans, [6, 6, 6])
    for j, (N, _, _) in enumerate(specs):
        mf.x[j].copy_(torch.rand(6, N * N, device=DEV))
    mf.count.fill_(6)
    mf.enqueue()
    torch.cuda.synchronize()
    for j, (N, S, st) in enumerate(specs):
        A = O.build_A(lib32.astype(np.float64), radii, N, S)
        tol = TOL if st == "bf16" else 1e-5
        y = mf.y[j].double().cpu().numpy()
        X = mf.x[j].double().cpu().numpy()
        for b in range(6):
            rel = O.bound_relative_error(y[b], A @ X[b], np.abs(A) @ np.abs(X[b]), floor=O.FLT_MIN)
            assert rel.max() <= tol, (st, b, rel.max())


def test_bf16_batched_256_sampled_rows():
    """One wavelength of the 256^2 batched workload in BF16 storage (8.6 GB of A), 64 scenes."""
    w = workloads.batched_256()
    lib32 = w.library(0).astype(np.float32)
    plan = _plan(lib32, w.radii, w.s, N=w.N, S=w.S)
    X = workloads.scene_batch(w, 64).astype(np.float32)
    Y = plan.forward(torch.from_numpy(X).to(DEV))
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    rng = np.random.default_rng(64)
    rows = np.sort(rng.choice(w.M, 32, replace=False))
    xs, ys = O.scene_offsets(w.N, w.S)
    A_r = O.A_rows(lib32.astype(np.float64), w.radii, xs, ys, rows)
    X64 = X.astype(np.float64)
    Yr = Y[:, torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
    rel = O.bound_relative_error(Yr, X64 @ A_r.T, np.abs(X64) @ np.abs(A_r).T, floor=O.FLT_MIN)
    assert rel.max() <= TOL, rel.max()
