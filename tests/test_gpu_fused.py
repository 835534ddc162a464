"""GPU parity of the fused path (A regenerated on chip, quadrant symmetry)
against the FP64 oracle and against the stored split-BF16 path.

Bound (per pixel, relative to sum_j |A_ij||x_j|): hi + lo storage of A on chip
(2^-17) + two-part bf16 split of x (2^-17) + the dropped lo * x2 product
(2^-18) + the drift of 64 accumulating MMAs between drains (64 * 2^-24) +
FP32 sums: 2.5e-5."""
import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O
from synth import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 2.5e-5


def _plan(lib32, radii, s, **kw):
    from paper_2106_09122_gb300 import Plan
    return Plan(torch.from_numpy(np.ascontiguousarray(lib32)).to(DEV), radii, s, **kw)


# B = 1 runs the 16-scene form with one scene; B = 33, 40 and 64 run the 64-scene form;
# B = 65 runs it and then the 16-scene form for the last scene; B = 100 runs it twice (64 + 36)
@pytest.mark.parametrize("n,N,S,B", [(32, 32, 0.3, 3), (24, 40, 0.2, 17), (40, 26, 0.33, 32), (16, 12, 0.5, 40),
                                     (32, 32, 0.3, 64), (24, 20, 0.4, 100), (20, 18, 0.45, 1), (18, 14, 0.6, 33),
                                     (28, 22, 0.35, 65)])
def test_fused_forward_matches_oracle(n, N, S, B):
    rng = np.random.default_rng(n * 7 + N)
    radii = np.linspace(0.0, 4.5, 12)
    lib32 = rng.uniform(0.0, 1.0, (12, n, n)).astype(np.float32)
    plan = _plan(lib32, radii, 0.5, N=N, S=S, storage="fused")
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    x = rng.uniform(0.0, 1.0, (B, N * N)).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    assert plan.sync_status() == 0
    for b in range(B):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], O.forward(A, x64), O.error_bound(A, x64), floor=O.FLT_MIN)
        assert rel.max() <= TOL, (b, rel.max())


def test_fused_512_crop_against_oracle_and_stored_path():
    """512^2 fused workload on a scene that is zero outside its central 256^2 crop."""
    w = workloads.fused_512()
    lib32 = w.library().astype(np.float32)
    scenes = workloads.scene_batch(w, 4, kind="two_ring").reshape(4, w.N, w.N)
    crop = np.zeros_like(scenes)
    lo, hi = w.N // 4, 3 * w.N // 4
    crop[:, lo:hi, lo:hi] = scenes[:, lo:hi, lo:hi]
    X = crop.reshape(4, -1).astype(np.float32)
    fused = _plan(lib32, w.radii, w.s, N=w.N, S=w.S, storage="fused")
    Y = fused.forward(torch.from_numpy(X).to(DEV))
    torch.cuda.synchronize()
    assert fused.sync_status() == 0
    # oracle on seeded sampled rows, columns restricted to the crop
    xs, ys = O.scene_offsets(w.N, w.S)
    iy, ix = np.divmod(np.arange(w.K), w.N)
    cols = np.nonzero((iy >= lo) & (iy < hi) & (ix >= lo) & (ix < hi))[0]
    rng = np.random.default_rng(61)
    rows = np.sort(rng.choice(w.M, 32, replace=False))
    A_r = O.A_rows(lib32.astype(np.float64), w.radii, xs[cols], ys[cols], rows)
    Xc = X[:, cols].astype(np.float64)
    Yr = Y[:, torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
    rel = O.bound_relative_error(Yr, Xc @ A_r.T, np.abs(Xc) @ np.abs(A_r).T, floor=O.FLT_MIN)
    assert rel.max() <= TOL, rel.max()
    # stored split-BF16 path over the crop's field points, every pixel: the two paths each
    # hold their own bound against the exact image (fused TOL, stored 1e-5), so they differ
    # by at most the sum, per pixel, relative to sum_j |A_ij||x_j|.  The library is
    # non-negative, so that sum is A |x|, taken from the stored path itself.
    assert lib32.min() >= 0.0
    pts = np.stack([xs[cols], ys[cols]], axis=1)
    stored = _plan(lib32, w.radii, w.s, points=pts, storage="split_bf16")
    Xc_d = torch.from_numpy(np.ascontiguousarray(X[:, cols])).to(DEV)
    Ys = stored.forward(Xc_d)
    bound = stored.forward(Xc_d.abs()).clamp_min(O.FLT_MIN)
    torch.cuda.synchronize()
    assert stored.sync_status() == 0
    rel = ((Ys - Y).abs() / bound).max().item()
    assert rel <= TOL + 1e-5, rel


def test_fused_with_nonuniform_radii():
    """IPAC-like offset sampling (dense near the centre, sparse further out)."""
    rng = np.random.default_rng(91)
    n, N, S = 28, 24, 0.25
    radii = np.unique(np.concatenate([np.arange(0.0, 1.5, 0.06), np.arange(1.5, 3.0, 0.5), [3.0, 3.25, 3.5]]))
    lib32 = rng.uniform(0.0, 1.0, (len(radii), n, n)).astype(np.float32)
    plan = _plan(lib32, radii, 0.25, N=N, S=S, storage="fused")
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    x = rng.uniform(0.0, 1.0, (5, N * N)).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    for b in range(5):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], A @ x64, np.abs(A) @ np.abs(x64), floor=O.FLT_MIN)
        assert rel.max() <= TOL, rel.max()
