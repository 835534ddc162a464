"""GPU parity of the multi-job persistent tensor-core forward (uneven scene
sizes and pixel scales, one launch), its autotuner, and graph-captured waves,
against the FP64 oracle (per-pixel bound-relative error <= 1e-5)."""
import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _setup(seed=71):
    from paper_2106_09122_gb300 import Plan
    rng = np.random.default_rng(seed)
    n, s = 24, 0.25
    radii = np.linspace(0.0, 4.0, 10)
    lib32 = rng.uniform(0.0, 1.0, (10, n, n)).astype(np.float32)
    lib = torch.from_numpy(lib32).to(DEV)
    buckets = [(N, S) for N in (8, 12, 16) for S in (0.3, 0.5)]
    plans = {k: Plan(lib, radii, s, N=k[0], S=k[1], storage="split_bf16") for k in buckets}
    As = {k: O.build_A(lib32.astype(np.float64), radii, k[0], k[1]) for k in buckets}
    return rng, buckets, plans, As


def _check(y, A, x):
    x64 = np.asarray(x, dtype=np.float64)
    rel = O.bound_relative_error(np.asarray(y, dtype=np.float64), A @ x64, np.abs(A) @ np.abs(x64), floor=O.FLT_MIN)
    assert rel.max() <= 1e-5, rel.max()


def test_multi_job_forward_and_counts():
    from paper_2106_09122_gb300.serve import MultiForward
    rng, buckets, plans, As = _setup()
    mf = MultiForward([plans[k] for k in buckets], [8] * len(buckets))
    counts = rng.integers(0, 9, len(buckets))
    for j, k in enumerate(buckets):
        mf.x[j].copy_(torch.rand(8, k[0] * k[0], device=DEV))
        mf.y[j].fill_(float("nan"))
    mf.count.copy_(torch.from_numpy(counts.astype(np.int32)))
    mf.enqueue()
    torch.cuda.synchronize()
    for j, k in enumerate(buckets):
        y = mf.y[j].cpu().numpy()
        for b in range(8):
            if b < counts[j]:
                _check(y[b], As[k], mf.x[j][b].cpu().numpy())
            else:
                assert np.all(np.isnan(y[b]))       # slots beyond the count are not written


def test_autotuner_picks_a_correct_shape():
    from paper_2106_09122_gb300.serve import MultiForward, autotune
    rng, buckets, plans, As = _setup(72)
    mf = MultiForward([plans[k] for k in buckets], [5] * len(buckets))
    for j, k in enumerate(buckets):
        mf.x[j].copy_(torch.rand(5, k[0] * k[0], device=DEV))
    mf.count.fill_(5)
    best, ms, results = autotune(mf, chunks=(1, 4, 8), units=(1, 4), reps=2)
    assert best in [r[0] for r in results] and ms == min(r[1] for r in results)
    mf.enqueue()
    torch.cuda.synchronize()
    for j, k in enumerate(buckets):
        for b in range(5):
            _check(mf.y[j][b].cpu().numpy(), As[k], mf.x[j][b].cpu().numpy())


def test_graph_replayed_waves_of_different_composition():
    from paper_2106_09122_gb300.serve import UnevenServer
    rng, buckets, plans, As = _setup(73)
    server = UnevenServer(plans, capacity=6)
    server.capture()
    for wave_no in range(3):
        keys = [buckets[i] for i in rng.integers(0, len(buckets), 12)]
        keys = [k for i, k in enumerate(keys) if keys[:i].count(k) < 6]
        wave = [(k, rng.uniform(0.0, 1.0, k[0] * k[0]).astype(np.float32)) for k in keys]
        out = server.run_wave(wave)
        for (k, x), y in zip(wave, out):
            _check(y.numpy(), As[k], x)
