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


@pytest.mark.parametrize("capacity", [None, 48])
def test_full_size_uneven_launch_against_oracle_rows(capacity):
    """The uneven workload's launch at full size: all 10 (N, S) buckets with their own
    split-BF16 A (16384 x N^2) on the 128^2 library, one multi-job persistent launch, with
    the capacity the bench's waves need (narrow accumulators, two CTAs per SM) and with 48
    scenes per bucket (wide accumulators, one CTA per SM).  Uneven counts, one of them zero;
    64 seeded rows per bucket against the oracle, every present scene."""
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.serve import MultiForward
    from synth import workloads
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    lib = torch.from_numpy(lib32).to(DEV)
    buckets = workloads.uneven_buckets()
    cap = capacity or workloads.uneven_arrivals(500, 50, w.seed + 9)[2]
    plans = [Plan(lib, w.radii, w.s, N=k[0], S=k[1], storage="split_bf16") for k in buckets]
    mf = MultiForward(plans, [cap] * len(buckets))
    rng = np.random.default_rng(404 + cap)
    counts = rng.integers(1, cap + 1, len(buckets))
    counts[3] = 0
    counts[7] = cap
    X = []
    for j, k in enumerate(buckets):
        xs = np.stack([workloads.random_ring_scene(k[0], k[1], w.r_max, 50000 + 100 * j + b).ravel()
                       for b in range(cap)]).astype(np.float32)
        X.append(xs)
        mf.x[j].copy_(torch.from_numpy(xs))
        mf.y[j].fill_(float("nan"))
    mf.count.copy_(torch.from_numpy(counts.astype(np.int32)))
    mf.enqueue()
    torch.cuda.synchronize()
    assert plans[0].sync_status() == 0
    for j, k in enumerate(buckets):
        rows = np.sort(np.random.default_rng(j).choice(w.M, 64, replace=False))
        xo, yo = O.scene_offsets(k[0], k[1])
        A_r = O.A_rows(lib32.astype(np.float64), w.radii, xo, yo, rows)
        y = mf.y[j].cpu().numpy()
        nb = int(counts[j])
        Xb = X[j][:nb].astype(np.float64)
        if nb:
            rel = O.bound_relative_error(y[:nb][:, rows], Xb @ A_r.T, np.abs(Xb) @ np.abs(A_r).T, floor=O.FLT_MIN)
            assert rel.max() <= 1e-5, (k, rel.max())
        assert np.all(np.isnan(y[nb:]))           # slots beyond the count are not written
    for p in plans:
        p.free()
