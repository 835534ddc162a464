"""GPU edge cases: large PSFs (global-tap build path), the maximum number of
radii, a library whose every column lies beyond the last radius, empty and
invalid batches, and the device status word."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _plan(lib32, radii, s, **kw):
    from paper_2106_09122_gb300 import Plan
    return Plan(torch.from_numpy(np.ascontiguousarray(lib32)).to(DEV), radii, s, **kw)


@pytest.mark.parametrize("n,storage", [(256, "fp32"), (320, "fp32"), (200, "split_bf16")])
def test_large_psfs_sampled_columns(n, storage):
    rng = np.random.default_rng(n)
    radii = np.linspace(0.0, 10.0, 6)
    lib32 = rng.uniform(0.0, 1.0, (6, n, n)).astype(np.float32)
    N, S = 6, 1.5
    plan = _plan(lib32, radii, 0.1, N=N, S=S, storage=storage)
    x = rng.uniform(0.0, 1.0, (2, N * N)).astype(np.float32)
    y = plan.forward(torch.from_numpy(x).to(DEV)).double().cpu().numpy()
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    for b in range(2):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b], A @ x64, np.abs(A) @ np.abs(x64), floor=O.FLT_MIN)
        assert rel.max() <= 1e-5


def test_maximum_number_of_radii_nonuniform():
    rng = np.random.default_rng(5)
    radii = np.concatenate([[0.0], np.cumsum(rng.uniform(0.005, 0.05, 255))])
    n, N, S = 16, 24, radii[-1] / 10
    lib32 = rng.uniform(0.0, 1.0, (256, n, n)).astype(np.float32)
    plan = _plan(lib32, radii, 0.2, N=N, S=S)
    A_gpu = plan.A_fp32().double().cpu().numpy()
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    assert np.all(np.abs(A_gpu - A) <= 1e-6 * np.abs(A) + 1e-9)


def test_every_column_beyond_the_last_radius_gives_zero_images():
    rng = np.random.default_rng(6)
    radii = np.array([0.0, 0.1, 0.2])
    lib32 = rng.uniform(0.0, 1.0, (3, 12, 12)).astype(np.float32)
    for storage in ("fp32", "split_bf16", "fused"):
        plan = _plan(lib32, radii, 0.5, N=8, S=1.0, storage=storage)
        y = plan.forward(torch.rand(3, 64, device=DEV))
        torch.cuda.synchronize()
        assert not torch.any(y) and plan.sync_status() == 0


def test_empty_and_invalid_batches_are_rejected():
    from paper_2106_09122_gb300 import _binding as B
    lib = B.load()
    rng = np.random.default_rng(7)
    plan = _plan(rng.uniform(0, 1, (3, 8, 8)).astype(np.float32), np.array([0.0, 1.0, 2.0]), 0.5, N=4, S=0.5)
    x = torch.zeros(16, device=DEV)
    y = torch.zeros(64, device=DEV)
    scr = torch.empty(1 << 20, dtype=torch.uint8, device=DEV)
    args = (ctypes.c_void_p(x.data_ptr()), 0, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(scr.data_ptr()),
            scr.numel(), None)
    assert lib.psfsim_forward(plan.handle, *args) == B.ERR_ARG
    assert lib.psfsim_adjoint(plan.handle, *args) == B.ERR_ARG
    # scratch too small
    assert lib.psfsim_forward(plan.handle, ctypes.c_void_p(x.data_ptr()), 1, ctypes.c_void_p(y.data_ptr()),
                              ctypes.c_void_p(scr.data_ptr()), 16, None) == B.ERR_WORKSPACE
    assert plan.sync_status() == 0
