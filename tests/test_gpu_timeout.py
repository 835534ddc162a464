"""The bounded-wait failure path of the tensor-core forwards (the stored
split-BF16 product and the fused on-chip one), driven on a GPU without
faulting, trapping or hanging it.

psfsim_debug_forward_stall runs the forward on one CTA with every device-side
wait limited to 1 ms and one shared-memory stage that the TMA producer never
fills.  The MMA issuer's wait for that stage runs out; the kernel must then
record PSFSIM_ERR_TIMEOUT, wait for the copies and MMAs it already issued,
release its tensor memory and return.  Afterwards the same plan, on the same
stream and context, must give correct images again.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

from oracle import psfsim_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _tiny_plan():
    from paper_2106_09122_gb300 import Plan
    rng = np.random.default_rng(303)
    n, N, S = 16, 8, 0.4
    radii = np.linspace(0.0, 3.0, 7)
    lib32 = rng.uniform(0.0, 1.0, (7, n, n)).astype(np.float32)
    plan = Plan(torch.from_numpy(lib32).to(DEV), radii, 0.5, N=N, S=S, storage="split_bf16")
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    x = rng.uniform(0.0, 1.0, (4, N * N)).astype(np.float32)
    return plan, A, x


def _stall(plan, x, y, scr, wait_ns, stall_load):
    from paper_2106_09122_gb300 import _binding as B
    lib = B.load()
    return lib.psfsim_debug_forward_stall(plan.handle, ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                          ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(scr.data_ptr()),
                                          scr.numel(), wait_ns, stall_load,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _check(y, A, x):
    for b in range(x.shape[0]):
        x64 = x[b].astype(np.float64)
        rel = O.bound_relative_error(y[b].astype(np.float64), A @ x64, np.abs(A) @ np.abs(x64), floor=O.FLT_MIN)
        assert rel.max() <= 1e-5, (b, rel.max())


def test_wait_that_runs_out_reports_timeout_and_leaves_the_plan_usable():
    from paper_2106_09122_gb300 import _binding as B
    plan, A, x_np = _tiny_plan()
    x = torch.from_numpy(x_np).to(DEV)
    y = torch.zeros((4, plan.M), device=DEV)
    scr = torch.empty(plan.forward_scratch_bytes(4), dtype=torch.uint8, device=DEV)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert _stall(plan, x, y, scr, 1_000_000, 0) == B.OK
    assert plan.sync_status() == B.ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    assert elapsed < 1.5, elapsed              # a few 1 ms waits, not the 2 s default
    # the status word is sticky until cleared
    assert plan.sync_status() == B.ERR_TIMEOUT
    assert plan._lib.psfsim_reset_status(plan.handle, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == B.OK
    assert plan.sync_status() == B.OK
    # same plan, same context: a normal launch is correct right after
    y2 = plan.forward(x)
    assert plan.sync_status() == B.OK
    _check(y2.cpu().numpy(), A, x_np)
    plan.free()


def test_stall_hook_without_a_stall_is_a_correct_one_cta_forward():
    from paper_2106_09122_gb300 import _binding as B
    plan, A, x_np = _tiny_plan()
    x = torch.from_numpy(x_np).to(DEV)
    y = torch.full((4, plan.M), float("nan"), device=DEV)
    scr = torch.empty(plan.forward_scratch_bytes(4), dtype=torch.uint8, device=DEV)
    assert _stall(plan, x, y, scr, 1_000_000_000, -1) == B.OK
    assert plan.sync_status() == B.OK
    _check(y.cpu().numpy(), A, x_np)
    plan.free()


def test_stall_hook_rejects_bad_limits():
    from paper_2106_09122_gb300 import _binding as B
    plan, _, x_np = _tiny_plan()
    x = torch.from_numpy(x_np).to(DEV)
    y = torch.zeros((4, plan.M), device=DEV)
    scr = torch.empty(plan.forward_scratch_bytes(4), dtype=torch.uint8, device=DEV)
    assert _stall(plan, x, y, scr, 10, 0) == B.ERR_ARG              # below 1 us
    assert _stall(plan, x, y, scr, 5_000_000_000, 0) == B.ERR_ARG   # above 2 s
    assert _stall(plan, x, y, scr, 1_000_000, -2) == B.ERR_ARG
    plan.free()


def _tiny_fused_plan(scenes=3):
    from paper_2106_09122_gb300 import Plan
    rng = np.random.default_rng(404)
    n, N, S = 40, 32, 0.3
    radii = np.linspace(0.0, 4.5, 12)
    lib32 = rng.uniform(0.0, 1.0, (12, n, n)).astype(np.float32)
    plan = Plan(torch.from_numpy(lib32).to(DEV), radii, 0.5, N=N, S=S, storage="fused")
    A = O.build_A(lib32.astype(np.float64), radii, N, S)
    x = rng.uniform(0.0, 1.0, (scenes, N * N)).astype(np.float32)
    return plan, A, x


def _check_fused(y, A, x):
    # the fused path's bound (split-BF16 A and x, dropped lo x2, 60-MMA accumulations)
    x64 = x.astype(np.float64)
    rel = O.bound_relative_error(y.astype(np.float64), x64 @ A.T, np.abs(x64) @ np.abs(A).T, floor=O.FLT_MIN)
    assert rel.max() <= 2.5e-5, rel.max()


@pytest.mark.parametrize("stall_load,scenes", [(0, 3), (1, 3), (3, 3), (1, 40)])
def test_fused_wait_that_runs_out_reports_timeout_and_leaves_the_plan_usable(stall_load, scenes):
    # 40 scenes run the 64-scene form (one accumulator, two boxes per scene tile)
    from paper_2106_09122_gb300 import _binding as B
    plan, A, x_np = _tiny_fused_plan(scenes)
    x = torch.from_numpy(x_np).to(DEV)
    y = torch.zeros((scenes, plan.M), device=DEV)
    scr = torch.empty(plan.forward_scratch_bytes(scenes), dtype=torch.uint8, device=DEV)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert _stall(plan, x, y, scr, 1_000_000, stall_load) == B.OK
    assert plan.sync_status() == B.ERR_TIMEOUT
    elapsed = time.perf_counter() - t0
    assert elapsed < 1.5, elapsed
    assert plan._lib.psfsim_reset_status(plan.handle, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == B.OK
    assert plan.sync_status() == B.OK
    y2 = plan.forward(x)
    assert plan.sync_status() == B.OK
    _check_fused(y2.cpu().numpy(), A, x_np)
    plan.free()


def test_fused_stall_hook_without_a_stall_is_a_correct_one_cta_forward():
    from paper_2106_09122_gb300 import _binding as B
    plan, A, x_np = _tiny_fused_plan()
    x = torch.from_numpy(x_np).to(DEV)
    y = torch.full((3, plan.M), float("nan"), device=DEV)
    scr = torch.empty(plan.forward_scratch_bytes(3), dtype=torch.uint8, device=DEV)
    assert _stall(plan, x, y, scr, 1_000_000_000, -1) == B.OK
    assert plan.sync_status() == B.OK
    _check_fused(y.cpu().numpy(), A, x_np)
    plan.free()


def test_fused_stall_hook_rejects_batches_beyond_one_launch():
    from paper_2106_09122_gb300 import _binding as B
    plan, _, _ = _tiny_fused_plan()
    x = torch.zeros((65, plan.K), device=DEV)
    y = torch.zeros((65, plan.M), device=DEV)
    scr = torch.empty(plan.forward_scratch_bytes(65), dtype=torch.uint8, device=DEV)
    assert _stall(plan, x, y, scr, 1_000_000, 0) == B.ERR_ARG
    plan.free()
