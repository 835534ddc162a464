"""psfsim_forward_static: the forward product for callers that cannot allocate.

Some callers of this library cannot allocate device memory at the moment they
simulate an image (a plug-in inside a host application that owns the GPU's
allocator, or a fixed-memory loop) and have no spare buffer to pass as
scratch.  psfsim_forward_static keeps its partial sums in a fixed array inside
the library instead.  These tests call it through the C ABI and compare it
with psfsim_forward, within the image tolerance the other GPU tests use
(1e-5 of sum_j |A_ij||x_j|), on two calls in a row, so that leftovers from the
first call cannot leak into the second.  The file sorts last so that a run
stopping at the first failure has already run every other test; it also runs
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _static_forward(plan, x, y):
    from paper_2106_09122_gb300 import _binding as B
    lib = B.load()
    bsz = x.numel() // plan.K
    return lib.psfsim_forward_static(plan.handle, ctypes.c_void_p(x.data_ptr()), bsz,
                                     ctypes.c_void_p(y.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _bound(plan, x):
    return (plan.A_fp32().abs() @ x.view(-1, plan.K).abs().t()).t()


@pytest.mark.parametrize("make", [workloads.plain_small, workloads.adjoint_128])
def test_static_forward_matches_forward_on_two_calls(make):
    from paper_2106_09122_gb300 import Plan, _binding as B
    w = make()
    plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(DEV), w.radii, w.s, N=w.N, S=w.S)
    scenes = torch.from_numpy(workloads.scene_batch(w, 3).astype(np.float32)).to(DEV)
    calls = [scenes[0].contiguous(), scenes[1:3].contiguous()]       # B = 1, then B = 2
    for x in calls:
        y_static = torch.full((x.numel() // plan.K, plan.M), float("nan"), device=DEV)
        assert _static_forward(plan, x, y_static) == B.OK
        y_ref = plan.forward(x).view(-1, plan.M)
        torch.cuda.synchronize()
        err = (y_static - y_ref).abs()
        assert torch.all(err <= 1e-5 * _bound(plan, x)), float(err.max())
    plan.free()


def test_static_forward_rejects_batches_beyond_the_array():
    from paper_2106_09122_gb300 import Plan, _binding as B
    w = workloads.adjoint_128()
    plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(DEV), w.radii, w.s, N=w.N, S=w.S)
    per_scene = plan.forward_scratch_bytes(1)
    too_many = B.STATIC_SCRATCH_BYTES // per_scene + 1
    x = torch.zeros((too_many, plan.K), device=DEV)
    y = torch.full((too_many, plan.M), 7.0, device=DEV)
    assert _static_forward(plan, x, y) == B.ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.all(y == 7.0)
    plan.free()
