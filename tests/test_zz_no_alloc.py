"""psfsim_forward_static: the forward product for callers that cannot allocate.

Some callers of this library cannot allocate device memory at the moment they
simulate an image (a plug-in inside a host application that owns the GPU's
allocator, or a fixed-memory loop) and have no spare buffer to pass as
scratch.  psfsim_forward_static keeps its partial sums in a fixed array inside
the library instead.  These tests call it through the C ABI and compare it
with psfsim_forward, within the image tolerance the other GPU tests use
(1e-5 of sum_j |A_ij||x_j|), on two calls in a row, so that leftovers from the
first call cannot leak into the second; they check that later calls leave the
device's free memory unchanged, and they repeat the two-call comparison in a
fresh Python process, where the library's device code is loaded by the first
static call itself.  The file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from synth import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_later_static_calls_leave_free_device_memory_unchanged():
    from paper_2106_09122_gb300 import Plan, _binding as B
    w = workloads.plain_small()
    plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(DEV), w.radii, w.s, N=w.N, S=w.S)
    x = torch.from_numpy(workloads.scene_batch(w, 2).astype(np.float32)).to(DEV)
    y = torch.empty((2, plan.M), device=DEV)
    assert _static_forward(plan, x, y) == B.OK       # loads the device code, if not yet loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _static_forward(plan, x, y) == B.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
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


_FRESH = textwrap.dedent("""
    import ctypes, sys
    import numpy as np, torch
    sys.path.insert(0, sys.argv[1])
    from paper_2106_09122_gb300 import Plan, _binding as B
    from synth import workloads
    w = workloads.plain_small()
    plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to("cuda:0"), w.radii, w.s, N=w.N, S=w.S)
    X = torch.from_numpy(workloads.scene_batch(w, 3).astype(np.float32)).to("cuda:0")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    bound = (plan.A_fp32().abs() @ X.abs().t()).t()
    for sl in (slice(0, 1), slice(1, 3)):
        x = X[sl].contiguous()
        y = torch.full((x.shape[0], plan.M), float("nan"), device="cuda:0")
        rc = B.load().psfsim_forward_static(plan.handle, ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                            ctypes.c_void_p(y.data_ptr()), st)
        assert rc == B.OK, rc
        ref = plan.forward(x)
        torch.cuda.synchronize()
        assert torch.all((y - ref).abs() <= 1e-5 * bound[sl]), float((y - ref).abs().max())
    print("fresh-process static forward OK")
""")


def test_static_forward_in_a_fresh_process():
    res = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "fresh-process static forward OK" in res.stdout
