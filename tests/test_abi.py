"""C-ABI checks that need no GPU: the library loads, exports every symbol the
headers declare, and rejects bad arguments on the host before any launch."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2106_09122_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names |= set(re.findall(r"\b(psfsim_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_2106_09122_gb300 import build_lib
        build_lib.build()
    return B.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert "psfsim_build" in names and "psfsim_forward" in names and "psfsim_adjoint" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in B.SIGNATURES, n


def test_status_strings(lib):
    for code in (B.OK, B.ERR_ARG, B.ERR_RADII, B.ERR_WORKSPACE, B.ERR_CUDA, B.ERR_UNSUPPORTED, B.ERR_TIMEOUT):
        assert B.status_string(code) and B.status_string(code) != "unknown status"


def test_workspace_bytes_covers_A(lib):
    out = ctypes.c_size_t()
    assert lib.psfsim_workspace_bytes(128, 40, 128 * 128, B.FP32, ctypes.byref(out)) == B.OK
    assert out.value >= 128 * 128 * 128 * 128 * 4
    assert lib.psfsim_workspace_bytes(128, 40, 128 * 128, B.SPLIT_BF16, ctypes.byref(out)) == B.OK
    assert out.value >= 2 * 2 * 128 * 128 * 128 * 128
    split = out.value
    assert lib.psfsim_workspace_bytes(128, 40, 128 * 128, B.BF16, ctypes.byref(out)) == B.OK
    assert 2 * 128 * 128 * 128 * 128 <= out.value < split - 128 ** 4  # hi alone: no lo array
    assert lib.psfsim_workspace_bytes(128, 40, 128 * 128, B.SPLIT_BF16_SYM, ctypes.byref(out)) == B.OK
    assert 4 * 128 * 128 * 128 * 128 // 4 <= out.value < split // 3  # hi + lo of the quadrant's columns
    assert lib.psfsim_workspace_bytes(512, 80, 512 * 512, B.FUSED, ctypes.byref(out)) == B.OK
    assert 79 * 513 * 513 * 32 <= out.value < 2 ** 30          # pair entries of the 79 radial brackets
    assert lib.psfsim_workspace_bytes(0, 4, 10, B.FP32, ctypes.byref(out)) == B.ERR_ARG
    assert lib.psfsim_workspace_bytes(16, 1, 10, B.FP32, ctypes.byref(out)) == B.ERR_ARG
    assert lib.psfsim_workspace_bytes(16, 4, 10, 7, ctypes.byref(out)) == B.ERR_ARG
    assert lib.psfsim_workspace_bytes(16, 4, 10, B.FP32, None) == B.ERR_ARG


def _build(lib, radii, lib_ptr=0x1000, ws_ptr=0x100000, ws_bytes=1 << 40, n=16, N=8, storage=B.FP32):
    h = ctypes.c_void_p()
    r = np.ascontiguousarray(radii, dtype=np.float64)
    rc = lib.psfsim_build(ctypes.c_void_p(lib_ptr), r.ctypes.data_as(ctypes.c_void_p), len(r), n, 0.5, N, 0.5,
                          storage, B.LINEAR, ctypes.c_void_p(ws_ptr), ws_bytes, None, ctypes.byref(h))
    return rc, h


def test_build_rejects_bad_arguments_before_launch(lib):
    good = [0.0, 1.0, 2.0]
    assert _build(lib, [0.0, 1.0, 1.0])[0] == B.ERR_RADII
    assert _build(lib, [0.0, np.nan])[0] == B.ERR_RADII
    assert _build(lib, [0.0])[0] == B.ERR_RADII
    assert _build(lib, good, lib_ptr=0)[0] == B.ERR_ARG
    assert _build(lib, good, lib_ptr=0x1004)[0] == B.ERR_ARG       # library not 16-byte aligned
    assert _build(lib, good, ws_ptr=0x100010)[0] == B.ERR_WORKSPACE  # workspace not 256-byte aligned
    assert _build(lib, good, ws_bytes=1024)[0] == B.ERR_WORKSPACE
    assert _build(lib, good, n=0)[0] == B.ERR_ARG
    assert _build(lib, good, N=0)[0] == B.ERR_ARG
    rc, h = _build(lib, good, n=0)
    assert h.value is None


def test_symmetric_storages_need_an_even_scene_grid(lib):
    assert _build(lib, [0.0, 1.0, 2.0], N=9, storage=B.FUSED)[0] == B.ERR_UNSUPPORTED
    assert _build(lib, [0.0, 1.0, 2.0], N=9, storage=B.FP32_SYM)[0] == B.ERR_UNSUPPORTED
    assert _build(lib, [0.0, 1.0, 2.0], N=9, storage=B.SPLIT_BF16_SYM)[0] == B.ERR_UNSUPPORTED


def test_products_reject_null_handles(lib):
    assert lib.psfsim_forward(None, None, 1, None, None, 0, None) == B.ERR_ARG
    assert lib.psfsim_adjoint(None, None, 1, None, None, 0, None) == B.ERR_ARG
    assert lib.psfsim_info(None, None) == B.ERR_ARG
    lib.psfsim_free(None)


def test_status_and_testing_hooks_reject_null_handles(lib):
    assert lib.psfsim_reset_status(None, None) == B.ERR_ARG
    assert lib.psfsim_sync_status(None, None) == B.ERR_ARG
    assert lib.psfsim_debug_forward_stall(None, None, 1, None, None, 0, 1_000_000, 0, None) == B.ERR_ARG
