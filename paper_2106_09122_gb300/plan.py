"""Python face of the psfsim C ABI: a built interpolated PSF library on one GPU.

PyTorch supplies device memory and streams; every computation is a call into
libpsfsim (argument marshalling only, no fallback path).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as B

_STORAGE = {"fp32": B.FP32, "split_bf16": B.SPLIT_BF16, "bf16": B.BF16, "fp32_sym": B.FP32_SYM, "fused": B.FUSED,
            "split_bf16_sym": B.SPLIT_BF16_SYM}
_INTERP = {"linear": B.LINEAR, "nearest": B.NEAREST}


def _stream_ptr(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def workspace_bytes(n: int, n_r: int, K: int, storage: str = "fp32") -> int:
    out = ctypes.c_size_t()
    B.check(B.load().psfsim_workspace_bytes(n, n_r, K, _STORAGE[storage], ctypes.byref(out)), "workspace_bytes")
    return out.value


class Plan:
    """A built library A (n^2 x K) living in a caller-owned (torch) workspace."""

    def __init__(self, lib: torch.Tensor, radii, s: float, *, N: int | None = None, S: float | None = None,
                 points=None, storage: str = "fp32", interp: str = "linear", stream=None):
        self._lib = B.load()
        self.lib = _dev_f32(lib, "lib")
        if lib.dim() != 3 or lib.shape[1] != lib.shape[2]:
            raise ValueError("lib must be [n_r, n, n]")
        self.n_r, self.n = int(lib.shape[0]), int(lib.shape[1])
        self.radii = np.ascontiguousarray(radii, dtype=np.float64)
        self.storage = storage
        if points is not None:
            pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
            K = pts.shape[0]
        else:
            K = int(N) * int(N)
        self.K, self.M = K, self.n * self.n
        ws = workspace_bytes(self.n, self.n_r, K, storage)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=lib.device)
        h = ctypes.c_void_p()
        rp = self.radii.ctypes.data_as(ctypes.c_void_p)
        if points is not None:
            rc = self._lib.psfsim_build_points(
                ctypes.c_void_p(lib.data_ptr()), rp, self.n_r, self.n, float(s),
                pts.ctypes.data_as(ctypes.c_void_p), K, _STORAGE[storage], _INTERP[interp],
                ctypes.c_void_p(self.workspace.data_ptr()), ws, _stream_ptr(stream), ctypes.byref(h))
        else:
            rc = self._lib.psfsim_build(
                ctypes.c_void_p(lib.data_ptr()), rp, self.n_r, self.n, float(s), int(N), float(S),
                _STORAGE[storage], _INTERP[interp], ctypes.c_void_p(self.workspace.data_ptr()), ws,
                _stream_ptr(stream), ctypes.byref(h))
        B.check(rc, "psfsim_build")
        self.handle = h
        self.info = B.Info()
        B.check(self._lib.psfsim_info(h, ctypes.byref(self.info)), "psfsim_info")

    # -- products -----------------------------------------------------------
    def forward_scratch_bytes(self, batch: int) -> int:
        out = ctypes.c_size_t()
        B.check(self._lib.psfsim_forward_scratch_bytes(self.handle, batch, ctypes.byref(out)), "scratch")
        return out.value

    def adjoint_scratch_bytes(self, batch: int) -> int:
        out = ctypes.c_size_t()
        B.check(self._lib.psfsim_adjoint_scratch_bytes(self.handle, batch, ctypes.byref(out)), "scratch")
        return out.value

    def _scratch(self, nbytes: int) -> torch.Tensor:
        return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.lib.device)

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None, scratch: torch.Tensor | None = None,
                stream=None, skip_zeros: bool = False) -> torch.Tensor:
        """S = A Z for x of shape [K] or [B, K] (float32, CUDA).  skip_zeros (FP32 storage): read
        only the columns of scene pixels that are non-zero in some scene (psfsim_forward_sparse)."""
        _dev_f32(x, "x")
        xb = x.view(-1, self.K)
        bsz = xb.shape[0]
        y = out if out is not None else torch.empty((bsz, self.M), dtype=torch.float32, device=x.device)
        name = "psfsim_forward_sparse" if skip_zeros else "psfsim_forward"
        nb = ctypes.c_size_t()
        B.check(getattr(self._lib, name + "_scratch_bytes")(self.handle, bsz, ctypes.byref(nb)), "scratch")
        if scratch is None or scratch.numel() < nb.value:
            scratch = self._scratch(nb.value)
        B.check(getattr(self._lib, name)(self.handle, ctypes.c_void_p(xb.data_ptr()), bsz,
                                         ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(scratch.data_ptr()),
                                         scratch.numel(), _stream_ptr(stream)), name)
        return y.view(self.M) if x.dim() == 1 else y

    def adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None, scratch: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
        """A^T g for g of shape [M] or [B, M] (float32, CUDA)."""
        _dev_f32(g, "g")
        gb = g.view(-1, self.M)
        bsz = gb.shape[0]
        gx = out if out is not None else torch.empty((bsz, self.K), dtype=torch.float32, device=g.device)
        need = self.adjoint_scratch_bytes(bsz)
        if scratch is None or scratch.numel() < need:
            scratch = self._scratch(need)
        B.check(self._lib.psfsim_adjoint(self.handle, ctypes.c_void_p(gb.data_ptr()), bsz,
                                         ctypes.c_void_p(gx.data_ptr()), ctypes.c_void_p(scratch.data_ptr()),
                                         scratch.numel(), _stream_ptr(stream)), "psfsim_adjoint")
        return gx.view(self.K) if g.dim() == 1 else gx

    def sync_status(self, stream=None) -> int:
        return self._lib.psfsim_sync_status(self.handle, _stream_ptr(stream))

    # -- views of the stored matrix (for tests and comparators) --------------
    def A_fp32(self) -> torch.Tensor:
        """The stored FP32 A as an [M, K] view (column-major in memory)."""
        if self.info.storage != B.FP32:
            raise ValueError("A_fp32 needs FP32 storage")
        ld = self.info.ld
        flat = self.workspace[self.info.a_offset:self.info.a_offset + ld * self.K * 4].view(torch.float32)
        return flat.view(self.K, ld)[:, : self.M].t()

    def A_split(self):
        """(hi [rows, ld] bf16, lo [rows, ld] bf16 or None, scale [ld] f32) views of split-BF16
        (or BF16: no lo) storage."""
        if self.info.storage not in (B.SPLIT_BF16, B.BF16, B.SPLIT_BF16_SYM):
            raise ValueError("A_split needs SPLIT_BF16, BF16 or SPLIT_BF16_SYM storage")
        ld = self.info.ld
        rows = (self.M + 127) // 128 * 128
        nb = rows * ld * 2
        hi = self.workspace[self.info.a_offset:self.info.a_offset + nb].view(torch.bfloat16).view(rows, ld)
        lo = None
        if self.info.lo_offset >= 0:
            lo = self.workspace[self.info.lo_offset:self.info.lo_offset + nb].view(torch.bfloat16).view(rows, ld)
        sc = self.workspace[self.info.scale_offset:self.info.scale_offset + ld * 4].view(torch.float32)
        return hi, lo, sc

    def free(self) -> None:
        if getattr(self, "handle", None):
            self._lib.psfsim_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
