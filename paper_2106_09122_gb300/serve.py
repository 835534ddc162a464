"""Uneven-size batches: many scenes of different sizes and pixel scales.

Each (N, S) bucket has its own stored split-BF16 A (n^2 x N^2, Sec. 3 with
n != N, s != S).  A wave of arriving scenes is simulated by ONE
psfsim_forward_multi call: a persistent tensor-core launch whose work units
interleave every bucket.  Scene counts per bucket live in device memory, so
that launch (split, GEMM, reductions) is captured once in a CUDA graph and
replayed for every wave whatever its composition; the copies around it move
exactly the scenes present and the images written.  The launch shape (drain
chunk, units per SM, pipeline stages) is picked by `autotune`, which times
candidate shapes on the actual job set.
"""
from __future__ import annotations

import ctypes
import itertools
import time

import numpy as np
import torch

from . import _binding as B
from .plan import Plan


def _vp(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class MultiForward:
    """Scene, image and count buffers and the C-ABI job table for one set of plans.

    The buffers are device memory by default; `x`, `y` and `count` may instead be given, e.g.
    pinned host tensors, which the kernels then read and write in place through the device's
    mapping of pinned memory (no staging copies)."""

    def __init__(self, plans: list[Plan], capacity: list[int], tuning=None, x=None, y=None, count=None):
        if not plans or len(plans) > 16:
            raise ValueError("1..16 plans")
        self.lib = B.load()
        self.plans = plans
        dev = plans[0].lib.device
        self.x = x if x is not None else [torch.zeros((c, p.K), dtype=torch.float32, device=dev)
                                          for p, c in zip(plans, capacity)]
        self.y = y if y is not None else [torch.zeros((c, p.M), dtype=torch.float32, device=dev)
                                          for p, c in zip(plans, capacity)]
        self.count = count if count is not None else torch.zeros(len(plans), dtype=torch.int32, device=dev)
        jobs = (B.Job * len(plans))()
        for j, (p, c) in enumerate(zip(plans, capacity)):
            jobs[j] = B.Job(p.handle, _vp(self.x[j]), _vp(self.y[j]), c,
                            ctypes.c_void_p(self.count.data_ptr() + 4 * j))
        self.jobs = jobs
        self.set_tuning(tuning)

    def set_tuning(self, tuning) -> None:
        self.tuning = B.Tuning(*tuning) if tuning else None
        tp = ctypes.byref(self.tuning) if self.tuning else None
        nb = ctypes.c_size_t()
        B.check(self.lib.psfsim_forward_multi_scratch_bytes(self.jobs, len(self.plans), tp, ctypes.byref(nb)),
                "multi scratch")
        self.scratch = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=self.plans[0].lib.device)

    def enqueue(self, stream=None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream()
        tp = ctypes.byref(self.tuning) if self.tuning else None
        B.check(self.lib.psfsim_forward_multi(self.jobs, len(self.plans), tp, _vp(self.scratch),
                                              self.scratch.numel(), ctypes.c_void_p(s.cuda_stream)),
                "psfsim_forward_multi")


def autotune(mf: MultiForward, chunks=(2, 4, 8), units=(2, 4, 8), stages=(0,), reps: int = 3):
    """Time every candidate launch shape on the job set; keep and return the fastest."""
    best, best_ms = None, float("inf")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    for ch, up, sg in itertools.product(chunks, units, stages):
        mf.set_tuning((ch, up, sg))
        mf.enqueue()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            mf.enqueue()
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        results.append(((ch, up, sg), ms))
        if ms < best_ms:
            best, best_ms = (ch, up, sg), ms
    mf.set_tuning(best)
    return best, best_ms, results


class UnevenServer:
    """Serve waves of scenes of mixed (N, S) through one persistent multi-job launch.

    Scenes, images and per-bucket counts live in pinned host memory that the kernels read and
    write directly through the device's mapping of pinned memory (over NVLink-C2C on
    Grace-Blackwell): each scene of a wave is copied once, into the next free slot of its
    bucket in the staging buffers; the whole wave (the multi-job split, GEMM and reductions,
    reading only the scenes present and writing only the images of present slots) is one
    captured CUDA graph per staging set.  Two staging sets let the next wave be packed while the
    GPU works on this one.
    """

    def __init__(self, plans: dict, capacity: int, tuning=None):
        self.keys = list(plans.keys())
        self.index = {k: j for j, k in enumerate(self.keys)}
        self.capacity = capacity
        dev = next(iter(plans.values())).lib.device
        self.stream = torch.cuda.Stream(device=dev)
        nb = len(self.keys)
        pl = [plans[k] for k in self.keys]
        self.h_count = [torch.zeros(nb, dtype=torch.int32).pin_memory() for _ in range(2)]
        self.h_x = [[torch.zeros((capacity, p.K), dtype=torch.float32).pin_memory() for p in pl] for _ in range(2)]
        self.h_y = [[torch.zeros((capacity, p.M), dtype=torch.float32).pin_memory() for p in pl] for _ in range(2)]
        self.sets = [MultiForward(pl, [capacity] * nb, tuning, x=self.h_x[i], y=self.h_y[i], count=self.h_count[i])
                     for i in range(2)]
        self.nx = [[t.numpy() for t in hx] for hx in self.h_x]   # numpy views of the staging
        self.ny = [[t.numpy() for t in hy] for hy in self.h_y]
        self.ncount = [t.numpy() for t in self.h_count]
        self.mf = self.sets[0]
        self.graphs = [None, None]
        self.done = [torch.cuda.Event() for _ in range(2)]
        self.copies = {"h2d_bytes": 0, "d2h_bytes": 0}

    def set_tuning(self, tuning) -> None:
        for mf in self.sets:
            mf.set_tuning(tuning)

    def capture(self) -> None:
        """Capture each staging set's whole wave (the multi-job forward on mapped buffers)."""
        torch.cuda.synchronize()
        for i, mf in enumerate(self.sets):
            with torch.cuda.stream(self.stream):
                mf.enqueue(self.stream)
            self.stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                mf.enqueue(self.stream)
            self.graphs[i] = g

    def _pack(self, buf: int, wave):
        """Copy each scene of the wave into the next free slot of its bucket in the staging set."""
        counts = [0] * len(self.keys)
        slots = []
        nx = self.nx[buf]
        for key, x in wave:
            j = self.index[key]
            b = counts[j]
            if b >= self.capacity:
                raise ValueError("bucket capacity exceeded")
            nx[j][b] = x
            counts[j] = b + 1
            slots.append((j, b))
        self.ncount[buf][:] = counts
        return counts, slots

    def _launch(self, buf: int, counts) -> None:
        # the kernels read exactly the scenes present and write exactly their images, in place
        for j, c in enumerate(counts):
            self.copies["h2d_bytes"] += c * self.h_x[buf][j].shape[1] * 4
            self.copies["d2h_bytes"] += c * self.h_y[buf][j].shape[1] * 4
        with torch.cuda.stream(self.stream):
            if self.graphs[buf] is not None:
                self.graphs[buf].replay()
            else:
                self.sets[buf].enqueue(self.stream)
            self.done[buf].record(self.stream)

    def _images(self, buf: int, counts, slots, copy: bool):
        """The wave's images in wave order.  copy=True: each bucket's present images leave the
        staging set in one block copy, and the images are views of those blocks; copy=False:
        views into the staging set, valid until the next wave that uses it."""
        if not copy:
            return [self.h_y[buf][j][b] for j, b in slots]
        ny = self.ny[buf]
        blocks = {j: torch.from_numpy(ny[j][:c].copy()) for j, c in enumerate(counts) if c}
        return [blocks[j][b] for j, b in slots]

    def run_wave(self, wave, copy: bool = True):
        """wave: list of (bucket key, scene vector).  Returns the images in wave order (see
        _images for copy)."""
        counts, slots = self._pack(0, wave)
        self._launch(0, counts)
        self.done[0].synchronize()
        return self._images(0, counts, slots, copy)

    def run_waves(self, waves):
        """Serve waves back to back: wave i + 1 is packed on the host while the GPU works on
        wave i.  Yields (images in wave order, seconds from the start of the wave's packing to
        its images being in host memory) per wave."""
        pending = None
        for i, wave in enumerate(waves):
            buf = i & 1
            t0 = time.perf_counter()
            # the staging set of wave i - 1 is still in use; wave i - 2's (this one) is free
            counts, slots = self._pack(buf, wave)
            self._launch(buf, counts)
            if pending is not None:
                yield self._collect(*pending)
            pending = (buf, counts, slots, t0)
        if pending is not None:
            yield self._collect(*pending)

    def _collect(self, buf, counts, slots, t0):
        self.done[buf].synchronize()
        images = self._images(buf, counts, slots, True)
        return images, time.perf_counter() - t0
