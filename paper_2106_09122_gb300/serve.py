"""Uneven-size batches: many scenes of different sizes and pixel scales.

Each (N, S) bucket has its own stored split-BF16 A (n^2 x N^2, Sec. 3 with
n != N, s != S).  A wave of arriving scenes is simulated by ONE
psfsim_forward_multi call: a persistent tensor-core launch whose work units
interleave every bucket.  Scene counts per bucket live in device memory, so
the whole wave (input gather, split, GEMM, reductions) is captured once in a
CUDA graph and replayed for every wave whatever its composition.  The launch
shape (drain chunk, units per SM, pipeline stages) is picked by `autotune`,
which times candidate shapes on the actual job set.
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
    """Device buffers and the C-ABI job table for one set of plans."""

    def __init__(self, plans: list[Plan], capacity: list[int], tuning=None):
        if not plans or len(plans) > 16:
            raise ValueError("1..16 plans")
        self.lib = B.load()
        self.plans = plans
        dev = plans[0].lib.device
        self.x = [torch.zeros((c, p.K), dtype=torch.float32, device=dev) for p, c in zip(plans, capacity)]
        self.y = [torch.zeros((c, p.M), dtype=torch.float32, device=dev) for p, c in zip(plans, capacity)]
        self.count = torch.zeros(len(plans), dtype=torch.int32, device=dev)
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
    """Serve waves of scenes of mixed (N, S) through one captured CUDA graph."""

    def __init__(self, plans: dict, capacity: int, tuning=None):
        self.keys = list(plans.keys())
        self.mf = MultiForward([plans[k] for k in self.keys], [capacity] * len(self.keys), tuning)
        self.capacity = capacity
        self.graph = None
        dev = self.mf.plans[0].lib.device
        self.h_count = torch.zeros(len(self.keys), dtype=torch.int32).pin_memory()
        self.h_x = [torch.zeros((capacity, p.K), dtype=torch.float32).pin_memory() for p in self.mf.plans]
        self.h_y = [torch.zeros((capacity, p.M), dtype=torch.float32).pin_memory() for p in self.mf.plans]
        self.stream = torch.cuda.Stream(device=dev)

    def _wave_ops(self) -> None:
        mf = self.mf
        mf.count.copy_(self.h_count, non_blocking=True)
        for j in range(len(self.keys)):
            mf.x[j].copy_(self.h_x[j], non_blocking=True)
        mf.enqueue(self.stream)
        for j in range(len(self.keys)):
            self.h_y[j].copy_(mf.y[j], non_blocking=True)

    def capture(self) -> None:
        """Capture one wave: H2D of counts and scenes, the multi-job forward, D2H of images."""
        # Warm up the exact op sequence eagerly before capturing it.
        torch.cuda.synchronize()
        with torch.cuda.stream(self.stream):
            self._wave_ops()
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self._wave_ops()
        self.graph = g

    def run_wave(self, wave):
        """wave: list of (bucket key, scene vector).  Returns images in wave order."""
        slots = []
        counts = [0] * len(self.keys)
        for key, x in wave:
            j = self.keys.index(key)
            if counts[j] >= self.capacity:
                raise ValueError("bucket capacity exceeded")
            self.h_x[j][counts[j]].copy_(torch.as_tensor(x, dtype=torch.float32))
            slots.append((j, counts[j]))
            counts[j] += 1
        self.h_count.copy_(torch.tensor(counts, dtype=torch.int32))
        # Replay on the capture stream and wait on that stream: replay() launches
        # on the current stream, and the pinned outputs are read right after.
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._wave_ops()
        self.stream.synchronize()
        return [self.h_y[j][b].clone() for j, b in slots]
