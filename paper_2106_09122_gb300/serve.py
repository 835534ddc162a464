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
    """Serve waves of scenes of mixed (N, S) through one persistent multi-job launch.

    A wave's scenes are grouped by bucket and stacked, one host copy per bucket,
    into pinned staging (two sets, so the next wave is packed while the GPU works
    on this one).  Only the bytes of the scenes present go to the device and only
    the images written come back (one copy per non-empty bucket each way); the
    multi-job forward itself, with its device-side counts, is one captured CUDA
    graph replayed every wave.
    """

    def __init__(self, plans: dict, capacity: int, tuning=None):
        self.keys = list(plans.keys())
        self.index = {k: j for j, k in enumerate(self.keys)}
        self.mf = MultiForward([plans[k] for k in self.keys], [capacity] * len(self.keys), tuning)
        self.capacity = capacity
        self.graph = None
        dev = self.mf.plans[0].lib.device
        self.stream = torch.cuda.Stream(device=dev)
        nb = len(self.keys)
        self.h_count = [torch.zeros(nb, dtype=torch.int32).pin_memory() for _ in range(2)]
        self.h_x = [[torch.zeros((capacity, p.K), dtype=torch.float32).pin_memory() for p in self.mf.plans]
                    for _ in range(2)]
        self.h_y = [[torch.zeros((capacity, p.M), dtype=torch.float32).pin_memory() for p in self.mf.plans]
                    for _ in range(2)]
        self.done = [torch.cuda.Event() for _ in range(2)]
        self.copies = {"h2d_bytes": 0, "d2h_bytes": 0}

    def capture(self) -> None:
        """Capture the multi-job forward (counts, scenes and images stay in device memory)."""
        torch.cuda.synchronize()
        with torch.cuda.stream(self.stream):
            self.mf.enqueue(self.stream)
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.mf.enqueue(self.stream)
        self.graph = g

    def _pack(self, buf: int, wave):
        """Group the wave's scenes by bucket and stack each group into pinned staging."""
        groups = {}
        for pos, (key, x) in enumerate(wave):
            groups.setdefault(self.index[key], []).append(pos)
        counts = [0] * len(self.keys)
        slots = [None] * len(wave)
        for j, poss in groups.items():
            if len(poss) > self.capacity:
                raise ValueError("bucket capacity exceeded")
            counts[j] = len(poss)
            np.stack([np.asarray(wave[p][1], dtype=np.float32).reshape(-1) for p in poss],
                     out=self.h_x[buf][j][:len(poss)].numpy())
            for b, p in enumerate(poss):
                slots[p] = (j, b)
        self.h_count[buf].copy_(torch.tensor(counts, dtype=torch.int32))
        return counts, slots

    def _launch(self, buf: int, counts) -> None:
        mf = self.mf
        with torch.cuda.stream(self.stream):
            mf.count.copy_(self.h_count[buf], non_blocking=True)
            for j, c in enumerate(counts):
                if c:
                    mf.x[j][:c].copy_(self.h_x[buf][j][:c], non_blocking=True)
                    self.copies["h2d_bytes"] += c * mf.x[j].shape[1] * 4
            if self.graph is not None:
                self.graph.replay()
            else:
                mf.enqueue(self.stream)
            for j, c in enumerate(counts):
                if c:
                    self.h_y[buf][j][:c].copy_(mf.y[j][:c], non_blocking=True)
                    self.copies["d2h_bytes"] += c * mf.y[j].shape[1] * 4
            self.done[buf].record(self.stream)

    def run_wave(self, wave):
        """wave: list of (bucket key, scene vector).  Returns images in wave order."""
        counts, slots = self._pack(0, wave)
        self._launch(0, counts)
        self.done[0].synchronize()
        return [self.h_y[0][j][b].clone() for j, b in slots]

    def run_waves(self, waves):
        """Serve waves back to back: wave i + 1 is packed on the host while the GPU
        works on wave i.  Yields (images in wave order, seconds from the start of
        the wave's packing to its images being back in host memory) per wave."""
        pending = None
        for i, wave in enumerate(waves):
            buf = i & 1
            t0 = time.perf_counter()
            counts, slots = self._pack(buf, wave)
            self._launch(buf, counts)
            if pending is not None:
                yield self._collect(*pending)
            pending = (buf, slots, t0)
        if pending is not None:
            yield self._collect(*pending)

    def _collect(self, buf, slots, t0):
        self.done[buf].synchronize()
        out = [self.h_y[buf][j][b].clone() for j, b in slots]
        return out, time.perf_counter() - t0
