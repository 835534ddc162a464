"""Benchmark: simulated images/s through the psfsim C ABI on one GB300 per rank.

Headline workload: the fused 512^2 configuration -- 80 synthetic Lyot PSFs of
512^2 at 0.0625 lambda/D applied to a 512^2 scene grid, so A would be
262144 x 262144 (275 GB in FP32) and is never stored: every product
regenerates A tile by tile on chip (radial lerp + bilinear rotation) and feeds
the tiles to the tensor cores.  One step is S = A Z (Eq. 6) for a batch of 32
two-ring exozodi scenes through psfsim_forward; value = images/s.  The
library copy the kernels read (665 MB) and the partial images (268 MB) exceed
the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the paper's method has no GPU
reference) on the host cores: each step is one seeded row of the image for
all 32 scenes, every A element of the row built from its definition;
images/s is extrapolated to all 262144 rows.  Multi-GPU (torchrun) runs
independent replicas: the path has no exchange step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "simulated images/s and GMAC/s (fraction of HBM/tensor roofline) vs plain FP32 GEMV at stated error"
CSRC = os.path.join(ROOT, "paper_2106_09122_gb300", "csrc")

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of a kernel, valid only for the kernel source it was taken on
# (sha256 prefix of the .cu file): a changed kernel reports traffic null until
# it is captured again.
NCU_TRAFFIC = {
    "fused_kernel": {"file": "fused.cu", "sha": "cce2519e41c5fb90", "bytes": 1.043801e9 + 0.244421e9},
    "fwd_ring_loss_kernel": {"file": "fit_gradient.cu", "sha": "b12c1c3a52352d28", "bytes": 1.073864e9 + 0.003710e9},
    "adj_chain_kernel": {"file": "fit_gradient.cu", "sha": "b12c1c3a52352d28", "bytes": 1.074243e9 + 0.003091e9},
    "tc_gemm_kernel_per_A_byte": {"file": "tc_gemm.cu", "sha": "643a1c8518b1b882",
                                  "bytes": (1086370560 + 28214528) / (4 * 16384 * 16384)},
}


def _traffic(name: str):
    t = NCU_TRAFFIC[name]
    if t["sha"] is None:
        return None
    with open(os.path.join(CSRC, t["file"]), "rb") as f:
        return t["bytes"] if hashlib.sha256(f.read()).hexdigest()[:16] == t["sha"] else None


def _peaks():
    """Measured peaks (MEASURED_PEAKS.json) or the documented fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm": float(p["hbm_gbs"]), "bf16": float(p["bf16_tflops"]),
                "bf16_sustained": float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), "kind": "measured"}
    except Exception:
        return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "kind": "fallback"}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world, int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def _allreduce_max(value: float, device) -> float:
    """Max of a per-rank scalar over all ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _timed(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _timed_build(make, stream):
    """A plan built twice: the first build leaves its workspace in the allocator's cache, so the
    timed second build (geometry, column sort, the build kernels) allocates nothing."""
    import torch
    plan = make()
    torch.cuda.synchronize()
    plan.free()
    del plan
    e0, e1 = _events(2)
    e0.record(stream)
    plan = make()
    e1.record(stream)
    torch.cuda.synchronize()
    return plan, e0.elapsed_time(e1)


def _build_roofline(a_bytes, ms, hbm):
    return {"bound": "hbm", "achieved": a_bytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": a_bytes / (ms / 1e3) / 1e9 / hbm,
            "bytes_note": "A written once over the whole build (geometry, column sort and the build kernels)"}


def _rows_error(lib32, radii, N, S, X, Y, rows, cols=None):
    """Bound-relative error of Y[:, rows] against the oracle (test-infrastructure leg only)."""
    from oracle import psfsim_oracle as O
    xs, ys = O.scene_offsets(N, S)
    if cols is None:
        cols = np.arange(N * N)
    A_r = O.A_rows(lib32.astype(np.float64), radii, xs[cols], ys[cols], rows)
    X64 = X[:, cols].astype(np.float64)
    rel = O.bound_relative_error(Y.astype(np.float64), X64 @ A_r.T, np.abs(X64) @ np.abs(A_r).T, floor=O.FLT_MIN)
    return {"max_bound_rel_error": float(rel.max()), "median": float(np.median(rel)),
            "rows_checked": int(len(rows)), "scenes_checked": int(X.shape[0])}


# ---------------------------------------------------------------------------
# headline: fused 512^2, 32 scenes
# ---------------------------------------------------------------------------

FUSED_SCENES = 32


def _fused_workload():
    from synth import workloads
    w = workloads.fused_512()
    lib32 = w.library().astype(np.float32)
    X = workloads.scene_batch(w, FUSED_SCENES, kind="two_ring").astype(np.float32)
    return w, lib32, X


def _fused_config(w, world):
    return {"workload": "fused_512: 80 Lyot PSFs 512^2 at 0.0625 lambda/D, 512^2 scene grid, A 262144^2 "
                        "regenerated on chip every product (never stored), batch of 32 two-ring scenes; step = "
                        "psfsim_forward of the batch (gather, fused tcgen05 kernel, reduction)",
            "M": w.M, "K": w.K, "n_radii": len(w.radii), "scenes_per_step": FUSED_SCENES, "storage": "fused",
            "l2": "inputs larger than L2 (library pair entries 665 MB, partial images 268 MB), no flush",
            "parallelism": f"replicas x{world}"}


def _fused_mma_flops(plan, scenes):
    """bf16 MMA flops one fused launch issues: per 128-row m-tile and 64-column k-tile of
    the quadrant's columns, three products (hi x1, hi x2, lo x1) of N = 4 Bp (Bp = 16, 32 or
    64 scenes per launch)."""
    Bp = 16 if scenes <= 16 else (32 if scenes <= 32 else 64)
    rows = (plan.M + 127) // 128 * 128
    ldx = (plan.info.K_stored + 63) // 64 * 64
    return 2.0 * rows * ldx * 4 * Bp * 3


def _oracle_rows_fused(w, lib32, X, rows):
    """FP64 oracle rows of the fused workload's images (every A element of a row from
    its definition, all K columns) and the seconds each row took."""
    from oracle import psfsim_oracle as O
    xs, ys = O.scene_offsets(w.N, w.S)
    X64 = X.astype(np.float64)
    ref, bound, secs = [], [], []
    for r in rows:
        t0 = time.perf_counter()
        a = O.A_rows(lib32.astype(np.float64), w.radii, xs, ys, np.array([r]))[0]
        ref.append(X64 @ a)
        secs.append(time.perf_counter() - t0)
        bound.append(np.abs(X64) @ np.abs(a))
    return np.array(ref).T, np.array(bound).T, np.array(secs)


def _headline(args, rank, world, local_rank):
    import torch
    from paper_2106_09122_gb300 import Plan

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    w, lib32, X_np = _fused_workload()
    lib = torch.from_numpy(lib32).to(dev)
    torch.cuda.synchronize()
    b0, b1 = _events(2)
    b0.record(stream)
    plan = Plan(lib, w.radii, w.s, N=w.N, S=w.S, storage="fused")
    b1.record(stream)
    torch.cuda.synchronize()
    build_ms = b0.elapsed_time(b1)
    X = torch.from_numpy(X_np).to(dev)
    Y = torch.empty((FUSED_SCENES, w.M), device=dev)
    scr = torch.empty(plan.forward_scratch_bytes(FUSED_SCENES), dtype=torch.uint8, device=dev)

    def step():
        plan.forward(X, out=Y, scratch=scr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0, t1 = _events(2)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = _allreduce_max(t0.elapsed_time(t1), dev)
    if world > 1:
        torch.distributed.barrier()

    # per-call duration of the fused launch sequence on the launching stream (the
    # x gather and the reduction of the partial images take about 1% of it)
    nk = max(3, min(args.steps, 10))
    ev = [_events(2) for _ in range(nk)]
    for i in range(nk):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    call_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    status = plan.sync_status()

    # e2e: every step's 32 scenes come from pinned host memory and its 32 images go
    # back to it, around the same C-ABI call.  Two device buffer sets and one copy
    # stream per direction let step i + 1's scenes arrive and step i - 1's images
    # leave while step i runs, as a caller streaming batches would.
    Y_dev = Y.clone()
    hX = torch.from_numpy(X_np).pin_memory()
    hY = [torch.empty((FUSED_SCENES, w.M), dtype=torch.float32).pin_memory() for _ in range(2)]
    Xd, Yd = [X, torch.empty_like(X)], [Y, torch.empty_like(Y)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_run(n):
        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        s_in.wait_event(start)
        fwd_done, out_done = [None, None], [None, None]
        for i in range(n):
            j = i & 1
            if fwd_done[j] is not None:  # step i - 2 has read Xd[j]
                s_in.wait_event(fwd_done[j])
            with torch.cuda.stream(s_in):
                Xd[j].copy_(hX, non_blocking=True)
            arrived = torch.cuda.Event()
            arrived.record(s_in)
            stream.wait_event(arrived)
            if out_done[j] is not None:  # step i - 2's images have left Yd[j]
                stream.wait_event(out_done[j])
            plan.forward(Xd[j], out=Yd[j], scratch=scr, stream=stream)
            fwd_done[j] = torch.cuda.Event()
            fwd_done[j].record(stream)
            s_out.wait_event(fwd_done[j])
            with torch.cuda.stream(s_out):
                hY[j].copy_(Yd[j], non_blocking=True)
            out_done[j] = torch.cuda.Event()
            out_done[j].record(s_out)
        stream.wait_event(out_done[(n - 1) & 1])
        end = torch.cuda.Event(enable_timing=True)
        end.record(stream)
        return start, end

    if args.warmup:
        e2e_run(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = e2e_run(args.steps)
    torch.cuda.synchronize()
    e2e_ms = _allreduce_max(e0.elapsed_time(e1), dev)
    last = (args.steps - 1) & 1
    e2e_equal = bool(torch.equal(hY[last], Y_dev.cpu()))

    peaks = _peaks()
    images = world * args.steps * FUSED_SCENES
    flops = _fused_mma_flops(plan, FUSED_SCENES)
    elems = plan.info.K_stored * w.M
    achieved = flops / (call_ms / 1e3) / 1e12
    ms_per_step = elapsed_ms / args.steps
    out = {
        "metric": METRIC,
        "value": images / (elapsed_ms / 1e3),
        "unit": "images/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16 (split hi+lo x split x, fp32 accumulate)",
        "data": "synthetic (seeded Lyot-coronagraph PSFs, two-ring exozodi scenes)",
        "config": _fused_config(w, world),
        "gmac_per_s": images * w.M * w.K / (elapsed_ms / 1e3) / 1e9,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_sustained"], "unit": "TFLOP/s",
                     "frac": achieved / peaks["bf16_sustained"], "traffic": _traffic("fused_kernel"),
                     "kernel": "fused_kernel (A tiles regenerated on chip + tcgen05); event pair around each "
                               "psfsim_forward call",
                     "flops_per_launch": flops,
                     "flops_note": "bf16 MMA flops the design issues: 2 x rows x 64-padded quadrant columns "
                                   "inside the last radius x 4 rotations x 32 scenes x 3 products (hi x1, hi x2, "
                                   "lo x1)",
                     "peak_source": f"{peaks['kind']} bf16_tflops_sustained"},
        "generation": {"elements_per_launch": elems, "elements_per_s": elems / (call_ms / 1e3),
                       "note": "A elements generated per launch: the quadrant's columns inside the last radius "
                               "x all image pixels (a quarter of the dense A's columns carry the rest exactly)"},
        "kernels_ms": {"fused_forward_call": call_ms, "build_once": build_ms},
        "e2e": {"value": images / (e2e_ms / 1e3), "unit": "images/s",
                "h2d_bytes_per_step": int(hX.numel() * 4), "d2h_bytes_per_step": int(hY[0].numel() * 4),
                "result_equals_device_path": e2e_equal,
                "transfer": "every step: cudaMemcpyAsync of its 32 scenes from pinned host memory and of its 32 "
                            "images back to pinned host memory, on one copy stream per direction, overlapping "
                            "the neighbouring steps' psfsim_forward calls (two device buffer sets)"},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "status": status,
    }
    return out, plan, Y, X, X_np, w, lib32


def _fused_crop_comparator(dev, stream, w, lib32, fused_plan, X_np, with_oracle):
    """Plain FP32 comparator for the fused workload: the scenes' central 256^2 crop (K =
    65536 columns) with its FP32 A stored (262144 x 65536, 68.7 GB) and multiplied by
    torch.mm (cuBLAS, TF32 off), against the fused path on the same cropped scenes; both
    checked against the oracle on seeded rows (crop columns only)."""
    import torch
    from paper_2106_09122_gb300 import Plan
    lo, hi = w.N // 4, 3 * w.N // 4
    iy, ix = np.divmod(np.arange(w.K), w.N)
    cols = np.nonzero((iy >= lo) & (iy < hi) & (ix >= lo) & (ix < hi))[0]
    Xc = np.zeros_like(X_np)
    Xc[:, cols] = X_np[:, cols]
    # the crop's field points (lambda/D): pixel centres (i - (N - 1) / 2) S of the scene grid
    c = (w.N - 1) / 2.0
    pts = np.stack([(ix[cols] - c) * w.S, (iy[cols] - c) * w.S], axis=1)
    fp = Plan(torch.from_numpy(lib32).to(dev), w.radii, w.s, points=pts, storage="fp32")
    A = fp.A_fp32()                                      # [M, 65536] view, column-major
    Xcrop = torch.from_numpy(np.ascontiguousarray(X_np[:, cols])).to(dev)
    allow = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        mm_ms = _timed(lambda: torch.mm(A, Xcrop.t()), 5, stream)
        Ymm = torch.mm(A, Xcrop.t()).t().contiguous()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = allow
    Xf = torch.from_numpy(Xc).to(dev)
    Yf = torch.empty((Xf.shape[0], w.M), device=dev)
    scr = torch.empty(fused_plan.forward_scratch_bytes(Xf.shape[0]), dtype=torch.uint8, device=dev)
    f_ms = _timed(lambda: fused_plan.forward(Xf, out=Yf, scratch=scr), 3, stream)
    out = {"workload": "fused_512 scenes cropped to their central 256^2 (65536 columns), 32 scenes",
           "fp32_torch_mm_ms": mm_ms, "fp32_A_bytes": int(4 * w.M * len(cols)),
           "fused_ms": f_ms, "speedup_fused_vs_fp32": mm_ms / f_ms,
           "note": "the stored FP32 A covers only the crop's columns (the full A would be 275 GB); the fused "
                   "call regenerates the whole quadrant whatever the scene, so this compares a quarter of the "
                   "method's columns on the GEMM side with all of them on the fused side"}
    if with_oracle:
        rows = np.sort(np.random.default_rng(86).choice(w.M, 16, replace=False))
        rsel = torch.from_numpy(rows).to(dev)
        e_mm = _rows_error(lib32, w.radii, w.N, w.S, X_np[:4], Ymm[:4, rsel].cpu().numpy(), rows, cols)
        e_f = _rows_error(lib32, w.radii, w.N, w.S, X_np[:4], Yf[:4, rsel].cpu().numpy(), rows, cols)
        out["error_vs_oracle"] = {"fp32_torch_mm": e_mm["max_bound_rel_error"], "fused": e_f["max_bound_rel_error"],
                                  "rows_checked": len(rows), "scenes_checked": 4}
    del fp, A, Xcrop, Ymm, Xf, Yf, scr
    torch.cuda.empty_cache()
    return out


def _fused_64_scenes(dev, stream, w, lib32, plan, peaks, with_oracle):
    """The fused 512^2 workload with 64 scenes per launch (the kernel's 64-scene form: MMA
    N = 256, one accumulator), beside the 32-scene headline: the same generation carries twice
    the tensor work."""
    import torch
    from synth import workloads
    B = 64
    X_np = workloads.scene_batch(w, B, kind="two_ring").astype(np.float32)
    X = torch.from_numpy(X_np).to(dev)
    Y = torch.empty((B, w.M), device=dev)
    scr = torch.empty(plan.forward_scratch_bytes(B), dtype=torch.uint8, device=dev)
    ms = _timed(lambda: plan.forward(X, out=Y, scratch=scr), 5, stream)
    flops = _fused_mma_flops(plan, B)
    out = {"workload": "fused_512 with 64 two-ring scenes per psfsim_forward call (one launch)",
           "images_per_s": B / (ms / 1e3), "ms_per_call": ms,
           "roofline": {"bound": "tensor", "achieved": flops / (ms / 1e3) / 1e12, "peak": peaks["bf16_sustained"],
                        "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / peaks["bf16_sustained"],
                        "flops_per_launch": flops},
           "status": plan.sync_status()}
    if with_oracle:
        from oracle import psfsim_oracle as O
        rows = np.sort(np.random.default_rng(64).choice(w.M, 8, replace=False))
        ref, bound, _ = _oracle_rows_fused(w, lib32, X_np, rows)
        Yr = Y[:, torch.from_numpy(rows).to(dev)].double().cpu().numpy()
        rel = O.bound_relative_error(Yr, ref, bound, floor=O.FLT_MIN)
        out["error_vs_oracle"] = {"max_bound_rel_error": float(rel.max()), "rows_checked": len(rows),
                                  "scenes_checked": B}
    del X, Y, scr
    return out


def _cpu_baseline_fused(w, lib32, X_np, Y_gpu, n_rows=64):
    """FP64 oracle on seeded rows of the headline images: time per row (extrapolated to all
    rows) and the bound-relative error of the GPU rows."""
    from oracle import psfsim_oracle as O
    rows = np.sort(np.random.default_rng(29).choice(w.M, n_rows, replace=False))
    ref, bound, secs = _oracle_rows_fused(w, lib32, X_np, rows)
    per_row = float(np.median(secs))
    base = {"value": FUSED_SCENES / (per_row * w.M), "unit": "images/s", "cores": _cores(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle: {n_rows} seeded rows of the 512^2 image for all 32 scenes, every A "
                      f"element of a row (all {w.K} columns) built from its definition; median {per_row:.3f} s "
                      f"per row, extrapolated to {w.M} rows ({float(np.sum(secs)):.1f} s of CPU work)"}
    rel = O.bound_relative_error(Y_gpu[:, rows].astype(np.float64), ref, bound, floor=O.FLT_MIN)
    err = {"max_bound_rel_error": float(rel.max()), "median": float(np.median(rel)), "rows_checked": int(n_rows),
           "scenes_checked": int(X_np.shape[0]), "tolerance": 2.5e-5}
    return base, err


def _reference_arm(args):
    """FP64 oracle arm: each step is one seeded image row for all 32 scenes."""
    rank, world, _ = _dist()
    if rank != 0:
        return None
    w, lib32, X_np = _fused_workload()
    rows = np.random.default_rng(31).choice(w.M, args.warmup + args.steps, replace=False)
    _oracle_rows_fused(w, lib32, X_np, rows[:max(args.warmup, 1)])
    t0 = time.perf_counter()
    _, _, secs = _oracle_rows_fused(w, lib32, X_np, rows[args.warmup:args.warmup + args.steps])
    wall = time.perf_counter() - t0
    per_row = float(np.mean(secs))
    value = FUSED_SCENES / (per_row * w.M)
    sample = (f"FP64 NumPy oracle, one seeded row of the 512^2 image per step for all 32 scenes (every A element "
              f"of the row from its definition), extrapolated to {w.M} rows ({wall:.1f} s wall for {len(secs)} "
              f"steps)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_row * w.M / FUSED_SCENES * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _fused_config(w, world),
            "cpu_baseline": {"value": value, "unit": "images/s", "cores": _cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------
# named entries: the other workloads (N = 1 only)
# ---------------------------------------------------------------------------

def _entry_fit128(dev, stream, with_oracle, steps=1000):
    """Adjoint/fit 128^2: one fit gradient per step (ring Z(theta), S = A Z with residual and
    FP64 loss, A^T r with the chain to the 5 ring parameters; two launches), A 16384^2 FP32."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.fit import RingProblem
    from synth import workloads
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    lib_d = torch.from_numpy(lib32).to(dev)
    plan, build_ms = _timed_build(lambda: Plan(lib_d, w.radii, w.s, N=w.N, S=w.S), stream)
    truth = np.array(w.extra["truth"])
    sigma = w.extra["sigma"]
    tmp = RingProblem(plan, w.N, w.S, w.r_max, torch.zeros(w.M, device=dev), sigma)
    d = plan.forward(tmp.scene(truth).clone()) + torch.from_numpy(
        workloads.fit_target_noise(w, w.M).astype(np.float32)).to(dev)
    prob = RingProblem(plan, w.N, w.S, w.r_max, d, sigma)
    theta = workloads.fit_init(w)

    def grad_steps(n):
        for _ in range(n):
            prob.enqueue_forward_loss(theta)
            prob.enqueue_adjoint_chain(theta)

    step_ms = _timed(lambda: grad_steps(steps), 1, stream) / steps
    nk = 300
    ev = [_events(4) for _ in range(nk)]
    for i in range(nk):
        ev[i][0].record(stream)
        prob.enqueue_forward_loss(theta)
        ev[i][1].record(stream)
        ev[i][2].record(stream)
        prob.enqueue_adjoint_chain(theta)
        ev[i][3].record(stream)
    torch.cuda.synchronize()
    fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    adj_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in ev]))
    dev_out6 = prob.out6.cpu().numpy().copy()
    # e2e: the target is read from, and the loss + gradient written to, pinned host
    # memory mapped into the GPU's address space, every step
    hd_m = d.cpu().pin_memory()
    hout_m = torch.zeros(6, dtype=torch.float64).pin_memory()
    prob_m = RingProblem(plan, w.N, w.S, w.r_max, hd_m, sigma)
    prob_m.out6 = hout_m
    prob_m.loss_d, prob_m.dtheta = hout_m[:1], hout_m[1:]
    e2e_ms = _timed(lambda: [prob_m.enqueue_gradient(theta) for _ in range(steps)], 1, stream) / steps
    # plain FP32 GEMV comparator (cuBLAS through torch) on the same stored A
    x = tmp.scene(theta).clone()
    g = torch.rand(w.M, device=dev)
    A = plan.A_fp32()
    cmp_ms = _timed(lambda: (torch.mv(A, x), torch.mv(A.t(), g)), 200, stream)
    hbm = _peaks()["hbm"]
    a_bytes = w.M * w.K * 4
    fwd_bytes = a_bytes + 3 * w.M * 4 + 6 * w.K * 4
    adj_bytes = a_bytes + w.M * 4 + 6 * w.K * 4
    f0 = time.perf_counter()
    theta_fit, hist = prob.fit(theta, steps=w.extra["steps"])
    fit_s = time.perf_counter() - f0
    out = {"workload": "adjoint_fit_128: 40 PSFs 128^2 at 0.25 lambda/D, A 16384^2 FP32 (1.07 GB); step = one fit "
                       "gradient in two launches",
           "images_per_s": 1e3 / step_ms, "ms_per_step": step_ms,
           "gmac_per_s": 2 * w.M * w.K / (step_ms / 1e3) / 1e9,
           "kernels_ms": {"forward_loss": fwd_ms, "adjoint_chain": adj_ms},
           "build_ms": build_ms, "build_roofline": _build_roofline(4 * w.M * w.K, build_ms, _peaks()["hbm"]),
           "roofline": {"bound": "hbm", "achieved": adj_bytes / (adj_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": adj_bytes / (adj_ms / 1e3) / 1e9 / hbm, "traffic": _traffic("adj_chain_kernel"),
                        "kernel": "adj_chain_kernel (event pair around psfsim_ring_adjoint_chain, timed alone)"},
           "roofline_frac": {"forward": fwd_bytes / (fwd_ms / 1e3) / 1e9 / hbm,
                             "adjoint": adj_bytes / (adj_ms / 1e3) / 1e9 / hbm},
           "e2e": {"images_per_s": 1e3 / e2e_ms, "h2d_bytes_per_step": w.M * 4, "d2h_bytes_per_step": 48,
                   "result_equals_device_path": bool(np.array_equal(hout_m.numpy(), dev_out6)),
                   "transfer": "target read from and result written to mapped pinned host memory"},
           "fp32_gemv_comparator": {"impl": "torch.mv forward + adjoint on the same A", "ms_per_step": cmp_ms,
                                    "images_per_s": 1e3 / cmp_ms, "speedup": cmp_ms / step_ms},
           "fit": {"steps": int(len(hist) - 1), "seconds": fit_s, "loss_first": float(hist[0]),
                   "loss_last": float(hist[-1]), "theta": [float(v) for v in theta_fit],
                   "truth": [float(v) for v in truth]}}
    if with_oracle:
        from oracle import psfsim_oracle as O
        rows = np.sort(np.random.default_rng(29).choice(w.M, 32, replace=False))
        y = plan.forward(x).cpu().numpy()
        out["error_vs_oracle"] = _rows_error(lib32, w.radii, w.N, w.S, x.cpu().numpy()[None, :], y[rows][None, :],
                                             rows)
        yc = torch.mv(A, x).cpu().numpy()
        out["fp32_gemv_comparator"]["error_vs_oracle"] = _rows_error(
            lib32, w.radii, w.N, w.S, x.cpu().numpy()[None, :], yc[rows][None, :], rows)["max_bound_rel_error"]
    plan.free()
    del plan, A, prob, prob_m, tmp
    torch.cuda.empty_cache()
    return out


def _path_batched(dev, stream, hbm, with_oracle):
    """Batched split-BF16 256^2 workload: 8 wavelengths x 64 scenes, each wavelength with its own
    A (8 x 17.2 GB resident), all products in one persistent multi-job tcgen05 launch; plus the
    plain FP32 comparator on one wavelength (FP32 A, 17.2 GB, torch.mm with TF32 off)."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.serve import MultiForward
    from synth import workloads
    w = workloads.batched_256()
    nl, B = len(w.lam_ratios), w.extra["scenes"]
    libs = [w.library(l).astype(np.float32) for l in range(nl)]

    def make(lb):
        return Plan(torch.from_numpy(lb).to(dev), w.radii, w.s, N=w.N, S=w.S, storage="split_bf16")

    p0, build_ms = _timed_build(lambda: make(libs[0]), stream)
    plans = [p0] + [make(lb) for lb in libs[1:]]
    mf = MultiForward(plans, [B] * nl)
    X_np = []
    for l in range(nl):
        xs = np.empty((B, w.K), dtype=np.float32)
        for b in range(B):
            xs[b] = workloads.random_ring_scene(w.N, w.S, w.r_max, w.seed + 100000 * (l + 1) + b).ravel()
        X_np.append(xs)
        mf.x[l].copy_(torch.from_numpy(xs))
    mf.count.fill_(B)
    ms = _timed(mf.enqueue, 10, stream)
    a_bytes = nl * (4 * w.M * w.K + B * w.K * 4 + B * w.M * 4)
    tr = _traffic("tc_gemm_kernel_per_A_byte")
    out = {"workload": "batched_split_bf16_256: 8 wavelengths x 64 scenes, 60 PSFs 256^2 per wavelength, "
                       "8 x A 65536^2 split-BF16 (137 GB) in one launch",
           "images_per_s": nl * B / (ms / 1e3), "ms_per_batch": ms, "build_ms_per_wavelength": build_ms,
           "build_roofline": _build_roofline(4 * w.M * w.K, build_ms, hbm),
           "gmac_per_s": nl * B * w.M * w.K / (ms / 1e3) / 1e9,
           "roofline": {"bound": "hbm", "achieved": a_bytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": a_bytes / (ms / 1e3) / 1e9 / hbm, "kernel": "tc_gemm_kernel, 8 jobs (+ split, reduce)",
                        "traffic": None if tr is None else tr * nl * 4 * w.M * w.K},
           "status": plans[0].sync_status()}
    Y0 = mf.y[0][:4].clone()
    per = []
    if with_oracle:
        for l in range(nl):
            rows = np.sort(np.random.default_rng(81 + l).choice(w.M, 12, replace=False))
            Yr = mf.y[l][:4, torch.from_numpy(rows).to(dev)].cpu().numpy()
            per.append(_rows_error(libs[l], w.radii, w.N, w.S, X_np[l][:4], Yr, rows)["max_bound_rel_error"])
        out["error_vs_oracle_per_wavelength"] = {"max_bound_rel_error": per, "rows_per_wavelength": 12,
                                                 "scenes_per_wavelength": 4}
    del plans, mf
    torch.cuda.empty_cache()
    # plain FP32 comparator: wavelength 0's A stored in FP32 (17.2 GB), 64 scenes by torch.mm
    fp = Plan(torch.from_numpy(libs[0]).to(dev), w.radii, w.s, N=w.N, S=w.S)
    A = fp.A_fp32()
    X0 = torch.from_numpy(X_np[0]).to(dev)
    allow = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        mm_ms = _timed(lambda: torch.mm(A, X0.t()), 5, stream)
        Ymm = torch.mm(A, X0.t()).t().contiguous()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = allow
    cmpd = {"impl": "torch.mm (cuBLAS, TF32 off) on wavelength 0's FP32 A (17.2 GB), 64 scenes",
            "ms_per_wavelength": mm_ms, "split_bf16_ms_per_wavelength": ms / nl,
            "speedup": mm_ms / (ms / nl)}
    if with_oracle:
        rows = np.sort(np.random.default_rng(81).choice(w.M, 12, replace=False))
        Yr = Ymm[:4, torch.from_numpy(rows).to(dev)].cpu().numpy()
        cmpd["error_vs_oracle"] = {"fp32_torch_mm": _rows_error(libs[0], w.radii, w.N, w.S, X_np[0][:4], Yr,
                                                                rows)["max_bound_rel_error"],
                                   "split_bf16": per[0]}
    out["fp32_gemm_comparator"] = cmpd
    fp.free()
    del fp, A, X0, Ymm
    torch.cuda.empty_cache()
    return out


def _path_uneven(dev, stream, hbm, with_oracle):
    """500 scenes of 10 (N, S) buckets, each with its own split-BF16 A; waves of 50, one
    persistent multi-job launch each (captured graph), copies of exactly the scenes present."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.serve import UnevenServer, autotune
    from synth import workloads
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    lib = torch.from_numpy(lib32).to(dev)
    buckets = workloads.uneven_buckets()
    plans = {k: Plan(lib, w.radii, w.s, N=k[0], S=k[1], storage="split_bf16") for k in buckets}
    W = 50
    order, waves, cap = workloads.uneven_arrivals(500, W, w.seed + 9)
    server = UnevenServer(plans, capacity=cap)
    mf = server.mf
    for j, k in enumerate(server.keys):
        mf.x[j].copy_(torch.rand(cap, k[0] * k[0], device=dev) * 1e-9)
    mf.count.fill_(cap)
    best, best_ms, _ = autotune(mf, chunks=(2, 4, 8), units=(2, 4, 8), reps=3)
    server.set_tuning(best)
    server.capture()
    scenes = [workloads.random_ring_scene(k[0], k[1], w.r_max, w.seed + 20000 + i).ravel().astype(np.float32)
              for i, k in enumerate(order)]
    wave_items = [[(k, scenes[wi * W + i]) for i, k in enumerate(wv)] for wi, wv in enumerate(waves)]
    for _ in server.run_waves(wave_items[:2]):   # warm
        pass
    # latency: one wave at a time (pack, copies, launch, images back in host memory)
    lat, lat_views = [], []
    for wv in wave_items:
        a = time.perf_counter()
        server.run_wave(wv)
        lat.append(time.perf_counter() - a)
        a = time.perf_counter()
        server.run_wave(wv, copy=False)
        lat_views.append(time.perf_counter() - a)
    # throughput: waves back to back, the next one packed while the GPU works
    server.copies = {"h2d_bytes": 0, "d2h_bytes": 0}
    outs = []
    t0 = time.perf_counter()
    for imgs, _ in server.run_waves(wave_items):
        outs += imgs
    total = time.perf_counter() - t0
    a_bytes = sum(p.M * p.info.ld * 4 for p in plans.values())
    wave_s = total / len(waves)
    out = {"workload": "uneven_500: 500 scenes, N in {64,96,128,192,256} x S in {0.3,0.5} lambda/D, per-bucket "
                       "split-BF16 A (17.3 GB), seeded arrival order, waves of 50; the kernels read the scenes from "
                       "and write the images to mapped pinned host memory",
           "images_per_s": len(order) / total, "p50_wave_ms": 1e3 * float(np.percentile(lat, 50)),
           "p99_wave_ms": 1e3 * float(np.percentile(lat, 99)),
           "p50_wave_ms_views": 1e3 * float(np.percentile(lat_views, 50)),
           "latency_note": "p50/p99: one wave at a time, from the scenes in the caller's arrays to copies of the "
                           "images in host memory (p50_wave_ms_views: the images left in the pinned staging the "
                           "kernels wrote); images_per_s: the 10 waves back to back, each packed while the GPU "
                           "runs the previous",
           "tuning": {"chunk": best[0], "units_per_sm": best[1]}, "multi_launch_ms": best_ms,
           "copies_per_wave_bytes": {"h2d": server.copies["h2d_bytes"] / len(waves),
                                     "d2h": server.copies["d2h_bytes"] / len(waves)},
           "roofline": {"bound": "hbm", "achieved": a_bytes / wave_s / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": a_bytes / wave_s / 1e9 / hbm,
                        "kernel": "served waves: packing, copies and the multi-job launch, back to back; A bytes "
                                  "of all buckets per wave over the wave time"}}
    fp = {k: Plan(lib, w.radii, w.s, N=k[0], S=k[1]) for k in buckets}
    xs_dev = [torch.from_numpy(sc).to(dev) for sc in scenes]
    torch.cuda.synchronize()
    c0 = time.perf_counter()
    for i, k in enumerate(order):
        torch.mv(fp[k].A_fp32(), xs_dev[i])
    torch.cuda.synchronize()
    out["fp32_gemv_loop"] = {"images_per_s": len(order) / (time.perf_counter() - c0)}
    if with_oracle:
        errs = []
        pick = np.random.default_rng(83).choice(len(order), 6, replace=False)
        for i in pick:
            k = order[i]
            rows = np.sort(np.random.default_rng(int(i)).choice(w.M, 8, replace=False))
            e = _rows_error(lib32, w.radii, k[0], k[1], scenes[i][None, :], outs[i].numpy()[rows][None, :], rows)
            errs.append(e["max_bound_rel_error"])
        out["error_vs_oracle"] = {"max_bound_rel_error": float(max(errs)), "scenes_checked": len(pick),
                                  "rows_per_scene": 8}
    del plans, fp, server, xs_dev, lib
    torch.cuda.empty_cache()
    return out


def _path_split_sym(dev, stream, hbm, with_oracle):
    """The batched 256^2 workload (8 wavelengths x 64 scenes) on split-BF16 storage compacted by
    the quarter-turn symmetry and the zero columns; one forward per wavelength (the four rotations
    of the 64 scenes as 256 scenes of the tcgen05 product).  Bytes are those of the compact A."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from synth import workloads
    w = workloads.batched_256()
    nl, B = len(w.lam_ratios), w.extra["scenes"]
    libs = [w.library(l).astype(np.float32) for l in range(nl)]
    plans = [Plan(torch.from_numpy(lb).to(dev), w.radii, w.s, N=w.N, S=w.S, storage="split_bf16_sym") for lb in libs]
    X_np, X, Y = [], [], []
    for l in range(nl):
        xs = np.empty((B, w.K), dtype=np.float32)
        for b in range(B):
            xs[b] = workloads.random_ring_scene(w.N, w.S, w.r_max, w.seed + 100000 * (l + 1) + b).ravel()
        X_np.append(xs)
        X.append(torch.from_numpy(xs).to(dev))
        Y.append(torch.empty((B, w.M), device=dev))
    scr = torch.empty(plans[0].forward_scratch_bytes(B), dtype=torch.uint8, device=dev)

    def run():
        for l in range(nl):
            plans[l].forward(X[l], out=Y[l], scratch=scr)

    ms = _timed(run, 10, stream)
    kst = plans[0].info.K_stored
    ld = plans[0].info.ld
    rows = (w.M + 127) // 128 * 128
    # the 4B = 256 rotated scenes run as interleaved jobs of at most 80 (padded to 16) against
    # one A: per job, MMAs of N = 3 Bp (hi) and 2 Bp (lo) over every (row, column) of A
    jobs = [min(80, 4 * B - b0) for b0 in range(0, 4 * B, 80)]
    bps = [-(-c // 16) * 16 for c in jobs]
    tc_flops = nl * 2.0 * rows * ld * sum(5 * bp for bp in bps)
    # the method's own work on this storage: every stored column against the 4B rotated scenes
    method_flops = nl * 2.0 * w.M * kst * 4 * B
    bf16_peak = _peaks()["bf16"]
    out = {"workload": "batched_split_bf16_sym_256: the batched 256^2 workload (8 wavelengths x 64 scenes) on "
                       f"split-BF16 storage of the quadrant's columns inside 12 lambda/D ({kst} of {w.K} columns, "
                       f"8 x {4 * rows * ld / 1e9:.2f} GB)",
           "images_per_s": nl * B / (ms / 1e3), "ms_per_batch": ms,
           "method_gmac_per_s": method_flops / 2 / (ms / 1e3) / 1e9,
           "roofline": {"bound": "tensor", "achieved": method_flops / (ms / 1e3) / 1e12, "peak": bf16_peak,
                        "unit": "TFLOP/s", "frac": method_flops / (ms / 1e3) / 1e12 / bf16_peak,
                        "kernel": "gather + tc_gemm_kernel (the 256 rotated scenes as 4 interleaved jobs against "
                                  "the compact A) + turned sum",
                        "numerator": "the method's MACs x 2: rows x stored columns x 4 rotations x scenes",
                        "issued_tflops": tc_flops / (ms / 1e3) / 1e12,
                        "issued_frac": tc_flops / (ms / 1e3) / 1e12 / bf16_peak,
                        "issued_note": "the tensor pipe issues 5 bf16 products per MAC for the 2^-17 split "
                                       "precision (hi x 3 parts of x, lo x 2) on scene counts padded to 16, so "
                                       "it is busy at issued_frac while the method's own work is frac; A "
                                       f"({4 * rows * ld / 1e9:.2f} GB per wavelength) is read from HBM once per "
                                       "wavelength and served from L2 to the other jobs"},
           "status": plans[0].sync_status()}
    if with_oracle:
        per = []
        for l in range(nl):
            rows_c = np.sort(np.random.default_rng(97 + l).choice(w.M, 12, replace=False))
            Yr = Y[l][:4, torch.from_numpy(rows_c).to(dev)].cpu().numpy()
            per.append(_rows_error(libs[l], w.radii, w.N, w.S, X_np[l][:4], Yr, rows_c)["max_bound_rel_error"])
        out["error_vs_oracle_per_wavelength"] = {"max_bound_rel_error": per, "rows_per_wavelength": 12,
                                                 "scenes_per_wavelength": 4}
    del plans, X, Y
    torch.cuda.empty_cache()
    return out


def _path_bf16(dev, stream, hbm, with_oracle):
    """The batched 256^2 workload with plain BF16 storage (hi alone: 8 x 8.6 GB), one multi-job
    tcgen05 launch: half the bytes of split-BF16 at 2^-8 instead of 2^-17 storage error."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.serve import MultiForward
    from synth import workloads
    w = workloads.batched_256()
    nl, B = len(w.lam_ratios), w.extra["scenes"]
    libs = [w.library(l).astype(np.float32) for l in range(nl)]

    def make(lb):
        return Plan(torch.from_numpy(lb).to(dev), w.radii, w.s, N=w.N, S=w.S, storage="bf16")

    p0, build_ms = _timed_build(lambda: make(libs[0]), stream)
    plans = [p0] + [make(lb) for lb in libs[1:]]
    mf = MultiForward(plans, [B] * nl)
    X_np = []
    for l in range(nl):
        xs = np.empty((B, w.K), dtype=np.float32)
        for b in range(B):
            xs[b] = workloads.random_ring_scene(w.N, w.S, w.r_max, w.seed + 100000 * (l + 1) + b).ravel()
        X_np.append(xs)
        mf.x[l].copy_(torch.from_numpy(xs))
    mf.count.fill_(B)
    ms = _timed(mf.enqueue, 10, stream)
    a_bytes = nl * (2 * w.M * w.K + B * w.K * 4 + B * w.M * 4)
    out = {"workload": "batched_bf16_256: the batched 256^2 workload (8 wavelengths x 64 scenes) with BF16 "
                       "storage, 8 x A 65536^2 (69 GB) in one launch",
           "images_per_s": nl * B / (ms / 1e3), "ms_per_batch": ms, "build_ms_per_wavelength": build_ms,
           "build_roofline": _build_roofline(2 * w.M * w.K, build_ms, hbm),
           "gmac_per_s": nl * B * w.M * w.K / (ms / 1e3) / 1e9,
           "roofline": {"bound": "hbm", "achieved": a_bytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": a_bytes / (ms / 1e3) / 1e9 / hbm,
                        "kernel": "tc_gemm_kernel, 8 jobs, one MMA (N = 2 x 64) per k-step (+ split, reduce)",
                        "intensity_note": "2 x 128 flop per 2-byte element = 128 flop/byte < bf16 ridge ~278"},
           "tolerance": 2.0 ** -8 + 2.5e-5,
           "status": plans[0].sync_status()}
    if with_oracle:
        per = []
        for l in range(nl):
            rows = np.sort(np.random.default_rng(91 + l).choice(w.M, 12, replace=False))
            Yr = mf.y[l][:4, torch.from_numpy(rows).to(dev)].cpu().numpy()
            per.append(_rows_error(libs[l], w.radii, w.N, w.S, X_np[l][:4], Yr, rows)["max_bound_rel_error"])
        out["error_vs_oracle_per_wavelength"] = {"max_bound_rel_error": per, "rows_per_wavelength": 12,
                                                 "scenes_per_wavelength": 4}
    del plans, mf
    torch.cuda.empty_cache()
    return out


def _path_convolution(dev, stream):
    """Sec. 3's comparison: the fit workload's exozodi ring simulated by the method and by
    convolution with the method's own PSF at 6 lambda/D (+x axis), masked to its core
    (radius 3 lambda/D) and re-centred; differences inside the working angles 3-9 lambda/D,
    for the scene as is and with its core (r < 3 lambda/D) masked."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.convolution import convolution_image
    from synth import workloads
    w = workloads.adjoint_128()
    plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S)
    xs = (np.arange(w.N) - (w.N - 1) / 2) * w.S
    ix_ref, iy_ref = int(np.argmin(np.abs(xs - 6.0))), int(np.argmin(np.abs(xs - 0.0)))
    one = torch.zeros(w.K, device=dev)
    one[iy_ref * w.N + ix_ref] = 1.0
    col = plan.forward(one).view(w.n, w.n)
    X, Y = np.meshgrid(xs, xs)
    r = np.hypot(X, Y)
    work = torch.from_numpy((r >= 3.0) & (r <= 9.0)).to(dev)
    out = {"workload": "adjoint_fit_128 ring scene (R = 5, i = 60 deg, g = 0.3): method vs convolution with the "
                       "method's PSF at (6, 0) lambda/D masked to 3 lambda/D, inside 3-9 lambda/D",
           "reference_offset_lambda_over_D": float(xs[ix_ref])}
    from synth import scenes
    base = scenes.ring_image(w.N, w.S, 5.0, 1.0, np.deg2rad(60.0), 0.3, 1e-9, w.r_max).astype(np.float32)
    for name, sc in (("scene", base), ("core_masked_scene", np.where(r < 3.0, 0.0, base).astype(np.float32))):
        x = torch.from_numpy(sc).to(dev)
        y_m = plan.forward(x.view(-1)).view(w.n, w.n)
        y_c = convolution_image(x, col, iy_ref, ix_ref, mask_radius_px=3.0 / w.s)
        peak = y_m[work].abs().max()
        d = ((y_c - y_m).abs() / peak)[work] * 100.0
        out[name] = {"max_pct_difference": float(d.max()), "mean_pct_difference": float(d.mean())}
    xsc = torch.from_numpy(base).to(dev)
    out["ms"] = {"method_forward": _timed(lambda: plan.forward(xsc.view(-1)), 50, stream),
                 "cufft_convolution": _timed(lambda: convolution_image(xsc, col, iy_ref, ix_ref, 3.0 / w.s), 50,
                                             stream)}
    plan.free()
    return out


def _path_sparse(dev, stream, hbm):
    """Skipping zero scene pixels (FP32 storage, 128^2 fit workload's A): the ring scene, which is
    zero beyond the 12 lambda/D outer working angle, and ten point sources; each against the dense
    forward.  Bytes are those of the columns actually read, never the dense A."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from synth import scenes, workloads
    w = workloads.adjoint_128()
    plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S)
    ring = scenes.ring_image(w.N, w.S, 5.0, 1.0, np.deg2rad(60.0), 0.3, 1e-9, w.r_max).astype(np.float32).ravel()
    pts = np.zeros(w.K, dtype=np.float32)
    rng = np.random.default_rng(93)
    pts[rng.choice(np.nonzero(ring)[0], 10, replace=False)] = 1e-8
    out = {"workload": "adjoint_fit_128 A (FP32, 1.07 GB): forward of one scene reading only the columns of "
                       "non-zero scene pixels"}
    for name, sc in (("ring_scene", ring), ("ten_point_sources", pts)):
        x = torch.from_numpy(sc).to(dev)
        y = torch.empty(w.M, device=dev)
        nnz = int(np.count_nonzero(sc))
        ms_s = _timed(lambda: plan.forward(x, out=y, skip_zeros=True), 50, stream)
        ms_d = _timed(lambda: plan.forward(x, out=y), 50, stream)
        ys = plan.forward(x, skip_zeros=True)
        yd = plan.forward(x)
        nbytes = nnz * w.M * 4 + w.K * 4 + w.M * 4
        out[name] = {"nonzero_pixels": nnz, "images_per_s": 1e3 / ms_s, "ms": ms_s, "dense_ms": ms_d,
                     "speedup_vs_dense": ms_d / ms_s,
                     "max_rel_diff_vs_dense": float(((ys - yd).abs().max() / yd.abs().max()).item()),
                     "roofline": {"bound": "hbm", "achieved": nbytes / (ms_s / 1e3) / 1e9, "peak": hbm,
                                  "unit": "GB/s", "frac": nbytes / (ms_s / 1e3) / 1e9 / hbm,
                                  "bytes_note": "columns of the non-zero pixels only"}}
    plan.free()
    return out


def _path_sym(dev, stream, hbm):
    """The fit gradient step on FP32 storage compacted by the quarter-turn symmetry and zero columns."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.fit import RingProblem
    from synth import workloads
    w = workloads.adjoint_128()
    lib = torch.from_numpy(w.library().astype(np.float32)).to(dev)
    dense = Plan(lib, w.radii, w.s, N=w.N, S=w.S)
    sym = Plan(lib, w.radii, w.s, N=w.N, S=w.S, storage="fp32_sym")
    truth = np.array(w.extra["truth"])
    sigma = w.extra["sigma"]
    tmp = RingProblem(dense, w.N, w.S, w.r_max, torch.zeros(w.M, device=dev), sigma)
    d = dense.forward(tmp.scene(truth).clone()) + torch.from_numpy(
        workloads.fit_target_noise(w, w.M).astype(np.float32)).to(dev)
    theta = workloads.fit_init(w)
    pd = RingProblem(dense, w.N, w.S, w.r_max, d, sigma)
    ps = RingProblem(sym, w.N, w.S, w.r_max, d, sigma)
    ld_, gd_ = pd.loss_and_grad(theta)
    ls_, gs_ = ps.loss_and_grad(theta)
    steps = 2000
    ms = _timed(lambda: [ps.enqueue_gradient(theta) for _ in range(steps)], 1, stream) / steps
    nk = 500
    ev = [_events(4) for _ in range(nk)]
    for i in range(nk):
        ev[i][0].record(stream)
        ps.enqueue_forward_loss(theta)
        ev[i][1].record(stream)
        ev[i][2].record(stream)
        ps.enqueue_adjoint_chain(theta)
        ev[i][3].record(stream)
    torch.cuda.synchronize()
    fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    adj_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in ev]))
    # A_Q0 (0.12 GB) fits in L2, so back-to-back steps can find some of it there; also time
    # single steps with L2 flushed before each (a 512 MB buffer rewritten between steps).
    flush = torch.empty(512 * 2**20 // 4, dtype=torch.float32, device=dev)
    nf = 200
    evf = [_events(2) for _ in range(nf)]
    for i in range(nf):
        flush.add_(1.0)
        evf[i][0].record(stream)
        ps.enqueue_gradient(theta)
        evf[i][1].record(stream)
    torch.cuda.synchronize()
    flushed_ms = float(np.median([e[0].elapsed_time(e[1]) for e in evf]))
    del flush
    kst = sym.info.K_stored
    stored = 4 * sym.info.ld * kst
    dom = "adjoint" if adj_ms > fwd_ms else "forward"
    dom_ms = max(adj_ms, fwd_ms)
    nbytes = stored + 24 * w.K + 8 * w.M   # compact A; scene, Jacobian; image, residual
    return {"workload": "adjoint_fit_128 gradient step on FP32_SYM storage: only the x>0, y>0 quadrant's columns "
                        f"inside 12 lambda/D are stored ({kst} of {w.K} columns, {stored / 1e9:.3f} GB); "
                        "three launches per gradient",
            "images_per_s": 1e3 / ms, "ms_per_step": ms,
            "l2": "back to back (A_Q0 is smaller than L2); flushed_l2 below rewrites 512 MB before each step",
            "flushed_l2": {"images_per_s": 1e3 / flushed_ms, "ms_per_step_median": flushed_ms},
            "kernels_ms": {"forward_half": fwd_ms, "adjoint_half": adj_ms},
            "roofline": {"bound": "hbm", "achieved": 2 * nbytes / (flushed_ms / 1e3) / 1e9,
                         "peak": hbm, "unit": "GB/s", "frac": 2 * nbytes / (flushed_ms / 1e3) / 1e9 / hbm,
                         "kernel": "the whole three-launch gradient step with L2 flushed before it",
                         "bytes_note": "the step's own bytes: both passes over the stored compact A (not the dense "
                                       "A) plus scene, Jacobian, image and residual",
                         "limit_note": f"HBM alone would take {2 * nbytes / hbm / 1e6 * 1e3:.1f} us; the rest of "
                                       "the step is the three launches' fixed costs and their reduction tails "
                                       f"(slowest half alone: {dom} at {dom_ms * 1e3:.1f} us)"},
            "agreement_with_dense": {"loss_rel": abs(ls_ - ld_) / abs(ld_),
                                     "grad_max_rel": float(np.max(np.abs(gs_ - gd_) / np.abs(gd_)))}}


def _path_ipac(dev, stream, hbm, with_oracle):
    """The paper's IPAC shape (128^2 PSFs at 0.2 lambda/D, 86 non-uniform offsets, 256^2 scene at
    3.529 mas): build and simulate timed like Tables 2 and 4 (linear and nearest)."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from synth import workloads
    w = workloads.ipac_shape()
    lib32 = w.library().astype(np.float32)
    lib = torch.from_numpy(lib32).to(dev)
    x_np = workloads.powerlaw_disk_scene(w.N, w.S, w.r_max).ravel().astype(np.float32)
    x = torch.from_numpy(x_np).to(dev)
    out = {"workload": "paper IPAC shape: 86 PSFs 128^2 at 0.2 lambda/D (offsets every 0.06 to 4, 0.5 to 9, "
                       "0.25 to 11 lambda/D), 256^2 power-law disk scene at 3.529 mas, A 16384 x 65536 FP32 (4.3 GB)",
           "paper_context": {"build_linear_s": 506.680, "build_nearest_s": 334.246, "simulate_s": 0.1642,
                             "hardware": "8-core 2.3 GHz CPU node, FP64 (Tables 1, 2, 4)"}}
    for interp in ("linear", "nearest"):
        plan, build_ms = _timed_build(lambda: Plan(lib, w.radii, w.s, N=w.N, S=w.S, interp=interp), stream)
        y = torch.empty(w.M, device=dev)
        scr = torch.empty(plan.forward_scratch_bytes(1), dtype=torch.uint8, device=dev)
        ms = _timed(lambda: plan.forward(x, out=y, scratch=scr), 50, stream)
        a_bytes = 4 * w.M * w.K + 4 * w.K + 4 * w.M
        out[interp] = {"build_ms": build_ms, "build_roofline": _build_roofline(4 * w.M * w.K, build_ms, hbm),
                       "simulate_ms": ms,
                       "speedup_vs_paper_simulate": 164.2 / ms,
                       "roofline": {"bound": "hbm", "achieved": a_bytes / (ms / 1e3) / 1e9, "peak": hbm,
                                    "unit": "GB/s", "frac": a_bytes / (ms / 1e3) / 1e9 / hbm}}
        if interp == "linear":
            y_lin = y.clone()
            if with_oracle:
                rows = np.sort(np.random.default_rng(85).choice(w.M, 16, replace=False))
                out["error_vs_oracle"] = _rows_error(lib32, w.radii, w.N, w.S, x_np[None, :],
                                                     y[torch.from_numpy(rows).to(dev)].cpu().numpy()[None, :], rows)
        else:
            c = (np.arange(w.n) - (w.n - 1) / 2) * w.s
            inside = torch.from_numpy((np.hypot(c[:, None], c[None, :]) <= 9.0).ravel()).to(dev)
            pct = (100 * (y_lin - y).abs() / y_lin.abs().clamp_min(1e-30))[inside & (y_lin.abs() > 0)]
            out["linear_vs_nearest_pct_within_9_lambda_over_D"] = {"max": float(pct.max()), "mean": float(pct.mean()),
                                                                   "paper_IPAC": {"max": 0.468, "mean": 0.114}}
        del plan, scr
        torch.cuda.empty_cache()
    return out


def _path_nearest(dev):
    """Linear vs nearest radial interpolation (Sec. 4.2): % difference of the images within 9 lambda/D."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from synth import workloads
    w = workloads.adjoint_128()
    lib = torch.from_numpy(w.library().astype(np.float32)).to(dev)
    x = torch.from_numpy(workloads.random_ring_scene(w.N, w.S, w.r_max, w.seed + 5).ravel()
                         .astype(np.float32)).to(dev)
    yl = Plan(lib, w.radii, w.s, N=w.N, S=w.S).forward(x)
    yn = Plan(lib, w.radii, w.s, N=w.N, S=w.S, interp="nearest").forward(x)
    c = (np.arange(w.n) - (w.n - 1) / 2) * w.s
    inside = torch.from_numpy((np.hypot(c[:, None], c[None, :]) <= 9.0).ravel()).to(dev)
    pct = (100 * (yl - yn).abs() / yl.abs().clamp_min(1e-30))[inside & (yl.abs() > 0)]
    return {"workload": "adjoint_fit_128 scene, linear vs nearest radial interpolation",
            "max_pct_difference_within_9_lambda_over_D": float(pct.max()),
            "mean_pct_difference_within_9_lambda_over_D": float(pct.mean())}


def _profile_case(name: str) -> None:
    """A few launches of one workload, small enough for a full ncu capture."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from synth import workloads
    dev = "cuda:0"
    if name == "fused512":
        w = workloads.fused_512()
        plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S,
                    storage="fused")
        X = torch.from_numpy(workloads.scene_batch(w, 32, kind="two_ring").astype(np.float32)).to(dev)
        for _ in range(2):
            plan.forward(X)
    elif name == "splitsym128":
        w = workloads.adjoint_128()
        plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S,
                    storage="split_bf16_sym")
        X = torch.rand(64, w.K, device=dev)
        for _ in range(3):
            plan.forward(X)
    elif name in ("tc128", "bf16_128"):
        w = workloads.adjoint_128()
        plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S,
                    storage="split_bf16" if name == "tc128" else "bf16")
        X = torch.rand(64, w.K, device=dev)
        for _ in range(3):
            plan.forward(X)
        g = torch.rand(1, w.M, device=dev)
        for _ in range(3):
            plan.adjoint(g)
    elif name == "fp32_128":
        w = workloads.adjoint_128()
        plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S)
        x = torch.rand(w.K, device=dev)
        g = torch.rand(w.M, device=dev)
        for _ in range(3):
            plan.forward(x)
            plan.adjoint(g)
    elif name == "sparse128":
        from synth import scenes
        w = workloads.adjoint_128()
        plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S)
        ring = scenes.ring_image(w.N, w.S, 5.0, 1.0, np.deg2rad(60.0), 0.3, 1e-9, w.r_max).astype(np.float32)
        x = torch.from_numpy(ring.ravel()).to(dev)
        for _ in range(3):
            plan.forward(x, skip_zeros=True)
    elif name == "builds":
        # each build of A twice: the even grid (quadrant generated, four turned copies) and the
        # same grid given as field points (the direct, column-by-column build)
        for wname, storage in (("adjoint_128", "fp32"), ("ipac_shape", "fp32"), ("batched_256", "split_bf16")):
            w = getattr(workloads, wname)()
            lib = torch.from_numpy((w.library(0) if wname == "batched_256" else w.library()).astype(np.float32)).to(dev)
            iy, ix = np.divmod(np.arange(w.N * w.N), w.N)
            pts = np.stack([(ix - (w.N - 1) / 2) * w.S, (iy - (w.N - 1) / 2) * w.S], axis=1)
            for grid in (True, False):
                plan = None
                torch.cuda.empty_cache()
                plan = (Plan(lib, w.radii, w.s, N=w.N, S=w.S, storage=storage) if grid
                        else Plan(lib, w.radii, w.s, points=pts, storage=storage))
                torch.cuda.synchronize()
                if plan.sync_status() != 0:
                    raise SystemExit(f"build {wname} status {plan.sync_status()}")
    elif name == "sym128":
        from paper_2106_09122_gb300.fit import RingProblem
        w = workloads.adjoint_128()
        plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S,
                    storage="fp32_sym")
        prob = RingProblem(plan, w.N, w.S, w.r_max, torch.rand(w.M, device=dev) * 1e-10, w.extra["sigma"])
        for _ in range(3):
            prob.enqueue_gradient(workloads.fit_init(w))
    elif name == "fit128":
        from paper_2106_09122_gb300.fit import RingProblem
        w = workloads.adjoint_128()
        plan = Plan(torch.from_numpy(w.library().astype(np.float32)).to(dev), w.radii, w.s, N=w.N, S=w.S)
        prob = RingProblem(plan, w.N, w.S, w.r_max, torch.rand(w.M, device=dev) * 1e-10, w.extra["sigma"])
        for _ in range(3):
            prob.enqueue_gradient(workloads.fit_init(w))
    else:
        raise SystemExit(f"unknown case {name}")
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "status": plan.sync_status()}))




def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="psfsim", choices=["psfsim", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--main-only", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--case", default=None,
                    help="run one small profiling case (fp32_128, fit128, sym128, sparse128, splitsym128, tc128, "
                         "bf16_128, fused512, builds)")
    args = ap.parse_args()
    if args.case:
        _profile_case(args.case)
        return
    rank, world, local_rank = _dist()
    if args.impl == "reference":
        out = _reference_arm(args)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out, plan, Y, X, X_np, w, lib32 = _headline(args, rank, world, local_rank)
    with_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    if with_oracle:
        out["cpu_baseline"], out["error_vs_oracle"] = _cpu_baseline_fused(w, lib32, X_np, Y.cpu().numpy())
    if not args.main_only and world == 1:
        dev = torch.device("cuda", local_rank)
        stream = torch.cuda.current_stream()
        out["fp32_gemm_comparator"] = _fused_crop_comparator(dev, stream, w, lib32, plan, X_np, with_oracle)
        fused64 = _fused_64_scenes(dev, stream, w, lib32, plan, _peaks(), with_oracle)
        del plan, Y, X
        torch.cuda.empty_cache()
        hbm = _peaks()["hbm"]
        out["other_workloads"] = {
            "fused_512_64_scenes": fused64,
            "adjoint_fit_128": _entry_fit128(dev, stream, with_oracle),
            "batched_split_bf16_256_8_wavelengths": _path_batched(dev, stream, hbm, with_oracle),
            "batched_bf16_256_8_wavelengths": _path_bf16(dev, stream, hbm, with_oracle),
            "batched_split_bf16_sym_256_8_wavelengths": _path_split_sym(dev, stream, hbm, with_oracle),
            "uneven_500": _path_uneven(dev, stream, hbm, with_oracle),
            "convolution_comparator_128": _path_convolution(dev, stream),
            "skip_zero_pixels_128": _path_sparse(dev, stream, hbm),
            "nearest_vs_linear_128": _path_nearest(dev),
            "compact_symmetric_fit_128": _path_sym(dev, stream, hbm),
            "paper_ipac_shape": _path_ipac(dev, stream, hbm, with_oracle),
        }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
