"""Benchmark: simulated images/s through the psfsim C ABI on one GB300 per rank.

Workload (default): the 128 x 128 adjoint/fit configuration -- 40 synthetic
Lyot PSFs of 128^2 at 0.25 lambda/D, a 128^2 scene, A = 16384 x 16384 FP32
(1.07 GB, larger than L2, so no flush is needed between steps).  One step is
one gradient evaluation of the ring fit: ring scene Z(theta), the forward
image S = A Z (Eq. 6), the float64 loss and residual, the adjoint A^T r and
the chain rule into the 5 ring parameters -- two full passes over A.
value = images simulated per second (one per step).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
column sample of the same workload (the paper's method has no GPU reference).
Multi-GPU (torchrun) runs independent replicas: the path has no exchange step.
"""
from __future__ import annotations

import argparse
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


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the current kernels (profiles/*.md).  The tensor-core figure is
# from the 128^2 case and scales with the bytes of A (traffic / A = 1.0364 there).
NCU_TRAFFIC = {
    "forward": 1.073864e9 + 0.003710e9,        # fwd_ring_loss_kernel, 128^2
    "adjoint": 1.074243e9 + 0.003091e9,        # adj_chain_kernel (two columns per pass), 128^2
    "tc_gemm_per_A_byte": (1.086396e9 + 0.026477e9) / (16384 * 16384 * 4),
    "fused": 2.031170e9 + 0.127913e9,          # fused_kernel, 512^2, 32 scenes
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


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


def _workload():
    from synth import workloads
    w = workloads.adjoint_128()
    lib32 = w.library().astype(np.float32)
    x = workloads.random_ring_scene(w.N, w.S, w.r_max, w.seed + 5).ravel().astype(np.float32)
    rng = np.random.default_rng(w.seed + 6)
    g = rng.standard_normal(w.M).astype(np.float32)
    return w, lib32, x, g


def _fit_config(w, world):
    """The fit gradient workload, as both arms report it."""
    return {"workload": f"{w.name}: n=N=128, s=S=0.25 lambda/D, 40 radii 0-12 lambda/D, "
                        "A 16384x16384 FP32; step = one fit gradient: ring Z(theta), S = A Z with residual "
                        "and FP64 loss, A^T r with the chain to the 5 ring parameters (2 launches)",
            "M": w.M, "K": w.K, "n_radii": len(w.radii), "storage": "fp32",
            "l2": "inputs larger than L2 (A is 1.07 GB), no flush",
            "parallelism": f"replicas x{world}"}


def _oracle_target(w):
    """Synthetic target image for the oracle's fit step (seeded noise; its values do not change the cost)."""
    from synth import workloads
    return workloads.fit_target_noise(w, w.M)


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


def _gpu_arm(args, rank, world, local_rank):
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.fit import RingProblem
    from synth import workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w, lib32, x_np, g_np = _workload()
    stream = torch.cuda.current_stream()
    lib_d = torch.from_numpy(lib32).to(dev)

    # one-off library build (the paper's Table 2 step), timed on its own
    torch.cuda.synchronize()
    b0, b1 = _events(2)
    b0.record(stream)
    plan = Plan(lib_d, w.radii, w.s, N=w.N, S=w.S)
    b1.record(stream)
    torch.cuda.synchronize()
    build_ms = b0.elapsed_time(b1)

    # target image: noisy simulated truth (the fit workload's inputs)
    truth = np.array(w.extra["truth"])
    sigma = w.extra["sigma"]
    tmp = RingProblem(plan, w.N, w.S, w.r_max, torch.zeros(w.M, device=dev), sigma)
    d = plan.forward(tmp.scene(truth).clone()) + torch.from_numpy(
        workloads.fit_target_noise(w, w.M).astype(np.float32)).to(dev)
    prob = RingProblem(plan, w.N, w.S, w.r_max, d, sigma)
    theta = workloads.fit_init(w)

    for _ in range(args.warmup):
        prob.enqueue_gradient(theta)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    nsteps = args.steps
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0, t1 = _events(2)
    prob.launches = 0
    t0.record(stream)
    for i in range(nsteps):
        # one gradient evaluation: [ring -> forward (+ residual, loss)], [adjoint (+ chain, sums)];
        # back to back, so one step's adjoint tail overlaps the next step's forward
        prob.enqueue_forward_loss(theta)
        prob.enqueue_adjoint_chain(theta)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = prob.launches
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    elapsed_ms = _allreduce_max(elapsed_ms, dev)

    # each half on its own: an event pair around each C-ABI call (the events
    # also stop the overlap between kernels), for the per-kernel roofline
    nk = min(nsteps, 500)
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

    # e2e: a new observed image arrives from pinned host memory every step and
    # the loss + gradient come back to the host, through the same C-ABI calls
    hd = d.cpu().pin_memory()
    hout = torch.empty(6, dtype=torch.float64).pin_memory()
    dd = torch.empty_like(d)
    prob_e = RingProblem(plan, w.N, w.S, w.r_max, dd, sigma)

    def e2e_step():
        dd.copy_(hd, non_blocking=True)
        prob_e.enqueue_gradient(theta)
        hout.copy_(prob_e.out6, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = _events(2)
    e0.record(stream)
    for _ in range(nsteps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = _allreduce_max(e2e_ms, dev)
    e2e_out = hout.numpy().copy()

    # the same, with no staging copies: the forward kernel reads the target
    # straight from pinned (mapped) host memory and the adjoint writes the loss
    # and gradient straight into it, over the CPU-GPU link, so that nothing
    # stands between one gradient's kernels and the next
    hd_m = d.cpu().pin_memory()
    hout_m = torch.zeros(6, dtype=torch.float64).pin_memory()
    prob_m = RingProblem(plan, w.N, w.S, w.r_max, hd_m, sigma)
    prob_m.out6 = hout_m
    prob_m.loss_d, prob_m.dtheta = hout_m[:1], hout_m[1:]
    for _ in range(args.warmup):
        prob_m.enqueue_gradient(theta)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(nsteps):
        prob_m.enqueue_gradient(theta)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_mapped_ms = _allreduce_max(e0.elapsed_time(e1), dev)
    e2e_mapped_out = hout_m.numpy().copy()

    # plain FP32 GEMV comparator (cuBLAS through torch) on the same stored A
    x = torch.from_numpy(x_np).to(dev)
    g = torch.from_numpy(g_np).to(dev)
    A = plan.A_fp32()
    for _ in range(3):
        torch.mv(A, x)
        torch.mv(A.t(), g)
    torch.cuda.synchronize()
    c0, c1 = _events(2)
    c0.record(stream)
    for _ in range(nsteps):
        torch.mv(A, x)
        torch.mv(A.t(), g)
    c1.record(stream)
    torch.cuda.synchronize()
    cmp_ms = c0.elapsed_time(c1) / nsteps
    y_gpu = plan.forward(x)
    y_cublas = torch.mv(A, x)
    agree = float(((y_gpu - y_cublas).abs().max() / y_cublas.abs().max()).item())

    # the 200-step fit itself (host line search reads the float64 loss each trial)
    torch.cuda.synchronize()
    f0 = time.perf_counter()
    theta_fit, hist = prob.fit(theta, steps=w.extra["steps"])
    fit_s = time.perf_counter() - f0

    hbm, _, peak_kind = _peaks()
    a_bytes = w.M * w.K * 4
    fwd_bytes = a_bytes + 3 * w.M * 4 + 6 * w.K * 4   # A, target; y, r; Z and dZ/dtheta
    adj_bytes = a_bytes + w.M * 4 + 6 * w.K * 4       # A, r; gz, dZ/dtheta
    ms_per_step = elapsed_ms / nsteps
    images = world * nsteps
    dominant = "adjoint" if adj_ms > fwd_ms else "forward"
    dom_ms, dom_bytes = (adj_ms, adj_bytes) if dominant == "adjoint" else (fwd_ms, fwd_bytes)
    out = {
        "metric": METRIC,
        "value": images / (elapsed_ms / 1e3),
        "unit": "images/s",
        "n_gpus": world,
        "steps": nsteps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded Lyot-coronagraph PSFs, exozodi ring scene)",
        "config": _fit_config(w, world),
        "gmac_per_s": images * 2 * w.M * w.K / (elapsed_ms / 1e3) / 1e9,
        "kernels_ms": {"forward": fwd_ms, "adjoint": adj_ms, "build_once": build_ms},
        "roofline": {"bound": "hbm", "achieved": dom_bytes / (dom_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": dom_bytes / (dom_ms / 1e3) / 1e9 / hbm, "traffic": NCU_TRAFFIC[dominant] / 1e9,
                     "kernel": f"psfsim {dominant} half of the gradient (one kernel streaming A once; event "
                               "pair around psfsim_ring_forward_loss / psfsim_ring_adjoint_chain, timed alone)",
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "roofline_frac": {"forward": fwd_bytes / (fwd_ms / 1e3) / 1e9 / hbm,
                          "adjoint": adj_bytes / (adj_ms / 1e3) / 1e9 / hbm},
        "fp32_gemv_comparator": {"impl": "torch.mv (cuBLAS) forward + adjoint on the same A",
                                 "ms_per_step": cmp_ms, "images_per_s": 1e3 / cmp_ms,
                                 "psfsim_forward_adjoint_ms": fwd_ms + adj_ms,
                                 "max_rel_diff_vs_psfsim": agree},
        "fit": {"steps": int(len(hist) - 1), "seconds": fit_s, "loss_first": float(hist[0]),
                "loss_last": float(hist[-1]), "theta": [float(v) for v in theta_fit],
                "truth": [float(v) for v in truth]},
        "e2e": {"value": images / (e2e_mapped_ms / 1e3), "unit": "images/s",
                "h2d_bytes_per_step": w.M * 4, "d2h_bytes_per_step": 6 * 8,
                "result_equals_device_path": bool(np.array_equal(e2e_mapped_out, dev_out6)),
                "transfer": "every step the forward kernel reads the new target (64 KB) from pinned host memory "
                            "and the adjoint writes the loss and gradient (48 B) into pinned host memory, both "
                            "mapped into the GPU's address space (no staging copies)"},
        "e2e_staged": {"value": images / (e2e_ms / 1e3), "unit": "images/s",
                       "h2d_bytes_per_step": w.M * 4, "d2h_bytes_per_step": 6 * 8,
                       "result_equals_device_path": bool(np.array_equal(e2e_out, dev_out6)),
                       "transfer": "cudaMemcpyAsync of the target from pinned host memory into device memory "
                                   "before each gradient, of the loss and gradient back after it"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    return out, plan, y_gpu, x_np, w, lib32


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


def _path_batched(dev, stream, hbm, with_oracle):
    """Batched split-BF16 256^2 workload: 8 wavelengths x 64 scenes, each wavelength with its own
    A (8 x 17.2 GB resident), all products in one persistent multi-job tcgen05 launch."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from paper_2106_09122_gb300.serve import MultiForward
    from synth import workloads
    w = workloads.batched_256()
    nl, B = len(w.lam_ratios), w.extra["scenes"]
    libs = [w.library(l).astype(np.float32) for l in range(nl)]
    torch.cuda.synchronize()
    b0, b1 = _events(2)
    b0.record(stream)
    plans = [Plan(torch.from_numpy(lb).to(dev), w.radii, w.s, N=w.N, S=w.S, storage="split_bf16") for lb in libs]
    b1.record(stream)
    torch.cuda.synchronize()
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
    out = {"workload": "batched_split_bf16_256: 8 wavelengths (575 nm, 10% band) x 64 scenes; 60 PSFs 256^2 "
                       "at 0.125 lambda0/D per wavelength; 8 x A 65536^2 split-BF16 (137 GB) in one launch",
           "images_per_s": nl * B / (ms / 1e3), "ms_per_batch": ms, "build_ms_all_wavelengths": b0.elapsed_time(b1),
           "gmac_per_s": nl * B * w.M * w.K / (ms / 1e3) / 1e9,
           "roofline": {"bound": "hbm", "achieved": a_bytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": a_bytes / (ms / 1e3) / 1e9 / hbm, "kernel": "tc_gemm_kernel, 8 jobs (+ split, reduce)",
                        "traffic": NCU_TRAFFIC["tc_gemm_per_A_byte"] * nl * 4 * w.M * w.K / 1e9,
                        "traffic_note": "ncu on the 128^2 case, scaled by the bytes of A"},
           "status": plans[0].sync_status()}
    if with_oracle:
        per = []
        for l in range(nl):
            rows = np.sort(np.random.default_rng(81 + l).choice(w.M, 12, replace=False))
            Yr = mf.y[l][:4, torch.from_numpy(rows).to(dev)].cpu().numpy()
            e = _rows_error(libs[l], w.radii, w.N, w.S, X_np[l][:4], Yr, rows)
            per.append(e["max_bound_rel_error"])
        out["error_vs_oracle_per_wavelength"] = {"max_bound_rel_error": per, "rows_per_wavelength": 12,
                                                 "scenes_per_wavelength": 4}
    del plans, mf
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
    _, bf16_peak, _ = _peaks()
    out = {"workload": "batched_split_bf16_sym_256: the batched 256^2 workload (8 wavelengths x 64 scenes) on "
                       f"split-BF16 storage of the quadrant's columns inside 12 lambda/D ({kst} of {w.K} columns, "
                       f"8 x {4 * rows * ld / 1e9:.2f} GB)",
           "images_per_s": nl * B / (ms / 1e3), "ms_per_batch": ms,
           "roofline": {"bound": "tensor", "achieved": tc_flops / (ms / 1e3) / 1e12, "peak": bf16_peak,
                        "unit": "TFLOP/s", "frac": tc_flops / (ms / 1e3) / 1e12 / bf16_peak,
                        "kernel": "gather + tc_gemm_kernel (the 256 rotated scenes as 4 interleaved jobs against "
                                  "the compact A) + turned sum",
                        "flops_note": "bf16 MMA flops issued: 2 x rows x ld x (3 + 2) x padded scenes per job; "
                                      f"the compact A is {4 * rows * ld / 1e9:.2f} GB per wavelength and is "
                                      "served mostly from L2 after the first job reads it"},
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
    plans = [Plan(torch.from_numpy(lb).to(dev), w.radii, w.s, N=w.N, S=w.S, storage="bf16") for lb in libs]
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
           "images_per_s": nl * B / (ms / 1e3), "ms_per_batch": ms,
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


def _path_fused(dev, stream, with_oracle):
    """Fused 512^2 workload: A (275 GB in FP32) regenerated on chip for 32 scenes."""
    import torch
    from paper_2106_09122_gb300 import Plan
    from synth import workloads
    w = workloads.fused_512()
    lib32 = w.library().astype(np.float32)
    plan = Plan(torch.from_numpy(lib32).to(dev), w.radii, w.s, N=w.N, S=w.S, storage="fused")
    X_np = workloads.scene_batch(w, 32, kind="two_ring").astype(np.float32)
    X = torch.from_numpy(X_np).to(dev)
    Y = torch.empty((32, w.M), device=dev)
    scr = torch.empty(plan.forward_scratch_bytes(32), dtype=torch.uint8, device=dev)
    ms = _timed(lambda: plan.forward(X, out=Y, scratch=scr), 3, stream)
    props = torch.cuda.get_device_properties(dev)
    # A elements generated per batch: the x>0, y>0 quadrant of the scene, columns inside the last radius.
    c = (np.arange(w.N // 2) + 0.5) * w.S
    q0 = np.hypot(c[:, None], c[None, :]) <= w.radii[-1]
    elems = int(q0.sum()) * w.M
    inst_per_elem = 87.1  # ncu: thread instructions per generated element (profiles/fused_kernel_512.md)
    peak_inst = props.multi_processor_count * 4 * 32 * 2.07e9
    achieved_inst = elems * inst_per_elem / (ms / 1e3)
    out = {"workload": "fused_512: 80 PSFs 512^2 at 0.0625 lambda/D, A 262144^2 never stored, 32 two-ring scenes",
           "images_per_s": 32 / (ms / 1e3), "ms_per_batch": ms,
           "elements_generated_per_s": elems / (ms / 1e3),
           "dense_equivalent_gmac_per_s": 32 * w.M * w.K / (ms / 1e3) / 1e9,
           "roofline": {"bound": "alu", "achieved": achieved_inst / 1e12, "peak": peak_inst / 1e12,
                        "unit": "Tinst/s", "frac": achieved_inst / peak_inst,
                        "kernel": "fused_kernel (A-tile generation + tcgen05)",
                        "traffic": NCU_TRAFFIC["fused"] / 1e9, "traffic_unit": "GB",
                        "peak_source": "SMs x 4 SMSPs x 32 lanes x 2070 MHz issue rate"},
           "status": plan.sync_status()}
    if with_oracle:
        rows = np.sort(np.random.default_rng(82).choice(w.M, 12, replace=False))
        Yr = Y[:2, torch.from_numpy(rows).to(dev)].cpu().numpy()
        out["error_vs_oracle"] = _rows_error(lib32, w.radii, w.N, w.S, X_np[:2], Yr, rows)
    del plan, X, Y, scr
    torch.cuda.empty_cache()
    return out


def _path_uneven(dev, stream, hbm, with_oracle):
    """500 scenes of 10 (N, S) buckets, each with its own split-BF16 A; waves of 50 via one CUDA graph."""
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
    server.capture()
    scenes = [workloads.random_ring_scene(k[0], k[1], w.r_max, w.seed + 20000 + i).ravel().astype(np.float32)
              for i, k in enumerate(order)]
    server.run_wave([(k, scenes[i]) for i, k in enumerate(waves[0])])  # warm replay
    lat = []
    outs = []
    t0 = time.perf_counter()
    for wi, wv in enumerate(waves):
        a = time.perf_counter()
        outs += server.run_wave([(k, scenes[wi * W + i]) for i, k in enumerate(wv)])
        lat += [time.perf_counter() - a] * len(wv)
    total = time.perf_counter() - t0
    a_bytes = sum(p.M * p.info.ld * 4 for p in plans.values())
    out = {"workload": "uneven_500: 500 scenes, N in {64,96,128,192,256} x S in {0.3,0.5} lambda/D, per-bucket "
                       "split-BF16 A (17.3 GB), seeded arrival order, waves of 50 through one CUDA graph",
           "images_per_s": len(order) / total, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
           "p99_ms": 1e3 * float(np.percentile(lat, 99)), "tuning": {"chunk": best[0], "units_per_sm": best[1]},
           "multi_launch_ms": best_ms,
           "roofline": {"bound": "hbm", "achieved": a_bytes / (best_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": a_bytes / (best_ms / 1e3) / 1e9 / hbm,
                        "kernel": "tc_gemm_kernel, 10 jobs in one persistent launch"}}
    # plain per-scene FP32 GEMV loop (cuBLAS) on FP32 A per bucket
    fp = {k: Plan(lib, w.radii, w.s, N=k[0], S=k[1]) for k in buckets}
    xs_dev = [torch.from_numpy(sc).to(dev) for sc in scenes]
    torch.cuda.synchronize()
    clat = []
    c0 = time.perf_counter()
    for i, k in enumerate(order):
        a = time.perf_counter()
        torch.mv(fp[k].A_fp32(), xs_dev[i])
        torch.cuda.synchronize()
        clat.append(time.perf_counter() - a)
    out["fp32_gemv_loop"] = {"images_per_s": len(order) / (time.perf_counter() - c0),
                             "p50_ms": 1e3 * float(np.percentile(clat, 50)),
                             "p99_ms": 1e3 * float(np.percentile(clat, 99))}
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
            "roofline": {"bound": "hbm", "achieved": nbytes / (dom_ms / 1e3) / 1e9,
                         "peak": hbm, "unit": "GB/s", "frac": nbytes / (dom_ms / 1e3) / 1e9 / hbm,
                         "kernel": f"{dom} half of the symmetric gradient (event pair around its C-ABI call)",
                         "bytes_note": "bytes of the stored compact A, not of the dense A"},
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
        torch.cuda.synchronize()
        e0, e1 = _events(2)
        e0.record(stream)
        plan = Plan(lib, w.radii, w.s, N=w.N, S=w.S, interp=interp)
        e1.record(stream)
        torch.cuda.synchronize()
        y = torch.empty(w.M, device=dev)
        scr = torch.empty(plan.forward_scratch_bytes(1), dtype=torch.uint8, device=dev)
        ms = _timed(lambda: plan.forward(x, out=y, scratch=scr), 50, stream)
        a_bytes = 4 * w.M * w.K + 4 * w.K + 4 * w.M
        out[interp] = {"build_ms": e0.elapsed_time(e1), "simulate_ms": ms,
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


def _oracle_sample(w, lib32, n_cols=512, seed=17):
    """Column sample of the oracle's A (FP64) and the sampled column indices."""
    from oracle import psfsim_oracle as O
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.choice(w.K, n_cols, replace=False))
    xs, ys = O.scene_offsets(w.N, w.S)
    A_s = O.build_points(lib32.astype(np.float64), w.radii, xs[cols], ys[cols])
    return cols, A_s


def _oracle_step_time(w, A_s, cols, d_np, budget_s=10.0, max_steps=None):
    """Seconds per full-size fit gradient step of the FP64 oracle.

    Per step: the ring scene and its Jacobian on the full N x N grid, the
    forward over the column sample, the residual and loss over all M pixels,
    the adjoint over the column sample and the chain dZ/dtheta^T (A^T r) over
    the same columns.  The column-sampled parts are scaled by K / len(cols);
    the ring scene and the loss are timed at full size.
    """
    from oracle import psfsim_oracle as O
    from oracle import ring_oracle as RO
    from synth import workloads
    theta = workloads.fit_init(w)
    sigma = float(w.extra["sigma"])
    d = d_np.astype(np.float64)
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        Z, J = RO.ring_scene_and_jacobian(theta, w.N, w.S, w.r_max)
        t1 = time.perf_counter()
        y = O.forward(A_s, Z[cols])
        t2 = time.perf_counter()
        r = (y - d) / sigma
        loss = 0.5 * float(r @ r)
        t3 = time.perf_counter()
        gz = O.adjoint(A_s, r / sigma)
        dtheta = J[cols].T @ gz
        t4 = time.perf_counter()
        assert np.isfinite(loss) and np.all(np.isfinite(dtheta))
        times.append((t1 - t0) + (t3 - t2) + ((t2 - t1) + (t4 - t3)) * w.K / len(cols))
        if (max_steps and len(times) >= max_steps) or (not max_steps and time.perf_counter() - t_start > budget_s):
            break
    return float(np.median(times)), len(times)


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def _cpu_baseline_and_error(w, lib32, x_np, g_np, y_gpu):
    from oracle import psfsim_oracle as O
    cols, A_s = _oracle_sample(w, lib32)
    per, reps = _oracle_step_time(w, A_s, cols, _oracle_target(w))
    base = {"value": 1.0 / per, "unit": "images/s", "cores": _cores(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle fit gradient step: ring scene, Jacobian and loss at full size, "
                      f"forward, adjoint and chain on a {len(cols)}-column seeded sample of A "
                      f"({len(cols)}/{w.K} columns, median of {reps} reps), extrapolated per column"}
    rng = np.random.default_rng(29)
    rows = np.sort(rng.choice(w.M, 64, replace=False))
    xs, ys = O.scene_offsets(w.N, w.S)
    A_r = O.A_rows(lib32.astype(np.float64), w.radii, xs, ys, rows)
    x64 = x_np.astype(np.float64)
    rel = O.bound_relative_error(y_gpu[rows], A_r @ x64, np.abs(A_r) @ np.abs(x64), floor=O.FLT_MIN)
    err = {"max_bound_rel_error": float(rel.max()), "median": float(np.median(rel)),
           "rows_checked": int(len(rows)), "tolerance": 1e-5}
    return base, err


def _reference_arm(args):
    rank, world, _ = _dist()
    if rank != 0:
        return None
    w, lib32, x_np, g_np = _workload()
    cols, A_s = _oracle_sample(w, lib32)
    d_np = _oracle_target(w)
    _oracle_step_time(w, A_s, cols, d_np, max_steps=max(args.warmup, 1))
    t0 = time.perf_counter()
    per, reps = _oracle_step_time(w, A_s, cols, d_np, max_steps=args.steps)
    wall = time.perf_counter() - t0
    value = 1.0 / per
    sample = (f"FP64 NumPy oracle fit gradient step per step: ring scene, Jacobian and loss at full size, "
              f"forward, adjoint and chain on a {len(cols)}-column seeded sample of A, extrapolated to all "
              f"{w.K} columns ({wall:.1f} s wall for {reps} steps)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _fit_config(w, world),
            "cpu_baseline": {"value": value, "unit": "images/s", "cores": _cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


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
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="psfsim", choices=["psfsim", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--main-only", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--case", default=None,
                    help="run one small profiling case (fp32_128, fit128, sym128, sparse128, splitsym128, tc128, "
                         "bf16_128, fused512)")
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
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out, plan, y, x_np, w, lib32 = _gpu_arm(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, _, _, g_np = _workload()
        out["cpu_baseline"], out["error_vs_oracle"] = _cpu_baseline_and_error(
            w, lib32, x_np, g_np, y.double().cpu().numpy())
    if not args.main_only and world == 1:
        del plan, y
        torch.cuda.empty_cache()
        dev = torch.device("cuda", local_rank)
        stream = torch.cuda.current_stream()
        hbm, _, _ = _peaks()
        oracle_ok = rank == 0 and world == 1 and not args.no_cpu_baseline
        out["other_workloads"] = {
            "batched_split_bf16_256_8_wavelengths": _path_batched(dev, stream, hbm, oracle_ok),
            "batched_bf16_256_8_wavelengths": _path_bf16(dev, stream, hbm, oracle_ok),
            "batched_split_bf16_sym_256_8_wavelengths": _path_split_sym(dev, stream, hbm, oracle_ok),
            "convolution_comparator_128": _path_convolution(dev, stream),
            "skip_zero_pixels_128": _path_sparse(dev, stream, hbm),
            "fused_512": _path_fused(dev, stream, oracle_ok),
            "uneven_500": _path_uneven(dev, stream, hbm, oracle_ok),
            "nearest_vs_linear_128": _path_nearest(dev),
            "compact_symmetric_fit_128": _path_sym(dev, stream, hbm),
            "paper_ipac_shape": _path_ipac(dev, stream, hbm, oracle_ok),
        }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
