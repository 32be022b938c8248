"""Benchmark of the compositing core: ms per forward+backward render of the 1M-Gaussian unbounded
scene at 1920x1080 (one training step of the hot path), through the C-ABI, on synthetic inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. `--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the oracle is test infrastructure; it is the reference arm here because the paper ships no
code). N > 1 (torchrun) runs independent replicas, one view per rank: the path has no exchange step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms per fwd+bwd render (1M Gaussians, 1080p)"
WORKLOAD = "unbounded 1M Gaussians SH3, one 1920x1080 view inside the foreground sphere, fwd+bwd"

# Per-unit FP32 work of the composite forward (counted from the kernel source):
#   per (pixel, record) test: 2 FADD (offsets) + 3 FFMA (cross) + 1 FMUL + 1 FFMA (|cross|^2)
#     + 5 FFMA (A) + 1 FMUL (threshold) = 13 FP32 instructions = 22 flops (FFMA = 2)
#   per hit: rcp + ex2 (2 MUFU) + 6 FP32 (m, alpha, od, t) = 11 flops
#   per composited hit: 1 FSUB + 2 FMUL (T, w) + 7 FFMA (colour, normal, depth) = 17 flops
FLOPS_PER_TEST = 22
FLOPS_PER_HIT = 11
FLOPS_PER_COMPOSITE = 17


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def make_workload(seed_offset=0):
    from paper_2506_19139_gb300 import synthetic as syn
    scene, cams = syn.unbounded_training(seed=2 + seed_offset)
    return scene, cams


def run_reference(args):
    """FP64 CPU oracle on a bounded pixel sample per step, extrapolated to the full frame (forward
    only: the oracle has no backward, so this under-counts the reference's work)."""
    import oracle
    ws, rank = _dist()
    if rank != 0:
        return
    scene, cams = make_workload()
    cam = cams[0]
    rng = np.random.default_rng(0)
    npx = cam.width * cam.height
    sample = int(os.environ.get("SOF_REF_PIXELS", "96"))
    times = []
    for step in range(args.warmup + args.steps):
        pix = rng.choice(npx, size=sample, replace=False).astype(np.int64)
        t0 = time.perf_counter()
        oracle.render(scene, cam, pixels=pix)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    per_frame_ms = statistics.mean(times) / sample * npx * 1e3
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": per_frame_ms, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_frame_ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_gaussians": scene.n, "width": cam.width, "height": cam.height},
        "cpu_baseline": {"value": per_frame_ms, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} random pixels per step of the 1920x1080 frame, forward only, "
                                   f"extrapolated to the full frame"},
        "e2e": {"value": per_frame_ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(scene, cam, seconds_target=12.0):
    import oracle
    rng = np.random.default_rng(1)
    npx = cam.width * cam.height
    pix = rng.choice(npx, size=16, replace=False).astype(np.int64)
    t0 = time.perf_counter()
    oracle.render(scene, cam, pixels=pix)
    dt = time.perf_counter() - t0
    n = int(max(16, min(4096, 16 * seconds_target / max(dt, 1e-3))))
    pix = rng.choice(npx, size=n, replace=False).astype(np.int64)
    t0 = time.perf_counter()
    oracle.render(scene, cam, pixels=pix)
    dt = time.perf_counter() - t0
    return {"value": dt / n * npx * 1e3, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} random pixels of the 1920x1080 frame (forward only), {dt:.1f} s, extrapolated "
                      f"to ms per full-frame forward"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2506_19139_gb300 import _lib as L
    from paper_2506_19139_gb300 import build as B
    from paper_2506_19139_gb300 import render as R

    world, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    scene, cams = make_workload(seed_offset=rank)
    cam = cams[0]
    ts = R.scene_tensors(scene, dev)
    opts = R.RenderOptions(chunk=args.chunk, reorder_k=args.reorder_k)
    ws = R.Workspace(dev)
    scene_c = R.scene_to_c(*ts)
    cams_c = R.cameras_to_c(cams)
    opts_c = opts.to_c()
    outs = R.alloc_outputs(cams, dev)
    grads = [torch.zeros_like(t) for t in ts]
    npx = cam.width * cam.height
    g = torch.Generator(device=dev).manual_seed(5)
    gin_t = {"color": torch.randn(3 * npx, device=dev, generator=g) / npx,
             "depth": torch.randn(npx, device=dev, generator=g) / npx,
             "exact": torch.randn(npx, device=dev, generator=g) / npx,
             "normal": torch.randn(3 * npx, device=dev, generator=g) / npx,
             "opacity": torch.randn(npx, device=dev, generator=g) / npx}
    gin = L.sof_render_grad_in()
    gin.d_color, gin.d_depth = gin_t["color"].data_ptr(), gin_t["depth"].data_ptr()
    gin.d_exact_depth, gin.d_normal = gin_t["exact"].data_ptr(), gin_t["normal"].data_ptr()
    gin.d_opacity, gin.d_median_depth = gin_t["opacity"].data_ptr(), 0
    sg = L.sof_scene_grad()
    sg.d_means, sg.d_log_scales, sg.d_quats = grads[0].data_ptr(), grads[1].data_ptr(), grads[2].data_ptr()
    sg.d_opacity_logits, sg.d_sh = grads[3].data_ptr(), grads[4].data_ptr()
    stream = torch.cuda.current_stream(dev)

    def step():
        R.render_forward_raw(scene_c, cams_c, 1, opts_c, outs, ws)
        L.check(L.sof_render_bwd(scene_c, cams_c, 1, opts_c, R._out_c(outs), gin, sg, ws.handle,
                                 stream.cuda_stream), "sof_render_bwd", ws.handle)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    stats = ws.stats()

    # per-kernel timing of the dominant kernels, on the launching stream, in separate passes
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    def timed_phases():
        ev[0].record(stream)
        R.render_forward_raw(scene_c, cams_c, 1, opts_c, outs, ws)
        ev[1].record(stream)
        L.check(L.sof_render_bwd(scene_c, cams_c, 1, opts_c, R._out_c(outs), gin, sg, ws.handle,
                                 stream.cuda_stream), "sof_render_bwd", ws.handle)
        ev[2].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

    fwd_ms, bwd_ms = [], []
    for _ in range(3):
        a, b = timed_phases()
        fwd_ms.append(a)
        bwd_ms.append(b)

    # timed region: exactly K steps, barrier + synchronize on both sides
    launches0 = L.sof_kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = (L.sof_kernel_launches() - launches0) // max(args.steps, 1)
    total_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps

    # end to end: host (pinned) inputs -> device, fwd+bwd through the C-ABI, result back to host
    host_in = [t.detach().cpu().pin_memory() for t in ts]
    dev_in = [torch.empty_like(t) for t in ts]
    host_out = torch.empty(3 * npx, dtype=torch.float32).pin_memory()
    scene_e = R.scene_to_c(*dev_in)
    h2d = sum(t.numel() * 4 for t in host_in)
    d2h = host_out.numel() * 4

    def e2e_step():
        for h, d in zip(host_in, dev_in):
            d.copy_(h, non_blocking=True)
        R.render_forward_raw(scene_e, cams_c, 1, opts_c, outs, ws)
        L.check(L.sof_render_bwd(scene_e, cams_c, 1, opts_c, R._out_c(outs), gin, sg, ws.handle,
                                 stream.cuda_stream), "sof_render_bwd", ws.handle)
        host_out.copy_(outs["color"], non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    peaks, peak_kind = _peaks()
    clocks = clk.summary()
    # roofline of the dominant kernel (the forward composite is timed with the forward phase;
    # its FP32 work comes from the counters of the last forward)
    fwd = statistics.median(fwd_ms)
    flops = stats["n_tests"] * FLOPS_PER_TEST + stats["n_hits"] * FLOPS_PER_HIT + \
        stats["n_composited"] * FLOPS_PER_COMPOSITE
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s, FFMA = 2 flops
    achieved = flops / (fwd * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": ms_per_step / world, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_gaussians": scene.n, "width": cam.width, "height": cam.height,
                   "l2": "inputs larger than L2 (scene 236 MB + records 96 MB + sorted pairs per step)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "tile": opts.tile, "chunk": opts.chunk, "reorder_k": opts.reorder_k},
        "phases_ms": {"fwd": fwd, "bwd": statistics.median(bwd_ms)},
        "work": stats,
        "roofline": {"bound": "alu", "kernel": "forward pass (composite-dominated)", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "peak_kind": f"FP32 FFMA issue: 152 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz"},
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_ms / world, "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(scene, cam)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chunk", type=int, default=64, help="records staged per shared-memory chunk")
    ap.add_argument("--reorder-k", type=int, default=16, help="per-pixel pending-hit buffer")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
