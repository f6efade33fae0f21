#!/usr/bin/env python3
"""Benchmark of the foveation path on one node.

Headline: foveated Mpix/s of one 1920x1080 RGB uint8 frame (sigma = 0.5 +
0.02 e, fixation at the centre, 32x32 blocks), frames resident in HBM,
rendered through the C ABI (fovea_render: sigma-table kernel, work-list
order kernel, persistent blur kernel). A step is one render of one frame.
Inputs rotate over a pool of distinct device buffers larger than L2.

Also reported on the same JSON line:
  e2e           same metric through fovea_render_host from pinned host
                memory (copies inside the timed region);
  roofline      the blur kernel timed alone with CUDA events on its stream,
                algorithmic FP32 FMAs per launch against the FP32 FMA peak;
  cpu_baseline  the FP64 oracle on a bounded sample of the frame's blocks;
  clocks        nvidia-smi samples taken during the timed region;
  batched       the 64-frame mixed batch in one launch vs one launch per frame;
  train         the 32x3x224x224 float32 batch, forward and forward+backward;
  block_sweep   render time and halo overhead for block sides 8, 16, 32, 64;
  served        p50/p99 latency of the served request stream (continuous
                batching) vs the plain one-request-per-launch loop.

`--impl reference` times the FP64 oracle (the reference arm of this build)
on bounded samples of the same workload and prints the same line.

Multi-GPU (torchrun, one process per GPU): replicas only; every rank renders
its own frames, there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import queue
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "foveated Mpix/s at 1080p RGB (% of roofline) + p50/p99 served-frame latency"
UNIT = "Mpix/s"
W, H, C, B = 1920, 1080, 3, 32
SIGMA0, K_SLOPE = 0.5, 0.02
FIX = (960.0, 540.0)
WORKLOAD = "1920x1080 RGB uint8 frame, 32x32 blocks, sigma = 0.5 + 0.02 e px, fixation at the centre"
L2_BYTES = 129 * 1024 * 1024
CSRC = os.path.join(ROOT, "paper_2012_08655_gb300", "csrc")
# Per forward kernel: committed ncu summary and the sources it was taken from.
KEV_EVERY = 16  # blur-kernel events on one step in KEV_EVERY of the timed region

KERNELS = {
    0: ("forward_kernel (fp32 FMA)", os.path.join(ROOT, "profiles", "forward_kernel_1080p_u8.txt"),
        ("forward.cu", "fwd_common.cuh", "fovea_internal.cuh")),
    1: ("tc_forward_kernel (tensor cores, mma.sync)", os.path.join(ROOT, "profiles", "tc_forward_kernel_1080p_u8.txt"),
        ("tc_forward.cu", "tc_common.cuh", "fwd_common.cuh", "fovea_internal.cuh")),
    2: ("umma_forward_kernel (vertical pass tcgen05 + TMEM, horizontal pass mma.sync)",
        os.path.join(ROOT, "profiles", "umma_forward_kernel_1080p_u8.txt"),
        ("umma_forward.cu", "tc05_common.cuh", "tc_common.cuh", "fwd_common.cuh", "fovea_internal.cuh")),
    3: ("tc05_forward_kernel (both passes tcgen05 + TMEM, warp-specialised pipeline)",
        os.path.join(ROOT, "profiles", "tc05_forward_kernel_1080p_u8.txt"),
        ("tc05_forward.cu", "tc05_common.cuh", "tc_common.cuh", "fwd_common.cuh", "fovea_internal.cuh")),
}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20000)
    p.add_argument("--warmup", type=int, default=200)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extras", action="store_true", help="skip the batched and served legs")
    p.add_argument("--served-seconds", type=float, default=10.0)
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--pixelwise-only", action="store_true",
                   help="run only the per-pixel foveation leg (--steps launches per kernel) and print it")
    p.add_argument("--train-only", action="store_true",
                   help="run only the float32 training leg (forward and backward) and print it")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline (profiling runs)")
    p.add_argument("--tensor-cores", type=int, choices=[0, 1, 2, 3], default=None,
                   help="force the forward kernel (0: fp32 FMA, 1: mma.sync, 2: tcgen05 vertical pass, "
                        "3: both passes on tcgen05) instead of autotuning")
    p.add_argument("--rows-per-chunk", type=int, choices=[16, 32, 64], default=32,
                   help="row chunk of the forced kernel (with --tensor-cores)")
    return p.parse_args()


# ------------------------------------------------------------------ helpers

def kernel_source_hash(tc: int) -> str:
    h = hashlib.sha256()
    for f in KERNELS[tc][2]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled(tc: int, rows_per_chunk: int):
    """Fields of the committed ncu summary of the timed kernel, or {} when it
    is missing, was taken with another row chunk, or the kernel's sources
    changed since it was taken."""
    try:
        vals = {}
        with open(KERNELS[tc][1]) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha256_16") != kernel_source_hash(tc):
            return {}
        if vals.get("rows_per_chunk") != str(rows_per_chunk):
            return {}
        return vals
    except OSError:
        return {}


def algorithmic_fmas(radius, width, height, channels, block):
    """Block-wise separable FMAs of one frame, halo rows included, clamping not
    folded: sum_b C (2 r_b + 1) bw (2 bh + 2 r_b)."""
    import numpy as np
    r = radius.astype(np.float64)
    nby, nbx = radius.shape
    bw = np.minimum(block, width - block * np.arange(nbx))[None, :].astype(np.float64)
    bh = np.minimum(block, height - block * np.arange(nby))[:, None].astype(np.float64)
    return float(np.sum(channels * (2 * r + 1) * bw * (2 * bh + 2 * r)))


def lower_bound_fmas(radius, width, height, channels, block):
    """Separable FMAs without halo overhead: 2 (2 r_b + 1) per output
    pixel-channel."""
    import numpy as np
    r = radius.astype(np.float64)
    nby, nbx = radius.shape
    bw = np.minimum(block, width - block * np.arange(nbx))[None, :].astype(np.float64)
    bh = np.minimum(block, height - block * np.arange(nby))[:, None].astype(np.float64)
    return float(np.sum(channels * 2 * (2 * r + 1) * bw * bh))


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples of one GPU (by UUID)."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or (self.uuid and self.uuid not in parts[0]):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(dev) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return ""


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle legs

def cpu_oracle_sample(target_s: float = 8.0, seed: int = 0):
    """Time the FP64 oracle on a bounded, seeded sample of the frame's blocks."""
    import numpy as np

    import oracle
    from paper_2012_08655_gb300 import workloads as wl
    frame = wl.frame_1080p()
    nb = ((W + B - 1) // B) * ((H + B - 1) // B)
    g = np.random.Generator(np.random.PCG64(seed))
    order = g.permutation(nb)
    threads = oracle.max_threads()
    # calibrate on a few blocks, then size the sample for about target_s seconds
    t0 = time.perf_counter()
    oracle.forward(frame.image, B, FIX[0], FIX[1], SIGMA0, K_SLOPE, "hwc", blocks=order[:threads].tolist())
    dt = max(time.perf_counter() - t0, 1e-3)
    n = int(min(nb, max(threads, threads * target_s / dt)))
    blocks = order[:n].tolist()
    t0 = time.perf_counter()
    oracle.forward(frame.image, B, FIX[0], FIX[1], SIGMA0, K_SLOPE, "hwc", blocks=blocks)
    dt = time.perf_counter() - t0
    px = n * B * B
    # the same oracle on one core, on a smaller sample (about a quarter of the time)
    n1 = max(1, int(n / threads / 4))
    t1 = time.perf_counter()
    oracle.forward(frame.image, B, FIX[0], FIX[1], SIGMA0, K_SLOPE, "hwc", blocks=order[:n1].tolist(), nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": px / dt / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} of {nb} blocks of the 1080p frame (seeded random), FP64 direct 2D sum, "
                      f"{threads} OpenMP threads, {dt:.2f} s",
            "one_core": {"value": n1 * B * B / dt1 / 1e6, "unit": UNIT,
                         "sample": f"first {n1} blocks of the same sample, 1 thread, {dt1:.2f} s"},
            "host": cpu_model()}


def cpu_model() -> str:
    """The host CPU as the OS reports it (model name, or Arm implementer/part)."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    name = fields.get("model name") or " ".join(
        f"{k} {fields[k]}" for k in ("CPU implementer", "CPU part") if k in fields)
    return f"{name or 'unknown'}, {os.cpu_count()} logical CPUs"


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2012_08655_gb300 import workloads as wl
    frame = wl.frame_1080p()
    nb = ((W + B - 1) // B) * ((H + B - 1) // B)
    order = np.random.Generator(np.random.PCG64(1)).permutation(nb)
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.forward(frame.image, B, FIX[0], FIX[1], SIGMA0, K_SLOPE, "hwc", blocks=order[:threads].tolist())
    per_block = max((time.perf_counter() - t0) / threads, 1e-4)
    # size each step so the whole run takes about two minutes of wall time
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = int(max(1, min(nb, budget * threads / per_block)))
    def step(i):
        sel = np.roll(order, -i * n)[:n].tolist()
        oracle.forward(frame.image, B, FIX[0], FIX[1], SIGMA0, K_SLOPE, "hwc", blocks=sel)
    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t0
    value = args.steps * n * B * B / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "block": B, "frame": f"{W}x{H}x{C}",
                                        "step": f"{n} blocks of the frame per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n} blocks per step, FP64 direct 2D sum, {threads} OpenMP threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU legs

def batched_leg(fv, torch):
    """64-frame mixed batch: one batched launch vs one render launch per frame."""
    from paper_2012_08655_gb300 import workloads as wl
    params = wl.mixed_batch_params(seed=0)
    content = {}
    ins, outs = [], []
    for (w, h, fx, fy, k) in params:
        if (w, h) not in content:
            content[(w, h)] = torch.from_numpy(wl.grating_frame(h, w, 3, seed=w)).cuda()
        ins.append(content[(w, h)].clone())
        outs.append(torch.empty_like(ins[-1]))
    frames = [fv.BatchFrame(ins[i], outs[i], p[2], p[3], 0.5, p[4]) for i, p in enumerate(params)]
    ctxs = {}
    px = sum(w * h for (w, h, _, _, _) in params)

    def batched():
        fv.foveate_batch(frames)

    def per_frame():
        for i, (w, h, fx, fy, k) in enumerate(params):
            key = (w, h, k)
            if key not in ctxs:
                ctxs[key] = fv.Context(w, h, 3, 32, 0.5, k, fv.U8_HWC)
            ctxs[key].render(ins[i], outs[i], fx, fy)

    # both arms autotuned: the batch on the batch itself, each per-frame
    # context on its own frame shape
    t0 = time.perf_counter()
    batch_cfg = fv.autotune_batch(frames, iters=3)
    tune_s = time.perf_counter() - t0
    for i, (w, h, fx, fy, k) in enumerate(params):
        key = (w, h, k)
        if key not in ctxs:
            ctxs[key] = fv.Context(w, h, 3, 32, 0.5, k, fv.U8_HWC)
            ctxs[key].autotune(iters=5)
    res = {}
    for name, fn in (("batched", batched), ("per_frame", per_frame)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": ms, "mpix_s": px / ms / 1e3}
    # the batch's algorithmic work (the method's separable FMAs, halo rows
    # included, clamping not folded) from each frame's radius table
    fmas = 0.0
    for (w, h, fx, fy, k) in params:
        _, rad = ctxs[(w, h, k)].sigma_table(fx, fy)
        fmas += algorithmic_fmas(rad.cpu().numpy(), w, h, 3, 32)
    tflops = 2 * fmas / (res["batched"]["ms"] * 1e-3) / 1e12
    return {"workload": "64 RGB uint8 frames: 16x640x480, 16x1280x720, 24x1920x1080, 8x3840x2160; "
                        "uniform fixations, k ~ U[0.01, 0.04]", "mpix": px / 1e6,
            "batched_mpix_s": res["batched"]["mpix_s"], "batched_ms": res["batched"]["ms"],
            "per_frame_mpix_s": res["per_frame"]["mpix_s"], "per_frame_ms": res["per_frame"]["ms"],
            "speedup": res["per_frame"]["ms"] / res["batched"]["ms"],
            "batch_config": batch_cfg, "batch_autotune_s": tune_s,
            "per_frame_configs": sorted({json.dumps(c.get_config(), sort_keys=True) for c in ctxs.values()}),
            "algorithmic_fmas": fmas, "batched_algorithmic_tflops": tflops,
            "note": "algorithmic FP32 FMAs of the whole batch over the batched time; the tensor-core "
                    "kernel does the work as fp16 MMAs, so the figure can exceed the FP32 peak"}


def sharded_batched_leg(fv, torch, world: int, rank: int, reps: int = 10):
    """The 64-frame mixed batch split over the ranks by estimated cost (LPT,
    the same assignment on every rank): each rank renders its frames as one
    autotuned batch on its GPU; time = max over ranks. Whole-job Mpix/s."""
    from paper_2012_08655_gb300 import replicas
    from paper_2012_08655_gb300 import workloads as wl
    params = wl.mixed_batch_params(seed=0)
    costs = [replicas.frame_cost(w, h, 3, replicas.frame_rmax(w, h, fx, fy, 0.5, k)) for (w, h, fx, fy, k) in params]
    mine = replicas.shard_frames(costs, world, rank)
    frames = []
    for i in mine:
        w, h, fx, fy, k = params[i]
        x = torch.from_numpy(wl.grating_frame(h, w, 3, seed=w)).cuda()
        frames.append(fv.BatchFrame(x, torch.empty_like(x), fx, fy, 0.5, k))
    cfg = fv.autotune_batch(frames, iters=3) if frames else None
    for _ in range(3):
        if frames:
            fv.foveate_batch(frames)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        if frames:
            fv.foveate_batch(frames)
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1) / reps, world)
    px = sum(w * h for (w, h, _, _, _) in params)
    return {"workload": "the 64-frame mixed batch split over the ranks", "ms": ms, "mpix_s": px / ms / 1e3,
            "frames_per_rank": [len(replicas.shard_frames(costs, world, r)) for r in range(world)],
            "rank0_config": cfg,
            "parallelism": f"frames sharded over {world} ranks by estimated cost (LPT), one batched launch per "
                           "GPU, max over ranks; no collective on the data path"}


def train_leg(fv, torch, reps: int = 20):
    """32x3x224x224 float32 batch (sigma = 0.5 + 0.08 e, random fixations):
    forward and backward through the autograd function (batched render and
    batched adjoint launches)."""
    from paper_2012_08655_gb300 import workloads as wl
    x_np, fix_np, s0, k = wl.train_batch(seed=0)
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    fix = torch.from_numpy(fix_np)
    g = torch.rand_like(x)
    n_img = x_np.shape[0]
    res = {}
    for name in ("forward", "forward_backward"):
        def step():
            y = fv.foveate_train(x, fix, s0, k)
            if name == "forward_backward":
                y.backward(g)
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            step()
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / reps
    # the same forward on the fp32 CUDA-core kernel (tensor cores off)
    b = fv._batch_ctx(32)
    b.set_config(256, 0, 32, tensor_cores=0)
    with torch.no_grad():
        for _ in range(3):
            fv.foveate_train(x, fix, s0, k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fv.foveate_train(x, fix, s0, k)
        e1.record()
        torch.cuda.synchronize()
    res["forward_fp32"] = e0.elapsed_time(e1) / reps
    # the backward alone (one batched adjoint launch per call): the fp32
    # adjoint every configuration but tensor_cores = 2 runs, then that one
    gi = torch.empty_like(g)
    frames = [fv.BatchFrame(g[i], gi[i], float(fix_np[i, 0]), float(fix_np[i, 1]), s0, k) for i in range(n_img)]
    for key, tc in (("backward", 1), ("backward_tensor_cores", 2)):
        b.set_config(256, 0, 32, tensor_cores=tc)
        for _ in range(3):
            b.backward_batch(frames)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.backward_batch(frames)
        e1.record()
        torch.cuda.synchronize()
        b.check()
        res[key] = e0.elapsed_time(e1) / reps
    b.set_config(256, 0, 32, tensor_cores=1)
    px = x_np.shape[0] * x_np.shape[2] * x_np.shape[3]
    # algorithmic work of the forward (the method's separable FMAs, halo
    # rows included, clamping not folded) from each image's radius table
    n, c, hh, ww = x_np.shape
    ctx = fv.Context(ww, hh, c, 32, s0, k, fv.F32_CHW)
    fmas = 0.0
    for i in range(n):
        _, rad = ctx.sigma_table(float(fix_np[i, 0]), float(fix_np[i, 1]))
        fmas += algorithmic_fmas(rad.cpu().numpy(), ww, hh, c, 32)
    tflops = 2 * fmas / (res["forward"] * 1e-3) / 1e12
    return {"workload": "32x3x224x224 float32 U[0,1), fixations uniform, sigma = 0.5 + 0.08 e",
            "forward_ms": res["forward"], "forward_backward_ms": res["forward_backward"],
            "forward_mpix_s": px / res["forward"] / 1e3,
            "forward_backward_mpix_s": px / res["forward_backward"] / 1e3,
            "forward_algorithmic_fmas": fmas,
            "forward_tflops": tflops,
            "forward_fp32_kernel_ms": res["forward_fp32"],
            "backward_ms": res["backward"],
            "backward_tensor_cores_ms": res["backward_tensor_cores"],
            "forward_note": "whole forward call (sigma, order and blur kernels, Python autograd overhead) "
                            "against the algorithmic FMAs; default configuration: float32 frames on the "
                            "mma.sync tensor-core kernel (fp16 hi + lo splits); forward_fp32_kernel_ms: the "
                            "same call on the fp32 CUDA-core kernel; backward_ms: one batched adjoint launch "
                            "(fovea_backward_batch) on the default fp32 adjoint, backward_tensor_cores_ms: the "
                            "same on the tensor-core adjoint (tensor_cores = 2)"}


def block_sweep_leg(fv, torch):
    """Fragment-size sweep at 1080p RGB: render time and the algorithmic work
    (halo overhead) for B in {8, 16, 32, 64}."""
    import numpy as np
    from paper_2012_08655_gb300 import workloads as wl
    frame = wl.frame_1080p(seed=0)
    x = torch.from_numpy(frame.image).cuda()
    y = torch.empty_like(x)
    res = {}
    for B in (8, 16, 32, 64):
        ctx = fv.Context(W, H, C, B, SIGMA0, K_SLOPE, fv.U8_HWC)
        cfg = ctx.autotune(iters=5)
        for _ in range(5):
            ctx.render(x, y, *FIX)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 50
        e0.record()
        for _ in range(reps):
            ctx.render(x, y, *FIX)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        _, rad = ctx.sigma_table(*FIX)
        fmas = algorithmic_fmas(rad.cpu().numpy(), W, H, C, B)
        res[str(B)] = {"ms": ms, "mpix_s": W * H / ms / 1e3, "algorithmic_fmas": fmas,
                       "fmas_per_pixel_channel": fmas / (W * H * C), "kernel_config": cfg}
    return {"workload": WORKLOAD.replace("32x32 blocks", "B x B blocks"), "by_block": res}


def plain_leg(fv, torch, reps: int = 2000):
    """The 256 x 256 single-channel float32 frame (sigma = 0.5 + 0.02 e,
    fixation at the centre): too small to fill the GPU, so it is reported as
    microseconds per render (launch latency), not against a roofline."""
    from paper_2012_08655_gb300 import workloads as wl
    spec = wl.plain_f32()
    x = torch.from_numpy(spec.image).cuda()
    y = torch.empty_like(x)
    h, w = spec.image.shape[-2:]
    ctx = fv.Context(w, h, 1, B, spec.sigma0, spec.k, fv.F32_CHW)
    for _ in range(20):
        ctx.render(x, y, spec.fix_x, spec.fix_y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.render(x, y, spec.fix_x, spec.fix_y)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / reps * 1e3
    # The same renders captured into a CUDA graph (100 per graph) and
    # replayed: the device time per render without host launch overhead,
    # the median over replays.
    graph = None
    try:
        import numpy as np
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            for _ in range(3):
                ctx.render(x, y, spec.fix_x, spec.fix_y)
        cs.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs):
            for _ in range(100):
                ctx.render(x, y, spec.fix_x, spec.fix_y)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        per = []
        cur = torch.cuda.current_stream()
        for _ in range(50):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(cur)
            g.replay()
            b.record(cur)
            b.synchronize()
            per.append(a.elapsed_time(b) * 10.0)  # ms per 100 renders -> us per render
        graph = {"us_per_render_median": float(np.median(per)), "replays": len(per), "renders_per_graph": 100}
    except Exception as ex:  # reported, not fatal: the eager figure stands
        graph = {"error": str(ex)[:200]}
    return {"workload": f"{w}x{h}x1 float32 U[0,1), sigma = {spec.sigma0} + {spec.k} e, fixation ({spec.fix_x}, "
                        f"{spec.fix_y})", "us_per_render": us, "renders": reps, "graph_replay": graph}


def pixel_radii(width, height, fix_x, fix_y, sigma0, k):
    """Per-pixel radius ceil(3 sigma) at pixel centres (the workload's size)."""
    import numpy as np
    x = np.arange(width) + 0.5
    y = np.arange(height) + 0.5
    e = np.sqrt((x[None, :] - fix_x) ** 2 + (y[:, None] - fix_y) ** 2)
    return np.ceil(3 * (sigma0 + k * e))


def pixelwise_mma_macs(width, height, channels, fix_x, fix_y, sigma0, k):
    """fp16 MMA multiply-adds one launch of the tensor-core per-pixel kernel
    issues: per 16 x 16 tile of radius R, per output column lx and channel
    plane, hi and lo products over ceil((16 + 2R) / 16) k-steps and the
    ceil((lx + 2R + 1) / 32) groups of 32 pixels (4 n-tiles) that hold the
    column's window."""
    import numpy as np
    r = pixel_radii(width, height, fix_x, fix_y, sigma0, k)
    macs = 0
    for y0 in range(0, height, 16):
        for x0 in range(0, width, 16):
            R = int(r[y0:y0 + 16, x0:x0 + 16].max())
            ks = (16 + 2 * R + 15) // 16
            lx = np.arange(min(16, width - x0))
            groups = int(((lx + 2 * R + 1 + 31) // 32).sum())
            macs += 2 * ks * 4 * groups * channels * 16 * 8 * 16
    return float(macs)


def pixelwise_leg(fv, torch, reps: int = 20):
    """Per-pixel ("perfect") foveation of the 1080p frame (Section 3.1's
    quality reference) on both kernels, and the SSIM of the block-wise output
    (anchored and fixation-centred grid) against it."""
    import numpy as np
    from paper_2012_08655_gb300 import workloads as wl
    frame = wl.frame_1080p(seed=0)
    x = torch.from_numpy(frame.image).cuda()
    y = torch.empty_like(x)
    r = pixel_radii(W, H, *FIX, SIGMA0, K_SLOPE)
    direct = float(C * ((2 * r + 1) ** 2).sum())
    res = {"workload": "1920x1080 RGB uint8 frame, every pixel its own sigma = 0.5 + 0.02 e px, "
                       "fixation at the centre",
           "direct_fmas_per_launch": direct, "max_radius": int(r.max())}
    for tc, n in ((1, reps), (0, max(2, reps // 8))):
        ctx = fv.Context(W, H, C, B, SIGMA0, K_SLOPE, fv.U8_HWC)
        ctx.set_config(256, 0, 32, tensor_cores=tc)
        for _ in range(3):
            ctx.render_pixelwise(x, y, *FIX)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            ctx.render_pixelwise(x, y, *FIX)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        leg = {"ms": ms, "mpix_s": W * H / ms / 1e3,
               "direct_tflops": 2 * direct / (ms * 1e-3) / 1e12}
        if tc:
            macs = pixelwise_mma_macs(W, H, C, *FIX, SIGMA0, K_SLOPE)
            leg["mma_flops_per_launch"] = 2 * macs
            leg["mma_tflops"] = 2 * macs / (ms * 1e-3) / 1e12
        res["tensor_core_kernel" if tc else "fp32_kernel"] = leg
    # Gaussian-pyramid (mipmap) foveation of the same frame: the comparison
    # approach of Section 3.2 (pyramid build + sampling, all launches)
    ctx = fv.Context(W, H, C, B, SIGMA0, K_SLOPE, fv.U8_HWC)
    for _ in range(3):
        ctx.render_pyramid(x, y, *FIX)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.render_pyramid(x, y, *FIX)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    res["pyramid"] = {"ms": ms, "mpix_s": W * H / ms / 1e3}
    ref = fv.foveate_pixelwise(x, *FIX, SIGMA0, K_SLOPE)
    pyr = fv.foveate_pyramid(x, *FIX, SIGMA0, K_SLOPE)
    outs = [("anchored_grid", fv.foveate(x, *FIX, SIGMA0, K_SLOPE, grid=fv.GRID_ANCHORED)),
            ("centred_grid", fv.foveate(x, *FIX, SIGMA0, K_SLOPE, grid=fv.GRID_CENTRED)), ("pyramid", pyr)]
    for name, blk in outs:
        m, mean = fv.ssim(blk, ref)
        mh = m.cpu().numpy()
        reg = mh[:H // 32 * 32, :W // 32 * 32].reshape(H // 32, 32, W // 32, 32).mean(axis=(1, 3))
        res["ssim_" + name] = {"mean": mean, "min": float(mh.min()), "worst_32px_region": float(reg.min())}
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fv.ssim(ref, ref, want_map=False)
    e1.record()
    torch.cuda.synchronize()
    res["ssim_ms"] = e0.elapsed_time(e1) / reps
    return res


def noalloc_leg(fv, torch, reps: int = 200):
    """fovea_render_noalloc (the entry point that allocates nothing: its
    scratch is a fixed array inside the library, and it always runs the fp32
    CUDA-core kernel) on the 1920x1080 RGB uint8 frame, against fovea_render
    on a context configured for the same kernel and on the context's default
    (tensor-core) configuration: ms per render, device-resident buffers, CUDA
    events over `reps` back-to-back calls."""
    from paper_2012_08655_gb300 import workloads as wl
    frame = wl.frame_1080p(seed=0)
    x = torch.from_numpy(frame.image).cuda()
    y = torch.empty_like(x)
    cur = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for _ in range(reps):
            fn()
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {"workload": "1920x1080 RGB uint8 frame, sigma = 0.5 + 0.02 e, fixation (960, 540)"}
    res["noalloc_ms"] = timed(lambda: fv.render_noalloc(x, y, *FIX, SIGMA0, K_SLOPE, block=B))
    fv.noalloc_check()
    ctx = fv.Context(W, H, C, B, SIGMA0, K_SLOPE, fv.U8_HWC)
    ctx.set_config(256, 0, 32, tensor_cores=0)
    res["render_fp32_kernel_ms"] = timed(lambda: ctx.render(x, y, *FIX))
    ctx.set_config(256, 0, 64, tensor_cores=1)
    res["render_tensor_core_ms"] = timed(lambda: ctx.render(x, y, *FIX))
    ctx.check()
    ctx.close()
    res["note"] = ("the no-allocation call runs the fp32 kernel with a fixed configuration; "
                   "render_fp32_kernel_ms is the regular entry point on that kernel")
    return res


def kernel_variants_leg(fv, torch, reps: int = 200):
    """Every forward kernel on the 1920x1080 RGB uint8 frame, each with its
    best row chunk: ms per render (sigma + blur, device-resident buffers,
    CUDA events over `reps` back-to-back renders) and the output's agreement
    with the mma.sync kernel's."""
    from paper_2012_08655_gb300 import workloads as wl
    frame = wl.frame_1080p(seed=0)
    x = torch.from_numpy(frame.image).cuda()
    cur = torch.cuda.current_stream()
    ctx = fv.Context(W, H, C, B, SIGMA0, K_SLOPE, fv.U8_HWC)
    outs, res = {}, {"workload": "1920x1080 RGB uint8 frame, sigma = 0.5 + 0.02 e, fixation (960, 540)"}
    for tc, rb in ((0, 32), (1, 64), (2, 32), (3, 16)):
        ctx.set_config(256, 0, rb, tensor_cores=tc)
        y = torch.empty_like(x)
        for _ in range(10):
            ctx.render(x, y, *FIX)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for _ in range(reps):
            ctx.render(x, y, *FIX)
        e1.record(cur)
        torch.cuda.synchronize()
        outs[tc] = y
        res[KERNELS[tc][0]] = {"ms": e0.elapsed_time(e1) / reps, "rows_per_chunk": rb}
    ctx.check()
    ctx.close()
    ref = outs[1].to(torch.int16)
    for tc in (0, 2, 3):
        d = (outs[tc].to(torch.int16) - ref).abs()
        res[KERNELS[tc][0]]["vs_mma_sync"] = {"max_lsb": int(d.max()), "equal": float((d == 0).float().mean())}
    return res


def served_leg(fv, torch, seconds: float, max_batch: int, world: int = 1, rank: int = 0):
    """Replay the Poisson request stream through the serving loop. With
    world > 1 each rank serves the requests of its streams (stream s on rank
    s mod world) on its own GPU and rank 0 merges the latencies."""
    import numpy as np

    from paper_2012_08655_gb300 import replicas
    from paper_2012_08655_gb300 import workloads as wl
    stream = wl.served_stream(seed=0, duration_s=seconds)
    mine = set(replicas.shard_streams(len(stream.stream_shapes), world, rank))
    reqs = [r for r in stream.requests if r.stream in mine]
    src, rings = {}, {}
    for s, (w, h, c) in enumerate(stream.stream_shapes):
        src[s] = torch.from_numpy(wl.grating_frame(h, w, c, seed=100 + s)).pin_memory()
        n = 32 if w * h < 100000 else 12
        rings[s] = [torch.empty_like(src[s]).pin_memory() for _ in range(n)]
    srv = fv.Server(device_budget_bytes=2 << 30, max_batch=max_batch, block=32, max_inflight=512)
    slot_owner = {}
    times = [None] * len(reqs)
    submitted = [0.0] * len(reqs)
    q = queue.Queue()

    def waiter():  # blocks on the queue and in the library, never polls
        for _ in range(len(reqs)):
            i, rid = q.get()
            times[i] = srv.wait(rid, timeout_ms=60000)

    th = threading.Thread(target=waiter, daemon=True)
    gc_was = gc.isenabled()
    gc.disable()  # no collector pauses inside the paced loop
    th.start()
    ring_pos = {s: 0 for s in rings}
    t0 = srv.now_us() + 200000.0
    try:
        for i, r in enumerate(reqs):
            s = r.stream
            slot = ring_pos[s] % len(rings[s])
            ring_pos[s] += 1
            prev = slot_owner.get((s, slot))
            if prev is not None:
                while times[prev] is None:  # output buffer still in use
                    time.sleep(0.0001)
            slot_owner[(s, slot)] = i
            arrival = t0 + r.arrival_s * 1e6
            while srv.now_us() < arrival:
                d = (arrival - srv.now_us()) * 1e-6
                if d > 0.0005:
                    time.sleep(d - 0.0003)
            submitted[i] = srv.now_us()
            q.put((i, srv.submit(src[s], rings[s][slot], r.fix_x, r.fix_y, stream.sigma0, stream.k,
                                 arrival_us=arrival)))
        th.join(timeout=120)
    finally:
        if gc_was:
            gc.enable()
    srv.close()
    done = [(i, t) for i, t in enumerate(times) if t]
    lat = np.array([(t["done_us"] - t["arrival_us"]) * 1e-3 for _, t in done])
    srv_lat = np.array([(t["done_us"] - submitted[i]) * 1e-3 for i, t in done])
    late = np.array([(submitted[i] - t["arrival_us"]) * 1e-3 for i, t in done])
    bs = np.array([t["batch_size"] for _, t in done])
    span = (max(t["done_us"] for _, t in done) - t0) * 1e-6
    px = sum(r.width * r.height for r in reqs)
    # Where the slowest 1 % of requests spend their time: waiting for
    # admission, waiting for their input copy and batch launch, and from the
    # batch launch until the worker saw their output copy finish.
    if world > 1:
        parts = replicas.gather_to_rank0({"lat": lat.tolist(), "px": px, "span": span, "n": len(reqs),
                                          "bs": bs.tolist(), "errors": int(sum(1 for _, t in done if t["status"]))})
        if parts is None:
            return None
        p50, p99 = replicas.merged_percentiles([p["lat"] for p in parts])
        return {"p50_ms": p50, "p99_ms": p99, "mpix_s": sum(p["px"] for p in parts) / max(p["span"] for p in parts) / 1e6,
                "requests": sum(p["n"] for p in parts), "errors": sum(p["errors"] for p in parts),
                "mean_batch": float(np.mean(np.concatenate([np.asarray(p["bs"]) for p in parts]))),
                "parallelism": f"streams sharded over {world} ranks (stream s on rank s mod {world}), one serving "
                               "loop per GPU, latencies merged on rank 0; no collective on the data path"}
    tail = lat >= np.percentile(lat, 99)
    ph = np.array([[t["admit_us"] - t["arrival_us"], t["start_us"] - t["admit_us"], t["done_us"] - t["start_us"]]
                   for _, t in done]) * 1e-3
    rpx = np.array([reqs[i].width * reqs[i].height for i, _ in done])
    tail_info = {"requests": int(tail.sum()), "mean_ms": float(lat[tail].mean()),
                 "admit_ms": float(ph[tail, 0].mean()), "copy_and_launch_ms": float(ph[tail, 1].mean()),
                 "render_and_d2h_ms": float(ph[tail, 2].mean()), "mean_mpix": float(rpx[tail].mean() / 1e6),
                 "mean_batch": float(bs[tail].mean())}
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "mpix_s": px / span / 1e6, "requests": len(reqs),
            "mean_batch": float(bs.mean()), "errors": int(sum(1 for _, t in done if t["status"] != 0)),
            "from_submit_p50_ms": float(np.percentile(srv_lat, 50)),
            "from_submit_p99_ms": float(np.percentile(srv_lat, 99)),
            "generator_late_p99_ms": float(np.percentile(late, 99)), "slowest_1pct": tail_info,
            "latency_note": "p50/p99 from the scheduled (Poisson) arrival; from_submit_* from the moment the "
                            "Python generator handed the request over (its lateness is generator_late_*)"}


def served_device_only(fv, torch, reps: int = 200):
    """Device-only time of the served stream's requests: per request class,
    one frame per batch launch from device-resident buffers (no copies),
    CUDA events around `reps` back-to-back launches with the stream's own
    fixations; the mean over the class mix weights each class by its share."""
    from paper_2012_08655_gb300 import workloads as wl
    stream = wl.served_stream(seed=0, duration_s=10.0)
    ctx = fv.batch_context(32)
    cur = torch.cuda.current_stream()
    by, wsum, tsum, psum = {}, 0.0, 0.0, 0.0
    for ci, (w, h, c, wt, _) in enumerate(wl.STREAM_CLASSES):
        x = torch.from_numpy(wl.grating_frame(h, w, c, seed=100 + ci)).cuda()
        o = torch.empty_like(x)
        fixes = [(r.fix_x, r.fix_y) for r in stream.requests if (r.width, r.height) == (w, h)][:reps]
        frames = [[fv.BatchFrame(x, o, fx, fy, stream.sigma0, stream.k)] for fx, fy in fixes]
        for f in frames[:20]:
            ctx.render_batch(f, cur)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(cur)
        for f in frames:
            ctx.render_batch(f, cur)
        e1.record(cur)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / len(frames)
        by[f"{w}x{h}x{c}"] = ms
        wsum += wt
        tsum += wt * ms
        psum += wt * w * h
    ctx.close()
    return {"per_request_ms": by, "mix_mean_ms": tsum / wsum, "mix_capacity_mpix_s": psum / (tsum * 1e-3) / 1e6,
            "note": "one frame per batch launch (sigma, order and blur kernels), device-resident buffers, "
                    f"CUDA events over {reps} back-to-back launches per class"}


def saturated_leg(fv, torch, seconds: float):
    """The served stream's requests all at once (no pacing): the serving loop
    (continuous batching) against the plain path, one fovea_render_host call
    per frame with the stream synchronised after each, as a one-request-at-
    a-time server would. Mpix/s of each."""
    from paper_2012_08655_gb300 import workloads as wl
    stream = wl.served_stream(seed=0, duration_s=seconds)
    reqs = stream.requests
    src, outs = {}, {}
    for s, (w, h, c) in enumerate(stream.stream_shapes):
        src[s] = torch.from_numpy(wl.grating_frame(h, w, c, seed=100 + s)).pin_memory()
        outs[s] = [torch.empty_like(src[s]).pin_memory() for _ in range(64 if w * h < 100000 else 16)]
    px = sum(r.width * r.height for r in reqs)
    # serving loop, every request submitted as soon as its output slot is free
    srv = fv.Server(device_budget_bytes=2 << 30, max_batch=64, block=32, max_inflight=512)
    pos = {s: 0 for s in outs}
    owner, ids = {}, []
    times = [None] * len(reqs)
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        slot = pos[r.stream] % len(outs[r.stream])
        pos[r.stream] += 1
        prev = owner.get((r.stream, slot))
        if prev is not None and times[prev] is None:  # the slot's previous result must be out
            times[prev] = srv.wait(ids[prev], timeout_ms=60000)
        owner[(r.stream, slot)] = i
        ids.append(srv.submit(src[r.stream], outs[r.stream][slot], r.fix_x, r.fix_y, stream.sigma0, stream.k))
    for i, rid in enumerate(ids):
        if times[i] is None:
            times[i] = srv.wait(rid, timeout_ms=60000)
    served_s = time.perf_counter() - t0
    srv.close()
    bs = [t["batch_size"] for t in times]
    # plain path: one render per request, synchronised
    shape_ctx = {}
    for s, (w, h, c) in enumerate(stream.stream_shapes):
        key = (w, h, c)
        if key not in shape_ctx:
            shape_ctx[key] = fv.Context(w, h, c, 32, stream.sigma0, stream.k, fv.U8_HWC)
    cur = torch.cuda.current_stream()
    for r in reqs[:50]:
        shape_ctx[(r.width, r.height, r.channels)].render_host(src[r.stream], outs[r.stream][0], r.fix_x, r.fix_y)
        cur.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        shape_ctx[(r.width, r.height, r.channels)].render_host(src[r.stream], outs[r.stream][0], r.fix_x, r.fix_y)
        cur.synchronize()
    plain_s = time.perf_counter() - t0
    # plain path pipelined: fovea_render_host calls back to back (each is
    # asynchronous, with two device slots per context), an output buffer
    # reused only once the call that last wrote it has completed
    pos = {s: 0 for s in outs}
    last = {}
    t0 = time.perf_counter()
    for r in reqs:
        slot = pos[r.stream] % len(outs[r.stream])
        pos[r.stream] += 1
        ev = last.get((r.stream, slot))
        if ev is not None:
            ev.synchronize()
        shape_ctx[(r.width, r.height, r.channels)].render_host(src[r.stream], outs[r.stream][slot], r.fix_x, r.fix_y)
        ev = torch.cuda.Event()
        ev.record(cur)
        last[(r.stream, slot)] = ev
    cur.synchronize()
    pipelined_s = time.perf_counter() - t0
    return {"workload": f"the served stream's {len(reqs)} requests ({px / 1e6:.0f} Mpix) submitted without pacing",
            "served_mpix_s": px / served_s / 1e6, "served_mean_batch": sum(bs) / len(bs),
            "plain_per_frame_mpix_s": px / plain_s / 1e6,
            "plain_pipelined_mpix_s": px / pipelined_s / 1e6,
            "plain_note": "plain_per_frame: fovea_render_host per request, stream synchronised after each; "
                          "plain_pipelined: the same calls back to back, synchronised only to reuse an output buffer",
            "errors": sum(1 for t in times if t["status"] != 0)}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    from paper_2012_08655_gb300 import fovea as fv
    if args.pixelwise_only:
        if rank == 0:
            print(json.dumps({"pixelwise": pixelwise_leg(fv, torch, reps=args.steps)}), flush=True)
        return 0
    if args.train_only:
        if rank == 0:
            print(json.dumps({"train": train_leg(fv, torch, reps=args.steps)}), flush=True)
        return 0
    from paper_2012_08655_gb300 import workloads as wl

    dev = torch.device("cuda", torch.cuda.current_device())
    frame = wl.frame_1080p(seed=rank)
    base = torch.from_numpy(frame.image).to(dev)
    fbytes = base.numel()
    pool_n = max(2, int(np.ceil(2 * L2_BYTES / (2 * fbytes))) + 1)  # in + out of the pool > 2x L2
    ins = [base.clone() for _ in range(pool_n)]
    outs = [torch.empty_like(base) for _ in range(pool_n)]
    ctx = fv.Context(W, H, C, B, SIGMA0, K_SLOPE, fv.U8_HWC)
    if args.tensor_cores is not None:
        ctx.set_config(256, 0, args.rows_per_chunk, tensor_cores=args.tensor_cores)
        cfg = ctx.get_config()
    else:
        cfg = ctx.get_config() if args.no_autotune else ctx.autotune(iters=20)
    stream = torch.cuda.current_stream()

    for i in range(args.warmup):
        ctx.render(ins[i % pool_n], outs[i % pool_n], *FIX)
    torch.cuda.synchronize()

    # The blur kernel is timed with CUDA events on every KEV_EVERY-th step of
    # the timed region; the other steps run without events between the sigma
    # and blur kernels, so the blur kernel's launch overlaps the sigma kernel
    # (programmatic dependent launch), as in an untimed render.
    n_kev = (args.steps + KEV_EVERY - 1) // KEV_EVERY
    ev_k = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_kev)]
    for a, b in ev_k:  # torch creates the CUDA events on first record
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(gpu_uuid(dev))
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.steps):
        if i % KEV_EVERY == 0:
            ctx.set_kernel_events(*ev_k[i // KEV_EVERY])
        elif i % KEV_EVERY == 1:
            ctx.set_kernel_events(None, None)
        ctx.render(ins[i % pool_n], outs[i % pool_n], *FIX)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ctx.set_kernel_events(None, None)
    ctx.check()  # raises if any kernel of the timed region recorded a device fault
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1), world)
    kernel_ms = float(np.mean([a.elapsed_time(b) for a, b in ev_k]))
    value = world * W * H * args.steps / (elapsed_ms * 1e-3) / 1e6

    # roofline of the blur kernel: algorithmic FP32 FMAs against the FP32 FMA peak
    sig, rad = ctx.sigma_table(*FIX)
    fmas = algorithmic_fmas(rad.cpu().numpy(), W, H, C, B)
    lower_fmas = lower_bound_fmas(rad.cpu().numpy(), W, H, C, B)
    props = torch.cuda.get_device_properties(dev)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak_tflops = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = 2 * fmas / (kernel_ms * 1e-3) / 1e12
    tc = int(cfg.get("tensor_cores", 0))
    prof = profiled(tc, int(cfg.get("rows_per_chunk", 32)))
    try:
        traffic = float(prof["dram_bytes_per_launch"]) if prof else None
    except (KeyError, ValueError):
        traffic = None
    measured_tflops = 2 * fv.measure_fma_rate() / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "peak_measured": measured_tflops, "frac_of_measured": achieved / measured_tflops,
                "lower_bound_fmas_per_launch": lower_fmas,
                "frac_lower_bound": 2 * lower_fmas / (kernel_ms * 1e-3) / 1e12 / peak_tflops,
                "kernel": KERNELS[tc][0], "kernel_ms": kernel_ms,
                "kernel_timing": f"CUDA events around the blur kernel on 1 step in {KEV_EVERY} of the timed region "
                                 f"({len(ev_k)} launches)",
                "algorithmic_fmas_per_launch": fmas,
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                              "(derived from unit counts and the maximum SM clock, not measured)",
                "hbm_bound_ms": 2 * fbytes / 6795.1e9 * 1e3}
    if tc and prof.get("mma_flops_per_launch"):
        # The same launch seen as a tensor-core contraction: fp16 MMA work per
        # launch (from the committed summary) against the measured dense
        # bf16 peak (fp16 has the same nominal rate).
        mma_tflops = float(prof["mma_flops_per_launch"]) / (kernel_ms * 1e-3) / 1e12
        roofline["tensor_view"] = {"achieved": mma_tflops, "peak": 1858.6, "unit": "TFLOP/s",
                                   "frac": mma_tflops / 1858.6, "peak_basis": "MEASURED_PEAKS bf16 burst (fp16 same rate)"}

    # end to end: pinned host frames through fovea_render_host
    hin = [torch.from_numpy(frame.image).pin_memory() for _ in range(4)]
    hout = [torch.empty_like(hin[0]).pin_memory() for _ in range(4)]
    for i in range(min(args.warmup, 50)):
        ctx.render_host(hin[i % 4], hout[i % 4], *FIX)
    torch.cuda.synchronize()
    ke = args.steps
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    t0 = time.perf_counter()
    for i in range(ke):
        ctx.render_host(hin[i % 4], hout[i % 4], *FIX)
    e1.record(stream)
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3
    ctx.check()
    barrier(world)
    e2e_ms = max_over_ranks(max(e0.elapsed_time(e1), wall_ms), world)
    e2e = {"value": world * W * H * ke / (e2e_ms * 1e-3) / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(hin[0].numel()), "d2h_bytes_per_step": int(hout[0].numel()),
           "ms_per_step": e2e_ms / ke}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["batched"] = batched_leg(fv, torch)
        extras["train"] = train_leg(fv, torch)
        extras["block_sweep"] = block_sweep_leg(fv, torch)
        extras["pixelwise"] = pixelwise_leg(fv, torch)
        extras["plain_256"] = plain_leg(fv, torch)
        extras["noalloc"] = noalloc_leg(fv, torch)
        extras["kernel_variants"] = kernel_variants_leg(fv, torch)
        served = served_leg(fv, torch, args.served_seconds, max_batch=64)
        plain = served_leg(fv, torch, args.served_seconds, max_batch=1)
        served["plain_per_frame"] = {k: plain[k] for k in ("p50_ms", "p99_ms", "mpix_s", "mean_batch")}
        served["device_only"] = served_device_only(fv, torch)
        extras["served"] = served
        extras["saturated"] = saturated_leg(fv, torch, args.served_seconds)

    if world > 1 and not args.no_extras:
        extras["sharded_batch"] = sharded_batched_leg(fv, torch, world, rank)
        served = served_leg(fv, torch, args.served_seconds, 64, world, rank)
        if rank == 0:
            extras["served_sharded"] = served

    cpu = cpu_oracle_sample() if (rank == 0 and world == 1 and not args.no_cpu) else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 MMA (hi/lo split taps, u8 data exact) + f32" if tc else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "block": B, "frame": f"{W}x{H}x{C}", "io": "uint8 HWC",
                       "l2": f"inputs rotate over {pool_n} distinct frame buffers "
                             f"({2 * pool_n * fbytes / 2**20:.0f} MiB in+out) > L2",
                       "kernel_config": cfg, "parallelism": f"replicas x{world}"},
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": 2 * args.steps, "clocks": clocks,  # sigma + blur kernel per render
            "device_faults": 0,  # fovea_check after each timed region (it raises otherwise)
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
