#!/usr/bin/env python3
"""Training-step throughput of the Student-splatting rasterizer on GB300.

One step = project + bin + sort + forward render of every view, L1 loss,
backward render + projection backward, SGHMC/Adam update -- the whole hot
path on a 1.5M-component scene (6 clusters + ground plane, SH degree 3,
nu in [1, 32], 30% scooping) seen by 4 views at 1297x840, seeded and
synthetic.  The step is captured once into a CUDA graph and replayed.

Prints one JSON line (rank 0).  Under torchrun every rank runs an
independent replica of the workload (no collective on the data path: the
path shards by scene/views without an exchange in this form), so scaling is
weak and `value` sums the pixels of all ranks over the slowest rank's time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on a bounded pixel sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s at 1.5M comps; serve p50/p99 ms, batched vs plain on one GB300"
UNIT = "Mpix/s"
WORKLOAD = ("clusters_1p5m_4views: 1.5M 3D t-components (6 Gaussian clusters + ground plane, log-scale "
            "N(-4,0.7), SH degree 3, nu log-uniform [1,32], 30% scooping), 4 views x 1297x840 per step, "
            "train step = project+bin+sort+render_fwd+loss(0.8 L1 + 0.2 D-SSIM, opacity/scale regularisers "
            "0.01)+render_bwd+project_bwd+sghmc_step")
WORKLOADS = {"clusters_1p5m_4views": "clusters_1p5m_4views", "shell_100k_8views": "shell_100k_8views",
             "gradcheck_cube_50k": "gradcheck_cube_50k"}
MUFU_PER_SM_CLK = 16    # MUFU (ex2/lg2) results per SM and clock
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0     # used only when neither nvidia-smi nor MEASURED_PEAKS.json gives it
# Algorithmic work of the render stages, the method's minimal per-pair work: the
# forward evaluates h (the cheap reject, 8 FP32 flops) for every evaluated
# (splat, pixel) pair and T2D, alpha and the compositing update (12 FP32
# flops + 2 MUFU: lg2, ex2) for every contributing pair; the backward does
# about 50 FP32 flops + 2 MUFU per contributing pair.
FWD_EVAL_FLOPS = 8
FWD_FLOPS, FWD_MUFU = 12, 2
BWD_FLOPS, BWD_MUFU = 50, 2
# A finer count of the backward's formulas written out (the same h, T2D, alpha
# and T recovery, dL/dalpha, dalpha/do, dalpha/dh, dalpha/dnu with its log,
# dh/dmean, dh/dconic, dL/drgb): 75 FP32 flops + 4 MUFU per contributing pair.
# Reported beside the minimal figure, labelled, never as the headline.
BWD_FLOPS_DETAILED, BWD_MUFU_DETAILED = 75, 4


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--tile", default=None, help="WxH tile, e.g. 16x16 (default: autotuned cache or 64x64)")
    ap.add_argument("--batch", type=int, default=None, help="records per warp and staging round with --tile: 32 or 64")
    ap.add_argument("--bwd-box-h", type=int, default=None,
                    help="height of the backward's warp box with --tile: 8 or 16 (16 needs tiles of at least 32x64)")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-frame-per-view comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-serve", action="store_true", help="skip the render-server leg")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="Poisson arrival window of the server leg at 200 req/s (the higher rates use 5 s)")
    ap.add_argument("--serve-tile", default="auto",
                    help="list tile of the server leg: 'auto' (per frame, the tuned tile of its largest view) "
                         "or WxH for every frame")
    ap.add_argument("--workload", default="clusters_1p5m_4views", choices=sorted(WORKLOADS),
                    help="smaller seeded workloads exist for profiling; the benchmark line uses the default")
    return ap.parse_args()


# ------------------------------------------------------------------ ranks

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (x itself with one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASON_NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t0 = time.time()

    def stop(self) -> dict | None:
        self.t1 = time.time()
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
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
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, val in zip(REASON_NAMES, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ ours

def _cfg(args):
    from paper_2503_10148_gb300 import autotune, frame
    if getattr(args, "tile", None):
        tw, th = (int(v) for v in args.tile.split("x"))
        return frame.make_cfg(tile_w=tw, tile_h=th, batch=getattr(args, "batch", None) or 32,
                              bwd_box_h=getattr(args, "bwd_box_h", None) or 8), "cli"
    best = autotune.cached(getattr(args, "workload", "clusters_1p5m_4views"))
    if best:
        return frame.make_cfg(tile_w=best["tile_w"], tile_h=best["tile_h"], batch=best.get("batch", 32),
                              bwd_box_h=best.get("bwd_box_h", 8)), "autotuned"
    return frame.make_cfg(), "default"


def stage_breakdown(ts, reps, device):
    """Eager steps with CUDA events between the stages (same stream); like
    the timed steps, each starts from the configured scene (the sampler
    writes its update beside it)."""
    import torch
    from paper_2503_10148_gb300 import frame as F
    fr = ts.frame
    st = torch.cuda.current_stream(device)
    names = ["project", "bin", "sort", "render_fwd", "loss", "render_bwd", "project_bwd", "sghmc_step"]
    acc = {n: 0.0 for n in names}
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record(st)
        fr.project(st); ev[1].record(st)
        fr.bin(st); ev[2].record(st)
        fr.sort(st); ev[3].record(st)
        fr.render_fwd(st); ev[4].record(st)
        if ts.loss_kind == "full":
            F.loss_image(fr, fr.rgb, ts.targets, ts.eps_dssim, ts.loss3, ts.scratch, st)
            F.loss_image_grad(fr, fr.rgb, ts.targets, ts.eps_dssim, ts.scratch, ts.dl, stream=st)
        else:
            F.loss_l1(fr.rgb, ts.targets, ts.dl, ts.loss, st)
        ev[5].record(st)
        fr.render_bwd(ts.dl, st); ev[6].record(st)
        fr.project_bwd([ts.grads], st); ev[7].record(st)
        ts.sample(st); ev[8].record(st)
        torch.cuda.synchronize(device)
        for i, n in enumerate(names):
            acc[n] += ev[i].elapsed_time(ev[i + 1])
    return {n: acc[n] / reps for n in names}


def count_pairs(ts, device):
    """Contributing and evaluated (splat, pixel) pairs of the frame a timed
    step renders: the step starts from the configured scene, so one counting
    forward of that scene (outside the timed region) gives them."""
    import torch
    assert ts.after is not None, "the timed steps must leave the configured scene unchanged"
    torch.cuda.synchronize(device)
    out = ts.frame.count_pairs()
    torch.cuda.synchronize(device)
    return out


def alu_ceiling(n_sms: int, mhz: float) -> tuple[float, float]:
    """(FP32 FLOP/s, MUFU op/s) of the device: unit counts x SM clock."""
    clk = mhz * 1e6
    return n_sms * FP32_LANES_PER_SM * 2 * clk, n_sms * MUFU_PER_SM_CLK * clk


def alu_roofline(kernel: str, ms: float, flops: float, mufu: float, n_sms: int, mhz: float, work: str) -> dict:
    """Achieved FP32 FLOP/s against the ALU ceiling: the shortest time the
    FP32 and MUFU pipes could do the work in, max(flops / P_fp32, mufu /
    P_mufu), divided by the measured time, is `frac`; `peak` is the FLOP rate
    at that ceiling."""
    t = ms * 1e-3
    p_fp32, p_mufu = alu_ceiling(n_sms, mhz)
    t_min = max(flops / p_fp32, mufu / p_mufu)
    return {"bound": "alu", "kernel": kernel, "achieved": round(flops / t / 1e12, 3),
            "peak": round(flops / t_min / 1e12, 3), "unit": "TFLOP/s", "frac": round(t_min / t, 4),
            "traffic": None, "peak_source": f"{n_sms} SMs x ({FP32_LANES_PER_SM} FP32 lanes x 2, "
                                           f"{MUFU_PER_SM_CLK} MUFU) x {mhz:.0f} MHz",
            "work": work}


def roofline(stage: str, ms: float, ts, pairs: tuple, peaks: dict, peak_src: str, n_sms: int, mhz: float):
    """Achieved vs peak for the dominant stage; ALU stages (the renders)
    against the FP32/MUFU ceiling derived from the device's SM count and
    maximum SM clock, memory stages against the measured copy bandwidth."""
    contrib, evaluated = pairs
    if stage == "render_bwd":
        r = alu_roofline(stage, ms, contrib * BWD_FLOPS, contrib * BWD_MUFU, n_sms, mhz,
                         f"{contrib} contributing pairs x ({BWD_FLOPS} FP32 flops + {BWD_MUFU} MUFU)")
        d = alu_roofline(stage, ms, contrib * BWD_FLOPS_DETAILED, contrib * BWD_MUFU_DETAILED, n_sms, mhz, "")
        r["detailed_count"] = {"work": f"{contrib} contributing pairs x ({BWD_FLOPS_DETAILED} FP32 flops + "
                                       f"{BWD_MUFU_DETAILED} MUFU), the formulas written out",
                               "achieved": d["achieved"], "peak": d["peak"], "frac": d["frac"]}
        return r
    if stage == "render_fwd":
        return alu_roofline(stage, ms, evaluated * FWD_EVAL_FLOPS + contrib * FWD_FLOPS, contrib * FWD_MUFU,
                            n_sms, mhz, f"{evaluated} evaluated pairs x {FWD_EVAL_FLOPS} FP32 flops + {contrib} "
                                        f"contributing pairs x ({FWD_FLOPS} FP32 flops + {FWD_MUFU} MUFU)")
    t = ms * 1e-3
    nbytes = algorithmic_bytes(stage, ts)
    achieved = nbytes / t / 1e9
    peak = float(peaks["hbm_gbs"])
    return {"bound": "hbm", "kernel": stage, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "peak_source": f"{peak_src} hbm_gbs",
            "work": f"{nbytes} algorithmic bytes"}


PROFILED_SOURCES = {"render_bwd": ("render_bwd.cu", "common.cuh"), "render_fwd": ("render_fwd.cu", "common.cuh")}


def code_hash(files) -> str:
    """First 16 hex digits of the sha256 of the C/CUDA sources `files` (under
    csrc/) with comments removed and whitespace runs collapsed: an edit of a
    comment leaves it unchanged, a change of the code does not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2503_10148_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    profiles/<kernel>_<workload>.md, or None when there is none or the kernel
    sources' code no longer hashes to the value recorded with the counters."""
    import re
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    srcs = PROFILED_SOURCES.get(kernel)
    if not srcs or not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"code_sha256_16:\s*([0-9a-f]{16})", text)
    m_b = re.search(r"dram_bytes_per_launch:\s*(\d+)", text)
    if not (m_sha and m_b):
        return None
    return int(m_b.group(1)) if code_hash(srcs) == m_sha.group(1) else None


def algorithmic_bytes(stage: str, ts) -> int:
    fr = ts.frame
    P = fr.plan
    n = ts.scene.n
    K = (ts.scene.sh_degree + 1) ** 2
    V = P.n_jobs
    pairs = fr.status()[1]
    if stage == "project":
        return n * (12 + 3 * K) * 4 + V * n * 64
    if stage == "project_bwd":
        return n * (12 + 3 * K) * 4 * 2 + V * n * 48
    if stage == "sghmc_step":
        return n * 4 * (3 * 4 + 1 + (9 + 3 * K) * 7)
    if stage == "sort":
        passes = (P.tile_bits + 7) // 8
        return pairs * (passes * 16 + 4)
    if stage == "bin":
        return V * n * 4 * (4 * 4 + 3) + pairs * 8
    return 0


def kernels_per_step(plan, form: str = "autograd", loss: str = "full") -> int:
    """Our kernel launches in one train step (memsets excluded)."""
    pair_passes = (plan.tile_bits + 7) // 8
    bin_k = 1 + 4 * 3 + 4  # init, 4 radix passes, count/scan/finish/emit
    sort_k = pair_passes * 3 + 2  # radix passes, range init and fix-up
    if loss == "full":
        loss_k = 3  # SSIM value, finish, gradient
    else:
        loss_k = 2 if form == "autograd" else 1  # value, then the gradient in the backward
    sampler_k = 3  # SGHMC, Adam rows, and the advance of the device step counter
    return 1 + bin_k + sort_k + 1 + loss_k + 1 + 1 + sampler_k


def run_ours(args):
    import torch
    from paper_2503_10148_gb300 import build, frame as F, inputs, train
    rank, world, local = dist_env()
    assert torch.cuda.is_available(), "bench.py needs a GPU (no CPU fallback)"
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init(world, "nccl")
    build.build()

    scene_np, cams = getattr(inputs, WORKLOADS[args.workload])()
    cams = [F.f32_camera(c) for c in cams]
    targets_np = np.concatenate([t.reshape(-1) for t in inputs.target_images(cams, seed=3)])
    scene = F.Scene.from_numpy(scene_np, device)
    targets = torch.as_tensor(targets_np, device=device)
    cfg, cfg_src = _cfg(args)
    # every timed step starts from the configured scene (the sampler writes
    # its update beside it), so the workload does not drift under the sampler
    ts = train.TrainStep(scene, cams, targets, cfg=cfg, device=device, loss="full", eps_dssim=0.2, reg_opacity=0.01,
                         reg_scale=0.01, restart=True)
    ts.calibrate()
    # one capture of the step per timed step, each with its own CUDA events
    # around the render launches (recorded as graph nodes) and all sharing
    # the first capture's memory pool: after the timed region every timed
    # step's kernel durations can be read, and averaged
    in_graph_timing = ts.time_kernels(("render_fwd", "render_bwd"))
    ts.capture()
    copies = [(ts.graph, ts.frame.timing)]
    if in_graph_timing:
        for _ in range(args.steps - 1):
            ts.time_kernels(("render_fwd", "render_bwd"))
            copies.append((ts.capture(pool=copies[0][0].pool(), warmup=0), ts.frame.timing))
    for g, _ in copies:  # a graph's first launch uploads it: every copy once before the timed region
        g.replay()
    for _ in range(max(args.warmup, 3)):
        ts.replay()
    torch.cuda.synchronize(device)

    mpix = sum(c.width * c.height for c in cams) / 1e6
    gpu_idx = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    clocks = ClockSampler(gpu_idx)
    st = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # one event between consecutive steps as well, for the per-step median
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps - 1)]
    barrier(world)
    torch.cuda.synchronize(device)
    clocks.start()
    e0.record(st)
    for k in range(args.steps):
        copies[k % len(copies)][0].replay()
        if k + 1 < args.steps:
            evs[k].record(st)
    e1.record(st)
    torch.cuda.synchronize(device)
    barrier(world)
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    marks = [e0, *evs, e1]
    step_ms = [a.elapsed_time(b) for a, b in zip(marks, marks[1:])]
    ms_median = statistics.median(step_ms)
    ms_max = max_over_ranks(ms, world, device)
    ts.check()
    # the render kernels' average duration over the timed steps (each timed
    # step is its own capture, whose events kept its launch's times); the
    # pair counts of the frame every timed step renders (the configured
    # scene), from one extra forward with counting on
    kern_ms = None
    if in_graph_timing:
        kern_ms = {k: round(statistics.fmean(t[k][0].elapsed_time(t[k][1]) for _, t in copies), 4)
                   for k in ("render_fwd", "render_bwd")}
    contrib_t, evaluated_t = count_pairs(ts, device)

    # end to end: every step's targets come from pinned host memory and its
    # loss goes back to the host.  The host->device copy of step k+1's
    # targets runs on a copy stream, into one of two staging buffers, while
    # step k computes; each step starts with a device copy of its staged
    # targets into the buffer the captured step reads.
    host_t = torch.empty(targets.numel(), dtype=torch.float32, pin_memory=True)
    host_t.copy_(torch.as_tensor(targets_np))
    host_loss = torch.empty(1, dtype=torch.float32, pin_memory=True)
    copy_st = torch.cuda.Stream(device)
    staging = [torch.empty_like(ts.targets), torch.empty_like(ts.targets)]
    staged = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]

    def h2d(k):
        b = k & 1
        with torch.cuda.stream(copy_st):
            if k >= 2:
                copy_st.wait_event(consumed[b])  # step k-2 has taken its targets
            staging[b].copy_(host_t, non_blocking=True)
            staged[b].record(copy_st)

    barrier(world)
    torch.cuda.synchronize(device)
    w0 = time.perf_counter()
    e0.record(st)
    h2d(0)
    for k in range(args.steps):
        if k + 1 < args.steps:
            h2d(k + 1)
        b = k & 1
        st.wait_event(staged[b])
        ts.targets.copy_(staging[b], non_blocking=True)
        consumed[b].record(st)
        ts.replay()
        host_loss.copy_(ts.loss, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize(device)
    wall = (time.perf_counter() - w0) * 1e3 / args.steps
    barrier(world)
    e2e_ms = max_over_ranks(max(e0.elapsed_time(e1) / args.steps, wall), world, device)
    ts.check()

    # per-stage breakdown and roofline of the dominant kernel (and of the
    # forward render), against the ceiling of this device: its SM count and
    # maximum SM clock
    stages = stage_breakdown(ts, 3, device)
    contrib, evaluated = contrib_t, evaluated_t
    dom = max(stages, key=stages.get)
    peaks, peak_src = measured_peaks()
    n_sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = float((clock_info or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or SM_MAX_MHZ)
    timing = {k: (kern_ms[k], "CUDA events around the launch inside the captured step, mean over the timed steps")
              if kern_ms and k in kern_ms else (stages[k], "CUDA events around the launch, eager step after the "
                                                           "timed region") for k in stages}
    roof = roofline(dom, timing[dom][0], ts, (contrib, evaluated), peaks, peak_src, n_sms, mhz)
    roof["timing"] = timing[dom][1]
    roof["traffic"] = profiled_traffic(dom, args.workload)
    roof_fwd = roofline("render_fwd", timing["render_fwd"][0], ts, (contrib, evaluated), peaks, peak_src, n_sms, mhz)
    roof_fwd["timing"] = timing["render_fwd"][1]
    roof_fwd["traffic"] = profiled_traffic("render_fwd", args.workload)
    _, pairs, _ = ts.frame.status()

    plain = None
    if not args.no_plain:
        ps = train.PlainStep(scene, cams, targets, cfg=cfg, device=device, loss="full", restart=True)
        ps.run()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        e0.record(st)
        reps = max(3, args.steps // 4)
        for _ in range(reps):
            ps.run()
        e1.record(st)
        torch.cuda.synchronize(device)
        pms = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3) / reps
        plain = {"form": "one frame per view, eager launches", "ms_per_step": round(pms, 3),
                 "value": round(world * mpix / (pms * 1e-3), 2)}

    result = {
        "metric": METRIC, "value": round(world * mpix / (ms_max * 1e-3), 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms_max, 3),
        "ms_per_step_median": round(ms_median, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded scene, cameras and target images)",
        "config": {"workload": WORKLOAD if args.workload == "clusters_1p5m_4views" else args.workload,
                   "views": len(cams), "width": cams[0].width, "height": cams[0].height,
                   "components": scene.n, "tile": f"{cfg.tile_w}x{cfg.tile_h}", "batch": cfg.batch, "bwd_box_h": cfg.bwd_box_h,
                   "cfg_source": cfg_src, "form": "batched frame through torch.autograd.Function (render, image loss), whole step in one CUDA graph, every step from the configured scene",
                   "pairs_per_step": pairs, "pair_capacity": ts.frame.pair_capacity,
                   "l2": "inputs larger than L2 (params 360 MB, pair lists > 1 GB, images 52 MB)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(world * mpix / (e2e_ms * 1e-3), 2), "unit": UNIT,
                "h2d_bytes_per_step": int(targets.numel() * 4), "d2h_bytes_per_step": 4},
        "gpu_launches": kernels_per_step(ts.frame.plan, ts.form, ts.loss_kind) * args.steps,
        "roofline": roof,
        "roofline_render_fwd": roof_fwd,
        "stages_ms": {k: round(v, 3) for k, v in stages.items()},
        "pairs": {"contributing": contrib, "evaluated": evaluated},
        "clocks": clock_info,
        "kernel_ms_in_graph": kern_ms,
        "plain": plain,
    }
    result["relocate"] = relocate_leg(scene_np, device)
    result["inference"] = inference_leg(scene_np, cams, device, cfg)
    if not args.no_serve:
        if args.serve_tile == "auto":
            from paper_2503_10148_gb300 import autotune
            result["serve"] = serve_leg(device, F.make_cfg(), args.serve_seconds, tile_of=autotune.serve_tile)
        else:
            stw, sth = (int(v) for v in args.serve_tile.split("x"))
            result["serve"] = serve_leg(device, F.make_cfg(tile_w=stw, tile_h=sth), args.serve_seconds)
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ recycling

def relocate_leg(scene_np, device, reps: int = 5) -> dict:
    """One sss_relocate call on the benchmark scene with 10 % of the
    opacities made transparent (seeded), timed with CUDA events; the
    parameters are restored between repetitions outside the timed call."""
    import torch
    from paper_2503_10148_gb300 import _abi, frame as F
    sc_np = dict(scene_np)
    rng = np.random.default_rng(31)
    n = sc_np["n"]
    raw = np.array(sc_np["opacity_raw"], np.float32, copy=True)
    dead = rng.random(n) < 0.10
    raw[dead] = rng.uniform(-0.004, 0.004, int(dead.sum())).astype(np.float32)
    sc_np["opacity_raw"] = raw
    sc = F.Scene.from_numpy(sc_np, device)
    pristine = {f: sc.t[f].clone() for f in F.FIELDS}
    st = F.SamplerState(sc)
    scratch = torch.empty(_abi.sss_relocate_scratch_bytes(n, 0.05) + 256, dtype=torch.uint8, device=device)
    moved = torch.zeros(1, dtype=torch.int32, device=device)
    times = []
    for k in range(reps + 1):
        for f in F.FIELDS:
            sc.t[f].copy_(pristine[f])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        F.relocate(sc, st, seed=7, step=k, moved_out=moved, scratch=scratch)
        e1.record()
        torch.cuda.synchronize(device)
        if k:
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    return {"workload": "clusters_1p5m_4views scene, 10 % of opacities transparent, at most 5 % moved per call, "
                        "<= 31 copies per target", "components": n, "moved": int(moved.cpu()[0]),
            "ms": round(ms, 4), "mcomponents_per_s": round(n / ms / 1e3, 1)}


def inference_leg(scene_np, cams, device, cfg, reps: int = 50) -> dict:
    """Inference-only rendering of the benchmark scene (project -> bin ->
    sort -> render_fwd, no backward): views per second at 1297x840 with one
    view per frame and with the four views in one frame, eager launches on
    one stream, timed with CUDA events over `reps` frames after a warm-up
    (the scene and cameras resident in HBM)."""
    import torch
    from paper_2503_10148_gb300 import frame as F
    sc = F.Scene.from_numpy(scene_np, device)
    out = {"workload": "clusters_1p5m_4views scene (1.5M components, SH degree 3), forward only, 1297x840"}
    for name, views in (("one_view", cams[:1]), ("four_views", cams)):
        fr = F.Frame([sc], views, cfg=cfg, device=device)
        fr.forward(grow=True)
        for _ in range(3):
            fr.forward(grow=False)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fr.forward(grow=False)
        e1.record()
        torch.cuda.synchronize(device)
        st, _, _ = fr.status()
        assert st == 0, st
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_frame": round(ms, 4), "views_per_s": round(len(views) * 1e3 / ms, 1)}
        del fr
    return out


# ------------------------------------------------------------------ serving

SERVE_WORKLOAD = ("3 resident scenes (200k, 1M, 3M components, clusters + ground distribution), Poisson "
                  "arrivals at 200 req/s (the configured rate) and at 500 and 1000 req/s, random camera on the "
                  "radius-3 sphere, resolution uniform over {256x256, 800x800, 1297x840, 1920x1080}; forward "
                  "render per request; then every request of the 200 req/s run arriving at once (burst)")
SERVE_RATES = (200.0, 500.0, 1000.0)


def serve_leg(device, cfg, seconds: float, tile_of=None) -> dict:
    """Render server (batched multi-scene frames) against one frame per
    request, on the same two arenas, streams and tile policy and the same
    seeded requests: latency at each arrival rate, then throughput with every
    request arriving at once."""
    import dataclasses
    import torch
    from paper_2503_10148_gb300 import frame as F, inputs, server
    scenes = [F.Scene.from_numpy(s, device) for s in inputs.serving_scenes()]
    budget = 16 << 30
    out = {"workload": SERVE_WORKLOAD, "hbm_budget_gb": budget >> 30,
           "tile": "per frame: the tuned tile of its largest view" if tile_of else f"{cfg.tile_w}x{cfg.tile_h}"}
    runs = []
    for rate in SERVE_RATES:
        window = seconds if rate == SERVE_RATES[0] else min(seconds, 5.0)
        reqs = server.poisson_requests(len(scenes), rate=rate, duration=window, seed=21)
        runs.append((f"poisson_{int(rate)}", reqs, window))
    runs.append(("burst", [dataclasses.replace(r, arrival=0.0) for r in runs[0][1]], 0.0))
    for name, rs, window in runs:
        srv = server.RenderServer(scenes, cfg, hbm_budget_bytes=budget, device=device, tile_of=tile_of)
        lat, ov = srv.serve(rs)
        b = server.summarize(lat, rs, srv)
        b["overflow_rerenders"] = ov
        del srv
        torch.cuda.empty_cache()
        lat_p, psrv = server.serve_plain(scenes, rs, cfg, hbm_budget_bytes=budget, device=device, tile_of=tile_of)
        p = server.summarize(lat_p, rs, psrv)
        del psrv
        torch.cuda.empty_cache()
        out[name] = {"arrival_window_s": window, "batched": b, "plain": p}
    return out


# ------------------------------------------------------------------ oracle

def _oracle_sample(scene_np, cams, n_pix, seed):
    """FP64 oracle forward + backward of n_pix seeded pixels per view (the
    projection of every (view, component) pair included)."""
    import oracle
    from paper_2503_10148_gb300 import inputs
    rng = np.random.default_rng(seed)
    pix = [rng.choice(c.width * c.height, n_pix, replace=False).astype(np.int64) for c in cams]
    w = inputs.linear_loss_weights(cams, seed)
    dl = [wv.reshape(3, -1)[:, p] for wv, p in zip(w, pix)]
    cfgd = dict(oracle.DEFAULT_CFG)
    t0 = time.perf_counter()
    oracle.backward(scene_np, cams, cfgd, dl, pix)
    return time.perf_counter() - t0


def cpu_baseline(budget_s: float):
    import oracle
    from paper_2503_10148_gb300 import inputs
    scene_np, cams = inputs.clusters_1p5m_4views()
    # two pilots fit t(n) = fixed (projection of all entries) + n x per-pixel
    t8 = _oracle_sample(scene_np, cams, 8, seed=100)
    t40 = _oracle_sample(scene_np, cams, 40, seed=99)
    per_px = max((t40 - t8) / 32.0, 1e-4)
    fixed = max(t8 - 8 * per_px, 0.0)
    n_pix = int(max(40, min(20000, (budget_s - fixed) / per_px)))
    t = _oracle_sample(scene_np, cams, n_pix, seed=101)
    if t < 0.5 * budget_s and n_pix < 20000:
        # the pilots overestimated the per-pixel cost (warm-up): rescale once
        n_pix = int(max(40, min(20000, n_pix * (budget_s - fixed) / max(t - fixed, 1e-3))))
        t = _oracle_sample(scene_np, cams, n_pix, seed=102)
    px = n_pix * len(cams)
    return {"value": round(px / t / 1e6, 8), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"FP64 oracle fwd+bwd of {n_pix} seeded pixels per view x {len(cams)} views of the "
                      f"1.5M-component workload, projection of all 6M (view, component) pairs included; "
                      f"{t:.1f} s"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2503_10148_gb300 import inputs
    oracle.build.build()
    scene_np, cams = inputs.clusters_1p5m_4views()
    warmup = max(args.warmup, 3)
    # each step a bounded sample: as many pixels per view as fit in
    # min(6 s, 150 s / (steps + warm-up)) beside the fixed projection of every
    # (view, component) pair, from two pilot samples that count as warm-up
    step_s = max(1.0, min(6.0, 150.0 / (args.steps + warmup)))
    t8 = _oracle_sample(scene_np, cams, 8, seed=1000)
    t40 = _oracle_sample(scene_np, cams, 40, seed=1001)
    per_px = max((t40 - t8) / 32.0, 1e-5)
    fixed = max(t8 - 8 * per_px, 0.0)
    n_pix = int(max(32, min(20000, (step_s - fixed) / per_px)))
    for w in range(warmup - 2):
        _oracle_sample(scene_np, cams, n_pix, seed=1002 + w)
    times = [_oracle_sample(scene_np, cams, n_pix, seed=2000 + k) for k in range(args.steps)]
    total = sum(times)
    px = n_pix * len(cams) * args.steps
    value = px / total / 1e6
    sample = (f"each step: FP64 oracle fwd+bwd of {n_pix} seeded pixels per view x {len(cams)} views of the "
              f"1.5M-component workload, projection of all (view, component) pairs included (pixels per view "
              f"sized from two pilots to about {step_s:.1f} s per step)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(total / args.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded scene and cameras)",
        "config": {"workload": WORKLOAD if args.workload == "clusters_1p5m_4views" else args.workload,
                   "views": len(cams), "width": cams[0].width, "height": cams[0].height,
                   "components": scene_np["n"]},
        "cpu_baseline": {"value": round(value, 8), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 8), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
