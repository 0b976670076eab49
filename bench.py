#!/usr/bin/env python3
"""Benchmark of the block-based CCL hot path on GB300.

Headline workload (one "step"): the 8192x8192 Bernoulli(p=0.5, seed 0) image
labelled with 8-connectivity through ``ccl_label`` 32 times.  Four device
copies of the image and four label buffers are cycled, so consecutive
labelings touch different memory; one labeling reads 67 MB and writes
268 MB, more than the 129 MB L2, so nothing of a labeling is still in L2 when
its buffers come back.  Inputs are resident in HBM when the timed region
starts.

The JSON line carries, besides the contract keys:
  roofline      the dominant kernel's algorithmic bytes per launch divided by
                its mean CUDA-event duration, taken in a second pass of the
                same steps with per-kernel events on the launching stream
                (the headline pass records no per-kernel events), against
                the measured HBM copy bandwidth;
  kernels       that pass's per-kernel launches, mean times and shares;
  cpu_baseline  the CPU oracle timed on a bounded sample of the same image
                (CPU model and core count recorded);
  e2e           the same metric through ``ccl_label_host_async`` from pinned
                host buffers on three streams (copies inside the timed region);
  clocks        SM clocks and throttle reasons sampled during the timed region;
  extra         the 4096x4096 noise set (density sweep and granular noise,
                both connectivities); single 512^2 and 4096^2 images, L2
                flushed and warm (min, median, mean, stdev); the 256-image
                uneven batch (batched graph vs plain launches, and the CPU
                oracle over the batch on every host core); the serving stream
                at 2k/5k/10k requests/s (p50/p99 and stage percentiles,
                Gpixel/s); the coarse-labelling variants of Sec. 4.2 (time,
                counters); component statistics of the 8192^2 labels; 512^3
                volumes (6/26-connectivity).

``--impl reference`` times the CPU oracle instead (the reference arm), on
the same 8192x8192 image.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpixel/s & % HBM roofline, plain vs batched persistent; serving p50/p99 ms"
UNIT = "Gpixel/s"
BYTES_PER_PIXEL = 5          # 1 B image read + 4 B label written
KERNEL_BYTES_PER_PIXEL = {   # the path's algorithmic bytes each kernel moves, per pixel
    "k_block_local": 1,      # reads the image once (lane-tile kernels: 4-connected images)
    "k_block_merge": 0,      # block border records only
    "k_block_write": 4,      # writes every label once
    "k_piece_local": 1,      # reads the image once (piece labeller: 8-connected images)
    "k_piece_write": 4,      # writes every label once
}
SIDE = 4096                  # the 4096x4096 noise set (an extra)
CONNS = (4, 8)
HEAD_N = 8192                # the headline image: 8192x8192 Bernoulli(0.5), seed 0
HEAD_CONN = 8
HEAD_COPIES = 4              # device copies of the image / label buffers cycled
HEAD_PER_STEP = 32           # labelings per step
HEAD_WORKLOAD = ("8192x8192 uint8 Bernoulli(p=0.5, seed 0) image, 8-connectivity, plain ccl_label path, "
                 "32 labelings per step")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured", float(p.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


# the sources that define the three labelling kernels of the step
KERNEL_SOURCES = ("ccl_block.cuh", "ccl_internal.h", "ccl_kernels.cu", "ccl_pieces.cuh")


def csrc_digest(sources=KERNEL_SOURCES):
    """Digest of the kernels' sources; a recorded ncu figure is used only
    while it matches."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1712_09789_gb300", "csrc")
    for name in sources:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when there is none or the kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"^csrc_digest:\s*([0-9a-f]+)", text, re.M)
    m_b = re.search(r"^dram_bytes_per_launch_8192:\s*([0-9.eE+]+)", text, re.M)
    if not m_sha or not m_b or m_sha.group(1) != csrc_digest():
        return None
    return float(m_b.group(1))


def recorded_figures(profile: str, sources):
    """The `name: number` lines of a committed ncu summary under profiles/,
    or None when it is missing or its csrc_digest does not match `sources`."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"^csrc_digest:\s*([0-9a-f]+)", text, re.M)
    if not m_sha or m_sha.group(1) != csrc_digest(sources):
        return None
    return {k: float(v) for k, v in re.findall(r"^(dram_bytes_per_[a-z0-9_.]+):\s*([0-9.eE+]+)\s*$", text, re.M)}


class ClockSampler:
    """nvidia-smi clock and throttle samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu_index), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks_tensor(torch, v: float, world: int, device) -> float:
    """Largest `v` over all ranks (the step time every rank waited for)."""
    if world == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, px_per_rank_step: int, steps: int, ms_max: float) -> float:
    """Whole-job Gpixel/s: every rank labels its own copy of the step's work
    (independent images, no collective on the data path), timed by the
    slowest rank."""
    return world * px_per_rank_step * steps / (ms_max / 1e3) / 1e9


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def noise_4096_images():
    from paper_1712_09789_gb300 import synth

    return list(synth.noise_4096_set(SIDE))


def host_cpu():
    """CPU model and online core count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    import platform

    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


# ---------------------------------------------------------------------------
def run_reference(args):
    """The reference arm: the CPU oracle on the host, on the headline image;
    each step is one labeling of the 8192x8192 image (a bounded sample of the
    headline step's 32)."""
    rank, world, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    from paper_1712_09789_gb300 import synth

    oracle.build()
    img = synth.bernoulli(HEAD_N, HEAD_N, 0.5, 0)
    for _ in range(args.warmup):
        oracle.label(img, HEAD_CONN)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.label(img, HEAD_CONN)
    dt = time.perf_counter() - t0
    px = HEAD_N * HEAD_N * args.steps
    value = px / dt / 1e9
    sample = (f"one labeling of the 8192x8192 Bernoulli(0.5) image per step, 8-connectivity, "
              f"single thread; the GPU arm's step labels it 32 times")
    cpu = host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": HEAD_WORKLOAD + " (CPU oracle: one labeling per step)",
                   "H": HEAD_N, "W": HEAD_N, "connectivity": HEAD_CONN},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, **cpu},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_1712_09789_gb300 import build as lib_build
    from paper_1712_09789_gb300 import ccl, synth

    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        lib_build.build()
    if world > 1:
        torch.distributed.barrier()
    ccl.load()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v: float) -> float:
        return max_over_ranks_tensor(torch, v, world, "cuda")

    img_np = synth.bernoulli(HEAD_N, HEAD_N, 0.5, 0)
    dev = [torch.from_numpy(img_np).cuda() for _ in range(HEAD_COPIES)]
    outs = [torch.empty((HEAD_N, HEAD_N), dtype=torch.int32, device="cuda") for _ in range(HEAD_COPIES)]
    px_step = HEAD_PER_STEP * HEAD_N * HEAD_N

    def step():
        for k in range(HEAD_PER_STEP):
            j = k % HEAD_COPIES
            ccl.ccl_label(dev[j], HEAD_CONN, labels=outs[j])

    for _ in range(args.warmup):
        step()
    status = ccl.ccl_get_device_status()
    if status != ccl.CCL_OK:
        raise RuntimeError(f"device status after warm-up: {ccl.ccl_status_string(status)}")

    # -- timed region: device time with CUDA events on the launching stream
    # (the current stream, which ccl_label uses); no per-kernel events here
    cvd = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    sampler = ClockSampler(cvd[local].strip() if local < len(cvd) else str(local))
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    status = ccl.ccl_get_device_status()
    if status != ccl.CCL_OK:
        raise RuntimeError(f"device status after timed region: {ccl.ccl_status_string(status)}")
    ms = max_over_ranks(e0.elapsed_time(e1))
    value = weak_scaling_value(world, px_step, args.steps, ms)

    # -- per-kernel pass: the same steps again, with CUDA events recorded on
    # the launching stream around every kernel
    ccl.ccl_debug_kernel_timing(True)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    ktimes = {k: v for k, v in ccl.ccl_debug_kernel_times().items() if v[1]}
    ccl.ccl_debug_kernel_timing(False)

    hbm_gbs, peak_kind, _ = load_peaks()
    total_kernel_ms = sum(v[0] for v in ktimes.values()) or 1.0
    dominant = max(ktimes, key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dominant]
    dom_avg_s = dom_ms / max(1, dom_n) / 1e3
    algo_bytes = KERNEL_BYTES_PER_PIXEL[dominant] * HEAD_N * HEAD_N
    achieved = algo_bytes / dom_avg_s / 1e9
    traffic = recorded_traffic(dominant)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": hbm_gbs,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm_gbs,
                "traffic": traffic, "algorithmic_bytes_per_launch": algo_bytes,
                "mean_launch_us": dom_avg_s * 1e6,
                "timing": "mean CUDA-event duration per launch, from a second pass of the same steps"}
    kernels = {}
    for k, (t, n) in ktimes.items():
        mean_us = (t / n * 1e3) if n else None
        kb = KERNEL_BYTES_PER_PIXEL.get(k, 0) * HEAD_N * HEAD_N
        kernels[k] = {"launches": n, "mean_us": mean_us, "share": t / total_kernel_ms,
                      "algorithmic_gbs": (kb / (mean_us * 1e3)) if (mean_us and kb) else None}
    path_frac = value * 1e9 / world * BYTES_PER_PIXEL / (hbm_gbs * 1e9)
    us_per_image = ms * 1e3 / (args.steps * HEAD_PER_STEP)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {
            "workload": HEAD_WORKLOAD, "H": HEAD_N, "W": HEAD_N, "connectivity": HEAD_CONN,
            "labelings_per_step": HEAD_PER_STEP, "pixels_per_step": px_step,
            "l2": "inputs larger than L2: each labeling reads 67 MB and writes 268 MB; 4 input copies "
                  "and 4 label buffers cycle",
        },
        "us_per_image": us_per_image,
        "hbm_roofline_frac_path": path_frac,
        "roofline": roofline,
        "kernels": kernels,
        "gpu_launches": 3 * HEAD_PER_STEP * args.steps,
        "clocks": clocks,
    }

    only = set(args.only_extra.split(",")) if args.only_extra else None

    def want(name):
        return only is None or name in only

    # -- the serving stream (Poisson arrivals of mixed-resolution host frames
    # through the continuous-batching server) runs first among the host-link
    # workloads: its copy stages lengthen the longer the process has been
    # moving frames (p99 of the copies grows from pass to pass even on one
    # server and one set of buffers)
    serving = None
    if rank == 0 and not args.no_extra and want("serving"):
        serving = bench_serving(torch, ccl, args.serving_seconds)

    # -- e2e through host buffers (copies inside the timed region)
    if not args.no_e2e:
        line["e2e"] = bench_e2e(torch, ccl, img_np, args, world, max_over_ranks)

    if rank == 0 and not args.no_extra:
        extra = line.setdefault("extra", {})

        # the 4096x4096 noise set, both connectivities
        if want("noise_4096"):
            extra["noise_4096"] = bench_noise_4096(torch, ccl, hbm_gbs)
        # single 512x512 and 4096x4096 images, L2 flushed and warm
        if want("single_512"):
            extra["single_512"] = bench_single(torch, ccl, 512, hbm_gbs)
        if want("single_4096"):
            extra["single_4096"] = bench_single(torch, ccl, 4096, hbm_gbs)
        # the uneven 256-image batch, batched graph vs plain launches
        if want("batched_256"):
            extra["batched_256"] = bench_batched(torch, ccl, hbm_gbs)
        if serving is not None:
            extra["serving"] = serving
        # the coarse-labelling variants of Sec. 4.2 (time and counters)
        if want("variants"):
            extra["variants"] = bench_variants(torch, ccl)
        # component statistics of the 8192^2 labels
        if want("component_stats"):
            extra["component_stats"] = bench_stats(torch, ccl)
        # 3D volumes (512^3 noise, 6- and 26-connectivity)
        if want("volume_512"):
            extra["volume_512"] = bench_volume(torch, ccl, hbm_gbs)
        # strip sharding of the 8192^2 image, emulated on one GPU
        if want("strips_8192"):
            extra["strips_8192"] = bench_strips(torch, ccl)

    # -- the CPU oracle over the whole uneven batch on every host core (after
    # the GPU extras: its worker processes load the host)
    if rank == 0 and world == 1 and "batched_256" in line.get("extra", {}) and not args.no_cpu:
        try:
            cores = oracle_all_cores(synth.batch_uneven(256, seed=0), 8)
        except Exception as exc:  # the CPU baseline must not cost the GPU numbers
            cores = {"unavailable": f"{type(exc).__name__}: {exc}"}
        line["extra"]["batched_256"]["cpu_oracle_all_cores"] = cores

    # -- CPU oracle on a bounded sample, rank 0 at N = 1 only
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = bench_cpu(img_np, outs[(HEAD_PER_STEP - 1) % HEAD_COPIES])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_single(torch, ccl, N, hbm_gbs, reps=100, warm=10):
    """One N x N Bernoulli(0.5) image (seed 0), 8-connectivity, plain path.
    Device time: the call (``ccl_label_ws`` with caller-owned scratch)
    captured once in a CUDA graph and replayed, CUDA events around each
    replay, `reps` repetitions with L2 flushed before each (a 512 MB write)
    and `reps` without, after `warm` warm-ups; min / median / mean / stdev in
    us.  Call time: the same through ``ccl_label`` from Python, one call
    between events, host launch work included (what a caller that waits for
    every image sees)."""
    from paper_1712_09789_gb300 import synth

    img = torch.from_numpy(synth.bernoulli(N, N, 0.5, 0)).cuda()
    out = torch.empty((N, N), dtype=torch.int32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    ws = torch.empty(ccl.ccl_workspace_size(N, N, 8), dtype=torch.uint8, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warm):
            ccl.ccl_label_ws(img, ws, 8, labels=out)
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        ccl.ccl_label_ws(img, ws, 8, labels=out)

    def stats(fn, cold):
        ts = []
        for _ in range(reps):
            if cold:
                flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) * 1e3)
        med = statistics.median(ts)
        return {"min_us": min(ts), "median_us": med, "mean_us": statistics.fmean(ts),
                "stdev_us": statistics.stdev(ts), "gpixel_s": N * N / (med / 1e6) / 1e9,
                "hbm_roofline_frac": N * N * BYTES_PER_PIXEL / (med / 1e6) / (hbm_gbs * 1e9)}

    for _ in range(warm):
        graph.replay()
    res = {"workload": f"{N}x{N} Bernoulli p=0.5 seed 0, 8-connectivity, plain path",
           "device_cold": stats(graph.replay, True), "device_warm": stats(graph.replay, False),
           "call_cold": stats(lambda: ccl.ccl_label(img, 8, labels=out), True)}
    if ccl.ccl_get_device_status() != ccl.CCL_OK:
        raise RuntimeError("single-image labelling reported a device error")
    return res


def bench_noise_4096(torch, ccl, hbm_gbs, reps=5):
    """The 4096x4096 noise set: Bernoulli p = 0.1..0.9 and granular noise
    (g = 4, 16) at p = 0.5, seeds 0..2 (33 images), each labelled with 4- and
    8-connectivity (66 labelings, 1.107 Gpixel per pass).  33 inputs and 66
    outputs (4.98 GB) cycle, so nothing of a pass is in L2 when the same
    image comes back.  `reps` timed passes after two warm-up passes, then one
    more pass with per-kernel events for the shares."""
    named = noise_4096_images()
    dev = [torch.from_numpy(img).cuda() for _, img in named]
    work = [(i, c) for c in CONNS for i in range(len(dev))]
    outs = [torch.empty((SIDE, SIDE), dtype=torch.int32, device="cuda") for _ in work]

    def one_pass():
        for k, (i, c) in enumerate(work):
            ccl.ccl_label(dev[i], c, labels=outs[k])

    for _ in range(2):
        one_pass()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        one_pass()
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    ccl.ccl_debug_kernel_timing(True)
    one_pass()
    torch.cuda.synchronize()
    kt = {k: v for k, v in ccl.ccl_debug_kernel_times().items() if v[1]}
    ccl.ccl_debug_kernel_timing(False)
    if ccl.ccl_get_device_status() != ccl.CCL_OK:
        raise RuntimeError("4096x4096 noise set reported a device error")
    px = len(work) * SIDE * SIDE
    gpx = px / (ms / 1e3) / 1e9
    tot = sum(t for t, _ in kt.values()) or 1.0
    res = {"workload": "4096x4096 noise set: Bernoulli p=0.1..0.9 and granular g=4,16 at p=0.5, seeds 0..2, "
                       "4- and 8-connectivity (66 labelings per pass)",
           "ms_per_pass": ms, "gpixel_s": gpx,
           "hbm_roofline_frac": gpx * 1e9 * BYTES_PER_PIXEL / (hbm_gbs * 1e9),
           "kernels": {k: {"mean_us": (t / n * 1e3 if n else None), "share": t / tot} for k, (t, n) in kt.items()}}
    del dev, outs
    torch.cuda.empty_cache()
    return res


def _oracle_batch_task(task):
    """Worker of oracle_all_cores: labels one image of the batch, read from
    the memory-mapped batch file, with the CPU oracle."""
    import numpy as np

    import oracle

    path, off, H, W, conn = task
    img = np.memmap(path, dtype=np.uint8, mode="r", offset=off, shape=(H, W))
    oracle.label(np.asarray(img), conn)
    return H * W


def oracle_all_cores(imgs, conn):
    """The CPU oracle over a whole batch, one image per task on every host
    core (spawned worker processes; the batch is shared through a
    memory-mapped file, so the timed region holds labelling only)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "batch.u8")
        tasks, off = [], 0
        with open(path, "wb") as f:
            for im in imgs:
                f.write(np.ascontiguousarray(im).tobytes())
                tasks.append((path, off, im.shape[0], im.shape[1], conn))
                off += im.size
        # a worker that cannot start makes the executor raise, not wait
        with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
            list(pool.map(_oracle_batch_task, tasks[:cores]))  # every worker loads the oracle
            t0 = time.perf_counter()
            px = sum(pool.map(_oracle_batch_task, tasks))
            dt = time.perf_counter() - t0
    return {"value": px / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": f"all {len(imgs)} images of the batch, one image per task"}


def bench_batched(torch, ccl, hbm_gbs):
    """256 images with H, W uniform in [64, 2048], density uniform in
    [0.2, 0.8] (half Bernoulli, half sigma=4 smoothed noise), 8-connectivity:
    one ccl_label_batched call (autotuned block shape, graph replay) against
    256 ccl_label calls on one stream.  Inputs 0.29 GB and outputs 1.1 GB
    exceed L2, so repetitions do not hit a warm cache."""
    from paper_1712_09789_gb300 import synth

    imgs = synth.batch_uneven(256, seed=0)
    pairs = [(torch.from_numpy(im).cuda(), torch.empty(im.shape, dtype=torch.int32, device="cuda"))
             for im in imgs]
    px = sum(im.size for im in imgs)
    tile = ccl.ccl_autotune_batched(pairs, 8)
    reps = 10

    def timed(fn):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    def batched():
        ccl.ccl_label_batched(pairs, 8)

    def plain():
        for img, lab in pairs:
            ccl.ccl_label(img, 8, labels=lab)

    ms_b = timed(batched)
    ms_p = timed(plain)
    # the same 256 plain calls captured once into a CUDA graph (caller-owned
    # scratch, so the capture allocates nothing): launch cost off the host
    ws = torch.empty(max(ccl.ccl_workspace_size(*im.shape) for im in imgs), dtype=torch.uint8, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for img, lab in pairs:
            ccl.ccl_label_ws(img, ws, 8, labels=lab)
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        for img, lab in pairs:
            ccl.ccl_label_ws(img, ws, 8, labels=lab)
    ms_pg = timed(graph.replay)
    status = ccl.ccl_get_device_status()
    res = {"workload": "256 images, H,W ~ U[64,2048], density ~ U[0.2,0.8], 8-connectivity",
           "pixels": px, "tile": ccl.ccl_tile_names()[tile],
           "batched_ms": ms_b, "batched_gpixel_s": px / (ms_b / 1e3) / 1e9,
           "plain_ms": ms_p, "plain_gpixel_s": px / (ms_p / 1e3) / 1e9,
           "plain_graph_ms": ms_pg, "plain_graph_gpixel_s": px / (ms_pg / 1e3) / 1e9,
           "batched_hbm_roofline_frac": px * BYTES_PER_PIXEL / (ms_b / 1e3) / (hbm_gbs * 1e9),
           "device_status": ccl.ccl_status_string(status)}
    return res


def bench_variants(torch, ccl):
    """Sec. 4.2's comparison of the coarse-to-fine strategy on random noise:
    C2FL (the method), RC2FL (coarse labelling along rows only), CC2FL (along
    columns only) and NC2FL (none).  Per variant: the median time of the three
    kernels (CUDA events, 5 runs after 2 warm-ups) and the step-1 counters
    (merges, root-walk steps, CAS attempts) per Mpixel; (a) sizes 256^2 to
    4096^2 at density 0.5, 4-connectivity (the paper's), (b) densities 0.1 to
    0.9 at 2048^2, both connectivities.  Every variant's labels are checked
    equal to C2FL's."""
    from paper_1712_09789_gb300 import synth

    names = ccl.VARIANTS

    def one(img, conn):
        d = torch.from_numpy(img).cuda()
        ref = ccl.ccl_label_variant(d, conn, 0)
        row = {}
        for v, name in enumerate(names):
            out = torch.empty_like(ref)
            for _ in range(2):
                ccl.ccl_label_variant(d, conn, v, labels=out)
            ts = []
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ccl.ccl_label_variant(d, conn, v, labels=out)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b) * 1e3)
            _, cnt = ccl.ccl_label_variant(d, conn, v, labels=out, counters=True)
            mpx = img.size / 1e6
            row[name] = {"us": sorted(ts)[2], "merges_per_mpx": cnt["merges"] / mpx,
                         "find_steps_per_mpx": cnt["find_steps"] / mpx, "atomics_per_mpx": cnt["atomics"] / mpx,
                         "same_labels": bool(torch.equal(out, ref))}
        return row

    res = {"workload": "Bernoulli noise; (a) side 256..4096 at p=0.5, 4-conn; (b) p=0.1..0.9 at 2048^2, 4/8-conn",
           "sizes": {}, "densities": {}}
    for side in (256, 1024, 4096):
        res["sizes"][str(side)] = one(synth.bernoulli(side, side, 0.5, 0), 4)
    for conn in (4, 8):
        for p in (0.1, 0.3, 0.5, 0.7, 0.9):
            res["densities"][f"conn{conn}_p{p}"] = one(synth.bernoulli(2048, 2048, p, 0), conn)
    return res


def bench_stats(torch, ccl):
    """Component statistics (area, bounding box, coordinate sums) of the
    8192x8192 Bernoulli(0.5) labels, both connectivities: one synchronous
    ccl_component_stats call per repetition with the records left on the
    device; median of 5 after 2 warm-ups (host clock around the call, which
    returns after its stream has finished)."""
    import ctypes

    from paper_1712_09789_gb300 import synth

    lib = ccl.load()
    img = torch.from_numpy(synth.bernoulli(8192, 8192, 0.5, 0)).cuda()
    res = {"workload": "8192x8192 Bernoulli p=0.5 seed 0 labels"}
    # DRAM bytes per pixel of a call (ncu) from
    # profiles/k_stats_8192_bernoulli.md while the sources match
    rec = recorded_figures("k_stats_8192_bernoulli.md", ("ccl_block.cuh", "ccl_internal.h", "ccl_stats.cu")) or {}
    for conn in (8, 4):
        lab = ccl.ccl_label(img, conn)
        n = ctypes.c_int(0)
        sp = torch.cuda.current_stream().cuda_stream
        lib.ccl_component_stats(lab.data_ptr(), 8192, 8192, None, 0, ctypes.byref(n), sp)
        buf = torch.empty(max(1, n.value) * 40, dtype=torch.uint8, device="cuda")
        ts = []
        for i in range(7):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = lib.ccl_component_stats(lab.data_ptr(), 8192, 8192, buf.data_ptr(), n.value, ctypes.byref(n), sp)
            t1 = time.perf_counter()
            if st != ccl.CCL_OK:
                raise RuntimeError(f"ccl_component_stats: {ccl.ccl_status_string(st)}")
            if i >= 2:
                ts.append((t1 - t0) * 1e3)
        ms = sorted(ts)[2]
        res[f"conn{conn}"] = {"components": n.value, "ms": ms, "gpixel_s": 8192 * 8192 / (ms / 1e3) / 1e9,
                              "ncu_dram_bytes_per_pixel": rec.get(f"dram_bytes_per_pixel_conn{conn}")}
    return res


def bench_strips(torch, ccl):
    """Strip sharding emulated on one GPU: the 8192x8192 Bernoulli(0.5) image,
    8-connectivity, cut into G strips that are labelled separately and joined
    at their seams (ccl_strip_begin per strip, edge rows to the host,
    ccl_strip_resolve, the seam map back, ccl_strip_finish per strip).  Host
    clock around each part with the stream synchronised, median of 7 after 2
    warm-ups; G = 1 is one plain ccl_label call for comparison.  On G GPUs
    each would run one strip's begin and finish; that is not measured here."""
    import numpy as np

    from paper_1712_09789_gb300 import strips, synth

    N = 8192
    img = torch.from_numpy(synth.bernoulli(N, N, 0.5, 0)).cuda()
    labels = torch.empty((N, N), dtype=torch.int32, device="cuda")
    res = {"workload": "8192x8192 Bernoulli p=0.5 seed 0, 8-connectivity, strips on one GPU"}

    def med(xs):
        return sorted(xs)[len(xs) // 2]

    ts = []
    for i in range(9):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ccl.ccl_label(img, 8, labels=labels)
        torch.cuda.synchronize()
        if i >= 2:
            ts.append((time.perf_counter() - t0) * 1e3)
    res["G1_plain_ms"] = med(ts)
    want = labels.clone()
    for G in (2, 4, 8):
        bounds = strips.strip_bounds(N, G)
        wss = [torch.empty(ccl.ccl_workspace_size(h, N, 8), dtype=torch.uint8, device="cuda") for _, h in bounds]
        parts = {"begin": [], "exchange_resolve": [], "finish": [], "total": []}
        pairs = None
        for i in range(9):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            edges = [ccl.ccl_strip_begin(img[y0:y0 + h], y0, N, ws, 8) for (y0, h), ws in zip(bounds, wss)]
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            pairs = ccl.ccl_strip_resolve(torch.stack(edges).cpu().numpy(), 8)
            seam = torch.from_numpy(pairs.view(np.int32)).cuda() if len(pairs) else None
            t2 = time.perf_counter()
            for (y0, h), ws in zip(bounds, wss):
                ccl.ccl_strip_finish(h, N, y0, N, seam, ws, 8, labels[y0:y0 + h])
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            if i >= 2:
                parts["begin"].append((t1 - t0) * 1e3)
                parts["exchange_resolve"].append((t2 - t1) * 1e3)
                parts["finish"].append((t3 - t2) * 1e3)
                parts["total"].append((t3 - t0) * 1e3)
        status = ccl.ccl_get_device_status()
        res[f"G{G}"] = {**{f"{k}_ms": med(v) for k, v in parts.items()}, "seam_pairs": int(len(pairs)),
                        "same_labels_as_plain": bool(torch.equal(labels, want)),
                        "device_status": ccl.ccl_status_string(status)}
    return res


def bench_volume(torch, ccl, hbm_gbs):
    """3D labelling (ccl_label_3d) of 512^3 Bernoulli volumes, seed 0: p = 0.3
    (near the 6-connected percolation threshold) and 0.5, both
    connectivities.  CUDA events around each call on its stream, median of 10
    after 3 warm-ups; the volume (134 MB) and labels (537 MB) are larger than
    L2.  Roofline: 1 B read + 4 B written per voxel against the measured copy
    bandwidth."""
    from paper_1712_09789_gb300 import synth

    res = {"workload": "512x512x512 Bernoulli volumes, seed 0", "bytes_per_voxel": BYTES_PER_PIXEL, "runs": {}}
    # DRAM bytes per voxel of the three kernels (ncu, 384^3 of the same
    # recipe) from profiles/k_vol_512_bernoulli.md while the sources match
    rec = recorded_figures("k_vol_512_bernoulli.md", ("ccl_block.cuh", "ccl_internal.h", "ccl_volume.cu"))
    n = 512 ** 3
    for p in (0.3, 0.5):
        d = torch.from_numpy(synth.bernoulli3d(512, 512, 512, p, 0)).cuda()
        out = torch.empty((512, 512, 512), dtype=torch.int32, device="cuda")
        for conn in (6, 26):
            for _ in range(3):
                ccl.ccl_label_3d(d, conn, labels=out)
            ts = []
            for _ in range(10):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ccl.ccl_label_3d(d, conn, labels=out)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            if ccl.ccl_get_device_status() != ccl.CCL_OK:
                raise RuntimeError("volume labelling reported a device error")
            ms = sorted(ts)[len(ts) // 2]
            gvx = n / (ms / 1e3) / 1e9
            res["runs"][f"p{p}_conn{conn}"] = {
                "ms": ms, "min_ms": min(ts), "gvoxel_s": gvx,
                "hbm_roofline_frac": gvx * 1e9 * BYTES_PER_PIXEL / (hbm_gbs * 1e9),
                "components": int(torch.unique(out).numel() - 1) if p == 0.3 else None,
                "ncu_dram_bytes_per_voxel_384": (rec or {}).get(f"dram_bytes_per_voxel_p{p}_conn{conn}")}
        del d, out
        torch.cuda.empty_cache()
    return res


def bench_serving(torch, ccl, seconds, rates=(2000, 5000, 10000), warm=0.5):
    """Serving stream: Poisson arrivals (exponential gaps, seeded per rate) of
    frames 640x480 (50%), 1920x1080 (35%), 3840x2160 (15%), sigma=6 smoothed
    noise at density 0.3..0.6 whose blobs move 1-4 px per frame, 8-connectivity,
    submitted from pinned host memory to ``CclServer`` (copies in both
    directions are part of every request).  Frames are generated before the
    clock starts.  After `warm` seconds the server's statistics are reset;
    p50/p99/max are submit -> labels in host memory, Gpixel/s is delivered
    pixels over the span from the first counted submission to the last
    completion."""
    from paper_1712_09789_gb300 import synth

    frames = synth.serving_frames(128, n_streams=4, seed=0)
    host = [torch.from_numpy(f).pin_memory() for f in frames]
    outs = [torch.empty(f.shape, dtype=torch.int32).pin_memory() for f in frames]
    hv = [h.numpy() for h in host]
    ov = [o.numpy() for o in outs]
    mean_px = sum(f.size for f in frames) / len(frames)
    res = {"workload": "Poisson arrivals of 640x480/1920x1080/3840x2160 frames (50/35/15%), smoothed noise "
                       "sigma=6 density 0.3-0.6, 8-connectivity, host frames in pinned memory",
           "seconds_per_rate": seconds, "pool_frames": len(frames), "mean_frame_px": mean_px, "rates": {}}
    with ccl.CclServer(max_slots=64, n_streams=4, max_batch=32, hbm_budget_bytes=8 << 30) as srv:
        for i in range(len(frames)):       # warm the server, its graphs and the autotuner
            srv.wait(srv.submit(hv[i], ov[i], 8))
        for _ in range(3):                 # and bursts, so that full batches have run on every stream
            for t in [srv.submit(hv[i], ov[i], 8) for i in range(len(frames))]:
                srv.wait(t)
        for rate in rates:
            arr = synth.poisson_arrivals(rate, warm + seconds, seed=rate)
            owner = [None] * len(frames)
            t0 = time.perf_counter()
            reset = False
            late = 0
            for i, ta in enumerate(arr):
                if not reset and ta >= warm:
                    srv.reset_stats()
                    reset = True
                while True:
                    now = time.perf_counter() - t0
                    if now >= ta:
                        break
                    if ta - now > 2e-4:
                        time.sleep(ta - now - 1e-4)
                if now - ta > 1e-3:
                    late += 1
                j = i % len(frames)
                if owner[j] is not None:
                    srv.wait(owner[j])     # the buffer's previous request is still out
                owner[j] = srv.submit(hv[j], ov[j], 8)
            for tk in owner:
                if tk is not None:
                    srv.wait(tk)
            st = srv.stats()
            res["rates"][str(rate)] = {
                "offered_gpixel_s": rate * mean_px / 1e9, "requests": int(st["completed"]),
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "mean_ms": st["mean_ms"],
                "delivered_gpixel_s": st["gpixel_s"], "rejected": int(st["rejected"]),
                "late_submissions": late,
                "stages_ms": {k: [st[f"{k}_p50_ms"], st[f"{k}_p99_ms"]] for k in ("queue", "h2d", "label", "d2h")},
                "batches": int(st["batches"]), "multi_request_batches": int(st["multi_request_batches"]),
                "overlapped_batches": int(st["overlapped_batches"]),
                "max_batch_requests": int(st["max_batch_requests"]),
                "max_batches_in_flight": int(st["max_batches_in_flight"])}
    return res


def bench_e2e(torch, ccl, img_np, args, world, max_over_ranks, n_streams=3):
    """The headline step end to end through ``ccl_label_host_async``: every
    labeling copies its image from pinned host memory to the device, labels
    it and copies the labels back to pinned host memory, on three streams in
    turn so that one image's copies overlap another's labelling.  The timed
    region ends when every stream has finished (host clock)."""
    pin_in = [torch.from_numpy(img_np).pin_memory().numpy() for _ in range(HEAD_COPIES)]
    pin_out = [torch.empty((HEAD_N, HEAD_N), dtype=torch.int32).pin_memory().numpy() for _ in range(n_streams)]
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    steps = max(1, min(3, args.steps))

    def step():
        for k in range(HEAD_PER_STEP):
            si = k % n_streams
            ccl.ccl_label_host_async(pin_in[k % HEAD_COPIES], pin_out[si], HEAD_CONN, stream=streams[si])

    step()  # warm-up: grows the library's staging buffers of each stream
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    for st in streams:
        st.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0)
    status = ccl.ccl_get_device_status()
    for st in streams:
        ccl.ccl_release_stream(st)
    if status != ccl.CCL_OK:
        raise RuntimeError(f"e2e: device status {ccl.ccl_status_string(status)}")
    px = HEAD_PER_STEP * HEAD_N * HEAD_N
    h2d = HEAD_PER_STEP * HEAD_N * HEAD_N
    d2h = HEAD_PER_STEP * HEAD_N * HEAD_N * 4
    return {"value": world * px * steps / dt / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "host_link_gbs": (h2d + d2h) * steps / dt / 1e9,
            "api": f"ccl_label_host_async on {n_streams} streams (pinned host buffers, copies in both "
                   f"directions inside the timed region)"}


def bench_cpu(img_np, gpu_labels, budget=12.0):
    """The CPU oracle, single thread, on the headline image: repeated until
    `budget` seconds of labelling; its first result is compared with the
    GPU's labels of the same image."""
    import numpy as np

    import oracle

    oracle.build()
    n, t_total, want = 0, 0.0, None
    while t_total < budget or n == 0:
        t0 = time.perf_counter()
        r = oracle.label(img_np, HEAD_CONN)
        t_total += time.perf_counter() - t0
        if want is None:
            want = r
        n += 1
    same = bool(np.array_equal(gpu_labels.cpu().numpy(), want))
    return {"value": n * img_np.size / t_total / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} labelings of the 8192x8192 Bernoulli(0.5) image, 8-connectivity, single thread "
                      f"({t_total:.1f} s)",
            **host_cpu(), "parity_bit_exact": same}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--only-extra", default="", help="comma-separated names of the extras to run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serving-seconds", type=float, default=3.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
