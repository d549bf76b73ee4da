#!/usr/bin/env python
"""Benchmark of the WSM hot path on GB300.

Workload (one step): 8 seeded 512x512 RGB images (noise amplitude swept
0..24, 18k..229k unique colors each), K = 256, fixed-iteration WSM
(10 iterations): for every image reduce -> init -> iterate -> map -> MSE.

  value   unique-color assignments per second (sum over the images of
          N' x iterations, divided by the step time), inputs resident in HBM;
  e2e     the same metric through the public API from pinned host buffers,
          with the host->device copy of the pixels and the device->host copy
          of the index image, palette and MSE inside the timed region;
  roofline  the persistent sort-means kernel (dominant): evaluated distances x
          8 FLOP per launch over its CUDA-event duration, against the FP32
          CUDA-core peak (SMs x 128 lanes x 2 FLOP x max SM clock);
  roofline_hbm  the HBM-bound kernels -- unique colors (a1), index images
          (a7), per-pixel MSE (a8) -- on 4 images of 4096x4096, each stage
          timed alone after the timed region: algorithmic bytes (3N + 8N',
          3N + N + N', 4N) over the mean CUDA-event time, against the
          measured HBM copy bandwidth;
  value_sustained  the step repeated back to back for about 2 s, with its
          own clock record;
  cpu_baseline  the CPU oracle on a bounded sample of the same workload
          (single thread; cpu_baseline_all_cores: one process per core).
The persistent kernel's launch shape comes from the library's autotuner,
run on the same images before the graphs are captured (untimed).

``--impl reference`` times the CPU oracle instead (the reference arm).
``--form batch`` times the batched form instead: 64 seeded images with sides
log-uniform in [256, 2048], K = 256, WSM 10 iterations, the whole path as one
replay of a captured CUDA graph (launch shape from the autotuner), against
64 sequential runs of the one-image path on the same images.
``--form serve`` drives the native serving loop instead: Poisson arrivals of
requests drawn from 48 seeded images with sides log-uniform in [128, 4096]
and K in {16, 64, 256}; p50/p99 latency and images/s over 10k requests.
``--form stability`` reports the stability statistic of Table 4,
100 (1 - sigma / mu) of the MSE over 100 seeds, for WSM and WSM-C on the 8
sweep images at K in {32, 64, 128, 256}.
``--form hbm`` times the HBM-bound steps on 4 images of 4096x4096: the
unique-color reduction, the pixel mapping and the per-pixel MSE of the
index images, each against the measured HBM peak (the final assignment and
the pipeline's MSE from it are timed beside them).
``--form wide`` times the iterations at K = 256, 512 and 1024 (16-bit
memberships above 256) on the 8 sweep images.
``--form grad`` times the differentiable form instead: forward + backward of
the weighted distortion D(C, X) of a 512x512 image's pixels at K = 64, and
200 Adam steps of palette refinement from the WSM palette.
Multi-GPU (torchrun): every rank quantizes its own 8 images (weak scaling,
no collective on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

K_PALETTE = 256
ITERS = 10
N_IMAGES = 8
H = W = 512
METRIC = "unique-color assignments/s per iter (K=256) vs FP32 peak; 512² images/s end-to-end"
WORKLOAD = "sweep 8x512x512 noise 0..24 (per GPU), K=256, WSM 10 iterations"
UNIT = "assignments/s"
L2_FLUSH_BYTES = 256 << 20
# per step, all images together: hist24, scan_count, scan_emit (up to 16 images
# per launch), init, the plan kernel (which also clears the launch's counters)
# and the sort-means launch (which also writes N' and the iteration counts) for
# the iterations, the plan kernel, the map-mode sort-means launch (which also
# sums the squared errors), the gather and the MSE kernel (up to 64 images per
# launch)
KERNELS_PER_STEP = 10


def workload(rank: int):
    """The rank's 8 images: seeds 1..8 (+8*rank), noise 0..24."""
    return [synth.image(H, W, 8 * rank + s + 1, a) for s, a in enumerate(synth.SWEEP_NOISE)]


def image_seed(rank: int, s: int) -> int:
    return 1000 * (8 * rank + s) + K_PALETTE


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def combine_ranks(total_ms: float, e2e_ms: float, units: float, device):
    """Whole-job figures of the replicas: the slowest rank's device and
    end-to-end times (max over ranks) and the units all ranks processed
    (sum).  Each rank quantizes its own images; this is the only exchange."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(u[0])


def profiled_traffic():
    """DRAM bytes (read + write) of one iterate launch from the committed ncu
    summary, or None if the kernel sources changed since that capture."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(root, "paper_1011_0093_gb300", "csrc")
    try:
        text = open(os.path.join(root, "profiles", "k_sortmeans_sweep8x512_K256.md")).read()
        src = b"".join(open(os.path.join(csrc, f), "rb").read()
                       for f in ("wsm_iterate.cu", "wsm_internal.cuh", "wsm_split.h"))
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines()
                  if line.startswith(("traffic_bytes_per_launch: ", "source_sha256: ")))
    if fields.get("source_sha256", "").strip() != hashlib.sha256(src).hexdigest():
        return None
    return int(fields["traffic_bytes_per_launch"])


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median and maximum SM clock and the throttle reasons seen active
        in `nvidia-smi --format=csv,noheader,nounits` lines of FIELDS."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm and CPU baseline: the CPU oracle
# ---------------------------------------------------------------------------

def oracle_sample(images, budget_s: float, start: int = 0):
    """Run the oracle on whole images (cycling) until budget_s has elapsed."""
    import oracle
    oracle.build()
    units, t0, n, s = 0, time.perf_counter(), 0, start
    while True:
        r = oracle.quantize(images[s % len(images)], K_PALETTE, image_seed(0, s % len(images)),
                            ITERS, 0.0)
        units += len(r["colors"]) * r["iters"]
        n += 1
        s += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            return units, el, n


def _oracle_worker(job):
    images, budget_s, start = job
    return oracle_sample(images, budget_s, start)


def oracle_parallel(images, budget_s: float):
    """One oracle process per core available to this process, each on whole
    images (different starting images) for budget_s: the sum of the
    processes' rates (they run at the same time), and the core count."""
    import multiprocessing as mp
    procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(images, budget_s, q) for q in range(procs)])
    return sum(u / t for u, t, _ in res), procs, sum(n for _, _, n in res)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    images = workload(0)
    oracle_sample(images, 0.0)                     # build + first touch
    for w in range(args.warmup):
        oracle_sample(images, 0.0, start=w)
    units, secs, nimg = 0, 0.0, 0
    for k in range(args.steps):
        u, t, n = oracle_sample(images, 0.0, start=k)   # one image per step
        units, secs, nimg = units + u, secs + t, nimg + n
    value = units / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{nimg} whole images of the workload, one per step, cycling "
                                   "through its 8 images, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    world, rank, local = dist_env()
    # the HBM workload's images are generated while the GPU runs the step
    hbm_pool = hbm_pending = None
    if rank == 0 and world == 1 and not args.no_hbm:
        hbm_pool, hbm_pending = hbm_images_async()            # spawned, before any CUDA call
    import torch
    import torch.distributed as dist

    import paper_1011_0093_gb300 as wsm
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    images = workload(rank)
    n = H * W
    h_imgs = [torch.from_numpy(im).pin_memory() for im in images]
    seeds = [image_seed(rank, s) for s in range(len(images))]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    plan = wsm.BatchPlan([im.shape for im in images], K_PALETTE, seeds, max_iter=ITERS)
    plan.load(h_imgs)
    # the iterations, once on their own, for the roofline (the same every step:
    # same inputs): the distances Algorithm 2's visits evaluate (the work
    # counted per unit), then the distances the launch computes with the
    # first pass started at the grid candidates (the default)
    wsm.wsm_set_first_pass_start(plan.handle, False)
    plan.run(wsm.STAGE_REDUCE | wsm.STAGE_INIT | wsm.STAGE_ITERATE)
    evaluated, _ = plan.stats()
    wsm.wsm_set_first_pass_start(plan.handle, True)
    # the launch shape of the persistent kernel, picked by the library's
    # autotuner on these images (untimed)
    if args.launch_shape >= 0:
        # a fixed shape (profiling runs: under a profiler the autotuner's
        # event timings include the profiler's own cost per launch)
        wsm.wsm_set_launch_shape(plan.handle, args.launch_shape)
        plan.weigh()
        best_shape, shape_ms = args.launch_shape, None
    else:
        best_shape, shape_ms = plan.tune(repeats=3)
    shape = wsm.wsm_launch_shape(plan.handle, best_shape)[1:3]
    plan.run(wsm.STAGE_REDUCE | wsm.STAGE_INIT | wsm.STAGE_ITERATE)
    executed, _ = plan.stats()
    # one step = three captured graphs replayed back to back: unique colors +
    # init, the iterations (one persistent launch over the 8 images), final
    # assignment + mapping + MSE; events between them
    # time the iterations inside the timed region
    parts = (wsm.STAGE_REDUCE | wsm.STAGE_INIT, wsm.STAGE_ITERATE,
             wsm.STAGE_MAP | wsm.STAGE_INDEX | wsm.STAGE_DISTORTION)
    plan.capture(parts)
    it_events = []

    def step(record: bool):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record else None
        if record:
            e[0].record(stream)
        plan.replay(0)
        if record:
            e[1].record(stream)
        plan.replay(1)
        if record:
            e[2].record(stream)
        plan.replay(2)
        if record:
            e[3].record(stream)
            it_events.append(e)

    for _ in range(args.warmup):
        step(False)
    plan.sync()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1)                                   # evict L2 between steps
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(True)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    barrier()
    plan.sync()
    n_unique = [int(v) for v in plan.n_unique.cpu()]
    units_step = sum(n_unique) * ITERS
    total_ms = sum(step_ms)

    # e2e through the public API from pinned host memory: pixels up, then the
    # same replay, then index images, palettes and MSE down (one copy per
    # field for all images: BatchPlan keeps each field in one buffer)
    e2e_ms = []
    h_packed = plan.pack(images)
    out = plan.host_outputs()
    h2d = h_packed.numel()
    d2h = sum(t.numel() * t.element_size() for t in out.values())

    def e2e_step():
        plan.load(h_packed)
        plan.replay()
        plan.fetch(out)

    for _ in range(max(args.warmup, 1)):
        e2e_step()
    barrier()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    barrier()
    clk = clocks.stop()
    plan.sync()

    # sustained: the same step back to back for about 2 s (L2 flushed between
    # steps, events around each, one synchronisation at the end), with its own
    # clock record
    n_sus = max(args.steps, int(2000.0 / max(statistics.median(step_ms), 1e-3)))
    sus_clocks = ClockSampler(local)
    sus_clocks.start()
    barrier()
    sus_ev = []
    for _ in range(n_sus):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(False)
        b.record(stream)
        sus_ev.append((a, b))
    barrier()
    sus_clk = sus_clocks.stop()
    sus_ms = sum(a.elapsed_time(b) for a, b in sus_ev)

    # roofline of the persistent sort-means kernel, from the timed steps
    it_ms = [e[1].elapsed_time(e[2]) for e in it_events]
    graph_ms = {name: statistics.median(e[q].elapsed_time(e[q + 1]) for e in it_events)
                for q, name in enumerate(("unique colors + init", "iterations",
                                          "final assignment + mapping + MSE"))}
    achieved_tflops = 8.0 * sum(evaluated) * len(it_ms) / (sum(it_ms) * 1e-3) / 1e12
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    fp32_measured = wsm.wsm_measure_fp32(plan.handle)     # after the timed region

    total_ms, e2e_total, all_units = combine_ranks(total_ms, sum(e2e_ms), units_step, dev)
    value = all_units * args.steps / (total_ms * 1e-3)
    e2e_value = all_units * args.steps / (e2e_total * 1e-3)
    sus_total, _, _ = combine_ranks(sus_ms, 0.0, units_step, dev)
    value_sustained = all_units * n_sus / (sus_total * 1e-3)

    # the HBM-bound kernels (a1, a7, a8) on large images, after the timed region
    roof_hbm = None
    if hbm_pending is not None:
        hbm_imgs = hbm_pending.get()
        hbm_pool.close()
        roof_hbm = roofline_hbm(*hbm_stages(hbm_imgs, 10, 3))
        del hbm_imgs

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        u, secs, nimg = oracle_sample(images, args.cpu_seconds)
        cpu = {"value": u / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nimg} whole 512x512 images of the same sweep (K=256, 10 iterations),"
                         f" single thread, {secs:.1f} s"}
        rate, procs, nimg_all = oracle_parallel(images, args.cpu_seconds)
        cpu_all = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": f"{procs} processes, one per core, {nimg_all} whole images in all, "
                             f"about {args.cpu_seconds:.0f} s each; the sum of their rates"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "unique_colors": n_unique,
                       "images_per_step": len(images) * world,
                       "images_per_s": len(images) * world * args.steps / (total_ms * 1e-3),
                       "images_per_s_e2e": len(images) * world * args.steps / (e2e_total * 1e-3),
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"replicas x{world}",
                       "graph_ms_median": graph_ms,
                       "launch_shape": {"threads": shape[0], "blocks_per_sm": shape[1],
                                        "autotune_iterate_ms": shape_ms}},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "alu", "kernel": "k_sortmeans<iterate> (8 images per launch)",
                         "achieved": achieved_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved_tflops / fp32_peak, "traffic": profiled_traffic(),
                         "peak_kind": f"FP32 {sms} SMs x 128 x 2 x {pk.get('sm_max_mhz')} MHz "
                                      f"({pk_kind} max clock)",
                         "fp32_measured_tflops": fp32_measured,
                         "frac_of_measured_fp32": achieved_tflops / fp32_measured,
                         "launch_ms": sum(it_ms) / len(it_ms),
                         "flop_per_launch": 8.0 * sum(evaluated),
                         "flop_per_launch_executed": 8.0 * sum(executed),
                         "timed": "the iterate graph (plan kernel with the counter clears, "
                                  "persistent launch) between CUDA events in every step"},
            "roofline_hbm": roof_hbm,
            "value_sustained": value_sustained,
            "sustained": {"steps": n_sus, "ms_per_step": sus_total / n_sus, "clocks": sus_clk,
                          "how": "the step back to back for about 2 s, L2 flushed between "
                                 "steps, CUDA events around each step"},
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "clocks": clk,
            "gpu_launches": KERNELS_PER_STEP * args.steps,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def adam_graph(wsm, X, C0, assign, h, lr=0.1):
    """A palette-refinement step (weighted distortion forward, backward, Adam
    with capturable state) captured into a CUDA graph; returns the palette
    parameter (reset to C0, optimizer state fresh), the graph and the
    assignment it warm-starts from."""
    import torch
    Cg = C0.clone().requires_grad_(True)
    opt = torch.optim.Adam([Cg], lr=lr, capturable=True)
    assign_g = assign.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            opt.zero_grad(set_to_none=True)
            wsm.weighted_distortion(X, Cg, assign=assign_g, warm_start=True, handle=h).backward()
            opt.step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    opt.zero_grad(set_to_none=True)
    with torch.cuda.graph(graph):
        wsm.weighted_distortion(X, Cg, assign=assign_g, warm_start=True, handle=h).backward()
        opt.step()
    with torch.no_grad():                       # start again from C0, fresh moments
        Cg.copy_(C0)
        for state in opt.state.values():
            for v in state.values():
                if torch.is_tensor(v):
                    v.zero_()
    return Cg, graph, assign_g


def run_grad(args):
    """Differentiable distortion, forward + backward (dD/dC and dD/dX) per step."""
    import torch

    import paper_1011_0093_gb300 as wsm

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    Kg = 64
    img = synth.image(512, 512, 41, 6)
    n = img.shape[0] * img.shape[1]
    q = wsm.quantize(torch.from_numpy(img).to(dev), Kg, 5, max_iter=ITERS, eps=0.0)
    C0 = q.centers[:, :3].contiguous()
    x_host = torch.from_numpy(img.reshape(-1, 3).astype(np.float32)).pin_memory()
    X = x_host.to(dev)
    h = wsm.Handle(Kg, 1, 1)
    assign = torch.empty(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step(X_in, C_in, warm):
        Xg = X_in.detach().requires_grad_(True)
        Cg = C_in.detach().requires_grad_(True)
        D = wsm.weighted_distortion(Xg, Cg, assign=assign, warm_start=warm, handle=h)
        D.backward()
        return D, Cg.grad, Xg.grad

    step(X, C0, False)
    for _ in range(args.warmup):
        step(X, C0, True)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(X, C0, True)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    # the same through the public API from pinned host memory: the points go
    # up, D and dD/dC come back every step
    e2e = []
    out_c = torch.empty((Kg, 3), dtype=torch.float32).pin_memory()
    out_d = torch.empty(1, dtype=torch.float32).pin_memory()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Xd = x_host.to(dev, non_blocking=True)
        D, gC, _ = step(Xd, C0, True)
        out_c.copy_(gC, non_blocking=True)
        out_d.copy_(D.detach().reshape(1), non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e.append(a.elapsed_time(b))
    # per-kernel view: forward call (rows + search + sums) and backward kernel
    fwd_ms, bwd_ms = [], []
    D = torch.empty(1, dtype=torch.float32, device=dev)
    resid = torch.empty((Kg, 4), dtype=torch.float32, device=dev)
    gD = torch.ones(1, dtype=torch.float32, device=dev)
    gC = torch.empty_like(C0)
    gX = torch.empty_like(X)
    for _ in range(args.steps):
        flush.fill_(1)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        wsm.wsm_distortion_fwd(h, X, None, C0, assign, True, D, resid)
        e[1].record(stream)
        wsm.wsm_distortion_bwd(h, X, None, C0, assign, resid, gD, gC, gX)
        e[2].record(stream)
        e[2].synchronize()
        fwd_ms.append(e[0].elapsed_time(e[1]))
        bwd_ms.append(e[1].elapsed_time(e[2]))
    # 200 Adam steps from the WSM palette, assignment carried as warm start
    # (after a few steps of a throwaway copy: the optimizer's first use loads
    # its kernels)
    Cw = C0.clone().requires_grad_(True)
    opt_w = torch.optim.Adam([Cw], lr=0.1)
    for _ in range(3):
        opt_w.zero_grad()
        wsm.weighted_distortion(X, Cw, assign=assign, warm_start=True, handle=h).backward()
        opt_w.step()
    Cp = C0.clone().requires_grad_(True)
    opt = torch.optim.Adam([Cp], lr=0.1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d_start = None
    for k in range(200):
        opt.zero_grad()
        Dk = wsm.weighted_distortion(X, Cp, assign=assign, warm_start=True, handle=h)
        Dk.backward()
        if d_start is None:
            d_start = float(Dk.detach())
        opt.step()
    torch.cuda.synchronize()
    adam_ms = (time.perf_counter() - t0) * 1e3
    d_end = float(wsm.weighted_distortion(X, Cp.detach(), assign=assign, warm_start=True,
                                          handle=h))
    # the same 200 steps, each one replay of a captured CUDA graph (forward,
    # backward and a capturable Adam step)
    Cg, graph, assign_g = adam_graph(wsm, X, C0, assign, h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(200):
        graph.replay()
    torch.cuda.synchronize()
    adam_graph_ms = (time.perf_counter() - t0) * 1e3
    d_end_graph = float(wsm.weighted_distortion(X, Cg.detach(), assign=assign_g, warm_start=True,
                                                handle=h))
    clk = clocks.stop()
    wsm.wsm_sync_status(h)

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        Xd64 = img.reshape(-1, 3).astype(np.float64)
        w64 = np.full(n, 1.0 / n)
        C64 = C0.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < min(args.cpu_seconds, 5.0) or reps == 0:
            oracle.distortion_grad(Xd64, w64, C64)
            reps += 1
        secs = time.perf_counter() - t0
        cpu = {"value": reps * n / secs, "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": f"{reps} FP64 forward+gradient passes (exhaustive) over the same "
                         f"{n} points, single thread, {secs:.1f} s"}
    step_ms = statistics.median(ms)
    bwd_bytes = n * (12 + 1 + 12)            # x read, assignment read, dD/dX written
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    bwd_gbs = bwd_bytes / (statistics.median(bwd_ms) * 1e-3) / 1e9
    line = {
        "metric": "differentiable weighted distortion, forward + backward (dD/dC, dD/dX)",
        "form": "grad", "value": n / (step_ms * 1e-3), "unit": "points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "512x512 image (seed 41, noise 6) as float points, w_i = 1/N, "
                               "K=64 palette from 10 WSM iterations, warm-started search",
                   "l2": "flushed between steps (256 MiB write)"},
        "e2e": {"value": n / (statistics.median(e2e) * 1e-3), "unit": "points/s",
                "h2d_bytes_per_step": n * 12, "d2h_bytes_per_step": Kg * 12 + 4},
        "kernels_ms": {"forward_call": statistics.median(fwd_ms),
                       "backward_call": statistics.median(bwd_ms)},
        "roofline": {"bound": "hbm", "kernel": "k_grad_bwd", "achieved": bwd_gbs, "peak": hbm,
                     "unit": "GB/s", "frac": bwd_gbs / hbm, "traffic": None,
                     "peak_kind": pk_kind, "bytes_per_launch": bwd_bytes},
        "adam": {"steps": 200, "lr": 0.1, "ms": adam_ms, "D_start": d_start, "D_end": d_end,
                 "graph_ms": adam_graph_ms, "graph_D_end": d_end_graph},
        "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": 4 * args.steps,
    }
    print(json.dumps(line), flush=True)
    h.close()


BATCH_COUNT = 64
BATCH_SEED = 3


def _batch_image(args):
    q, (h, w) = args
    return synth.image(h, w, 7000 + q, (5 * q) % 25)


def batch_workload():
    """64 images, sides log-uniform in [256, 2048] (seeded), noise 0..24, built
    by a pool of spawned processes (no CUDA state is shared)."""
    import multiprocessing as mp
    sizes = synth.batch_sizes(BATCH_SEED, BATCH_COUNT, 256, 2048)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_batch_image, list(enumerate(sizes)))


def run_batch(args):
    """Batched form: one graph replay per step vs the one-image path."""
    images = batch_workload()                     # before any CUDA call
    import torch

    import paper_1011_0093_gb300 as wsm

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    n_img = len(images)
    seeds = [9000 + q for q in range(n_img)]
    h_imgs = [torch.from_numpy(im).pin_memory() for im in images]
    d_imgs = [t.to(dev) for t in h_imgs]
    plan = wsm.BatchPlan([im.shape for im in images], K_PALETTE, seeds, max_iter=ITERS)
    plan.load(d_imgs)
    # Algorithm 2's distance counts (the work per unit), then the tuned launch
    # with the default first pass (its counts: the distances it computes)
    wsm.wsm_set_first_pass_start(plan.handle, False)
    plan.run(wsm.STAGE_REDUCE | wsm.STAGE_INIT | wsm.STAGE_ITERATE)
    evaluated, _ = plan.stats()
    wsm.wsm_set_first_pass_start(plan.handle, True)
    best, shape_ms = plan.tune(repeats=2)
    executed, _ = plan.stats()
    shapes = [wsm.wsm_launch_shape(plan.handle, q)[1:3] for q in range(len(shape_ms))]
    plan.capture()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        plan.replay()
    plan.sync()
    clocks = ClockSampler(0)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.replay()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    plan.sync()
    # end to end: pixels up from pinned host memory, index images, palettes and
    # MSE back (one copy per field for all images), around the same replay
    h_packed = plan.pack(images)
    out = plan.host_outputs()
    e2e = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.load(h_packed)
        plan.replay()
        plan.fetch(out)
        b.record(stream)
        b.synchronize()
        e2e.append(a.elapsed_time(b))
    clk = clocks.stop()
    plan.sync()
    # the one-image path, image after image, on the same device-resident inputs
    h1 = wsm.Handle(K_PALETTE, max(im.shape[0] * im.shape[1] for im in images))
    seq = []
    same = True
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = [wsm.quantize(d_imgs[q], K_PALETTE, seeds[q], max_iter=ITERS, handle=h1)
                for q in range(n_img)]
        torch.cuda.synchronize()
        seq.append((time.perf_counter() - t0) * 1e3)
    for q, o in enumerate(outs):
        r = plan.result(q)
        same &= (torch.equal(o.centers, r["centers"]) and torch.equal(o.index, r["index"])
                 and o.mse == r["mse"] and o.iters == r["iters"])
    n_unique = [plan.result(q)["n_unique"] for q in range(n_img)]
    step_ms = statistics.median(ms)
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    it_ms = shape_ms[best]
    tflops = 8.0 * sum(evaluated) / (it_ms * 1e-3) / 1e12
    chunks16, chunks48 = -(-n_img // 16), -(-n_img // 48)
    launches = 3 * chunks16 + 1 * chunks48 + 2 * chunks48 + 1 + 3 * chunks48 + 2 * chunks48
    line = {
        "metric": "batched WSM: images/s, 64 images 256^2..2048^2, K=256, one CUDA-graph replay",
        "form": "batch", "value": n_img / (step_ms * 1e-3), "unit": "images/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{n_img} images, sides log-uniform in [256, 2048] (seed "
                               f"{BATCH_SEED}), noise 0..24, K=256, WSM 10 iterations",
                   "pixels": int(sum(im.shape[0] * im.shape[1] for im in images)),
                   "unique_colors_min_max": [min(n_unique), max(n_unique)],
                   "unique_colors_total": int(sum(n_unique)),
                   "l2": "flushed between steps (256 MiB write)"},
        "e2e": {"value": n_img / (statistics.median(e2e) * 1e-3), "unit": "images/s",
                "h2d_bytes_per_step": int(h_packed.numel()),
                "d2h_bytes_per_step": int(sum(t.numel() * t.element_size()
                                              for t in out.values()))},
        "sequential_one_image_path": {"ms": min(seq), "images_per_s": n_img / (min(seq) * 1e-3),
                                      "speedup": min(seq) / step_ms,
                                      "identical_results": bool(same)},
        "autotune": {"chosen": {"threads": shapes[best][0], "blocks_per_sm": shapes[best][1]},
                     "iterate_ms_by_shape": {f"{t}x{b}": m for (t, b), m in zip(shapes, shape_ms)}},
        "roofline": {"bound": "alu", "kernel": "k_sortmeans<iterate> (all launches of the batch)",
                     "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": tflops / fp32_peak, "traffic": None,
                     "peak_kind": "FP32 SMs x 128 x 2 x max SM clock",
                     "flop": 8.0 * sum(evaluated), "flop_executed": 8.0 * sum(executed),
                     "launch_ms": it_ms},
        "cpu_baseline": None, "clocks": clk,
        "gpu_launches": launches * args.steps,
    }
    print(json.dumps(line), flush=True)
    h1.close()


SERVE_BANK = 48


def _serve_image(args):
    q, (h, w) = args
    return synth.image(h, w, 11000 + q, (7 * q) % 25)


def serve_workload():
    """48 images, sides log-uniform in [128, 4096] (seeded), noise 0..24."""
    import multiprocessing as mp
    sizes = synth.batch_sizes(5, SERVE_BANK, 128, 4096)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_serve_image, list(enumerate(sizes)))


def _drive(srv, bank, plan, rate):
    """Submit the planned requests (bank index, K, seed) at Poisson times of
    the given rate (None: all at once) and collect them; per-request latency
    from the server's own clock, and the throughput over the whole run."""
    import threading
    rng = np.random.default_rng(23)
    gaps = rng.exponential(1.0 / rate, len(plan)) if rate else np.zeros(len(plan))
    pending = []
    lock = threading.Condition()

    def submitter():
        t = time.perf_counter()
        for (b, K, seed), g in zip(plan, gaps):
            t += g
            d = t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            p = srv.submit(bank[b], K, seed)
            with lock:
                pending.append(p)
                lock.notify()

    th = threading.Thread(target=submitter)
    th.start()
    lat, first, last = [], None, None
    for i in range(len(plan)):
        with lock:
            while len(pending) <= i:
                lock.wait()
            p = pending[i]
            pending[i] = None
        r = srv.wait(p)
        lat.append(r["latency"])
        first = r["t_submit"] if first is None else min(first, r["t_submit"])
        last = r["t_done"] if last is None else max(last, r["t_done"])
    th.join()
    lat = np.array(lat) * 1e3
    return {"requests": len(plan), "offered_rate": rate, "images_per_s": len(plan) / (last - first),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}


def run_serve(args):
    bank_np = serve_workload()                    # before any CUDA call
    import torch

    import paper_1011_0093_gb300 as wsm

    torch.cuda.set_device(0)
    bank = [torch.from_numpy(im).pin_memory() for im in bank_np]
    rng = np.random.default_rng(19)
    n_req = args.requests

    def plan(n):
        return [(int(rng.integers(0, len(bank))), int(rng.choice([16, 64, 256])),
                 int(rng.integers(0, 1 << 40))) for _ in range(n)]

    with wsm.Server(lanes=args.lanes, slots_per_lane=16, arena_bytes=8 << 30) as srv:
        _drive(srv, bank, plan(2 * SERVE_BANK), None)              # warm-up
        sat = _drive(srv, bank, plan(min(n_req, 2000)), None)      # closed loop: capacity
        clocks = ClockSampler(0)
        clocks.start()
        main = _drive(srv, bank, plan(n_req), 0.8 * sat["images_per_s"])
        clk = clocks.stop()
        sweep = [_drive(srv, bank, plan(min(n_req, 1500)), f * sat["images_per_s"])
                 for f in (0.3, 0.6, 0.95)]
        st = srv.stats()
    px = [im.shape[0] * im.shape[1] for im in bank_np]
    line = {
        "metric": "serving: images/s and p50/p99 latency, Poisson arrivals, images 128^2..4096^2",
        "form": "serve", "value": main["images_per_s"], "unit": "images/s", "n_gpus": 1,
        "steps": n_req, "warmup": 2 * SERVE_BANK, "ms_per_step": main["mean_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{n_req} requests drawn from {len(bank)} seeded images (sides "
                               "log-uniform in [128, 4096], noise 0..24), K in {16, 64, 256}, "
                               "WSM 10 iterations; Poisson arrivals at 0.8x the closed-loop "
                               "capacity", "pixels_min_max": [min(px), max(px)],
                   "lanes": args.lanes, "slots_per_lane": 16, "arena_bytes": 8 << 30},
        "latency_ms": {"p50": main["p50_ms"], "p99": main["p99_ms"], "mean": main["mean_ms"]},
        "capacity_closed_loop": sat, "rate_sweep": sweep,
        "server": st,
        "e2e": {"value": main["images_per_s"], "unit": "images/s",
                "h2d_bytes_per_step": int(np.mean([im.nbytes for im in bank_np])),
                "d2h_bytes_per_step": int(np.mean(px))},
        "cpu_baseline": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_stability(args):
    """Table 4's statistic on the synthetic sweep: 100 seeded runs per image,
    palette size and variant, all runs of one (image, K, variant) in one batch."""
    import torch

    import paper_1011_0093_gb300 as wsm

    torch.cuda.set_device(0)
    images = workload(0)
    runs = args.runs
    h = wsm.Handle(K_PALETTE, H * W, H * W)
    wsm.wsm_reserve_batch(h, runs)
    table = []
    t0 = time.perf_counter()
    for s_img, img in enumerate(images):
        d = torch.from_numpy(img).cuda()
        for K in (32, 64, 128, 256):
            for name, max_iter, eps in (("WSM", 10, 0.0), ("WSM-C", 100, 1e-4)):
                plan = wsm.BatchPlan([img.shape] * runs, K, [7919 * r + 1 for r in range(runs)],
                                     max_iter=max_iter, eps=eps, handle=h)
                plan.load([d] * runs)
                plan.run()
                plan.sync()
                mse = plan.mse.cpu().numpy()
                iters = plan.iters.cpu().numpy()
                mu, sigma = float(mse.mean()), float(mse.std())
                table.append({"image": f"sweep {s_img} (noise {synth.SWEEP_NOISE[s_img]})",
                              "K": K, "variant": name, "mse_mean": mu, "mse_std": sigma,
                              "stability": 100.0 * (1.0 - sigma / mu),
                              "iterations_mean": float(iters.mean())})
    secs = time.perf_counter() - t0
    means = {v: float(np.mean([r["stability"] for r in table if r["variant"] == v]))
             for v in ("WSM", "WSM-C")}
    line = {"metric": "stability 100(1 - sigma/mu) of the MSE over seeded runs (Table 4)",
            "form": "stability", "value": means["WSM-C"], "unit": "percent", "n_gpus": 1,
            "steps": len(table), "warmup": 0, "ms_per_step": 1e3 * secs / len(table),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"8 sweep images 512x512, K in (32, 64, 128, 256), {runs} "
                                   "seeds each, WSM (10 iterations) and WSM-C (1e-4, <= 100)"},
            "mean_stability": means, "table": table}
    print(json.dumps(line), flush=True)
    h.close()


def run_wide(args):
    """Palettes of 256, 512 and 1024 colors on the 8 sweep images: the
    iterations (WSM, 10) of all 8 in one persistent launch, timed with CUDA
    events (L2 flushed before each), with 8-bit memberships at K = 256 and
    16-bit ones (a wide handle) above; Algorithm 2's distance count as the
    work, as in the headline roofline."""
    import torch

    import paper_1011_0093_gb300 as wsm

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    images = workload(0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    pk, _ = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    rows = []
    for K in (256, 512, 1024):
        h = wsm.Handle(K, H * W, H * W)
        plan = wsm.BatchPlan([im.shape for im in images], K, list(range(8)), max_iter=ITERS,
                             handle=h)
        plan.load([torch.from_numpy(im) for im in images])
        wsm.wsm_set_first_pass_start(h, False)
        plan.run(wsm.STAGE_REDUCE | wsm.STAGE_INIT | wsm.STAGE_ITERATE)
        evaluated, _ = plan.stats()
        wsm.wsm_set_first_pass_start(h, True)
        ms = []
        for rep in range(args.warmup + args.steps):
            plan.run(wsm.STAGE_INIT)
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.run(wsm.STAGE_ITERATE)
            b.record(stream)
            b.synchronize()
            if rep >= args.warmup:
                ms.append(a.elapsed_time(b))
        plan.sync()
        t = statistics.median(ms)
        nu = [int(v) for v in plan.n_unique.cpu()]
        tflops = 8.0 * sum(evaluated) / (t * 1e-3) / 1e12
        rows.append({"K": K, "labels": "uint16" if h.wide else "uint8", "iterate_ms": t,
                     "assignments_per_s": sum(nu) * ITERS / (t * 1e-3),
                     "algorithm2_tflops": tflops, "frac_fp32": tflops / fp32_peak})
        h.close()
    line = {"metric": "unique-color assignments/s per iter at K = 256, 512, 1024 (8 sweep "
                      "images, one persistent launch)", "form": "wide",
            "value": rows[-1]["assignments_per_s"], "unit": "assignments/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows[-1]["iterate_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "sweep 8x512x512 noise 0..24, WSM 10 iterations",
                       "l2": "flushed before each timed launch (256 MiB write)"},
            "by_K": rows, "fp32_peak": fp32_peak}
    print(json.dumps(line), flush=True)


HBM_IMAGES = 4
HBM_WORKLOAD = "4 images 4096x4096 (seeds 12000..12003, noise 5, 13, 21, 4), K=256"


def _hbm_image(q):
    return synth.image(4096, 4096, 12000 + q, (8 * q + 5) % 25)


def hbm_images_async():
    """Start generating the HBM workload's images in spawned processes (the
    caller collects them with .get() once it needs them)."""
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(HBM_IMAGES)
    return pool, pool.map_async(_hbm_image, range(HBM_IMAGES))


def hbm_stages(images, steps: int, warmup: int):
    """The HBM-bound stages on the given images, each timed on its own (CUDA
    events around the stage on the launching stream, inputs resident, L2
    flushed before each): unique colors (a1), the final assignment, the index
    images through the color -> label table (a7), the pipeline's MSE from the
    assignment and the per-pixel MSE of Eq. 2 (a8).  Returns per stage the
    mean and median ms and, for a1 / a7 / a8, the algorithmic bytes (the
    per-unit figures: 3N + 8N', 3N + N + N', 4N), GB/s from the mean and the
    fraction of the measured HBM peak; plus N and the N' values."""
    import torch

    import paper_1011_0093_gb300 as wsm

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    n_img = len(images)
    plan = wsm.BatchPlan([im.shape for im in images], K_PALETTE, list(range(n_img)), max_iter=2)
    plan.load([torch.from_numpy(im) for im in images])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stages = {"reduce": wsm.STAGE_REDUCE, "init+iterate": wsm.STAGE_INIT | wsm.STAGE_ITERATE,
              "assign": wsm.STAGE_MAP, "index": wsm.STAGE_INDEX,
              "mse_from_assign": wsm.STAGE_DISTORTION,
              "mse_pixels": None}                # Eq. 2 over the pixels and the index images
    times = {k: [] for k in stages}
    for rep in range(warmup + steps):
        for name, st in stages.items():
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if st is None:
                wsm.wsm_distortion_batch(plan.handle, plan.images, sync=False)
            else:
                plan.run(st)
            b.record(stream)
            b.synchronize()
            if rep >= warmup:
                times[name].append(a.elapsed_time(b))
    plan.sync()
    n_unique = [int(v) for v in plan.n_unique.cpu()]
    N = sum(im.shape[0] * im.shape[1] for im in images)
    NU = sum(n_unique)
    algo = {"reduce": 3 * N + 8 * NU,                     # pixels in, (color, count) out
            "index": 3 * N + N + NU,                      # pixels in, index out, table entries
            "mse_pixels": 4 * N}                          # pixels and index in
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    rows = {}
    for name in stages:
        mean = sum(times[name]) / len(times[name])
        rows[name] = {"ms": statistics.median(times[name]), "ms_mean": mean}
        if name in algo:
            gbs = algo[name] / (mean * 1e-3) / 1e9
            rows[name].update({"algorithmic_bytes": algo[name], "GB/s": gbs, "frac": gbs / hbm})
    del plan
    torch.cuda.empty_cache()
    return rows, N, n_unique, hbm, pk_kind


def roofline_hbm(rows, N, n_unique, hbm, pk_kind):
    """The bench line's record of the HBM-bound kernels (a1, a7, a8)."""
    names = {"reduce": ("a1 unique colors", "k_hist24 + k_scan_count + k_scan_emit", "3N + 8N'"),
             "index": ("a7 index images", "k_pixels_batch<1,0> (gather)", "3N + N + N'"),
             "mse_pixels": ("a8 per-pixel MSE", "k_pixels_batch<0,1> + k_mse_final_batch",
                            "4N")}
    out = {"workload": HBM_WORKLOAD, "pixels": N, "unique_colors": n_unique,
           "bound": "hbm", "peak": hbm, "unit": "GB/s",
           "peak_kind": f"{pk_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
           "timed": "each stage alone between CUDA events on the launching stream, L2 flushed "
                    "(256 MiB write) before each, inputs resident; achieved from the mean"}
    for key, (row, kernels, per_unit) in names.items():
        r = rows[key]
        out[row] = {"kernels": kernels, "algorithmic_bytes": r["algorithmic_bytes"],
                    "bytes_per_unit": per_unit, "ms_mean": r["ms_mean"], "ms_median": r["ms"],
                    "achieved": r["GB/s"], "frac": r["frac"]}
    return out


def run_hbm(args):
    """The HBM-bound stages on 4096x4096 images, each timed on its own (CUDA
    events around the stage, inputs resident, L2 flushed before each)."""
    pool, pending = hbm_images_async()                     # before any CUDA call
    images = pending.get()
    pool.close()
    import torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rows, N, n_unique, hbm, pk_kind = hbm_stages(images, args.steps, args.warmup)
    n_img = len(images)
    line = {"metric": "HBM-bound steps on 4096x4096 images: algorithmic GB/s vs measured HBM peak",
            "form": "hbm", "value": rows["reduce"]["GB/s"], "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows["reduce"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": HBM_WORKLOAD, "images": n_img,
                       "pixels": N, "unique_colors": n_unique,
                       "l2": "flushed before each stage (256 MiB write)"},
            "stages": rows, "peak": hbm, "peak_kind": pk_kind}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wsm", choices=["wsm", "reference"])
    ap.add_argument("--form", default="plain",
                    choices=["plain", "grad", "batch", "serve", "stability", "hbm", "wide"])
    ap.add_argument("--runs", type=int, default=100)
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--lanes", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch-shape", type=int, default=-1,
                    help="fix the persistent kernel's launch shape (index into the library's "
                         "shapes; default: the autotuner picks it)")
    ap.add_argument("--no-hbm", action="store_true",
                    help="skip the HBM-bound stages on 4096x4096 images in the default form")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "grad":
        run_grad(args)
    elif args.form == "batch":
        run_batch(args)
    elif args.form == "serve":
        run_serve(args)
    elif args.form == "stability":
        run_stability(args)
    elif args.form == "hbm":
        run_hbm(args)
    elif args.form == "wide":
        run_wide(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
