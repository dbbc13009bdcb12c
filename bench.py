"""Benchmark of the Köhler contrast-curve path (curve + thresholds) on GB300.

Default line (one GPU): the 5184 x 3456 uint8 Voronoi image (~18 Mpixel, M = 256).
A step is one fused launch of the whole path on one image: the pair-histogram
pass, the exact scans that give |B(t)| and the summed contrast for every t, C(t)
and the ranked local-maximum thresholds.  Inputs are resident in HBM; the
timed steps cycle through a pool of distinct images whose total size exceeds
the L2 cache, so every step reads its image from HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun, one process per GPU) every rank processes its
own images (replicas: weak scaling, no data-path collective); rank 0 prints the
line with the whole-job throughput, timed as the slowest rank.
`--impl reference` times the CPU oracle (the definitional per-threshold loop) on
the host cores instead.

At N = 1 the same line carries "forms": the batched form (one launch over a
96-image uint8 batch, and over 16 uint16 12-bit images with M = 4096) timed
against one launch per image on the same resident images, and the served form
(2000 Poisson-arriving video frames of mixed resolution through the
continuous-batching server: p50/p99 latency, closed-loop frames/s, and one
synchronous host call per frame for comparison), segmentation of the 18-Mpixel
images by their ranked thresholds, and the whole path with the 8- and hexagonal
6-neighbourhoods beside the 4-neighbourhood.  Every form checks its results
against the oracle.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpixel/s of Köhler curve + % HBM roofline; p50/p99 frame latency (served)"
UNIT = "Gpixel/s"
MAX_K = 16
POOL = 12  # distinct 17.9 MB images per rank: 215 MB > 129 MB of L2


# ----------------------------------------------------------------------------- distributed plumbing
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def init_dist(world: int):
    if world <= 1:
        return None
    import torch.distributed as dist

    if not dist.is_initialized():
        dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float) -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 20):
        self.rows = []
        self.t0 = self.t1 = None
        self.proc = None
        self.thread = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", str(period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        inside = [r for t, r in self.rows if self.t0 is not None and self.t0 <= t <= (self.t1 or t)]
        use = inside if inside else [r for _, r in self.rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in use:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(use), "window": "timed region" if inside else "whole run"}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Device sources each profiled kernel is compiled from (its pass and the common
# epilogue); a change to another pass leaves its counters valid.
KERNEL_SOURCES = {"k_u8h": ("kohler_common.cuh", "kohler_u8h.cuh")}


def device_source_digest(kernel: str) -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1707_05062_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, if it was taken on the kernel's current device source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
        digest = device_source_digest(kernel)
    except (OSError, KeyError):
        return None
    traffic = source = None
    for line in text.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1])
        if line.startswith("device_source_sha256_16:"):
            source = line.split(":", 1)[1].strip()
    return traffic if (traffic is not None and source == digest) else None


# ----------------------------------------------------------------------------- CPU baseline (oracle)
def cpu_baseline(img: np.ndarray, M: int, budget_s: float = 12.0):
    """The CPU oracle as it stands (definitional loop over thresholds and N4*
    pairs, OpenMP over thresholds) on a bounded sample of the workload."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    # sample: a band of rows sized from a quick probe so the run stays near budget_s
    probe_rows = max(2, min(img.shape[0], 64))
    t = time.perf_counter()
    card, sumc = oracle.curve(img[:probe_rows], M)
    oracle.thresholds(card, sumc, MAX_K)
    dt = max(time.perf_counter() - t, 1e-6)
    rows = int(min(img.shape[0], max(probe_rows, probe_rows * (budget_s / 3.0) / dt)))
    band = np.ascontiguousarray(img[:rows])
    reps, elapsed = 0, 0.0
    while reps < 3 and (reps == 0 or elapsed < budget_s / 2):
        t = time.perf_counter()
        card, sumc = oracle.curve(band, M)
        oracle.normalise(card, sumc)
        oracle.thresholds(card, sumc, MAX_K)
        elapsed += time.perf_counter() - t
        reps += 1
    px = band.shape[0] * band.shape[1] * reps
    return {"value": px / elapsed / 1e9, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", cores)),
            "kind": "oracle",
            "sample": f"rows 0..{rows - 1} of the {img.shape[1]}x{img.shape[0]} image ({band.size / 1e6:.2f} Mpixel), "
                      f"{reps} run(s), {elapsed:.1f} s: per-threshold loop over N4* pairs + normalisation + thresholds",
            "single_thread": cpu_single_thread(M)}


_SINGLE = r'''
import json, sys, time
sys.path.insert(0, ROOT)
import numpy as np, oracle, synth
oracle.build()
out = {}
for name, img in (("blobs_256", synth.blobs_image()), ("voronoi_18mp_rows_0_47", synth.voronoi_18mp()[:48])):
    img = np.ascontiguousarray(img)
    n, t = 0, time.perf_counter()
    while n == 0 or time.perf_counter() - t < 1.5:
        card, sumc = oracle.curve(img, M)
        oracle.normalise(card, sumc)
        oracle.thresholds(card, sumc, MAX_K)
        n += 1
    dt = (time.perf_counter() - t) / n
    out[name] = {"ms_per_image": dt * 1e3, "gpx_s": img.size / dt / 1e9, "runs": n}
print(json.dumps(out))
'''


def cpu_single_thread(M: int):
    """The oracle on one host thread (a fresh process with OMP_NUM_THREADS=1),
    on the 256x256 image and a 48-row band of the 18-Mpixel image, as the paper's
    single-thread rows are timed."""
    import subprocess

    code = _SINGLE.replace("ROOT", repr(ROOT)).replace("MAX_K", str(MAX_K)).replace("M)", f"{M})")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        res = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal
        return {"error": repr(e)[:200]}
    res["cores"] = 1
    return res


# ----------------------------------------------------------------------------- workloads
def make_pool(rank: int, n: int):
    import synth

    return synth.voronoi_18mp_pool(n, seed=synth.SEEDS["voronoi_18mp"] + 1000 * rank)


def bench_ours(args, rank, local, world, dist):
    import torch

    import paper_1707_05062_gb300 as K
    from paper_1707_05062_gb300 import build as kbuild

    kbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pool_np = make_pool(rank, POOL)
    H, W = pool_np[0].shape
    px = W * H
    pool = [torch.from_numpy(im).to(dev) for im in pool_np]
    stream = torch.cuda.current_stream(dev)
    M = 256
    outs = alloc_outputs(torch, dev, 1, M)
    for i in range(args.warmup):
        K.analyze_batch([pool[i % POOL]], M, MAX_K, out=outs)
    torch.cuda.synchronize(dev)
    if K.stream_status(stream) != K.OK:
        raise RuntimeError("warm-up reported an error")
    # parity spot check of the timed configuration against the oracle (rank 0, one image)
    parity = None
    if rank == 0 and not args.no_check:
        import oracle

        oracle.build()
        card, sumc, c, ts, cnt, t0 = K.analyze_batch([pool[0]], M, MAX_K, out=outs)
        torch.cuda.synchronize(dev)
        ocard, osumc, oc, ots, ocnt, ot0 = oracle.analyze(pool_np[0], M, MAX_K, method="alg1")
        parity = bool(np.array_equal(card[0].cpu().numpy().view(np.uint64), ocard)
                      and np.array_equal(sumc[0].cpu().numpy().view(np.uint64), osumc)
                      and np.array_equal(c[0].cpu().numpy(), oc) and np.array_equal(ts[0].cpu().numpy(), ots)
                      and int(cnt[0]) == ocnt and int(t0[0]) == ot0)
    # The K steps are one CUDA graph of K fused launches (the pool cycled
    # inside; at most 512 launches per graph, several graphs for larger K), so
    # the host's per-call cost does not pace the GPU.  The graph is replayed R
    # times; each replay is one timed block of exactly K steps between a
    # barrier and a synchronize on both sides, timed by an event pair on the
    # launching stream (events inside a block would stop a launch from
    # overlapping the previous one's epilogue).  ms_per_step is the median
    # block over K; p90 is reported beside it.
    # Every kernel before a call on these streams is the library's own previous
    # call.  The timed stream is pipelined (kohler_stream_overlap mode 2): each
    # call's pass overlaps the previous call's epilogue, and two consecutive
    # calls run side by side on half the SMs each.  `stream` (isolated and
    # Python-launched references) and `wstream` (the same graph with whole-GPU
    # launches, reported beside the headline) use mode 1.
    gstream = torch.cuda.Stream(dev)
    wstream = torch.cuda.Stream(dev)
    K.stream_overlap(gstream, pipeline=True)
    K.stream_overlap(wstream)
    K.stream_overlap(stream)
    G = 512

    def capture(j0, n, st):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for j in range(j0, j0 + n):
                K.analyze_batch([pool[j % POOL]], M, MAX_K, out=outs, stream=st)
        return g

    for st in (gstream, wstream):
        with torch.cuda.stream(st):
            for i in range(3):  # creates the library's workspace for this stream before capture
                K.analyze_batch([pool[i % POOL]], M, MAX_K, out=outs, stream=st)
    torch.cuda.synchronize(dev)
    graphs = [capture(j0, min(G, args.steps - j0), gstream) for j0 in range(0, args.steps, G)]

    def replay_all(gs=None, st=None):
        with torch.cuda.stream(st or gstream):
            for g in (gs or graphs):
                g.replay()

    replay_all()  # warm replay
    torch.cuda.synchronize(dev)
    est_block_s = args.steps * 16e-6
    # about one second of blocks, so that the clock samples (every 20 ms) cover them
    R = args.reps if args.reps > 0 else int(max(5, min(2000, 1.0 / max(est_block_s, 1e-9))))
    sampler = ClockSampler(local)
    time.sleep(0.3)
    blocks = []
    barrier(dist)
    torch.cuda.synchronize(dev)
    sampler.mark_start()
    t_start = time.perf_counter()
    for _ in range(R):
        barrier(dist)
        torch.cuda.synchronize(dev)
        e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_start.record(gstream)
        replay_all()
        e_end.record(gstream)
        torch.cuda.synchronize(dev)
        barrier(dist)
        blocks.append(e_start.elapsed_time(e_end) / 1e3)
    t_host = time.perf_counter() - t_start
    sampler.mark_end()
    time.sleep(0.1)
    sampler.stop()
    st = K.stream_status(gstream)
    if st != K.OK:
        raise RuntimeError(f"timed run reported status {st}")
    dev_s = float(np.median(blocks))
    dev_p90 = float(np.percentile(blocks, 90))
    # the same K steps with whole-GPU launches (mode 1), a few blocks, for reference
    wgraphs = [capture(j0, min(G, args.steps - j0), wstream) for j0 in range(0, args.steps, G)]
    replay_all(wgraphs, wstream)
    torch.cuda.synchronize(dev)
    wblocks = []
    for _ in range(max(5, min(200, R // 4))):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(wstream)
        replay_all(wgraphs, wstream)
        b.record(wstream)
        torch.cuda.synchronize(dev)
        wblocks.append(a.elapsed_time(b) / 1e3)
    whole_gpu_ms_per_step = float(np.median(wblocks)) * 1e3 / args.steps
    del wgraphs
    # the same steps launched one by one from Python through the binding, for reference
    outt = outs
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_host = min(args.steps, 1000)
    h0.record(stream)
    for i in range(n_host):
        K.analyze_batch([pool[i % POOL]], M, MAX_K, out=outt)
    h1.record(stream)
    torch.cuda.synchronize(dev)
    host_launched_us = h0.elapsed_time(h1) * 1e3 / n_host
    # isolated launches (each bracketed by events; no overlap), for reference
    launch_ms = []
    for i in range(min(50, args.steps)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        K.analyze_batch([pool[i % POOL]], M, MAX_K, out=outt)
        b.record(stream)
        b.synchronize()
        launch_ms.append(a.elapsed_time(b))
    elapsed = max_over_ranks(dist, dev_s)  # one block of K steps: the median over the R blocks
    host_elapsed = max_over_ranks(dist, t_host)
    total_px = sum_over_ranks(dist, float(px * args.steps))
    value = total_px / elapsed / 1e9
    # one fused launch (pass + epilogue kernel) per step; with two launches in
    # flight a launch lasts about two steps, so the rate is taken over the block
    mean_launch_s = dev_s / args.steps
    peak, peak_src = measured_peak_hbm()
    achieved = px / mean_launch_s / 1e9  # algorithmic bytes: one read of each 1-byte pixel, per step time
    traffic = kernel_traffic("k_u8h", "voronoi_18mp")
    e2e = bench_e2e(args, pool_np, M, rank, dist) if not args.no_e2e else None
    cpu = cpu_baseline(pool_np[0], M) if (rank == 0 and world == 1 and not args.no_cpu) else None
    del pool
    torch.cuda.empty_cache()
    forms = run_forms(args, K, torch, dev, peak) if (world == 1 and args.forms) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": {"workload": "voronoi_18mp", "image": f"{W}x{H} uint8", "M": M, "max_k": MAX_K,
                   "images_per_step": 1, "per_gpu_pool": f"{POOL} distinct images ({POOL * px / 1e6:.0f} MB) cycled",
                   "l2": "inputs larger than L2 (rotating pool), no flush", "parallelism": f"replicas x{world}",
                   "launch": f"one CUDA graph of the K fused launches, replayed R = {R} times; pipelined stream: "
                             "two consecutive launches side by side on half the SMs each (programmatic dependent "
                             "launch)",
                   "timing": {"blocks_R": R, "steps_per_block": args.steps,
                              "whole_gpu_launches_ms_per_step": whole_gpu_ms_per_step,
                              "block_ms_median": dev_s * 1e3, "block_ms_p90": dev_p90 * 1e3,
                              "ms_per_step_p90": dev_p90 * 1e3 / args.steps,
                              "statistic": "median block / K (p90 beside it); max over ranks"}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": f"hbm_gbs of {peak_src}",
                     "kernel": "k_u8h (strip pass) + k_finish (curve, thresholds), one step",
                     "rate": "algorithmic bytes of the K steps / the timed block (two launches in flight)",
                     "mean_launch_us": mean_launch_s * 1e6,
                     "isolated_launch_p50_us": float(np.median(launch_ms)) * 1e3,
                     "host_launched_us_per_step": host_launched_us},
        # every step launches two of the library's kernels (the strip pass and
        # k_finish); the timed region holds R blocks of K steps
        "e2e": e2e, "gpu_launches": 2 * args.steps * R, "gpu_launches_per_step": 2,
        "clocks": sampler.summary(), "host_elapsed_s": host_elapsed,
        "parity_spot_check": parity,
        "paper_context": {"gpx_s": 0.138, "workload": "Tulips 3672x4896, 0.130 s (Table 1)",
                          "hardware": "Intel i7-4702HQ, 4 cores / 8 threads, OpenMP + SIMD"},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if forms is not None:
        line["forms"] = forms
        line["forms_summary"] = forms_summary(forms)  # last key: stays in a tail of the output
    return line


def alloc_outputs(torch, dev, n, M):
    return (torch.empty((n, M), dtype=torch.int64, device=dev), torch.empty((n, M), dtype=torch.int64, device=dev),
            torch.empty((n, M), dtype=torch.float64, device=dev), torch.empty((n, MAX_K), dtype=torch.int32, device=dev),
            torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev))


def bench_e2e(args, pool_np, M, rank, dist):
    """Same metric through the host-buffer C-ABI call: pinned host image in,
    host curve + thresholds out, copies inside the timed region."""
    import torch

    import paper_1707_05062_gb300 as K

    steps = max(3, min(args.steps, args.e2e_steps))
    pinned = [torch.from_numpy(im).pin_memory() for im in pool_np[:4]]
    out = K.host_outputs(M, MAX_K)  # the caller's result arrays, reused every step
    for i in range(3):
        K.analyze_host(pinned[i % 4], M, MAX_K, out=out)
    barrier(dist)
    t = time.perf_counter()
    for i in range(steps):
        K.analyze_host(pinned[i % 4], M, MAX_K, out=out)
    dt = time.perf_counter() - t
    dt = max_over_ranks(dist, dt)
    px = pool_np[0].size
    total = sum_over_ranks(dist, float(px * steps))
    return {"value": total / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(px),
            "d2h_bytes_per_step": int(M * 8 * 3 + MAX_K * 4 + 8), "steps": steps,
            "call": "kohler_analyze_host (pinned host image -> host curve and thresholds; "
                    "recorded as one CUDA graph per geometry and replayed)"}


# ----------------------------------------------------------------------------- batched and served forms
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _graph_of(torch, dev, fn, pipeline=False):
    """Captures fn(stream) into a CUDA graph on a side stream (after two eager
    calls there, which create the library's workspace for that stream)."""
    import paper_1707_05062_gb300 as K

    s = torch.cuda.Stream(dev)
    K.stream_overlap(s, pipeline=pipeline)  # the stream holds only the library's calls
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        fn(s)
        fn(s)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn(s)
    torch.cuda.synchronize(dev)
    return g, s


def _time_graph(torch, g, s, reps):
    a, b = _events(torch)
    with torch.cuda.stream(s):
        g.replay()
        a.record(s)
        for _ in range(reps):
            g.replay()
        b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def _time_host(torch, fn, s, reps):
    a, b = _events(torch)
    fn(s)
    a.record(s)
    for _ in range(reps):
        fn(s)
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def form_batched(K, torch, dev, imgs_np, M, name, check_idx, peak):
    """One launch over the whole batch (per-image histogram slices, per-image
    epilogues) against one launch per image, on the same device-resident images."""
    import oracle

    n = len(imgs_np)
    imgs = [torch.from_numpy(im).to(dev) for im in imgs_np]
    px = sum(im.size for im in imgs_np)
    nbytes = sum(im.nbytes for im in imgs_np)
    outs = alloc_outputs(torch, dev, n, M)
    rows = [tuple(t[j:j + 1] for t in outs) for j in range(n)]

    def batched(s):
        K.analyze_batch(imgs, M, MAX_K, out=outs, stream=s)

    per_graph = 8  # batch launches per graph: back to back, as the headline times its launches

    def batched_run(s):
        for _ in range(per_graph):
            batched(s)

    def plain(s):
        for j in range(n):
            K.analyze_batch([imgs[j]], M, MAX_K, out=rows[j], stream=s)

    res = {"images": n, "mpixel": px / 1e6, "bytes": nbytes, "M": M}
    gb, sb = _graph_of(torch, dev, batched_run)
    t1 = _time_graph(torch, gb, sb, 2) / per_graph
    reps = int(min(100, max(5, 0.5 / max(t1 * per_graph, 1e-6))))
    tb = _time_graph(torch, gb, sb, reps) / per_graph
    g1, s1 = _graph_of(torch, dev, batched)
    tb_single = _time_graph(torch, g1, s1, reps)
    tb_host = _time_host(torch, batched, sb, reps)
    if K.stream_status(sb) != K.OK or K.stream_status(s1) != K.OK:
        raise RuntimeError(f"{name}: batched launch reported an error")
    gp, sp = _graph_of(torch, dev, plain)
    tp = _time_graph(torch, gp, sp, max(3, reps // 4))
    tp_host = _time_host(torch, plain, sp, max(3, reps // 4))
    if K.stream_status(sp) != K.OK:
        raise RuntimeError(f"{name}: per-image launches reported an error")
    res["batched"] = {"launches_per_step": (n + 127) // 128, "ms_graph": tb * 1e3, "gpx_s_graph": px / tb / 1e9,
                      "hbm_frac_graph": nbytes / tb / 1e9 / peak, "graph": f"{per_graph} batch launches per graph",
                      "ms_graph_single": tb_single * 1e3, "ms_host": tb_host * 1e3,
                      "gpx_s_host": px / tb_host / 1e9, "reps": reps}
    res["plain"] = {"launches_per_step": n, "ms_graph": tp * 1e3, "gpx_s_graph": px / tp / 1e9,
                    "hbm_frac_graph": nbytes / tp / 1e9 / peak, "ms_host": tp_host * 1e3,
                    "gpx_s_host": px / tp_host / 1e9}
    res["batched_over_plain_graph"] = tp / tb
    res["batched_over_plain_host"] = tp_host / tb_host

    def parity():
        # sampled images of the batch from a fresh batched call must equal the oracle
        batched(torch.cuda.current_stream(dev))
        torch.cuda.synchronize(dev)
        ok = True
        for j in check_idx:
            ocard, osumc, oc, ots, ocnt, ot0 = oracle.analyze(imgs_np[j], M, MAX_K, method="alg1")
            ok = ok and bool(np.array_equal(outs[0][j].cpu().numpy().view(np.uint64), ocard)
                             and np.array_equal(outs[1][j].cpu().numpy().view(np.uint64), osumc)
                             and np.array_equal(outs[2][j].cpu().numpy(), oc)
                             and np.array_equal(outs[3][j].cpu().numpy(), ots)
                             and int(outs[4][j]) == ocnt and int(outs[5][j]) == ot0)
        return ok

    res["parity_spot_check"] = {"images": list(check_idx), "equal": parity()}
    # the autotuner's choice for this batch (every candidate checked exact by the
    # tuner), then the same batched graph timed again with it
    if n <= 128:
        t0 = time.perf_counter()
        rep = K.autotune(imgs, M, reps=5)
        tune_s = time.perf_counter() - t0
        gt, st = _graph_of(torch, dev, batched_run)
        tt = _time_graph(torch, gt, st, reps) / per_graph
        gt1, st1 = _graph_of(torch, dev, batched)
        tt_single = _time_graph(torch, gt1, st1, reps)
        if K.stream_status(st) != K.OK or K.stream_status(st1) != K.OK:
            raise RuntimeError(f"{name}: tuned batched launch reported an error")
        res["tuned"] = {"ms_graph": tt * 1e3, "gpx_s_graph": px / tt / 1e9, "hbm_frac_graph": nbytes / tt / 1e9 / peak,
                        "ms_graph_single": tt_single * 1e3, "over_default": tb / tt, "tune_wall_s": tune_s,
                        "candidates": sum(len(g["candidates"]) for g in rep["groups"]),
                        "all_candidates_exact": all(c["exact"] for g in rep["groups"] for c in g["candidates"]),
                        "choice": [{"pass": g["pass"], "default_us": g["default_us"], **g["best"]}
                                   for g in rep["groups"]],
                        "parity_spot_check": parity()}
        K.tune_clear()
        del gt, gt1
    del imgs, outs, rows, gb, g1, gp
    torch.cuda.empty_cache()
    return res


class _Server:
    def __init__(self, K, M, max_k):
        import ctypes

        self.K, self.L, self.ct = K, K.lib(), ctypes
        self.h = ctypes.c_void_p()
        self.max_k = max_k
        rc = self.L.kohler_server_create(ctypes.byref(self.h), M, max_k, 0, 0)
        if rc != 0:
            raise RuntimeError(f"kohler_server_create: {rc}")

    def submit(self, frame):
        # the frames are pinned and live for the whole run: the server reads them
        # asynchronously (kohler_submit_borrowed), several copies in flight
        ct = self.ct
        t = ct.c_uint64()
        while True:
            rc = self.L.kohler_submit_borrowed(self.h, frame.ctypes.data, 1, frame.shape[1], frame.shape[0],
                                               frame.strides[0], ct.byref(t))
            if rc != self.K.ERR_BUSY:
                break
            time.sleep(0.0002)
        if rc != 0:
            raise RuntimeError(f"kohler_submit: {rc}")
        return t.value

    def submit_segment(self, frame, out):
        ct = self.ct
        t = ct.c_uint64()
        while True:
            rc = self.L.kohler_submit_segment(self.h, frame.ctypes.data, 1, frame.shape[1], frame.shape[0],
                                              frame.strides[0], out.ctypes.data, out.strides[0], ct.byref(t))
            if rc != self.K.ERR_BUSY:
                break
            time.sleep(0.0002)
        if rc != 0:
            raise RuntimeError(f"kohler_submit_segment: {rc}")
        return t.value

    def poll(self, ticket):
        ct = self.ct
        ts = (ct.c_int32 * max(1, self.max_k))()
        res = self.K.KohlerResult()
        res.thresholds = ct.cast(ts, ct.c_void_p)
        rc = self.L.kohler_poll(self.h, ct.c_uint64(ticket), ct.byref(res), -1)
        if rc != 0:
            raise RuntimeError(f"kohler_poll: {rc}")
        return res.t0, res.count, list(ts)[:self.max_k], res.latency_s

    def submit_many(self, frs):
        # one call for a batch of pinned frames (kohler_submit_borrowed_many)
        ct = self.ct
        arr = (self.K.KohlerFrame * len(frs))()
        for j, f in enumerate(frs):
            arr[j] = self.K.KohlerFrame(f.ctypes.data, f.shape[1], f.shape[0], f.strides[0])
        tickets = (ct.c_uint64 * len(frs))()
        rc = self.L.kohler_submit_borrowed_many(self.h, arr, len(frs), 1, tickets, None)
        if rc != 0:
            raise RuntimeError(f"kohler_submit_borrowed_many: {rc}")
        return list(tickets)

    def poll_many(self, tickets):
        ct = self.ct
        n = len(tickets)
        bufs = [(ct.c_int32 * max(1, self.max_k))() for _ in range(n)]
        res = (self.K.KohlerResult * n)()
        for j in range(n):
            res[j].thresholds = ct.cast(bufs[j], ct.c_void_p)
        st = (ct.c_int32 * n)()
        rc = self.L.kohler_poll_many(self.h, (ct.c_uint64 * n)(*tickets), n, res, st, -1)
        if rc != 0 or any(st):
            raise RuntimeError(f"kohler_poll_many: {rc} {list(st)}")
        return [(res[j].t0, res[j].count, list(bufs[j])[:self.max_k], res[j].latency_s) for j in range(n)]

    def stats(self):
        ct = self.ct
        v = [ct.c_uint64() for _ in range(4)]
        self.L.kohler_server_stats(self.h, *[ct.byref(x) for x in v])
        return [x.value for x in v]

    def close(self):
        self.L.kohler_server_destroy(self.h)


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def form_served(K, torch, dev, n_frames=2000, fps=240.0, distinct=8, closed_frames=2000, plain_frames=300):
    """Poisson-arriving video frames of mixed resolutions through the server
    (continuous batching), against one synchronous host call per frame."""
    import queue

    import oracle
    import synth

    arrivals, res_idx = synth.video_schedule(n_frames, fps)
    scene = synth.VideoScene()
    # `distinct` rendered frames per resolution, cycled in arrival order
    # frames sit in pinned host memory (numpy views of pinned tensors), as a
    # capture pipeline would deliver them
    frames = {r: [torch.from_numpy(scene.frame(k, *synth.VIDEO_SIZES[r])).pin_memory().numpy() for k in range(distinct)]
              for r in range(len(synth.VIDEO_SIZES))}
    src = []
    seen = [0] * len(synth.VIDEO_SIZES)
    for r in res_idx:
        src.append((int(r), seen[r] % distinct))
        seen[r] += 1
    want = {}
    for r, fl in frames.items():
        for k, f in enumerate(fl):
            card, sumc = oracle.curve_alg1(f, 256)
            ts, cnt, t0 = oracle.thresholds(card, sumc, MAX_K)
            want[(r, k)] = (int(t0), int(cnt), ts.tolist())
    px = np.array([frames[r][k].size for r, k in src], dtype=np.float64)
    out = {"frames": n_frames, "fps_offered": fps, "mean_mpixel_per_frame": float(px.mean() / 1e6),
           "resolutions": {f"{w}x{h}": int((res_idx == r).sum()) for r, (w, h) in enumerate(synth.VIDEO_SIZES)},
           "content": f"{distinct} rendered frames per resolution, cycled in arrival order, in pinned host memory"}

    def run(order, times):
        srv = _Server(K, 256, MAX_K)
        q = queue.Queue()
        results = [None] * len(order)
        t_base = time.perf_counter() + 0.05

        def producer():
            for j, (r, k) in enumerate(order):
                if times is not None:
                    # sleep until shortly before the arrival, then spin: a plain
                    # sleep overshoots by tens of microseconds
                    target = t_base + times[j]
                    dt = target - time.perf_counter()
                    if dt > 3e-4:
                        time.sleep(dt - 3e-4)
                    while time.perf_counter() < target:
                        pass
                t_arr = t_base + times[j] if times is not None else time.perf_counter()
                t_sub = time.perf_counter()
                q.put((j, srv.submit(frames[r][k]), t_arr, t_sub))

        th = threading.Thread(target=producer)
        t_start = time.perf_counter()
        th.start()
        for _ in range(len(order)):
            j, ticket, t_arr, t_sub = q.get()
            t0, cnt, ts, lat_srv = srv.poll(ticket)
            t_done = time.perf_counter()
            results[j] = (t0, cnt, ts, t_done - t_arr, lat_srv, t_done - t_sub, t_sub - t_arr)
        th.join()
        t_end = time.perf_counter()
        stats = srv.stats()
        srv.close()
        return results, (t_start if times is None else t_base), t_end, stats

    ok = True
    # (i) open loop: Poisson arrivals at `fps`
    results, t_a, t_b, stats = run(src, arrivals)
    lat = [r[3] for r in results]
    ok = ok and all((r[0], r[1], r[2]) == want[s] for r, s in zip(results, src))
    out["open_loop"] = {"fps_achieved": n_frames / (t_b - t_a), "latency_ms_p50": _pct(lat, 50) * 1e3,
                        "latency_ms_p99": _pct(lat, 99) * 1e3, "latency_ms_max": max(lat) * 1e3,
                        "submit_to_result_ms_p50": _pct([r[5] for r in results], 50) * 1e3,
                        "submit_to_result_ms_p99": _pct([r[5] for r in results], 99) * 1e3,
                        "producer_lateness_ms_p99": _pct([r[6] for r in results], 99) * 1e3,
                        "server_latency_ms_p50": _pct([r[4] for r in results], 50) * 1e3,
                        "server_latency_ms_p99": _pct([r[4] for r in results], 99) * 1e3,
                        "launches": stats[2], "max_frames_per_launch": stats[3],
                        "submit": "kohler_submit_borrowed (pinned frames read asynchronously)",
                        "latency": "scheduled arrival -> thresholds in host memory (poll returned)",
                        "by_resolution": {f"{w}x{h}": {"p50_ms": _pct([x[3] for x, (r, _) in zip(results, src) if r == ri], 50) * 1e3,
                                                       "p99_ms": _pct([x[3] for x, (r, _) in zip(results, src) if r == ri], 99) * 1e3}
                                          for ri, (w, h) in enumerate(synth.VIDEO_SIZES)}}
    def run_batched(order, B):
        # closed loop with batched calls: the producer hands over B frames per
        # kohler_submit_borrowed_many, the consumer collects them with one
        # kohler_poll_many
        srv = _Server(K, 256, MAX_K)
        q = queue.Queue()
        results = [None] * len(order)

        def producer():
            for j0 in range(0, len(order), B):
                js = list(range(j0, min(len(order), j0 + B)))
                t_sub = time.perf_counter()
                q.put((js, srv.submit_many([frames[order[j][0]][order[j][1]] for j in js]), t_sub))

        th = threading.Thread(target=producer)
        t_start = time.perf_counter()
        th.start()
        done = 0
        while done < len(order):
            js, tickets, t_sub = q.get()
            res = srv.poll_many(tickets)
            t_done = time.perf_counter()
            for j, r in zip(js, res):
                results[j] = (r[0], r[1], r[2], t_done - t_sub, r[3], t_done - t_sub, 0.0)
            done += len(js)
        th.join()
        t_end = time.perf_counter()
        stats = srv.stats()
        srv.close()
        return results, t_start, t_end, stats

    # (ii) closed loop: batches of 8 frames handed over and collected per call
    sub = src[:closed_frames]
    results, t_a, t_b, stats = run_batched(sub, 8)
    ok = ok and all((r[0], r[1], r[2]) == want[s] for r, s in zip(results, sub))
    lat = [r[3] for r in results]
    out["closed_loop"] = {"frames": len(sub), "fps": len(sub) / (t_b - t_a),
                          "gpx_s": float(px[:len(sub)].sum()) / (t_b - t_a) / 1e9,
                          "latency_ms_p50": _pct(lat, 50) * 1e3, "latency_ms_p99": _pct(lat, 99) * 1e3,
                          "launches": stats[2], "max_frames_per_launch": stats[3],
                          "mean_frames_per_launch": len(sub) / max(1, stats[2]),
                          "submit": "kohler_submit_borrowed_many, 8 frames per call; kohler_poll_many per batch",
                          "h2d_gb_s": float(sum(frames[r][k].nbytes for r, k in sub)) / (t_b - t_a) / 1e9}
    # (iii) plain: one synchronous host call per frame (pinned frames), in arrival order
    pinned = {key: torch.from_numpy(frames[key[0]][key[1]]) for key in want}
    sub = src[:plain_frames]
    lat = []
    t_a = time.perf_counter()
    for key in sub:
        t = time.perf_counter()
        card, sumc, c, ts, cnt, t0 = K.analyze_host(pinned[key], 256, MAX_K)
        lat.append(time.perf_counter() - t)
        ok = ok and (t0, cnt, ts.tolist()) == want[key]
    t_b = time.perf_counter()
    out["plain_per_frame"] = {"frames": len(sub), "fps": len(sub) / (t_b - t_a),
                              "gpx_s": float(px[:len(sub)].sum()) / (t_b - t_a) / 1e9,
                              "latency_ms_p50": _pct(lat, 50) * 1e3, "latency_ms_p99": _pct(lat, 99) * 1e3,
                              "call": "kohler_analyze_host per frame"}
    # (iv) open loop again, every frame also segmented into two classes at its t0
    # and copied back (the paper's video experiment, Section 4 and Table 2);
    # outputs in per-resolution rings of pinned buffers, a slot reused only
    # after its frame was polled
    ring = 16
    outs = {r: [torch.empty(frames[r][0].shape, dtype=torch.uint8).pin_memory().numpy() for _ in range(ring)]
            for r in frames}
    want_seg = {key: oracle.segment(frames[key[0]][key[1]], 256, [want[key][0]]) for key in want}
    free = {r: threading.Semaphore(ring) for r in frames}
    srv = _Server(K, 256, MAX_K)
    q = queue.Queue()
    t_base = time.perf_counter() + 0.05

    def producer():
        used = {r: 0 for r in frames}
        for j, (r, k) in enumerate(src):
            target = t_base + arrivals[j]
            dt = target - time.perf_counter()
            if dt > 3e-4:
                time.sleep(dt - 3e-4)
            while time.perf_counter() < target:
                pass
            free[r].acquire()
            slot = used[r] % ring
            used[r] += 1
            q.put((j, srv.submit_segment(frames[r][k], outs[r][slot]), target, r, k, slot))

    # the comparisons run in their own thread, off the poll path; it frees the slot
    checks = queue.Queue()
    all_equal = [True]

    def checker():
        while True:
            item = checks.get()
            if item is None:
                return
            r, k, slot, t0 = item
            all_equal[0] = all_equal[0] and t0 == want[(r, k)][0] and np.array_equal(outs[r][slot], want_seg[(r, k)])
            free[r].release()

    th = threading.Thread(target=producer)
    tc = threading.Thread(target=checker)
    tc.start()
    th.start()
    lat = []
    for _ in range(n_frames):
        j, ticket, t_arr, r, k, slot = q.get()
        t0, cnt, ts, lat_srv = srv.poll(ticket)
        lat.append(time.perf_counter() - t_arr)
        checks.put((r, k, slot, t0))
    th.join()
    t_end = time.perf_counter()
    checks.put(None)
    tc.join()
    seg_ok = all_equal[0]
    srv.close()
    out["segmented_open_loop"] = {"fps_achieved": n_frames / (t_end - t_base),
                                  "latency_ms_p50": _pct(lat, 50) * 1e3, "latency_ms_p99": _pct(lat, 99) * 1e3,
                                  "latency_ms_max": max(lat) * 1e3,
                                  "latency": "scheduled arrival -> two-class frame in host memory (poll returned)",
                                  "parity_all_frames": bool(seg_ok),
                                  "paper_context": "97 frames/s segmented, 502x480 video, i7-4702HQ (Table 2)"}
    out["parity_all_frames"] = ok
    return out


def form_segment(K, torch, dev, peak, n_pool=6):
    """Segmentation of the 18-Mpixel images by their own ranked thresholds (each
    pixel replaced by its class mean), the thresholds and their count passed
    on the device from a preceding analyze call: kohler_segment alone, and the
    whole analyze + segment per image, both as CUDA-graph replays cycling
    n_pool images and outputs (more bytes than L2)."""
    import oracle
    import synth

    pool_np = synth.voronoi_18mp_pool(n_pool)
    H, W = pool_np[0].shape
    px = W * H
    imgs = [torch.from_numpy(im).to(dev) for im in pool_np]
    outs = [torch.empty_like(im) for im in imgs]
    res_an = [K.analyze_batch([im], 256, 6) for im in imgs]
    torch.cuda.synchronize(dev)

    def seg_only(s):
        for j in range(n_pool):
            K.segment(imgs[j], 256, res_an[j][3][0], res_an[j][4][0], out=outs[j], stream=s)

    def whole(s):
        for j in range(n_pool):
            K.analyze_batch([imgs[j]], 256, 6, out=res_an[j], stream=s)
            K.segment(imgs[j], 256, res_an[j][3][0], res_an[j][4][0], out=outs[j], stream=s)

    g1, s1 = _graph_of(torch, dev, seg_only)
    t_seg = _time_graph(torch, g1, s1, 20) / n_pool
    g2, s2 = _graph_of(torch, dev, whole)
    t_all = _time_graph(torch, g2, s2, 20) / n_pool
    if K.stream_status(s1) != K.OK or K.stream_status(s2) != K.OK:
        raise RuntimeError("segment: a launch reported an error")
    ts = res_an[0][3][0].cpu().numpy()
    want = oracle.segment(pool_np[0], 256, [int(t) for t in ts if t >= 0])
    moved = 3 * px  # the image read by the level-count pass and by the map pass, the output written
    return {"workload": f"{W}x{H} uint8 Voronoi images, M = 256, their 6 ranked thresholds (7 classes)",
            "segment_ms": t_seg * 1e3, "segment_gpx_s": px / t_seg / 1e9,
            "segment_bytes_per_image": moved, "segment_hbm_frac": moved / t_seg / 1e9 / peak,
            "analyze_plus_segment_ms": t_all * 1e3, "analyze_plus_segment_gpx_s": px / t_all / 1e9,
            "parity_spot_check": bool(np.array_equal(outs[0].cpu().numpy(), want)),
            "launch": f"CUDA-graph replays of {n_pool} images"}


def form_nbhd(K, torch, dev, peak, n_pool=6):
    """The whole path (curve + thresholds) of the 18-Mpixel images with the 8- and
    the hexagonal 6-neighbourhood, beside the 4-neighbourhood, as CUDA-graph
    replays cycling n_pool images (more bytes than L2); one image of each checked
    against the oracle."""
    import oracle
    import synth

    pool_np = synth.voronoi_18mp_pool(n_pool)
    H, W = pool_np[0].shape
    px = W * H
    imgs = [torch.from_numpy(im).to(dev) for im in pool_np]
    out = {"workload": f"{W}x{H} uint8 Voronoi images, M = 256",
           "launch": f"CUDA-graph replays of {n_pool} images on a pipelined stream (whole-GPU launches beside)"}
    for nb in (4, 8, 6):
        res = [K.analyze_batch([im], 256, 16, nbhd=nb) for im in imgs]
        torch.cuda.synchronize(dev)

        def run(s, nb=nb, res=res):
            for j in range(n_pool):
                K.analyze_batch([imgs[j]], 256, 16, out=res[j], stream=s, nbhd=nb)

        g, st = _graph_of(torch, dev, run, pipeline=True)
        t = _time_graph(torch, g, st, 20) / n_pool
        gw, sw = _graph_of(torch, dev, run)
        tw = _time_graph(torch, gw, sw, 20) / n_pool
        if K.stream_status(st) != K.OK or K.stream_status(sw) != K.OK:
            raise RuntimeError(f"N{nb}: a launch reported an error")
        want = oracle.analyze(pool_np[0], 256, 16, nbhd=nb)
        got = (res[0][0][0].cpu().numpy().view(np.uint64), res[0][1][0].cpu().numpy().view(np.uint64),
               res[0][2][0].cpu().numpy(), res[0][3][0].cpu().numpy(), int(res[0][4][0]), int(res[0][5][0]))
        ok = all(np.array_equal(got[k], want[k]) for k in range(4)) and got[4:] == want[4:]
        pairs = {4: 2, 8: 4, 6: 3}[nb]
        out[f"N{nb}"] = {"ms": t * 1e3, "gpx_s": px / t / 1e9, "gpairs_s": pairs * px / t / 1e9,
                         "hbm_frac": px / t / 1e9 / peak, "whole_gpu_ms": tw * 1e3, "parity_spot_check": bool(ok)}
    return out


def form_ceiling(K, torch, dev, peak):
    """Microbenchmarks of the ceilings the strip pass runs into (libkohler_probe):
    conflict-free shared-memory additions and three-input integer additions per
    clock per SM, and the per-row work of the four-addition (k_u8h) and the
    three-addition formulations on register data, in pixels per clock per SM,
    with the rates they imply on this GPU."""
    import ctypes

    from paper_1707_05062_gb300 import build as kbuild

    L = ctypes.CDLL(kbuild.PROBE_LIB)
    L.kohler_probe_run.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cyc = torch.zeros(sms, dtype=torch.int64, device=dev)
    sink = torch.zeros(1024, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev)
    out = {"sms": sms, "warps_per_sm": 16}

    def run(which, iters):
        for _ in range(2):
            a, b = _events(torch)
            a.record(s)
            if L.kohler_probe_run(which, sms, iters, cyc.data_ptr(), sink.data_ptr(), ctypes.c_void_p(s.cuda_stream)):
                raise RuntimeError("probe launch failed")
            b.record(s)
            b.synchronize()
        c = cyc.cpu().numpy().astype(np.float64)
        return float(np.median(c)), a.elapsed_time(b) / 1e3

    cyc_red, t_red = run(0, 4000)
    out["shared_add_warp_inst_per_clk_sm"] = 16 * 4000 * 16 / cyc_red
    cyc_add, _ = run(1, 4000)
    out["int_add3_warp_inst_per_clk_sm"] = 16 * 4000 * 32 / cyc_add
    mhz = cyc_red / t_red / 1e6  # clock seen by the probe (cycles of the median block over the launch time)
    out["sm_mhz_during_probe"] = mhz
    for which, name, upd in ((2, "rows_4_additions", 4), (3, "rows_3_additions", 3)):
        c, _ = run(which, 200)
        ppc = 16 * 200 * 4 * 256 / c
        gpx = ppc * sms * mhz * 1e6 / 1e9
        out[name] = {"px_per_clk_sm": ppc, "implied_gpx_s": gpx, "implied_hbm_frac_u8": gpx / peak,
                     "shared_add_bound_px_per_clk_sm": out["shared_add_warp_inst_per_clk_sm"] * 32 / upd}
    out["reading"] = ("the per-row work alone runs at the shared-add bound for 4 additions per pixel; the strip "
                      "pass adds the ring's tensor-copy writes and row loads to the same shared-memory pipe "
                      "(profiles/k_u8h_voronoi_18mp.md) and pays fixed per-launch phases")
    return out


def form_blobs(K, torch, dev, reps=300):
    """Config 1: one 256 x 256 uint8 blobs image, M = 256, the plain single-image
    path.  Launch-bound, so reported as latency: one call as a CUDA-graph replay
    (device events around each replay), one call through the host-buffer entry
    point (host wall clock, copies included), and back-to-back graph throughput."""
    import oracle
    import synth

    img_np = synth.blobs_image()
    img = torch.from_numpy(img_np).to(dev)
    outs = alloc_outputs(torch, dev, 1, 256)
    g1, s1 = _graph_of(torch, dev, lambda s: K.analyze_batch([img], 256, MAX_K, out=outs, stream=s))
    lat = []
    for _ in range(reps):
        a, b = _events(torch)
        with torch.cuda.stream(s1):
            a.record(s1)
            g1.replay()
            b.record(s1)
        b.synchronize()
        lat.append(a.elapsed_time(b) * 1e3)
    n = 100
    gN, sN = _graph_of(torch, dev, lambda s: [K.analyze_batch([img], 256, MAX_K, out=outs, stream=s) for _ in range(n)])
    t_n = _time_graph(torch, gN, sN, 5)
    pinned = torch.from_numpy(img_np).pin_memory()
    hout = K.host_outputs(256, MAX_K)
    for _ in range(5):
        K.analyze_host(pinned, 256, MAX_K, out=hout)
    hl = []
    for _ in range(reps):
        t = time.perf_counter()
        K.analyze_host(pinned, 256, MAX_K, out=hout)
        hl.append((time.perf_counter() - t) * 1e6)
    if K.stream_status(s1) != K.OK or K.stream_status(sN) != K.OK:
        raise RuntimeError("blobs_256: a launch reported an error")
    ocard, osumc, oc, ots, ocnt, ot0 = oracle.analyze(img_np, 256, MAX_K, method="def")
    ok = bool(np.array_equal(outs[0][0].cpu().numpy().view(np.uint64), ocard)
              and np.array_equal(outs[1][0].cpu().numpy().view(np.uint64), osumc)
              and np.array_equal(outs[2][0].cpu().numpy(), oc) and np.array_equal(outs[3][0].cpu().numpy(), ots))
    return {"workload": "256x256 uint8 blobs image, M = 256, plain single-image path",
            "graph_call_us_p50": _pct(lat, 50), "graph_call_us_p99": _pct(lat, 99),
            "host_call_us_p50": _pct(hl, 50), "host_call_us_p99": _pct(hl, 99),
            "back_to_back_us_per_image": t_n * 1e6 / n, "back_to_back_gpx_s": img_np.size * n / t_n / 1e9,
            "host_call": "kohler_analyze_host: pinned image in, curve and thresholds out", "calls": reps,
            "parity_spot_check": ok}


def forms_summary(forms):
    """The forms' headline numbers in a few hundred bytes."""
    out = {}

    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return round(d, 4) if isinstance(d, float) else d

    for name, f in forms.items():
        if not isinstance(f, dict) or "error" in f:
            out[name] = {"error": (f or {}).get("error") if isinstance(f, dict) else "?"}
            continue
        if name in ("batch96", "cosine_u16_batch16"):
            out[name] = {"batched_ms": g(f, "batched", "ms_graph"), "batched_gpx_s": g(f, "batched", "gpx_s_graph"),
                         "batched_hbm_frac": g(f, "batched", "hbm_frac_graph"), "plain_ms": g(f, "plain", "ms_graph"),
                         "batched_over_plain": g(f, "batched_over_plain_graph"), "tuned_ms": g(f, "tuned", "ms_graph"),
                         "tuned_hbm_frac": g(f, "tuned", "hbm_frac_graph"),
                         "parity": g(f, "parity_spot_check", "equal")}
        elif name == "served":
            out[name] = {"open_p50_ms": g(f, "open_loop", "latency_ms_p50"), "open_p99_ms": g(f, "open_loop", "latency_ms_p99"),
                         "open_max_frames_per_launch": g(f, "open_loop", "max_frames_per_launch"),
                         "closed_fps": g(f, "closed_loop", "fps"), "closed_gpx_s": g(f, "closed_loop", "gpx_s"),
                         "closed_max_frames_per_launch": g(f, "closed_loop", "max_frames_per_launch"),
                         "plain_fps": g(f, "plain_per_frame", "fps"),
                         "seg_p99_ms": g(f, "segmented_open_loop", "latency_ms_p99"), "parity": f.get("parity_all_frames")}
        elif name == "segment":
            out[name] = {"ms": g(f, "segment_ms"), "hbm_frac": g(f, "segment_hbm_frac"), "parity": f.get("parity_spot_check")}
        elif name == "nbhd":
            out[name] = {k: {"ms": g(f, k, "ms"), "hbm_frac": g(f, k, "hbm_frac"), "whole_gpu_ms": g(f, k, "whole_gpu_ms")}
                         for k in ("N4", "N8", "N6")}
        elif name == "ceiling":
            out[name] = {"shared_add_per_clk_sm": g(f, "shared_add_warp_inst_per_clk_sm"),
                         "rows4_px_per_clk_sm": g(f, "rows_4_additions", "px_per_clk_sm"),
                         "rows4_hbm_frac": g(f, "rows_4_additions", "implied_hbm_frac_u8"),
                         "rows3_px_per_clk_sm": g(f, "rows_3_additions", "px_per_clk_sm")}
        elif name == "blobs_256":
            out[name] = {"graph_us_p50": g(f, "graph_call_us_p50"), "graph_us_p99": g(f, "graph_call_us_p99"),
                         "host_us_p50": g(f, "host_call_us_p50"), "host_us_p99": g(f, "host_call_us_p99"),
                         "parity": f.get("parity_spot_check")}
    return out


def run_forms(args, K, torch, dev, peak):
    forms = {}
    names = [x for x in args.forms.split(",") if x]
    for name in names:
        t = time.perf_counter()
        try:
            if name == "batch96":
                import synth

                specs = synth.batch96_specs()
                imgs = synth.voronoi_batch(specs, workers=os.cpu_count() or 1)
                small = min(range(len(imgs)), key=lambda j: imgs[j].size)
                large = max(range(len(imgs)), key=lambda j: imgs[j].size)
                forms[name] = form_batched(K, torch, dev, imgs, 256, name, (small, large), peak)
                forms[name]["workload"] = "96 Voronoi uint8 images, sizes 320x240 .. 4096x3072, M = 256"
            elif name == "cosine_u16_batch16":
                import synth

                imgs = synth.cosine_u16_batch()
                forms[name] = form_batched(K, torch, dev, imgs, 4096, name, (), peak)
                forms[name]["workload"] = "16 uint16 2048x2048 12-bit cosine fields, M = 4096"
                forms[name]["parity_spot_check"]["note"] = "full-size parity: tests/test_gpu_parity.py (slow mark)"
            elif name == "served":
                forms[name] = form_served(K, torch, dev)
            elif name == "segment":
                forms[name] = form_segment(K, torch, dev, peak)
            elif name == "nbhd":
                forms[name] = form_nbhd(K, torch, dev, peak)
            elif name == "ceiling":
                forms[name] = form_ceiling(K, torch, dev, peak)
            elif name == "blobs_256":
                forms[name] = form_blobs(K, torch, dev)
            else:
                forms[name] = {"error": "unknown form"}
        except Exception as e:  # a failing form is reported, not hidden
            forms[name] = {"error": f"{type(e).__name__}: {e}"}
        forms[name]["wall_s"] = time.perf_counter() - t
    return forms


def bench_reference(args, rank, world):
    """The CPU oracle as the reference arm: each step a bounded band of the
    same workload on the host cores."""
    import oracle
    import synth

    oracle.build()
    img = synth.voronoi_18mp()
    M = 256
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    rows = 96
    band = np.ascontiguousarray(img[:rows])
    for _ in range(args.warmup):
        card, sumc = oracle.curve(band, M)
        oracle.thresholds(card, sumc, MAX_K)
    t = time.perf_counter()
    for _ in range(args.steps):
        card, sumc = oracle.curve(band, M)
        oracle.normalise(card, sumc)
        oracle.thresholds(card, sumc, MAX_K)
    dt = time.perf_counter() - t
    value = band.size * args.steps / dt / 1e9
    sample = f"rows 0..{rows - 1} of the 5184x3456 image per step ({band.size / 1e6:.2f} Mpixel)"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "voronoi_18mp", "image": "5184x3456 uint8", "M": M, "max_k": MAX_K,
                       "parallelism": "host cores of rank 0"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", cores)),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# Small fixed workloads for ncu captures of one kernel: a few untimed launches,
# then `launches` launches of the case, nothing else on the GPU.
NCU_CASES = ("u8_18mp", "u8_18mp_pipelined", "u16_batch16", "u16_batch16_tuned", "n8_18mp", "n6_18mp", "segment_18mp")


def ncu_case(name: str, launches: int = 3) -> int:
    import tempfile

    import torch

    import paper_1707_05062_gb300 as K
    import synth
    from paper_1707_05062_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    if name.startswith("u16_batch16"):
        imgs_np = synth.cosine_u16_batch()
        imgs = [torch.from_numpy(im.view(np.int16)).to(dev) for im in imgs_np]
        M = 4096
        if name.endswith("_tuned"):
            # the autotuner's choice for this batch: 16 warps, 8 pixels per lane, 64 rows per warp
            px = sum(im.size for im in imgs_np)
            entry = {"pass": "u16_fast", "M": M, "px_class": int(px).bit_length() - 1, "route": "u16_fast",
                     "warps": 16, "px": 8, "per_sm": 0, "upw": 64, "us": 0.0}
            with tempfile.NamedTemporaryFile("w", suffix=".json", delete=False) as f:
                json.dump({"kohler_tune": 1, "entries": [entry]}, f)
            K.tune_load(f.name)
            os.unlink(f.name)
        run = lambda: K.analyze_batch(imgs, M, MAX_K)
    else:
        img = torch.from_numpy(synth.voronoi_18mp()).to(dev)
        if name == "segment_18mp":
            res = K.analyze_batch([img], 256, 6)
            out = torch.empty_like(img)
            run = lambda: K.segment(img, 256, res[3][0], res[4][0], out=out)
        elif name == "u8_18mp":
            run = lambda: K.analyze_batch([img], 256, MAX_K)
        elif name == "u8_18mp_pipelined":
            # the headline's launch configuration: a pipelined stream (half the SMs per pass)
            ps = torch.cuda.Stream(dev)
            K.stream_overlap(ps, pipeline=True)

            def run():
                with torch.cuda.stream(ps):
                    K.analyze_batch([img], 256, MAX_K, stream=ps)
                ps.synchronize()
                if K.stream_status(ps) != K.OK:
                    raise RuntimeError("pipelined case reported an error")
        else:
            nb = 8 if name == "n8_18mp" else 6
            run = lambda: K.analyze_batch([img], 256, MAX_K, nbhd=nb)
    for _ in range(2 + launches):
        run()
    torch.cuda.synchronize(dev)
    return 0 if K.stream_status() == K.OK else 1


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="voronoi_18mp")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--reps", type=int, default=0, help="timed blocks of K steps (0: about 1 s of blocks, 5..2000)")
    ap.add_argument("--forms", default="ceiling,blobs_256,batch96,cosine_u16_batch16,served,segment,nbhd",
                    help="comma list of extra forms reported in the same line (N = 1 only); empty for none")
    ap.add_argument("--ncu-case", choices=NCU_CASES, default=None,
                    help="run only a small fixed workload of one kernel (for ncu captures) and exit")
    args = ap.parse_args(argv)
    if args.ncu_case:
        return ncu_case(args.ncu_case)
    if args.warmup < 3:
        args.warmup = 3
    rank, local, world = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(bench_reference(args, rank, world)), flush=True)
        return 0
    dist = init_dist(world)
    if args.workload != "voronoi_18mp":
        raise SystemExit(f"unknown workload {args.workload}")
    line = bench_ours(args, rank, local, world, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
