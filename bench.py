#!/usr/bin/env python3
"""Block-matching throughput benchmark (one JSON line on stdout, rank 0).

Metric: reference patches matched per second on 512x512 float32 grey images
(8x8 patches, reference stride 3, 39x39 search window, K = 16) -- the
BM3D-shaped workload.  One step = one batch of `--images` such images
already resident in HBM, matched through the C ABI (bm_match_batch): box
filter, bf16 planes, tcgen05 cross term + top-K, FP32/FP64 re-rank.  The
batch is larger than the 129 MB L2, so no L2 flush is needed between
steps.  Timing: CUDA events on the launch stream, barrier + synchronize on
both sides, max over ranks.  Multi-GPU (torchrun): every rank matches its
own batch (weak scaling, no collective on the data path).

--impl reference times the CPU oracle (the plain brute-force definition)
on the host cores instead, each step a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WL = dict(H=512, W=512, C=1, patch=8, window=39, stride=3, K=16, sigma=25.0)
METRIC = "ref patches matched/s at 512^2, 8x8 patch, 39^2 window, K=16"
SEED_BASE = 2000


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--images", type=int, default=160, help="512^2 images per step per GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving latency stream")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream (a seeded prefix of the 2000-request stream)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--minimal", action="store_true",
                    help="timed loop only (no baselines, latency or e2e); for profiler runs")
    return ap.parse_args()


def useful_pairs(H, W, p, win, s):
    """Exact number of (reference, candidate) pairs over clipped windows."""
    h = (win - 1) // 2
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    Hc, Wc = H - p + 1, W - p + 1
    ys = np.arange(ny) * s
    xs = np.arange(nx) * s
    cy = np.minimum(Hc - 1, ys + h) - np.maximum(0, ys - h) + 1
    cx = np.minimum(Wc - 1, xs + h) - np.maximum(0, xs - h) + 1
    return int(cy.sum()) * int(cx.sum())


def tc_issued_flop_per_image(H, W, p, win, s, ty=16, tx=8, products=3):
    """Tensor-core FLOP the tc kernel issues per float32 grey image, for a
    tile of ty x tx references (the tile the library picks for the 512^2,
    p 8, s 3, window 39 class): per tile, every candidate column of the
    window union gets products x p*p/16 K-steps plus the norm step, each an
    MMA of 128 references x Rb candidate rows x 16 (Rb = the union's rows
    plus p - 1, rounded up to 16)."""
    h = (win - 1) // 2
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    rows = (ty - 1) * s + 2 * h + 1
    cols = (tx - 1) * s + 2 * h + 1
    Rb = (rows + p - 1 + 15) // 16 * 16
    tiles = -(-ny // ty) * -(-nx // tx)
    mmas_per_col = products * (p * p // 16) + 1
    return float(tiles * cols * mmas_per_col * 2 * 128 * Rb * 16)


# ---------------------------------------------------------------- distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle timing

def cpu_oracle_rate(seconds: float, images_seed: int, threads: int = 0):
    """Oracle (as it stands) on whole 512^2 images, `threads` host cores (0: all),
    ~`seconds` of work."""
    from oracle import oracle as O
    from paper_2006_13714_gb300 import synth
    threads = threads or O.max_threads()
    refs = 0
    t0 = time.perf_counter()
    n = 0
    while True:
        img = synth.gray(WL["H"], WL["W"], WL["sigma"], images_seed + n, np.float32)
        t1 = time.perf_counter()
        idx, _ = O.match(img, WL["patch"], WL["window"], WL["stride"], WL["K"], threads=threads)
        refs += idx.shape[0]
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
        del t1
    el = time.perf_counter() - t0
    return refs / el, threads, n, el


# ---------------------------------------------------------------- reference arm

def run_reference(args, world, rank, dist):
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2006_13714_gb300 import synth
    threads = O.max_threads()
    ny, nx = (WL["H"] - WL["patch"]) // WL["stride"] + 1, (WL["W"] - WL["patch"]) // WL["stride"] + 1
    n_refs = ny * nx
    # bounded sample per step: a seeded quarter of one image's references
    per_step = n_refs // 4
    rng = np.random.default_rng(SEED_BASE)
    imgs = [synth.gray(WL["H"], WL["W"], WL["sigma"], SEED_BASE + i, np.float32) for i in range(2)]
    samples = [np.sort(rng.choice(n_refs, size=per_step, replace=False)).astype(np.int32)
               for _ in range(2)]
    for w in range(args.warmup):
        O.match(imgs[w % 2], WL["patch"], WL["window"], WL["stride"], WL["K"],
                refs=samples[w % 2], threads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.match(imgs[k % 2], WL["patch"], WL["window"], WL["stride"], WL["K"],
                refs=samples[k % 2], threads=threads)
    el = time.perf_counter() - t0
    value = per_step * args.steps / el
    sample = f"{per_step} seeded references of one 512x512 float32 image per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ref_patches/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512x512 f32 grey, patch 8, stride 3, window 39, K 16",
                   "refs_per_step": per_step, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "ref_patches/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "ref_patches/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def profiled_counters(images_per_launch):
    """From the committed ncu summary of the tensor-core kernel (16-image
    capture): DRAM bytes (read + write) per launch, scaled by images per
    launch (the traffic is per image), and the tensor pipe's active
    percentage; (None, None) when the kernel source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "tc_match_kernel_512x512_f32_batch16.md")
    src = os.path.join(ROOT, "paper_2006_13714_gb300", "csrc", "selfconv_tc.cu")
    try:
        fields = dict(line.split(": ", 1) for line in open(path).read().splitlines()
                      if line.startswith(("traffic_bytes_per_image:", "source_sha256_16:",
                                          "tensor_pipe_active_pct:")))
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if fields.get("source_sha256_16", "").strip() != digest:
            return None, None
        pipe = float(fields["tensor_pipe_active_pct"]) if "tensor_pipe_active_pct" in fields else None
        return float(fields["traffic_bytes_per_image"]) * images_per_launch, pipe
    except (OSError, KeyError, ValueError):
        return None, None


def serve_stream(ctx, pkg, synth, dev, n=2000, seed=SEED_BASE + 55, side=2048):
    """Serving workload: n seeded requests (uint8 / float32, C 1 or 4, sides
    uniform in [128, side], patch 8 (stride 3) or 7 (stride 4), window 39 or
    61, K 16 / 32 / 70) admitted under the context's 40 GB workspace budget,
    with every input and output resident on the device.  Each request's
    image is a seeded crop of one of four side x side synthetic base images
    (one per dtype and channel count), cut on the device.  Three passes over
    the same requests:
      serial     bm_match one request at a time (synchronised after each);
      saturated  every request submitted at once: aggregate ref-patches/s;
      poisson    submitted at seeded Poisson arrival times at 0.7 x the
                 serial request rate: latency = completion seen by polling
                 minus arrival, p50 / p99.
    """
    import torch
    draws = synth.serve_requests(2000, seed, 1.0)[:n]
    bases = {
        ("u8", 1): synth.gray(side, side, 20.0, seed + 1, np.uint8),
        ("f32", 1): synth.gray(side, side, 20.0, seed + 2, np.float32),
        ("u8", 4): synth.rgbnir(side, side, 20.0, seed + 3),
        ("f32", 4): synth.rgbnir(side, side, 20.0, seed + 4).astype(np.float32),
    }
    dbases = {k: torch.from_numpy(v).to(dev) for k, v in bases.items()}
    jobs = []
    refs = []
    for d in draws:
        H = min(side, d["H"])
        W = min(side, d["W"])
        rng = np.random.default_rng(d["seed"])
        y0 = int(rng.integers(0, side - H + 1))
        x0 = int(rng.integers(0, side - W + 1))
        t = dbases[(d["dtype"], d["C"])][y0:y0 + H, x0:x0 + W].contiguous()
        idx, dist_t = ctx.outputs(t, d["patch"], d["stride"], d["K"])
        req = pkg.Context.request(t, d["patch"], d["window"], d["stride"], d["K"], idx, dist_t)
        jobs.append((t, idx, dist_t, req, d))
        ny, nx = pkg.bm_num_refs(H, W, d["patch"], d["stride"])
        refs.append(ny * nx)
    del dbases
    torch.cuda.synchronize(dev)
    total_refs = float(sum(refs))
    in_bytes = sum(j[0].numel() * j[0].element_size() for j in jobs)
    out_bytes = sum(j[1].numel() * 4 + j[2].numel() * 4 for j in jobs)

    def wait(ticket, limit=300.0):
        t_end = time.perf_counter() + limit
        while True:
            if time.perf_counter() > t_end:
                raise RuntimeError("serving request did not finish")
            done, st = ctx.poll(ticket)
            if done:
                if st != 0:
                    raise pkg.BMError(st, "serving request failed")
                return
            time.sleep(0.00005)

    # warm-up: one request of every class (kernel loads, workspaces)
    seen = set()
    for j in jobs:
        d = j[4]
        key = (d["dtype"], d["C"], d["patch"], d["window"], d["K"])
        if key not in seen:
            seen.add(key)
            wait(ctx.submit(j[3]))
    torch.cuda.synchronize(dev)

    # serial: bm_match one request at a time
    stream = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    for t, idx, dist_t, req, d in jobs:
        ctx.match(t, d["patch"], d["window"], d["stride"], d["K"], out=(idx, dist_t), stream=stream)
        stream.synchronize()
    serial_s = time.perf_counter() - t0

    # saturated: everything submitted at once
    t0 = time.perf_counter()
    tks = [ctx.submit(j[3]) for j in jobs]
    for tk in tks:
        wait(tk)
    sat_s = time.perf_counter() - t0

    # Poisson arrivals at 0.7 x the serial request rate
    serial_rps = n / serial_s
    rate = 0.7 * serial_rps
    arrivals = np.cumsum(np.random.default_rng(seed + 9).exponential(1.0 / rate, size=n))
    lat = [None] * n
    tickets = {}
    start = time.perf_counter()
    i = 0
    while i < n or tickets:
        now = time.perf_counter() - start
        if now > arrivals[-1] + 300.0:
            raise RuntimeError("serving stream did not finish in 300 s after the last arrival")
        while i < n and arrivals[i] <= now:
            tickets[ctx.submit(jobs[i][3])] = i
            i += 1
        for tk in list(tickets):
            done, st = ctx.poll(tk)
            if done:
                if st != 0:
                    raise pkg.BMError(st, "serving request failed")
                k = tickets.pop(tk)
                lat[k] = (time.perf_counter() - start) - arrivals[k]
        time.sleep(0.00005)
    wall = time.perf_counter() - start
    lat_ms = np.array(lat) * 1e3
    cls = {}
    for k, (t, idx, dist_t, req, d) in enumerate(jobs):
        key = "f32_c4_p8" if (d["dtype"], d["C"], d["patch"]) == ("f32", 4, 8) else "other"
        cls.setdefault(key, []).append(lat_ms[k])
    out = {
        "requests": n, "ref_patches": total_refs,
        "serial": {"seconds": serial_s, "ref_patches_per_s": total_refs / serial_s,
                   "req_per_s": serial_rps, "api": "bm_match, synchronised after each"},
        "saturated": {"seconds": sat_s, "ref_patches_per_s": total_refs / sat_s,
                      "vs_serial": serial_s / sat_s, "api": "bm_submit all, bm_poll"},
        "poisson": {"rate_req_per_s": rate, "p50_ms": float(np.percentile(lat_ms, 50)),
                    "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
                    "seconds": wall, "ref_patches_per_s": total_refs / wall},
        "p99_ms_by_class": {k: float(np.percentile(v, 99)) for k, v in cls.items()},
        "resident_bytes": {"inputs": in_bytes, "outputs": out_bytes},
        "workload": f"{n} seeded requests (of the 2000-request stream): u8/f32, C 1/4, sides U[128,{side}], patch 8 (s 3) / 7 (s 4), "
                    "window 39/61, K 16/32/70, 40 GB workspace budget; images are seeded crops "
                    f"of four {side}x{side} synthetic base images",
    }
    for j in jobs:
        del j
    return out


def tiny_row(ctx, pkg, synth, dev, stream):
    """The tiny plain-method configuration: one 64x64 uint8 image, patch 8,
    stride 1 (all 57 x 57 references), window 21, K 16, matched alone
    through bm_match (its windows split across CTAs: window_split parts per
    tile) -- latency from CUDA events, median of 50 calls after warm-up."""
    import torch
    img = torch.from_numpy(synth.gray(64, 64, 25.0, SEED_BASE + 1, np.uint8)).to(dev)
    idx, dist_t = ctx.outputs(img, 8, 1, 16)
    for _ in range(5):
        ctx.match(img, 8, 21, 1, 16, out=(idx, dist_t), stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    for _ in range(50):
        e0.record(stream)
        ctx.match(img, 8, 21, 1, 16, out=(idx, dist_t), stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        lat.append(e0.elapsed_time(e1))
    med = statistics.median(lat)
    e0.record(stream)
    for _ in range(20):
        ctx.match_direct(img, 8, 21, 1, 16, out=(idx, dist_t), stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    d_ms = e0.elapsed_time(e1) / 20
    return {"workload": "64x64 uint8 grey, patch 8, stride 1, window 21, K 16, alone (bm_match)",
            "latency_ms": {"median": med, "min": min(lat)},
            "ref_patches_per_s": 57 * 57 / (med / 1e3),
            "window_split": pkg.bm_window_split(64, 64, 1, pkg.BM_U8, 8, 21, 1, 16),
            "direct_fp32_gpu_ms": d_ms}


def batch_row(ctx, pkg, dev, nps, p, win, s, K, label, peaks, steps=5, n_direct=None):
    """Throughput of one batch workload through bm_match_batch (the graph-
    captured persistent launches): ref-patches/s, useful cross-term TMAC/s
    (pairs x p*p*C), the tensor-core kernel's share and its algorithmic
    fraction of the bf16 peak, and the plain FP32 direct kernel on (a prefix
    of) the same batch."""
    import torch
    stream = torch.cuda.Stream(dev)
    imgs, outs, reqs, nref = [], [], [], []
    pairs_mac = 0
    for a in nps:
        t = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        idx, dist_t = ctx.outputs(t, p, s, K)
        imgs.append(t)
        outs.append((idx, dist_t))
        reqs.append(pkg.Context.request(t, p, win, s, K, idx, dist_t))
        H, W = a.shape[0], a.shape[1]
        C = 1 if a.ndim == 2 else a.shape[2]
        ny, nx = pkg.bm_num_refs(H, W, p, s)
        nref.append(ny * nx)
        pairs_mac += useful_pairs(H, W, p, win, s) * p * p * C
    refs = sum(nref)
    for _ in range(3):
        ctx.match_batch(reqs, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.match_batch(reqs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    ctx.timing(reset=True)
    ctx.set_timing(True)
    ctx.match_batch(reqs, stream=stream)
    torch.cuda.synchronize(dev)
    ctx.set_timing(False)
    tm = ctx.timing(reset=True)
    tc = tm["tc"]
    peak = peaks.get("bf16_tflops_sustained") or 1700.0
    tc_tflops = 2.0 * pairs_mac / (tc["ms"] / 1e3) / 1e12 if tc["ms"] > 0 else None
    nd = len(imgs) if n_direct is None else min(n_direct, len(imgs))
    e0.record(stream)
    for i in range(nd):
        ctx.match_direct(imgs[i], p, win, s, K, out=outs[i], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    d_ms = e0.elapsed_time(e1)
    d_refs = sum(nref[:nd])
    direct_rate = d_refs / (d_ms / 1e3)
    return {
        "workload": label, "images": len(nps), "ms_per_batch": ms,
        "ref_patches_per_s": refs / (ms / 1e3), "useful_tmac_per_s": pairs_mac / (ms / 1e3) / 1e12,
        "tc": {"launches": tc["launches"], "ms": tc["ms"], "share": tc["ms"] / max(1e-9, sum(v["ms"] for v in tm.values())),
               "algorithmic_tflops": tc_tflops,
               "frac_of_bf16": (tc_tflops / peak) if tc_tflops else None,
               "peak_source": "of measured (bf16 sustained)" if peaks.get("bf16_tflops_sustained") else "of fallback"},
        "stage_ms": {k: v["ms"] for k, v in tm.items() if v["launches"]},
        "direct_fp32_gpu": {"images": nd, "ref_patches_per_s": direct_rate,
                            "speedup": (refs / (ms / 1e3)) / direct_rate},
    }


def groups_throughput(ctx, imgs, outs, peaks, stream, dev, n=16):
    """Patch-group gather and reconstruction (the steps on either side of the
    matching, §IV) on n images of the workload, from their matches: CUDA
    events on the launch stream; every image's groups are written before the
    first is read back, so the reconstruction reads them from HBM."""
    import torch
    H, W, p, s, K = WL["H"], WL["W"], WL["patch"], WL["stride"], WL["K"]
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    n = min(n, len(imgs))
    gbufs = [torch.empty((ny * nx, K, p * p), dtype=torch.float32, device=dev) for _ in range(n)]
    obufs = [(torch.empty((H, W, 1), dtype=torch.float32, device=dev),
              torch.empty((H, W), dtype=torch.float32, device=dev)) for _ in range(n)]
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    times = []
    for rep in range(4):  # 1 warm-up + 3 timed
        e[0].record(stream)
        for i in range(n):
            ctx.gather_groups(imgs[i], p, outs[i][0], ny, nx, out=gbufs[i], stream=stream)
        e[1].record(stream)
        for i in range(n):
            ctx.aggregate(gbufs[i], outs[i][0], H, W, 1, p, ny, nx, out=obufs[i], stream=stream)
        e[2].record(stream)
        torch.cuda.synchronize(dev)
        if rep:
            times.append((e[0].elapsed_time(e[1]) / n, e[1].elapsed_time(e[2]) / n))
    g_ms = min(t[0] for t in times)
    a_ms = min(t[1] for t in times)
    group_bytes = ny * nx * K * p * p * 4
    idx_bytes = ny * nx * K * 4
    g_alg = group_bytes + idx_bytes + H * W * 4           # write groups, read idx + image
    a_alg = group_bytes + idx_bytes + H * W * 4 * 2       # read groups + idx, write image + weights
    peak = peaks.get("hbm_gbs")
    gbs_g, gbs_a = g_alg / (g_ms / 1e3) / 1e9, a_alg / (a_ms / 1e3) / 1e9
    return {"images": n, "gather_us_per_image": 1e3 * g_ms, "aggregate_us_per_image": 1e3 * a_ms,
            "gather_bytes_per_image": g_alg, "aggregate_bytes_per_image": a_alg,
            "gather_GBps": gbs_g, "aggregate_GBps": gbs_a,
            "hbm_peak_GBps": peak, "peak_source": "of measured (copy)" if peak else None,
            "gather_frac": gbs_g / peak if peak else None,
            "aggregate_frac": gbs_a / peak if peak else None,
            "groups_per_image": ny * nx, "layout": "float32 [refs][K][p*p]"}


NLM_B = 283.0  # b of Eq. equ:nlm for the 512^2, sigma 25, 8x8 workload: d / b^2 ~ 1 for similar patches


def nlm_throughput(ctx, imgs, stream, dev, pairs, n=16):
    """Non-local means (Eq. equ:nlm) on n images of the workload: full-window
    weights and patch estimates, CUDA events on the launch stream.  Roofline:
    ALU (FP32), 4 p^2 C FLOP per (reference, candidate) pair against the
    nominal FP32 FMA rate of 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz."""
    import torch
    H, W, p, win, s = WL["H"], WL["W"], WL["patch"], WL["window"], WL["stride"]
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    n = min(n, len(imgs))
    outs = [(torch.empty((ny * nx, p * p), dtype=torch.float32, device=dev),
             torch.empty((ny * nx,), dtype=torch.float32, device=dev)) for _ in range(n)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for rep in range(3):  # 1 warm-up + 2 timed
        e0.record(stream)
        for i in range(n):
            ctx.nlm(imgs[i], p, win, s, NLM_B, out=outs[i], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rep:
            times.append(e0.elapsed_time(e1) / n)
    ms = min(times)
    flop = 4.0 * pairs * p * p
    peak = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = flop / (ms / 1e3) / 1e12
    return {"images": n, "us_per_image": 1e3 * ms, "ref_patches_per_s": ny * nx / (ms / 1e3),
            "b": NLM_B, "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                                    "unit": "TFLOP/s", "frac": achieved / peak,
                                    "peak_source": "nominal FP32 FMA rate (152 SMs x 128 lanes x 2.07 GHz)",
                                    "algorithmic_flop_per_image": flop}}


def ncc_throughput(ctx, imgs, stream, dev, pairs, n=16):
    """NCC block matching (Eq. equ:cor) on n images of the workload (K 16),
    CUDA events on the launch stream.  Roofline: ALU (FP32) against the
    nominal FP32 FMA rate; the work is the cross term, 2 p^2 C FLOP per pair,
    plus one norm (2 p^2 C FLOP) per patch position of the image: a
    candidate's norm does not depend on the reference, and the kernel forms
    it once."""
    import torch
    H, W, p, win, s, K = WL["H"], WL["W"], WL["patch"], WL["window"], WL["stride"], WL["K"]
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    n = min(n, len(imgs))
    outs = [(torch.empty((ny * nx, K), dtype=torch.int32, device=dev),
             torch.empty((ny * nx, K), dtype=torch.float32, device=dev)) for _ in range(n)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for rep in range(3):
        e0.record(stream)
        for i in range(n):
            ctx.match_ncc(imgs[i], p, win, s, K, out=outs[i], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rep:
            times.append(e0.elapsed_time(e1) / n)
    ms = min(times)
    # the same on uint8 stand-ins (the tensor-core form: exact cross terms on
    # tcgen05, a pool of 32 ranked exactly)
    u8 = [torch.clamp(imgs[i], 0, 255).round().to(torch.uint8).contiguous() for i in range(n)]
    times8 = []
    for rep in range(3):
        e0.record(stream)
        for i in range(n):
            ctx.match_ncc(u8[i], p, win, s, K, out=outs[i], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rep:
            times8.append(e0.elapsed_time(e1) / n)
    ms8 = min(times8)
    flop = 2.0 * pairs * p * p + 2.0 * (H - p + 1) * (W - p + 1) * p * p
    peak = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = flop / (ms / 1e3) / 1e12
    return {"images": n, "us_per_image": 1e3 * ms, "ref_patches_per_s": ny * nx / (ms / 1e3),
            "uint8_tensor_core": {"us_per_image": 1e3 * ms8, "ref_patches_per_s": ny * nx / (ms8 / 1e3),
                                  "useful_tmac_per_s": pairs * p * p / (ms8 / 1e3) / 1e12},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "peak_source": "nominal FP32 FMA rate (152 SMs x 128 lanes x 2.07 GHz)",
                         "algorithmic_flop_per_image": flop}}


def match3d_throughput(ctx, synth, dev, stream, n=4):
    """3-D block matching across channels (§IV) on n seeded 512 x 512 x 4
    uint8 RGB-NIR stand-ins: patch 8 x 8 x depth 2, window 39, stride 3,
    K 16, three channel offsets.  This shape runs the integer kernel (the
    Self-Convolution identity with dp4a on packed bytes).  Roofline: ALU,
    the cross term's p*p*depth byte multiply-accumulates per (reference,
    candidate) pair against dp4a issued by every scheduler every clock (four
    byte MACs per lane).  The FP32-equivalent rate (3 FLOP per element of the
    direct form) is reported beside it."""
    import torch
    H = W = 512
    p, d, win, s, K = 8, 4 // 2, WL["window"], WL["stride"], WL["K"]
    imgs = [torch.from_numpy(synth.rgbnir(H, W, 20.0, SEED_BASE + 300 + i)).to(dev) for i in range(n)]
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    nc = 4 - d + 1
    outs = [(torch.empty((ny * nx * nc, K), dtype=torch.int32, device=dev),
             torch.empty((ny * nx * nc, K), dtype=torch.int32, device=dev)) for _ in range(n)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for rep in range(3):
        e0.record(stream)
        for i in range(n):
            ctx.match_3d(imgs[i], p, d, win, s, K, out=outs[i], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if rep:
            times.append(e0.elapsed_time(e1) / n)
    ms = min(times)
    pairs = useful_pairs(H, W, p, win, s) * nc * nc
    macs = float(pairs * p * p * d)
    peak = 152 * 4 * 32 * 4 * 2.07e9 / 1e12
    achieved = macs / (ms / 1e3) / 1e12
    return {"images": n, "workload": "512x512x4 u8, patch 8x8x2, window 39, stride 3, K 16",
            "us_per_image": 1e3 * ms, "refs_per_s": ny * nx * nc / (ms / 1e3),
            "fp32_equivalent_tflops": 3.0 * macs / (ms / 1e3) / 1e12,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tmac/s",
                         "frac": achieved / peak,
                         "peak_source": "nominal dp4a issue rate (152 SMs x 4 schedulers x 32 lanes"
                                        " x 4 byte MACs x 2.07 GHz)",
                         "algorithmic_byte_macs_per_image": macs}}


def time_row_oracles(img, idx, synth, groups, nlm, ncc, m3d, seconds=1.0):
    """The oracles of the rows beside block matching, as they stand, on bounded
    seeded samples of the same workloads (one host thread, numpy): each result
    dict gains "cpu_oracle" with the rate in the row's unit and the sample."""
    from oracle import bm3d as O3
    from oracle import groups as OG
    from oracle import ncc as ON
    from oracle import nlm as ONL
    H, W, p, win, s, K = WL["H"], WL["W"], WL["patch"], WL["window"], WL["stride"], WL["K"]
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    rng = np.random.default_rng(SEED_BASE + 900)

    def rate(fn, unit_count, what):
        n, t0 = 0, time.perf_counter()
        while True:
            fn()
            n += 1
            el = time.perf_counter() - t0
            if el >= seconds:
                return {"value": unit_count * n / el, "cores": 1, "kind": "oracle",
                        "sample": f"{what}, {n} run(s) in {el:.1f} s"}

    if groups:
        sel = np.sort(rng.choice(ny * nx, size=1000, replace=False))
        sub = idx[sel]
        g = OG.gather_groups(img, p, sub)
        groups["cpu_oracle"] = {
            "gather": rate(lambda: OG.gather_groups(img, p, sub), len(sel),
                           "groups of 1000 seeded references of one 512x512 image (groups/s)"),
            "aggregate": rate(lambda: OG.aggregate(g, sub, H, W, 1, p), len(sel),
                              "reconstruction from those 1000 groups (groups/s)")}
    if nlm:
        refs = np.sort(rng.choice(ny * nx, size=100, replace=False))
        nlm["cpu_oracle"] = rate(lambda: ONL.nlm(img, p, win, s, NLM_B, refs=refs), len(refs),
                                 "100 seeded references of one 512x512 image (ref_patches/s)")
    if ncc:
        refs = np.sort(rng.choice(ny * nx, size=20, replace=False))
        ncc["cpu_oracle"] = rate(lambda: ON.match_ncc(img, p, win, s, K, refs=refs), len(refs),
                                 "20 seeded references of one 512x512 image (ref_patches/s)")
    if m3d:
        img4 = synth.rgbnir(H, W, 20.0, SEED_BASE + 300)
        refs = np.sort(rng.choice(ny * nx * 3, size=20, replace=False))
        m3d["cpu_oracle"] = rate(lambda: O3.match_3d(img4, p, 2, win, s, K, refs=refs), len(refs),
                                 "20 seeded references of one 512x512x4 image (refs/s)")


def run_ours(args, world, rank, local, dist):
    import torch
    import paper_2006_13714_gb300 as pkg
    from paper_2006_13714_gb300 import synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    B = args.images
    H, W, p, win, s, K = WL["H"], WL["W"], WL["patch"], WL["window"], WL["stride"], WL["K"]
    ny, nx = (H - p) // s + 1, (W - p) // s + 1
    nR = ny * nx
    pairs = useful_pairs(H, W, p, win, s)
    macs_per_image = pairs * p * p * WL["C"]

    ctx = pkg.Context(local)
    base = [synth.gray(H, W, WL["sigma"], SEED_BASE + 7919 * rank + i, np.float32) for i in range(8)]
    imgs, outs, reqs = [], [], []
    for i in range(B):
        # distinct images: seeded base images with a per-image offset and flip pattern
        a = base[i % 8]
        a = a[::-1] if (i // 8) % 2 else a
        a = a[:, ::-1] if (i // 16) % 2 else a
        t = torch.from_numpy(np.ascontiguousarray(a + float(i // 32))).to(dev)
        idx, dist_t = ctx.outputs(t, p, s, K)
        imgs.append(t)
        outs.append((idx, dist_t))
        reqs.append(pkg.Context.request(t, p, win, s, K, idx, dist_t))
    # a stream of our own: repeated batches replay one captured CUDA graph
    stream = torch.cuda.Stream(dev)

    def step():
        ctx.match_batch(reqs, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    st0 = ctx.stats()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    elapsed_ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(dist, elapsed_ms, dev)
    # per-kernel device times: the same steps again with the library's stage
    # events (CUDA events on the launch stream around every kernel launch)
    ctx.timing(reset=True)
    ctx.set_timing(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    ctx.set_timing(False)
    tm = ctx.timing(reset=True)
    total_refs = nR * B * args.steps * world
    value = total_refs / (elapsed_ms / 1e3)
    st1 = ctx.stats()

    if args.minimal:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "ref_patches/s",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": elapsed_ms / args.steps, "minimal": True,
                              "tc_ms_per_launch": tm["tc"]["ms"] / max(1, tm["tc"]["launches"])}),
                  flush=True)
        ctx.close()
        return 0

    staged_ms = sum(v["ms"] for v in tm.values()) / args.steps

    # roofline of the dominant kernel (tensor-core cross term + top-K)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    tc = tm["tc"]
    n_tc = max(1, tc["launches"])
    imgs_per_launch = B * args.steps / n_tc  # one persistent launch covers up to 64 images
    tc_ms = tc["ms"] / n_tc
    flop_per_launch = 2.0 * macs_per_image * imgs_per_launch
    achieved = flop_per_launch / (tc_ms / 1e3) / 1e12  # algorithmic TFLOP/s per launch
    issued_per_launch = tc_issued_flop_per_image(H, W, p, win, s) * imgs_per_launch
    peak = peaks.get("bf16_tflops_sustained")
    peak_src = "of measured (bf16 sustained)"
    if peak is None:
        peak, peak_src = 1700.0, "of fallback (bf16 sustained)"
    traffic, pipe_pct = profiled_counters(imgs_per_launch)
    stage_share = {k: round(v["ms"] / max(1e-9, sum(x["ms"] for x in tm.values())), 4)
                   for k, v in tm.items() if v["launches"]}

    # plain FP32 CUDA-core baseline on the same batch
    n_direct = min(B, 32)
    e0.record(stream)
    for i in range(n_direct):
        ctx.match_direct(imgs[i], p, win, s, K, out=outs[i], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    direct_ms_img = e0.elapsed_time(e1) / n_direct
    tc_ms_img = elapsed_ms / (B * args.steps)

    # single-image latency through bm_match
    lat = []
    for _ in range(20):
        e0.record(stream)
        ctx.match(imgs[0], p, win, s, K, out=outs[0], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        lat.append(e0.elapsed_time(e1))

    # end to end through the host-buffer batch entry point (pinned host memory):
    # every step copies its images in and its results out inside the timed region
    n_e2e = min(B, 64)
    host_imgs = [imgs[i].cpu().pin_memory() for i in range(n_e2e)]
    h_outs = [(torch.empty((nR, K), dtype=torch.int32).pin_memory(),
               torch.empty((nR, K), dtype=torch.float32).pin_memory()) for _ in range(n_e2e)]
    h_reqs = (pkg.bm_request * n_e2e)(*[
        pkg.bm_request(hi.data_ptr(), H, W, 1, pkg.BM_F32, p, win, s, K, o[0].data_ptr(), o[1].data_ptr())
        for hi, o in zip(host_imgs, h_outs)])
    rc = pkg.bm_match_host_batch(ctx.handle, h_reqs, n_e2e)  # warm-up (staging, workspaces)
    if rc != 0:
        raise pkg.BMError(rc, pkg.bm_last_error(ctx.handle))
    e2e_steps = 3
    torch.cuda.synchronize(dev)
    barrier(dist)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = pkg.bm_match_host_batch(ctx.handle, h_reqs, n_e2e)
        if rc != 0:
            raise pkg.BMError(rc, pkg.bm_last_error(ctx.handle))
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(dist, e2e_s, dev)
    e2e_value = nR * n_e2e * e2e_steps * world / e2e_s

    cfg3 = batch_row(ctx, pkg, dev, [synth.gray(Hh, Ww, sg, SEED_BASE + 300 + i, np.float32)
                                     for i, (Hh, Ww, sg) in enumerate(synth.batch_sizes(32, SEED_BASE + 3))],
                     7, 61, 4, 70, "32 float32 grey images of seeded uneven sizes (256^2 .. 1024^2, "
                     "sigma 15/25/50), patch 7, stride 4, window 61, K 70", peaks, n_direct=8)
    rgbnir4 = [synth.rgbnir(1024, 1024, 20.0, SEED_BASE + 400 + i) for i in range(4)]
    # 16 distinct images: four seeded stacks, each also flipped three ways
    rgbnir16 = [np.ascontiguousarray(a[::fy, ::fx]) for a in rgbnir4 for fy, fx in ((1, 1), (-1, 1), (1, -1), (-1, -1))]
    cfg4 = batch_row(ctx, pkg, dev, rgbnir16,
                     8, 39, 3, 32, "16 uint8 RGB-NIR 1024x1024x4 images, patch 8, stride 3, window 39, K 32",
                     peaks, n_direct=4)
    tiny = tiny_row(ctx, pkg, synth, dev, stream)
    serve = serve_stream(ctx, pkg, synth, dev, n=args.serve_requests) if not args.no_serve else None
    groups = groups_throughput(ctx, imgs, outs, peaks, stream, dev)
    nlm = nlm_throughput(ctx, imgs, stream, dev, pairs)
    ncc = ncc_throughput(ctx, imgs, stream, dev, pairs)
    m3d = match3d_throughput(ctx, synth, dev, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        time_row_oracles(base[0], outs[0][0].cpu().numpy(), synth, groups, nlm, ncc, m3d)
        rate, cores, n_img, el = cpu_oracle_rate(args.cpu_seconds, SEED_BASE + 100)
        rate1, _, n1, el1 = cpu_oracle_rate(min(args.cpu_seconds, 5.0), SEED_BASE + 200, threads=1)
        cpu = {"value": rate, "unit": "ref_patches/s", "cores": cores, "kind": "oracle",
               "sample": f"{n_img} whole 512x512 float32 images ({el:.1f} s, all host cores)",
               "single_thread": {"value": rate1, "unit": "ref_patches/s",
                                 "sample": f"{n1} whole 512x512 float32 image(s) ({el1:.1f} s, one core)"}}

    launches_per_step = sum(v["launches"] for v in tm.values()) / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "ref_patches/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "512x512 f32 grey, patch 8, stride 3, window 39, K 16",
                   "images_per_step_per_gpu": B, "refs_per_image": nR,
                   "useful_pairs_per_image": pairs, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "ref_patches/s",
                "h2d_bytes_per_step": H * W * 4 * n_e2e,
                "d2h_bytes_per_step": nR * K * 8 * n_e2e,
                "images_per_step": n_e2e, "api": "bm_match_host_batch (pinned host buffers)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "tc_match_kernel",
                     "peak_source": peak_src, "tc_ms_per_launch": tc_ms,
                     "algorithmic_flop_per_launch": flop_per_launch,
                     "issued_flop_per_launch": issued_per_launch,
                     "issued_frac": issued_per_launch / (tc_ms / 1e3) / 1e12 / peak,
                     "images_per_launch": imgs_per_launch,
                     "tensor_pipe_active_ncu": pipe_pct,
                     "tensor_pipe_note": "sm__pipe_tensor_cycles_active (pct of peak, active) of one "
                                         "16-image launch, ncu; issued MMAs, not the algorithmic fraction"},
        "cpu_baseline": cpu,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk,
        "stage_ms_share": stage_share,
        "kernel_ms_per_step_with_stage_events": staged_ms,
        "config1_tiny": tiny,
        "config3_batch": cfg3,
        "config4_rgbnir": cfg4,
        "serve": serve,
        "groups": groups,
        "nlm": nlm,
        "ncc": ncc,
        "match_3d": m3d,
        "direct_fp32_gpu": {"ms_per_image": direct_ms_img, "ms_per_image_selfconv": tc_ms_img,
                            "speedup": direct_ms_img / tc_ms_img},
        "single_image_latency_ms": {"min": min(lat), "median": statistics.median(lat),
                                    "window_split": pkg.bm_window_split(H, W, 1, pkg.BM_F32, p, win, s, K)},
        "stats": {k: st1[k] - st0[k] for k in ("rerank_overflow", "fp64_rechecks",
                                               "bound_violations", "tc_jobs")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = parse_args()
    world, rank, local, dist = dist_setup(args)
    try:
        if args.impl == "reference":
            rc = run_reference(args, world, rank, dist)
        else:
            rc = run_ours(args, world, rank, local, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
