#!/usr/bin/env python
"""Benchmark of the XPCS correlation hot path on one GB300 (replicas on N GPUs).

Workload (512x512 detector, T = 10,000 frames, uint16 Poisson counts of mean 0.1 from
AR(1) speckle with D = 5e-4, 36 equal-width q-rings, basis of rank k = 64 fit in FP64 on
the first 1000 frames).  One step = the compressed path over the whole series:
encode A = X V_K (Eq. 7) + two-time C_q for every ring from the coefficients
(Eq. 10 with ring factors, C stored as the float32 lower triangle) + g2.  The exact raw
path (Eq. 1-2 on integer counts) is timed in the same run for the speed-up.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64 oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(H=512, W=512, T=10000, dtype="uint16", mean=0.1, D=5e-4, n_q=36, k=64, n_fit=1000,
                seed=20356002)
# smaller case of the same kernels for profiler captures: inputs and outputs still exceed L2
SMALL = dict(H=256, W=256, T=4096, dtype="uint16", mean=0.1, D=2e-3, n_q=16, k=64, n_fit=500, seed=20356012)
WORKLOAD_NAME = ("512x512 detector, T=10000 frames, uint16 Poisson AR(1) speckle mean 0.1 D=5e-4, "
                 "36 q-rings, k=64 basis fit on the first 1000 frames; step = encode + two-time (C stored, "
                 "float32 lower triangle) + g2")
METRIC = "frames/s correlated (compressed vs exact raw path) at stated err; p99 frame latency"
# grouped batching: 64 uneven ring-plus-sector masks (100 .. 20000 px) on a 1 Mpx detector
GROUPED = dict(H=1024, W=1024, T=20000, dtype="uint16", mean=0.05, D=5e-4, n_q=64, min_px=100, max_px=20000,
               k=128, n_fit=1000, seed=20356003)
GROUPED_NAME = ("1024x1024 detector, 64 ring-plus-sector masks of 100..20000 px (246813 masked px, X holds "
                "those only), T=20000 frames, uint16 Poisson AR(1) speckle mean 0.05 D=5e-4, k=128 basis fit "
                "on the first 1000 frames; step = encode + two-time with g2 fused (C not stored: 102 GB)")
# smaller case of the grouped kernels for profiler captures (X and the operands exceed L2)
GROUPED_SMALL = dict(H=512, W=512, T=4096, dtype="uint16", mean=0.05, D=5e-4, n_q=64, min_px=100, max_px=3000,
                     k=128, n_fit=500, seed=20356013)
# multi-stream serving: four detectors of different sizes at their own rates, 100 q-rings
# each, coefficient histories capped at 2e5 frames, one server with continuous batching
SERVING = dict(streams=[dict(H=1536, W=2048, rate_hz=2000.0, k=256, D=1e-4),
                        dict(H=1024, W=1024, rate_hz=10000.0, k=128, D=4.64e-4),
                        dict(H=512, W=512, rate_hz=50000.0, k=128, D=2.15e-3),
                        dict(H=256, W=256, rate_hz=100000.0, k=64, D=1e-2)],
               n_q=100, history=200000, max_batch=128, mean=0.02, n_fit=1000, pool=128, seed=20356005)
# online stream: one 1 Mpx detector at 10 kHz, history of 1e5 frames
STREAM = dict(H=1024, W=1024, dtype="uint16", mean=0.02, D=5e-4, n_q=36, k=128, n_fit=1000, history=100000,
              rate_hz=10000.0, pool=2048, max_batch=128, seed=20356003)
STREAM_NAME = ("1024x1024 uint16 stream, Poisson AR(1) speckle mean 0.02 D=5e-4, 36 q-rings, k=128 basis fit on "
               "a 1000-frame calibration run, history 100000 frames, frames arriving at 10 kHz in device memory")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], bf16_tflops=d["bf16_tflops"],
                    bf16_tflops_sustained=d.get("bf16_tflops_sustained"), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="fallback")


# ---------------------------------------------------------------- clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.t_lo = self.t_hi = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def mark(self, lo, hi):
        self.t_lo, self.t_hi = lo, hi

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.samples:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((t, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        win = [r for r in rows if self.t_lo is not None and self.t_lo - 0.15 <= r[0] <= self.t_hi + 0.15] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in win for i, v in enumerate(r[3]) if v.lower() == "active"})
        sm = sorted(r[1] for r in win)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[2] for r in win), "reasons": reasons,
                "samples": len(win)}


# ---------------------------------------------------------------- distributed plumbing

def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if n_gpus > 0 else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def T_pad_of(T):
    return (T + 127) // 128 * 128


def rings_padded(rings):
    """Row length of the raw path's ring-sorted operand: every ring padded to 64 pixels."""
    return int(sum(max(1, (int(m) + 63) // 64) * 64 for m in rings.sizes()))


# ---------------------------------------------------------------- oracle timing (CPU)

def oracle_cpu(frames_host, qmap, wl, n_rings_sample=1, enc_frames=None):
    """Time the oracle on a bounded sample and extrapolate to the whole workload.

    Encode runs over `enc_frames` frames (all if None); the two-time + g2 runs for
    `n_rings_sample` rings at the full T.  Returns (frames/s, seconds, details).
    """
    import oracle as O

    T, n_q, k = wl["T"], wl["n_q"], wl["k"]
    t0 = time.perf_counter()
    B, _ = O.fit_basis(frames_host[: wl["n_fit"]], k)
    t_fit = time.perf_counter() - t0
    G, s, Mq = O.ring_factors(B, qmap, n_q)
    ne = T if enc_frames is None else enc_frames
    t0 = time.perf_counter()
    A = np.concatenate([O.encode(frames_host[i:i + 500], B) for i in range(0, ne, 500)])
    t_enc = (time.perf_counter() - t0) * (T / ne)
    t0 = time.perf_counter()
    for q in range(n_rings_sample):
        if ne < T:
            break
        Cq = O.twotime_from_gram(O.compressed_ring_gram(A, G[q]), A @ s[q], A @ s[q], Mq[q])
        O.g2_from_twotime(Cq)
        del Cq
    t_ring = (time.perf_counter() - t0) / max(1, n_rings_sample)
    total = t_enc + t_ring * n_q
    return T / total, total, dict(t_fit=t_fit, t_encode_full=t_enc, t_ring=t_ring, B=B, G=G, s=s, Mq=Mq, A=A)


def run_reference(args, wl):
    world, rank, local = dist_init(0)
    if rank != 0:
        return
    from synth import ring_qmap, speckle_counts

    import oracle as O

    # same workload, generated on the host (a prefix is enough for the sampled steps)
    qmap = ring_qmap(wl["H"], wl["W"], wl["n_q"])
    n_host = wl["n_fit"] + 200
    frames = speckle_counts(wl["H"], wl["W"], n_host, wl["mean"], wl["D"], wl["seed"], np.uint16)
    B, _ = O.fit_basis(frames[: wl["n_fit"]], wl["k"])
    G, s, Mq = O.ring_factors(B, qmap, wl["n_q"])
    T = wl["T"]
    rng = np.random.default_rng(0)

    def step():
        # bounded sample: encode 200 frames (scaled to T) + two-time and g2 of one ring
        # at the full T on coefficients of the same statistics (scaled to all rings)
        t0 = time.perf_counter()
        A = O.encode(frames[wl["n_fit"]:wl["n_fit"] + 200], B)
        t_enc = (time.perf_counter() - t0) * T / 200
        Af = A[rng.integers(0, 200, size=T)]
        t0 = time.perf_counter()
        q = int(rng.integers(0, wl["n_q"]))
        Cq = O.twotime_from_gram(O.compressed_ring_gram(Af, G[q]), Af @ s[q], Af @ s[q], Mq[q])
        O.g2_from_twotime(Cq)
        t_ring = time.perf_counter() - t0
        return t_enc + t_ring * wl["n_q"]

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    est = [step() for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    per_step = float(np.mean(est))
    value = T / per_step
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "impl": "CPU FP64 oracle (numpy)"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": "extrapolated: per step, oracle encode of 200 frames scaled to T=10000, "
                                   "plus oracle two-time + g2 of one ring at T=10000 scaled to 36 rings",
                         "wall_s": wall},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm

def run_ours(args, wl):
    import torch

    world, rank, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2407_20356_gb300 import xpcs as X
    from synth import ring_qmap
    from synth.speckle import TorchSpeckle

    H, W, T, n_q, k = wl["H"], wl["W"], wl["T"], wl["n_q"], wl["k"]
    M = H * W
    prec = args.prec
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    # ---- synthetic input, resident in HBM
    t0 = time.time()
    gen = TorchSpeckle(H, W, wl["mean"], wl["D"], wl["seed"] + rank, dtype=wl["dtype"], device=str(dev))
    Xd = torch.empty((T, M), dtype=torch.uint16, device=dev)
    for i in range(0, T, 1000):
        Xd[i:i + 1000].copy_(gen.next(min(1000, T - i)))
    del gen
    qmap = ring_qmap(H, W, n_q)
    torch.cuda.synchronize()
    t_gen = time.time() - t0

    ctx = X.Context(local, 0, stream.cuda_stream)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), M, n_q)
    t0 = time.time()
    basis = X.xpcs_fit_basis(ctx, rings, Xd, wl["n_fit"], k)
    t_fit = time.time() - t0

    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    C = torch.empty((n_q, T, T), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    ctx.set_async(True)

    def step(p=prec):
        X.xpcs_encode(ctx, basis, Xd, T, A)
        X.xpcs_twotime(ctx, basis, A, T, p, C_out=C, g2_out=g2, count_out=cnt)

    def timed(fn, K, Wm, profile=False, sampler=None):
        for _ in range(Wm):
            fn()
        ctx.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        if profile:
            ctx.profile_enable(True)
        n0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lo = time.time()
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        ctx.synchronize()
        torch.cuda.synchronize()
        hi = time.time()
        barrier(world)
        if sampler:
            sampler.mark(lo, hi)
        ms = e0.elapsed_time(e1) / K
        prof = ctx.profile() if profile else {}
        if profile:
            ctx.profile_enable(False)
        return ms, ctx.launch_count() - n0, prof

    # the two-time configuration for this shape, chosen by the library's autotuner
    X.xpcs_encode(ctx, basis, Xd, T, A)
    tuned = X.xpcs_autotune_twotime(ctx, basis, A, T, prec, C_out=C, g2_out=g2, count_out=cnt, reps=2)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ms, launches, prof = timed(step, args.steps, args.warmup, profile=True, sampler=sampler)
    if sampler:
        sampler.stop()
    ms = max_over_ranks(ms, world, dev)

    # ---- the same step captured once as a CUDA graph and replayed (one launch per step)
    X.xpcs_capture_begin(ctx)
    step()
    graph = X.xpcs_capture_end(ctx)
    graph_ms, graph_launches, _ = timed(graph.launch, args.steps, args.warmup)
    graph_ms = max_over_ranks(graph_ms, world, dev)
    graph_res = {"ms_per_step": graph_ms, "frames_per_s": world * T / (graph_ms * 1e-3),
                 "kernels_per_step": graph.kernels(), "gpu_launches": graph_launches}
    graph.close()

    # ---- g2 over the stored C of the last step (the standalone xpcs_g2 call): HBM-bound,
    # it reads the lower triangle once (C = 14.4 GB, far larger than L2)
    g2s = torch.empty_like(g2)
    cs = torch.empty_like(cnt)
    g2c_ms, _, g2c_prof = timed(lambda: X.xpcs_g2(ctx, C, n_q, T, g2s, cs), max(1, min(args.steps, 5)), 3,
                                profile=True)
    pk = peaks()
    g2c_bytes = n_q * T * (T + 1) // 2 * 4 + n_q * T * 16  # lower triangle read + g2 and counts written
    g2c_kern = {k_: v[0] / max(1, v[1]) for k_, v in g2c_prof.items()}
    g2c_k = g2c_kern.get("g2_from_C")
    g2_res = {"ms_per_call": g2c_ms, "kernels_ms": g2c_kern,
              "roofline": {"bound": "hbm", "kernel": "g2_from_C", "algorithmic_bytes": g2c_bytes,
                           "bytes_model": "lower triangle of C read once (float32) + g2 and counts written",
                           "achieved": g2c_bytes / (g2c_k * 1e-3) / 1e9 if g2c_k else None,
                           "peak": pk["hbm_gbs"], "unit": "GB/s",
                           "frac": g2c_bytes / (g2c_k * 1e-3) / 1e9 / pk["hbm_gbs"] if g2c_k else None,
                           "peak_source": pk["source"]}}
    del g2s, cs

    # ---- raw exact path on the same frames (the comparison of the metric)
    raw_ms = None
    raw_res = None
    if not args.no_raw:
        def raw_step():
            X.xpcs_twotime_raw(ctx, rings, Xd, T, C_out=C, g2_out=g2, count_out=cnt)

        raw_tuned = X.xpcs_autotune_twotime_raw(ctx, rings, Xd, T, C_out=C, g2_out=g2, count_out=cnt, reps=1)
        raw_ms, _, raw_prof = timed(raw_step, max(1, min(args.steps, 3)), 1, profile=True)
        raw_ms = max_over_ranks(raw_ms, world, dev)
        raw_kern = {k_: v[0] / max(1, v[1]) for k_, v in raw_prof.items()}
        Mq_sum = int(np.asarray(rings.sizes()).sum())
        raw_flops = 2.0 * Mq_sum * T * (T + 1) / 2  # exact Gram over the upper triangle, all ring pixels
        rg = raw_kern.get("twotime_gram")
        rpeak = pk["bf16_tflops_sustained"] or pk["bf16_tflops"]
        ing = raw_kern.get("ingest")
        ing_bytes = T * M * 2 + T_pad_of(T) * rings_padded(rings) * 2  # X read (uint16) + bf16 operand written
        raw_res = {
            "frames_per_s": world * T / (raw_ms * 1e-3), "ms_per_step": raw_ms, "kernels_ms": raw_kern,
            "autotuned": raw_tuned,
            "roofline": {"bound": "tensor", "kernel": "twotime_gram", "flops": raw_flops,
                         "flops_model": "2 sum_q M_q T(T+1)/2 (bf16 operands, exact integer Gram)",
                         "achieved": raw_flops / (rg * 1e-3) / 1e12 if rg else None, "peak": rpeak,
                         "unit": "TFLOP/s", "frac": raw_flops / (rg * 1e-3) / 1e12 / rpeak if rg else None,
                         "peak_source": pk["source"] + (" sustained" if pk["bf16_tflops_sustained"] else "")},
            "ingest_roofline": {"bound": "hbm", "kernel": "ingest", "algorithmic_bytes": ing_bytes,
                                "bytes_model": "X read once (uint16) + ring-sorted bf16 operand written",
                                "achieved": ing_bytes / (ing * 1e-3) / 1e9 if ing else None, "peak": pk["hbm_gbs"],
                                "unit": "GB/s", "frac": ing_bytes / (ing * 1e-3) / 1e9 / pk["hbm_gbs"] if ing else None},
        }

    # ---- other precision modes: time and error
    variants = {}
    for p in ("fp16", "bf16", "bf16x3"):
        if p == prec:
            continue
        vms, _, _ = timed(lambda: step(p), max(1, min(args.steps, 5)), 1)
        variants[p] = {"ms_per_step": vms}

    # ---- online stream: sustained rate and per-frame latency (every replica runs its own)
    stream_res = None
    if not (args.no_stream or args.no_host):
        stream_res = run_stream_leg(X, ctx, dev, args)

    # ---- grouped workload: 64 uneven masks in one encode and one two-time launch
    grouped_res = None
    if not (args.no_grouped or args.no_host) and args.workload == "c2":
        grouped_res = run_grouped_leg(X, dev, args)

    # ---- multi-stream serving: four detectors at their own rates on one server
    serving_res = None
    if not (args.no_serving or args.no_host) and args.workload == "c2":
        serving_res = run_serving_leg(X, dev, args)

    # ---- ceiling of the serving workload: two-time tiles it needs per second at full
    # history against the tile rate the online stream sustains on this GPU (steps of 128
    # frames: every ring x every tile diagonal of the history per step)
    if serving_res and stream_res:
        sv, sw = SERVING, STREAM
        nd = lambda W: (W + 126) // 128 + 1
        need = sum(st["rate_hz"] for st in sv["streams"]) * sv["n_q"] * nd(sv["history"]) / 128
        have = stream_res["sustained_frames_per_s"] * sw["n_q"] * nd(sw["history"]) / 128
        serving_res["ceiling_model"] = {
            "tiles_per_s_needed_at_full_history": need, "tiles_per_s_sustained_by_stream_leg": have,
            "ratio": need / have,
            "note": "a 128-frame step of a stream with n_q rings and history W runs n_q x (ceil(W/128)+1) "
                    "two-time tiles; at the 2e5-frame cap the four streams' arrival rates need the ratio "
                    "times the tile rate the online stream sustains, so they cannot all keep up on one GPU"}

    # ---- the small raw workload, timed in full beside the oracle
    c1_res = None
    if not args.no_host and rank == 0:
        c1_res = run_c1_leg(X, dev, args)

    # ---- end to end through the public API from pinned host memory
    if args.no_host:
        if rank == 0:
            print(json.dumps({"workload": args.workload, "ms_per_step": ms, "frames_per_s": world * T / (ms * 1e-3),
                              "raw_ms": raw_ms, "variants_ms": {p: v["ms_per_step"] for p, v in variants.items()},
                              "kernels_ms": {k_: v[0] / max(1, v[1]) for k_, v in prof.items()},
                              "gpu_launches": launches}), flush=True)
        return
    Xh = torch.empty((T, M), dtype=torch.uint16, pin_memory=True)
    Xh.copy_(Xd)
    g2h = torch.empty((n_q, T), dtype=torch.float64, pin_memory=True)
    cnth = torch.empty((n_q, T), dtype=torch.int64, pin_memory=True)

    def e2e_step():
        # frames from pinned host memory: the library copies them in blocks on two copy
        # streams while it encodes the blocks already on the device
        X.xpcs_encode_host(ctx, basis, Xh, T, A)
        X.xpcs_twotime(ctx, basis, A, T, prec, C_out=C, g2_out=g2, count_out=cnt)
        g2h.copy_(g2, non_blocking=True)
        cnth.copy_(cnt, non_blocking=True)

    e2e_ms, _, _ = timed(e2e_step, max(1, min(args.steps, 5)), 1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    # the bound of the end-to-end step: one plain copy of the frames from pinned host memory
    copy_ms, _, _ = timed(lambda: Xd.copy_(Xh, non_blocking=True), 3, 1)
    del Xh

    # ---- parity at full size on sampled outputs, and the CPU oracle baseline (rank 0)
    result = {}
    if rank == 0:
        step()
        ctx.synchronize()
        frames_host = Xd.cpu().numpy()
        cpu_fps, cpu_s, info = oracle_cpu(frames_host, qmap, wl, n_rings_sample=1)
        import oracle as O

        rng = np.random.default_rng(1)
        nsamp = 4096
        qs = rng.integers(0, n_q, size=nsamp)
        t1 = rng.integers(0, T, size=nsamp)
        t2 = rng.integers(0, T, size=nsamp)
        t1, t2 = np.minimum(t1, t2), np.maximum(t1, t2)
        errs = {}
        # g2 of ring 0 at the full T from the oracle
        Cq = O.twotime_from_gram(O.compressed_ring_gram(info["A"], info["G"][0]), info["A"] @ info["s"][0],
                                 info["A"] @ info["s"][0], info["Mq"][0])
        gref, _ = O.g2_from_twotime(Cq)
        del Cq
        order = np.concatenate([np.flatnonzero(qs == q) for q in range(n_q)])
        ref = np.concatenate([O.compressed_pair_values(info["A"], info["G"][q], info["s"][q], info["Mq"][q],
                                                       t1[qs == q], t2[qs == q]) for q in range(n_q)])
        idx = torch.from_numpy(((qs * T + t2) * T + t1).astype(np.int64)).to(dev)  # lower triangle
        for p in ("fp16", "bf16", "bf16x3"):
            step(p)
            ctx.synchronize()
            gotq = C.view(-1)[idx].cpu().numpy().astype(np.float64)[order]
            ok = ~np.isnan(ref) & ~np.isnan(gotq)
            d = np.abs(gotq[ok] - ref[ok])
            c_max = float(d.max() / np.abs(ref[ok]).max())
            c_rms = float(np.sqrt((d ** 2).sum() / (ref[ok] ** 2).sum()))
            gg = g2[0].cpu().numpy()
            okg = ~np.isnan(gref) & ~np.isnan(gg)
            g_max = float(np.abs(gg[okg] - gref[okg]).max() / np.abs(gref[okg]).max())
            errs[p] = {"C_rel_max": c_max, "C_rel_rms": c_rms, "g2_rel_max_ring0": g_max,
                       "pairs_sampled": int(ok.sum()),
                       "nan_mismatch": int((np.isnan(ref) != np.isnan(gotq)).sum())}
        result = dict(cpu_fps=cpu_fps, cpu_s=cpu_s, info=info, errs=errs)

    if rank != 0:
        return

    # ---- roofline of the dominant kernel (timed live over the timed region)
    pk = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms_total, dom_n) = dom
    dom_ms = dom_ms_total / max(1, dom_n)
    nT = (T + 127) // 128
    T_pad = nT * 128
    Kc = ((3 if prec == "bf16x3" else 1) * k + 63) // 64 * 64
    if dom_name == "twotime_gram":
        c_elems = 0
        for I in range(nT):
            rows = min(128, T - 128 * I)
            for J in range(I, nT):
                c_elems += rows * min(128, T - 128 * J)
        maxC = (nT + 7) // 8
        alg = n_q * c_elems * 4 + 2 * n_q * T_pad * Kc * 2 + n_q * nT * maxC * 256 * 4
        alg_note = "C triangle tiles written (float32) + both operand matrices read once + diagonal partials"
    elif dom_name == "encode":
        kp = (k + 15) // 16 * 16
        alg = T * M * 2 + 2 * kp * M * 2 + T_pad * k * 4
        alg_note = "X read once (uint16) + hi/lo basis read once + partial coefficients"
    else:
        alg = None
        alg_note = "no byte model"
    achieved = alg / (dom_ms * 1e-3) / 1e9 if alg else None
    traffic = None
    prof_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof_file):
        tr = json.load(open(prof_file)).get(dom_name, {}).get(prec)
        if tr:
            traffic = tr
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": (achieved / pk["hbm_gbs"]) if achieved else None, "traffic": traffic,
                "algorithmic_bytes": alg, "kernel_ms": dom_ms, "peak_source": pk["source"], "bytes_model": alg_note}

    value = world * T / (ms * 1e-3)
    h2d = T * M * 2
    d2h = n_q * T * 16
    # the long objects first and the metric's own figures (latency, raw path, speed-up,
    # error) last, so that a reader keeping only the end of the line still has them
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "precision": prec, "l2": "inputs larger than L2 (X = 5.24 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "grouped": grouped_res,
        "serving": serving_res,
        "cuda_graph": graph_res,
        "autotuned": tuned,
        "setup_s": {"generate": t_gen, "fit_basis_gpu": t_fit},
        "kernels_ms": {k_: v[0] / max(1, v[1]) for k_, v in prof.items()},
        "precision_variants_ms": {p: v["ms_per_step"] for p, v in variants.items()},
        "xpcs_g2": g2_res,
        "c1_raw": c1_res,
        "roofline": roofline,
        "cpu_baseline": {"value": result["cpu_fps"], "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "extrapolated: oracle FP64 encode of all 10000 frames + two-time and g2 of ring 0 "
                                   "at T=10000 timed, the two-time scaled x36 rings (BLAS multithreaded, "
                                   "reductions single-threaded)",
                         "seconds": result["cpu_s"]},
        "e2e": {"value": world * T / (e2e_ms * 1e-3), "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "h2d_gbs_over_step": h2d / (e2e_ms * 1e-3) / 1e9,
                "h2d_copy_only_ms": copy_ms, "h2d_copy_only_gbs": h2d / (copy_ms * 1e-3) / 1e9,
                "path": "xpcs_encode_host (copies of 256 MB blocks, on one or two copy streams as the context calibrates on its first call, overlapped with the "
                        "encode) + xpcs_twotime + g2/count read back"},
        "gpu_launches": launches,
        "clocks": sampler.summary() if sampler else None,
        "error_vs_fp64_oracle": result["errs"],
        "raw_path": raw_res,
        "speedup_vs_raw": (raw_ms / ms) if raw_ms else None,
        "latency": stream_res,
    }
    print(json.dumps(line), flush=True)


def run_grouped_leg(X, dev, args, gw=GROUPED):
    """Grouped workload: all 64 uneven masks through one encode and one two-time launch.

    X (masked pixels only, padded to 16-byte rows with zero columns outside every mask) is
    resident in HBM (9.9 GB, larger than L2).  One step = encode + two-time (bf16x3) with
    g2 and counts fused; C is not stored.  Timed with CUDA events on the library's
    stream; the roofline is the two-time kernel's tensor work against the measured bf16
    peak (algorithmic flops of one product; the hi/lo scheme issues three)."""
    import torch
    from synth import sector_qmap
    from synth.speckle import TorchSpeckle

    H, W, T, n_q, k = gw["H"], gw["W"], gw["T"], gw["n_q"], gw["k"]
    stream = torch.cuda.current_stream(dev)
    qfull = sector_qmap(H, W, n_annuli=8, n_sectors=8, min_px=gw["min_px"], max_px=gw["max_px"], seed=gw["seed"])
    pix = np.flatnonzero(qfull >= 0)
    M = (pix.size + 7) // 8 * 8
    qmap = np.full(M, -1, dtype=np.int32)
    qmap[:pix.size] = qfull[pix]
    pix_d = torch.from_numpy(pix.astype(np.int64)).to(dev)
    t0 = time.time()
    gen = TorchSpeckle(H, W, gw["mean"], gw["D"], gw["seed"], dtype=gw["dtype"], device=str(dev))
    Xd = torch.zeros((T, M), dtype=torch.uint16, device=dev)
    for i in range(0, T, 1000):
        Xd[i:i + 1000, :pix.size].copy_(gen.next(min(1000, T - i)).index_select(1, pix_d))
    del gen
    torch.cuda.synchronize()
    t_gen = time.time() - t0
    ctx = X.Context(dev.index or 0, 0, stream.cuda_stream)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), M, n_q)
    t0 = time.time()
    basis = X.xpcs_fit_basis(ctx, rings, Xd, gw["n_fit"], k)
    t_fit = time.time() - t0
    A = torch.empty((T, k), dtype=torch.float32, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    ctx.set_async(True)

    def step():
        X.xpcs_encode(ctx, basis, Xd, T, A)
        X.xpcs_twotime(ctx, basis, A, T, "bf16x3", g2_out=g2, count_out=cnt)

    X.xpcs_encode(ctx, basis, Xd, T, A)
    tuned = X.xpcs_autotune_twotime(ctx, basis, A, T, "bf16x3", g2_out=g2, count_out=cnt, reps=1)
    K = max(1, min(args.steps, 5))
    for _ in range(3):
        step()
    ctx.synchronize()
    ctx.profile_enable(True)
    n0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        step()
    e1.record(stream)
    ctx.synchronize()
    ms = e0.elapsed_time(e1) / K
    launches = ctx.launch_count() - n0
    prof = ctx.profile()
    ctx.profile_enable(False)
    kern = {k_: v[0] / max(1, v[1]) for k_, v in prof.items()}
    # the same step as one CUDA graph (all masks' encode and two-time kernels, one launch)
    X.xpcs_capture_begin(ctx)
    step()
    graph = X.xpcs_capture_end(ctx)
    for _ in range(3):
        graph.launch()
    ctx.synchronize()
    e0.record(stream)
    for _ in range(K):
        graph.launch()
    e1.record(stream)
    ctx.synchronize()
    graph_ms = e0.elapsed_time(e1) / K
    graph_kernels = graph.kernels()
    graph.close()
    sizes = np.bincount(qmap[qmap >= 0], minlength=n_q)
    nT = (T + 127) // 128
    flops = 2.0 * n_q * k * T * (T + 1) / 2  # one product over the upper triangle
    gram_ms = kern.get("twotime_gram")
    pk = peaks()
    peak = pk["bf16_tflops_sustained"] or pk["bf16_tflops"]
    achieved = flops / (gram_ms * 1e-3) / 1e12 if gram_ms else None
    # every precision of the g2-only two-time: time (autotuned per precision) and the error
    # of g2 against the FP64 oracle of the same coefficients on the smallest and the largest
    # mask (whole g2 at the full T)
    import oracle as O

    g2h = {}
    per_prec = {}
    for p in ("bf16x3", "fp16", "bf16"):
        tp = X.xpcs_autotune_twotime(ctx, basis, A, T, p, g2_out=g2, count_out=cnt, reps=1)
        for _ in range(2):
            X.xpcs_twotime(ctx, basis, A, T, p, g2_out=g2, count_out=cnt)
        ctx.synchronize()
        ctx.profile_enable(True)
        e0.record(stream)
        for _ in range(K):
            X.xpcs_twotime(ctx, basis, A, T, p, g2_out=g2, count_out=cnt)
        e1.record(stream)
        ctx.synchronize()
        kp = {k_: v[0] / max(1, v[1]) for k_, v in ctx.profile().items()}
        ctx.profile_enable(False)
        gm = kp.get("twotime_gram")
        g2h[p] = g2.cpu().numpy()
        per_prec[p] = {"twotime_ms": e0.elapsed_time(e1) / K, "gram_ms": gm, "autotuned": tp,
                       "gram_tflops_one_product": flops / (gm * 1e-3) / 1e12 if gm else None,
                       "frac_of_peak_one_product": flops / (gm * 1e-3) / 1e12 / peak if gm else None}
    Ah = A.cpu().numpy().astype(np.float64)
    _, Gh, sh = basis.export()
    for p in per_prec:
        per_prec[p]["g2_rel_max"] = {}
    for m in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        Sq = Ah @ sh[m]
        Cq = O.twotime_from_gram(O.compressed_ring_gram(Ah, Gh[m]), Sq, Sq, sizes[m])
        gref, _ = O.g2_from_twotime(Cq)
        del Cq
        okr = ~np.isnan(gref)
        for p in per_prec:
            gg = g2h[p][m]
            ok = okr & ~np.isnan(gg)
            per_prec[p]["g2_rel_max"][f"mask{m}_{int(sizes[m])}px"] = float(
                np.abs(gg[ok] - gref[ok]).max() / np.abs(gref[ok]).max())
    del Ah
    # the cheapest precision whose g2 error stays within the 1e-3 target on both masks
    enc_ms = kern.get("encode", 0.0) + kern.get("encode_reduce", 0.0)
    ok = [p for p in ("fp16", "bf16", "bf16x3") if max(per_prec[p]["g2_rel_max"].values()) <= 1e-3]
    chosen = min(ok, key=lambda p: per_prec[p]["twotime_ms"]) if ok else "bf16x3"
    chosen_ms = enc_ms + per_prec[chosen]["twotime_ms"]
    out = {
        "workload": GROUPED_NAME, "frames_per_s": T / (ms * 1e-3), "ms_per_step": ms, "steps": K, "warmup": 3,
        "chosen_precision": chosen, "chosen_ms_per_step": chosen_ms, "chosen_frames_per_s": T / (chosen_ms * 1e-3),
        "chosen_note": "the cheapest precision whose g2 error against the FP64 oracle is within 1e-3 on the "
                       "smallest and the largest mask; its step = the encode plus its two-time call "
                       "(event-timed separately); frames_per_s above is the bf16x3 step",
        "masks": n_q, "mask_px": {"min": int(sizes.min()), "max": int(sizes.max()), "total": int(sizes.sum())},
        "tiles_per_step": int(n_q * nT * (nT + 1) // 2), "kernels_ms": kern, "gpu_launches": launches,
        "cuda_graph": {"ms_per_step": graph_ms, "frames_per_s": T / (graph_ms * 1e-3),
                       "kernels_per_step": graph_kernels},
        "autotuned": tuned,
        # the roofline of the chosen precision's two-time kernel (fp16 and bf16 have the same
        # nominal dense rate, so the measured bf16 peak is theirs too), and the bf16x3 step's
        "roofline": {"bound": "tensor", "kernel": "twotime_gram", "precision": chosen,
                     "achieved": per_prec[chosen]["gram_tflops_one_product"], "peak": peak, "unit": "TFLOP/s",
                     "frac": per_prec[chosen]["frac_of_peak_one_product"], "traffic": None,
                     "peak_source": pk["source"] + (" sustained" if pk["bf16_tflops_sustained"] else ""),
                     "flops_model": "2 n_q k T(T+1)/2 (one 16-bit product; bf16x3 issues three)"},
        "roofline_bf16x3": {"bound": "tensor", "kernel": "twotime_gram", "precision": "bf16x3", "achieved": achieved,
                            "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                            "frac_counting_issued_products": (3 * achieved / peak) if achieved else None},
        "setup_s": {"generate": t_gen, "fit_basis_gpu": t_fit},
        "precision": "bf16x3", "l2": "inputs larger than L2 (X = %.2f GB)" % (T * M * 2 / 1e9),
        "precisions": per_prec,
        "precision_note": "g2 error vs the FP64 oracle of the same coefficients (target 1e-3); the cheapest "
                          "precision within it is the caller's choice",
    }
    del Xd, A
    basis.close()
    rings.close()
    ctx.close()
    torch.cuda.empty_cache()
    return out


C1 = dict(H=64, W=64, T=500, n_q=8, mean=0.1, D=1e-3, seed=20356001)
C1_NAME = ("64x64 detector, T=500 frames, uint8 Poisson AR(1) speckle mean 0.1 D=1e-3, 8 q-rings; "
           "raw path: exact integer Gram N, C, g2 and counts")


def run_c1_leg(X, dev, args, w=C1):
    """The small raw workload timed in full on the GPU and on the oracle, with bit-exactness."""
    import torch

    import oracle as O
    from synth import ring_qmap, speckle_counts

    H, W, T, n_q = w["H"], w["W"], w["T"], w["n_q"]
    frames = speckle_counts(H, W, T, w["mean"], w["D"], w["seed"], np.uint8)
    qmap = ring_qmap(H, W, n_q)
    stream = torch.cuda.current_stream(dev)
    ctx = X.Context(dev.index or 0, 0, stream.cuda_stream)
    rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), H * W, n_q)
    Xd = torch.from_numpy(frames).to(dev)
    C = torch.empty((n_q, T, T), dtype=torch.float32, device=dev)
    N = torch.empty((n_q, T, T), dtype=torch.int64, device=dev)
    g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
    cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
    ctx.set_async(True)

    def call():
        X.xpcs_twotime_raw(ctx, rings, Xd, T, C_out=C, N_out=N, g2_out=g2, count_out=cnt)

    for _ in range(3):
        call()
    ctx.synchronize()
    K = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        call()
    e1.record(stream)
    ctx.synchronize()
    gpu_ms = e0.elapsed_time(e1) / K
    t0 = time.perf_counter()
    Cref, Nref, _, _ = O.raw_twotime(frames, qmap, n_q)
    gref = [O.g2_from_twotime(Cref[q]) for q in range(n_q)]
    t_or = time.perf_counter() - t0
    il = np.tril_indices(T)
    Nh, gh = N.cpu().numpy(), g2.cpu().numpy()
    exact = all(np.array_equal(Nh[q][il], Nref[q][il]) for q in range(n_q))
    gerr = max(float(np.nanmax(np.abs(gh[q] - gref[q][0]) / np.nanmax(np.abs(gref[q][0])))) for q in range(n_q))
    rings.close()
    ctx.close()
    return {"workload": C1_NAME, "gpu": {"ms_per_step": gpu_ms, "frames_per_s": T / (gpu_ms * 1e-3), "steps": K},
            "oracle": {"seconds": t_or, "frames_per_s": T / t_or, "cores": os.cpu_count(),
                       "sample": "the whole workload (all 8 rings at T=500), not extrapolated"},
            "N_bit_exact": bool(exact), "g2_rel_max": gerr}


def run_serving_leg(X, dev, args, sv=SERVING):
    """Multi-stream serving: four streams of different detector sizes on one server.

    Each stream gets its own basis (k per stream, fitted on a 1000-frame calibration run of
    its detector) and 100 equal-width q-rings, and is opened on one xpcs_server with a
    2e5-frame history cap and batches of up to 64 frames.  A client thread per stream
    submits frames in device memory (a detector feeding the GPU directly; cycled from a
    pool of distinct generated frames, queued by pointer with xpcs_server_submit_device)
    at the stream's rate for `--serving-seconds`, starting from empty histories; the server's
    scheduler batches continuously and the streams overlap on the device.  Afterwards each
    stream is drained.  Reported per stream: target rate, frames submitted and dropped
    (a client keeps at most about 256 MB of frames outstanding per stream, at least 64;
    frames that arrive beyond that are dropped and counted), the rate at which the submitted frames were
    folded in (frames / time until the last one completed), whether the stream kept up
    (nothing dropped, folded rate within 2 % of the arrival rate), and the per-frame latency
    (submit to completion) p50/p99."""
    import threading

    import torch
    from synth import ring_qmap
    from synth.speckle import TorchSpeckle

    ctx = X.Context(dev.index or 0)
    server = X.Server(ctx)
    n_q, Wl, mb = sv["n_q"], sv["history"], sv["max_batch"]
    streams = []
    t0 = time.time()
    for i, st in enumerate(sv["streams"]):
        H, W, k = st["H"], st["W"], st["k"]
        gen = TorchSpeckle(H, W, sv["mean"], st["D"], sv["seed"] + 100 + i, dtype="uint16", device=str(dev))
        calib = gen.next(sv["n_fit"])
        rings = X.Rings(ctx, torch.from_numpy(ring_qmap(H, W, n_q)).to(dev), H * W, n_q)
        basis = X.xpcs_fit_basis(ctx, rings, calib, sv["n_fit"], k)
        del calib, gen
        gen = TorchSpeckle(H, W, sv["mean"], st["D"], sv["seed"] + i, dtype="uint16", device=str(dev))
        pool = gen.next(sv["pool"])  # device frames, read in place by the stream
        del gen
        sid = server.open(basis, Wl, mb)
        streams.append(dict(cfg=st, rings=rings, basis=basis, pool=pool, id=sid, sent=0, dropped=0, ticket=0))
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    secs = args.serving_seconds
    start = time.perf_counter() + 0.05
    stop_at = start + secs

    def client(e):
        # frames arrive at the stream's rate; while more than `cap` submitted frames are not
        # yet folded in (about 256 MB of frames, at least 64), arriving frames are dropped
        # and counted, as a detector that outruns its consumer loses them
        rate, P = e["cfg"]["rate_hz"], e["pool"]
        cap = max(64, (256 << 20) // (P.shape[1] * 2))
        e["cap"] = cap
        while True:
            now = time.perf_counter()
            if now >= stop_at:
                break
            due = int((now - start) * rate) - (e["sent"] + e["dropped"])
            if due <= 0:
                time.sleep(50e-6)
                continue
            if e["sent"] > cap and not server.poll(e["id"], e["sent"] - cap, 0):
                e["dropped"] += due
                continue
            o = e["sent"] % P.shape[0]
            n = min(due, P.shape[0] - o)
            e["ticket"] = server.submit_device(e["id"], P[o:o + n])
            e["sent"] += n

    threads = [threading.Thread(target=client, args=(e,)) for e in streams]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    out = []
    total = 0.0
    for e in streams:
        ok = server.poll(e["id"], e["ticket"], 60000) if e["ticket"] else True
        t_done = time.perf_counter() - start
        lat = server.latency(e["id"])
        st = e["cfg"]
        rate = e["sent"] / t_done if (ok and t_done > 0) else None
        total += rate or 0.0
        out.append({"detector": f"{st['H']}x{st['W']}", "k": st["k"], "D": st["D"], "rate_hz": st["rate_hz"],
                    "frames": e["sent"], "dropped": e["dropped"], "backlog_cap": e.get("cap"), "drained": bool(ok),
                    "folded_frames_per_s": rate,
                    "kept_up": bool(e["dropped"] == 0 and rate is not None and rate >= 0.98 * st["rate_hz"]),
                    "p50_us": lat["p50_us"], "p99_us": lat["p99_us"], "max_us": lat["max_us"],
                    "history_reached": min(e["sent"], Wl)})
    res = {"workload": "four uint16 streams (1536x2048 at 2 kHz k=256 D=1e-4, 1024x1024 at 10 kHz k=128 "
                       "D=4.64e-4, 512x512 at 50 kHz k=128 D=2.15e-3, 256x256 at 100 kHz k=64 D=1e-2), "
                       "Poisson AR(1) speckle mean 0.02, 100 q-rings each, history cap 200000, batches <= 64, "
                       "one server, device frames submitted at each stream's rate from empty histories",
           "seconds": secs, "streams": out, "total_folded_frames_per_s": total,
           "target_frames_per_s": sum(s_["rate_hz"] for s_ in sv["streams"]), "batches": server.batches(),
           "setup_s": t_setup}
    server.close()
    for e in streams:
        e["basis"].close()
        e["rings"].close()
    ctx.close()
    torch.cuda.empty_cache()
    return res


def run_stream_leg(X, ctx, dev, args, sw=STREAM):
    """Online stream at the stated arrival rate: sustained frames/s and p50/p99 latency.

    Frames come from a device pool of `pool` distinct generated frames, pushed in order and
    cycled (the work per frame does not depend on the frame's content beyond its nonzero
    count).  Phases: fill the history unpaced (batches of max_batch), time a further
    unpaced run (sustained rate), time an unpaced run in batches of one frame, then push
    at rate_hz with each frame stamped at its scheduled arrival time; latency counts from
    that arrival to the end of the device work of the frame's batch."""
    import torch
    from synth import ring_qmap
    from synth.speckle import TorchSpeckle

    H, W, n_q, k, Wl = sw["H"], sw["W"], sw["n_q"], sw["k"], sw["history"]
    M = H * W
    rings = X.Rings(ctx, torch.from_numpy(ring_qmap(H, W, n_q)).to(dev), M, n_q)
    gen = TorchSpeckle(H, W, sw["mean"], sw["D"], sw["seed"] + 100, dtype=sw["dtype"], device=str(dev))
    cal = gen.next(sw["n_fit"])
    basis = X.xpcs_fit_basis(ctx, rings, cal, sw["n_fit"], k)
    del cal, gen
    gen = TorchSpeckle(H, W, sw["mean"], sw["D"], sw["seed"], dtype=sw["dtype"], device=str(dev))
    P = sw["pool"]
    pool = torch.empty((P, M), dtype=torch.uint16, device=dev)
    for i in range(0, P, 256):
        pool[i:i + 256].copy_(gen.next(min(256, P - i)))
    del gen
    nnz_per_frame = float((pool[:64].view(torch.int16) != 0).sum().item()) / 64
    torch.cuda.synchronize()
    def measure(prec, seconds):
        """Fill, sustained, one-frame and paced phases of one stream of precision `prec`."""
        st = X.Stream(ctx, basis, Wl, sw["max_batch"], dtype=sw["dtype"], prec=prec)
        pushed = 0

        def push(n, batch):
            nonlocal pushed
            t = 0
            while n > 0:
                i = pushed % P
                m = min(n, P - i, batch)
                t = st.push(pool[i:i + m])
                pushed += m
                n -= m
            return t

        def run_unpaced(n, batch):
            t0 = time.perf_counter()
            ticket = push(n, batch)
            assert st.poll(ticket, 600000)
            return n / (time.perf_counter() - t0)

        run_unpaced(Wl, sw["max_batch"])  # fill the history
        fps_sustained = run_unpaced(20000, sw["max_batch"])
        fps_b1 = run_unpaced(4000, 1)
        st.latency(reset=True)

        # paced: frame j arrives at t0 + j / rate.  Continuous batching: whenever fewer than
        # two batches are in flight, every frame that has arrived (up to max_batch) goes out
        # as one batch, so the batch grows with the load instead of a queue.
        n_paced = int(sw["rate_hz"] * seconds)
        period = 1e9 / sw["rate_hz"]
        t0 = X.clock_ns() + 1_000_000
        arrive = (t0 + np.arange(n_paced) * period).astype(np.int64)
        j = 0
        batches = 0
        inflight = []
        ticket = 0
        while j < n_paced:
            while inflight and st.poll(inflight[0], 0):
                inflight.pop(0)
            if len(inflight) >= 2:
                continue
            now = X.clock_ns()
            due = min(n_paced, int((now - t0) // period) + 1) if now >= t0 else 0
            if due <= j:
                continue
            n = min(due - j, sw["max_batch"])
            i = pushed % P
            n = min(n, P - i)
            ticket = st.push_at(pool[i:i + n], arrive[j:j + n])
            inflight.append(ticket)
            pushed += n
            j += n
            batches += 1
        assert st.poll(ticket, 600000)
        t_end = X.clock_ns()
        lat = st.latency(reset=True)
        st.close()
        return {"sustained": fps_sustained, "b1": fps_b1, "lat": lat, "n_paced": n_paced, "batches": batches,
                "paced_fps": n_paced / ((t_end - t0) * 1e-9)}

    m3 = measure("bf16x3", args.stream_seconds)
    m16 = measure("fp16", min(args.stream_seconds, 3.0))
    fps_sustained, fps_b1, lat, n_paced, batches = m3["sustained"], m3["b1"], m3["lat"], m3["n_paced"], m3["batches"]
    nb = Wl  # history length
    ka = (k + 31) // 32 * 32
    bytes_batch_fixed = nb * ka * 4 + nb * n_q * 4 + 2 * n_q * nb * 16
    bytes_frame = M * 2 + nnz_per_frame * k * 4
    raw_frame_bytes = Wl * M * 2
    pk = peaks()
    out = {
        "workload": STREAM_NAME, "frames_paced": n_paced, "rate_hz": sw["rate_hz"],
        "p50_us": lat["p50_us"], "p99_us": lat["p99_us"], "max_us": lat["max_us"],
        "frames_measured": lat["batches"], "batches_paced": batches, "mean_batch": n_paced / max(1, batches),
        "paced_frames_per_s": m3["paced_fps"],
        "sustained_frames_per_s": fps_sustained, "sustained_batch": sw["max_batch"],
        "batch1_frames_per_s": fps_b1,
        "bytes_model": {"per_batch_fixed": bytes_batch_fixed, "per_frame": bytes_frame,
                        "note": "history rows + ring factors read once and g2 sums/counts read+written per batch; "
                                "frame scan + basis rows of nonzero pixels per frame"},
        "sustained_gbs": (bytes_batch_fixed / sw["max_batch"] + bytes_frame) * fps_sustained / 1e9,
        "raw_equivalent_frames_per_s_model": pk["hbm_gbs"] * 1e9 / raw_frame_bytes,
        "raw_equivalent_note": "cross-check only: a raw row update that reads the uint16 history (history x M) "
                               "once per frame at the measured HBM bandwidth",
        "pool_frames": P, "nnz_per_frame": nnz_per_frame,
        "precision": "bf16x3",
        "fp16": {"note": "the same stream in f16 (one product, half the history bytes; 1e-3 of max|g2|)",
                 "sustained_frames_per_s": m16["sustained"], "batch1_frames_per_s": m16["b1"],
                 "p50_us": m16["lat"]["p50_us"], "p99_us": m16["lat"]["p99_us"],
                 "frames_paced": m16["n_paced"], "mean_batch": m16["n_paced"] / max(1, m16["batches"])},
    }
    out["raw_equivalent"] = run_raw_stream_equivalent(X, ctx, basis, rings, pool, sw)
    basis.close()
    rings.close()
    del pool
    torch.cuda.empty_cache()
    return out


def run_raw_stream_equivalent(X, ctx, basis, rings, pool, sw, histories=(10000, 20000)):
    """The raw-path equivalent of the online stream, measured: xpcs_raw_stream (every pushed
    frame's exact raw two-time row against the window, integer Gram on the tensor cores)
    on the same 1 Mpx frames, at histories that fit HBM as bf16 rows, in 64-frame steps and
    one frame at a time; the compressed stream is timed at the same history beside it.
    Both cost in proportion to the history, which the two histories show."""
    P = pool.shape[0]

    def feed(push, wait, n, batch, pushed):
        t0 = time.perf_counter()
        last = None
        while n > 0:
            i = pushed % P
            m = min(n, P - i, batch)
            last = push(pool[i:i + m])
            pushed += m
            n -= m
        wait(last)
        return time.perf_counter() - t0, pushed

    out = {"note": "exact raw row update (bf16 counts, f32 integer Gram on the tensor cores, FP64 g2 sums) "
                   "against the compressed stream (bf16x3) on the same frames and history"}
    for Wr in histories:
        rs = X.RawStream(ctx, rings, Wr, dtype=sw["dtype"])
        rwait = lambda _t: ctx.synchronize()  # the raw stream runs on the context's stream
        _, pushed = feed(rs.push, rwait, Wr, sw["max_batch"], 0)  # fill the history
        t64, pushed = feed(rs.push, rwait, 1280, sw["max_batch"], pushed)
        t1, pushed = feed(rs.push, rwait, 64, 1, pushed)
        rs.close()
        st = X.Stream(ctx, basis, Wr, sw["max_batch"], dtype=sw["dtype"])
        swait = lambda t: st.poll(t, 600000)  # the stream runs on its own CUDA stream
        _, pc = feed(st.push, swait, Wr, sw["max_batch"], 0)
        c64, pc = feed(st.push, swait, 4096, sw["max_batch"], pc)
        c1, pc = feed(st.push, swait, 1024, 1, pc)
        st.close()
        out[f"history_{Wr}"] = {
            "batch": sw["max_batch"],
            "raw_frames_per_s_batch": 1280 / t64, "raw_frames_per_s_batch1": 64 / t1,
            "compressed_frames_per_s_batch": 4096 / c64, "compressed_frames_per_s_batch1": 1024 / c1,
            "speedup_batch": (4096 / c64) / (1280 / t64), "speedup_batch1": (1024 / c1) / (64 / t1),
            "raw_history_gb": (128 * ((Wr + 126) // 128 + 2)) * rings_padded(rings) * 2 / 1e9,
        }
    return out


def stream_capture(mode, path, prec="bf16x3"):
    """A short stream run for profiling one single-frame step at the full history.

    make: fit the basis of the online-stream workload, fill a stream with history + 64
    frames, and save the basis and a checkpoint under `path`.  run: import that basis,
    restore the checkpoint into a fresh stream and push three single frames, each waited
    for, then a 64-frame and a 128-frame step, so a profiler sees about twenty launches
    before them.  prec: the stream's precision (the checkpoint records it, so make and run
    take the same).
    Prints no bench line."""
    import torch
    from paper_2407_20356_gb300 import xpcs as X
    from synth import ring_qmap
    from synth.speckle import TorchSpeckle

    sw = STREAM
    dev = torch.device("cuda", 0)
    H, W, n_q, k, Wl = sw["H"], sw["W"], sw["n_q"], sw["k"], sw["history"]
    ctx = X.Context(0)
    rings = X.Rings(ctx, torch.from_numpy(ring_qmap(H, W, n_q)).to(dev), H * W, n_q)
    f_basis, f_ckpt = os.path.join(path, "stream_basis.npy"), os.path.join(path, f"stream_ckpt_{prec}.bin")
    if mode == "make":
        gen = TorchSpeckle(H, W, sw["mean"], sw["D"], sw["seed"] + 100, dtype=sw["dtype"], device=str(dev))
        np.save(f_basis, X.xpcs_fit_basis(ctx, rings, gen.next(sw["n_fit"]), sw["n_fit"], k).export()[0])
    basis = X.xpcs_basis_import(ctx, rings, np.load(f_basis))
    pool = TorchSpeckle(H, W, sw["mean"], sw["D"], sw["seed"], dtype=sw["dtype"], device=str(dev)).next(64)
    st = X.Stream(ctx, basis, Wl, 64, dtype=sw["dtype"], prec=prec)
    if mode == "make":
        t = 0
        for _ in range(0, Wl + 64, 64):
            t = st.push(pool)
        assert st.poll(t, 600000)
        st.checkpoint().tofile(f_ckpt)
    else:
        st.restore(np.fromfile(f_ckpt, dtype=np.uint8))
        for j in range(3):
            assert st.poll(st.push(pool[j:j + 1]), 60000)
        assert st.poll(st.push(pool[:64]), 60000)  # then a 64-frame step (to the block's end)
        assert st.poll(st.push(pool[:128]), 60000)  # and a whole 128-frame block
    print(f"stream capture {mode}: {st.frames()} frames", file=sys.stderr)
    st.close()
    ctx.close()


def profile_leg(args):
    """Profiling aid, no bench line: run one leg alone so that a profiler sees few launches.

    raw: the exact raw path (ingest, integer Gram with C, g2 and counts) on the chosen
    workload, `--steps` calls after `--warmup`; compressed: the compressed two-time of the
    chosen workload with C stored, g2 and counts (default configuration); grouped: the
    grouped masks' g2-only two-time on the small grouped case.  Prints a short JSON line of
    event-timed milliseconds per call."""
    import torch
    from paper_2407_20356_gb300 import xpcs as X
    from synth import ring_qmap
    from synth.speckle import TorchSpeckle

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    out = {"leg": args.leg, "workload": args.workload}
    if args.leg == "raw":
        wl = dict(WORKLOAD if args.workload == "c2" else SMALL)
        H, W, T, n_q = wl["H"], wl["W"], wl["T"], wl["n_q"]
        gen = TorchSpeckle(H, W, wl["mean"], wl["D"], wl["seed"], dtype=wl["dtype"], device=str(dev))
        Xd = torch.empty((T, H * W), dtype=torch.uint16, device=dev)
        for i in range(0, T, 1000):
            Xd[i:i + 1000].copy_(gen.next(min(1000, T - i)))
        del gen
        ctx = X.Context(0, 0, stream.cuda_stream)
        rings = X.Rings(ctx, torch.from_numpy(ring_qmap(H, W, n_q)).to(dev), H * W, n_q)
        C = torch.empty((n_q, T, T), dtype=torch.float32, device=dev)
        g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
        cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)

        def call():
            X.xpcs_twotime_raw(ctx, rings, Xd, T, C_out=C, g2_out=g2, count_out=cnt)

        flops = 2.0 * H * W * T * (T + 1) / 2
    elif args.leg == "compressed":
        wl = dict(WORKLOAD if args.workload == "c2" else SMALL)
        H, W, T, n_q, k = wl["H"], wl["W"], wl["T"], wl["n_q"], wl["k"]
        gen = TorchSpeckle(H, W, wl["mean"], wl["D"], wl["seed"], dtype=wl["dtype"], device=str(dev))
        Xd = torch.empty((T, H * W), dtype=torch.uint16, device=dev)
        for i in range(0, T, 1000):
            Xd[i:i + 1000].copy_(gen.next(min(1000, T - i)))
        del gen
        ctx = X.Context(0, 0, stream.cuda_stream)
        rings = X.Rings(ctx, torch.from_numpy(ring_qmap(H, W, n_q)).to(dev), H * W, n_q)
        basis = X.xpcs_fit_basis(ctx, rings, Xd, wl["n_fit"], k)
        A = torch.empty((T, k), dtype=torch.float32, device=dev)
        X.xpcs_encode(ctx, basis, Xd, T, A)
        C = torch.empty((n_q, T, T), dtype=torch.float32, device=dev)
        g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
        cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)

        def call():
            X.xpcs_twotime(ctx, basis, A, T, args.prec, C_out=C, g2_out=g2, count_out=cnt)

        flops = 2.0 * n_q * k * T * (T + 1) / 2
    else:
        gw = dict(GROUPED_SMALL)
        from synth import sector_qmap

        H, W, T, n_q, k = gw["H"], gw["W"], gw["T"], gw["n_q"], gw["k"]
        qfull = sector_qmap(H, W, n_annuli=8, n_sectors=8, min_px=gw["min_px"], max_px=gw["max_px"],
                            seed=gw["seed"])
        pix = np.flatnonzero(qfull >= 0)
        M = (pix.size + 7) // 8 * 8
        qmap = np.full(M, -1, dtype=np.int32)
        qmap[:pix.size] = qfull[pix]
        gen = TorchSpeckle(H, W, gw["mean"], gw["D"], gw["seed"], dtype=gw["dtype"], device=str(dev))
        Xd = torch.zeros((T, M), dtype=torch.uint16, device=dev)
        pix_d = torch.from_numpy(pix.astype(np.int64)).to(dev)
        for i in range(0, T, 1000):
            Xd[i:i + 1000, :pix.size].copy_(gen.next(min(1000, T - i)).index_select(1, pix_d))
        del gen
        ctx = X.Context(0, 0, stream.cuda_stream)
        rings = X.Rings(ctx, torch.from_numpy(qmap).to(dev), M, n_q)
        basis = X.xpcs_fit_basis(ctx, rings, Xd, gw["n_fit"], k)
        A = torch.empty((T, k), dtype=torch.float32, device=dev)
        g2 = torch.empty((n_q, T), dtype=torch.float64, device=dev)
        cnt = torch.empty((n_q, T), dtype=torch.int64, device=dev)
        X.xpcs_encode(ctx, basis, Xd, T, A)

        def call():
            X.xpcs_twotime(ctx, basis, A, T, args.prec, g2_out=g2, count_out=cnt)

        flops = 2.0 * n_q * k * T * (T + 1) / 2
        out["masks_px"] = int(pix.size)
    ctx.set_async(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed():
        for _ in range(args.warmup):
            call()
        ctx.synchronize()
        ctx.profile_enable(True)
        e0.record(stream)
        for _ in range(args.steps):
            call()
        e1.record(stream)
        ctx.synchronize()
        kern = {k_: v[0] / max(1, v[1]) for k_, v in ctx.profile().items()}
        ctx.profile_enable(False)
        return e0.elapsed_time(e1) / args.steps, kern

    if args.sweep:  # every (tiles per item, schedule) of the two-time kernel
        sweep = {}
        for sched in X.SCHEDULES:
            for tiles in (1, 2, 4, 8, 16, 32):
                ctx.twotime_config(tiles, sched)
                _, kern = timed()
                sweep[f"{sched}/{tiles}"] = kern.get("twotime_gram")
        ctx.twotime_config(0)
        out["gram_ms_by_config"] = sweep
    out["ms_per_call"], out["kernels_ms"] = timed()
    gm = out["kernels_ms"].get("twotime_gram")
    out["gram_tflops_one_product"] = flops / (gm * 1e-3) / 1e12 if gm else None
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp16", "bf16", "bf16x3"])
    ap.add_argument("--no-raw", action="store_true")
    ap.add_argument("--no-host", action="store_true",
                    help="skip the host-side legs (e2e, sampled parity, CPU baseline); for profiler runs")
    ap.add_argument("--workload", default="c2", choices=["c2", "small"])
    ap.add_argument("--no-stream", action="store_true", help="skip the online stream leg")
    ap.add_argument("--no-grouped", action="store_true", help="skip the grouped 64-mask leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the multi-stream serving leg")
    ap.add_argument("--serving-seconds", type=float, default=5.0, help="arrival window of the serving leg")
    ap.add_argument("--stream-seconds", type=float, default=10.0, help="paced part of the stream leg")
    ap.add_argument("--stream-capture", choices=["make", "run"],
                    help="profiling aid, no bench line: make = fill the online stream and checkpoint it; "
                         "run = restore it and push three single frames, a 64-frame and a 128-frame step")
    ap.add_argument("--capture-dir", default="/tmp", help="where --stream-capture keeps its basis and checkpoint")
    ap.add_argument("--stream-prec", default="bf16x3", choices=["fp16", "bf16x3"],
                    help="precision of the --stream-capture stream")
    ap.add_argument("--sweep", action="store_true",
                    help="with --leg: also time the two-time kernel in every configuration")
    ap.add_argument("--leg", choices=["raw", "compressed", "grouped"],
                    help="profiling aid, no bench line: run only the raw path or the compressed two-time with C "
                         "stored (on --workload), or the grouped g2-only two-time (small grouped case), and print "
                         "its event-timed call time")
    args = ap.parse_args()
    if args.stream_capture:
        stream_capture(args.stream_capture, args.capture_dir, args.stream_prec)
        return
    if args.leg:
        profile_leg(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = dict(WORKLOAD if args.workload == "c2" else SMALL)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
