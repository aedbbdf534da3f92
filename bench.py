#!/usr/bin/env python3
"""Throughput of the stencil hot path on one GB300 (or N replicas under torchrun).

One step = the non-separable correlation of one 8192x8192 f32 image (pixels uniform
[0, 1)) with a 5x5 and an 11x11 filter (N(0,1) taps divided by their L1 norm),
clamp-to-edge, each through ``imagecl_conv2d`` with the variant the auto-tuner picked.
``value`` is output Mpixel/s of the whole job (both filters, all ranks).  Inputs and
outputs (268 MB each) are larger than L2, so no flush is needed between steps.

Also reported: per-stencil tuned vs plain throughput and roofline fractions, the
dominant kernel's roofline (CUDA events on its own stream over the timed region), the
end-to-end rate through the C ABI with host buffers, SM clocks sampled during the timed
region, and the CPU oracle timed on a bounded sample (``cpu_baseline``).

``--impl reference`` times the CPU oracle itself (the reference arm) on the same
workload, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import ctypes
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
sys.path.insert(0, ROOT)

METRIC = "Mpixel/s and % HBM roofline per stencil, tuned vs plain, at stated tol"
WORKLOAD = ("non-separable 2D correlation, one 8192x8192 f32 image (uniform [0,1)), "
            "5x5 and 11x11 N(0,1) taps normalised to unit L1 sum, clamp-to-edge")
SIDE = 8192
KS = (5, 11)
FALLBACK_HBM_GBS, FALLBACK_BF16_TFS = 6800.0, 1900.0
FP32_FMA_PER_SM_CLK = 128          # FP32 lanes per SM (4 sub-partitions x 32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="weak", choices=["weak", "strong"],
                    help="weak: every rank runs the whole workload (replicas); strong: the one image is "
                         "split into row bands across the ranks, with a halo exchange every step")
    ap.add_argument("--tune-budget", type=float, default=20.0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-stencil measurements of the other workloads")
    ap.add_argument("--tune-cache", default=None,
                    help="tuning cache file: loaded (and tuning skipped) if it exists, "
                         "written after tuning otherwise")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers

def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return rank, world, local, pg


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return FALLBACK_HBM_GBS, FALLBACK_BF16_TFS, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.device_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_id_for_smi(local_rank):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local_rank).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[local_rank]
        return str(local_rank)


def kernel_source_hash():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1605_06399_gb300", "csrc")
    for f in ("common.cuh", "tile_common.cuh", "conv2d_kernels.cuh", "conv2d_tiled.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def variant_key(v):
    return ",".join(f"{f}={v[f]}" for f in ("px", "py", "bx", "by", "load", "filt", "map"))


def traffic_record(k, variant):
    """(DRAM bytes read + written per launch, note) for the k x k kernel in this variant,
    from a committed ncu capture, if the kernel sources are unchanged since; (None, why)
    otherwise.  A block shape that was not captured takes the mean over the captured
    shapes of the same per-thread form (they differ by well under 1%), and says so."""
    p = os.path.join(ROOT, "profiles", f"conv2d_tiled_k{k}_8192_f32.traffic.json")
    if not os.path.exists(p):
        return None, "no capture committed"
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash():
        return None, "kernel sources changed since the capture"
    recs = d.get("dram_bytes_per_launch", {})
    key = variant_key(variant)
    if key in recs:
        return recs[key], f"ncu capture of this variant ({os.path.basename(p)})"
    form = {f: variant[f] for f in ("px", "py", "load", "filt", "map")}
    same = [v for kk, v in recs.items()
            if all(f"{f}={form[f]}" in kk.split(",") for f in form)]
    if same:
        return sum(same) / len(same), (f"mean of {len(same)} captured block shapes of this form "
                                       f"({os.path.basename(p)}); this block shape was not captured")
    return None, "this variant was not captured"


def config_of(world):
    """The workload description both arms print."""
    return {"workload": WORKLOAD, "image": f"{SIDE}x{SIDE} f32", "filters": list(KS), "border": "clamp",
            "l2": "inputs and outputs larger than L2 (no flush)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def workload():
    from paper_1605_06399_gb300 import synth
    img, w5 = synth.workload_conv_f32(5)
    _, w11 = synth.workload_conv_f32(11)
    return img, {5: w5, 11: w11}


# ----------------------------------------------------------------------------- CPU oracle

class omp_threads:
    """Run the oracle's OpenMP loops on `n` threads inside the block (the OpenMP runtime
    the oracle library was linked with, set through its own API); restores the count."""

    def __init__(self, n):
        self.n = n
        self.gomp = None
        self.prev = None

    def __enter__(self):
        import oracle
        oracle.default()
        try:
            self.gomp = ctypes.CDLL("libgomp.so.1")
            self.prev = int(self.gomp.omp_get_max_threads())
            self.gomp.omp_set_num_threads(int(self.n))
        except OSError:
            self.gomp = None
        return self

    def __exit__(self, *exc):
        if self.gomp is not None:
            self.gomp.omp_set_num_threads(self.prev)


def oracle_rate(img, taps_by_k, seconds, gpu_outs=None):
    import oracle
    h, w = img.shape
    # calibrate on a thin band, then size the timed sample to about `seconds`
    t0 = time.perf_counter()
    for k, taps in taps_by_k.items():
        r = k // 2
        oracle.conv2d(img[h // 2 - r:h // 2 + 8 + r], taps, rows=(r, r + 8))
    t_cal = time.perf_counter() - t0
    n = max(8, min(h, int(8 * seconds / max(t_cal, 1e-6))))
    y0 = (h - n) // 2
    t0 = time.perf_counter()
    passes = 0
    while True:   # whole passes over the band until the time budget is used
        for k, taps in taps_by_k.items():
            r = k // 2
            a, b = max(0, y0 - r), min(h, y0 + n + r)
            oracle.conv2d(img[a:b], taps, rows=(y0 - a, y0 + n - a))
        passes += 1
        if time.perf_counter() - t0 >= 0.9 * seconds:
            break
    dt = time.perf_counter() - t0
    px = passes * n * w * len(taps_by_k)
    errs = {}
    if gpu_outs is not None:
        for k, taps in taps_by_k.items():
            r = k // 2
            a, b = max(0, y0 - r), min(h, y0 + n + r)
            ref = oracle.conv2d(img[a:b], taps, rows=(y0 - a, y0 + n - a))
            s = oracle.conv2d(np.abs(img[a:b].astype(np.float64)), np.abs(taps.astype(np.float64)),
                              rows=(y0 - a, y0 + n - a))
            g = gpu_outs[k][y0:y0 + n].astype(np.float64)
            errs[k] = float(np.max(np.abs(g - ref) / np.maximum(s, 1e-30)))
    return px / dt / 1e6, (n, passes), oracle.num_threads(), dt, errs


def _scaled(gpu, ref, scale):
    g = np.asarray(gpu, dtype=np.float64)
    return float(np.max(np.abs(g - ref) / np.maximum(scale, 1e-30))) if g.size else 0.0


def _host64(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def error_report(dev):
    """Errors against the float64 oracle, stated per result as the workloads ask.  Each
    error is scaled by the magnitude of the summed terms (the oracle applied to absolute
    values; T^2 for Harris, T = |G| (*) (Ax^2 + Ay^2), A = |S| (*) |I|).

    * separable Gaussian, 8192^2, radius 1..16, every storage pair: the arithmetic error
      (oracle on the rounded pixels the GPU reads) and the storage error (oracle on the
      unrounded f32 pixels, so it includes the 16-bit rounding of the input and output);
    * Harris 5x5 on the 4096^2 rectangles image;
    * the ragged batch forward (f16 outputs) and its adjoint on a sample of images.
    Row bands at the top, middle and bottom of each large image, every column."""
    import torch

    import oracle
    from paper_1605_06399_gb300 import Batch, ops, synth
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    rep = {}

    g = np.random.default_rng(1605003)
    base = synth.uniform_f32(g, SIDE, SIDE)
    bands = [(0, 4), (SIDE // 2 - 2, SIDE // 2 + 2), (SIDE - 4, SIDE)]
    xs = {d: synth.to_storage(base, d) for d in ("f32", "f16", "bf16")}
    xd = {d: xs[d].to(dev) for d in xs}
    sep = {}
    for R in range(1, 17):
        t = synth.gaussian_taps(R)
        at = np.abs(t.astype(np.float64))
        per = {}
        for ind, outd in (("f32", "f32"), ("bf16", "f32"), ("f16", "f32"), ("f16", "f16"), ("bf16", "bf16")):
            y = ops.sepconv(xd[ind], t, t, out_dtype=tdt[outd])
            arith = storage = 0.0
            for (y0, y1) in bands:
                a, b = max(0, y0 - R), min(SIDE, y1 + R)
                rows = (y0 - a, y1 - a)
                yb = _host64(y[y0:y1])
                xr = xs[ind][a:b].double().numpy()
                arith = max(arith, _scaled(yb, oracle.sepconv(xr, t, t, rows=rows),
                                           oracle.sepconv(np.abs(xr), at, at, rows=rows)))
                xu = base[a:b].astype(np.float64)
                storage = max(storage, _scaled(yb, oracle.sepconv(xu, t, t, rows=rows),
                                               oracle.sepconv(np.abs(xu), at, at, rows=rows)))
            per[f"{ind}->{outd}"] = {"arith": arith, "storage": storage}
        sep[f"R{R}"] = per
    rep["sep_8192_per_radius"] = {
        "errors": sep, "sample": "rows 0-3, 4094-4097 and 8188-8191, all columns, default variant",
        "gate": "arith <= 1e-5 for f32 outputs and 2e-3 for f16 outputs (bf16 outputs: one bf16 ulp plus "
                "the f32 bound, checked by the tests); storage error reported, not gated"}
    del xd, xs, base

    img, sx, sy, win, k = synth.workload_harris()
    R_gpu = ops.harris(torch.from_numpy(img).to(dev), sx, sy, win, k)
    e = 0.0
    for (y0, y1) in [(0, 4), (2046, 2050), (4092, 4096)]:
        a, b = max(0, y0 - 4), min(4096, y1 + 4)
        rows = (y0 - a, y1 - a)
        ai = np.abs(img[a:b].astype(np.float64))
        ax, ay = oracle.conv2d(ai, np.abs(sx)), oracle.conv2d(ai, np.abs(sy))
        T = oracle.conv2d(ax * ax + ay * ay, np.abs(win), rows=rows)
        e = max(e, _scaled(_host64(R_gpu[y0:y1]), oracle.harris(img[a:b], sx, sy, win, k, rows=rows), T * T))
    rep["harris_4096"] = {"max_scaled_err": e, "gate": 1e-5, "sample": "rows 0-3, 2046-2049, 4092-4095"}
    del R_gpu

    items = synth.workload_batch()
    gb = np.random.default_rng(1605005)
    bitems, grads = [], []
    for it in items:
        gr = gb.standard_normal((it.height, it.width)).astype(np.float32)
        d = {"op": it.op, "x": it.image.to(dev), "taps": torch.from_numpy(it.taps).to(dev),
             "out_dtype": torch.float16, "grad_out": torch.from_numpy(gr).to(dev)}
        if it.op == "sep":
            d["col_taps"] = torch.from_numpy(it.col_taps).to(dev)
        bitems.append(d)
        grads.append(gr)
    b = Batch(bitems, tune_budget_s=1.0)
    outs = b.run()
    gin, gt, gt2 = b.backward()
    torch.cuda.synchronize()
    px = [it.width * it.height for it in items]
    small = [i for i in range(len(items)) if px[i] <= 1 << 20]
    conv = sorted((i for i in small if items[i].op == "conv"), key=lambda i: -px[i] * items[i].k ** 2)
    sepi = sorted((i for i in small if items[i].op == "sep"), key=lambda i: -px[i])
    sample = sorted(set(conv[:2] + sepi[:2] + conv[-1:] + sepi[-1:]))
    ef = eb = 0.0
    for i in sample:
        it, gr = items[i], grads[i]
        x64 = it.image.double().numpy()
        if it.op == "conv":
            ef = max(ef, _scaled(_host64(outs[i]), oracle.conv2d(x64, it.taps),
                                 oracle.conv2d(np.abs(x64), np.abs(it.taps))))
            dx64, dw64 = oracle.conv2d_backward(x64, it.taps, gr)
            sdx, sdw = oracle.conv2d_backward(np.abs(x64), np.abs(it.taps), np.abs(gr))
            eb = max(eb, _scaled(_host64(gin[i]), dx64, sdx), _scaled(_host64(gt[i]), dw64, sdw))
        else:
            ef = max(ef, _scaled(_host64(outs[i]), oracle.sepconv(x64, it.taps, it.col_taps),
                                 oracle.sepconv(np.abs(x64), np.abs(it.taps), np.abs(it.col_taps))))
            dx64, dr64, dc64 = oracle.sepconv_backward(x64, it.taps, it.col_taps, gr)
            sdx, sdr, sdc = oracle.sepconv_backward(np.abs(x64), np.abs(it.taps), np.abs(it.col_taps), np.abs(gr))
            eb = max(eb, _scaled(_host64(gin[i]), dx64, sdx), _scaled(_host64(gt[i]), dr64, sdr),
                     _scaled(_host64(gt2[i]), dc64, sdc))
    b.close()
    rep["batch256_f16"] = {"fwd_max_scaled_err": ef, "fwd_gate": 2e-3, "bwd_max_scaled_err": eb, "bwd_gate": 1e-4,
                           "sample": f"whole images {sample} (the largest conv and separable items up to 1 Mpx "
                                     "and the smallest of each), forward f16 output, adjoint f32"}
    return rep


# ----------------------------------------------------------------------------- other stencils

def _flush_l2(flush, r):
    """Leave L2 cold and clean before a timed call: overwrite one buffer larger than L2,
    then read another one.  After the write alone L2 is full of that buffer's dirty lines,
    and the timed kernel would pay for writing them back to HBM as its own lines evict
    them; the read pushes them out before the timed region and leaves clean lines only."""
    w, rd = flush
    w.fill_(float(r))
    rd.sum()


def _median_ms(fn, reps, flush=None, calls=8):
    """Median device time of one fn() call.  `calls` calls are recorded in a CUDA graph
    (so host-side argument marshalling is not timed), the graph is replayed `reps` times
    between CUDA events on the current stream, and each replay is divided by `calls`.
    With `flush` (two buffers larger than L2), L2 is flushed before each replay, outside
    the events (_flush_l2), and one call is recorded per replay so that every timed call
    starts cold."""
    import torch
    if flush is not None and calls > 1:
        calls = 1
    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    if calls == 0:   # fn itself replays a CUDA graph: time it directly
        ts = []
        for r in range(reps):
            if flush is not None:
                _flush_l2(flush, r)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[len(ts) // 2]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(calls):
            fn()
    g.replay()
    torch.cuda.synchronize()
    ts = []
    for r in range(reps):
        if flush is not None:
            _flush_l2(flush, r)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / calls)
    ts.sort()
    del g
    return ts[len(ts) // 2]


def _entry(px, tuned_ms, plain_ms, bytes_px, flops_px, hbm_gbs, fp32_peak, variant=None, note=None):
    t = tuned_ms / 1e3
    d = {"tuned_mpx_s": px / t / 1e6, "tuned_ms": tuned_ms,
         "hbm_gbs": bytes_px * px / t / 1e9, "hbm_frac": bytes_px * px / t / 1e9 / hbm_gbs,
         "fp32_tflops": flops_px * px / t / 1e12, "fp32_frac": flops_px * px / t / 1e12 / fp32_peak}
    if plain_ms is not None:
        d.update({"plain_mpx_s": px / (plain_ms / 1e3) / 1e6, "plain_ms": plain_ms,
                  "speedup_vs_plain": plain_ms / tuned_ms})
    if variant is not None:
        d["variant"] = variant
    if note:
        d["note"] = note
    return d


def tc_mma_flops(k, dt, W, H):
    """Flops the tensor-core conv2d variant issues as MMAs for a W x H image: per 128-row
    tile and 16 output columns, two groups of J = (k+1)/2 filter rows, the 32-element K
    window, M = 128, N = 16 J, and three (tf32 split) or two (16-bit taps split) products."""
    J = (k + 1) // 2
    bh = 129 - J
    blocks = -(-H // bh) * -(-W // 16)
    products = 3 if dt == "f32" else 2
    return blocks * 2 * products * 2 * 128 * 16 * J * 32


def extra_stencils(hbm_gbs, fp32_peak, budget, imad_peak=None, bf16_tflops=FALLBACK_BF16_TFS):
    """Tuned vs plain for the other workloads (inputs resident; L2 flushed between runs
    when a working set would fit in L2)."""
    import torch
    from paper_1605_06399_gb300 import Batch, _abi, ops, synth
    out = {}
    dev = torch.device("cuda")
    flush = (torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev),    # 256 MB each, > L2
             torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev))
    plain = {"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16}

    # 512x512 u8, 3x3 integer taps: launch-latency bound, timed by CUDA-graph replay
    img, taps = synth.workload_int3x3()
    x = torch.from_numpy(img).to(dev)
    y = torch.empty((512, 512), dtype=torch.int32, device=dev)
    res = ops.tune(ops.problem(_abi.OP_CONV2D, "u8", "i32", 3, 3, 512, 512), budget_s=budget, reps=5)
    times = {name: _median_ms(lambda v=v: ops.conv2d(x, taps, out=y, variant=v), 7, calls=100)
             for name, v in (("tuned", None), ("plain", plain))}
    out["conv3x3_512_u8_i32"] = _entry(512 * 512, times["tuned"], times["plain"], 5, 18, hbm_gbs, fp32_peak,
                                       res["variant"], "L2-resident, launch-latency bound: % roofline not "
                                       "meaningful; per-launch time from 100 launches in a CUDA graph")
    del x, y

    # separable Gaussian, 8192x8192, radius R, storage types
    g = np.random.default_rng(3)
    base = synth.uniform_f32(g, SIDE, SIDE)
    for R in (2, 8, 16):
        t = synth.gaussian_taps(R)
        for ind, outd in (("f32", "f32"), ("bf16", "f32"), ("f16", "f16"), ("bf16", "bf16")):
            x = synth.to_storage(base, ind).to(dev)
            od = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[outd]
            y = torch.empty((SIDE, SIDE), dtype=od, device=dev)
            res = ops.tune(ops.problem(_abi.OP_SEPCONV, ind, outd, 2 * R + 1, 2 * R + 1, SIDE, SIDE),
                           budget_s=budget, reps=3)
            ws = torch.empty(SIDE * SIDE * 4, dtype=torch.uint8, device=dev)
            tt = _median_ms(lambda: ops.sepconv(x, t, t, out=y), 7)
            tp = _median_ms(lambda: ops.sepconv(x, t, t, out=y, variant=plain, workspace=ws), 5)
            bpx = x.element_size() + y.element_size()
            out[f"sep_R{R}_8192_{ind}_{outd}"] = _entry(SIDE * SIDE, tt, tp, bpx, 4 * (2 * R + 1), hbm_gbs,
                                                        fp32_peak, res["variant"])
            del x, y, ws

    base_large = base
    # the paper's own benchmark shapes (§6): 4096^2 f32 separable 5x5 with the constant
    # border, and 8192^2 u8 non-separable 5x5 with the clamped border
    x = torch.from_numpy(synth.uniform_f32(g, 4096, 4096)).to(dev)
    y = torch.empty_like(x)
    t = synth.gaussian_taps(2)
    res = ops.tune(ops.problem(_abi.OP_SEPCONV, "f32", "f32", 5, 5, 4096, 4096, "constant"), budget_s=budget, reps=3)
    ws = torch.empty(4096 * 4096 * 4, dtype=torch.uint8, device=dev)
    tt = _median_ms(lambda: ops.sepconv(x, t, t, "constant", 0.0, out=y), 7, flush)
    tp = _median_ms(lambda: ops.sepconv(x, t, t, "constant", 0.0, out=y, variant=plain, workspace=ws), 5, flush)
    out["paper_sep5x5_4096_f32_constant"] = _entry(4096 * 4096, tt, tp, 8, 20, hbm_gbs, fp32_peak, res["variant"])
    del x, y, ws
    x = torch.from_numpy(synth.uniform_u8(g, SIDE, SIDE)).to(dev)
    y = torch.empty((SIDE, SIDE), dtype=torch.int32, device=dev)
    w5 = synth.int_filter(g, 5)
    res = ops.tune(ops.problem(_abi.OP_CONV2D, "u8", "i32", 5, 5, SIDE, SIDE), budget_s=budget, reps=3)
    tt = _median_ms(lambda: ops.conv2d(x, w5, out=y), 7)
    tp = _median_ms(lambda: ops.conv2d(x, w5, out=y, variant=plain), 5)
    e = _entry(SIDE * SIDE, tt, tp, 5, 50, hbm_gbs, fp32_peak, res["variant"],
               "50 integer ops per pixel (25 multiply-adds); a tuned variant with unroll=3 (F32_EXACT) does them "
               "as f32 FMAs, exact below 2^24 (fp32_frac is its pipe); int_frac is against the measured int32 "
               "multiply-add rate (imagecl_probe_imad), the pipe of the integer-accumulating variants")
    if imad_peak:
        e["int_tops"] = 50 * SIDE * SIDE / (tt / 1e3) / 1e12
        e["int_frac"] = e["int_tops"] / imad_peak
    out["paper_conv5x5_8192_u8_i32"] = e
    del x, y

    # large filters, where the tensor-core (tcgen05 banded-Toeplitz) variant competes with
    # the FP32-pipe ones: the tuned pick, and both families timed on the same launch
    tensor_peak = {"f32": bf16_tflops * 0.5, "f16": bf16_tflops, "bf16": bf16_tflops}   # tf32 = 1/2 of bf16 (nominal)
    for dt, od, k in (("f32", torch.float32, 13), ("f32", torch.float32, 15), ("bf16", torch.bfloat16, 11),
                      ("bf16", torch.bfloat16, 15), ("f16", torch.float32, 13)):
        x = synth.to_storage(base_large, dt).to(dev)
        y = torch.empty((SIDE, SIDE), dtype=od, device=dev)
        w = synth.normal_filter_l1(g, k)
        prob = ops.problem(_abi.OP_CONV2D, dt, od, k, k, SIDE, SIDE)
        res = ops.tune(prob, budget_s=budget, reps=3)
        vs = ops.variants(prob)
        tcv = [v for v in vs if v["kind"] == _abi.KIND_TENSOR][0]
        tiled = [v for v in vs if v["kind"] == _abi.KIND_TILED][0]
        tt = _median_ms(lambda: ops.conv2d(x, w, out=y), 7)
        t_tc = min(_median_ms(lambda nb=nb: ops.conv2d(x, w, out=y, variant=dict(tcv, bx=nb)), 5) for nb in (4, 8))
        t_fp = _median_ms(lambda: ops.conv2d(x, w, out=y, variant=tiled), 5)
        bpx = x.element_size() + y.element_size()
        e = _entry(SIDE * SIDE, tt, None, bpx, 2 * k * k, hbm_gbs, fp32_peak, res["variant"])
        mma = tc_mma_flops(k, dt, SIDE, SIDE)
        e["tensor_variant"] = {"ms": t_tc, "mpx_s": SIDE * SIDE / t_tc / 1e3,
                               "mma_tflops": mma / (t_tc / 1e3) / 1e12,
                               "mma_frac": mma / (t_tc / 1e3) / 1e12 / tensor_peak[dt],
                               "mma_flops_per_launch": mma, "algorithmic_flops_per_launch": 2 * k * k * SIDE * SIDE,
                               "peak": f"{'tf32' if dt == 'f32' else dt} tensor peak {tensor_peak[dt]:.0f} TFLOP/s "
                                       "(measured bf16 x nominal ratio)"}
        e["fp32_pipe_variant"] = {"ms": t_fp, "mpx_s": SIDE * SIDE / t_fp / 1e3, "variant": tiled}
        e["tensor_speedup_vs_fp32_pipe"] = t_fp / t_tc
        out[f"conv{k}x{k}_8192_{dt}_{str(od)[6:]}"] = e
        del x, y
    del base_large

    # Harris, 4096x4096 rectangles: forward tuned vs the two-kernel form, and the backward
    img, sx, sy, win, k = synth.workload_harris()
    x = torch.from_numpy(img).to(dev)
    y = torch.empty_like(x)
    res = ops.tune(ops.problem(_abi.OP_HARRIS, "f32", "f32", 5, 5, 4096, 4096), budget_s=budget, reps=3)
    ws = torch.empty(2 * 4096 * 4096 * 4, dtype=torch.uint8, device=dev)
    tt = _median_ms(lambda: ops.harris(x, sx, sy, win, k, out=y), 7, flush)
    tp = _median_ms(lambda: ops.harris(x, sx, sy, win, k, out=y, variant=plain, workspace=ws), 5, flush)
    px = 4096 * 4096
    flops_fwd = 2 * 18 * (4100 * 4100) / px + 3 + 2 * 3 * 25 + 7
    out["harris_4096_fwd"] = _entry(px, tt, tp, 8, flops_fwd, hbm_gbs, fp32_peak, res["variant"])
    gR = torch.randn(4096, 4096, device=dev)
    tb = _median_ms(lambda: ops.harris_backward(gR, x, sx, sy, win, k), 5, calls=2)
    # algorithmic: read I and gR, write dI (12 B/px); forward recomputed (flops_fwd) plus
    # the window adjoint and window gradient (2 x 3 x 2 x 25), the Sobel adjoint and
    # Sobel gradients (2 x 2 x 2 x 9) and the product / response derivatives (~16)
    flops_bwd = flops_fwd + 2 * 3 * 2 * 25 + 2 * 2 * 2 * 9 + 16
    out["harris_4096_bwd"] = _entry(px, tb, None, 12, flops_bwd, hbm_gbs, fp32_peak,
                                    note="image, Sobel and window gradients: one fused tile kernel, then the "
                                         "three tap-gradient reductions")
    del x, y, ws, gR

    # conv2d and separable backward on the 8192^2 f32 image: input and tap gradients
    img, w11 = synth.workload_conv_f32(11)
    x = torch.from_numpy(img).to(dev)
    gO = torch.randn_like(x)
    tb = _median_ms(lambda: ops.conv2d_backward(gO, x, w11), 5, calls=2)
    # read g and x, write dx (12 B/px); dx and dw are each a K^2 correlation (4 K^2 flop/px)
    out["conv2d_bwd_11x11_8192_f32"] = _entry(SIDE * SIDE, tb, None, 12, 4 * 121, hbm_gbs, fp32_peak,
                                              note="dx (zero-border correlation + clamp folds) and dw (two-stage)")
    t5 = synth.gaussian_taps(2)
    tb = _median_ms(lambda: ops.sepconv_backward(gO, x, t5, t5), 5, calls=2)
    # dx (two 1D passes), drow and dcol (a 1D pass each to rebuild their operand, then a
    # dot product per tap): 6 x 2 x 5 flop/px; read g and x, write dx
    out["sep_bwd_R2_8192_f32"] = _entry(SIDE * SIDE, tb, None, 12, 6 * 2 * 5, hbm_gbs, fp32_peak,
                                        note="dx, row-tap and column-tap gradients")
    del x, gO

    # the paper's Harris shape (§6): 5120x5120 f32 with a 2x2 box block (offsets -1, 0)
    img, sx, sy, _, k = synth.workload_harris(5120, 5120)
    win2 = synth.box_window(2)
    x = torch.from_numpy(img).to(dev)
    y = torch.empty_like(x)
    res = ops.tune(ops.problem(_abi.OP_HARRIS, "f32", "f32", 2, 2, 5120, 5120), budget_s=budget, reps=3)
    ws = torch.empty(2 * 5120 * 5120 * 4, dtype=torch.uint8, device=dev)
    tt = _median_ms(lambda: ops.harris(x, sx, sy, win2, k, out=y), 7, flush)
    tp = _median_ms(lambda: ops.harris(x, sx, sy, win2, k, out=y, variant=plain, workspace=ws), 5, flush)
    px = 5120 * 5120
    flops_box2 = 2 * 18 * (5122 * 5122) / px + 3 + 2 * 3 * 4 + 7   # algorithmic: a 2x2 window
    out["paper_harris_5120_f32_box2"] = _entry(px, tt, tp, 8, flops_box2, hbm_gbs, fp32_peak, res["variant"],
                                               "the 2x2 block runs in its own fused kernels (products over one extra row and column, 4 window taps)")
    del x, y, ws

    # ragged batch: 256 f16 images, one graph launch forward and one backward
    items = synth.workload_batch()
    bitems = []
    for it in items:
        xi = it.image.to(dev)
        d = {"op": it.op, "x": xi, "taps": torch.from_numpy(it.taps).to(dev), "out_dtype": torch.float16,
             "grad_out": torch.randn(xi.shape, device=dev)}
        if it.op == "sep":
            d["col_taps"] = torch.from_numpy(it.col_taps).to(dev)
        bitems.append(d)
    b = Batch(bitems, tune_budget_s=budget)
    info = b.info()
    tf = _median_ms(b.run, 7, calls=0)
    tbw = _median_ms(b.backward, 5, calls=0)

    def plain_loop():
        for d in bitems:
            if d["op"] == "conv":
                ops.conv2d(d["x"], d["taps"], out_dtype=torch.float16, variant=plain)
            else:
                ops.sepconv(d["x"], d["taps"], d["col_taps"], out_dtype=torch.float16, variant=plain)
    tpl = _median_ms(plain_loop, 3, calls=1)
    bytes_total = sum(it.width * it.height * 4 for it in items)
    flops_total = sum(it.width * it.height * (2 * it.k * it.k if it.op == "conv" else 4 * it.k) for it in items)
    # per-image roofline time: sum of max(bytes / BW, flops / P_fp32)
    roof_ms = sum(max(it.width * it.height * 4 / (hbm_gbs * 1e9),
                      it.width * it.height * (2 * it.k * it.k if it.op == "conv" else 4 * it.k) / (fp32_peak * 1e12))
                  for it in items) * 1e3
    e = _entry(info["pixels"], tf, tpl, bytes_total / info["pixels"], flops_total / info["pixels"], hbm_gbs,
               fp32_peak, note=f"{info['images']} images, {info['tiles']} tiles of {info['tile']}; plain = "
                               "one untuned launch per image")
    e["roofline_frac"] = roof_ms / tf
    out["batch256_f16_fwd"] = e
    # backward, per image: read the f32 upstream gradient and the f16 input, write the f32
    # input gradient (10 B/px); dx and dw each a correlation of the forward's size
    bw_flops = [it.width * it.height * 2 * (2 * it.k * it.k if it.op == "conv" else 4 * it.k) for it in items]
    roof_bwd_ms = sum(max(it.width * it.height * 10 / (hbm_gbs * 1e9), f / (fp32_peak * 1e12))
                      for it, f in zip(items, bw_flops)) * 1e3
    eb = _entry(info["pixels"], tbw, None, 10.0, sum(bw_flops) / info["pixels"], hbm_gbs, fp32_peak,
                note="input and tap gradients of every image, one graph launch (the input gradients in the pipelined tile kernel beside the tap-gradient tiles, then per-image reductions)")
    eb["roofline_frac"] = roof_bwd_ms / tbw
    out["batch256_f16_bwd"] = eb
    b.close()
    return out


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    from paper_1605_06399_gb300 import _abi, ops, shard

    rank, world, local, pg = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hbm_gbs, bf16_tflops, sm_max_mhz, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    fp32_peak = n_sm * FP32_FMA_PER_SM_CLK * 2 * sm_max_mhz * 1e6 / 1e12   # TFLOP/s

    img, taps = workload()
    x = torch.from_numpy(img).to(dev)
    ys = {k: torch.empty_like(x) for k in KS}
    stream = torch.cuda.current_stream()
    lib = _abi.lib()

    # tune each stencil (untimed), then time plain and tuned
    tuned = {}
    cached = args.tune_cache is not None and os.path.exists(args.tune_cache)
    if cached:
        ops.tune_load(args.tune_cache)
    for k in KS:
        prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", k, k, SIDE, SIDE)
        if cached:
            tuned[k] = {"variant": ops.default_variant(prob)}
        else:
            t0 = time.perf_counter()
            tuned[k] = ops.tune(prob, budget_s=args.tune_budget, reps=5)
            tuned[k]["seconds"] = time.perf_counter() - t0
    if args.tune_cache is not None and not cached and rank == 0:
        ops.tune_save(args.tune_cache)
    xi = ops.image(x)
    yi = {k: ops.image(ys[k]) for k in KS}
    tp = {k: np.ascontiguousarray(taps[k], np.float32) for k in KS}
    variants = {k: _abi.Variant.from_dict(tuned[k]["variant"]) for k in KS}
    plain = _abi.Variant.from_dict({"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16})
    sh = ctypes.c_void_p(stream.cuda_stream)

    def launch(k, variant):
        return lib.imagecl_conv2d(ctypes.byref(xi), ctypes.byref(yi[k]),
                                  ctypes.c_void_p(tp[k].ctypes.data), _abi.F32, k, k,
                                  _abi.MEM_HOST, _abi.BORDER_CLAMP, 0.0, ctypes.byref(variant), sh)

    def time_kernel(k, variant, n):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for _ in range(3):
            _abi.check(launch(k, variant))
        torch.cuda.synchronize()
        evs[0].record(stream)
        for _ in range(n):
            _abi.check(launch(k, variant))
        evs[1].record(stream)
        torch.cuda.synchronize()
        return evs[0].elapsed_time(evs[1]) / n

    plain_ms = {k: time_kernel(k, plain, 10) for k in KS}

    # ---------------- timed region: K steps, each = conv 5x5 + conv 11x11
    for _ in range(args.warmup):
        for k in KS:
            _abi.check(launch(k, variants[k]))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(KS) + 1)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(gpu_id_for_smi(local)) if rank == 0 else None
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.2)
    start.record(stream)
    for s in range(args.steps):
        ev[s][0].record(stream)
        for i, k in enumerate(KS):
            launch(k, variants[k])
            ev[s][i + 1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    st = ops.device_status()
    assert st == 0, f"kernel status {st}"
    elapsed_ms = start.elapsed_time(end)
    per_k_ms = {k: sum(ev[s][i].elapsed_time(ev[s][i + 1]) for s in range(args.steps)) / args.steps
                for i, k in enumerate(KS)}
    elapsed_ms = shard.max_over_ranks(elapsed_ms, pg)

    px = SIDE * SIDE
    ms_per_step = elapsed_ms / args.steps
    value = world * px * len(KS) / (ms_per_step / 1e3) / 1e6

    # ---------------- end to end: host buffers, copies inside the timed region.  Each step
    # copies the image in from pinned host memory, runs both filters through the C ABI and
    # copies both results out; steps are pipelined over three streams (copy in, compute,
    # copy out) with two device buffer sets, so one step's copies overlap its neighbours'
    # kernels.  Events: from before the first timed copy-in to after the last copy-out.
    h_in = torch.from_numpy(img).pin_memory()
    h_out = {k: torch.empty((SIDE, SIDE), dtype=torch.float32).pin_memory() for k in KS}
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    xb = [x, torch.empty_like(x)]
    yb = [ys, {k: torch.empty_like(ys[k]) for k in KS}]
    xib = [ops.image(b) for b in xb]
    yib = [{k: ops.image(yb[j][k]) for k in KS} for j in range(2)]
    in_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for i in range(args.e2e_steps + 2):
        j = i % 2
        if i == 2:
            torch.cuda.synchronize()
            if pg:
                pg.barrier()
            e0.record(s_in)
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(comp_done[j])        # step i-2 has read this input buffer
            xb[j].copy_(h_in, non_blocking=True)
            in_done[j].record(s_in)
        stream.wait_event(in_done[j])
        if i >= 2:
            stream.wait_event(out_done[j])          # step i-2 has copied these outputs out
        for k in KS:
            _abi.check(lib.imagecl_conv2d(ctypes.byref(xib[j]), ctypes.byref(yib[j][k]),
                                          ctypes.c_void_p(tp[k].ctypes.data), _abi.F32, k, k, _abi.MEM_HOST,
                                          _abi.BORDER_CLAMP, 0.0, ctypes.byref(variants[k]), sh))
        comp_done[j].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(comp_done[j])
            for k in KS:
                h_out[k].copy_(yb[j][k], non_blocking=True)
            out_done[j].record(s_out)
    e1.record(s_out)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
    e2e_ms = shard.max_over_ranks(e2e_ms, pg)
    e2e_value = world * px * len(KS) / (e2e_ms / 1e3) / 1e6

    # the host link's own rate: plain pinned copies of one step's input (host to device)
    # and outputs (device to host), each alone on its stream; the slower direction bounds
    # the pipelined end-to-end rate
    def copy_ms(fn, stream_):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 1e30
        for _ in range(4):
            torch.cuda.synchronize()
            c0.record(stream_)
            with torch.cuda.stream(stream_):
                fn()
            c1.record(stream_)
            c1.synchronize()
            best = min(best, c0.elapsed_time(c1))
        return best
    h2d_ms = copy_ms(lambda: xb[1].copy_(h_in, non_blocking=True), s_in)
    d2h_ms = copy_ms(lambda: [h_out[k].copy_(yb[1][k], non_blocking=True) for k in KS], s_out)
    link = {"h2d_gbs": px * 4 / (h2d_ms / 1e3) / 1e9, "d2h_gbs": px * 4 * len(KS) / (d2h_ms / 1e3) / 1e9,
            "copy_bound_mpx_s": world * px * len(KS) / (max(h2d_ms, d2h_ms) / 1e3) / 1e6}

    if rank != 0:
        pg.destroy_process_group()
        return

    # ---------------- roofline of the dominant kernel
    bytes_px = 8.0                       # 4 B read + 4 B written per output pixel
    per_stencil = {}
    for k in KS:
        flops = 2.0 * k * k * px
        t = per_k_ms[k] / 1e3
        per_stencil[f"{k}x{k}"] = {
            "tuned_mpx_s": px / t / 1e6,
            "plain_mpx_s": px / (plain_ms[k] / 1e3) / 1e6,
            "speedup_vs_plain": plain_ms[k] / per_k_ms[k],
            "tuned_ms": per_k_ms[k],
            "plain_ms": plain_ms[k],
            "hbm_gbs": bytes_px * px / t / 1e9,
            "hbm_frac": bytes_px * px / t / 1e9 / hbm_gbs,
            "fp32_tflops": flops / t / 1e12,
            "fp32_frac": flops / t / 1e12 / fp32_peak,
            "variant": tuned[k]["variant"],
        }
    dom = max(KS, key=lambda k: per_k_ms[k])
    d = per_stencil[f"{dom}x{dom}"]
    ai = 2.0 * dom * dom / bytes_px                          # flop per HBM byte
    ridge = fp32_peak * 1e3 / hbm_gbs
    traffic, traffic_note = traffic_record(dom, d["variant"])
    if ai > ridge:
        roof = {"bound": "alu", "achieved": d["fp32_tflops"], "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": d["fp32_frac"], "traffic": traffic, "traffic_source": traffic_note,
                "kernel": f"k_conv2d_tiled {dom}x{dom} f32",
                "peak_source": f"{n_sm} SMs x 128 FMA/clk x 2 x {sm_max_mhz:.0f} MHz ({peak_src} max clock)"}
    else:
        roof = {"bound": "hbm", "achieved": d["hbm_gbs"], "peak": hbm_gbs, "unit": "GB/s",
                "frac": d["hbm_frac"], "traffic": traffic, "traffic_source": traffic_note,
                "kernel": f"k_conv2d_tiled {dom}x{dom} f32", "peak_source": f"{peak_src} copy bandwidth"}

    probe = {"ffma_tflops": ops.probe_fp32(False), "ffma2_tflops": ops.probe_fp32(True),
             "imad_tops": ops.probe_imad()}

    # the model-guided tuner (§4: random sample, neural-network cost model, best predicted
    # confirmed) against the exhaustive search on the same problems; the exhaustive
    # winner stays cached
    tuning = {}
    if not cached:
        for k in KS:
            prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", k, k, SIDE, SIDE)
            m = ops.tune_model(prob, n_sample=36, n_confirm=10, reps=5, seed=1605)
            ops.tune_set(prob, tuned[k]["variant"])
            tuning[f"{k}x{k}"] = {
                "exhaustive": {"seconds": tuned[k].get("seconds"), "best_ms": tuned[k].get("best_ms"),
                               "candidates": m["report"]["candidates"]},
                "model_guided": {"seconds": m["report"]["seconds"], "best_ms": m["best_ms"],
                                 "timed": m["report"]["sampled"] + m["report"]["confirmed"] + m["report"]["holdout"],
                                 "timed_fraction": (m["report"]["sampled"] + m["report"]["confirmed"]
                                                    + m["report"]["holdout"]) / m["report"]["candidates"],
                                 "model_rmse_log_train": m["report"]["model_rmse"],
                                 "model_rmse_log_holdout": m["report"]["holdout_rmse"],
                                 "holdout_valid": m["report"]["holdout_valid"],
                                 "found_vs_exhaustive": m["best_ms"] / tuned[k]["best_ms"]},
                "paper": "about 1700 candidates and 2 hours per device and benchmark (compile-per-candidate)",
            }
    if not args.no_extras:
        per_stencil.update(extra_stencils(hbm_gbs, fp32_peak, max(2.0, args.tune_budget / 4), probe["imad_tops"],
                                          bf16_tflops))

    gpu_outs = None
    cpu = None
    errs = {}
    error_rep = None
    if not args.no_cpu_baseline:
        for k in KS:
            launch(k, variants[k])
        torch.cuda.synchronize()
        gpu_outs = {k: ys[k].cpu().numpy() for k in KS}
        rate, rows, threads, secs, errs = oracle_rate(img, taps, args.cpu_seconds, gpu_outs)
        cpu = {"value": rate, "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
               "sample": f"{rows[1]} pass(es) over rows {rows[0]} of 8192 (all 8192 columns) "
                         f"through both filters, fp64, {secs:.1f} s"}
        with omp_threads(1) as ot:
            rate1, rows1, _, secs1, _ = oracle_rate(img, taps, args.cpu_seconds / 3)
        if ot.gomp is not None:
            cpu["one_thread"] = {"value": rate1, "unit": "Mpixel/s", "cores": 1,
                                 "sample": f"{rows1[1]} pass(es) over rows {rows1[0]} of 8192, {secs1:.1f} s"}
        if not args.no_extras:
            error_rep = error_report(dev)

    line = {
        "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": config_of(world),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "Mpixel/s",
                "h2d_bytes_per_step": px * 4, "d2h_bytes_per_step": px * 4 * len(KS),
                "mode": "pipelined: copy in / compute / copy out on three streams, two device buffer sets",
                "host_link": link},
        "clocks": clocks,
        "gpu_launches": args.steps * len(KS),
        "per_stencil": per_stencil,
        "fp32_probe": probe,
        "tuning": tuning,
        "max_scaled_err": {f"{k}x{k}": errs.get(k) for k in KS} if errs else None,
        "tolerance": 1e-5,
        "errors_vs_fp64": error_rep,
    }
    print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    img, taps = workload()
    h, w = img.shape
    # one bounded sample per step: a band of rows sized from a calibration run
    t0 = time.perf_counter()
    for k in KS:
        r = k // 2
        oracle.conv2d(img[h // 2 - r:h // 2 + 8 + r], taps[k], rows=(r, r + 8))
    t_cal = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)            # seconds per step
    rows = int(max(8, min(h, 8 * budget / max(t_cal, 1e-6))))
    y0 = (h - rows) // 2

    def step():
        for k in KS:
            r = k // 2
            a, b = max(0, y0 - r), min(h, y0 + rows + r)
            oracle.conv2d(img[a:b], taps[k], rows=(y0 - a, y0 + rows - a))
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = rows * w * len(KS) / dt / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": config_of(int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"rows {rows} of 8192 (all columns), both filters, per step"},
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_strong(args):
    """Strong scaling of one 8192x8192 image over the ranks: each rank owns a band of
    rows plus a halo of r = 5 rows on each side (the 11x11 filter's reach), refreshes the
    halo from its neighbours every step (one batched point-to-point exchange, NCCL
    between GPUs) and runs both filters on its extended band.  value = image pixels x 2
    filters / the slowest rank's time per step.  The input and outputs stay resident;
    e2e adds the band's host copies."""
    import torch
    from paper_1605_06399_gb300 import _abi, ops, shard

    rank, world, local, pg = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    img, taps = workload()
    halo = max(KS) // 2
    bands = shard.row_bands(SIDE, world, halo)
    y0, y1, e0, e1 = bands[rank]
    ext = torch.from_numpy(img[e0:e1]).to(dev)
    outs = {k: torch.empty_like(ext) for k in KS}
    tuned = {}
    for k in KS:
        prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", k, k, SIDE, e1 - e0)
        tuned[k] = ops.tune(prob, budget_s=args.tune_budget, reps=3)["variant"]

    def step():
        if pg is not None:
            shard.exchange_halos(ext, bands, rank, pg)
        for k in KS:
            ops.conv2d(ext, taps[k], out=outs[k], variant=tuned[k])

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(gpu_id_for_smi(local)) if rank == 0 else None
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.2)
    e_start.record(stream)
    for _ in range(args.steps):
        step()
    e_end.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    assert ops.device_status() == 0
    ms = shard.max_over_ranks(e_start.elapsed_time(e_end) / args.steps, pg)
    px = SIDE * SIDE
    value = px * len(KS) / (ms / 1e3) / 1e6

    # end to end: the band's rows in from pinned host memory, its own output rows out
    h_in = torch.from_numpy(img[e0:e1]).pin_memory()
    h_out = {k: torch.empty((y1 - y0, SIDE), dtype=torch.float32).pin_memory() for k in KS}
    for _ in range(2):
        ext.copy_(h_in, non_blocking=True)
        step()
        for k in KS:
            h_out[k].copy_(outs[k][y0 - e0:y1 - e0], non_blocking=True)
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(args.e2e_steps):
        ext.copy_(h_in, non_blocking=True)
        step()
        for k in KS:
            h_out[k].copy_(outs[k][y0 - e0:y1 - e0], non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = shard.max_over_ranks(c0.elapsed_time(c1) / args.e2e_steps, pg)
    if rank != 0:
        pg.destroy_process_group()
        return
    cfg = config_of(world)
    cfg["parallelism"] = f"row bands over {world} rank(s), halo {halo} rows, batched point-to-point exchange"
    line = {
        "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "e2e": {"value": px * len(KS) / (e2e_ms / 1e3) / 1e6, "unit": "Mpixel/s",
                "h2d_bytes_per_step": (e1 - e0) * SIDE * 4, "d2h_bytes_per_step": (y1 - y0) * SIDE * 4 * len(KS),
                "mode": "serial on one stream: band copy in, exchange, both filters, own rows out"},
        "clocks": clocks, "gpu_launches": args.steps * len(KS), "variants": {f"{k}x{k}": tuned[k] for k in KS},
    }
    print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "ours" and args.mode == "strong":
        run_strong(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
