"""Run one stencil workload a few times with a fixed variant, for profiling.

    python -m paper_1605_06399_gb300.profile_cases CASE [--variant JSON] [--reps N] ...

CASE: conv (8192x8192, --k, --in, --out), sep (8192x8192, --radius, --in, --out), harris
(4096x4096 rectangles), batch / batch_bwd (the 256-image ragged batch), conv_bwd,
sep_bwd, harris_bwd.  No tuning runs, so the kernel launch sequence is fixed: one
warm-up call, then --reps calls (the batch also times its 4 tile shapes at creation,
4 launches each, before its first run).
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import Batch, _abi, ops, synth

DT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--variant", default=None,
                    help="variant as key=value pairs, e.g. kind=1,bx=32,by=8,px=4,py=8,load=2 or "
                         "kind=2,bx=8,px=16,py=123,load=2,filt=1 (the tensor-core conv2d, 11x11) "
                         "(default: the built-in choice)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--k", type=int, default=11)
    ap.add_argument("--radius", type=int, default=2)
    ap.add_argument("--in", dest="ind", default="f32")
    ap.add_argument("--out", dest="outd", default="f32")
    a = ap.parse_args(argv)
    v = None
    if a.variant:
        v = {"kind": 1, "unroll": 1, "persistent": 1}
        v.update({kv.split("=")[0]: int(kv.split("=")[1]) for kv in a.variant.split(",")})
    dev = torch.device("cuda")
    c = a.case
    if c in ("conv", "conv_bwd"):
        img, taps = synth.workload_conv_f32(a.k)
        x = synth.to_storage(img, a.ind).to(dev)
        y = torch.empty(x.shape, dtype=DT[a.outd], device=dev)
        g = torch.randn_like(x)
        fn = (lambda: ops.conv2d(x, taps, out=y, variant=v)) if c == "conv" else \
            (lambda: ops.conv2d_backward(g, x, taps))
    elif c in ("sep", "sep_bwd"):
        img, row, col = synth.workload_sep(a.radius)
        x = synth.to_storage(img, a.ind).to(dev)
        y = torch.empty(x.shape, dtype=DT[a.outd], device=dev)
        g = torch.randn(x.shape, device=dev)
        fn = (lambda: ops.sepconv(x, row, col, out=y, variant=v)) if c == "sep" else \
            (lambda: ops.sepconv_backward(g, x, row, col))
    elif c in ("harris", "harris_bwd"):
        img, sx, sy, win, k = synth.workload_harris()
        x = torch.from_numpy(img).to(dev)
        y = torch.empty_like(x)
        g = torch.randn_like(x)
        fn = (lambda: ops.harris(x, sx, sy, win, k, out=y, variant=v)) if c == "harris" else \
            (lambda: ops.harris_backward(g, x, sx, sy, win, k))
    elif c in ("batch", "batch_bwd"):
        items = []
        for it in synth.workload_batch():
            xi = it.image.to(dev)
            d = {"op": it.op, "x": xi, "taps": torch.from_numpy(it.taps).to(dev), "out_dtype": torch.float16}
            if it.op == "sep":
                d["col_taps"] = torch.from_numpy(it.col_taps).to(dev)
            if c == "batch_bwd":
                d["grad_out"] = torch.randn(xi.shape, device=dev)
            items.append(d)
        b = Batch(items, tune_budget_s=1e9)
        fn = b.run if c == "batch" else b.backward
    else:
        raise SystemExit(f"unknown case {c}")
    fn()
    torch.cuda.synchronize()
    for _ in range(a.reps):
        fn()
    torch.cuda.synchronize()
    assert ops.device_status() == 0
    print(f"{c}: ok")


if __name__ == "__main__":
    main()
