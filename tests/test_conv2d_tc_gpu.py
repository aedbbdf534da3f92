"""The tensor-core (tcgen05, banded-Toeplitz) conv2d variant against the oracle.

The variant covers sides 9..15 for f32 (tf32 operands split into high and low parts),
f16 and bf16 images (exact operands, split taps).  Its results are held to the same
gates as the FP32-pipe variants: the scaled 1e-5 error for f32 outputs, 2e-3 for f16
outputs, one bf16 ulp plus the f32 bound for bf16 outputs.  Sizes span several row
bands (129 - J output rows each) and column segments, ragged right and bottom edges
and images narrower or shorter than one band.
"""
import numpy as np
import pytest
import torch

from gpu_util import assert_pads_intact, empty_padded, padded
from metrics import check_float_output, conv_reference
from paper_1605_06399_gb300 import ImclError, _abi, ops, synth

pytestmark = pytest.mark.gpu

PAIRS = [("f32", torch.float32), ("f16", torch.float32), ("f16", torch.float16), ("bf16", torch.float32),
         ("bf16", torch.bfloat16)]


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert ops.device_status() == 0


def _tensor_variants(dt, out_dtype, k, w, h, taps_mem=_abi.MEM_HOST):
    prob = ops.problem(_abi.OP_CONV2D, dt, out_dtype, k, k, w, h, "clamp", taps_mem)
    vs = [v for v in ops.variants(prob) if v["kind"] == _abi.KIND_TENSOR]
    assert vs, f"no tensor-core variant compiled for {dt}->{out_dtype} {k}x{k}"
    return vs


@pytest.mark.parametrize("k", [9, 11, 13, 15])
@pytest.mark.parametrize("dt,out_dtype", PAIRS, ids=[f"{a}-{str(b)[6:]}" for a, b in PAIRS])
def test_tensor_variant_matches_oracle(dt, out_dtype, k):
    g = np.random.default_rng(11000 + k)
    w = synth.normal_filter_l1(g, k)
    v0 = _tensor_variants(dt, out_dtype, k, 64, 64)[0]
    for (h, wd) in [(1, 1), (7, 13), (130, 259), (300, 517), (251, 40)]:
        x = synth.to_storage(synth.uniform_f32(g, h, wd), dt)
        for border, bv in (("clamp", 0.0), ("constant", 0.375)):
            ref, s = conv_reference(x, w, border, bv)
            for nb, mem, layout in ((16, "host", "dense"), (1, "device", "padded"), (4, "host", "padded")):
                xd = x.cuda() if layout == "dense" else padded(x)
                taps = torch.from_numpy(w).cuda() if mem == "device" else w
                out = empty_padded(h, wd, out_dtype) if layout == "padded" else None
                if xd.stride(0) * xd.element_size() % 16:   # TMA staging needs 16-byte rows
                    with pytest.raises(ImclError) as ei:
                        ops.conv2d(xd, taps, border, bv, out=out, out_dtype=out_dtype, variant=dict(v0, bx=nb))
                    assert ei.value.status == _abi.ERR_ALIGN
                    continue
                y = ops.conv2d(xd, taps, border, bv, out=out, out_dtype=out_dtype, variant=dict(v0, bx=nb))
                if out is not None:
                    assert_pads_intact(out, "tensor conv2d")
                check_float_output(y, ref, s, out_dtype, f"{dt}->{out_dtype} k={k} {h}x{wd} {border} nb={nb} {mem}")


@pytest.mark.parametrize("k,dt,out_dtype", [(11, "f32", torch.float32), (15, "bf16", torch.bfloat16),
                                            (9, "f16", torch.float16), (13, "f32", torch.float32)])
def test_tensor_variant_multitile_whole_image(k, dt, out_dtype):
    """2048x2304: 17 bands x 9 segments of 256 columns (several units per persistent CTA,
    the slab ring and the double-buffered accumulator wrapping many times)."""
    g = np.random.default_rng(11100 + k)
    x = synth.to_storage(synth.uniform_f32(g, 2048, 2304), dt)
    w = synth.normal_filter_l1(g, k)
    v = _tensor_variants(dt, out_dtype, k, 2304, 2048)[0]
    y = ops.conv2d(x.cuda(), w, out_dtype=out_dtype, variant=v)
    ref, s = conv_reference(x, w)
    check_float_output(y, ref, s, out_dtype, f"{dt} {k}x{k} 2048x2304")


@pytest.mark.parametrize("k", [11, 15])
def test_tensor_variant_8192_workload_rows(k):
    """The 8192x8192 f32 workload with unit-L1 N(0,1) taps, every tensor unit width the
    tuner may pick, checked on row bands at the top, across a band seam and at the bottom."""
    img, w = synth.workload_conv_f32(k) if k == 11 else (synth.workload_conv_f32(11)[0],
                                                          synth.normal_filter_l1(np.random.default_rng(5), 15))
    x = torch.from_numpy(img).cuda()
    for v in _tensor_variants("f32", torch.float32, k, 8192, 8192)[:1]:
        for nb in (16, 32):
            y = ops.conv2d(x, w, variant=dict(v, bx=nb))
            for rows in [(0, 6), (117, 129), (4090, 4101), (8186, 8192)]:
                ref, s = conv_reference(img, w, rows=rows, halo=k // 2)
                check_float_output(y[rows[0]:rows[1]], ref, s, torch.float32, f"k={k} nb={nb} rows={rows}")
    del x
    torch.cuda.empty_cache()


def test_tensor_variant_rejects_unaligned_input():
    g = np.random.default_rng(11200)
    base = synth.to_storage(synth.uniform_f32(g, 64, 81), "f32").cuda()
    v = _tensor_variants("f32", torch.float32, 11, 80, 64)[0]
    with pytest.raises(ImclError) as ei:
        ops.conv2d(base[:, 1:], synth.normal_filter_l1(g, 11), variant=v)
    assert ei.value.status == _abi.ERR_ALIGN


def test_tuner_offers_the_tensor_variant_and_its_pick_is_correct():
    """The exhaustive tuner times the tensor variant beside the FP32-pipe ones (it passes
    the tuner's own check against PLAIN); whatever wins, the cached pick matches the oracle."""
    g = np.random.default_rng(11300)
    x = synth.to_storage(synth.uniform_f32(g, 1536, 2048), "bf16")
    w = synth.normal_filter_l1(g, 13)
    prob = ops.problem(_abi.OP_CONV2D, "bf16", torch.float32, 13, 13, 2048, 1536)
    res = ops.tune(prob, budget_s=5.0, reps=3)
    y = ops.conv2d(x.cuda(), w)
    ref, s = conv_reference(x, w)
    check_float_output(y, ref, s, torch.float32, f"tuned {res['variant']}")
