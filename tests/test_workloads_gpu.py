"""Parity of the launches the benchmark times, at sizes where they run.

The persistent kernels loop over tiles: a CTA that owns more than one tile refills its
staging ring and carries partial sums from tile to tile.  Small images give every CTA
at most one tile, so these tests use images with at least two tiles per resident CTA
(or the benchmark's own shapes) and compare with the oracle element by element:
bit for bit for integer results, the scaled 1e-5 (forward) or 1e-4 (adjoint) gates for
floating ones.  Adjoint scales are the adjoint applied to absolute values (the size of
the terms each entry sums).
"""
import numpy as np
import pytest
import torch

import oracle
from metrics import (check_float_output, check_grad, check_harris_output, conv_reference, harris_backward_scale,
                     harris_reference, sep_reference, to_f64)
from paper_1605_06399_gb300 import Batch, _abi, ops, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert ops.device_status() == 0
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ forward, the paper's shapes

def test_paper_conv5x5_8192_u8_tuned_bit_exact():
    """§6 non-separable benchmark shape: 8192x8192 u8, 5x5 integer taps in [-4, 4],
    clamped, the tuned launch; the whole int32 result bit for bit."""
    g = np.random.default_rng(1605100)
    img = synth.uniform_u8(g, 8192, 8192)
    w5 = synth.int_filter(g, 5)
    x = torch.from_numpy(img).cuda()
    ops.tune(ops.problem(_abi.OP_CONV2D, "u8", "i32", 5, 5, 8192, 8192), budget_s=4.0, reps=3)
    y = ops.conv2d(x, w5).cpu().numpy()
    ref = oracle.conv2d(img, w5)
    bad = np.argwhere(y != ref)
    assert bad.size == 0, f"{len(bad)} pixels differ, first at {bad[:3].tolist()}"


def test_paper_sep5x5_4096_constant_tuned_whole_image():
    """§6 separable benchmark shape: 4096x4096 f32, 5x5 Gaussian, constant border 0, the
    tuned launch; every pixel within the scaled 1e-5 gate."""
    g = np.random.default_rng(1605101)
    img = synth.uniform_f32(g, 4096, 4096)
    t = synth.gaussian_taps(2)
    x = torch.from_numpy(img).cuda()
    ops.tune(ops.problem(_abi.OP_SEPCONV, "f32", "f32", 5, 5, 4096, 4096, "constant"), budget_s=4.0, reps=3)
    y = ops.sepconv(x, t, t, "constant", 0.0)
    ref, s = sep_reference(img, t, t, "constant", 0.0)
    check_float_output(y, ref, s, torch.float32, "sep 5x5 4096 constant")


@pytest.mark.parametrize("k,dt,out_dtype", [(5, "f16", torch.float32), (11, "bf16", torch.bfloat16),
                                            (15, "f16", torch.float16), (11, "f16", torch.float32)])
def test_conv_16bit_2048_tuned_whole_image(k, dt, out_dtype):
    """16-bit images at 2048x2048 (many tiles per persistent CTA), the tuned launch, the
    whole image against the oracle on the same rounded pixels."""
    g = np.random.default_rng(1605102 + k)
    x = synth.to_storage(synth.uniform_f32(g, 2048, 2048), dt)
    w = synth.normal_filter_l1(g, k)
    ops.tune(ops.problem(_abi.OP_CONV2D, dt, out_dtype, k, k, 2048, 2048), budget_s=3.0, reps=3)
    y = ops.conv2d(x.cuda(), w, out_dtype=out_dtype)
    ref, s = conv_reference(x, w)
    check_float_output(y, ref, s, out_dtype, f"{dt}->{out_dtype} {k}x{k} 2048")


def test_plain_kernels_taller_than_a_grid():
    """1,100,000-row images need more row blocks than a grid may be high (65535 x 16):
    the untuned kernels walk their rows, and the first and last rows match the oracle."""
    g = np.random.default_rng(1605103)
    h = 1_100_000
    img = synth.uniform_f32(g, h, 3)
    x = torch.from_numpy(img).cuda()
    plain = {"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16}
    w = synth.normal_filter_l1(g, 5)
    t = synth.gaussian_taps(2)
    y_conv = ops.conv2d(x, w, variant=plain)
    y_sep = ops.sepconv(x, t, t, variant=plain)
    sx, sy, win = synth.sobel_x(), synth.sobel_y(), synth.gaussian_window(5, 1.0)
    y_har = ops.harris(x, sx, sy, win, 0.04, variant=plain)
    for rows in [(0, 40), (h // 2, h // 2 + 8), (h - 40, h)]:
        ref, s = conv_reference(img, w, rows=rows, halo=2)
        check_float_output(y_conv[rows[0]:rows[1]], ref, s, torch.float32, f"conv rows={rows}")
        ref, s = sep_reference(img, t, t, rows=rows, halo=2)
        check_float_output(y_sep[rows[0]:rows[1]], ref, s, torch.float32, f"sep rows={rows}")
    for rows in [(0, 40), (h - 40, h)]:
        R64, sc = harris_reference(img, sx, sy, win, rows=rows, halo=4)
        check_harris_output(y_har[rows[0]:rows[1]], R64, sc, f"harris rows={rows}")
    # the multi-pass Harris adjoint (a 7x7 window) walks its rows the same way
    del x, y_conv, y_sep, y_har
    img2 = synth.rectangles_image(g, h, 2, n_rect=2000, side_lo=1, side_hi=2000)
    gR = g.standard_normal((h, 2)).astype(np.float32)
    win7 = synth.gaussian_window(7, 1.5)
    dI, dsx, dsy, dw = ops.harris_backward(torch.from_numpy(gR).cuda(), torch.from_numpy(img2).cuda(), sx, sy, win7)
    ref = oracle.harris_backward(img2, sx, sy, win7, gR, 0.04)
    sc = harris_backward_scale(img2, sx, sy, win7, gR, 0.04)
    for got, want, s, name in zip((dI, dsx, dsy, dw), ref, sc, ("dI", "dsx", "dsy", "dwin")):
        check_grad(got, want, s, f"tall harris 7x7 {name}")


# ------------------------------------------------------------------ adjoints, multi-tile

SEP_BWD_CASES = [(2, "f32", "clamp", 0.0), (2, "f32", "constant", 0.25), (8, "f32", "clamp", 0.0),
                 (2, "f16", "clamp", 0.0), (8, "bf16", "constant", 0.25), (8, "f16", "constant", -0.5)]


@pytest.mark.parametrize("radius,dt,border,bv", SEP_BWD_CASES)
def test_sep_backward_fused_multitile(radius, dt, border, bv):
    """The fused separable adjoint (64x32 tiles, persistent CTAs carrying their tap sums
    from tile to tile, a two-stage TMA ring for f32 operands) on 2048x1536: 1536 tiles,
    several per resident CTA.  dx, drow and dcol element by element."""
    g = np.random.default_rng(1605200 + radius)
    h, w = 1536, 2048
    x = synth.to_storage(synth.uniform_f32(g, h, w), dt)
    gr = g.standard_normal((h, w)).astype(np.float32)
    r = synth.gaussian_taps(radius)
    c = g.standard_normal(2 * radius + 1).astype(np.float32)
    dx, dr, dc = ops.sepconv_backward(torch.from_numpy(gr).cuda(), x.cuda(), r, c, border, bv)
    dx64, dr64, dc64 = oracle.sepconv_backward(x, r, c, gr, border, bv)
    sdx, sdr, sdc = oracle.sepconv_backward(np.abs(to_f64(x)), np.abs(r), np.abs(c), np.abs(gr), border, abs(bv))
    what = f"R={radius} {dt} {border}"
    check_grad(dx, dx64, sdx, "dx " + what)
    check_grad(dr, dr64, sdr, "drow " + what)
    check_grad(dc, dc64, sdc, "dcol " + what)


def test_sep_backward_8192_benchmark_shape():
    """The benchmark's separable adjoint: 8192x8192 f32, radius 2 Gaussian taps, clamped.
    The tap gradients entry by entry over the whole image, dx on the whole image."""
    img, _ = synth.workload_conv_f32(11)
    g = np.random.default_rng(1605210)
    gr = g.standard_normal((8192, 8192), dtype=np.float32)
    t5 = synth.gaussian_taps(2)
    dx, dr, dc = ops.sepconv_backward(torch.from_numpy(gr).cuda(), torch.from_numpy(img).cuda(), t5, t5)
    dx64, dr64, dc64 = oracle.sepconv_backward(img, t5, t5, gr)
    sdx, sdr, sdc = oracle.sepconv_backward(img.astype(np.float64), np.abs(t5), np.abs(t5), np.abs(gr))
    check_grad(dr, dr64, sdr, "drow 8192")
    check_grad(dc, dc64, sdc, "dcol 8192")
    check_grad(dx, dx64, sdx, "dx 8192")


@pytest.mark.parametrize("k,h,w", [(5, 2048, 4096), (11, 3072, 3072), (3, 1024, 5000)])
def test_conv2d_backward_taps_multitile(k, h, w):
    """conv2d adjoint with the TMA-staged tap-gradient reduction (128x64 tiles, grid capped
    at the resident CTAs, so each CTA reduces several tiles): dw entry by entry and dx
    element by element over the whole image."""
    g = np.random.default_rng(1605300 + k)
    x = synth.uniform_f32(g, h, w)
    gr = g.standard_normal((h, w)).astype(np.float32)
    wt = synth.normal_filter_l1(g, k)
    for border, bv in (("clamp", 0.0), ("constant", 0.5)):
        dx, dw = ops.conv2d_backward(torch.from_numpy(gr).cuda(), torch.from_numpy(x).cuda(), wt, border, bv)
        dx64, dw64 = oracle.conv2d_backward(x, wt, gr, border, bv)
        sdx, sdw = oracle.conv2d_backward(x.astype(np.float64), np.abs(wt), np.abs(gr), border, abs(bv))
        check_grad(dw, dw64, sdw, f"dw {k}x{k} {h}x{w} {border}")
        check_grad(dx, dx64, sdx, f"dx {k}x{k} {h}x{w} {border}")


def test_harris_backward_4096_entrywise():
    """The benchmark's Harris adjoint (4096x4096 rectangles, Sobel, 5x5 Gaussian window):
    dI over the whole image and the Sobel and window gradients entry by entry, each
    scaled by the adjoint on absolute values."""
    img, sx, sy, win, k = synth.workload_harris()
    g = np.random.default_rng(1605400)
    gR = g.standard_normal((4096, 4096), dtype=np.float32)
    dI, dsx, dsy, dw = ops.harris_backward(torch.from_numpy(gR).cuda(), torch.from_numpy(img).cuda(), sx, sy, win, k)
    ref = oracle.harris_backward(img, sx, sy, win, gR, k)
    sc = harris_backward_scale(img, sx, sy, win, gR, k)
    for got, want, s, name in zip((dI, dsx, dsy, dw), ref, sc, ("dI", "dsx", "dsy", "dwin")):
        check_grad(got, want, s, f"harris 4096 {name}")


def test_batch_backward_workload_sampled():
    """The benchmark's ragged batch (256 f16 images, f16 outputs) with an f32 upstream
    gradient per image, forward then adjoint in their graph launches.  A sample of
    images (the largest conv and separable ones, and a spread of others) is checked
    against the oracle adjoint: the input gradient over the whole image, the tap
    gradients entry by entry."""
    items = synth.workload_batch()
    g = np.random.default_rng(1605500)
    bitems, grads = [], []
    for it in items:
        gr = g.standard_normal((it.height, it.width)).astype(np.float32)
        d = {"op": it.op, "x": it.image.cuda(), "taps": torch.from_numpy(it.taps).cuda(),
             "out_dtype": torch.float16, "grad_out": torch.from_numpy(gr).cuda()}
        if it.op == "sep":
            d["col_taps"] = torch.from_numpy(it.col_taps).cuda()
        bitems.append(d)
        grads.append(gr)
    b = Batch(bitems, tune_budget_s=2.0)
    b.run()
    gin, gt, gt2 = b.backward()
    torch.cuda.synchronize()
    px = [it.width * it.height for it in items]
    conv = sorted((i for i, it in enumerate(items) if it.op == "conv"), key=lambda i: -px[i] * items[i].k ** 2)
    sep = sorted((i for i, it in enumerate(items) if it.op == "sep"), key=lambda i: -px[i])
    sample = sorted(set(conv[:3] + sep[:2] + conv[-1:] + sep[-1:] + list(range(0, 256, 37))))
    for i in sample:
        it, gr = items[i], grads[i]
        x64 = it.image.double().numpy()
        what = f"item {i} {it.op} k={it.k} {it.height}x{it.width}"
        if it.op == "conv":
            dx64, dw64 = oracle.conv2d_backward(it.image, it.taps, gr)
            sdx, sdw = oracle.conv2d_backward(np.abs(x64), np.abs(it.taps), np.abs(gr))
            check_grad(gin[i], dx64, sdx, "dx " + what)
            check_grad(gt[i], dw64, sdw, "dw " + what)
        else:
            dx64, dr64, dc64 = oracle.sepconv_backward(it.image, it.taps, it.col_taps, gr)
            sdx, sdr, sdc = oracle.sepconv_backward(np.abs(x64), np.abs(it.taps), np.abs(it.col_taps), np.abs(gr))
            check_grad(gin[i], dx64, sdx, "dx " + what)
            check_grad(gt[i], dr64, sdr, "drow " + what)
            check_grad(gt2[i], dc64, sdc, "dcol " + what)
    b.close()
