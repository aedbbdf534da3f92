"""Adjoint passes and autograd on the GPU against the oracle's adjoints.

Gradients are compared element by element with the oracle (float64) on the same inputs.
The error of each entry is scaled by the adjoint applied to absolute values (the size of
the terms it sums), gate 1e-4 (f32 accumulation over up to a few thousand terms).  At
full workload size the bands the oracle can afford are checked element by element and
the whole result through identities that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import place
from metrics import band, check_grad, harris_backward_scale, to_f64
from paper_1605_06399_gb300 import _abi, autograd, ops, synth

pytestmark = pytest.mark.gpu
TOL_GRAD = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert ops.device_status() == 0


def _gate(gpu, ref, scale, what):
    e = np.abs(to_f64(gpu) - ref) / np.maximum(scale, 1e-30)
    emax = float(e.max()) if e.size else 0.0
    assert emax <= TOL_GRAD, f"{what}: scaled error {emax:.3e}"


SIZES = [(1, 1), (1, 13), (13, 1), (2, 3), (9, 14), (37, 70), (130, 131)]


@pytest.mark.parametrize("k", [1, 3, 5, 7, 11, 15])
@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_conv2d_backward_matches_oracle(k, dt):
    g = np.random.default_rng(5000 + k)
    w = g.standard_normal((k, k)).astype(np.float32)
    for (h, wd) in SIZES:
        x = synth.to_storage(synth.uniform_f32(g, h, wd), dt)
        gr = g.standard_normal((h, wd)).astype(np.float32)
        for border, bv in (("clamp", 0.0), ("constant", 0.5)):
            dx64, dw64 = oracle.conv2d_backward(x, w, gr, border, bv)
            sdx, _ = oracle.conv2d_backward(np.abs(to_f64(x)), np.abs(w), np.abs(gr), border, abs(bv))
            _, sdw = oracle.conv2d_backward(np.abs(to_f64(x)), np.abs(w), np.abs(gr), border, abs(bv))
            for mem, layout in (("host", "dense"), ("device", "padded")):
                taps = torch.from_numpy(w).cuda() if mem == "device" else w
                dx, dw = ops.conv2d_backward(place(torch.from_numpy(gr), layout), place(x, layout), taps,
                                             border, bv)
                what = f"k={k} {dt} {h}x{wd} {border} {mem}"
                _gate(dx, dx64, sdx, "dx " + what)
                _gate(dw, dw64, sdw, "dw " + what)


# equal sides up to 17 run the fused one-pass adjoint, the others the multi-pass form
@pytest.mark.parametrize("nr,nc", [(1, 1), (3, 3), (5, 5), (17, 17), (19, 19), (5, 9), (33, 1), (1, 33), (15, 7)])
@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_sepconv_backward_matches_oracle(nr, nc, dt):
    g = np.random.default_rng(6000 + nr * 40 + nc)
    r = g.standard_normal(nr).astype(np.float32)
    c = g.standard_normal(nc).astype(np.float32)
    for (h, wd) in SIZES:
        x = synth.to_storage(synth.uniform_f32(g, h, wd), dt)
        gr = g.standard_normal((h, wd)).astype(np.float32)
        for border, bv in (("clamp", 0.0), ("constant", 0.25)):
            dx64, dr64, dc64 = oracle.sepconv_backward(x, r, c, gr, border, bv)
            sdx, sdr, sdc = oracle.sepconv_backward(np.abs(to_f64(x)), np.abs(r), np.abs(c), np.abs(gr), border,
                                                    abs(bv))
            for mem, layout in (("host", "dense"), ("device", "padded")):
                rt = torch.from_numpy(r).cuda() if mem == "device" else r
                ct = torch.from_numpy(c).cuda() if mem == "device" else c
                dx, dr, dc = ops.sepconv_backward(place(torch.from_numpy(gr), layout), place(x, layout), rt, ct,
                                                  border, bv)
                what = f"{nr}x{nc} {dt} {h}x{wd} {border} {mem}"
                _gate(dx, dx64, sdx, "dx " + what)
                _gate(dr, dr64, sdr, "drow " + what)
                _gate(dc, dc64, sdc, "dcol " + what)


@pytest.mark.parametrize("wk", [2, 3, 4, 5, 7])
def test_harris_backward_matches_oracle(wk):
    g = np.random.default_rng(7000 + wk)
    sx = synth.sobel_x() + 0.1 * g.standard_normal((3, 3)).astype(np.float32)
    sy = synth.sobel_y() + 0.1 * g.standard_normal((3, 3)).astype(np.float32)
    win = synth.gaussian_window(wk, 1.0) if wk % 2 else (g.random((wk, wk)) + 0.5).astype(np.float32)
    # 150 x 300 holds interior tiles of the fused adjoint (64 x 32 tiles with a 6-pixel halo)
    for (h, wd) in [(1, 1), (3, 7), (16, 16), (45, 60), (100, 133), (150, 300)]:
        img = synth.rectangles_image(g, h, wd, n_rect=10, side_lo=2, side_hi=max(3, min(h, wd)))
        gR = g.standard_normal((h, wd)).astype(np.float32)
        ref = oracle.harris_backward(img, sx, sy, win, gR, 0.04)
        scale = harris_backward_scale(img, sx, sy, win, gR, 0.04)
        for mem in ("host", "device"):
            taps = [torch.from_numpy(np.ascontiguousarray(t)).cuda() if mem == "device" else t for t in (sx, sy, win)]
            dI, dsx, dsy, dw = ops.harris_backward(torch.from_numpy(gR).cuda(), torch.from_numpy(img).cuda(),
                                                   *taps, k=0.04)
            for got, want, s, name in zip((dI, dsx, dsy, dw), ref, scale, ("dI", "dsx", "dsy", "dwin")):
                check_grad(got, want, s, f"{name} wk={wk} {h}x{wd} {mem}")


def test_autograd_wiring():
    g = np.random.default_rng(8000)
    x = synth.to_storage(synth.uniform_f32(g, 40, 57), "f32").cuda().requires_grad_(True)
    w = torch.from_numpy(synth.normal_filter(g, 5)).cuda().requires_grad_(True)
    up = torch.from_numpy(g.standard_normal((40, 57)).astype(np.float32)).cuda()
    (autograd.conv2d(x, w) * up).sum().backward()
    dx64, dw64 = oracle.conv2d_backward(x.detach().cpu(), w.detach().cpu(), up.cpu())
    sdx, sdw = oracle.conv2d_backward(x.detach().cpu().abs(), w.detach().cpu().abs(), up.cpu().abs())
    check_grad(x.grad, dx64, sdx, "autograd conv dx")
    check_grad(w.grad, dw64, sdw, "autograd conv dw")

    x.grad = None
    r = torch.from_numpy(synth.gaussian_taps(3)).cuda().requires_grad_(True)
    c = torch.from_numpy(g.standard_normal(5).astype(np.float32)).cuda().requires_grad_(True)
    (autograd.sepconv(x, r, c) * up).sum().backward()
    dx64, dr64, dc64 = oracle.sepconv_backward(x.detach().cpu(), r.detach().cpu(), c.detach().cpu(), up.cpu())
    sdx, sdr, sdc = oracle.sepconv_backward(x.detach().cpu().abs(), r.detach().cpu().abs(), c.detach().cpu().abs(),
                                            up.cpu().abs())
    check_grad(x.grad, dx64, sdx, "autograd sep dx")
    check_grad(r.grad, dr64, sdr, "autograd sep drow")
    check_grad(c.grad, dc64, sdc, "autograd sep dcol")

    img = torch.from_numpy(synth.rectangles_image(g, 48, 64, n_rect=8, side_lo=4, side_hi=30)).cuda()
    img.requires_grad_(True)
    sx = torch.from_numpy(synth.sobel_x()).cuda().requires_grad_(True)
    sy = torch.from_numpy(synth.sobel_y()).cuda().requires_grad_(True)
    win = torch.from_numpy(synth.gaussian_window(5, 1.0)).cuda().requires_grad_(True)
    upR = torch.from_numpy(g.standard_normal((48, 64)).astype(np.float32)).cuda()
    (autograd.harris(img, sx, sy, win) * upR).sum().backward()
    args = (img.detach().cpu(), synth.sobel_x(), synth.sobel_y(), synth.gaussian_window(5, 1.0), upR.cpu(), 0.04)
    ref = oracle.harris_backward(*args)
    scale = harris_backward_scale(*args)
    for got, want, s, name in zip((img.grad, sx.grad, sy.grad, win.grad), ref, scale, ("dI", "dsx", "dsy", "dwin")):
        check_grad(got, want, s, "autograd harris " + name)


def test_conv2d_backward_8192_bands_and_identities():
    """8192x8192 f32, 11x11 taps: dx checked on row bands against the oracle; dx and dw
    checked over the whole image with <A x, g> = <x, A^T g> and <A_w x, g> = <dw, w>."""
    img, w = synth.workload_conv_f32(11)
    g = np.random.default_rng(8100)
    gr = torch.from_numpy(g.standard_normal((8192, 8192), dtype=np.float32)).cuda()
    x = torch.from_numpy(img).cuda()
    dx, dw = ops.conv2d_backward(gr, x, w)
    grc = gr.cpu().numpy()
    for rows in [(0, 4), (4095, 4099), (8188, 8192)]:
        xb, rb = band(img, rows, 10)
        gb, _ = band(grc, rows, 10)
        dx64, _ = oracle.conv2d_backward(xb, w, gb)
        sdx, _ = oracle.conv2d_backward(np.abs(xb.astype(np.float64)), np.abs(w), np.abs(gb))
        _gate(dx[rows[0]:rows[1]], dx64[rb[0]:rb[1]], sdx[rb[0]:rb[1]], f"dx rows={rows}")
    y = ops.conv2d(x, w)
    lhs = torch.sum(y.double() * gr.double()).item()
    rhs = torch.sum(x.double() * dx.double()).item()
    scale = torch.sum((y.double() * gr.double()).abs()).item()
    assert abs(lhs - rhs) <= 1e-6 * scale
    rhs_w = float(np.sum(dw.cpu().numpy().astype(np.float64) * w.astype(np.float64)))
    assert abs(lhs - rhs_w) <= 1e-6 * scale


def test_harris_backward_4096_identities():
    """4096x4096 rectangles: the Euler identities of the degree-4 (image, Sobel taps)
    and degree-2 (window) homogeneous response hold over the whole image (the element-wise
    comparison with the oracle at this size is in the workload tests)."""
    img, sx, sy, win, k = synth.workload_harris()
    g = np.random.default_rng(8200)
    gR = torch.from_numpy(g.standard_normal((4096, 4096), dtype=np.float32)).cuda()
    x = torch.from_numpy(img).cuda()
    R = ops.harris(x, sx, sy, win, k)
    dI, dsx, dsy, dw = ops.harris_backward(gR, x, sx, sy, win, k)
    ip = torch.sum(gR.double() * R.double()).item()
    scale = torch.sum((gR.double() * R.double()).abs()).item()
    assert abs(torch.sum(dI.double() * x.double()).item() - 4 * ip) <= 1e-4 * scale
    assert abs(float(np.sum(dw.cpu().numpy() * win.astype(np.float64))) - 2 * ip) <= 1e-4 * scale
    t = float(np.sum(dsx.cpu().numpy() * sx.astype(np.float64)) + np.sum(dsy.cpu().numpy() * sy.astype(np.float64)))
    assert abs(t - 4 * ip) <= 1e-4 * scale
