"""Harris response on the GPU (fused and two-kernel forms) against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import assert_pads_intact, out_buffer, place
from metrics import check_harris_output, harris_reference
from paper_1605_06399_gb300 import ImclError, _abi, ops, synth

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (1, 23), (23, 1), (4, 5), (40, 70), (133, 261), (64, 300)]


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert ops.device_status() == 0


def _variants(wk, w, h, mem):
    prob = ops.problem(_abi.OP_HARRIS, "f32", "f32", wk, wk, w, h, "clamp", mem)
    vs = ops.variants(prob)
    extra = [dict(v, bx=bx, by=by) for v in vs if v["kind"] == _abi.KIND_TILED and v["load"] == _abi.LOAD_TMA
             for bx, by in ((32, 8), (8, 32), (16, 8))]
    return [None] + vs + extra


def _window(g, wk):
    if wk == 1:
        return np.ones((1, 1), np.float32)
    if wk % 2:
        return synth.gaussian_window(wk, 1.0)
    return (g.random((wk, wk)) + 0.5).astype(np.float32)   # even: no symmetry to hide the anchor


@pytest.mark.parametrize("wk", [1, 2, 3, 4, 5, 6, 7])
def test_harris_every_variant_matches_oracle(wk):
    g = np.random.default_rng(3000 + wk)
    sx = synth.sobel_x() + 0.1 * g.standard_normal((3, 3)).astype(np.float32)
    sy = synth.sobel_y() + 0.1 * g.standard_normal((3, 3)).astype(np.float32)
    win = _window(g, wk)
    n = 0
    for (h, w) in SIZES:
        img = synth.rectangles_image(g, h, w, n_rect=12, side_lo=2, side_hi=max(3, min(h, w)))
        R64, sc = harris_reference(img, sx, sy, win)
        x = torch.from_numpy(img)
        for mem, layout in ((_abi.MEM_HOST, "dense"), (_abi.MEM_HOST, "padded"), (_abi.MEM_DEVICE, "padded"),
                            (_abi.MEM_DEVICE, "dense")):
            xd = place(x, layout)
            taps = [torch.from_numpy(np.ascontiguousarray(t)).cuda() if mem == _abi.MEM_DEVICE else t
                    for t in (sx, sy, win)]
            for v in _variants(wk, w, h, mem):
                out = out_buffer(h, w, torch.float32, layout)
                try:
                    y = ops.harris(xd, *taps, k=0.04, out=out, variant=v)
                except ImclError as e:
                    assert e.status in (_abi.ERR_UNSUPPORTED, _abi.ERR_ALIGN), str(e)
                    continue
                if out is not None:
                    assert_pads_intact(out, f"harris {v}")
                check_harris_output(y, R64, sc, f"wk={wk} {h}x{w} mem={mem} {layout} {v}")
                n += 1
    assert n > 0


def test_harris_workload_4096_sampled_rows():
    """4096x4096 rectangles + noise, Sobel, 5x5 Gaussian window sigma=1, k=0.04: the
    tuned launch, checked on row bands at the top, middle and bottom."""
    img, sx, sy, win, k = synth.workload_harris()
    x = torch.from_numpy(img).cuda()
    ops.tune(ops.problem(_abi.OP_HARRIS, "f32", "f32", 5, 5, 4096, 4096), budget_s=6.0, reps=3)
    y = ops.harris(x, sx, sy, win, k)
    for rows in [(0, 7), (2040, 2050), (4089, 4096)]:
        R64, sc = harris_reference(img, sx, sy, win, k, rows=rows, halo=3)
        check_harris_output(y[rows[0]:rows[1]], R64, sc, f"rows={rows}")
    yp = ops.harris(x, sx, sy, win, k, variant={"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16})
    R64, sc = harris_reference(img, sx, sy, win, k, rows=(100, 104), halo=3)
    check_harris_output(yp[100:104], R64, sc, "plain")


def test_harris_corners_found():
    """Noise-free rectangles: the 16 strongest 3x3 maxima of the GPU response lie within
    2 pixels of the 16 rectangle corners."""
    import scipy.ndimage as ndi
    rects = [(12, 14, 30, 22, 0.9), (70, 10, 40, 35, 0.6), (15, 70, 25, 40, 0.8), (66, 72, 45, 30, 0.7)]
    img = synth.rectangles_noise_free(128, 128, rects)
    R = ops.harris(torch.from_numpy(img).cuda(), synth.sobel_x(), synth.sobel_y(),
                   synth.gaussian_window(5, 1.0)).cpu().numpy()
    peak = (R == ndi.maximum_filter(R, size=3, mode="nearest")) & (R > 0)
    ys, xs = np.nonzero(peak)
    order = np.argsort(-R[ys, xs])[:16]
    found = list(zip(xs[order], ys[order]))
    for (x0, y0, rw, rh, _) in rects:
        for (cx, cy) in [(x0, y0), (x0 + rw - 1, y0), (x0, y0 + rh - 1), (x0 + rw - 1, y0 + rh - 1)]:
            assert min(max(abs(cx - fx), abs(cy - fy)) for fx, fy in found) <= 2


def test_harris_rejects_window_above_7():
    x = torch.rand(16, 16, device="cuda")
    with pytest.raises(ImclError) as ei:
        ops.harris(x, synth.sobel_x(), synth.sobel_y(), np.ones((8, 8), np.float32))
    assert ei.value.status == _abi.ERR_UNSUPPORTED


def test_harris_box2_block_5120_sampled_rows():
    """The paper's Harris benchmark shape: 5120x5120 f32 rectangles + noise with a 2x2
    box block (offsets -1, 0), tuned launch, checked on row bands (top, middle, bottom)."""
    img, sx, sy, _, k = synth.workload_harris(5120, 5120)
    win = synth.box_window(2)
    x = torch.from_numpy(img).cuda()
    ops.tune(ops.problem(_abi.OP_HARRIS, "f32", "f32", 2, 2, 5120, 5120), budget_s=4.0, reps=3)
    y = ops.harris(x, sx, sy, win, k)
    for rows in [(0, 6), (2555, 2565), (5114, 5120)]:
        R64, sc = harris_reference(img, sx, sy, win, k, rows=rows, halo=3)
        check_harris_output(y[rows[0]:rows[1]], R64, sc, f"box2 rows={rows}")
