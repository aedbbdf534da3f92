"""Pins for the CPU oracle: facts fixed by the definitions, not by the oracle itself.

Each ``check_*`` takes an oracle object (``oracle.Oracle``) and raises AssertionError
when the oracle disagrees with the fact.  ``tests/test_oracle_pins.py`` runs them on the
real oracle; ``tests/test_oracle_mutations.py`` runs them on deliberately broken copies
of the oracle source and expects them to fail.

What pins what:
  * hand-derived fixtures (tests/golden): Listing 1's box filter, tap orientation,
    both boundary rules (§5, Fig. 3), and a Harris value on a step edge;
  * special cases: a delta filter is the identity, a normalised filter keeps a
    constant image constant, linearity, translation of the interior;
  * library routines doing the same definition another way: scipy.ndimage.correlate
    (mode 'nearest' is the clamped rule, 'constant' the constant rule), numpy edge
    padding plus shifted sums, torch conv2d on a replicate-padded input;
  * brute force on 4x4 inputs;
  * separable = 2D with the outer-product filter (clamped rule);
  * Harris: R = 0 on a constant image, R <= 0 on a straight edge, transpose symmetry,
    degree-4 homogeneity, corners of rectangles found at their positions; even windows
    against scipy, a delta window's closed form and the zero-padded odd window;
  * adjoints: <A x, g> = <x, A^T g>, linearity in the taps, torch autograd on the
    library formulation, Euler's identity for the homogeneous Harris response and
    central finite differences.
"""
from __future__ import annotations

import numpy as np
import scipy.ndimage as ndi
import torch
import torch.nn.functional as F

import golden_io
from paper_1605_06399_gb300 import synth

CONV_GOLDEN = ["listing1_box_center.txt", "listing1_box_corner.txt", "box_corner_4x4.txt",
               "correlation_orientation.txt", "box_constant_border.txt"]
SHAPES = [(1, 1), (1, 9), (9, 1), (2, 3), (7, 13), (13, 7), (16, 16), (33, 20)]


def _rel(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300)) if a.size else 0.0


def _padded_sum(x, w, border, bv):
    """Correlation as extension-by-padding plus a sum of shifted views."""
    kh, kw = w.shape
    ry, rx = (kh - 1) // 2, (kw - 1) // 2
    if border == "clamp":
        xp = np.pad(x, ((ry, ry), (rx, rx)), mode="edge")
    else:
        xp = np.pad(x, ((ry, ry), (rx, rx)), mode="constant", constant_values=bv)
    h, wd = x.shape
    out = np.zeros((h, wd), dtype=np.result_type(xp, w, np.float64))
    for j in range(kh):
        for i in range(kw):
            out += w[j, i] * xp[j:j + h, i:i + wd]
    return out


def _scipy_corr(x, w, border, bv=0.0):
    mode = "nearest" if border == "clamp" else "constant"
    return ndi.correlate(np.asarray(x, np.float64), np.asarray(w, np.float64), mode=mode,
                         cval=bv)


def _torch_corr(x, w):
    """Clamped correlation via torch: replicate padding then a valid conv2d (torch's
    conv2d is itself a correlation)."""
    kh, kw = w.shape
    ry, rx = (kh - 1) // 2, (kw - 1) // 2
    xt = torch.as_tensor(np.asarray(x, np.float64))[None, None]
    wt = torch.as_tensor(np.asarray(w, np.float64))[None, None]
    xp = F.pad(xt, (rx, rx, ry, ry), mode="replicate")
    return F.conv2d(xp, wt)[0, 0].numpy()


# ------------------------------------------------------------------ conv2d forward

def check_golden_conv(ora):
    for name in CONV_GOLDEN:
        g = golden_io.read(name)
        out = ora.conv2d(g["image"], g["filter"], g["border"], g["border_value"]) / g["divide"]
        assert np.array_equal(out, g["expected"]), name
        oi = ora.conv2d(g["image"].astype(np.int32), g["filter"].astype(np.int32),
                        g["border"], int(g["border_value"]))
        assert np.array_equal(oi, (g["expected"] * g["divide"]).astype(np.int32)), name


def check_delta_identity(ora):
    g = np.random.default_rng(11)
    for (h, w) in SHAPES:
        for (kh, kw) in [(1, 1), (3, 3), (5, 5), (15, 15), (3, 7), (9, 1)]:
            d = np.zeros((kh, kw))
            d[(kh - 1) // 2, (kw - 1) // 2] = 1.0
            x = g.random((h, w))
            assert np.array_equal(ora.conv2d(x, d, "clamp"), x)
            assert np.array_equal(ora.conv2d(x, d, "constant", 3.5), x)
            xi = g.integers(0, 256, (h, w)).astype(np.uint8)
            assert np.array_equal(ora.conv2d(xi, d.astype(np.int32)), xi.astype(np.int32))


def check_constant_image(ora):
    for k in (3, 5, 11, 15):
        c = 0.7310585786300049
        x = np.full((9, 12), c)
        box = np.full((k, k), 1.0 / (k * k))
        assert _rel(ora.conv2d(x, box), np.full_like(x, c)) < 1e-14
        t = synth.gaussian_taps((k - 1) // 2).astype(np.float64)
        gw = np.outer(t, t)
        assert _rel(ora.conv2d(x, gw), np.full_like(x, c * gw.sum())) < 1e-14
    xi = np.full((7, 5), 201, dtype=np.uint8)
    assert np.array_equal(ora.conv2d(xi, np.ones((3, 3), np.int32)), np.full((7, 5), 9 * 201))


def check_linearity(ora):
    g = np.random.default_rng(12)
    x, y = g.random((17, 23)), g.random((17, 23))
    w = g.standard_normal((5, 5))
    lhs = ora.conv2d(2.5 * x - 0.75 * y, w)
    rhs = 2.5 * ora.conv2d(x, w) - 0.75 * ora.conv2d(y, w)
    assert _rel(lhs, rhs) < 1e-13
    xi = g.integers(0, 100, (11, 9)).astype(np.int32)
    yi = g.integers(0, 100, (11, 9)).astype(np.int32)
    wi = g.integers(-4, 5, (3, 3)).astype(np.int32)
    assert np.array_equal(ora.conv2d(3 * xi - 2 * yi, wi),
                          3 * ora.conv2d(xi, wi) - 2 * ora.conv2d(yi, wi))


def check_brute_force_4x4(ora):
    g = np.random.default_rng(13)
    for _ in range(40):
        x = g.integers(-9, 10, (4, 4)).astype(np.float64)
        w = g.integers(-5, 6, (3, 3)).astype(np.float64)
        # enumerate every tap of every pixel from the clamped index sets
        exp = np.zeros((4, 4))
        for py in range(4):
            for px in range(4):
                for j in range(3):
                    for i in range(3):
                        qy = min(max(py + j - 1, 0), 3)
                        qx = min(max(px + i - 1, 0), 3)
                        exp[py, px] += w[j, i] * x[qy, qx]
        assert np.array_equal(ora.conv2d(x, w), exp)
        assert np.array_equal(ora.conv2d(x.astype(np.int32), w.astype(np.int32)),
                              exp.astype(np.int32))


def check_library_conv(ora):
    g = np.random.default_rng(14)
    for (h, w) in SHAPES:
        for k in (1, 3, 5, 11):
            x = g.random((h, w))
            f = g.standard_normal((k, k))
            ref = _scipy_corr(x, f, "clamp")
            out = ora.conv2d(x, f)
            assert _rel(out, ref, np.abs(f).sum()) < 1e-13, (h, w, k)
            assert _rel(out, _torch_corr(x, f), np.abs(f).sum()) < 1e-13
            assert _rel(out, _padded_sum(x, f, "clamp", 0.0), np.abs(f).sum()) < 1e-13
            outc = ora.conv2d(x, f, "constant", -0.5)
            assert _rel(outc, _scipy_corr(x, f, "constant", -0.5), np.abs(f).sum()) < 1e-13
    fr = g.standard_normal((3, 7))
    x = g.random((12, 10))
    assert _rel(ora.conv2d(x, fr), _padded_sum(x, fr, "clamp", 0.0), 10) < 1e-13


def check_translation(ora):
    g = np.random.default_rng(15)
    x = g.random((40, 40))
    w = g.standard_normal((5, 5))
    xs = np.roll(x, (3, -2), axis=(0, 1))
    a = ora.conv2d(x, w)
    b = ora.conv2d(xs, w)
    # away from the border and the roll seam, the output moves with the input
    assert _rel(np.roll(a, (3, -2), axis=(0, 1))[8:-8, 8:-8], b[8:-8, 8:-8]) < 1e-14


def check_int_wraparound(ora):
    x = np.full((3, 3), 1 << 20, dtype=np.int32)
    w = np.full((3, 3), 1 << 11, dtype=np.int32)
    exact = 9 * (1 << 31)                      # 9 * 2^20 * 2^11, beyond int32
    wrapped = ((exact + (1 << 31)) % (1 << 32)) - (1 << 31)
    assert np.all(ora.conv2d(x, w) == wrapped)


def check_row_range(ora):
    g = np.random.default_rng(16)
    x = g.random((30, 17))
    w = g.standard_normal((7, 7))
    full = ora.conv2d(x, w)
    assert np.array_equal(ora.conv2d(x, w, rows=(5, 12)), full[5:12])
    assert ora.conv2d(x, w, rows=(4, 4)).shape == (0, 17)
    r, c = g.standard_normal(5), g.standard_normal(9)
    sfull = ora.sepconv(x, r, c)
    assert np.array_equal(ora.sepconv(x, r, c, rows=(0, 3)), sfull[0:3])
    assert np.array_equal(ora.sepconv(x, r, c, rows=(26, 30)), sfull[26:30])


# ------------------------------------------------------------------ sepconv forward

def check_sep_outer_product(ora):
    g = np.random.default_rng(21)
    for (h, w) in SHAPES:
        for (nr, nc) in [(3, 3), (5, 9), (33, 7)]:
            x = g.random((h, w))
            r, c = g.standard_normal(nr), g.standard_normal(nc)
            scale = np.abs(r).sum() * np.abs(c).sum()
            assert _rel(ora.sepconv(x, r, c), ora.conv2d(x, np.outer(c, r)), scale) < 1e-13


def check_sep_library(ora):
    g = np.random.default_rng(22)
    for (h, w) in SHAPES:
        x = g.random((h, w))
        r, c = g.standard_normal(5), g.standard_normal(7)
        scale = np.abs(r).sum() * np.abs(c).sum()
        ref = ndi.correlate1d(ndi.correlate1d(x, r, axis=1, mode="nearest"), c, axis=0,
                              mode="nearest")
        assert _rel(ora.sepconv(x, r, c), ref, scale) < 1e-13
        refc = ndi.correlate1d(ndi.correlate1d(x, r, axis=1, mode="constant", cval=0.25), c,
                               axis=0, mode="constant", cval=0.25)
        assert _rel(ora.sepconv(x, r, c, "constant", 0.25), refc, scale) < 1e-13


def check_sep_constant_and_mirror(ora):
    for rad in (1, 4, 16):
        t = synth.gaussian_taps(rad).astype(np.float64)
        x = np.full((8, 21), 0.3)
        assert _rel(ora.sepconv(x, t, t), np.full_like(x, 0.3 * t.sum() ** 2)) < 1e-14
    g = np.random.default_rng(23)
    x = g.random((19, 26))
    t = synth.gaussian_taps(5).astype(np.float64)
    a = ora.sepconv(x, t, t)
    assert _rel(ora.sepconv(x[:, ::-1], t, t), a[:, ::-1]) < 1e-14
    assert _rel(ora.sepconv(x[::-1, :], t, t), a[::-1, :]) < 1e-14


def check_sep_constant_border_differs(ora):
    # Under the constant rule each stage pads its own input, so the separable result is
    # not the 2D result with the outer product unless the pad value vanishes.
    g = np.random.default_rng(24)
    x = g.random((10, 10))
    r, c = np.array([0.5, 1.0, 0.25]), np.array([1.0, 0.5, 2.0])
    a = ora.sepconv(x, r, c, "constant", 1.0)
    b = ora.conv2d(x, np.outer(c, r), "constant", 1.0)
    assert np.abs(a - b).max() > 1e-3
    a0 = ora.sepconv(x, r, c, "constant", 0.0)
    b0 = ora.conv2d(x, np.outer(c, r), "constant", 0.0)
    assert _rel(a0, b0, 5.0) < 1e-14


# ------------------------------------------------------------------ Harris forward

SX, SY = synth.sobel_x().astype(np.float64), synth.sobel_y().astype(np.float64)
WIN5 = synth.gaussian_window(5, 1.0).astype(np.float64)


def _harris_library(img, sx, sy, win, k):
    ix = ndi.correlate(img, sx, mode="nearest")
    iy = ndi.correlate(img, sy, mode="nearest")
    sxx = ndi.correlate(ix * ix, win, mode="nearest")
    syy = ndi.correlate(iy * iy, win, mode="nearest")
    sxy = ndi.correlate(ix * iy, win, mode="nearest")
    return sxx * syy - sxy * sxy - k * (sxx + syy) ** 2, ix, iy


def check_golden_harris(ora):
    g = golden_io.read("harris_vertical_step.txt")
    R = ora.harris(g["image"], SX, SY, g["window"], g["k"])
    assert _rel(R, g["expected"]) < 1e-14


def check_harris_library(ora):
    g = np.random.default_rng(31)
    for (h, w) in [(1, 1), (2, 9), (9, 2), (17, 23), (40, 31)]:
        img = g.random((h, w))
        win = g.random((5, 5))
        ref, ix, _ = _harris_library(img, SX, SY, win, 0.04)
        R, inter = ora.harris(img, SX, SY, win, 0.04, intermediates=True)
        scale = max(np.abs(ref).max(), 1.0)
        assert _rel(R, ref, scale) < 1e-12
        assert _rel(inter["Ix"], ndi.sobel(img, axis=1, mode="nearest"), 8) < 1e-14
        assert _rel(inter["Iy"], ndi.sobel(img, axis=0, mode="nearest"), 8) < 1e-14
        assert _rel(R[2:5], ora.harris(img, SX, SY, win, 0.04, rows=(2, 5)), scale) == 0.0 \
            if h >= 5 else True


def check_harris_invariants(ora):
    g = np.random.default_rng(32)
    assert np.all(ora.harris(np.full((12, 9), 0.77), SX, SY, WIN5) == 0.0)
    for _ in range(3):
        step = np.where(np.arange(20)[None, :] >= g.integers(2, 18), g.random(), g.random())
        img = np.repeat(step, 14, axis=0)                      # vertical edge
        assert np.all(ora.harris(img, SX, SY, WIN5) <= 0.0)
        assert np.all(ora.harris(img.T.copy(), SX, SY, WIN5) <= 0.0)   # horizontal edge
    img = g.random((21, 16))
    a = ora.harris(img, SX, SY, WIN5)
    assert _rel(ora.harris(img.T.copy(), SX, SY, WIN5), a.T) < 1e-13
    assert np.array_equal(ora.harris(2.0 * img, SX, SY, WIN5), 16.0 * a)
    assert _rel(ora.harris(0.37 * img, SX, SY, WIN5), 0.37 ** 4 * a) < 1e-13


def check_harris_corners(ora):
    rects = [(12, 14, 30, 22, 0.9), (70, 10, 40, 35, 0.6), (15, 70, 25, 40, 0.8),
             (66, 72, 45, 30, 0.7)]
    img = synth.rectangles_noise_free(128, 128, rects).astype(np.float64)
    R = ora.harris(img, SX, SY, WIN5)
    corners = []
    for (x0, y0, rw, rh, _) in rects:
        corners += [(x0, y0), (x0 + rw - 1, y0), (x0, y0 + rh - 1), (x0 + rw - 1, y0 + rh - 1)]
    peak = (R == ndi.maximum_filter(R, size=3, mode="nearest")) & (R > 0)
    ys, xs = np.nonzero(peak)
    order = np.argsort(-R[ys, xs])[:16]
    found = list(zip(xs[order], ys[order]))
    assert len(found) == 16
    for (cx, cy) in corners:
        d = min(max(abs(cx - fx), abs(cy - fy)) for fx, fy in found)
        assert d <= 2, (cx, cy, d)


def _pad_window(win):
    """An even wk x wk window as the (wk+1) x (wk+1) centred window with the same offsets:
    tap (j, i) reads offset (i - wk/2, j - wk/2) in both, so a zero last row and column."""
    wk = win.shape[0]
    out = np.zeros((wk + 1, wk + 1))
    out[:wk, :wk] = win
    return out


def check_harris_even_window(ora):
    """Even windows (the 2x2 block of the Harris benchmark, §6) anchored at offsets
    -wk/2 .. wk/2 - 1: scipy.ndimage.correlate centres an even filter at index size // 2,
    the same offsets; a delta window gives the closed form -k (Ix^2 + Iy^2)^2 at the
    delta's offset; and the window equals its zero-padded odd form exactly, forward and
    backward."""
    g = np.random.default_rng(33)
    k = 0.04
    for (h, w) in [(1, 1), (2, 3), (9, 7), (16, 21)]:
        img = g.random((h, w))
        for wk in (2, 4, 6):
            win = g.random((wk, wk))
            ref, _, _ = _harris_library(img, SX, SY, win, k)
            R = ora.harris(img, SX, SY, win, k)
            assert _rel(R, ref, max(np.abs(ref).max(), 1.0)) < 1e-12
            assert np.array_equal(R, ora.harris(img, SX, SY, _pad_window(win), k))
        ix = ndi.correlate(img, SX, mode="nearest")
        iy = ndi.correlate(img, SY, mode="nearest")
        m = ix * ix + iy * iy
        closed = -k * m * m
        scale = max(np.abs(closed).max(), 1e-300)
        for (j, i) in ((1, 1), (0, 0), (0, 1), (1, 0)):   # offsets (i - 1, j - 1)
            delta = np.zeros((2, 2))
            delta[j, i] = 1.0
            R = ora.harris(img, SX, SY, delta, k)
            ys = np.clip(np.arange(h) + j - 1, 0, h - 1)
            xs = np.clip(np.arange(w) + i - 1, 0, w - 1)
            assert _rel(R, closed[np.ix_(ys, xs)], scale) < 1e-12, (j, i)
    img = g.random((8, 9))
    gR = g.standard_normal((8, 9))
    win = g.random((2, 2))
    dI, dsx, dsy, dwin = ora.harris_backward(img, SX, SY, win, gR, k)
    pI, psx, psy, pwin = ora.harris_backward(img, SX, SY, _pad_window(win), gR, k)
    assert np.array_equal(dI, pI) and np.array_equal(dsx, psx) and np.array_equal(dsy, psy)
    assert np.array_equal(dwin, pwin[:2, :2])
    L = lambda a: np.sum(gR * ora.harris(img, SX, SY, a, k))
    for idx in [(0, 0), (1, 1), (0, 1)]:
        fd = _fd(L, win, idx)
        assert abs(fd - dwin[idx]) < 1e-6 * (abs(dwin[idx]) + abs(fd) + 1e-3)


# ------------------------------------------------------------------ adjoints

def check_conv_adjoint(ora):
    g = np.random.default_rng(41)
    for (h, w) in [(1, 1), (3, 2), (9, 14), (16, 11)]:
        for k in (1, 3, 5, 7):
            x, gr = g.standard_normal((h, w)), g.standard_normal((h, w))
            f = g.standard_normal((k, k))
            for border, bv in (("clamp", 0.0), ("constant", 0.0), ("constant", 1.5)):
                ax = ora.conv2d(x, f, border, bv) - ora.conv2d(np.zeros_like(x), f, border, bv)
                dx, dw = ora.conv2d_backward(x, f, gr, border, bv)
                scale = np.abs(ax).sum() * np.abs(gr).max() + 1.0
                assert abs(np.sum(ax * gr) - np.sum(x * dx)) < 1e-12 * scale
                f2 = g.standard_normal((k, k))
                y2 = ora.conv2d(x, f2, border, bv)
                assert abs(np.sum(y2 * gr) - np.sum(dw * f2)) < 1e-12 * (np.abs(y2).sum() + 1)


def check_conv_backward_autograd(ora):
    g = np.random.default_rng(42)
    for (h, w, k) in [(6, 9, 3), (12, 7, 5), (3, 3, 7)]:
        x = torch.tensor(g.standard_normal((h, w)), requires_grad=True)
        f = torch.tensor(g.standard_normal((k, k)), requires_grad=True)
        gr = g.standard_normal((h, w))
        r = (k - 1) // 2
        y = F.conv2d(F.pad(x[None, None], (r, r, r, r), mode="replicate"), f[None, None])
        (y[0, 0] * torch.as_tensor(gr)).sum().backward()
        dx, dw = ora.conv2d_backward(x.detach().numpy(), f.detach().numpy(), gr)
        assert _rel(dx, x.grad.numpy()) < 1e-12
        assert _rel(dw, f.grad.numpy()) < 1e-12


def check_sep_adjoint(ora):
    g = np.random.default_rng(43)
    for (h, w) in [(1, 1), (5, 3), (12, 17)]:
        for (nr, nc) in [(3, 3), (5, 9), (1, 7)]:
            x, gr = g.standard_normal((h, w)), g.standard_normal((h, w))
            r, c = g.standard_normal(nr), g.standard_normal(nc)
            for border, bv in (("clamp", 0.0), ("constant", 0.0)):
                y = ora.sepconv(x, r, c, border, bv)
                dx, drow, dcol = ora.sepconv_backward(x, r, c, gr, border, bv)
                ip = np.sum(y * gr)
                tol = 1e-12 * (np.abs(y).sum() * np.abs(gr).max() + 1)
                assert abs(ip - np.sum(x * dx)) < tol
                assert abs(ip - np.sum(drow * r)) < tol
                assert abs(ip - np.sum(dcol * c)) < tol


def _fd(f, x, idx, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp[idx] += h
    xm[idx] -= h
    return (f(xp) - f(xm)) / (2 * h)


def check_harris_backward(ora):
    g = np.random.default_rng(44)
    for (h, w) in [(6, 7), (11, 9)]:
        img = g.random((h, w))
        sx = SX + 0.1 * g.standard_normal((3, 3))
        sy = SY + 0.1 * g.standard_normal((3, 3))
        win = WIN5 + 0.01 * g.random((5, 5))
        gR = g.standard_normal((h, w))
        k = 0.04
        R = ora.harris(img, sx, sy, win, k)
        dI, dsx, dsy, dwin = ora.harris_backward(img, sx, sy, win, gR, k)
        ip = np.sum(gR * R)
        # Euler: R is homogeneous of degree 4 in I, 2 in the window, 4 in (Sx, Sy)
        assert abs(np.sum(dI * img) - 4 * ip) < 1e-10 * (abs(ip) + 1)
        assert abs(np.sum(dwin * win) - 2 * ip) < 1e-10 * (abs(ip) + 1)
        assert abs(np.sum(dsx * sx) + np.sum(dsy * sy) - 4 * ip) < 1e-10 * (abs(ip) + 1)
        # central finite differences
        L = lambda im: np.sum(gR * ora.harris(im, sx, sy, win, k))
        for idx in [(0, 0), (h - 1, w - 1), (h // 2, 1), (2, w // 2), (h - 1, 0)]:
            fd = _fd(L, img, idx)
            assert abs(fd - dI[idx]) < 1e-6 * (abs(dI[idx]) + abs(fd) + 1e-3)
        for name, arr, grad in (("sx", sx, dsx), ("sy", sy, dsy), ("win", win, dwin)):
            for idx in [(0, 0), (1, 2), (2, 1)]:
                def Lw(a, name=name):
                    kw = dict(sx=sx, sy=sy, win=win)
                    kw[name] = a
                    return np.sum(gR * ora.harris(img, kw["sx"], kw["sy"], kw["win"], k))
                fd = _fd(Lw, arr, idx)
                assert abs(fd - grad[idx]) < 1e-6 * (abs(grad[idx]) + abs(fd) + 1e-3), name


def check_conv_sep_fd(ora):
    g = np.random.default_rng(45)
    x, gr = g.standard_normal((7, 8)), g.standard_normal((7, 8))
    f = g.standard_normal((5, 5))
    dx, dw = ora.conv2d_backward(x, f, gr)
    L = lambda a: np.sum(gr * ora.conv2d(a, f))
    for idx in [(0, 0), (6, 7), (3, 4), (0, 5)]:
        assert abs(_fd(L, x, idx) - dx[idx]) < 1e-7 * (abs(dx[idx]) + 1)
    r, c = g.standard_normal(5), g.standard_normal(3)
    dx, drow, dcol = ora.sepconv_backward(x, r, c, gr)
    L = lambda a: np.sum(gr * ora.sepconv(a, r, c))
    for idx in [(0, 0), (6, 7), (3, 4)]:
        assert abs(_fd(L, x, idx) - dx[idx]) < 1e-7 * (abs(dx[idx]) + 1)


ALL_CHECKS = [check_golden_conv, check_delta_identity, check_constant_image, check_linearity,
              check_brute_force_4x4, check_library_conv, check_translation,
              check_int_wraparound, check_row_range, check_sep_outer_product,
              check_sep_library, check_sep_constant_and_mirror,
              check_sep_constant_border_differs, check_golden_harris, check_harris_library,
              check_harris_invariants, check_harris_corners, check_harris_even_window,
              check_conv_adjoint,
              check_conv_backward_autograd, check_sep_adjoint, check_harris_backward,
              check_conv_sep_fd]
