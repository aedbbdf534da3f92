"""Error measures used by the parity tests.

Floating results are compared with the oracle's float64 result y64 on the same
(storage-rounded) inputs.  The error of an output is scaled by the magnitude of the
terms that were summed, s(p) = sum |w| |x| (the forward-error bound of a dot product,
Higham §3.1), so outputs that cancel to near zero are judged fairly:

    e(p) = |y_gpu - y64| / max(s(p), 1e-30)         gate: 1e-5 (f32 storage)

A 16-bit output carries one rounding of its own: f16 (unit roundoff 2^-11) stays within
2e-3 of s; bf16 (unit roundoff 2^-8 = 3.9e-3, above 2e-3) is gated at one bf16 ulp of
y64 plus the f32 arithmetic bound.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

TOL_F32 = 1e-5
TOL_16 = 2e-3


def to_f64(t) -> np.ndarray:
    if isinstance(t, torch.Tensor):
        return t.detach().cpu().to(torch.float64).numpy()
    return np.asarray(t, dtype=np.float64)


def ulp(v: np.ndarray, mant_bits: int) -> np.ndarray:
    """Spacing of a float format with `mant_bits` stored mantissa bits at |v|."""
    a = np.maximum(np.abs(v), np.finfo(np.float64).tiny)
    return np.exp2(np.floor(np.log2(a)) - mant_bits)


def scaled_error(gpu, y64: np.ndarray, s: np.ndarray) -> np.ndarray:
    return np.abs(to_f64(gpu) - y64) / np.maximum(s, 1e-30)


def check_float_output(gpu, y64, s, out_dtype: torch.dtype, what: str = "") -> float:
    """Assert the gate for the output type; return the max scaled error."""
    g = to_f64(gpu)
    e = np.abs(g - y64) / np.maximum(s, 1e-30)
    emax = float(e.max()) if e.size else 0.0
    if out_dtype == torch.float32:
        assert emax <= TOL_F32, f"{what}: max scaled error {emax:.3e} > {TOL_F32}"
    elif out_dtype == torch.float16:
        assert emax <= TOL_16, f"{what}: max scaled error {emax:.3e} > {TOL_16}"
    elif out_dtype == torch.bfloat16:
        bound = ulp(y64, 7) + TOL_F32 * s
        bad = np.abs(g - y64) > bound
        assert not bad.any(), f"{what}: {int(bad.sum())} bf16 outputs beyond 1 ulp + f32 bound"
    else:
        raise ValueError(out_dtype)
    return emax


def band(x, rows, halo):
    """Rows [y0 - halo, y1 + halo) of x (cut at the image) and the band's rows inside it.
    Output rows of the band read only rows of the crop, and the crop meets the image's
    own edge wherever the boundary rule applies, so the oracle on the crop gives the same
    values as on the whole image."""
    h = x.shape[0]
    y0, y1 = rows
    a, b = max(0, y0 - halo), min(h, y1 + halo)
    return x[a:b], (y0 - a, y1 - a)


def conv_reference(x, w, border="clamp", bv=0.0, rows=None, halo=None):
    """(y64, s) for conv2d: the oracle result and the scale sum |w||x|."""
    if rows is not None and halo is not None:
        x, rows = band(x, rows, halo)
    y64 = oracle.conv2d(x, w, border, bv, rows=rows)
    if np.issubdtype(y64.dtype, np.integer):
        return y64, None
    s = oracle.conv2d(np.abs(to_f64(x)), np.abs(to_f64(w)), border, abs(bv), rows=rows)
    return y64, s


def sep_reference(x, row, col, border="clamp", bv=0.0, rows=None, halo=None):
    """(y64, s) for sepconv; s = (|c| x |r|) applied to |x| (|bv| outside), the scale of
    the summed terms of both passes."""
    if rows is not None and halo is not None:
        x, rows = band(x, rows, halo)
    y64 = oracle.sepconv(x, row, col, border, bv, rows=rows)
    s = oracle.sepconv(np.abs(to_f64(x)), np.abs(to_f64(row)), np.abs(to_f64(col)), border, abs(bv),
                       rows=rows)
    return y64, s


TOL_HARRIS = 1e-5


def harris_reference(img, sx, sy, win, k=0.04, rows=None, halo=None):
    """(R64, scale) for Harris.  scale = T^2 with T = |G| (*) (Ax^2 + Ay^2) and
    A = |S| (*) |I|: a bound on |Sxx|, |Syy|, |Sxy| that also covers the rounding of the
    Sobel sums (|Ix| <= Ax), so e = |R - R64| / T^2 is the forward error of R relative
    to the size of its terms."""
    if rows is not None and halo is not None:
        img, rows = band(img, rows, halo)
    R = oracle.harris(img, sx, sy, win, k, rows=rows)
    ai = np.abs(to_f64(img))
    ax = oracle.conv2d(ai, np.abs(to_f64(sx)))
    ay = oracle.conv2d(ai, np.abs(to_f64(sy)))
    aw = np.abs(to_f64(win))
    if aw.shape[0] % 2 == 0:   # even window: offsets -wk/2 .. wk/2-1, the centred odd one padded
        aw = np.pad(aw, ((0, 1), (0, 1)))
    T = oracle.conv2d(ax * ax + ay * ay, aw, rows=rows)
    return R, T * T


def check_harris_output(gpu, R64, scale, what=""):
    e = np.abs(to_f64(gpu) - R64) / np.maximum(scale, 1e-30)
    emax = float(e.max()) if e.size else 0.0
    assert emax <= TOL_HARRIS, f"{what}: max scaled error {emax:.3e} > {TOL_HARRIS}"
    return emax


def harris_backward_scale(img, sx, sy, win, gR, k=0.04):
    """Element-wise scales (sdI, dsx, dsy, dwin) for the Harris adjoint: the adjoint
    evaluated on absolute values, every product and sum of the chain rule taken with the
    magnitudes of its terms.  The forward planes are Ax = |Sx| (*) |I| (>= |Ix|, and the
    same for y), their products, and |G| (*) those; the response derivatives become
    |gR| (Syy + 2k tr), |gR| (Sxx + 2k tr) and 2 |gR| Sxy; each adjoint step then runs
    with |taps| on non-negative planes.  The computed gradient's rounding error is
    bounded by a modest multiple of the unit roundoff times this scale (the first-order
    forward-error bound of the chain), which is what the 1e-4 gate measures against."""
    ai = np.abs(to_f64(img))
    asx, asy, aw = np.abs(to_f64(sx)), np.abs(to_f64(sy)), np.abs(to_f64(win))
    wk = aw.shape[0]
    if wk % 2 == 0:   # even window: offsets -wk/2 .. wk/2-1, the centred odd one padded
        aw = np.pad(aw, ((0, 1), (0, 1)))
    ag = np.abs(to_f64(gR))
    ax = oracle.conv2d(ai, asx)
    ay = oracle.conv2d(ai, asy)
    p = {"xx": ax * ax, "yy": ay * ay, "xy": ax * ay}
    s = {c: oracle.conv2d(p[c], aw) for c in p}
    tr = s["xx"] + s["yy"]
    gs = {"xx": ag * (s["yy"] + 2 * k * tr), "yy": ag * (s["xx"] + 2 * k * tr), "xy": 2 * ag * s["xy"]}
    gp, dwin = {}, np.zeros_like(aw)
    for c in p:
        gp[c], dw_c = oracle.conv2d_backward(p[c], aw, gs[c])
        dwin += dw_c
    gix = 2 * ax * gp["xx"] + ay * gp["xy"]
    giy = 2 * ay * gp["yy"] + ax * gp["xy"]
    di_x, dsx = oracle.conv2d_backward(ai, asx, gix)
    di_y, dsy = oracle.conv2d_backward(ai, asy, giy)
    return di_x + di_y, dsx, dsy, dwin[:wk, :wk]


TOL_GRAD = 1e-4


def check_grad(gpu, ref, scale, what="", tol=TOL_GRAD):
    """Element-wise scaled gradient error, |g - g64| / scale, gated at `tol`; returns the max."""
    e = np.abs(to_f64(gpu) - ref) / np.maximum(scale, 1e-30)
    emax = float(e.max()) if e.size else 0.0
    assert emax <= tol, f"{what}: scaled error {emax:.3e} > {tol}"
    return emax
