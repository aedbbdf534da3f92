"""Python entry points over the C ABI: argument marshalling only.

Every function takes CUDA tensors (2D, unit stride along x), passes their device
pointers, sizes and row pitches to ``libimagecl.so`` and launches on the current torch
stream (or ``stream``).  All stencil arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import check, lib

TORCH_TO_DT = {torch.uint8: _abi.U8, torch.int32: _abi.I32, torch.float32: _abi.F32,
               torch.float16: _abi.F16, torch.bfloat16: _abi.BF16}
DT_TO_TORCH = {v: k for k, v in TORCH_TO_DT.items()}
NAME_TO_DT = {"u8": _abi.U8, "i32": _abi.I32, "f32": _abi.F32, "f16": _abi.F16, "bf16": _abi.BF16}
BORDERS = {"clamp": _abi.BORDER_CLAMP, "constant": _abi.BORDER_CONSTANT}


def image(t: torch.Tensor) -> _abi.Image:
    """Describe a 2D CUDA tensor (H, W) with unit x stride as an ``imcl_image``."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("images must be CUDA tensors")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("images must be 2D (H, W) with unit stride along x")
    if t.dtype not in TORCH_TO_DT:
        raise TypeError(f"unsupported pixel type {t.dtype}")
    return _abi.Image(t.data_ptr(), TORCH_TO_DT[t.dtype], t.size(1), t.size(0), 0,
                      t.stride(0) * t.element_size())


def stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _variant(v):
    if v is None:
        return None
    if isinstance(v, _abi.Variant):
        return ctypes.byref(v)
    return ctypes.byref(_abi.Variant.from_dict(v))


class Taps:
    """Filter taps as the C ABI wants them: a pointer, its memory kind and the sides.

    CUDA tensors are passed as device taps; anything else (numpy, CPU tensors, lists)
    becomes a contiguous host array kept alive by this object."""

    def __init__(self, taps, integer: bool, ndim: int = 2):
        want_np = np.int32 if integer else np.float32
        want_t = torch.int32 if integer else torch.float32
        if isinstance(taps, torch.Tensor) and taps.is_cuda:
            t = taps.detach().to(want_t).contiguous()
            self.keep = t
            self.ptr = t.data_ptr()
            self.mem = _abi.MEM_DEVICE
            shape = tuple(t.shape)
        else:
            if isinstance(taps, torch.Tensor):
                taps = taps.detach().cpu().numpy()
            a = np.ascontiguousarray(taps, dtype=want_np)
            self.keep = a
            self.ptr = a.ctypes.data
            self.mem = _abi.MEM_HOST
            shape = a.shape
        if len(shape) != ndim:
            raise ValueError(f"taps must be {ndim}-D, got shape {shape}")
        self.shape = shape
        self.dtype = _abi.I32 if integer else _abi.F32


def _out_like(x: torch.Tensor, out, out_dtype, integer: bool) -> torch.Tensor:
    if out is not None:
        return out
    if integer:
        dt = torch.int32
    elif out_dtype is None:
        dt = torch.float32
    else:
        dt = out_dtype if isinstance(out_dtype, torch.dtype) else DT_TO_TORCH[NAME_TO_DT[out_dtype]]
    return torch.empty(x.shape, dtype=dt, device=x.device)


def conv2d(x: torch.Tensor, taps, border: str = "clamp", border_value: float = 0.0, out=None,
           out_dtype=None, variant=None, stream=None) -> torch.Tensor:
    """Non-separable correlation of ``x`` (H, W) with ``taps`` (kh, kw), centred, no flip.

    u8 / i32 images take integer taps and give i32; f32 / f16 / bf16 images take f32
    taps and give f32 (default) or their own 16-bit type (``out_dtype``)."""
    integer = x.dtype in (torch.uint8, torch.int32)
    tp = Taps(taps, integer)
    y = _out_like(x, out, out_dtype, integer)
    xi, yi = image(x), image(y)
    kh, kw = tp.shape
    check(lib().imagecl_conv2d(ctypes.byref(xi), ctypes.byref(yi), ctypes.c_void_p(tp.ptr), tp.dtype,
                               kw, kh, tp.mem, BORDERS[border], float(border_value),
                               _variant(variant), ctypes.c_void_p(stream_handle(stream))))
    return y


def sepconv(x: torch.Tensor, row_taps, col_taps=None, border: str = "clamp",
            border_value: float = 0.0, out=None, out_dtype=None, variant=None, workspace=None,
            stream=None) -> torch.Tensor:
    """Row pass with ``row_taps`` then column pass with ``col_taps`` (default: the same
    taps), each applying the boundary rule to its own input; t is kept in f32."""
    if x.dtype in (torch.uint8, torch.int32):
        raise TypeError("sepconv takes f32, f16 or bf16 images")
    rt = Taps(row_taps, False, ndim=1)
    ct = Taps(row_taps if col_taps is None else col_taps, False, ndim=1)
    if rt.mem != ct.mem:
        raise ValueError("row and column taps must both be on the host or both on the device")
    y = _out_like(x, out, out_dtype, False)
    xi, yi = image(x), image(y)
    vptr = _variant(variant)
    prob = problem(_abi.OP_SEPCONV, x.dtype, y.dtype, rt.shape[0], ct.shape[0], x.size(1), x.size(0), border,
                   rt.mem)
    need = lib().imagecl_sepconv_workspace_size(ctypes.byref(prob), vptr)
    ws_ptr, ws_bytes = None, 0
    if need:
        if workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    check(lib().imagecl_sepconv(ctypes.byref(xi), ctypes.byref(yi), ctypes.c_void_p(rt.ptr),
                                rt.shape[0], ctypes.c_void_p(ct.ptr), ct.shape[0], rt.mem,
                                BORDERS[border], float(border_value), vptr,
                                ctypes.c_void_p(ws_ptr), ws_bytes,
                                ctypes.c_void_p(stream_handle(stream))))
    return y


def harris(x: torch.Tensor, sobel_x, sobel_y, window, k: float = 0.04, out=None, variant=None,
           workspace=None, stream=None) -> torch.Tensor:
    """Harris response of the f32 image ``x`` with the given 3x3 Sobel taps and odd
    window (clamped boundary on every stage)."""
    if x.dtype != torch.float32:
        raise TypeError("harris takes an f32 image")
    sx, sy = Taps(sobel_x, False), Taps(sobel_y, False)
    win = Taps(window, False)
    if not (sx.mem == sy.mem == win.mem):
        raise ValueError("all Harris taps must be on the host or all on the device")
    if sx.shape != (3, 3) or sy.shape != (3, 3) or win.shape[0] != win.shape[1]:
        raise ValueError("Sobel taps must be 3x3 and the window square")
    y = out if out is not None else torch.empty_like(x)
    xi, yi = image(x), image(y)
    vptr = _variant(variant)
    prob = problem(_abi.OP_HARRIS, torch.float32, torch.float32, win.shape[0], win.shape[0], x.size(1),
                   x.size(0), "clamp", sx.mem)
    need = lib().imagecl_harris_workspace_size(ctypes.byref(prob), vptr)
    ws_ptr, ws_bytes = None, 0
    if need:
        if workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    check(lib().imagecl_harris(ctypes.byref(xi), ctypes.byref(yi), ctypes.c_void_p(sx.ptr),
                               ctypes.c_void_p(sy.ptr), ctypes.c_void_p(win.ptr), win.shape[0],
                               float(k), sx.mem, vptr, ctypes.c_void_p(ws_ptr), ws_bytes,
                               ctypes.c_void_p(stream_handle(stream))))
    return y


def _grad_buffers(x, need_dx):
    dx = torch.empty(x.shape, dtype=torch.float32, device=x.device) if need_dx else None
    return dx, (ctypes.byref(image(dx)) if dx is not None else None)


def _ws(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def _f32_grad(g):
    return g.detach().to(torch.float32).contiguous()


def conv2d_backward(g, x, taps, border="clamp", border_value=0.0, need_dx=True, need_dw=True,
                    stream=None):
    """(dx, dtaps) of ``conv2d(x, taps)`` for the upstream gradient ``g`` (f32 results;
    None for what is not requested)."""
    g = _f32_grad(g)
    tp = Taps(taps, False)
    kh, kw = tp.shape
    dx, dx_ref = _grad_buffers(x, need_dx)
    dw = torch.empty((kh, kw), dtype=torch.float32, device=x.device) if need_dw else None
    ws = _ws(lib().imagecl_conv2d_backward_workspace_size(x.size(1), x.size(0), kw, kh), x.device)
    gi, xi = image(g), image(x)
    check(lib().imagecl_conv2d_backward(ctypes.byref(gi), ctypes.byref(xi), ctypes.c_void_p(tp.ptr), kw, kh,
                                        tp.mem, BORDERS[border], float(border_value), dx_ref,
                                        ctypes.c_void_p(dw.data_ptr() if dw is not None else None),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                        ctypes.c_void_p(stream_handle(stream))))
    return dx, dw


def sepconv_backward(g, x, row_taps, col_taps=None, border="clamp", border_value=0.0, need_dx=True,
                     need_drow=True, need_dcol=True, stream=None):
    """(dx, drow, dcol) of ``sepconv(x, row_taps, col_taps)`` for the upstream ``g``."""
    g = _f32_grad(g)
    rt = Taps(row_taps, False, ndim=1)
    ct = Taps(row_taps if col_taps is None else col_taps, False, ndim=1)
    nr, nc = rt.shape[0], ct.shape[0]
    dx, dx_ref = _grad_buffers(x, need_dx)
    drow = torch.empty(nr, dtype=torch.float32, device=x.device) if need_drow else None
    dcol = torch.empty(nc, dtype=torch.float32, device=x.device) if need_dcol else None
    ws = _ws(lib().imagecl_sepconv_backward_workspace_size(x.size(1), x.size(0), nr, nc), x.device)
    gi, xi = image(g), image(x)
    check(lib().imagecl_sepconv_backward(ctypes.byref(gi), ctypes.byref(xi), ctypes.c_void_p(rt.ptr), nr,
                                         ctypes.c_void_p(ct.ptr), nc, rt.mem, BORDERS[border],
                                         float(border_value), dx_ref,
                                         ctypes.c_void_p(drow.data_ptr() if drow is not None else None),
                                         ctypes.c_void_p(dcol.data_ptr() if dcol is not None else None),
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                         ctypes.c_void_p(stream_handle(stream))))
    return dx, drow, dcol


def harris_backward(g, x, sobel_x, sobel_y, window, k=0.04, need_dx=True, need_taps=True, stream=None):
    """(dI, dsobel_x, dsobel_y, dwindow) of ``harris`` for the upstream gradient ``g``."""
    g = _f32_grad(g)
    sx, sy, win = Taps(sobel_x, False), Taps(sobel_y, False), Taps(window, False)
    wk = win.shape[0]
    dx, dx_ref = _grad_buffers(x, need_dx)
    mk = (lambda shape: torch.empty(shape, dtype=torch.float32, device=x.device) if need_taps else None)
    dsx, dsy, dwin = mk((3, 3)), mk((3, 3)), mk((wk, wk))
    ws = _ws(lib().imagecl_harris_backward_workspace_size(x.size(1), x.size(0), wk), x.device)
    gi, xi = image(g), image(x)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else None)
    check(lib().imagecl_harris_backward(ctypes.byref(gi), ctypes.byref(xi), ctypes.c_void_p(sx.ptr),
                                        ctypes.c_void_p(sy.ptr), ctypes.c_void_p(win.ptr), wk, float(k),
                                        sx.mem, dx_ref, ptr(dsx), ptr(dsy), ptr(dwin),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                        ctypes.c_void_p(stream_handle(stream))))
    return dx, dsx, dsy, dwin


def problem(op: int, in_dtype, out_dtype, kw: int, kh: int, width: int, height: int,
            border: str = "clamp", taps_mem: int = _abi.MEM_HOST) -> _abi.Problem:
    def dt(d):
        if isinstance(d, torch.dtype):
            return TORCH_TO_DT[d]
        return NAME_TO_DT[d] if isinstance(d, str) else int(d)
    return _abi.Problem(op, dt(in_dtype), dt(out_dtype), kw, kh, width, height, BORDERS[border],
                        taps_mem)


def variants(prob: _abi.Problem) -> list[dict]:
    """Every compiled variant applicable to ``prob`` (default block shapes)."""
    n = lib().imagecl_variant_count(ctypes.byref(prob))
    out = []
    for i in range(n):
        v = _abi.Variant()
        check(lib().imagecl_variant_get(ctypes.byref(prob), i, ctypes.byref(v)))
        out.append(v.as_dict())
    return out


def default_variant(prob: _abi.Problem) -> dict:
    v = _abi.Variant()
    check(lib().imagecl_variant_default(ctypes.byref(prob), ctypes.byref(v)))
    return v.as_dict()


def tune_model(prob: _abi.Problem, n_sample: int = 32, n_confirm: int = 8, reps: int = 3, seed: int = 0,
               stream=None) -> dict:
    """Model-guided tuning of ``prob`` (random sample, neural-network cost model, the best
    predicted confirmed by timing); returns the winner, its time, PLAIN's and the report."""
    v = _abi.Variant()
    best_ms, plain_ms = ctypes.c_double(0), ctypes.c_double(0)
    rep = _abi.TuneReport()
    check(lib().imagecl_tune_model(ctypes.byref(prob), int(n_sample), int(n_confirm), int(reps), int(seed),
                                   ctypes.byref(v), ctypes.byref(best_ms), ctypes.byref(plain_ms),
                                   ctypes.byref(rep), ctypes.c_void_p(stream_handle(stream))))
    return {"variant": v.as_dict(), "best_ms": best_ms.value, "plain_ms": plain_ms.value,
            "report": rep.as_dict()}


def tune(prob: _abi.Problem, budget_s: float = 20.0, reps: int = 5, stream=None) -> dict:
    """Run the auto-tuner on ``prob``; returns the winner and its time against PLAIN."""
    v = _abi.Variant()
    best_ms, plain_ms = ctypes.c_double(0), ctypes.c_double(0)
    check(lib().imagecl_tune(ctypes.byref(prob), float(budget_s), int(reps), ctypes.byref(v),
                             ctypes.byref(best_ms), ctypes.byref(plain_ms),
                             ctypes.c_void_p(stream_handle(stream))))
    return {"variant": v.as_dict(), "best_ms": best_ms.value, "plain_ms": plain_ms.value}


def tune_set(prob: _abi.Problem, variant) -> None:
    v = variant if isinstance(variant, _abi.Variant) else _abi.Variant.from_dict(variant)
    check(lib().imagecl_tune_set(ctypes.byref(prob), ctypes.byref(v)))


def tune_clear() -> None:
    lib().imagecl_tune_clear()


def tune_save(path: str) -> None:
    check(lib().imagecl_tune_save(path.encode()))


def tune_load(path: str) -> None:
    check(lib().imagecl_tune_load(path.encode()))


def device_status(stream=None) -> int:
    """Synchronise, then read and clear the device status word (0: no kernel gave up)."""
    code = ctypes.c_int32(0)
    st = lib().imagecl_device_status(ctypes.byref(code), ctypes.c_void_p(stream_handle(stream)))
    if st not in (_abi.OK, _abi.ERR_TIMEOUT):
        check(st)
    return int(code.value)


def probe_fp32(packed: bool = False, stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU in TFLOP/s."""
    v = ctypes.c_double(0)
    check(lib().imagecl_probe_fp32(int(packed), ctypes.byref(v), ctypes.c_void_p(stream_handle(stream))))
    return v.value


def probe_imad(stream=None) -> float:
    """Measured int32 multiply-add throughput of the current GPU in Tops/s (2 per IMAD)."""
    v = ctypes.c_double(0)
    check(lib().imagecl_probe_imad(ctypes.byref(v), ctypes.c_void_p(stream_handle(stream))))
    return v.value


def selftest_wait_timeout(rounds: int = 1000, stream=None) -> None:
    """Launch the bounded-wait self-test (a wait that runs out and records code 1)."""
    check(lib().imagecl_selftest_wait_timeout(int(rounds), ctypes.c_void_p(stream_handle(stream))))


def version() -> str:
    return lib().imagecl_version().decode()


class Batch:
    """A ragged batch plan: one persistent, graph-replayed launch over many images.

    ``items`` is a list of dicts with keys ``op`` ('conv' or 'sep'), ``x`` (CUDA tensor),
    ``taps`` (CUDA tensor: conv (kh, kw), sep row taps), ``col_taps`` (sep, CUDA tensor),
    optional ``out`` / ``out_dtype``, ``border``, ``border_value``, and for the backward
    ``grad_out`` (f32 CUDA tensor).  The plan keeps references to every tensor it uses."""

    def __init__(self, items, tune_budget_s: float = 2.0):
        self.keep = []
        arr = (_abi.BatchItem * len(items))()
        self.outputs = []
        self.grad_in, self.grad_taps, self.grad_taps2 = [], [], []
        for i, it in enumerate(items):
            x = it["x"]
            op = _abi.OP_CONV2D if it["op"] == "conv" else _abi.OP_SEPCONV
            taps = it["taps"].detach().to(torch.float32).contiguous()
            col = it.get("col_taps")
            col = col.detach().to(torch.float32).contiguous() if col is not None else None
            if not taps.is_cuda or (col is not None and not col.is_cuda):
                raise ValueError("batch taps must be CUDA tensors")
            out = it.get("out")
            if out is None:
                od = it.get("out_dtype", x.dtype)
                out = torch.empty(x.shape, dtype=od, device=x.device)
            a = arr[i]
            a.op = op
            a.border = BORDERS[it.get("border", "clamp")]
            if op == _abi.OP_CONV2D:
                a.kh, a.kw = taps.shape
            else:
                a.kw, a.kh = taps.numel(), col.numel()
            a.border_value = float(it.get("border_value", 0.0))
            a.in_ = image(x)
            a.out = image(out)
            a.taps = taps.data_ptr()
            a.taps2 = col.data_ptr() if col is not None else None
            g = it.get("grad_out")
            if g is not None:
                g = g.detach().to(torch.float32).contiguous()
                gi = torch.empty(x.shape, dtype=torch.float32, device=x.device)
                gt = torch.empty(taps.shape, dtype=torch.float32, device=x.device)
                gt2 = torch.empty(col.shape, dtype=torch.float32, device=x.device) if col is not None else None
                a.grad_out = image(g)
                a.grad_in = image(gi)
                a.grad_taps = gt.data_ptr()
                a.grad_taps2 = gt2.data_ptr() if gt2 is not None else None
                self.keep += [g]
            else:
                gi = gt = gt2 = None
            self.grad_in.append(gi)
            self.grad_taps.append(gt)
            self.grad_taps2.append(gt2)
            self.keep += [x, taps, col, out, gi, gt, gt2]
            self.outputs.append(out)
        h = ctypes.c_void_p()
        check(lib().imagecl_batch_create(arr, len(items), float(tune_budget_s), ctypes.byref(h)))
        self.handle = h
        self._items = arr

    def run(self, stream=None):
        check(lib().imagecl_batch_run(self.handle, ctypes.c_void_p(stream_handle(stream))))
        return self.outputs

    def backward(self, stream=None):
        """Run the batch's adjoint: fills ``grad_in``, ``grad_taps`` (and ``grad_taps2``)."""
        check(lib().imagecl_batch_backward(self.handle, ctypes.c_void_p(stream_handle(stream))))
        return self.grad_in, self.grad_taps, self.grad_taps2

    def info(self) -> dict:
        i = _abi.BatchInfo()
        check(lib().imagecl_batch_info(self.handle, ctypes.byref(i)))
        return {"images": i.images, "tiles": i.tiles, "tile": (i.tile_w, i.tile_h), "pixels": i.pixels,
                "fwd_ms_at_create": i.fwd_ms_at_create, "shape_ms": list(i.shape_ms),
                "has_backward": bool(i.has_backward)}

    def close(self):
        if getattr(self, "handle", None):
            lib().imagecl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
