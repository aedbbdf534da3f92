"""ctypes declarations of the C ABI in ``include/imagecl.h``.

Loading fails loudly (ImportError) when ``libimagecl.so`` has not been built: there is
no fallback implementation behind this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libimagecl.so")

c_int32, c_int64, c_void_p, c_double = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double

# imcl_status
OK, ERR_INVALID, ERR_UNSUPPORTED, ERR_ALIGN, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = range(7)
STATUS_NAMES = ["IMCL_OK", "IMCL_ERR_INVALID", "IMCL_ERR_UNSUPPORTED", "IMCL_ERR_ALIGN",
                "IMCL_ERR_OOM", "IMCL_ERR_CUDA", "IMCL_ERR_TIMEOUT"]
# imcl_dtype
U8, I32, F32, F16, BF16 = range(5)
# imcl_border / imcl_mem / imcl_op
BORDER_CLAMP, BORDER_CONSTANT = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
OP_CONV2D, OP_SEPCONV, OP_HARRIS = 0, 1, 2
# imcl_kind / imcl_load / imcl_filt / imcl_map / imcl_unroll
KIND_PLAIN, KIND_TILED, KIND_TENSOR = 0, 1, 2
LOAD_GLOBAL, LOAD_SMEM, LOAD_TMA = 0, 1, 2
FILT_PARAM, FILT_SMEM = 0, 1
MAP_BLOCKED, MAP_INTERLEAVED, MAP_REGISTER = 0, 1, 2
UNROLL_NONE, UNROLL_FULL, UNROLL_PACKED, UNROLL_F32_EXACT = 0, 1, 2, 3


class Image(ctypes.Structure):
    _fields_ = [("data", c_void_p), ("dtype", c_int32), ("width", c_int32), ("height", c_int32),
                ("reserved", c_int32), ("pitch_bytes", c_int64)]


VARIANT_FIELDS = ("kind", "bx", "by", "px", "py", "load", "filt", "map", "unroll", "persistent")


class Variant(ctypes.Structure):
    _fields_ = [(n, c_int32) for n in VARIANT_FIELDS]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n in VARIANT_FIELDS}

    @classmethod
    def from_dict(cls, d: dict) -> "Variant":
        v = cls()
        for n in VARIANT_FIELDS:
            setattr(v, n, int(d.get(n, UNROLL_FULL if n == "unroll" else 0)))
        return v

    def __repr__(self):
        return f"Variant({self.as_dict()})"


PROBLEM_FIELDS = ("op", "in_dtype", "out_dtype", "kw", "kh", "width", "height", "border", "taps_mem")


class Problem(ctypes.Structure):
    _fields_ = [(n, c_int32) for n in PROBLEM_FIELDS]


class BatchItem(ctypes.Structure):
    _fields_ = [("op", c_int32), ("border", c_int32), ("kw", c_int32), ("kh", c_int32),
                ("border_value", c_double), ("in_", Image), ("out", Image), ("taps", c_void_p),
                ("taps2", c_void_p), ("grad_out", Image), ("grad_in", Image), ("grad_taps", c_void_p),
                ("grad_taps2", c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("images", c_int32), ("tiles", c_int32), ("tile_w", c_int32), ("tile_h", c_int32),
                ("pixels", c_double), ("fwd_ms_at_create", c_double), ("shape_ms", c_double * 4),
                ("has_backward", c_int32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("candidates", c_int32), ("sampled", c_int32), ("confirmed", c_int32), ("valid", c_int32),
                ("model_rmse", c_double), ("seconds", c_double), ("holdout", c_int32), ("holdout_valid", c_int32),
                ("holdout_rmse", c_double)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class ImclError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


P = ctypes.POINTER
# name -> (restype, argtypes)
SIGNATURES = {
    "imagecl_conv2d": (c_int32, [P(Image), P(Image), c_void_p, c_int32, c_int32, c_int32, c_int32,
                                 c_int32, c_double, P(Variant), c_void_p]),
    "imagecl_sepconv": (c_int32, [P(Image), P(Image), c_void_p, c_int32, c_void_p, c_int32, c_int32,
                                  c_int32, c_double, P(Variant), c_void_p, ctypes.c_size_t, c_void_p]),
    "imagecl_sepconv_workspace_size": (ctypes.c_size_t, [P(Problem), P(Variant)]),
    "imagecl_harris": (c_int32, [P(Image), P(Image), c_void_p, c_void_p, c_void_p, c_int32,
                                 ctypes.c_float, c_int32, P(Variant), c_void_p, ctypes.c_size_t,
                                 c_void_p]),
    "imagecl_harris_workspace_size": (ctypes.c_size_t, [P(Problem), P(Variant)]),
    "imagecl_sepconv_noalloc": (c_int32, [P(Image), P(Image), c_void_p, c_int32, c_void_p, c_int32,
                                          c_int32, c_int32, c_double, c_void_p]),
    "imagecl_conv2d_backward": (c_int32, [P(Image), P(Image), c_void_p, c_int32, c_int32, c_int32,
                                          c_int32, c_double, P(Image), c_void_p, c_void_p,
                                          ctypes.c_size_t, c_void_p]),
    "imagecl_conv2d_backward_workspace_size": (ctypes.c_size_t, [c_int32, c_int32, c_int32, c_int32]),
    "imagecl_sepconv_backward": (c_int32, [P(Image), P(Image), c_void_p, c_int32, c_void_p, c_int32,
                                           c_int32, c_int32, c_double, P(Image), c_void_p, c_void_p,
                                           c_void_p, ctypes.c_size_t, c_void_p]),
    "imagecl_sepconv_backward_workspace_size": (ctypes.c_size_t, [c_int32, c_int32, c_int32, c_int32]),
    "imagecl_harris_backward": (c_int32, [P(Image), P(Image), c_void_p, c_void_p, c_void_p, c_int32,
                                          ctypes.c_float, c_int32, P(Image), c_void_p, c_void_p,
                                          c_void_p, c_void_p, ctypes.c_size_t, c_void_p]),
    "imagecl_harris_backward_workspace_size": (ctypes.c_size_t, [c_int32, c_int32, c_int32]),
    "imagecl_batch_create": (c_int32, [P(BatchItem), c_int32, c_double, P(c_void_p)]),
    "imagecl_batch_run": (c_int32, [c_void_p, c_void_p]),
    "imagecl_batch_backward": (c_int32, [c_void_p, c_void_p]),
    "imagecl_batch_info": (c_int32, [c_void_p, P(BatchInfo)]),
    "imagecl_batch_destroy": (None, [c_void_p]),
    "imagecl_variant_count": (c_int32, [P(Problem)]),
    "imagecl_variant_get": (c_int32, [P(Problem), c_int32, P(Variant)]),
    "imagecl_variant_default": (c_int32, [P(Problem), P(Variant)]),
    "imagecl_tune": (c_int32, [P(Problem), c_double, c_int32, P(Variant), P(c_double), P(c_double),
                               c_void_p]),
    "imagecl_tune_model": (c_int32, [P(Problem), c_int32, c_int32, c_int32, ctypes.c_uint64, P(Variant),
                                     P(c_double), P(c_double), P(TuneReport), c_void_p]),
    "imagecl_tune_set": (c_int32, [P(Problem), P(Variant)]),
    "imagecl_tune_clear": (None, []),
    "imagecl_tune_save": (c_int32, [ctypes.c_char_p]),
    "imagecl_tune_load": (c_int32, [ctypes.c_char_p]),
    "imagecl_probe_fp32": (c_int32, [c_int32, P(c_double), c_void_p]),
    "imagecl_probe_imad": (c_int32, [P(c_double), c_void_p]),
    "imagecl_selftest_wait_timeout": (c_int32, [c_int32, c_void_p]),
    "imagecl_last_error": (ctypes.c_char_p, []),
    "imagecl_device_status": (c_int32, [P(c_int32), c_void_p]),
    "imagecl_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded library (built with ``paper_1605_06399_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it first "
                                  "(python -m paper_1605_06399_gb300.build)")
            import torch  # noqa: F401  (loads the CUDA runtime the library links against)
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def check(status: int) -> None:
    if status != OK:
        raise ImclError(status, lib().imagecl_last_error().decode(errors="replace"))
