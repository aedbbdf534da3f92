"""CPU oracle for the stencil operators -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``imagecl_oracle.c`` (plain loops, double / int64
accumulation, each function citing the paper passage it writes out); this module
only builds it with gcc, converts arrays to float64 / int64 and calls it.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against facts the definitions fix (identities, library routines, brute force,
hand-derived fixtures, adjoint identities and finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "imagecl_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

BORDER = {"clamp": 0, "constant": 1}

def build(force: bool = False, src: str = _SRC, out: str = _SO) -> str:
    """Compile the oracle with gcc (OpenMP if available) into ``out``."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=os.path.dirname(out))
    os.close(fd)
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", src, "-o", tmp]
    try:
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    INT = ctypes.c_int
    D = ctypes.c_double
    lib.ora_num_threads.restype = INT
    lib.ora_conv2d_f64.argtypes = [P, I64, I64, P, INT, INT, INT, D, I64, I64, P]
    lib.ora_conv2d_i64.argtypes = [P, I64, I64, P, INT, INT, INT, I64, I64, I64, P]
    lib.ora_sepconv_f64.argtypes = [P, I64, I64, P, INT, P, INT, INT, D, I64, I64, P]
    lib.ora_harris_f64.argtypes = [P, I64, I64, P, P, P, INT, D, I64, I64, P, P]
    lib.ora_conv2d_bwd_f64.argtypes = [P, I64, I64, P, INT, INT, INT, D, P, P, P]
    lib.ora_sepconv_bwd_f64.argtypes = [P, I64, I64, P, INT, P, INT, INT, D, P, P, P, P]
    lib.ora_harris_bwd_f64.argtypes = [P, I64, I64, P, P, P, INT, D, P, P, P, P, P]
    for f in ("ora_conv2d_f64", "ora_conv2d_i64", "ora_sepconv_f64", "ora_harris_f64",
              "ora_conv2d_bwd_f64", "ora_sepconv_bwd_f64", "ora_harris_bwd_f64"):
        getattr(lib, f).restype = INT
    return lib


def _f64(a) -> np.ndarray:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().to(torch.float64).numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a) -> np.ndarray:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().to(torch.int64).numpy()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(a, dtype=np.int64)


def _is_int(a) -> bool:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return not (a.is_floating_point() or a.is_complex())
    except ImportError:  # pragma: no cover
        pass
    return np.issubdtype(np.asarray(a).dtype, np.integer)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _rows(rows, h):
    y0, y1 = (0, h) if rows is None else rows
    if not (0 <= y0 <= y1 <= h):
        raise ValueError(f"row range {rows} outside [0, {h}]")
    return int(y0), int(y1)


HARRIS_PLANES = ("Ix", "Iy", "Pxx", "Pyy", "Pxy", "Sxx", "Syy", "Sxy")


class Oracle:
    """The oracle's entry points bound to one compiled copy of ``imagecl_oracle.c``."""

    def __init__(self, path: str):
        self.path = path
        self.lib = _bind(path)

    def num_threads(self) -> int:
        """Threads the parallel loops use (OMP_NUM_THREADS, else all cores)."""
        return int(self.lib.ora_num_threads())

    def conv2d(self, x, w, border: str = "clamp", border_value: float = 0.0, rows=None) -> np.ndarray:
        """Correlation of image ``x`` (H, W) with taps ``w`` (kh, kw), centred, no flip.

        Integer image and integer taps -> exact int64 sum wrapped to int32.  Otherwise the
        sum is taken in float64 over the float64 values of the inputs as given (so an f32,
        f16 or bf16 input is used exactly as stored).  ``rows=(y0, y1)`` returns those
        output rows only."""
        lib = self.lib
        h, wd = np.shape(x)
        kh, kw = np.shape(w)
        y0, y1 = _rows(rows, h)
        if _is_int(x) and _is_int(w):
            xi, wi = _i64(x), _i64(w)
            out = np.empty((y1 - y0, wd), dtype=np.int32)
            rc = lib.ora_conv2d_i64(_ptr(xi), wd, h, _ptr(wi), kw, kh, BORDER[border],
                                    int(border_value), y0, y1, _ptr(out))
        else:
            xf, wf = _f64(x), _f64(w)
            out = np.empty((y1 - y0, wd), dtype=np.float64)
            rc = lib.ora_conv2d_f64(_ptr(xf), wd, h, _ptr(wf), kw, kh, BORDER[border],
                                    float(border_value), y0, y1, _ptr(out))
        if rc != 0:
            raise ValueError(f"oracle conv2d rejected its arguments (code {rc})")
        return out


    def sepconv(self, x, row, col, border: str = "clamp", border_value: float = 0.0,
                rows=None) -> np.ndarray:
        """Row pass with ``row`` taps, then column pass with ``col`` taps (float64)."""
        lib = self.lib
        h, wd = np.shape(x)
        y0, y1 = _rows(rows, h)
        xf, rf, cf = _f64(x), _f64(row).ravel(), _f64(col).ravel()
        out = np.empty((y1 - y0, wd), dtype=np.float64)
        rc = lib.ora_sepconv_f64(_ptr(xf), wd, h, _ptr(rf), rf.size, _ptr(cf), cf.size,
                                 BORDER[border], float(border_value), y0, y1, _ptr(out))
        if rc != 0:
            raise ValueError(f"oracle sepconv rejected its arguments (code {rc})")
        return out




    def harris(self, img, sx, sy, win, k: float = 0.04, rows=None, intermediates: bool = False):
        """Harris response R (float64), clamped boundary on every stage.

        With ``intermediates=True`` also returns a dict of the 8 intermediate planes."""
        lib = self.lib
        h, wd = np.shape(img)
        y0, y1 = _rows(rows, h)
        xf, sxf, syf, gf = _f64(img), _f64(sx), _f64(sy), _f64(win)
        wk = gf.shape[0]
        out = np.empty((y1 - y0, wd), dtype=np.float64)
        inter = np.empty((8, y1 - y0, wd), dtype=np.float64) if intermediates else None
        rc = lib.ora_harris_f64(_ptr(xf), wd, h, _ptr(sxf), _ptr(syf), _ptr(gf), wk, float(k),
                                y0, y1, _ptr(out), _ptr(inter) if intermediates else None)
        if rc != 0:
            raise ValueError(f"oracle harris rejected its arguments (code {rc})")
        if intermediates:
            return out, {n: inter[i] for i, n in enumerate(HARRIS_PLANES)}
        return out


    def conv2d_backward(self, x, w, g, border: str = "clamp", border_value: float = 0.0):
        """(dx, dw): adjoint of ``conv2d`` applied to the upstream gradient ``g``."""
        lib = self.lib
        h, wd = np.shape(x)
        kh, kw = np.shape(w)
        xf, wf, gf = _f64(x), _f64(w), _f64(g)
        dx = np.empty((h, wd))
        dw = np.empty((kh, kw))
        rc = lib.ora_conv2d_bwd_f64(_ptr(xf), wd, h, _ptr(wf), kw, kh, BORDER[border],
                                    float(border_value), _ptr(gf), _ptr(dx), _ptr(dw))
        if rc != 0:
            raise ValueError(f"oracle conv2d_backward failed (code {rc})")
        return dx, dw


    def sepconv_backward(self, x, row, col, g, border: str = "clamp", border_value: float = 0.0):
        """(dx, drow, dcol): adjoint of ``sepconv`` applied to ``g``."""
        lib = self.lib
        h, wd = np.shape(x)
        xf, rf, cf, gf = _f64(x), _f64(row).ravel(), _f64(col).ravel(), _f64(g)
        dx = np.empty((h, wd))
        drow = np.empty(rf.size)
        dcol = np.empty(cf.size)
        rc = lib.ora_sepconv_bwd_f64(_ptr(xf), wd, h, _ptr(rf), rf.size, _ptr(cf), cf.size,
                                     BORDER[border], float(border_value), _ptr(gf), _ptr(dx),
                                     _ptr(drow), _ptr(dcol))
        if rc != 0:
            raise ValueError(f"oracle sepconv_backward failed (code {rc})")
        return dx, drow, dcol


    def harris_backward(self, img, sx, sy, win, gR, k: float = 0.04):
        """(dI, dsx, dsy, dwin): adjoint of ``harris`` applied to the upstream gradient."""
        lib = self.lib
        h, wd = np.shape(img)
        xf, sxf, syf, gf, gRf = _f64(img), _f64(sx), _f64(sy), _f64(win), _f64(gR)
        wk = gf.shape[0]
        dI = np.empty((h, wd))
        dsx = np.empty((3, 3))
        dsy = np.empty((3, 3))
        dwin = np.empty((wk, wk))
        rc = lib.ora_harris_bwd_f64(_ptr(xf), wd, h, _ptr(sxf), _ptr(syf), _ptr(gf), wk, float(k),
                                    _ptr(gRf), _ptr(dI), _ptr(dsx), _ptr(dsy), _ptr(dwin))
        if rc != 0:
            raise ValueError(f"oracle harris_backward failed (code {rc})")
        return dI, dsx, dsy, dwin


_default: Oracle | None = None


def default() -> Oracle:
    """The oracle built from ``imagecl_oracle.c`` (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def from_source(src: str, out: str) -> Oracle:
    """Compile another copy of the oracle source (used by the mutation tests)."""
    return Oracle(build(force=True, src=src, out=out))


def num_threads() -> int:
    return default().num_threads()


def conv2d(*a, **k):
    return default().conv2d(*a, **k)


def sepconv(*a, **k):
    return default().sepconv(*a, **k)


def harris(*a, **k):
    return default().harris(*a, **k)


def conv2d_backward(*a, **k):
    return default().conv2d_backward(*a, **k)


def sepconv_backward(*a, **k):
    return default().sepconv_backward(*a, **k)


def harris_backward(*a, **k):
    return default().harris_backward(*a, **k)
