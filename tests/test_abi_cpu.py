"""Host-side checks of the C ABI: the library loads, exports every entry point the
header declares, its structs match the ctypes layout, and argument validation rejects
bad calls before anything touches a GPU (no compute here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1605_06399_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "imagecl.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_abi.LIB_PATH):
        build.build()
    return _abi.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(imagecl_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    assert "imagecl_conv2d" in names and "imagecl_tune" in names
    assert len(names) >= 10


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (imagecl_\w+)", out))
    for name in declared_functions():
        assert name in exported, f"{name} declared in imagecl.h but not exported"
        assert hasattr(lib, name)
        assert name in _abi.SIGNATURES, f"{name} has no ctypes signature"


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "imagecl.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(imcl_image), '
                   'sizeof(imcl_variant), sizeof(imcl_problem), offsetof(imcl_image, pitch_bytes), '
                   'sizeof(imcl_batch_item), offsetof(imcl_batch_item, grad_in), sizeof(imcl_batch_info_t), '
                   'sizeof(imcl_tune_report), offsetof(imcl_tune_report, model_rmse));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                            check=True).stdout.split()]
    assert sizes == [ctypes.sizeof(_abi.Image), ctypes.sizeof(_abi.Variant),
                     ctypes.sizeof(_abi.Problem), _abi.Image.pitch_bytes.offset,
                     ctypes.sizeof(_abi.BatchItem), _abi.BatchItem.grad_in.offset,
                     ctypes.sizeof(_abi.BatchInfo), ctypes.sizeof(_abi.TuneReport),
                     _abi.TuneReport.model_rmse.offset]


def test_version_and_last_error(lib):
    assert lib.imagecl_version().decode().startswith("imagecl-gb300")
    assert isinstance(lib.imagecl_last_error(), bytes)


def _img(ptr, dt, w, h, pitch):
    return _abi.Image(ptr, dt, w, h, 0, pitch)


def _call(lib, xin, xout, taps_dt=_abi.F32, kw=3, kh=3, border=0, bv=0.0):
    taps = (ctypes.c_float * 225)()
    return lib.imagecl_conv2d(ctypes.byref(xin) if xin is not None else None,
                              ctypes.byref(xout) if xout is not None else None,
                              ctypes.cast(taps, ctypes.c_void_p), taps_dt, kw, kh, _abi.MEM_HOST,
                              border, bv, None, None)


def test_validation_rejects_bad_calls_before_any_launch(lib):
    # fake, never-dereferenced device addresses: every case fails in host validation
    a, b = 1 << 40, 1 << 41
    good_in = _img(a, _abi.F32, 64, 32, 256)
    good_out = _img(b, _abi.F32, 64, 32, 256)
    assert _call(lib, None, good_out) == _abi.ERR_INVALID
    assert _call(lib, _img(0, _abi.F32, 64, 32, 256), good_out) == _abi.ERR_INVALID
    assert _call(lib, _img(a, _abi.F32, 0, 32, 256), good_out) == _abi.ERR_INVALID
    assert _call(lib, _img(a, _abi.F32, 64, 32, 100), good_out) == _abi.ERR_INVALID   # pitch < row
    assert _call(lib, _img(a, _abi.F32, 64, 32, 258), good_out) == _abi.ERR_INVALID   # pitch % 4
    assert _call(lib, _img(a, 9, 64, 32, 256), good_out) == _abi.ERR_INVALID          # dtype
    assert _call(lib, good_in, _img(b, _abi.F32, 63, 32, 256)) == _abi.ERR_INVALID     # shape
    assert _call(lib, good_in, _img(a + 128, _abi.F32, 64, 32, 256)) == _abi.ERR_INVALID  # overlap
    assert _call(lib, good_in, good_out, kw=4, kh=4) == _abi.ERR_UNSUPPORTED          # even side
    assert _call(lib, good_in, good_out, kw=17, kh=17) == _abi.ERR_UNSUPPORTED        # too large
    assert _call(lib, good_in, good_out, taps_dt=_abi.I32) == _abi.ERR_INVALID        # taps type
    assert _call(lib, good_in, _img(b, _abi.I32, 64, 32, 256)) == _abi.ERR_INVALID     # out type
    assert _call(lib, good_in, good_out, border=5) == _abi.ERR_INVALID
    u8_in = _img(a, _abi.U8, 64, 32, 64)
    i32_out = _img(b, _abi.I32, 64, 32, 256)
    assert _call(lib, u8_in, i32_out, taps_dt=_abi.I32, border=1, bv=300.0) == _abi.ERR_INVALID
    assert _call(lib, u8_in, i32_out, taps_dt=_abi.I32, border=1, bv=2.5) == _abi.ERR_INVALID
    assert b"border_value" in lib.imagecl_last_error()
    assert lib.imagecl_selftest_wait_timeout(0, None) == _abi.ERR_INVALID          # unbounded wait
    assert lib.imagecl_selftest_wait_timeout(1 << 21, None) == _abi.ERR_INVALID


def test_build_units_cover_every_tiled_side():
    names = [u[2] for u in build.units()]
    for k in build.TILED_K:
        for g in build.TILED_GROUPS:
            assert f"conv2d_tiled_k{k}_g{g}.o" in names
