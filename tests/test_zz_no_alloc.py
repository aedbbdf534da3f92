"""imagecl_sepconv_noalloc: the separable correlation for callers that must not
allocate device memory (plugins inside a framework that owns all device memory,
real-time loops that cannot take an allocation's synchronisation).  Its row-pass
intermediate lives in a fixed library array instead of a caller workspace.

This file is named so that pytest collects it last.  Each check calls the entry point
through the C ABI twice in a row, with different inputs, and compares both results with
the existing imagecl_sepconv: bit for bit against its PLAIN variant (the same kernels)
and within the scaled 1e-5 tolerance of the other tests against its default variant.
"""
import ctypes

import numpy as np
import pytest
import torch

from metrics import check_float_output, sep_reference
from paper_1605_06399_gb300 import _abi, ops, synth

pytestmark = pytest.mark.gpu


def _noalloc(x, y, row, col, border=0, bv=0.0, mem=_abi.MEM_HOST):
    xi, yi = ops.image(x), ops.image(y)
    r_ptr = row.data_ptr() if mem == _abi.MEM_DEVICE else row.ctypes.data
    c_ptr = col.data_ptr() if mem == _abi.MEM_DEVICE else col.ctypes.data
    st = _abi.lib().imagecl_sepconv_noalloc(ctypes.byref(xi), ctypes.byref(yi), ctypes.c_void_p(r_ptr),
                                            len(row), ctypes.c_void_p(c_ptr), len(col), mem, border, bv,
                                            ctypes.c_void_p(ops.stream_handle()))
    return st


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def test_noalloc_matches_sepconv_two_calls_in_a_row():
    g = np.random.default_rng(404)
    plain = {"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16}
    cases = [((333, 517), 3, "f32", torch.float32, ("clamp", 0.0)),
             ((1024, 2048), 7, "bf16", torch.float32, ("constant", 0.375))]
    for (h, w), radius, dt, out_dt, (border, bv) in cases:
        x = synth.to_storage(synth.uniform_f32(g, h, w), dt)
        row = synth.gaussian_taps(radius)
        col = g.standard_normal(2 * radius + 1).astype(np.float32)
        xd = x.cuda()
        y = torch.full((h, w), float("nan"), dtype=out_dt, device="cuda")
        st = _noalloc(xd, y, row, col, ops.BORDERS[border], bv)
        assert st == _abi.OK, _abi.lib().imagecl_last_error()
        ref_plain = ops.sepconv(xd, row, col, border, bv, out_dtype=out_dt, variant=plain)
        ref_default = ops.sepconv(xd, row, col, border, bv, out_dtype=out_dt)
        torch.cuda.synchronize()
        assert torch.equal(y, ref_plain), f"{dt} {h}x{w}: differs from the PLAIN variant"
        y64, s = sep_reference(x, row, col, border, bv)
        check_float_output(y, y64, s, out_dt, "no-alloc vs oracle")
        check_float_output(ref_default, y64, s, out_dt, "default vs oracle")
        diff = (y.double() - ref_default.double()).abs().cpu().numpy()
        assert float((diff / np.maximum(s, 1e-30)).max()) <= 2e-5


def test_noalloc_device_taps_and_f16_output():
    g = np.random.default_rng(405)
    for _ in range(2):
        x = synth.to_storage(synth.uniform_f32(g, 200, 300), "f16").cuda()
        row = torch.from_numpy(synth.gaussian_taps(4)).cuda()
        col = torch.from_numpy(synth.gaussian_taps(2)).cuda()
        y = torch.empty((200, 300), dtype=torch.float16, device="cuda")
        assert _noalloc(x, y, row, col, mem=_abi.MEM_DEVICE) == _abi.OK
        ref = ops.sepconv(x, row, col, out_dtype=torch.float16,
                          variant={"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16})
        torch.cuda.synchronize()
        assert torch.equal(y, ref)


def test_noalloc_rejects_images_beyond_its_scratch():
    x = torch.zeros((2049, 2048), device="cuda")            # 4,196,352 pixels > 16 MiB / 4
    y = torch.empty_like(x)
    t = synth.gaussian_taps(1)
    assert _noalloc(x, y, t, t) == _abi.ERR_UNSUPPORTED
    assert b"IMAGECL_NOALLOC_SCRATCH_BYTES" in _abi.lib().imagecl_last_error()
    x2 = torch.zeros((2048, 2048), device="cuda")           # exactly at the limit
    assert _noalloc(x2, torch.empty_like(x2), t, t) == _abi.OK
    torch.cuda.synchronize()


def test_noalloc_images_taller_than_a_grid():
    """2 x 2,000,000 pixels fit the scratch array but need more row blocks than a grid
    can be high (65535): the kernels walk the rows, so the result still equals PLAIN."""
    g = np.random.default_rng(406)
    x = torch.from_numpy(synth.uniform_f32(g, 2_000_000, 2)).cuda()
    row, col = synth.gaussian_taps(1), synth.gaussian_taps(3)
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        assert _noalloc(x, y, row, col) == _abi.OK, _abi.lib().imagecl_last_error()
        ref = ops.sepconv(x, row, col, variant={"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16})
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
    y64, s = sep_reference(x.cpu(), row, col, rows=(0, 64), halo=3)
    check_float_output(y[:64], y64, s, torch.float32, "tall no-alloc top rows")
    y64, s = sep_reference(x.cpu(), row, col, rows=(1_999_936, 2_000_000), halo=3)
    check_float_output(y[-64:], y64, s, torch.float32, "tall no-alloc bottom rows")

