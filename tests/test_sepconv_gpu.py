"""Separable correlation on the GPU (fused and two-kernel forms) against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import assert_pads_intact, out_buffer, place
from metrics import check_float_output, sep_reference
from paper_1605_06399_gb300 import ImclError, _abi, ops, synth

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (1, 19), (19, 1), (5, 3), (33, 65), (130, 259), (70, 300)]
CASES = [("f32", torch.float32), ("f16", torch.float32), ("f16", torch.float16),
         ("bf16", torch.float32), ("bf16", torch.bfloat16)]


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert ops.device_status() == 0


def _all_variants(dt, out_dtype, nr, nc, w, h, mem):
    prob = ops.problem(_abi.OP_SEPCONV, dt, out_dtype, nr, nc, w, h, "clamp", mem)
    vs = ops.variants(prob)
    extra = [dict(v, bx=bx, by=by) for v in vs if v["kind"] == _abi.KIND_TILED and v["load"] == _abi.LOAD_TMA
             for bx, by in ((16, 8), (8, 16), (32, 4))]
    return [None] + vs + extra


@pytest.mark.parametrize("radius", list(range(1, 17)))
@pytest.mark.parametrize("dt,out_dtype", CASES, ids=[f"{a}-{str(b)[6:]}" for a, b in CASES])
def test_sepconv_every_variant_matches_oracle(dt, out_dtype, radius):
    g = np.random.default_rng(2000 + radius)
    row = synth.gaussian_taps(radius)
    col = (g.standard_normal(2 * radius + 1)).astype(np.float32)   # asymmetric column taps
    n = 0
    for (h, w) in SIZES:
        x = synth.to_storage(synth.uniform_f32(g, h, w), dt)
        for border, bv in (("clamp", 0.0), ("constant", 0.375)):
            ref, s = sep_reference(x, row, col, border, bv)
            for mem, layout in ((_abi.MEM_HOST, "dense"), (_abi.MEM_HOST, "padded"),
                                (_abi.MEM_DEVICE, "padded"), (_abi.MEM_DEVICE, "dense")):
                xd = place(x, layout)
                r_arg = torch.from_numpy(row).cuda() if mem == _abi.MEM_DEVICE else row
                c_arg = torch.from_numpy(col).cuda() if mem == _abi.MEM_DEVICE else col
                for v in _all_variants(dt, out_dtype, row.size, col.size, w, h, mem):
                    out = out_buffer(h, w, out_dtype, layout)
                    try:
                        y = ops.sepconv(xd, r_arg, c_arg, border, bv, out=out, out_dtype=out_dtype,
                                        variant=v)
                    except ImclError as e:
                        assert e.status in (_abi.ERR_UNSUPPORTED, _abi.ERR_ALIGN), str(e)
                        continue
                    if out is not None:
                        assert_pads_intact(out, f"sepconv {v}")
                    check_float_output(y, ref, s, out_dtype,
                                       f"{dt}->{out_dtype} R={radius} {h}x{w} {border} mem={mem} {layout} {v}")
                    n += 1
    assert n > 0


@pytest.mark.parametrize("nr,nc", [(5, 9), (9, 5), (1, 33), (33, 1), (3, 1), (1, 1)])
def test_unequal_tap_counts(nr, nc):
    g = np.random.default_rng(nr * 100 + nc)
    x = synth.to_storage(synth.uniform_f32(g, 77, 140), "f32")
    row = g.standard_normal(nr).astype(np.float32)
    col = g.standard_normal(nc).astype(np.float32)
    ref, s = sep_reference(x, row, col)
    for v in [None] + ops.variants(ops.problem(_abi.OP_SEPCONV, "f32", "f32", nr, nc, 140, 77)):
        y = ops.sepconv(x.cuda(), row, col, variant=v)
        check_float_output(y, ref, s, torch.float32, f"{nr}x{nc} {v}")


def test_plain_needs_workspace():
    x = torch.rand(40, 50, device="cuda")
    t = synth.gaussian_taps(2)
    plain = {"kind": _abi.KIND_PLAIN, "bx": 16, "by": 16}
    xi, yi = ops.image(x), ops.image(torch.empty_like(x))
    import ctypes
    st = _abi.lib().imagecl_sepconv(ctypes.byref(xi), ctypes.byref(yi), ctypes.c_void_p(t.ctypes.data), 5,
                                    ctypes.c_void_p(t.ctypes.data), 5, _abi.MEM_HOST, 0, 0.0,
                                    ctypes.byref(_abi.Variant.from_dict(plain)), None, 0, None)
    assert st == _abi.ERR_INVALID
    assert ops.sepconv(x, t, variant=plain).shape == x.shape


@pytest.mark.parametrize("radius", [1, 4, 8, 16])
@pytest.mark.parametrize("dt,out_dtype", [("f32", torch.float32), ("bf16", torch.float32),
                                          ("f16", torch.float16), ("bf16", torch.bfloat16)])
def test_workload_8192_sampled_rows(radius, dt, out_dtype):
    """8192x8192 Gaussian (sigma = R/3) separable filter, the tuned launch, checked on row
    bands at the top, middle and bottom (every column)."""
    img, row, col = synth.workload_sep(radius)
    x = synth.to_storage(img, dt)
    xd = x.cuda()
    prob = ops.problem(_abi.OP_SEPCONV, dt, out_dtype, 2 * radius + 1, 2 * radius + 1, 8192, 8192)
    ops.tune(prob, budget_s=6.0, reps=3)
    y = ops.sepconv(xd, row, col, out_dtype=out_dtype)
    for rows in [(0, 5), (4090, 4099), (8187, 8192)]:
        ref, s = sep_reference(x, row, col, rows=rows, halo=radius)
        check_float_output(y[rows[0]:rows[1]], ref, s, out_dtype, f"R={radius} {dt} rows={rows}")
    del xd, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("radius", [1, 2, 4, 8, 13])
@pytest.mark.parametrize("dt,out_dtype", [("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float32)])
def test_packed_fma_form_gives_the_scalar_bits(dt, out_dtype, radius):
    """Both passes of UNROLL_PACKED keep the scalar operation order per lane: its output
    equals the scalar variant with the same axes bit for bit."""
    g = np.random.default_rng(5200 + radius)
    x = place(synth.to_storage(synth.uniform_f32(g, 263, 301), dt), "padded")
    row = synth.gaussian_taps(radius)
    col = g.standard_normal(2 * radius + 1).astype(np.float32)
    prob = ops.problem(_abi.OP_SEPCONV, dt, out_dtype, row.size, col.size, 301, 263)
    vs = ops.variants(prob)
    packed = [v for v in vs if v["unroll"] == _abi.UNROLL_PACKED]
    assert packed, "no packed variant compiled"
    axes = ("kind", "px", "py", "load", "filt", "map")
    for border, bv in (("clamp", 0.0), ("constant", 0.25)):
        for v in packed:
            twins = [u for u in vs if u["unroll"] == _abi.UNROLL_FULL and all(u[f] == v[f] for f in axes)]
            yp = ops.sepconv(x, row, col, border, bv, out=out_buffer(263, 301, out_dtype, "padded"), variant=v)
            if twins:
                ys = ops.sepconv(x, row, col, border, bv, out=out_buffer(263, 301, out_dtype, "padded"),
                                 variant=dict(twins[0], bx=v["bx"], by=v["by"]))
                assert torch.equal(ys, yp), f"packed {v} differs from its scalar form"
            else:
                ref, s = sep_reference(x.cpu(), row, col, border, bv)
                check_float_output(yp, ref, s, out_dtype, f"packed {v}")
