"""conv2d on the GPU (through the C ABI) against the CPU oracle, element by element."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_pads_intact, empty_padded, padded
from metrics import check_float_output, conv_reference, to_f64
from paper_1605_06399_gb300 import ImclError, _abi, ops, synth

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (1, 17), (17, 1), (3, 2), (7, 13), (33, 65), (130, 259), (67, 300)]
EXTRA_SHAPES = [(16, 8), (64, 4), (8, 16)]


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    yield
    assert ops.device_status() == 0


def _inputs(g, h, w, dt):
    if dt == "u8":
        return torch.from_numpy(synth.uniform_u8(g, h, w))
    return synth.to_storage(synth.uniform_f32(g, h, w), dt)


def _variants_for(in_t, out_t, k, h, w, taps_mem, border):
    prob = ops.problem(_abi.OP_CONV2D, in_t, out_t, k, k, w, h, border, taps_mem)
    vs = ops.variants(prob)
    extra = []
    for v in vs:
        if v["kind"] == _abi.KIND_TILED and v["load"] == _abi.LOAD_TMA and v["py"] == 4:
            for bx, by in EXTRA_SHAPES:
                extra.append(dict(v, bx=bx, by=by))
    return [None] + vs + extra


def _run_all(x_cpu, taps, out_dtype, border, bv, taps_mem, layout):
    """Run every compiled variant; yield (variant, output) for those that launch.
    layout 'dense': contiguous tensors; 'padded': rows padded to 128 bytes (TMA-able)."""
    x = x_cpu.cuda() if layout == "dense" else padded(x_cpu)
    integer = x.dtype == torch.uint8
    k = taps.shape[0]
    t_dev = torch.from_numpy(taps).cuda() if taps_mem == _abi.MEM_DEVICE else taps
    out_t = torch.int32 if integer else out_dtype
    for v in _variants_for(x.dtype, out_t, k, x.shape[0], x.shape[1], taps_mem, border):
        out = None if layout == "dense" else empty_padded(x.shape[0], x.shape[1], out_t)
        try:
            y = ops.conv2d(x, t_dev, border, bv, out=out, out_dtype=out_t, variant=v)
        except ImclError as e:
            assert e.status in (_abi.ERR_UNSUPPORTED, _abi.ERR_ALIGN), str(e)
            continue
        if out is not None:
            assert_pads_intact(out, f"conv2d {v}")
        yield v, y


CASES = [("u8", torch.int32), ("f32", torch.float32), ("f16", torch.float32),
         ("f16", torch.float16), ("bf16", torch.float32), ("bf16", torch.bfloat16)]


@pytest.mark.parametrize("k", [1, 3, 5, 7, 9, 11, 13, 15])
@pytest.mark.parametrize("dt,out_dtype", CASES, ids=[f"{a}-{str(b)[6:]}" for a, b in CASES])
def test_conv2d_every_variant_matches_oracle(dt, out_dtype, k):
    g = np.random.default_rng(1000 + k)
    taps = synth.int_filter(g, k) if dt == "u8" else synth.normal_filter_l1(g, k)
    n_checked = 0
    for (h, w) in SIZES:
        x = _inputs(g, h, w, dt)
        for border, bv in (("clamp", 0.0), ("constant", 3.0 if dt == "u8" else 0.375)):
            ref, s = conv_reference(x, taps, border, bv)
            for mem, layout in ((_abi.MEM_HOST, "dense"), (_abi.MEM_HOST, "padded"),
                                (_abi.MEM_DEVICE, "padded"), (_abi.MEM_DEVICE, "dense")):
                for v, y in _run_all(x, taps, out_dtype, border, bv, mem, layout):
                    what = f"{dt}->{out_dtype} k={k} {h}x{w} {border} mem={mem} {layout} {v}"
                    if dt == "u8":
                        assert np.array_equal(y.cpu().numpy(), ref), what
                    else:
                        check_float_output(y, ref, s, out_dtype, what)
                    n_checked += 1
    assert n_checked > 0


def test_rectangular_filter_uses_plain_and_matches():
    g = np.random.default_rng(5)
    x = synth.to_storage(synth.uniform_f32(g, 45, 71), "f32")
    taps = g.standard_normal((3, 7)).astype(np.float32)
    y = ops.conv2d(x.cuda(), taps)
    ref, s = conv_reference(x, taps)
    check_float_output(y, ref, s, torch.float32, "3x7")


def test_workload_int3x3_bit_exact():
    """512x512 u8, 3x3 integer taps in [-4, 4], i32 accumulation: bit-exact."""
    img, taps = synth.workload_int3x3()
    x = torch.from_numpy(img).cuda()
    ref = oracle.conv2d(img, taps)
    for v in [None] + ops.variants(ops.problem(_abi.OP_CONV2D, "u8", "i32", 3, 3, 512, 512)):
        y = ops.conv2d(x, taps, variant=v)
        assert np.array_equal(y.cpu().numpy(), ref), v


def test_int_wraparound_matches_oracle():
    """Taps far past the f32-exact bound: the F32_EXACT variants run their integer twin,
    and every variant wraps like the oracle."""
    x = torch.full((20, 24), 255, dtype=torch.uint8)
    taps = np.full((15, 15), 2 ** 25, dtype=np.int32)   # 225 * 255 * 2^25 wraps int32
    ref = oracle.conv2d(x.numpy(), taps)
    vs = [None] + ops.variants(ops.problem(_abi.OP_CONV2D, "u8", "i32", 15, 15, 24, 20))
    assert any(v and v["unroll"] == _abi.UNROLL_F32_EXACT for v in vs)
    for v in vs:
        assert np.array_equal(ops.conv2d(padded(x), taps, variant=v).cpu().numpy(), ref), v


@pytest.mark.parametrize("wval", [292, 293])
def test_f32_exact_u8_at_the_bound(wval):
    """225 taps of 292 keep sum |w| * 255 = 16,753,500 below 2^24 (f32 accumulation is
    exact); 293 crosses it (16,810,875: the integer form runs).  Both bit-exact, on a
    saturated image and on random pixels with mixed-sign taps."""
    g = np.random.default_rng(wval)
    prob = ops.problem(_abi.OP_CONV2D, "u8", "i32", 15, 15, 300, 130)
    facc = [v for v in ops.variants(prob) if v["unroll"] == _abi.UNROLL_F32_EXACT]
    assert facc
    for x in (np.full((130, 300), 255, np.uint8), synth.uniform_u8(g, 130, 300)):
        taps = (wval * np.where(g.random((15, 15)) < 0.5, -1, 1)).astype(np.int32)
        if x[0, 0] == 255 and x.min() == 255:
            taps = np.abs(taps)
        ref = oracle.conv2d(x, taps)
        for v in facc:
            y = ops.conv2d(padded(torch.from_numpy(x)), taps, variant=v)
            assert np.array_equal(y.cpu().numpy(), ref), (wval, v)


@pytest.mark.parametrize("k", [5, 11])
def test_workload_8192_f32_tuned_sampled_rows(k):
    """8192x8192 f32, unit-L1 N(0,1) taps, the tuned launch the benchmark times; checked
    on row bands at the top, bottom and interior (every column of each band)."""
    img, taps = synth.workload_conv_f32(k)
    x = torch.from_numpy(img).cuda()
    prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", k, k, 8192, 8192)
    res = ops.tune(prob, budget_s=15.0, reps=3)
    y = ops.conv2d(x, taps)
    for rows in [(0, 6), (4093, 4101), (8186, 8192), (1234, 1236)]:
        ref, s = conv_reference(img, taps, rows=rows, halo=k // 2)
        check_float_output(y[rows[0]:rows[1]], ref, s, torch.float32, f"k={k} rows={rows} {res}")
    del x, y
    torch.cuda.empty_cache()


def test_unaligned_buffers_fall_back_and_match():
    g = np.random.default_rng(9)
    base = synth.to_storage(synth.uniform_f32(g, 50, 81), "f32").cuda()
    x = base[:, 1:]                                   # base address off by 4 bytes
    taps = synth.normal_filter_l1(g, 5)
    tma = {"kind": 1, "bx": 32, "by": 8, "px": 4, "py": 4, "load": _abi.LOAD_TMA, "filt": 0,
           "map": 0, "unroll": 1, "persistent": 1}
    with pytest.raises(ImclError) as ei:
        ops.conv2d(x, taps, variant=tma)
    assert ei.value.status == _abi.ERR_ALIGN
    y = ops.conv2d(x, taps)
    ref, s = conv_reference(x.cpu(), taps)
    check_float_output(y, ref, s, torch.float32, "unaligned")


def test_wide_and_tall_images():
    g = np.random.default_rng(10)
    taps = synth.normal_filter_l1(g, 7)
    for (h, w) in [(3, 70001), (40001, 5)]:
        x = synth.to_storage(synth.uniform_f32(g, h, w), "f32")
        y = ops.conv2d(x.cuda(), taps)
        ref, s = conv_reference(x, taps)
        check_float_output(y, ref, s, torch.float32, f"{h}x{w}")


def test_aliasing_rejected():
    x = torch.rand(32, 32, device="cuda")
    with pytest.raises(ImclError) as ei:
        ops.conv2d(x, np.ones((3, 3), np.float32), out=x)
    assert ei.value.status == _abi.ERR_INVALID


def test_tuner_reports_and_caches(tmp_path):
    prob = ops.problem(_abi.OP_CONV2D, "f32", "f32", 5, 5, 1024, 768)
    ops.tune_clear()
    res = ops.tune(prob, budget_s=5.0, reps=3)
    assert res["best_ms"] > 0 and res["plain_ms"] > 0
    assert res["best_ms"] <= res["plain_ms"] * 1.05
    assert ops.default_variant(prob) == res["variant"]
    path = str(tmp_path / "cache.txt")
    ops.tune_save(path)
    ops.tune_clear()
    ops.tune_load(path)
    assert ops.default_variant(prob) == res["variant"]


@pytest.mark.parametrize("k,border,bv", [(5, "clamp", 0.0), (11, "constant", 0.25)])
def test_row_bands_on_one_gpu_match_whole_image(k, border, bv):
    """The row-band partition of one image (what each rank of a multi-GPU run computes
    after its halo exchange), run band by band on one GPU: the band's own rows of the
    result on its extended band equal the whole image's rows bit for bit, and match the
    oracle on the whole image's rows."""
    from paper_1605_06399_gb300 import shard
    g = np.random.default_rng(6100 + k)
    x = torch.from_numpy(g.random((517, 301), dtype=np.float32)).cuda()
    taps = g.standard_normal((k, k)).astype(np.float32)
    whole = ops.conv2d(x, taps, border, bv)
    xc = x.cpu().numpy()
    for (y0, y1, e0, e1) in shard.row_bands(517, 4, (k - 1) // 2):
        band = ops.conv2d(x[e0:e1].contiguous(), taps, border, bv)
        assert torch.equal(band[y0 - e0:y1 - e0], whole[y0:y1]), (y0, y1)
        ref, s = conv_reference(xc, taps, border, bv, rows=(y0, y1), halo=k // 2)
        check_float_output(band[y0 - e0:y1 - e0], ref, s, torch.float32, f"band rows {y0}..{y1}")
