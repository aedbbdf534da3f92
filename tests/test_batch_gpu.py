"""The ragged batch (one persistent, graph-replayed launch) against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import assert_pads_intact, empty_padded
from metrics import check_float_output, conv_reference, sep_reference
from paper_1605_06399_gb300 import Batch, ops, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert ops.device_status() == 0


def _mixed_items(g):
    shapes = [(1, 1), (1, 33), (33, 1), (7, 5), (64, 64), (130, 200), (257, 511), (31, 97), (300, 20)]
    storage = [("f16", torch.float16), ("f16", torch.float32), ("bf16", torch.bfloat16), ("f32", torch.float32)]
    items, meta = [], []
    i = 0
    for (h, w) in shapes:
        for conv_k in (1, 3, 7, 15, (3, 7)):
            st, od = storage[i % len(storage)]
            border, bv = (("clamp", 0.0), ("constant", 0.375))[i % 2]
            x = synth.to_storage(synth.uniform_f32(g, h, w), st)
            kh, kw = conv_k if isinstance(conv_k, tuple) else (conv_k, conv_k)
            taps = g.standard_normal((kh, kw)).astype(np.float32)
            items.append({"op": "conv", "x": x.cuda(), "taps": torch.from_numpy(taps).cuda(), "out_dtype": od,
                          "border": border, "border_value": bv})
            meta.append(("conv", x, taps, None, od, border, bv))
            i += 1
        for (nr, nc) in ((3, 3), (15, 15), (5, 9), (1, 7)):
            st, od = storage[i % len(storage)]
            border, bv = (("clamp", 0.0), ("constant", 0.375))[i % 2]
            x = synth.to_storage(synth.uniform_f32(g, h, w), st)
            r = g.standard_normal(nr).astype(np.float32)
            c = g.standard_normal(nc).astype(np.float32)
            items.append({"op": "sep", "x": x.cuda(), "taps": torch.from_numpy(r).cuda(),
                          "col_taps": torch.from_numpy(c).cuda(), "out_dtype": od, "border": border,
                          "border_value": bv})
            meta.append(("sep", x, r, c, od, border, bv))
            i += 1
    return items, meta


def _check(meta, outs):
    for k, ((op, x, t1, t2, od, border, bv), y) in enumerate(zip(meta, outs)):
        if op == "conv":
            ref, s = conv_reference(x, t1, border, bv)
        else:
            ref, s = sep_reference(x, t1, t2, border, bv)
        check_float_output(y, ref, s, od, f"item {k} {op} {tuple(x.shape)} {border}")


def test_mixed_batch_matches_oracle_and_replays():
    g = np.random.default_rng(9000)
    items, meta = _mixed_items(g)
    b = Batch(items, tune_budget_s=1.0)
    info = b.info()
    assert info["images"] == len(items) and info["tiles"] > len(items)
    outs = b.run()
    torch.cuda.synchronize()
    _check(meta, outs)
    first = [o.clone() for o in outs]
    b.run()
    torch.cuda.synchronize()
    for a, o in zip(first, outs):
        assert torch.equal(a, o), "graph replay changed a result"
    # change inputs in place: the replayed plan sees the new pixels
    for it, m in zip(items, meta):
        newx = synth.to_storage(synth.uniform_f32(g, *it["x"].shape), {torch.float16: "f16", torch.bfloat16: "bf16",
                                                                       torch.float32: "f32"}[it["x"].dtype])
        it["x"].copy_(newx.cuda())
    meta = [(m[0], it["x"].cpu()) + m[2:] for it, m in zip(items, meta)]
    b.run()
    torch.cuda.synchronize()
    _check(meta, outs)
    b.close()


def test_batch_pitched_views_unaligned():
    """Images that are column windows of wider buffers: rows start off 16-byte boundaries
    (the first rows and last rows of such images are read without bulk copies) and the
    pitch exceeds the width.  Outputs are views into padded buffers with guard bands that
    must stay untouched."""
    g = np.random.default_rng(9100)
    items, meta = [], []
    i = 0
    for st, od in (("f16", torch.float16), ("bf16", torch.float32), ("f32", torch.float32)):
        for (h, w, o) in ((1, 5, 1), (9, 70, 3), (130, 77, 5), (70, 260, 7), (300, 9, 2)):
            border, bv = (("clamp", 0.0), ("constant", -0.625))[i % 2]
            full = synth.to_storage(synth.uniform_f32(g, h, w + o + 11), st).cuda()
            x = full[:, o:o + w]
            if i % 2 == 0:
                k = (3, 7, 15)[i % 3]
                taps = g.standard_normal((k, k)).astype(np.float32)
                items.append({"op": "conv", "x": x, "taps": torch.from_numpy(taps).cuda(),
                              "out": empty_padded(h, w, od), "border": border, "border_value": bv})
                meta.append(("conv", x.cpu(), taps, None, od, border, bv))
            else:
                r = g.standard_normal(2 * (i % 7) + 1).astype(np.float32)
                c = g.standard_normal(2 * ((i + 3) % 7) + 1).astype(np.float32)
                items.append({"op": "sep", "x": x, "taps": torch.from_numpy(r).cuda(),
                              "col_taps": torch.from_numpy(c).cuda(), "out": empty_padded(h, w, od),
                              "border": border, "border_value": bv})
                meta.append(("sep", x.cpu(), r, c, od, border, bv))
            i += 1
    b = Batch(items, tune_budget_s=0.5)
    outs = b.run()
    torch.cuda.synchronize()
    _check(meta, outs)
    for k, it in enumerate(items):
        assert_pads_intact(it["out"], f"batch item {k}")
    b.close()


def test_workload_256_images_sampled():
    """256 f16 images, sides log-uniform in [64, 2048], each with an N(0,1) conv filter of
    odd side 3..15 or a Gaussian separable pair of radius 1..7: the whole batch in one
    graph launch, every small image checked in full and row bands of the large ones."""
    items = synth.workload_batch()
    bitems, meta = [], []
    for it in items:
        x = it.image.cuda()
        if it.op == "conv":
            bitems.append({"op": "conv", "x": x, "taps": torch.from_numpy(it.taps).cuda(),
                           "out_dtype": torch.float16})
        else:
            bitems.append({"op": "sep", "x": x, "taps": torch.from_numpy(it.taps).cuda(),
                           "col_taps": torch.from_numpy(it.col_taps).cuda(), "out_dtype": torch.float16})
        meta.append(it)
    b = Batch(bitems, tune_budget_s=3.0)
    outs = b.run()
    torch.cuda.synchronize()
    info = b.info()
    assert 80e6 < info["pixels"] < 90e6
    for it, y in zip(meta, outs):
        r = it.k // 2
        if it.width * it.height <= 160 * 160:
            rows, halo = None, None
        else:
            rows, halo = (it.height // 2, it.height // 2 + 3), r
        yy = y if rows is None else y[rows[0]:rows[1]]
        if it.op == "conv":
            ref, s = conv_reference(it.image, it.taps, rows=rows, halo=halo)
        else:
            ref, s = sep_reference(it.image, it.taps, it.col_taps, rows=rows, halo=halo)
        check_float_output(yy, ref, s, torch.float16, f"{it.op} k={it.k} {it.height}x{it.width}")
    b.close()


TOL_GRAD = 1e-4


def _gate(gpu, ref, scale, what):
    e = np.abs(gpu.detach().cpu().double().numpy() - ref) / np.maximum(scale, 1e-30)
    assert float(e.max()) <= TOL_GRAD, f"{what}: scaled error {float(e.max()):.3e}"


def test_batch_backward_matches_oracle():
    """Batch adjoint against the single-image oracle adjoints, item by item."""
    import oracle
    g = np.random.default_rng(9100)
    shapes = [(1, 1), (5, 3), (40, 70), (130, 257), (64, 300), (300, 31)]
    items, meta = [], []
    i = 0
    for (h, w) in shapes:
        for spec in (("conv", 3), ("conv", 15), ("conv", (5, 9)), ("sep", (3, 3)), ("sep", (15, 5)), ("sep", (1, 7))):
            # six specs per shape: shift the storage type and border per shape so that each
            # spec meets every type and both borders
            st = ("f16", "f32", "bf16")[(i + i // 6) % 3]
            border, bv = (("clamp", 0.0), ("constant", 0.375))[(i + i // 6) % 2]
            x = synth.to_storage(synth.uniform_f32(g, h, w), st)
            gr = torch.from_numpy(g.standard_normal((h, w)).astype(np.float32))
            if spec[0] == "conv":
                kh, kw = spec[1] if isinstance(spec[1], tuple) else (spec[1], spec[1])
                t = g.standard_normal((kh, kw)).astype(np.float32)
                items.append({"op": "conv", "x": x.cuda(), "taps": torch.from_numpy(t).cuda(), "border": border,
                              "border_value": bv, "grad_out": gr.cuda(), "out_dtype": torch.float32})
                meta.append(("conv", x, t, None, gr.numpy(), border, bv))
            else:
                nr, nc = spec[1]
                r = g.standard_normal(nr).astype(np.float32)
                c = g.standard_normal(nc).astype(np.float32)
                items.append({"op": "sep", "x": x.cuda(), "taps": torch.from_numpy(r).cuda(),
                              "col_taps": torch.from_numpy(c).cuda(), "border": border, "border_value": bv,
                              "grad_out": gr.cuda(), "out_dtype": torch.float32})
                meta.append(("sep", x, r, c, gr.numpy(), border, bv))
            i += 1
    b = Batch(items, tune_budget_s=1.0)
    assert b.info()["has_backward"]
    b.run()
    gin, gt, gt2 = b.backward()
    torch.cuda.synchronize()
    for k, (op, x, t1, t2, gr, border, bv) in enumerate(meta):
        ax = np.abs(x.double().numpy())
        what = f"item {k} {op} {tuple(x.shape)} {border}"
        if op == "conv":
            dx64, dw64 = oracle.conv2d_backward(x, t1, gr, border, bv)
            sdx, sdw = oracle.conv2d_backward(ax, np.abs(t1), np.abs(gr), border, abs(bv))
            _gate(gin[k], dx64, sdx, "dx " + what)
            _gate(gt[k], dw64, sdw, "dw " + what)
        else:
            dx64, dr64, dc64 = oracle.sepconv_backward(x, t1, t2, gr, border, bv)
            sdx, sdr, sdc = oracle.sepconv_backward(ax, np.abs(t1), np.abs(t2), np.abs(gr), border, abs(bv))
            _gate(gin[k], dx64, sdx, "dx " + what)
            _gate(gt[k], dr64, sdr, "drow " + what)
            _gate(gt2[k], dc64, sdc, "dcol " + what)
    b.close()
