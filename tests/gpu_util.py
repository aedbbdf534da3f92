"""Layout helpers for the GPU tests: dense tensors, or rows padded to 128 bytes so
that TMA-staged variants and vector stores are exercised on ragged widths.

Padded output buffers carry canary guard bands: every byte of the pad columns and of
one extra row below the image is set to a sentinel before the call, and
``assert_pads_intact`` checks afterwards that no kernel wrote outside the image."""
import torch

SENTINEL = 0xA5


def padded(t: torch.Tensor, device="cuda") -> torch.Tensor:
    """A (h, w) view of a buffer whose rows are padded to a multiple of 128 bytes."""
    h, w = t.shape
    per = 128 // t.element_size()
    buf = torch.zeros((h, (w + per - 1) // per * per), dtype=t.dtype, device=device)
    v = buf[:, :w]
    v.copy_(t.to(device))
    return v


def empty_padded(h, w, dtype):
    """An (h, w) output view into a buffer of rows padded to 128 bytes plus one guard row,
    all bytes set to the sentinel."""
    per = 128 // torch.empty((), dtype=dtype).element_size()
    buf = torch.empty((h + 1, (w + per - 1) // per * per), dtype=dtype, device="cuda")
    buf.view(torch.uint8).fill_(SENTINEL)
    return buf[:h, :w]


def assert_pads_intact(v: torch.Tensor, what: str = "") -> None:
    """The pad columns and the guard row of an ``empty_padded`` view still hold the
    sentinel."""
    buf = v._base
    assert buf is not None and buf.dim() == 2, "not a view made by empty_padded"
    h, w = v.shape
    raw = buf.view(torch.uint8)
    esz = v.element_size()
    pads = raw[:h, w * esz:]
    guard = raw[h:]
    bad = int((pads != SENTINEL).sum().item()) + int((guard != SENTINEL).sum().item())
    assert bad == 0, f"{what}: {bad} bytes written outside the image (pad columns or guard row)"


def place(t_cpu: torch.Tensor, layout: str) -> torch.Tensor:
    return t_cpu.cuda() if layout == "dense" else padded(t_cpu)


def out_buffer(h, w, dtype, layout):
    return None if layout == "dense" else empty_padded(h, w, dtype)
