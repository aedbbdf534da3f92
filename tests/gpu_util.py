"""Layout helpers for the GPU tests: dense tensors, or rows padded to 128 bytes so
that TMA-staged variants and vector stores are exercised on ragged widths."""
import torch


def padded(t: torch.Tensor, device="cuda") -> torch.Tensor:
    """A (h, w) view of a buffer whose rows are padded to a multiple of 128 bytes."""
    h, w = t.shape
    per = 128 // t.element_size()
    buf = torch.zeros((h, (w + per - 1) // per * per), dtype=t.dtype, device=device)
    v = buf[:, :w]
    v.copy_(t.to(device))
    return v


def empty_padded(h, w, dtype):
    per = 128 // torch.empty((), dtype=dtype).element_size()
    return torch.empty((h, (w + per - 1) // per * per), dtype=dtype, device="cuda")[:, :w]


def place(t_cpu: torch.Tensor, layout: str) -> torch.Tensor:
    return t_cpu.cuda() if layout == "dense" else padded(t_cpu)


def out_buffer(h, w, dtype, layout):
    return None if layout == "dense" else empty_padded(h, w, dtype)
