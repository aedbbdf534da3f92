"""torch.autograd.Function wrappers: forward and backward both run the library's kernels.

Taps given as CUDA tensors stay on the device (the kernels read them from there), so a
training step never copies them to the host.  Gradients are f32.
"""
from __future__ import annotations

import torch

from . import ops


class Conv2dFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, taps, border="clamp", border_value=0.0):
        ctx.border, ctx.border_value = border, border_value
        ctx.save_for_backward(x, taps)
        return ops.conv2d(x, taps, border, border_value)

    @staticmethod
    def backward(ctx, g):
        x, taps = ctx.saved_tensors
        dx, dw = ops.conv2d_backward(g, x, taps, ctx.border, ctx.border_value,
                                     need_dx=ctx.needs_input_grad[0], need_dw=ctx.needs_input_grad[1])
        return dx, dw, None, None


class SepConvFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, row_taps, col_taps, border="clamp", border_value=0.0):
        ctx.border, ctx.border_value = border, border_value
        ctx.save_for_backward(x, row_taps, col_taps)
        return ops.sepconv(x, row_taps, col_taps, border, border_value)

    @staticmethod
    def backward(ctx, g):
        x, r, c = ctx.saved_tensors
        dx, dr, dc = ops.sepconv_backward(g, x, r, c, ctx.border, ctx.border_value,
                                          need_dx=ctx.needs_input_grad[0],
                                          need_drow=ctx.needs_input_grad[1],
                                          need_dcol=ctx.needs_input_grad[2])
        return dx, dr, dc, None, None


class HarrisFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, sobel_x, sobel_y, window, k=0.04):
        ctx.k = k
        ctx.save_for_backward(x, sobel_x, sobel_y, window)
        return ops.harris(x, sobel_x, sobel_y, window, k)

    @staticmethod
    def backward(ctx, g):
        x, sx, sy, win = ctx.saved_tensors
        need_taps = any(ctx.needs_input_grad[1:4])
        dx, dsx, dsy, dwin = ops.harris_backward(g, x, sx, sy, win, ctx.k,
                                                 need_dx=ctx.needs_input_grad[0], need_taps=need_taps)
        return dx, dsx, dsy, dwin, None


def conv2d(x, taps, border="clamp", border_value=0.0):
    """Differentiable conv2d (input and taps)."""
    return Conv2dFn.apply(x, taps, border, border_value)


def sepconv(x, row_taps, col_taps=None, border="clamp", border_value=0.0):
    """Differentiable separable correlation (input, row taps, column taps)."""
    return SepConvFn.apply(x, row_taps, row_taps if col_taps is None else col_taps, border, border_value)


def harris(x, sobel_x, sobel_y, window, k=0.04):
    """Differentiable Harris response (image, both Sobel tap sets and the window)."""
    return HarrisFn.apply(x, sobel_x, sobel_y, window, k)
