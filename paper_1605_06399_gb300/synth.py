"""Seeded synthetic inputs shaped like the paper's benchmark workloads (§6).

This module only draws inputs: images, filter taps and batch descriptions. It holds
none of the stencil arithmetic, so the CUDA path and the CPU oracle can both be fed
from it without sharing any of the method.

Every generator takes an explicit ``numpy.random.Generator`` (PCG64).  The workload
seeds are ``SEED_BASE + n`` for workload ``n`` (1: 512x512 u8 3x3 integer filter,
2: 8192x8192 f32 non-separable, 3: 8192x8192 separable Gaussian, 4: 4096x4096 Harris
on rectangles, 5: ragged batch of 256 f16 images).

Storage rounding (f32 -> f16 / bf16) is round-to-nearest-even and is done here, once,
so that both sides see bit-identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

SEED_BASE = 1605000


def rng(seed_offset: int) -> np.random.Generator:
    """PCG64 generator for workload ``seed_offset`` (seed = 1605000 + offset)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(seed_offset)))


# --------------------------------------------------------------------------- images

def uniform_u8(g: np.random.Generator, h: int, w: int) -> np.ndarray:
    """u8 image, pixels uniform in 0..255 (the 8-bit grayscale benchmark image, §6)."""
    return g.integers(0, 256, size=(h, w), dtype=np.uint8)


def uniform_f32(g: np.random.Generator, h: int, w: int) -> np.ndarray:
    """f32 image, pixels uniform in [0, 1)."""
    return g.random((h, w), dtype=np.float32)


def rectangles_image(g: np.random.Generator, h: int, w: int, n_rect: int = 400,
                     side_lo: int = 16, side_hi: int = 512, noise_sd: float = 0.02) -> np.ndarray:
    """Corner-detection test image: axis-aligned rectangles plus Gaussian noise.

    ``n_rect`` rectangles with sides uniform in {side_lo..side_hi} (capped at the image
    size), top-left corner uniform such that the rectangle fits, intensity uniform in
    [0, 1), painted in order over a 0 background (later ones overwrite earlier ones);
    then N(0, noise_sd) noise is added in f32, without clipping.
    """
    img = np.zeros((h, w), dtype=np.float32)
    for _ in range(n_rect):
        rw = int(g.integers(side_lo, side_hi + 1))
        rh = int(g.integers(side_lo, side_hi + 1))
        rw, rh = min(rw, w), min(rh, h)
        x0 = int(g.integers(0, w - rw + 1))
        y0 = int(g.integers(0, h - rh + 1))
        img[y0:y0 + rh, x0:x0 + rw] = np.float32(g.random())
    if noise_sd > 0:
        img += g.normal(0.0, noise_sd, size=(h, w)).astype(np.float32)
    return img


def rectangles_noise_free(h: int, w: int, rects) -> np.ndarray:
    """Image with the given ``(x0, y0, rw, rh, value)`` rectangles on 0, no noise."""
    img = np.zeros((h, w), dtype=np.float32)
    for x0, y0, rw, rh, v in rects:
        img[y0:y0 + rh, x0:x0 + rw] = np.float32(v)
    return img


# --------------------------------------------------------------------------- filters

def int_filter(g: np.random.Generator, k: int, lo: int = -4, hi: int = 4) -> np.ndarray:
    """k x k int32 taps uniform in [lo, hi]."""
    return g.integers(lo, hi + 1, size=(k, k)).astype(np.int32)


def normal_filter_l1(g: np.random.Generator, k: int) -> np.ndarray:
    """k x k taps drawn N(0, 1) then divided by their L1 norm (in f64), stored f32."""
    w = g.standard_normal((k, k))
    w = w / np.abs(w).sum()
    return w.astype(np.float32)


def normal_filter(g: np.random.Generator, k: int) -> np.ndarray:
    """k x k taps drawn N(0, 1), stored f32 (the ragged-batch filters)."""
    return g.standard_normal((k, k)).astype(np.float32)


def gaussian_taps(radius: int, sigma: float | None = None) -> np.ndarray:
    """1-D Gaussian taps exp(-k^2 / (2 sigma^2)), k = -radius..radius, sigma = radius/3
    by default; normalised to unit sum in f64 and rounded to f32 once."""
    if sigma is None:
        sigma = radius / 3.0
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    t = np.exp(-(k * k) / (2.0 * sigma * sigma))
    t = t / t.sum()
    return t.astype(np.float32)


def gaussian_window(size: int, sigma: float) -> np.ndarray:
    """size x size Gaussian window exp(-(i^2 + j^2) / (2 sigma^2)), unit sum in f64, f32."""
    r = size // 2
    k = np.arange(-r, r + 1, dtype=np.float64)
    t = np.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2.0 * sigma * sigma))
    t = t / t.sum()
    return t.astype(np.float32)


def sobel_x() -> np.ndarray:
    """Unnormalised 3x3 Sobel taps for d/dx (row j = dy, column i = dx)."""
    return np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], dtype=np.float32)


def sobel_y() -> np.ndarray:
    """Unnormalised 3x3 Sobel taps for d/dy (the transpose of ``sobel_x``)."""
    return np.ascontiguousarray(sobel_x().T)


HARRIS_K = 0.04


# --------------------------------------------------------------------------- storage

def to_storage(a: np.ndarray, dtype: str) -> torch.Tensor:
    """Round an f32 array to the storage type ('f32', 'f16', 'bf16') with RN-even.

    Returns a CPU torch tensor (numpy has no bf16)."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    if dtype == "f32":
        return t.clone()
    if dtype == "f16":
        return t.to(torch.float16)
    if dtype == "bf16":
        return t.to(torch.bfloat16)
    raise ValueError(dtype)


TORCH_DTYPE = {"u8": torch.uint8, "i32": torch.int32, "f32": torch.float32,
               "f16": torch.float16, "bf16": torch.bfloat16}


# --------------------------------------------------------------------------- workloads

def workload_int3x3(h: int = 512, w: int = 512, k: int = 3, seed_offset: int = 1):
    """512x512 u8 image, 3x3 integer taps in [-4, 4] (int32 accumulation)."""
    g = rng(seed_offset)
    return uniform_u8(g, h, w), int_filter(g, k)


def workload_conv_f32(k: int, h: int = 8192, w: int = 8192, seed_offset: int = 2):
    """8192x8192 f32 image, k x k N(0,1) taps normalised to unit L1 sum."""
    g = rng(seed_offset)
    img = uniform_f32(g, h, w)
    return img, normal_filter_l1(g, k)


def workload_sep(radius: int, h: int = 8192, w: int = 8192, seed_offset: int = 3):
    """8192x8192 f32 image and the radius-R Gaussian (sigma = R/3) row/column taps."""
    g = rng(seed_offset)
    img = uniform_f32(g, h, w)
    t = gaussian_taps(radius)
    return img, t, t.copy()


def box_window(size: int) -> np.ndarray:
    """size x size box window with unit sum (the Harris benchmark's 2x2 block, §6)."""
    return np.full((size, size), 1.0 / (size * size), dtype=np.float32)


def workload_harris(h: int = 4096, w: int = 4096, seed_offset: int = 4):
    """4096x4096 rectangles + noise image, Sobel taps, 5x5 sigma=1 Gaussian window."""
    g = rng(seed_offset)
    img = rectangles_image(g, h, w)
    return img, sobel_x(), sobel_y(), gaussian_window(5, 1.0), HARRIS_K


@dataclass
class BatchItem:
    """One image of the ragged batch and the stencil paired with it."""
    width: int
    height: int
    op: str                      # 'conv' (k x k taps) or 'sep' (Gaussian row/col taps)
    k: int                       # filter side (conv) or 2R+1 (sep)
    image: torch.Tensor          # (height, width) f16, CPU
    taps: np.ndarray             # conv: (k, k) f32; sep: (k,) f32 row taps
    col_taps: np.ndarray | None = field(default=None)


def log_uniform_side(g: np.random.Generator, lo: int, hi: int) -> int:
    return int(math.floor(math.exp(g.uniform(math.log(lo), math.log(hi)))))


def workload_batch(n: int = 256, lo: int = 64, hi: int = 2048, seed_offset: int = 5,
                   dtype: str = "f16") -> list[BatchItem]:
    """Ragged batch: n images with log-uniform sides in [lo, hi], pixels uniform [0, 1)
    stored f16; each paired (p = 0.5) with an N(0,1) conv filter of odd side 3..15 or a
    Gaussian separable filter of radius 1..7."""
    g = rng(seed_offset)
    items = []
    for _ in range(n):
        w = log_uniform_side(g, lo, hi)
        h = log_uniform_side(g, lo, hi)
        img = to_storage(uniform_f32(g, h, w), dtype)
        if g.random() < 0.5:
            k = int(g.choice([3, 5, 7, 9, 11, 13, 15]))
            items.append(BatchItem(w, h, "conv", k, img, normal_filter(g, k)))
        else:
            r = int(g.integers(1, 8))
            t = gaussian_taps(r)
            items.append(BatchItem(w, h, "sep", 2 * r + 1, img, t, t.copy()))
    return items
