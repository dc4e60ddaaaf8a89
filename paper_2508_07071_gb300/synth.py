"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random inputs (images, crop rectangles, NV12 frames,
float tensors, chain constants, request arrivals). It holds none of the
preprocessing arithmetic, so both the CUDA path and the CPU checker can take
their inputs from it without sharing any computation.

Every generator takes an explicit integer seed and uses numpy's PCG64
(`numpy.random.default_rng(seed)`), so a (function, arguments, seed) triple
always yields the same bytes on x86 and Arm.
"""
from __future__ import annotations

import numpy as np

# Op kinds of the vertical Mul/Add chain (paper §VI-B, "Mul and Add" pairs).
KIND_MUL = 0
KIND_ADD = 1


def packed_image(seed: int, height: int, width: int, channels: int = 3,
                 lo: int = 0, hi: int = 255) -> np.ndarray:
    """uint8 HWC image, each byte uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(height, width, channels), dtype=np.uint8)


def crop_rois(seed: int, n: int, frame_w: int, frame_h: int,
              w_range: tuple[int, int], h_range: tuple[int, int]) -> np.ndarray:
    """n crop rectangles (x, y, w, h) as int32 [n, 4].

    w ~ U{w_range}, h ~ U{h_range} (inclusive), then the top-left corner is
    uniform over every position that keeps the rectangle inside the frame.
    """
    rng = np.random.default_rng(seed)
    w = rng.integers(w_range[0], w_range[1] + 1, size=n)
    h = rng.integers(h_range[0], h_range[1] + 1, size=n)
    x = np.array([rng.integers(0, frame_w - wi + 1) for wi in w])
    y = np.array([rng.integers(0, frame_h - hi + 1) for hi in h])
    return np.stack([x, y, w, h], axis=1).astype(np.int32)


def nv12_frames(seed: int, n: int, height: int, width: int,
                lo: int = 16, hi: int = 235) -> np.ndarray:
    """n NV12 frames as uint8 [n, height*3//2, width].

    Rows [0, height) are the luma plane; rows [height, height*3//2) are the
    interleaved chroma plane (U, V byte pairs at half resolution). Every byte,
    luma and chroma alike, is uniform in [lo, hi].
    """
    if height % 2 or width % 2:
        raise ValueError("NV12 needs even width and height")
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n, height * 3 // 2, width), dtype=np.uint8)


def f32_uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n float32 values uniform in [lo, hi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n).astype(np.float32)


def linear_values(seed: int, n: int, dtype: str) -> np.ndarray:
    """n values of one element type for the typed chains: u8 uniform in
    [0, 255], u16 uniform in [0, 65535], f32 and f64 uniform in [-1, 1) (the
    f64 values carry all 53 mantissa bits, so a cast to f32 rounds)."""
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        return rng.integers(0, 256, size=n, dtype=np.uint8)
    if dtype == "u16":
        return rng.integers(0, 65536, size=n, dtype=np.uint16)
    if dtype == "f32":
        return rng.uniform(-1.0, 1.0, size=n).astype(np.float32)
    if dtype == "f64":
        return rng.uniform(-1.0, 1.0, size=n)
    raise ValueError(f"unknown element type {dtype}")


def chain_constants(seed: int, length: int,
                    mul_range: tuple[float, float] = (0.99, 1.01),
                    add_range: tuple[float, float] = (-0.01, 0.01)):
    """Kinds and float32 constants of an alternating Mul/Add chain.

    Position i is a Mul when i is even and an Add when i is odd, so the chain
    starts with a Mul. Mul constants are uniform in mul_range, Add constants
    in add_range, all drawn from one stream in position order.
    """
    rng = np.random.default_rng(seed)
    kinds = np.array([KIND_MUL if i % 2 == 0 else KIND_ADD for i in range(length)],
                     dtype=np.int32)
    consts = np.empty(length, dtype=np.float32)
    for i in range(length):
        lo, hi = mul_range if kinds[i] == KIND_MUL else add_range
        consts[i] = np.float32(rng.uniform(lo, hi))
    return kinds, consts


def poisson_arrivals(seed: int, rate_per_s: float, n_requests: int) -> np.ndarray:
    """Arrival times in seconds of a Poisson process (exponential gaps)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_requests))


def serving_requests(seed: int, n_requests: int,
                     n_range=(1, 64), w_range=(320, 3840), h_range=(240, 2160)):
    """Per request: a list of (h, w, image seed) with n ~ U{n_range} images."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_requests):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        imgs = []
        for _ in range(n):
            w = int(rng.integers(w_range[0], w_range[1] + 1))
            h = int(rng.integers(h_range[0], h_range[1] + 1))
            imgs.append((h, w, int(rng.integers(0, 2**31 - 1))))
        out.append(imgs)
    return out
