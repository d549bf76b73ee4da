"""Seeded synthetic RGB images shaped like the test set of the WSM paper.

The paper evaluates on eight classic photographs and drawings (Sec. 3.1:
512x512-class natural images and two synthetic images, 7%..58% of the pixels
carrying a unique color, heavy-tailed color frequencies).  Those images are
not available here, so this module generates stand-ins of the same shape:

    base(x, y)  smooth two-axis gradient
                (255 x/(W-1), 255 y/(H-1), 255 (1 - (x+y)/(W+H-2))),
                posterized to multiples of ``BASE_STEP`` (flat regions, like
                sky and background in a photograph, give the heavy head of the
                frequency distribution);
    4 blobs     Gaussian spatial weight a = exp(-|p - p_b|^2 / (2 r_b^2)),
                center p_b ~ U(image), radius r_b ~ U(W/10, W/4), blob color
                U[0,255]^3 plus a N(0, 20^2) offset per channel; the pixel is
                lerp(base, blob color, a) -- smooth shading;
    noise       a luminance offset U{-A..A} shared by the three channels plus
                a chroma offset U{-A//4..A//4} per channel (the long tail of
                count-1 colors), then round-half-up and clamp to [0, 255].

Every random draw comes from a counter-based splitmix64 stream (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
draw i of stream s under seed S is mix64(S + gamma * (s * 2^40 + i + 1)).

This module holds none of the quantizer's arithmetic; it only produces
inputs, and both the CUDA path and the oracle consume what it returns.
"""
from __future__ import annotations

import math

import numpy as np

BASE_STEP = 64.0          # posterization step of the base gradient
BLOB_COUNT = 4
BLOB_SIGMA = 20.0         # spread of each blob's color, per channel
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def stream_u64(seed: int, stream: int, n: int) -> np.ndarray:
    """n raw 64-bit draws of stream ``stream`` under ``seed``."""
    ctr = (np.arange(n, dtype=np.uint64) + np.uint64(1)
           + (np.uint64(stream) << np.uint64(40)))
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GAMMA * ctr)


def stream_unif(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform on [0, 1) (top 53 bits of each draw)."""
    return (stream_u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def image(H: int, W: int, seed: int, noise: int) -> np.ndarray:
    """One seeded uint8 image of shape [H, W, 3] (see the module docstring)."""
    if H < 2 or W < 2:
        raise ValueError("image needs H, W >= 2")
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.stack([255.0 * x / (W - 1), 255.0 * y / (H - 1),
                    255.0 * (1.0 - (x + y) / (W + H - 2))], axis=-1)
    img = BASE_STEP * np.floor(img / BASE_STEP + 0.5)
    p = stream_unif(seed, 1, BLOB_COUNT * 9).reshape(BLOB_COUNT, 9)
    for b in range(BLOB_COUNT):
        cx, cy = p[b, 0] * W, p[b, 1] * H
        r = W / 10.0 + p[b, 2] * (W / 4.0 - W / 10.0)
        # Box-Muller on (p[6..8], p[7,8,6]) gives the N(0, sigma^2) offset
        gauss = np.sqrt(-2.0 * np.log1p(-p[b, 6:9])) * np.cos(2.0 * math.pi * p[b, [7, 8, 6]])
        color = 255.0 * p[b, 3:6] + BLOB_SIGMA * gauss
        a = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * r * r))[..., None]
        img = img * (1.0 - a) + a * color
    if noise > 0:
        chroma = noise // 4
        lum = (stream_u64(seed, 20, H * W) % np.uint64(2 * noise + 1)).astype(np.int64)
        img = img + (lum.reshape(H, W, 1) - noise)
        if chroma > 0:
            ch = (stream_u64(seed, 21, H * W * 3) % np.uint64(2 * chroma + 1)).astype(np.int64)
            img = img + (ch.reshape(H, W, 3) - chroma)
    return np.clip(np.floor(img + 0.5), 0, 255).astype(np.uint8)


# ---- the workloads -----------------------------------------------------------

def plain_256() -> np.ndarray:
    """256x256, seed 0, noise 6: the single-image parity workload (K=16)."""
    return image(256, 256, 0, 6)


SWEEP_NOISE = (0, 3, 7, 10, 14, 17, 21, 24)   # round(24 s / 7), s = 0..7


def sweep_512() -> list[np.ndarray]:
    """8 images 512x512, seeds 1..8, noise swept 0..24 (K in {32,64,128,256})."""
    return [image(512, 512, s + 1, a) for s, a in enumerate(SWEEP_NOISE)]


def sweep_512_one(s: int) -> np.ndarray:
    return image(512, 512, s + 1, SWEEP_NOISE[s])


def batch_sizes(seed: int, count: int, lo: int, hi: int) -> list[tuple[int, int]]:
    """Seeded (H, W) pairs, each side log-uniform in [lo, hi]."""
    u = stream_unif(seed, 30, 2 * count).reshape(count, 2)
    sides = np.floor(lo * (hi / lo) ** u + 0.5).astype(np.int64)
    return [(int(h), int(w)) for h, w in sides]


def tiny(H: int, W: int, seed: int, levels: int) -> np.ndarray:
    """Small image whose channels take only ``levels`` distinct values.

    Used to force duplicate colors and exact distance ties on tiny cases.
    """
    u = stream_u64(seed, 40, H * W * 3) % np.uint64(levels)
    step = 255 // max(levels - 1, 1)
    return (u.astype(np.int64) * step).reshape(H, W, 3).astype(np.uint8)
