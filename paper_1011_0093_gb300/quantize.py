"""One image through the whole path: reduce -> init -> iterate -> map -> MSE.

Only allocation (torch) and the sequence of C-ABI calls live here.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _native as N


@dataclass
class Quantized:
    centers: torch.Tensor     # float32 [K, 4] palette (R, G, B, unused), device
    index: torch.Tensor       # uint8 [H, W] palette index per pixel, device
    colors: torch.Tensor      # uint32 [N'] unique colors, device
    counts: torch.Tensor      # uint32 [N'] pixel counts, device
    labels: torch.Tensor      # uint8 [N'] final membership of each unique color, device
    n_unique: int
    iters: int
    sse_trace: list
    mse: float | None
    palette8: torch.Tensor | None = None   # uint8 [K, 4] 8-bit palette (ties to even), device
    mse8: float | None = None               # Eq. 2 with the 8-bit palette


def quantize(rgb: torch.Tensor, K: int, seed: int = 0, max_iter: int = 10, eps: float = 0.0,
             handle: N.Handle | None = None, mse: bool = True, palette8: bool = False,
             stream=None) -> Quantized:
    """Quantize one uint8 [H, W, 3|4] CUDA image to K colors.

    eps <= 0 runs exactly max_iter iterations (WSM); eps > 0 stops on the
    relative SSE change (WSM-C, Sec. 3.2) or at max_iter.  With mse, the MSE
    of Eq. 2 with the FP32 palette; with palette8 also the 8-bit palette and
    the MSE with it.
    """
    if not rgb.is_cuda or rgb.dtype != torch.uint8 or rgb.dim() != 3:
        raise ValueError("rgb must be a uint8 CUDA tensor of shape [H, W, 3|4]")
    rgb = rgb.contiguous()
    H, W, _ = rgb.shape
    n = H * W
    h = handle if handle is not None else N.Handle(max(K, 1), n, n)
    dev = rgb.device
    colors = torch.empty(n, dtype=torch.uint32, device=dev)
    counts = torch.empty(n, dtype=torch.uint32, device=dev)
    nu = N.wsm_reduce(h, rgb, colors, counts, stream=stream)
    colors, counts = colors[:nu], counts[:nu]
    centers = torch.empty((K, 4), dtype=torch.float32, device=dev)
    labels = torch.empty(nu, dtype=N.label_dtype(h), device=dev)
    N.wsm_init(h, colors, nu, K, seed, centers, labels, stream=stream)
    iters, trace = N.wsm_iterate(h, colors, counts, nu, K, centers, labels, max_iter, eps,
                                 stream=stream)
    index = torch.empty((H, W), dtype=N.label_dtype(h), device=dev)
    N.wsm_map(h, rgb, colors, nu, centers, K, labels, index, stream=stream)
    m = m8 = pal8 = None
    if mse:
        m = N.wsm_distortion(h, rgb, centers, K, index, stream=stream)
    if palette8:
        pal8, rounded = N.wsm_round_palette(h, centers, K, stream=stream)
        m8 = N.wsm_distortion(h, rgb, rounded, K, index, stream=stream)
    return Quantized(centers, index, colors, counts, labels, nu, iters, trace, m, pal8, m8)


def quantize_batch(images: list, K: int, seeds: list, max_iter: int = 10, eps: float = 0.0,
                   handle: N.Handle | None = None, mse: bool = True, stream=None) -> list:
    """Quantize several uint8 [H, W, 3|4] CUDA images to K colors each: one
    batched call per step of the path (unique colors, initialisation, the
    Sort-Means iterations in one persistent launch per 64 images, mapping,
    MSE), with the results of quantize() image by image."""
    if handle is None:
        biggest = max(int(im.shape[0]) * int(im.shape[1]) for im in images)
        handle = N.Handle(K, biggest, biggest)
    N.wsm_reserve_batch(handle, len(images))
    items = []
    for rgb in images:
        if not rgb.is_cuda or rgb.dtype != torch.uint8 or rgb.dim() != 3:
            raise ValueError("each image must be a uint8 CUDA tensor of shape [H, W, 3|4]")
        rgb = rgb.contiguous()
        H, W, _ = rgb.shape
        n = H * W
        dev = rgb.device
        items.append(dict(rgb=rgb, K=K,
                          colors=torch.empty(n, dtype=torch.uint32, device=dev),
                          counts=torch.empty(n, dtype=torch.uint32, device=dev),
                          centers=torch.empty((K, 4), dtype=torch.float32, device=dev),
                          labels=torch.empty(n, dtype=N.label_dtype(handle), device=dev),
                          index=torch.empty((H, W), dtype=N.label_dtype(handle), device=dev)))
    N.wsm_reduce_batch(handle, items, stream=stream)
    N.wsm_init_batch(handle, items, seeds, stream=stream)
    iters = N.wsm_iterate_batch(handle, items, max_iter, eps, stream=stream)
    N.wsm_map_batch(handle, items, stream=stream)
    mses = N.wsm_distortion_batch(handle, items, stream=stream) if mse else [None] * len(items)
    out = []
    for it, done, m in zip(items, iters, mses):
        nu = it["n_unique"]
        out.append(Quantized(it["centers"], it["index"], it["colors"][:nu], it["counts"][:nu],
                             it["labels"][:nu], nu, done, [], m))
    return out
