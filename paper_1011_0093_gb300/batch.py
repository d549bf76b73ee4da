"""A fixed batch of images through the whole path as one enqueue
(wsm_quantize_batch), optionally tuned (wsm_autotune_batch) and captured
into a CUDA graph, then replayed on new pixels.

Only buffer management and argument marshalling live here; every step of
the path runs in libwsm's CUDA kernels.  The pixels, index images and
palettes of all images live in one device buffer each (every image's part
256-byte aligned), so that loading a batch and reading its results take one
copy per field instead of one per image.
"""
from __future__ import annotations

import torch

from . import _native as N

_ALIGN = 256   # bytes: each image's part of a shared buffer starts on this boundary


def _offsets(nbytes):
    """Start offsets (bytes) of consecutive parts of the given sizes, each
    aligned to _ALIGN, and the total size."""
    offs, at = [], 0
    for b in nbytes:
        offs.append(at)
        at += (int(b) + _ALIGN - 1) // _ALIGN * _ALIGN
    return offs, at


def _pack_into(buf, offsets, shapes, images):
    """Write each image's bytes at its offset of the flat uint8 buffer `buf`,
    after checking that there is one image per shape and each has its shape."""
    images = list(images)
    if len(images) != len(shapes):
        raise ValueError(f"{len(images)} images for a plan of {len(shapes)}")
    for q, (im, shape, off) in enumerate(zip(images, shapes, offsets)):
        t = torch.as_tensor(im)
        if t.dtype != torch.uint8 or tuple(t.shape) != tuple(shape):
            raise ValueError(f"image {q}: expected uint8 {tuple(shape)}, got "
                             f"{t.dtype} {tuple(t.shape)}")
        buf[off:off + t.numel()].copy_(t.reshape(-1))
    return buf


class BatchPlan:
    """Static device buffers for images of the given (H, W, channels) shapes,
    palette sizes K and seeds; run() enqueues the path for all of them."""

    def __init__(self, shapes, K, seeds, max_iter: int = 10, eps: float = 0.0,
                 handle: N.Handle | None = None, device=None):
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        Ks = list(K) if isinstance(K, (list, tuple)) else [int(K)] * len(shapes)
        if len(Ks) != len(shapes) or len(seeds) != len(shapes):
            raise ValueError("one K and one seed per image")
        self.n_items = len(shapes)
        self.max_iter, self.eps = int(max_iter), float(eps)
        biggest = max(int(h) * int(w) for h, w, _ in shapes)
        self.handle = handle if handle is not None else N.Handle(max(Ks), biggest, biggest)
        N.wsm_reserve_batch(self.handle, self.n_items)
        dev = self.device
        self.shapes = [(int(h), int(w), int(c)) for h, w, c in shapes]
        lab = N.label_dtype(self.handle)       # uint8, or int16 for a wide handle
        self._rgb_off, rgb_total = _offsets(h * w * c for h, w, c in self.shapes)
        self._idx_off, idx_total = _offsets(h * w * lab.itemsize for h, w, _ in self.shapes)
        self._pal_off, pal_total = _offsets(16 * k for k in Ks)
        self.rgb_all = torch.zeros(rgb_total, dtype=torch.uint8, device=dev)
        self.index_all = torch.zeros(idx_total // lab.itemsize, dtype=lab, device=dev)
        self.centers_all = torch.zeros(pal_total // 4, dtype=torch.float32, device=dev)
        self.images = []
        for q, ((h, w, c), k) in enumerate(zip(self.shapes, Ks)):
            n = h * w
            r0, p0 = self._rgb_off[q], self._pal_off[q] // 4
            i0 = self._idx_off[q] // lab.itemsize
            self.images.append(dict(
                rgb=self.rgb_all[r0:r0 + n * c].view(h, w, c), K=int(k),
                colors=torch.empty(n, dtype=torch.uint32, device=dev),
                counts=torch.empty(n, dtype=torch.uint32, device=dev),
                centers=self.centers_all[p0:p0 + 4 * k].view(k, 4),
                labels=torch.empty(n, dtype=lab, device=dev),
                index=self.index_all[i0:i0 + n].view(h, w)))
        self.n_unique = torch.zeros(self.n_items, dtype=torch.int64, device=dev)
        self.iters = torch.zeros(self.n_items, dtype=torch.int32, device=dev)
        self.mse = torch.zeros(self.n_items, dtype=torch.float64, device=dev)
        self._items = N.pipeline_items(self.images, self.handle.wide)
        self._seeds = N._seeds(list(seeds), self.n_items)
        self.graph = None
        self.graphs = []

    def pack(self, images, pin: bool = True) -> torch.Tensor:
        """A host buffer laid out like the device pixel buffer, holding the
        given images (uint8 [H, W, C] arrays or tensors): load() copies it
        in one transfer."""
        buf = torch.zeros(self.rgb_all.numel(), dtype=torch.uint8)
        if pin:
            buf = buf.pin_memory()
        return _pack_into(buf, self._rgb_off, self.shapes, images)

    def load(self, images, non_blocking: bool = True):
        """Copy new pixels into the static input buffers, on the current
        stream: a buffer from pack() in one copy, or a list of uint8
        [H, W, C] tensors (host or device) one copy each."""
        if isinstance(images, torch.Tensor) and images.dim() == 1:
            self.rgb_all.copy_(images, non_blocking=non_blocking)
            return
        images = list(images)
        if len(images) != self.n_items:
            raise ValueError(f"{len(images)} images for a plan of {self.n_items}")
        for dst, src in zip((im["rgb"] for im in self.images), images):
            dst.copy_(torch.as_tensor(src), non_blocking=non_blocking)

    def host_outputs(self, pin: bool = True) -> dict:
        """Host buffers for fetch(): index images, palettes and MSE of all
        images, laid out like the device buffers."""
        def mk(t):
            h = torch.empty(t.shape, dtype=t.dtype)
            return h.pin_memory() if pin else h
        return dict(index=mk(self.index_all), centers=mk(self.centers_all), mse=mk(self.mse))

    def fetch(self, out: dict, non_blocking: bool = True):
        """Copy the index images, palettes and MSE of all images into the
        buffers of host_outputs(), one copy each, on the current stream;
        image i's parts are at index_offset(i) and palette_offset(i)."""
        out["index"].copy_(self.index_all, non_blocking=non_blocking)
        out["centers"].copy_(self.centers_all, non_blocking=non_blocking)
        out["mse"].copy_(self.mse, non_blocking=non_blocking)

    def index_offset(self, i: int) -> int:
        """Where image i's index image starts in index_all (elements)."""
        return self._idx_off[i] // self.index_all.element_size()

    def palette_offset(self, i: int) -> int:
        """Where image i's palette starts in centers_all (floats)."""
        return self._pal_off[i] // 4

    def run(self, stages: int = N.STAGE_ALL, stream=None):
        """Enqueue unique colors -> init -> iterations -> mapping -> MSE (or
        the given stages, on the state the earlier ones left)."""
        N.wsm_quantize_batch(self.handle, self._items, self.n_items, self._seeds, self.max_iter,
                             self.eps, self.n_unique, self.iters, self.mse, stages=stages,
                             stream=stream)

    def tune(self, repeats: int = 2):
        """Pick the persistent kernel's launch shape on the loaded images."""
        return N.wsm_autotune_batch(self.handle, self._items, self.n_items, self._seeds,
                                    self.max_iter, self.eps, repeats)

    def weigh(self):
        """Weigh the loaded images for the current launch shape (the second
        half of tune(), for a shape fixed with wsm_set_launch_shape)."""
        N.wsm_weigh_batch(self.handle, self._items, self.n_items, self._seeds, self.max_iter,
                          self.eps)

    def stats(self):
        """(distances evaluated, iterations) per image of the last persistent
        launch (after tune(): of the Sort-Means iterations)."""
        return N.wsm_batch_stats(self.handle, self.n_items)

    def capture(self, parts=(N.STAGE_ALL,)):
        """Capture run() into CUDA graphs, one per entry of `parts` (stage
        bits, replayed in that order by replay()), after one eager run."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            for stages in parts:
                self.run(stages)
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        N.wsm_sync_status(self.handle)
        self.graphs = []
        for stages in parts:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.run(stages)
            self.graphs.append(g)
        self.graph = self.graphs[0]
        return self.graphs

    def replay(self, part: int | None = None):
        """Replay the captured graphs in order (or only graph `part`)."""
        if self.graph is None:
            raise RuntimeError("capture() first")
        for g in (self.graphs if part is None else [self.graphs[part]]):
            g.replay()

    def sync(self):
        """Wait for the work and raise any device-side error (e.g. an image
        with fewer unique colors than K)."""
        torch.cuda.synchronize(self.device)
        N.wsm_sync_status(self.handle)

    def result(self, i: int) -> dict:
        """Image i's outputs as device tensors (after sync())."""
        im = self.images[i]
        nu = int(self.n_unique[i])
        return dict(centers=im["centers"], index=im["index"], colors=im["colors"][:nu],
                    counts=im["counts"][:nu], labels=im["labels"][:nu], n_unique=nu,
                    iters=int(self.iters[i]), mse=float(self.mse[i]))
