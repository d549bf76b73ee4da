"""A fixed batch of images through the whole path as one enqueue
(wsm_quantize_batch), optionally tuned (wsm_autotune_batch) and captured
into a CUDA graph, then replayed on new pixels.

Only buffer management and argument marshalling live here; every step of
the path runs in libwsm's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import _native as N


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
        self.images = []
        for (h, w, c), k in zip(shapes, Ks):
            n = int(h) * int(w)
            self.images.append(dict(
                rgb=torch.zeros((h, w, c), dtype=torch.uint8, device=dev), K=int(k),
                colors=torch.empty(n, dtype=torch.uint32, device=dev),
                counts=torch.empty(n, dtype=torch.uint32, device=dev),
                centers=torch.zeros((k, 4), dtype=torch.float32, device=dev),
                labels=torch.empty(n, dtype=torch.uint8, device=dev),
                index=torch.empty((h, w), dtype=torch.uint8, device=dev)))
        self.n_unique = torch.zeros(self.n_items, dtype=torch.int64, device=dev)
        self.iters = torch.zeros(self.n_items, dtype=torch.int32, device=dev)
        self.mse = torch.zeros(self.n_items, dtype=torch.float64, device=dev)
        self._items = N.pipeline_items(self.images)
        self._seeds = N._seeds(list(seeds), self.n_items)
        self.graph = None
        self.graphs = []

    def load(self, images, non_blocking: bool = True):
        """Copy new pixels (uint8 [H, W, C] tensors, host or device) into the
        static input buffers, on the current stream."""
        for dst, src in zip((im["rgb"] for im in self.images), images):
            dst.copy_(torch.as_tensor(src), non_blocking=non_blocking)

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
