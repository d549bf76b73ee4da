"""A quantization server over the library's native scheduler (wsm_server_*
in include/wsm.h): requests are queued from any thread, admitted into
lanes by device-memory footprint, batched, and run while other lanes'
batches are on the GPU.

Only argument marshalling lives here.  Inputs and outputs are page-locked
host tensors, so the lanes' copies overlap with the device work.
"""
from __future__ import annotations

import ctypes as C
import threading

import torch

from . import _native as N


class Pending:
    """A submitted request: its id, its page-locked outputs, and the input it
    keeps alive until the result is collected."""

    def __init__(self, rid: int, rgb: torch.Tensor, index: torch.Tensor, palette: torch.Tensor):
        self.id, self.rgb, self.index, self.palette = rid, rgb, index, palette


class Server:
    def __init__(self, max_K: int = N.MAX_K, max_pixels: int = N.MAX_PIXELS, lanes: int = 2,
                 slots_per_lane: int = 16, arena_bytes: int = 8 << 30):
        cfg = N.ServerConfig(int(max_K), int(max_pixels), int(lanes), int(slots_per_lane),
                             int(arena_bytes))
        ptr = C.c_void_p()
        N._check(N.lib().wsm_server_create(C.byref(ptr), C.byref(cfg)))
        self.ptr = ptr
        self._lock = threading.Lock()

    def submit(self, rgb: torch.Tensor, K: int, seed: int, max_iter: int = 10,
               eps: float = 0.0) -> Pending:
        """Queue one uint8 [H, W, 3|4] host image (page-locked for overlap)."""
        if rgb.is_cuda or rgb.dtype != torch.uint8 or rgb.dim() != 3 or not rgb.is_contiguous():
            raise ValueError("rgb must be a contiguous uint8 host tensor [H, W, 3|4]")
        H, W, stride = rgb.shape
        index = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
        palette = torch.empty((K, 4), dtype=torch.float32, pin_memory=True)
        r = N.Request(rgb.data_ptr(), H * W, stride, int(K), int(seed) & (2**64 - 1),
                      int(max_iter), float(eps), index.data_ptr(), palette.data_ptr())
        rid = C.c_uint64(0)
        N._check(N.lib().wsm_server_submit(self.ptr, C.byref(r), C.byref(rid)))
        return Pending(rid.value, rgb, index, palette)

    def wait(self, p: Pending, timeout: float | None = None) -> dict:
        """Block until the request is done; its results, times in seconds."""
        res = N.Result()
        rc = N.lib().wsm_server_wait(self.ptr, p.id, -1.0 if timeout is None else float(timeout),
                                     C.byref(res))
        N._check(rc)
        return dict(index=p.index, palette=p.palette, n_unique=res.n_unique, iters=res.iters,
                    mse=res.mse, t_submit=res.t_submit, t_admit=res.t_admit, t_done=res.t_done,
                    latency=res.t_done - res.t_submit)

    def stats(self) -> dict:
        st = N.ServerStats()
        N._check(N.lib().wsm_server_stats_get(self.ptr, C.byref(st)))
        return {name: getattr(st, name) for name, _ in N.ServerStats._fields_}

    def close(self):
        with self._lock:
            if self.ptr:
                N.lib().wsm_server_destroy(self.ptr)
                self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
