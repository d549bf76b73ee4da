"""The weighted distortion D(C, X) = sum_i w_i min_k ||x_i - c_k||^2 (Eq. 1
with the sample weights of Sec. 2) as a torch.autograd.Function over the
library's forward and backward kernels (wsm_distortion_fwd / _bwd).

Only argument marshalling lives here: the nearest-center search, the sums and
both gradients run in libwsm's CUDA kernels.
"""
from __future__ import annotations

import threading

import torch

from . import _native as N

_handles: dict[int, N.Handle] = {}
_handles_lock = threading.Lock()


def _default_handle(device: torch.device) -> N.Handle:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    with _handles_lock:
        h = _handles.get(idx)
        if h is None:
            with torch.cuda.device(idx):
                h = N.Handle(N.MAX_K, 1, 1)
            _handles[idx] = h
        return h


class WeightedDistortion(torch.autograd.Function):
    """D(C, X); gradients dD/dC = -2 sum_{m_i=k} w_i (x_i - c_k) and
    dD/dX = 2 w_i (x_i - c_{m_i}), valid away from ties."""

    @staticmethod
    def forward(ctx, x, centers, w, assign, warm_start, handle):
        x = x.detach().contiguous()
        c = centers.detach().contiguous()
        wd = w.detach().contiguous() if w is not None else None
        K = c.shape[0]
        D = torch.empty(1, dtype=torch.float32, device=x.device)
        resid = torch.empty((K, 4), dtype=torch.float32, device=x.device)
        N.wsm_distortion_fwd(handle, x, wd, c, assign, warm_start, D, resid)
        ctx.save_for_backward(x, c, assign, resid)
        ctx.w = wd
        ctx.handle = handle
        return D[0]

    @staticmethod
    def backward(ctx, gD):
        x, c, assign, resid = ctx.saved_tensors
        g = gD.detach().reshape(1).to(torch.float32).contiguous()
        gC = torch.empty_like(c) if ctx.needs_input_grad[1] else None
        gX = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        N.wsm_distortion_bwd(ctx.handle, x, ctx.w, c, assign, resid, g, gC, gX)
        return gX, gC, None, None, None, None


def weighted_distortion(x: torch.Tensor, centers: torch.Tensor, w: torch.Tensor | None = None,
                        assign: torch.Tensor | None = None, warm_start: bool = False,
                        handle: N.Handle | None = None) -> torch.Tensor:
    """D(C, X) for float32 CUDA x [n, 3|4] and centers [K, 3|4] (K <= 256),
    with weights w [n] (None: w_i = 1/n).  Differentiable in x and centers.

    assign (uint8 [n], optional) receives each point's nearest center; with
    warm_start=True its contents are where each search starts, so passing
    the previous call's assignment makes a slowly moving palette cheap.
    """
    if not (x.is_cuda and centers.is_cuda):
        raise ValueError("x and centers must be CUDA tensors")
    if x.dtype != torch.float32 or centers.dtype != torch.float32:
        raise ValueError("x and centers must be float32")
    if assign is None:
        if warm_start:
            raise ValueError("warm_start needs an assignment tensor")
        assign = torch.empty(x.shape[0], dtype=torch.uint8, device=x.device)
    h = handle if handle is not None else _default_handle(x.device)
    return WeightedDistortion.apply(x, centers, w, assign, warm_start, h)
