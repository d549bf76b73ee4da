"""GB300-native Weighted Sort-Means (WSM) color quantization.

Implements the method of M. E. Celebi, "Fast Color Quantization Using
Weighted Sort-Means Clustering" (arXiv:1011.0093) as hand-written CUDA for
sm_103a behind the C ABI of include/wsm.h (libwsm.so).  This package is the
thin Python layer above it: ``_native`` marshals arguments to the C entry
points; ``quantize`` chains them for one image or a batch; ``batch`` holds a
fixed batch's buffers and captures the whole path into a CUDA graph;
``serve`` queues requests to the native continuous-batching server;
``distortion`` wraps the weighted distortion and its gradients as a
torch.autograd.Function.  PyTorch only provides device memory and streams.
"""
from ._native import (MAX_K, MAX_K_WIDE, MAX_PIXELS, STAGE_ALL, STAGE_DISTORTION, STAGE_INDEX,
                      STAGE_INIT, STAGE_ITERATE, STAGE_MAP, STAGE_REDUCE, Handle, WsmError,
                      label_dtype, lib,
                      pipeline_items, wsm_autotune_batch, wsm_batch_stats, wsm_distortion,
                      wsm_distortion_batch, wsm_distortion_bwd, wsm_distortion_fwd, wsm_init,
                      wsm_init_batch, wsm_iterate, wsm_iterate_batch, wsm_iterate_noalloc,
                      wsm_iterate_stats, wsm_launch_shape, wsm_map, wsm_map_batch,
                      wsm_quantize_batch, wsm_reduce, wsm_reduce_batch, wsm_reserve_batch,
                      wsm_measure_fp32, wsm_round_palette,
                      wsm_set_first_pass_start, wsm_set_grid_limit, wsm_set_launch_shape,
                      wsm_set_reduce_path, wsm_weigh_batch,
                      wsm_sync_status)
from .batch import BatchPlan
from .serve import Server
from .distortion import WeightedDistortion, weighted_distortion
from .quantize import Quantized, quantize, quantize_batch

__all__ = [
    "MAX_K", "MAX_K_WIDE", "MAX_PIXELS", "Handle", "WsmError", "label_dtype", "lib",
    # one image, step by step
    "wsm_reduce", "wsm_init", "wsm_iterate", "wsm_iterate_stats", "wsm_iterate_noalloc",
    "wsm_map", "wsm_distortion", "wsm_round_palette", "wsm_sync_status", "Quantized",
    "quantize",
    # batches of images
    "wsm_reserve_batch", "wsm_reduce_batch", "wsm_init_batch", "wsm_iterate_batch",
    "wsm_map_batch", "wsm_distortion_batch", "quantize_batch",
    # the whole path with N' on the device, graphs, launch shapes, autotuner
    "wsm_quantize_batch", "pipeline_items", "STAGE_REDUCE", "STAGE_INIT", "STAGE_ITERATE",
    "STAGE_MAP", "STAGE_INDEX", "STAGE_DISTORTION", "STAGE_ALL", "wsm_autotune_batch",
    "wsm_launch_shape", "wsm_set_launch_shape", "wsm_set_grid_limit", "wsm_set_first_pass_start",
    "wsm_set_reduce_path", "wsm_weigh_batch",
    "wsm_batch_stats", "BatchPlan", "wsm_measure_fp32",
    # serving
    "Server",
    # differentiable distortion
    "wsm_distortion_fwd", "wsm_distortion_bwd", "WeightedDistortion", "weighted_distortion",
]
