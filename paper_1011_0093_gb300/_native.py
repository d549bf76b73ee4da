"""ctypes binding of libwsm (include/wsm.h): argument marshalling only.

Every function here has the name of the C entry point it calls, checks the
tensors it is given (device, dtype, contiguity, size), passes their device
pointers and the current CUDA stream, and turns a non-zero status into a
WsmError.  All computation happens in the library's CUDA kernels; there is
no other code path.  If libwsm.so has not been built, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwsm.so")

WSM_OK = 0
ERRORS = {-1: "WSM_E_INVAL", -2: "WSM_E_NOMEM", -3: "WSM_E_CUDA", -4: "WSM_E_TIMEOUT",
          -5: "WSM_E_STATE", -6: "WSM_E_CAPACITY"}
MAX_K = 256          # palettes with 8-bit memberships
MAX_K_WIDE = 1024    # palettes of a wide handle (16-bit memberships)
MAX_PIXELS = 1 << 24

_lock = threading.Lock()
_lib = None
_P = C.c_void_p
_I64 = C.c_int64

class WsmItem(C.Structure):
    """wsm_item of include/wsm.h: one image of a batch call."""
    _fields_ = [("d_rgb", C.c_void_p), ("n_pixels", C.c_int64), ("pixel_stride", C.c_int),
                ("K", C.c_int), ("d_colors", C.c_void_p), ("d_counts", C.c_void_p),
                ("n_unique", C.c_int64), ("d_centers", C.c_void_p), ("d_labels", C.c_void_p),
                ("d_index", C.c_void_p)]


class ServerConfig(C.Structure):
    """wsm_server_config of include/wsm.h."""
    _fields_ = [("max_K", C.c_int), ("max_pixels", C.c_int64), ("lanes", C.c_int),
                ("slots_per_lane", C.c_int), ("arena_bytes", C.c_int64)]


class Request(C.Structure):
    """wsm_request of include/wsm.h."""
    _fields_ = [("rgb", C.c_void_p), ("n_pixels", C.c_int64), ("pixel_stride", C.c_int),
                ("K", C.c_int), ("seed", C.c_uint64), ("max_iter", C.c_int),
                ("eps", C.c_double), ("index_out", C.c_void_p), ("palette_out", C.c_void_p)]


class Result(C.Structure):
    """wsm_result of include/wsm.h."""
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("n_unique", C.c_int64),
                ("mse", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


class ServerStats(C.Structure):
    """wsm_server_stats of include/wsm.h."""
    _fields_ = [(name, C.c_int64) for name in
                ("submitted", "completed", "failed", "batches", "in_flight", "max_in_flight",
                 "queued", "arena_bytes", "arena_used", "arena_peak")]


SIGNATURES = {
    "wsm_last_error": (C.c_char_p, []),
    "wsm_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _I64, _I64]),
    "wsm_destroy": (C.c_int, [_P]),
    "wsm_sync_status": (C.c_int, [_P, _P]),
    "wsm_reduce": (C.c_int, [_P, _P, _I64, C.c_int, _P, _P, _I64, _P, C.POINTER(_I64), _P]),
    "wsm_init": (C.c_int, [_P, _P, _I64, C.c_int, C.c_uint64, _P, _P, _P]),
    "wsm_iterate": (C.c_int, [_P, _P, _P, _I64, C.c_int, _P, _P, C.c_int, C.c_double,
                              C.POINTER(C.c_int), _P, _P]),
    "wsm_iterate_stats": (C.c_int, [_P, C.c_int, C.POINTER(_I64), _P, _P, _P]),
    "wsm_iterate_noalloc": (C.c_int, [_P, _P, _I64, C.c_int, _P, _P, C.c_int, C.c_double,
                                      C.POINTER(C.c_int), _P, _P]),
    "wsm_map": (C.c_int, [_P, _P, _I64, C.c_int, _P, _I64, _P, C.c_int, _P, _P, _P]),
    "wsm_reserve_batch": (C.c_int, [_P, C.c_int]),
    "wsm_iterate_batch": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_double, _P, _P]),
    "wsm_map_batch": (C.c_int, [_P, _P, C.c_int, _P]),
    "wsm_reduce_batch": (C.c_int, [_P, _P, C.c_int, _P]),
    "wsm_init_batch": (C.c_int, [_P, _P, C.c_int, _P, _P]),
    "wsm_distortion_batch": (C.c_int, [_P, _P, C.c_int, _P, _P, _P]),
    "wsm_quantize_batch": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_double, _P, _P, _P, _P]),
    "wsm_quantize_batch_stages": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_double, _P, _P, _P,
                                            C.c_uint, _P]),
    "wsm_launch_shape": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]),
    "wsm_set_launch_shape": (C.c_int, [_P, C.c_int]),
    "wsm_batch_stats": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "wsm_selftest_barrier_timeout": (C.c_int, [_P, C.c_int, _P]),
    "wsm_set_grid_limit": (C.c_int, [_P, C.c_int]),
    "wsm_set_first_pass_start": (C.c_int, [_P, C.c_int]),
    "wsm_set_reduce_path": (C.c_int, [_P, C.c_int]),
    "wsm_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(ServerConfig)]),
    "wsm_server_submit": (C.c_int, [_P, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "wsm_server_wait": (C.c_int, [_P, C.c_uint64, C.c_double, C.POINTER(Result)]),
    "wsm_server_stats_get": (C.c_int, [_P, C.POINTER(ServerStats)]),
    "wsm_server_destroy": (C.c_int, [_P]),
    "wsm_autotune_batch": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_double, C.c_int, _P, _P]),
    "wsm_weigh_batch": (C.c_int, [_P, _P, C.c_int, _P, C.c_int, C.c_double, _P]),
    "wsm_distortion_fwd": (C.c_int, [_P, _P, C.c_int, _P, _I64, _P, C.c_int, C.c_int, _P,
                                     C.c_int, _P, _P, _P]),
    "wsm_distortion_bwd": (C.c_int, [_P, _P, C.c_int, _P, _I64, _P, C.c_int, C.c_int, _P, _P,
                                     _P, _P, _P, _P]),
    "wsm_distortion": (C.c_int, [_P, _P, _I64, C.c_int, _P, C.c_int, _P, _P,
                                 C.POINTER(C.c_double), _P]),
    "wsm_round_palette": (C.c_int, [_P, _P, C.c_int, _P, _P, _P]),
    "wsm_measure_fp32": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), _P]),
}


class WsmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """The loaded libwsm (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libwsm.so not found at {LIB_PATH}: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            so = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(so, name)
                f.restype = res
                f.argtypes = args
            _lib = so
    return _lib


def _check_index(rc: int) -> int:
    """For calls that return an index >= 0 or a negative error code."""
    if rc < 0:
        _check(rc)
    return rc


def _check(rc: int):
    if rc != WSM_OK:
        raise WsmError(rc, lib().wsm_last_error().decode(errors="replace"))


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _dev(t: torch.Tensor | None, dtype, name: str, min_numel: int = 0) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < min_numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {min_numel}")
    return t.data_ptr()


def label_dtype(h) -> torch.dtype:
    """The dtype of memberships and index images for handle h: uint8, or for
    a wide handle (max_K > 256) int16, whose bits the library reads as
    uint16 (palette indices stay below 1024)."""
    return torch.int16 if int(h.max_K) > MAX_K else torch.uint8


def _lab(t: torch.Tensor | None, wide: bool, name: str, min_numel: int = 0) -> int | None:
    """A membership or index array: uint8, or for a wide handle int16/uint16."""
    if t is None:
        return None
    ok = (torch.int16, getattr(torch, "uint16", torch.int16)) if wide else (torch.uint8,)
    if t.dtype not in ok:
        raise ValueError(f"{name} must be {ok[0]} for this handle, got {t.dtype}")
    return _dev(t, t.dtype, name, min_numel)


def _pixels(rgb: torch.Tensor) -> tuple[int, int]:
    stride = rgb.shape[-1]
    if stride not in (3, 4):
        raise ValueError("pixels must have 3 or 4 channels in the last dimension")
    return rgb.numel() // stride, stride


class Handle:
    """Owns a wsm_handle (library scratch on the current device)."""

    def __init__(self, max_K: int, max_pixels: int, max_unique: int | None = None):
        h = C.c_void_p()
        _check(lib().wsm_create(C.byref(h), int(max_K), int(max_pixels),
                                int(max_unique if max_unique is not None else max_pixels)))
        self.ptr = h.value
        self.max_K = int(max_K)
        self.wide = self.max_K > MAX_K      # 16-bit memberships and index images
        self.max_pixels = int(max_pixels)
        self.max_unique = int(max_unique if max_unique is not None else max_pixels)

    def close(self):
        if self.ptr:
            lib().wsm_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def wsm_sync_status(h: Handle, stream=None):
    _check(lib().wsm_sync_status(h.ptr, _stream(stream)))


def wsm_reduce(h: Handle, rgb: torch.Tensor, colors: torch.Tensor, counts: torch.Tensor,
               d_n_unique: torch.Tensor | None = None, sync: bool = True, stream=None):
    """Unique colors + counts; returns N' (host int) if sync, else None."""
    n, stride = _pixels(rgb)
    cap = min(colors.numel(), counts.numel())
    nu = _I64(0)
    _check(lib().wsm_reduce(h.ptr, _dev(rgb, torch.uint8, "rgb"), n, stride,
                            _dev(colors, torch.uint32, "colors"),
                            _dev(counts, torch.uint32, "counts"), cap,
                            _dev(d_n_unique, torch.int64, "d_n_unique", 1),
                            C.byref(nu) if sync else None, _stream(stream)))
    return int(nu.value) if sync else None


def wsm_init(h: Handle, colors: torch.Tensor, n_unique: int, K: int, seed: int,
             centers: torch.Tensor, labels: torch.Tensor, stream=None):
    _check(lib().wsm_init(h.ptr, _dev(colors, torch.uint32, "colors", n_unique), n_unique, K,
                          seed & (2 ** 64 - 1), _dev(centers, torch.float32, "centers", 4 * K),
                          _lab(labels, h.wide, "labels", n_unique), _stream(stream)))


def wsm_iterate(h: Handle, colors: torch.Tensor, counts: torch.Tensor, n_unique: int, K: int,
                centers: torch.Tensor, labels: torch.Tensor, max_iter: int, eps: float,
                sync: bool = True, stream=None):
    """Returns (iterations done, SSE trace list) if sync, else None."""
    it = C.c_int(0)
    trace = (C.c_double * max(max_iter, 1))()
    _check(lib().wsm_iterate(h.ptr, _dev(colors, torch.uint32, "colors", n_unique),
                             _dev(counts, torch.uint32, "counts", n_unique), n_unique, K,
                             _dev(centers, torch.float32, "centers", 4 * K),
                             _lab(labels, h.wide, "labels", n_unique), max_iter, float(eps),
                             C.byref(it) if sync else None,
                             C.cast(trace, C.c_void_p) if sync else None, _stream(stream)))
    if not sync:
        return None
    return it.value, [trace[i] for i in range(min(it.value, max_iter))]


def wsm_iterate_noalloc(colors: torch.Tensor, counts: torch.Tensor, n_unique: int, K: int,
                        centers: torch.Tensor, labels: torch.Tensor, max_iter: int, eps: float,
                        sync: bool = True, stream=None):
    """wsm_iterate without a handle and without any device allocation, for
    callers that cannot allocate (see include/wsm.h).  Same arguments and
    results as wsm_iterate; calls that overlap on the GPU race."""
    it = C.c_int(0)
    trace = (C.c_double * max(max_iter, 1))()
    _check(lib().wsm_iterate_noalloc(_dev(colors, torch.uint32, "colors", n_unique),
                                     _dev(counts, torch.uint32, "counts", n_unique), n_unique, K,
                                     _dev(centers, torch.float32, "centers", 4 * K),
                                     _dev(labels, torch.uint8, "labels", n_unique), max_iter,
                                     float(eps), C.byref(it) if sync else None,
                                     C.cast(trace, C.c_void_p) if sync else None,
                                     _stream(stream)))
    if not sync:
        return None
    return it.value, [trace[i] for i in range(min(it.value, max_iter))]


def wsm_iterate_stats(h: Handle, K: int, sums: bool = True, stream=None):
    """(evaluated distances, S [K,3] int64 or None, W [K] int64 or None)."""
    ev = _I64(0)
    S = (_I64 * (3 * K))()
    W = (_I64 * K)()
    _check(lib().wsm_iterate_stats(h.ptr, K, C.byref(ev), C.cast(S, C.c_void_p) if sums else None,
                                   C.cast(W, C.c_void_p) if sums else None, _stream(stream)))
    if not sums:
        return ev.value, None, None
    return (ev.value, torch.tensor(list(S), dtype=torch.int64).view(K, 3),
            torch.tensor(list(W), dtype=torch.int64))


def wsm_map(h: Handle, rgb: torch.Tensor, colors: torch.Tensor, n_unique: int,
            centers: torch.Tensor, K: int, labels: torch.Tensor, index: torch.Tensor,
            stream=None):
    n, stride = _pixels(rgb)
    _check(lib().wsm_map(h.ptr, _dev(rgb, torch.uint8, "rgb"), n, stride,
                         _dev(colors, torch.uint32, "colors", n_unique), n_unique,
                         _dev(centers, torch.float32, "centers", 4 * K), K,
                         _lab(labels, h.wide, "labels", n_unique),
                         _lab(index, h.wide, "index", n), _stream(stream)))


def wsm_reserve_batch(h: Handle, max_items: int):
    _check(lib().wsm_reserve_batch(h.ptr, int(max_items)))


def _items(images: list[dict], need_pixels: bool, need_counts: bool, wide: bool = False):
    """Marshal dicts with tensors (rgb, colors, counts, n_unique, K, centers,
    labels, index) into a wsm_item array."""
    arr = (WsmItem * max(len(images), 1))()
    for q, im in enumerate(images):
        K, nu = int(im["K"]), int(im["n_unique"])
        it = arr[q]
        it.K = K
        it.n_unique = nu
        it.d_colors = _dev(im["colors"], torch.uint32, "colors", nu)
        it.d_centers = _dev(im["centers"], torch.float32, "centers", 4 * K)
        it.d_labels = _lab(im["labels"], wide, "labels", nu)
        if need_counts:
            it.d_counts = _dev(im["counts"], torch.uint32, "counts", nu)
        if need_pixels:
            n, stride = _pixels(im["rgb"])
            it.d_rgb = _dev(im["rgb"], torch.uint8, "rgb")
            it.n_pixels = n
            it.pixel_stride = stride
            it.d_index = _lab(im["index"], wide, "index", n)
    return arr


def wsm_iterate_batch(h: Handle, images: list[dict], max_iter: int, eps: float,
                      sync: bool = True, stream=None):
    """Iterate every image of the batch; returns the iteration counts if sync."""
    arr = _items(images, False, True, h.wide)
    done = (C.c_int * max(len(images), 1))()
    _check(lib().wsm_iterate_batch(h.ptr, C.cast(arr, C.c_void_p), len(images), max_iter,
                                   float(eps), C.cast(done, C.c_void_p) if sync else None,
                                   _stream(stream)))
    return [done[i] for i in range(len(images))] if sync else None


def wsm_map_batch(h: Handle, images: list[dict], stream=None):
    arr = _items(images, True, False, h.wide)
    _check(lib().wsm_map_batch(h.ptr, C.cast(arr, C.c_void_p), len(images), _stream(stream)))


def wsm_reduce_batch(h: Handle, images: list[dict], stream=None) -> list[int]:
    """Unique colors of every image (dicts with rgb, colors, counts; colors and
    counts hold n_pixels entries); sets each dict's n_unique and returns them."""
    arr = (WsmItem * max(len(images), 1))()
    for q, im in enumerate(images):
        n, stride = _pixels(im["rgb"])
        it = arr[q]
        it.d_rgb = _dev(im["rgb"], torch.uint8, "rgb")
        it.n_pixels = n
        it.pixel_stride = stride
        it.d_colors = _dev(im["colors"], torch.uint32, "colors", n)
        it.d_counts = _dev(im["counts"], torch.uint32, "counts", n)
    _check(lib().wsm_reduce_batch(h.ptr, C.cast(arr, C.c_void_p), len(images), _stream(stream)))
    out = [int(arr[q].n_unique) for q in range(len(images))]
    for im, nu in zip(images, out):
        im["n_unique"] = nu
    return out


def wsm_init_batch(h: Handle, images: list[dict], seeds: list[int], stream=None):
    """Initial centers and labels of every image (dicts with colors, n_unique,
    K, centers, labels)."""
    arr = (WsmItem * max(len(images), 1))()
    for q, im in enumerate(images):
        K, nu = int(im["K"]), int(im["n_unique"])
        it = arr[q]
        it.K = K
        it.n_unique = nu
        it.d_colors = _dev(im["colors"], torch.uint32, "colors", nu)
        it.d_centers = _dev(im["centers"], torch.float32, "centers", 4 * K)
        it.d_labels = _lab(im["labels"], h.wide, "labels", nu)
    if len(seeds) != len(images):
        raise ValueError("one seed per image")
    sd = (C.c_uint64 * max(len(images), 1))(*[int(x) & (2**64 - 1) for x in seeds])
    _check(lib().wsm_init_batch(h.ptr, C.cast(arr, C.c_void_p), len(images),
                                C.cast(sd, C.c_void_p), _stream(stream)))


def wsm_distortion_batch(h: Handle, images: list[dict], d_mse: torch.Tensor | None = None,
                         sync: bool = True, stream=None):
    """MSE of Eq. 2 of every image (dicts with rgb, K, centers, index); returns
    the host floats if sync, else None."""
    arr = (WsmItem * max(len(images), 1))()
    for q, im in enumerate(images):
        n, stride = _pixels(im["rgb"])
        K = int(im["K"])
        it = arr[q]
        it.d_rgb = _dev(im["rgb"], torch.uint8, "rgb")
        it.n_pixels = n
        it.pixel_stride = stride
        it.K = K
        it.d_centers = _dev(im["centers"], torch.float32, "centers", 4 * K)
        it.d_index = _lab(im["index"], h.wide, "index", n)
    m = (C.c_double * max(len(images), 1))()
    _check(lib().wsm_distortion_batch(h.ptr, C.cast(arr, C.c_void_p), len(images),
                                      _dev(d_mse, torch.float64, "d_mse", len(images)),
                                      C.cast(m, C.c_void_p) if sync else None,
                                      _stream(stream)))
    return [m[q] for q in range(len(images))] if sync else None


def wsm_distortion(h: Handle, rgb: torch.Tensor, centers: torch.Tensor, K: int,
                   index: torch.Tensor, d_mse: torch.Tensor | None = None, sync: bool = True,
                   stream=None):
    """MSE of Eq. 2; returns the host float if sync, else None."""
    n, stride = _pixels(rgb)
    m = C.c_double(0.0)
    _check(lib().wsm_distortion(h.ptr, _dev(rgb, torch.uint8, "rgb"), n, stride,
                                _dev(centers, torch.float32, "centers", 4 * K), K,
                                _lab(index, h.wide, "index", n),
                                _dev(d_mse, torch.float64, "d_mse", 1),
                                C.byref(m) if sync else None, _stream(stream)))
    return m.value if sync else None


def wsm_measure_fp32(h: Handle, repeats: int = 3, stream=None) -> float:
    """Measured FP32 TFLOP/s of this GPU (independent FMA chains)."""
    v = C.c_double(0.0)
    _check(lib().wsm_measure_fp32(h.ptr, int(repeats), C.byref(v), _stream(stream)))
    return v.value


def wsm_round_palette(h: Handle, centers: torch.Tensor, K: int, stream=None):
    """The palette as 8-bit colors (ties to even, clamped): (uint8 [K, 4],
    float32 [K, 4] of the same values, for wsm_distortion)."""
    pal = torch.empty((K, 4), dtype=torch.uint8, device=centers.device)
    rounded = torch.empty((K, 4), dtype=torch.float32, device=centers.device)
    _check(lib().wsm_round_palette(h.ptr, _dev(centers, torch.float32, "centers", 4 * K), K,
                                   _dev(pal, torch.uint8, "palette", 4 * K),
                                   _dev(rounded, torch.float32, "rounded", 4 * K),
                                   _stream(stream)))
    return pal, rounded


def _points(t: torch.Tensor, name: str) -> tuple[int, int]:
    if t.dim() != 2 or t.shape[1] not in (3, 4):
        raise ValueError(f"{name} must be float32 [n, 3|4]")
    return t.shape[0], t.shape[1]


def wsm_distortion_fwd(h: Handle, x: torch.Tensor, w: torch.Tensor | None, centers: torch.Tensor,
                       assign: torch.Tensor, warm_start: bool, D: torch.Tensor,
                       resid: torch.Tensor, stream=None):
    """Forward pass of the weighted distortion: fills D [1], resid [K, 4] and assign [n]."""
    n, xs = _points(x, "x")
    K, cs = _points(centers, "centers")
    _check(lib().wsm_distortion_fwd(h.ptr, _dev(x, torch.float32, "x"), xs,
                                    _dev(w, torch.float32, "w", n), n,
                                    _dev(centers, torch.float32, "centers"), cs, K,
                                    _dev(assign, torch.uint8, "assign", n), int(bool(warm_start)),
                                    _dev(D, torch.float32, "D", 1),
                                    _dev(resid, torch.float32, "resid", 4 * K), _stream(stream)))


def wsm_distortion_bwd(h: Handle, x: torch.Tensor, w: torch.Tensor | None, centers: torch.Tensor,
                       assign: torch.Tensor, resid: torch.Tensor, gD: torch.Tensor,
                       gC: torch.Tensor | None, gX: torch.Tensor | None, stream=None):
    """Backward pass: fills gC [K, 3|4] and gX [n, 3|4] (either may be None)."""
    n, xs = _points(x, "x")
    K, cs = _points(centers, "centers")
    if gC is not None and tuple(gC.shape) != (K, cs):
        raise ValueError("gC must have the shape of centers")
    if gX is not None and tuple(gX.shape) != (n, xs):
        raise ValueError("gX must have the shape of x")
    _check(lib().wsm_distortion_bwd(h.ptr, _dev(x, torch.float32, "x"), xs,
                                    _dev(w, torch.float32, "w", n), n,
                                    _dev(centers, torch.float32, "centers"), cs, K,
                                    _dev(assign, torch.uint8, "assign", n),
                                    _dev(resid, torch.float32, "resid", 4 * K),
                                    _dev(gD, torch.float32, "gD", 1),
                                    _dev(gC, torch.float32, "gC"), _dev(gX, torch.float32, "gX"),
                                    _stream(stream)))


N_SHAPES = 5


def pipeline_items(images: list[dict], wide: bool = False):
    """Marshal dicts with rgb, K, colors, counts, centers, labels, index (device
    buffers of wsm_quantize_batch) into a wsm_item array; the array keeps the
    pointers, so it can be reused for as long as the tensors live."""
    arr = (WsmItem * max(len(images), 1))()
    for q, im in enumerate(images):
        n, stride = _pixels(im["rgb"])
        K = int(im["K"])
        it = arr[q]
        it.d_rgb = _dev(im["rgb"], torch.uint8, "rgb")
        it.n_pixels = n
        it.pixel_stride = stride
        it.K = K
        it.d_colors = _dev(im["colors"], torch.uint32, "colors", n)
        it.d_counts = _dev(im["counts"], torch.uint32, "counts", n)
        it.n_unique = 0
        it.d_centers = _dev(im["centers"], torch.float32, "centers", 4 * K)
        it.d_labels = _lab(im["labels"], wide, "labels", n)
        it.d_index = _lab(im["index"], wide, "index", n)
    return arr


def _seeds(seeds, n):
    if len(seeds) != n:
        raise ValueError("one seed per image")
    return (C.c_uint64 * max(n, 1))(*[int(x) & (2**64 - 1) for x in seeds])


STAGE_REDUCE, STAGE_INIT, STAGE_ITERATE, STAGE_MAP, STAGE_DISTORTION = 1, 2, 4, 8, 16
STAGE_INDEX = 32
STAGE_ALL = 63


def wsm_quantize_batch(h: Handle, items, n_items: int, seeds, max_iter: int, eps: float,
                       d_n_unique: torch.Tensor | None = None, d_iters: torch.Tensor | None = None,
                       d_mse: torch.Tensor | None = None, stages: int = STAGE_ALL, stream=None):
    """Enqueue the path (or the given stages of it) for a batch (items: a
    pipeline_items array); nothing is synchronised, so a CUDA graph can
    capture it."""
    sd = seeds if isinstance(seeds, C.Array) else _seeds(seeds, n_items)
    _check(lib().wsm_quantize_batch_stages(h.ptr, C.cast(items, C.c_void_p), n_items,
                                           C.cast(sd, C.c_void_p), int(max_iter), float(eps),
                                           _dev(d_n_unique, torch.int64, "d_n_unique", n_items),
                                           _dev(d_iters, torch.int32, "d_iters", n_items),
                                           _dev(d_mse, torch.float64, "d_mse", n_items),
                                           int(stages), _stream(stream)))


def wsm_launch_shape(h: Handle, shape: int = -1) -> tuple[int, int, int, bool]:
    """(shape, threads per block, blocks per SM, resident) of a launch shape."""
    t, b, r = C.c_int(0), C.c_int(0), C.c_int(0)
    q = _check_index(lib().wsm_launch_shape(h.ptr, int(shape), C.byref(t), C.byref(b),
                                            C.byref(r)))
    return q, t.value, b.value, bool(r.value)


def wsm_set_launch_shape(h: Handle, shape: int):
    _check(lib().wsm_set_launch_shape(h.ptr, int(shape)))


def wsm_autotune_batch(h: Handle, items, n_items: int, seeds, max_iter: int, eps: float,
                       repeats: int = 2, stream=None) -> tuple[int, list[float]]:
    """Time every resident launch shape on the batch; keeps and returns the
    fastest, with each shape's best time in ms (-1: not resident)."""
    sd = seeds if isinstance(seeds, C.Array) else _seeds(seeds, n_items)
    times = (C.c_float * N_SHAPES)()
    q = _check_index(lib().wsm_autotune_batch(h.ptr, C.cast(items, C.c_void_p), n_items,
                                              C.cast(sd, C.c_void_p), int(max_iter), float(eps),
                                              int(repeats), C.cast(times, C.c_void_p),
                                              _stream(stream)))
    return q, [times[i] for i in range(N_SHAPES)]


def wsm_weigh_batch(h: Handle, items, n_items: int, seeds, max_iter: int, eps: float,
                    stream=None) -> None:
    """Set the images' work weights for the handle's current launch shape."""
    sd = seeds if isinstance(seeds, C.Array) else _seeds(seeds, n_items)
    _check(lib().wsm_weigh_batch(h.ptr, C.cast(items, C.c_void_p), n_items,
                                 C.cast(sd, C.c_void_p), int(max_iter), float(eps),
                                 _stream(stream)))


def wsm_batch_stats(h: Handle, n_items: int, stream=None) -> tuple[list[int], list[int]]:
    """(distances evaluated, iterations) of the last persistent launch per slot."""
    ev = (C.c_int64 * max(n_items, 1))()
    it = (C.c_int * max(n_items, 1))()
    _check(lib().wsm_batch_stats(h.ptr, int(n_items), C.cast(ev, C.c_void_p),
                                 C.cast(it, C.c_void_p), _stream(stream)))
    return [ev[i] for i in range(n_items)], [it[i] for i in range(n_items)]


def wsm_set_grid_limit(h: Handle, blocks: int):
    _check(lib().wsm_set_grid_limit(h.ptr, int(blocks)))


def wsm_set_first_pass_start(h: Handle, candidate: bool):
    _check(lib().wsm_set_first_pass_start(h.ptr, int(bool(candidate))))


def wsm_set_reduce_path(h: Handle, path: int):
    """0: by size (default), 1: direct histogram, 2: bucketed (include/wsm.h)."""
    _check(lib().wsm_set_reduce_path(h.ptr, int(path)))
