"""Python access to the plain FP64 CPU oracle of Weighted Sort-Means.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The oracle
(``wsm_oracle.c``) is compiled with the host C compiler into
``oracle/libwsm_oracle.so`` on first use; it shares nothing with the CUDA
library.  Every wrapper below names the part of the paper (Celebi,
arXiv:1011.0093) that the C function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wsm_oracle.c")
_LIB = os.path.join(_HERE, "libwsm_oracle.so")
_lock = threading.Lock()
_lib = None

_P = C.c_void_p
_I64 = C.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle (no fused multiply-add: x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["cc", "-std=c11", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    """Load a compiled oracle library and declare its signatures."""
    lib = C.CDLL(path)
    sig = {
        "wsmo_unique": (_I64, [_P, _I64, C.c_int, _P, _P]),
        "wsmo_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
        "wsmo_init_indices": (C.c_int, [_I64, C.c_int, C.c_uint64, _P]),
        "wsmo_init_centers": (None, [_P, _I64, _P, C.c_int, _P, _P]),
        "wsmo_center_distances": (None, [_P, C.c_int, _P]),
        "wsmo_sort_rows": (None, [_P, C.c_int, _P]),
        "wsmo_assign": (_I64, [_P, _I64, _P, C.c_int, _P, _P, _P, _P]),
        "wsmo_update": (None, [_P, _P, _I64, _P, C.c_int, _P, _P, _P]),
        "wsmo_update_normalised": (None, [_P, _P, _I64, _P, C.c_int, _P]),
        "wsmo_iteration": (C.c_double, [_P, _P, _I64, C.c_int, _P, _P, _P, _P, _P]),
        "wsmo_run": (C.c_int, [_P, _P, _I64, C.c_int, _P, _P, C.c_int, C.c_double,
                               _P, _P]),
        "wsmo_exhaustive": (None, [_P, _I64, _P, C.c_int, _P, _P, _P]),
        "wsmo_kmeans_pixels_iteration": (C.c_double, [_P, _I64, C.c_int, C.c_int,
                                                      _P, _P]),
        "wsmo_map": (C.c_int, [_P, _I64, C.c_int, _P, _P, _I64, _P]),
        "wsmo_mse": (C.c_double, [_P, _I64, C.c_int, _P, C.c_int, _P]),
        "wsmo_psnr": (C.c_double, [C.c_double]),
        "wsmo_distortion_grad": (C.c_double, [_P, _P, _I64, _P, C.c_int, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def compile_variant(source: str, path: str):
    """Compile C source text (a modified copy of the oracle) and bind it.

    Used by the planted-mistake tests, which swap the result in for the real
    oracle to show that the pins reject it."""
    src = path + ".c"
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["cc", "-std=c11", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", path, src, "-lm"])
    return _bind(path)


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _pixels(rgb: np.ndarray) -> tuple[np.ndarray, int, int]:
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    stride = rgb.shape[-1]
    if stride not in (3, 4):
        raise ValueError("pixels must have 3 or 4 channels")
    return rgb, rgb.size // stride, stride


# ---- Sec. 2, data sampling and sample weighting ------------------------------

def unique(rgb: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Unique packed colors 0xRRGGBB (ascending) and their pixel counts."""
    rgb, n, stride = _pixels(rgb)
    colors = np.empty(max(n, 1), np.uint32)
    counts = np.empty(max(n, 1), np.uint32)
    nu = _load().wsmo_unique(_ptr(rgb), n, stride, _ptr(colors), _ptr(counts))
    if nu < 0:
        raise ValueError("oracle unique failed")
    return colors[:nu].copy(), counts[:nu].copy()


def unpack(colors: np.ndarray) -> np.ndarray:
    c = colors.astype(np.int64)
    return np.stack([(c >> 16) & 255, (c >> 8) & 255, c & 255], axis=-1).astype(np.float64)


# ---- Algorithm 2, initialisation ---------------------------------------------

def splitmix64(seed: int, i: int) -> int:
    return int(_load().wsmo_splitmix64(seed & (2**64 - 1), i))


def init_indices(n_unique: int, K: int, seed: int) -> np.ndarray:
    idx = np.empty(K, np.int64)
    if _load().wsmo_init_indices(n_unique, K, seed & (2**64 - 1), _ptr(idx)) != 0:
        raise ValueError("K must satisfy 1 <= K <= N'")
    return idx


def init(colors: np.ndarray, K: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Initial centers [K,3] (FP64) and memberships (all 0)."""
    colors = np.ascontiguousarray(colors, np.uint32)
    idx = init_indices(len(colors), K, seed)
    centers = np.empty((K, 3), np.float64)
    labels = np.empty(len(colors), np.int32)
    _load().wsmo_init_centers(_ptr(colors), len(colors), _ptr(idx), K, _ptr(centers),
                              _ptr(labels))
    return centers, labels


# ---- Algorithm 2, the steps of one pass ---------------------------------------

def center_distances(centers: np.ndarray) -> np.ndarray:
    centers = np.ascontiguousarray(centers, np.float64)
    K = centers.shape[0]
    d = np.empty((K, K), np.float64)
    _load().wsmo_center_distances(_ptr(centers), K, _ptr(d))
    return d


def sort_rows(d: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(d, np.float64)
    K = d.shape[0]
    M = np.empty((K, K), np.int32)
    _load().wsmo_sort_rows(_ptr(d), K, _ptr(M))
    return M


def assign(colors, centers, labels, d=None, M=None):
    """Pruned assignment; returns (new labels, min_dist per color, #distances)."""
    colors = np.ascontiguousarray(colors, np.uint32)
    centers = np.ascontiguousarray(centers, np.float64)
    K = centers.shape[0]
    if d is None:
        d = center_distances(centers)
    if M is None:
        M = sort_rows(d)
    lab = np.ascontiguousarray(labels, np.int32).copy()
    mind = np.empty(len(colors), np.float64)
    ev = _load().wsmo_assign(_ptr(colors), len(colors), _ptr(centers), K,
                             _ptr(np.ascontiguousarray(d)), _ptr(np.ascontiguousarray(M)),
                             _ptr(lab), _ptr(mind))
    return lab, mind, int(ev)


def update(colors, counts, labels, centers):
    """Weighted means; returns (new centers, S [K,3] int64, W [K] int64)."""
    colors = np.ascontiguousarray(colors, np.uint32)
    counts = np.ascontiguousarray(counts, np.uint32)
    lab = np.ascontiguousarray(labels, np.int32)
    c = np.ascontiguousarray(centers, np.float64).copy()
    K = c.shape[0]
    S = np.empty((K, 3), np.int64)
    W = np.empty(K, np.int64)
    _load().wsmo_update(_ptr(colors), _ptr(counts), len(colors), _ptr(lab), K, _ptr(c),
                        _ptr(S), _ptr(W))
    return c, S, W


def update_normalised(colors, counts, labels, centers):
    colors = np.ascontiguousarray(colors, np.uint32)
    counts = np.ascontiguousarray(counts, np.uint32)
    lab = np.ascontiguousarray(labels, np.int32)
    c = np.ascontiguousarray(centers, np.float64).copy()
    _load().wsmo_update_normalised(_ptr(colors), _ptr(counts), len(colors), _ptr(lab),
                                   c.shape[0], _ptr(c))
    return c


def iteration(colors, counts, centers, labels):
    """One pass of Algorithm 2.

    Returns dict(centers, labels, S, W, sse, evaluated); inputs are not modified.
    """
    colors = np.ascontiguousarray(colors, np.uint32)
    counts = np.ascontiguousarray(counts, np.uint32)
    c = np.ascontiguousarray(centers, np.float64).copy()
    lab = np.ascontiguousarray(labels, np.int32).copy()
    K = c.shape[0]
    S = np.empty((K, 3), np.int64)
    W = np.empty(K, np.int64)
    ev = np.zeros(1, np.int64)
    sse = _load().wsmo_iteration(_ptr(colors), _ptr(counts), len(colors), K, _ptr(c),
                                 _ptr(lab), _ptr(S), _ptr(W), _ptr(ev))
    return dict(centers=c, labels=lab, S=S, W=W, sse=float(sse), evaluated=int(ev[0]))


def run(colors, counts, centers, labels, max_iter: int, eps: float):
    """Algorithm 2 with the Sec. 3.2 termination (eps <= 0: fixed max_iter).

    Returns dict(centers, labels, iters, sse_trace, evaluated).
    """
    colors = np.ascontiguousarray(colors, np.uint32)
    counts = np.ascontiguousarray(counts, np.uint32)
    c = np.ascontiguousarray(centers, np.float64).copy()
    lab = np.ascontiguousarray(labels, np.int32).copy()
    trace = np.zeros(max(max_iter, 1), np.float64)
    ev = np.zeros(1, np.int64)
    it = _load().wsmo_run(_ptr(colors), _ptr(counts), len(colors), c.shape[0], _ptr(c),
                          _ptr(lab), max_iter, eps, _ptr(trace), _ptr(ev))
    if it < 0:
        raise ValueError("oracle run: bad arguments")
    return dict(centers=c, labels=lab, iters=int(it), sse_trace=trace[:it].copy(),
                evaluated=int(ev[0]))


# ---- checkers without pruning --------------------------------------------------

def exhaustive(colors, centers):
    """(best, second best, lowest argmin) over all K centers, per color."""
    colors = np.ascontiguousarray(colors, np.uint32)
    centers = np.ascontiguousarray(centers, np.float64)
    n = len(colors)
    b = np.empty(n, np.float64)
    s = np.empty(n, np.float64)
    a = np.empty(n, np.int32)
    _load().wsmo_exhaustive(_ptr(colors), n, _ptr(centers), centers.shape[0], _ptr(b), _ptr(s),
                            _ptr(a))
    return b, s, a


def kmeans_pixels_iteration(rgb, centers):
    """One iteration of Algorithm 1 over every pixel; returns (centers, labels, mse)."""
    rgb, n, stride = _pixels(rgb)
    c = np.ascontiguousarray(centers, np.float64).copy()
    lab = np.empty(n, np.int32)
    mse = _load().wsmo_kmeans_pixels_iteration(_ptr(rgb), n, stride, c.shape[0], _ptr(c),
                                               _ptr(lab))
    return c, lab, float(mse)


# ---- Sec. 1 pixel mapping, Sec. 3.1 Eq. 2 and Eq. 3 ---------------------------

def map_pixels(rgb, colors, labels) -> np.ndarray:
    rgb, n, stride = _pixels(rgb)
    colors = np.ascontiguousarray(colors, np.uint32)
    lab = np.ascontiguousarray(labels, np.int32)
    out = np.empty(n, np.int32)             # palette indices (K may exceed 256)
    if _load().wsmo_map(_ptr(rgb), n, stride, _ptr(colors), _ptr(lab), len(colors),
                        _ptr(out)) != 0:
        raise ValueError("pixel color missing from the unique list")
    return out


def mse(rgb, palette, index) -> float:
    rgb, n, stride = _pixels(rgb)
    pal = np.ascontiguousarray(palette, np.float64)
    idx = np.ascontiguousarray(index, np.int32).reshape(-1)
    v = _load().wsmo_mse(_ptr(rgb), n, stride, _ptr(pal), pal.shape[0], _ptr(idx))
    if v < 0:
        raise ValueError("index out of palette range")
    return float(v)


def psnr(m: float) -> float:
    return float(_load().wsmo_psnr(m))


def round_palette(palette) -> np.ndarray:
    """The palette as 8-bit colors (Sec. 3.1: a quantized image stores 8-bit
    colors; the paper does not say whether its MSE uses them, so this is the
    secondary palette): every coordinate rounded to the nearest integer, ties
    to even, clamped to [0, 255]; float64 [K, 3]."""
    p = np.asarray(palette, np.float64)[:, :3]
    return np.clip(np.rint(p), 0.0, 255.0)


def distortion_grad(X, w, centers):
    """D(C, X) = sum w_i min_k ||x_i - c_k||^2 and its gradients (dC, dX)."""
    X = np.ascontiguousarray(X, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    c = np.ascontiguousarray(centers, np.float64)
    n, K = X.shape[0], c.shape[0]
    dC = np.empty((K, 3), np.float64)
    dX = np.empty((n, 3), np.float64)
    a = np.empty(n, np.int32)
    D = _load().wsmo_distortion_grad(_ptr(X), _ptr(w), n, _ptr(c), K, _ptr(dC), _ptr(dX),
                                     _ptr(a))
    return float(D), dC, dX, a


# ---- the whole quantizer, for reference runs ------------------------------------

def quantize(rgb, K: int, seed: int, max_iter: int, eps: float):
    """Unique colors -> init -> Algorithm 2 -> final assignment -> mapping -> MSE.

    Returns dict(colors, counts, init_centers, centers, labels, iters, sse_trace,
    index, mse, evaluated).
    """
    colors, counts = unique(rgb)
    c0, lab0 = init(colors, K, seed)
    r = run(colors, counts, c0, lab0, max_iter, eps)
    lab, _, ev = assign(colors, r["centers"], r["labels"])
    index = map_pixels(rgb, colors, lab)
    m = mse(rgb, r["centers"], index)
    return dict(colors=colors, counts=counts, init_centers=c0, centers=r["centers"],
                labels=lab, iters=r["iters"], sse_trace=r["sse_trace"], index=index, mse=m,
                evaluated=r["evaluated"] + ev)
