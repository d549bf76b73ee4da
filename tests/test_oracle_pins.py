"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties one oracle function to something fixed independently of it:
a published test vector, a hand-worked case, brute force on tiny inputs, an
exact-fraction closed form, a library routine, or a mathematical invariant of
the method (Celebi, arXiv:1011.0093: Sec. 2, Algorithms 1 and 2, Sec. 3.1-3.2).
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


# ---- generators for tiny cases (inputs only) -----------------------------------

def tiny_colors(seed, n, levels):
    """Distinct packed colors from a lattice of `levels` values per channel."""
    rng = np.random.default_rng(seed)
    step = 255 // max(levels - 1, 1)
    pts = rng.integers(0, levels, size=(4 * n, 3)) * step
    keys = np.unique((pts[:, 0] << 16) | (pts[:, 1] << 8) | pts[:, 2]).astype(np.uint32)
    rng.shuffle(keys)
    return np.sort(keys[:n])


def brute_unique(rgb):
    counts = {}
    for px in rgb.reshape(-1, rgb.shape[-1]):
        k = (int(px[0]) << 16) | (int(px[1]) << 8) | int(px[2])
        counts[k] = counts.get(k, 0) + 1
    keys = sorted(counts)
    return np.array(keys, np.uint32), np.array([counts[k] for k in keys], np.uint32)


def sq(a, b):
    return sum((float(a[c]) - float(b[c])) ** 2 for c in range(3))


# ---- Sec. 2, data sampling and sample weighting ---------------------------------

@pytest.mark.parametrize("shape,levels,stride", [((7, 5), 3, 3), ((16, 16), 4, 3),
                                                  ((9, 13), 6, 4), ((1, 1), 2, 3)])
def test_unique_matches_brute_force(shape, levels, stride):
    img = synth.tiny(shape[0], shape[1], 11 + levels, levels)
    if stride == 4:
        img = np.concatenate([img, np.full(shape + (1,), 77, np.uint8)], axis=-1)
    c, n = oracle.unique(img)
    bc, bn = brute_unique(img)
    assert np.array_equal(c, bc) and np.array_equal(n, bn)


def test_unique_matches_numpy_on_plain_image():
    img = synth.plain_256()
    c, n = oracle.unique(img)
    keys = ((img[..., 0].astype(np.uint32) << 16) | (img[..., 1].astype(np.uint32) << 8)
            | img[..., 2]).ravel()
    uc, un = np.unique(keys, return_counts=True)
    assert np.array_equal(c, uc) and np.array_equal(n, un)
    assert int(n.sum()) == img.shape[0] * img.shape[1]
    assert np.all(np.diff(c.astype(np.int64)) > 0)


def test_unique_empty_and_single():
    c, n = oracle.unique(np.zeros((0, 3), np.uint8))
    assert len(c) == 0
    c, n = oracle.unique(np.full((4, 4, 3), 9, np.uint8))
    assert list(c) == [0x090909] and list(n) == [16]


# ---- initialisation: splitmix64 and Floyd sampling -------------------------------

def test_splitmix64_published_vector():
    for seed, i, val in read_golden("splitmix64.txt"):
        assert oracle.splitmix64(int(seed), int(i)) == int(val, 16)


def test_init_indices_valid():
    for seed in range(50):
        for n, K in [(1, 1), (5, 5), (17, 3), (1000, 256), (300000, 16)]:
            idx = oracle.init_indices(n, K, seed)
            assert len(idx) == K and len(set(idx.tolist())) == K
            assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < n
    with pytest.raises(ValueError):
        oracle.init_indices(3, 4, 0)
    with pytest.raises(ValueError):
        oracle.init_indices(3, 0, 0)


def test_init_subsets_uniform():
    """Floyd's algorithm draws every K-subset with the same probability."""
    n, K, trials = 6, 2, 15000
    hist = {}
    for seed in range(trials):
        key = tuple(oracle.init_indices(n, K, seed * 7919 + 1).tolist())
        hist[key] = hist.get(key, 0) + 1
    assert len(hist) == math.comb(n, K)
    expect = trials / math.comb(n, K)
    chi2 = sum((v - expect) ** 2 / expect for v in hist.values())
    assert chi2 < 45.0      # 14 degrees of freedom: p < 1e-4 beyond this


def test_init_floyd_on_the_published_stream():
    """Step r of Floyd's sample (Bentley & Floyd 1987) reduces draw r of the
    seed's stream, which for seed 0 is the published splitmix64 output r
    (tests/golden/splitmix64.txt): t = draw_r mod (j + 1) for j = n - K + r,
    taken unless already taken, else j.  The sizes are ones where a draw
    repeats an earlier pick at the second or the third step."""
    draws = [int(v, 16) for seed, _, v in read_golden("splitmix64.txt") if seed == "0"]
    K = len(draws)
    for n in (3, 7, 8, 13, 22, 32, 1000):
        picks = []
        for r, j in enumerate(range(n - K, n)):
            t = draws[r] % (j + 1)
            picks.append(j if t in picks else t)
        assert oracle.init_indices(n, K, 0).tolist() == sorted(picks), n


def test_init_centers_are_the_drawn_colors():
    colors = tiny_colors(3, 40, 6)
    c0, lab = oracle.init(colors, 7, 123)
    idx = oracle.init_indices(40, 7, 123)
    assert np.array_equal(c0, oracle.unpack(colors[idx]))
    assert np.all(lab == 0)


# ---- Algorithm 2: center distances and the sorted matrix M -----------------------

def test_center_distances_closed_form():
    c = np.array([[0, 0, 0], [3, 4, 0], [0, 0, 12], [3, 4, 12]], np.float64)
    d = oracle.center_distances(c)
    expect = np.array([[0, 25, 144, 169], [25, 0, 169, 144],
                       [144, 169, 0, 25], [169, 144, 25, 0]], np.float64)
    assert np.array_equal(d, expect)


def test_sort_rows_order_and_ties():
    c = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 0], [5, 5, 5]], np.float64)
    M = oracle.sort_rows(oracle.center_distances(c))
    assert M[0].tolist() == [0, 3, 1, 2, 4]   # p first, then duplicate 3 (d=0), ties by index
    assert M[3].tolist() == [3, 0, 1, 2, 4]
    assert M[1].tolist() == [1, 0, 3, 2, 4]   # d: 0->1, 3->1, 2->2, 4->66
    rng = np.random.default_rng(5)
    for _ in range(20):
        K = int(rng.integers(1, 40))
        c = rng.integers(0, 6, size=(K, 3)).astype(np.float64)
        d = oracle.center_distances(c)
        M = oracle.sort_rows(d)
        for p in range(K):
            assert sorted(M[p].tolist()) == list(range(K))
            assert M[p, 0] == p
            dd = d[p, M[p]]
            assert np.all(np.diff(dd) >= 0)


# ---- Algorithm 2: the pruned assignment ---------------------------------------

def test_assign_hand_worked_cases():
    for row in read_golden("sortmeans_hand.txt"):
        v = list(map(int, row[1:]))
        centers = np.array(v[0:9], np.float64).reshape(3, 3)
        x = v[9:12]
        color = np.array([(x[0] << 16) | (x[1] << 8) | x[2]], np.uint32)
        lab, mind, ev = oracle.assign(color, centers, np.array([v[12]], np.int32))
        assert (lab[0], mind[0], ev) == (v[13], float(v[14]), v[15]), row[0]


@pytest.mark.parametrize("levels", [3, 5, 256])
def test_assign_finds_exhaustive_minimum_from_any_start(levels):
    """The triangle-inequality stop never loses the nearest center (Sec. 2)."""
    rng = np.random.default_rng(levels)
    trials = 0
    for t in range(400):
        n = int(rng.integers(1, 120))
        K = int(rng.integers(1, 17))
        colors = tiny_colors(1000 * levels + t, n, levels)
        n = len(colors)
        if rng.random() < 0.5:
            centers = oracle.unpack(colors[rng.integers(0, n, size=K)])   # duplicates allowed
        else:
            centers = rng.random((K, 3)) * 255.0
        start = rng.integers(0, K, size=n).astype(np.int32)
        lab, mind, ev = oracle.assign(colors, centers, start)
        x = oracle.unpack(colors)
        full = ((x[:, None, :] - centers[None, :, :]) ** 2).sum(-1)
        best = full.min(axis=1)
        assert np.array_equal(mind, full[np.arange(n), lab])   # reported min is the label's
        assert np.all(mind == best)
        srt = np.sort(full, axis=1)
        gap = (srt[:, 1] - srt[:, 0]) if K > 1 else np.full(n, np.inf)
        clear = gap > 0
        assert np.array_equal(lab[clear], full.argmin(axis=1)[clear])
        assert n <= ev <= n * K
        trials += 1
    assert trials == 400


def test_assign_finds_exhaustive_minimum_with_large_palettes():
    """The same for palettes of more than 256 colors (memberships past one
    byte), from random starting memberships."""
    rng = np.random.default_rng(1024)
    for t, K in enumerate((257, 600, 1024)):
        colors = np.unique(rng.integers(0, 1 << 24, size=3000).astype(np.uint32))
        centers = rng.random((K, 3)) * 255.0
        start = rng.integers(0, K, size=len(colors)).astype(np.int32)
        lab, mind, ev = oracle.assign(colors, centers, start)
        x = oracle.unpack(colors)
        full = ((x[:, None, :] - centers[None, :, :]) ** 2).sum(-1)
        assert np.all(mind == full.min(axis=1))
        assert np.array_equal(mind, full[np.arange(len(colors)), lab])
        assert lab.max() >= 256
        assert len(colors) <= ev < len(colors) * K


def test_assign_stops_early_on_separated_clusters():
    """Well separated clusters: after convergence each color computes one distance."""
    base = np.array([[10, 10, 10], [200, 10, 10], [10, 200, 10], [10, 10, 200]])
    pts = []
    for b in base:
        for dx in range(3):
            for dy in range(3):
                pts.append(((b[0] + dx) << 16) | ((b[1] + dy) << 8) | b[2])
    colors = np.array(sorted(pts), np.uint32)
    counts = np.ones(len(colors), np.uint32)
    centers = base.astype(np.float64) + 1.0
    r = oracle.run(colors, counts, centers, np.zeros(len(colors), np.int32), 5, 1e-4)
    lab, mind, ev = oracle.assign(colors, r["centers"], r["labels"])
    assert ev == len(colors)


# ---- Algorithm 2: weighted means -------------------------------------------------

def test_update_matches_exact_fractions():
    rng = np.random.default_rng(9)
    for t in range(30):
        colors = tiny_colors(t, 50, 7)
        n = len(colors)
        counts = rng.integers(1, 1000, size=n).astype(np.uint32)
        K = int(rng.integers(1, 9))
        labels = rng.integers(0, K, size=n).astype(np.int32)
        old = rng.random((K, 3)) * 255
        c, S, W = oracle.update(colors, counts, labels, old)
        x = oracle.unpack(colors).astype(np.int64)
        for k in range(K):
            members = labels == k
            Wk = int(counts[members].astype(np.int64).sum())
            assert W[k] == Wk
            for ch in range(3):
                Sk = int((counts[members].astype(np.int64) * x[members, ch]).sum())
                assert S[k, ch] == Sk
                if Wk:
                    assert c[k, ch] == float(Fraction(Sk, Wk))   # correctly rounded mean
                else:
                    assert c[k, ch] == old[k, ch]                 # empty cluster keeps its center
        cn = oracle.update_normalised(colors, counts, labels, old)
        assert np.allclose(cn, c, rtol=1e-12, atol=1e-12)


def test_k1_closed_form():
    img = synth.tiny(12, 10, 4, 5)
    colors, counts = oracle.unique(img)
    x = oracle.unpack(colors)
    c0, lab = oracle.init(colors, 1, 0)
    r = oracle.run(colors, counts, c0, lab, 3, 0.0)
    N = int(counts.sum())
    for ch in range(3):
        mean = Fraction(int((counts.astype(np.int64) * x[:, ch].astype(np.int64)).sum()), N)
        assert r["centers"][0, ch] == float(mean)
    # second pass measures the distortion around the mean: the weighted variance
    var = sum(Fraction(int(counts[i]), N) * sum((Fraction(int(x[i, ch])) - Fraction(
        int((counts.astype(np.int64) * x[:, ch].astype(np.int64)).sum()), N)) ** 2
        for ch in range(3)) for i in range(len(colors)))
    assert math.isclose(r["sse_trace"][1], float(var), rel_tol=1e-12)


def test_empty_cluster_keeps_its_center_and_sse_is_taken_before_the_update():
    """Worked by hand.  Colors (0,0,0) x1, (10,0,0) x2, (12,0,0) x3; centers
    c0 = (0,0,0), c1 = (11,0,0), c2 = (200,200,200); every color starts in
    cluster 0.  Row 0 is c0, c1 (d = 121), c2 (d = 120000).  (0,0,0): prev = 0,
    the visit stops at once.  (10,0,0): prev = 100, 121 < 400 so c1 is visited
    at distance 1 and taken; 120000 >= 400 stops.  (12,0,0): prev = 144, c1 at
    distance 1.  So the memberships are 0, 1, 1; nothing joins c2, which keeps
    its place (reading R3); c0 = (0,0,0), c1 = ((2*10 + 3*12) / 5, 0, 0) =
    (11.2, 0, 0).  The SSE of the assignment step (reading R4) is
    (1*0 + 2*1 + 3*1) / 6 = 5/6; measured after the update it would be
    (2*1.2^2 + 3*0.8^2) / 6 = 0.8."""
    colors = np.array([0x000000, 0x0A0000, 0x0C0000], np.uint32)
    counts = np.array([1, 2, 3], np.uint32)
    centers = np.array([[0.0, 0.0, 0.0], [11.0, 0.0, 0.0], [200.0, 200.0, 200.0]])
    r = oracle.iteration(colors, counts, centers, np.zeros(3, np.int32))
    assert list(r["labels"]) == [0, 1, 1]
    assert list(r["W"]) == [1, 5, 0]
    assert r["centers"][2].tolist() == [200.0, 200.0, 200.0]
    assert r["centers"][0].tolist() == [0.0, 0.0, 0.0]
    assert r["centers"][1].tolist() == [56 / 5, 0.0, 0.0]
    assert math.isclose(r["sse"], 5 / 6, rel_tol=1e-15)    # FP64 sum of w_i * d_i


def test_k_equals_unique_count_is_lossless():
    img = synth.tiny(8, 8, 2, 3)
    colors, counts = oracle.unique(img)
    K = len(colors)
    assert K <= 64
    r = oracle.quantize(img, K, 5, 10, 1e-4)
    assert r["iters"] == 1 and r["sse_trace"][0] == 0.0 and r["mse"] == 0.0
    assert np.array_equal(np.sort(oracle.unpack(colors), axis=0),
                          np.sort(r["centers"], axis=0))


# ---- weighted k-means on unique colors == batch k-means on pixels ---------------

def test_weighted_equals_batch_kmeans():
    """Sec. 2 "Sample weighting" vs Algorithm 1: with the same initial centers,
    WSM on (unique color, count) moves the centers exactly like conventional
    k-means on every pixel, iteration by iteration (checked wherever no color
    is equidistant from two centers, since Algorithm 1 leaves ties open)."""
    compared = 0
    for seed in range(40):
        H, W = (12 + seed % 9, 10 + seed % 7)
        img = (synth.image(H, W, 100 + seed, seed % 4) if seed % 2
               else synth.tiny(H, W, 100 + seed, 24))
        colors, counts = oracle.unique(img)
        K = min(len(colors), 2 + seed % 7)
        c_w, lab_w = oracle.init(colors, K, seed)
        c_b = c_w.copy()
        for it in range(8):
            best, second, _ = oracle.exhaustive(colors, c_w)
            if K > 1 and np.any(second - best <= 0):
                break
            step = oracle.iteration(colors, counts, c_w, lab_w)
            c_b2, lab_b, mse_b = oracle.kmeans_pixels_iteration(img, c_b)
            assert np.array_equal(step["centers"], c_b2), (seed, it)
            assert math.isclose(step["sse"], mse_b, rel_tol=1e-12, abs_tol=1e-12)
            c_w, lab_w, c_b = step["centers"], step["labels"], c_b2
            compared += 1
    assert compared >= 150


# ---- Lloyd monotonicity and the termination rule (Sec. 3.2) ----------------------

def test_sse_never_increases_and_termination_rule():
    for img, K, seed in [(synth.plain_256(), 16, 0), (synth.image(64, 48, 3, 9), 8, 1),
                         (synth.tiny(20, 20, 7, 5), 6, 2)]:
        colors, counts = oracle.unique(img)
        c0, lab = oracle.init(colors, K, seed)
        full = oracle.run(colors, counts, c0, lab, 100, 0.0)["sse_trace"]
        assert np.all(full[1:] <= full[:-1] * (1 + 1e-12))
        for eps in (0.5, 0.3, 0.1, 0.03, 1e-2, 1e-3, 1e-4):
            r = oracle.run(colors, counts, c0, lab, 100, eps)
            tr = r["sse_trace"]
            assert np.array_equal(tr, full[:len(tr)])
            stop = 100
            for i in range(100):
                if full[i] == 0 or (i >= 1 and (full[i - 1] - full[i]) / full[i] <= eps):
                    stop = i + 1
                    break
            assert r["iters"] == stop, eps
        f = oracle.run(colors, counts, c0, lab, 10, 0.0)
        assert f["iters"] == 10


# ---- pixel mapping, Eq. 2 and Eq. 3 ---------------------------------------------

def test_map_and_mse_brute_force():
    img = synth.tiny(9, 11, 8, 4)
    colors, counts = oracle.unique(img)
    labels = (np.arange(len(colors)) % 5).astype(np.int32)
    idx = oracle.map_pixels(img, colors, labels)
    lut = {int(c): int(l) for c, l in zip(colors, labels)}
    flat = img.reshape(-1, 3)
    for p in range(len(flat)):
        k = (int(flat[p, 0]) << 16) | (int(flat[p, 1]) << 8) | int(flat[p, 2])
        assert idx[p] == lut[k]
    pal = np.array([[0, 0, 0], [255, 255, 255], [1.5, 2.5, 3.5], [100, 0, 50], [7, 7, 7]])
    m = oracle.mse(img, pal, idx)
    exact = sum(sq(flat[p], pal[idx[p]]) for p in range(len(flat))) / len(flat)
    assert math.isclose(m, exact, rel_tol=1e-13)


def test_map_and_mse_with_indices_beyond_one_byte():
    """Palettes of more than 256 colors: labels up to 999 reach the index image
    unchanged, an out-of-range index is refused, and the MSE of a palette that
    holds every pixel's own color is 0."""
    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, (20, 30, 3), dtype=np.uint8)
    colors, counts = oracle.unique(img)
    assert len(colors) <= 1000
    labels = (np.arange(len(colors)) * 7 % 1000).astype(np.int32)   # distinct: gcd(7, 1000) = 1
    idx = oracle.map_pixels(img, colors, labels)
    assert idx.dtype == np.int32 and idx.max() >= 256
    lut = {int(c): int(l) for c, l in zip(colors, labels)}
    keys = ((img[..., 0].astype(np.int64) << 16) | (img[..., 1].astype(np.int64) << 8)
            | img[..., 2]).ravel()
    assert all(idx[p] == lut[int(keys[p])] for p in range(len(keys)))
    pal = np.zeros((1000, 3))
    pal[labels] = oracle.unpack(colors)
    assert oracle.mse(img, pal, idx) == 0.0
    top = int(idx.max())                       # the smallest palette that holds every index
    assert oracle.mse(img, pal[:top + 1], idx) == 0.0
    for short in (500, top):
        with pytest.raises(ValueError):
            oracle.mse(img, pal[:short], idx)


def test_mse_psnr_closed_forms():
    img = np.array([[[0, 0, 0], [10, 20, 30]]], np.uint8)
    pal = np.array([[1, 2, 2], [10, 20, 33]], np.float64)
    # (1+4+4 + 0+0+9) / 2 pixels = 9
    assert oracle.mse(img, pal, np.array([0, 1], np.uint8)) == 9.0
    assert math.isclose(oracle.psnr(1.0), 20 * math.log10(255.0), rel_tol=1e-15)
    assert oracle.psnr(255.0 ** 2) == 0.0


def test_round_palette_ties_to_even_and_clamps():
    """Round half to even (0.5 -> 0, 1.5 -> 2, 2.5 -> 2, 254.5 -> 254), plain
    rounding elsewhere, clamping outside [0, 255]; the fourth column of a
    [K, 4] palette is dropped."""
    pal = np.array([[0.5, 1.5, 2.5, 9.0],
                    [254.5, 255.49, 300.0, 9.0],
                    [-0.2, 3.4999, 3.5001, 9.0],
                    [127.5, 128.5, 0.0, 9.0]])
    expect = np.array([[0, 2, 2], [254, 255, 255], [0, 3, 4], [128, 128, 0]], np.float64)
    assert np.array_equal(oracle.round_palette(pal), expect)
    # the MSE with the rounded palette of an image whose colors are the
    # palette's rounded colors is 0
    img = expect.astype(np.uint8)[None]
    assert oracle.mse(img, oracle.round_palette(pal), np.arange(4, dtype=np.uint8)) == 0.0


# ---- gradient of the weighted distortion ----------------------------------------

def test_distortion_gradient_finite_differences():
    rng = np.random.default_rng(21)
    for t in range(6):
        n, K = 40, 5
        X = rng.random((n, 3)) * 255
        w = rng.random(n)
        C = rng.random((K, 3)) * 255
        D, dC, dX, a = oracle.distortion_grad(X, w, C)
        h = 1e-3
        for k in range(K):
            for ch in range(3):
                Cp, Cm = C.copy(), C.copy()
                Cp[k, ch] += h
                Cm[k, ch] -= h
                Dp, _, _, ap = oracle.distortion_grad(X, w, Cp)
                Dm, _, _, am = oracle.distortion_grad(X, w, Cm)
                if np.array_equal(ap, a) and np.array_equal(am, a):
                    assert math.isclose((Dp - Dm) / (2 * h), dC[k, ch], rel_tol=1e-6,
                                        abs_tol=1e-6)
        for i in range(0, n, 7):
            for ch in range(3):
                Xp, Xm = X.copy(), X.copy()
                Xp[i, ch] += h
                Xm[i, ch] -= h
                Dp, _, _, ap = oracle.distortion_grad(Xp, w, C)
                Dm, _, _, am = oracle.distortion_grad(Xm, w, C)
                if np.array_equal(ap, a) and np.array_equal(am, a):
                    assert math.isclose((Dp - Dm) / (2 * h), dX[i, ch], rel_tol=1e-6,
                                        abs_tol=1e-6)


def test_gradient_vanishes_at_a_lloyd_fixed_point():
    img = synth.image(48, 40, 5, 6)
    colors, counts = oracle.unique(img)
    c0, lab = oracle.init(colors, 6, 3)
    r = oracle.run(colors, counts, c0, lab, 500, 1e-15)
    x = oracle.unpack(colors)
    w = counts / counts.sum()
    D, dC, _, _ = oracle.distortion_grad(x, w, r["centers"])
    assert np.abs(dC).max() < 1e-9
