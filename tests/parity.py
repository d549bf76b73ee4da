"""Comparison of the CUDA path with the CPU oracle, shared by the GPU tests.

Bars (Celebi, arXiv:1011.0093, Algorithm 2; tolerances of the FP32-vs-FP64
contract):
  - unique colors, counts, initial centers, the integer cluster sums S_k / W_k
    of every cluster no differing color touches, the index image, and
    Algorithm 2's distance count wherever the arithmetic is exact: bit-exact;
  - a membership may differ from the oracle's only where FP32 rounding can
    decide it.  That needs (i) a near-tie: the oracle's best and second-best
    squared distances differ by at most GAP, and (ii) a decision that is not
    taken on exactly computed values.  When the two candidate centers are
    the same point, or both of the color's distances to them are computed
    without any rounding in FP32 from the same centers the oracle uses, the
    decision (an exact tie included) rests on Algorithm 2's visit order
    alone -- the later visit wins -- and the GPU must take it as the oracle
    does, unless that order itself (the two centers' places in row p, or
    whether the visit of row p reaches one of them) is decided on values
    within rounding of each other;
  - centers within 1e-4, and equal to fl32(S_k / W_k) where the sums agree;
    SSE and MSE within 1e-5 relative.
Teacher forcing gives both sides the same state: the oracle's centers
rounded to FP32 (the values the GPU holds) and the oracle's memberships.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

GAP = 1e-3
# Whole-path divergences seen in this session: (run, pass, flipped colors);
# every compared run: (run, iterations GPU / oracle, divergence pass or None,
# relative difference of the free runs' MSEs).
DIVERGENCES: list[tuple[str, int, int]] = []
RUNS: list[tuple[str, int, int, int | None, float]] = []


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pad4(c):
    out = np.zeros((c.shape[0], 4), np.float32)
    out[:, :3] = c
    return out


def fl32(c):
    """Centers as the FP32 values a GPU holds, in float64."""
    return np.asarray(c, np.float64).astype(np.float32).astype(np.float64)


def f32_centers(S, W, fallback):
    """fl32 of the exact quotient S/W (the oracle's FP64 quotient rounded)."""
    c = np.array(fallback, np.float64).copy()
    nz = W > 0
    c[nz] = S[nz].astype(np.float64) / W[nz, None].astype(np.float64)
    return c.astype(np.float32)


def gaps_of(colors, centers):
    best, second, _ = oracle.exhaustive(colors, centers)
    return second - best


def _is32(v):
    return v.astype(np.float32).astype(np.float64) == v


def exact_sq(a, b):
    """Whether the squared distance between points a and b ([..., 3] float64
    holding FP32 values) is computed without any rounding by the kernel's
    FP32 difference form (three subtractions, one product, two fused
    multiply-adds, channels in order): every difference, square and running
    sum is then an FP32 value, so FP32 and FP64 give the exact distance."""
    e = a - b
    ok = np.all(_is32(e), axis=-1)
    e2 = e * e
    ok &= np.all(_is32(e2), axis=-1)
    s = e2[..., 0]
    for ch in (1, 2):
        t = s + e2[..., ch]
        ok &= (t - s == e2[..., ch]) & (t - e2[..., ch] == s) & _is32(t)
        s = t
    return ok


def all_exact(c32):
    """Centers whose coordinates are multiples of 1/8 in [0, 255]: then every
    distance between an integer color and a center, or between two centers,
    is an FP32 value with every intermediate exact (11-bit differences,
    22-bit squares, sums below 2^18 in steps of 2^-6)."""
    c = np.asarray(c32, np.float64)
    return bool(np.all(c * 8 == np.round(c * 8)) and np.all((c >= 0) & (c <= 255)))


def sq(a, b):
    d = a - b
    return np.sum(d * d, axis=-1)


def unexplained_flips(colors, c64, c32, lab, got, ref):
    """Indices of colors whose GPU membership `got` differs from the oracle's
    `ref` in a way FP32 rounding cannot explain (see the module docstring).
    c64: the centers the oracle's pass started from; c32: the FP32 centers
    the GPU's pass started from; lab: the memberships both started from."""
    diff = np.flatnonzero(got != ref)
    if diff.size == 0:
        return diff
    x = oracle.unpack(colors[diff])
    g = gaps_of(colors[diff], c64)
    p, a, b = lab[diff].astype(np.int64), got[diff].astype(np.int64), ref[diff].astype(np.int64)
    same_in = np.all(c64 == c32, axis=1)                # the oracle's centers are FP32 values
    ca, cb, cp = c32[a], c32[b], c32[p]
    same_pt = np.all(ca == cb, axis=1)
    exact_pair = same_in[a] & same_in[b] & (same_pt | (exact_sq(x, ca) & exact_sq(x, cb)))

    def tol(v):
        return 1e-6 * np.abs(v) + 1e-6

    # order of a and b in row p
    dpa, dpb = sq(cp, ca), sq(cp, cb)
    row_exact = same_in[p] & (same_pt | (exact_sq(cp, ca) & exact_sq(cp, cb)))
    row_near = ~row_exact & (np.abs(dpa - dpb) <= tol(np.maximum(dpa, dpb)))
    # whether the visit of row p reaches a / b: d[p][t] >= 4 prev stops it
    prev = sq(x, cp)
    prev_exact = same_in[p] & exact_sq(x, cp)

    def reach_near(t, dpt):
        ex = prev_exact & same_in[t] & exact_sq(cp, c32[t])
        return (t != p) & ~ex & (np.abs(dpt - 4 * prev) <= tol(dpt))

    near_order = row_near | reach_near(a, dpa) | reach_near(b, dpb)
    explained = (g <= GAP) & (~exact_pair | near_order)
    return diff[~explained]


def check_pass(colors, counts, c, lab, got_labels, got_centers, got_S, got_W, got_sse, got_ev,
               it, paper_scan=True, c_gpu=None):
    """Compare one GPU pass with one oracle pass started from the oracle's
    state (centers c, memberships lab); the GPU started from c_gpu (default
    fl32(c)) and the same memberships.  Returns the oracle's pass and the
    number of colors whose membership differs (each explained by rounding)."""
    c_gpu = fl32(c) if c_gpu is None else np.asarray(c_gpu, np.float64)
    step = oracle.iteration(colors, counts, c, lab)
    bad = unexplained_flips(colors, np.asarray(c, np.float64), c_gpu, lab, got_labels,
                            step["labels"])
    assert bad.size == 0, (it, bad[:5], got_labels[bad[:5]], step["labels"][bad[:5]],
                           lab[bad[:5]])
    diff = got_labels != step["labels"]
    exact = all_exact(c_gpu) and np.array_equal(c_gpu, np.asarray(c, np.float64))
    if exact:       # every decision on exactly computed values: no difference at all
        assert not diff.any(), (it, np.flatnonzero(diff)[:5])
    assert abs(got_sse - step["sse"]) <= 1e-5 * step["sse"], (it, got_sse, step["sse"])
    # clusters that no differing color left or joined must match bit for bit
    touched = np.zeros(c.shape[0], bool)
    touched[got_labels[diff]] = True
    touched[step["labels"][diff]] = True
    ok = ~touched
    assert np.array_equal(got_S[ok], step["S"][ok]) and np.array_equal(got_W[ok], step["W"][ok])
    expect = f32_centers(step["S"], step["W"], c_gpu)
    assert np.array_equal(got_centers[ok], expect[ok]), it
    assert np.abs(got_centers[ok] - step["centers"][ok]).max(initial=0.0) <= 1e-4
    if paper_scan and exact:
        assert got_ev == step["evaluated"], (it, got_ev, step["evaluated"])
    return step, int(diff.sum())


def gpu_pass(wsm, h, cd, nd, nu, K, centers, labels):
    """One pass (one persistent launch with max_iter = 1) from the given
    state; returns memberships, centers, S, W, SSE and distance count."""
    done, trace = wsm.wsm_iterate(h, cd, nd, nu, K, centers, labels, 1, 0.0)
    assert done == 1
    ev, S, W = wsm.wsm_iterate_stats(h, K)
    return (labels.cpu().numpy(), centers.cpu().numpy()[:, :3], S.numpy(), W.numpy(), trace[0],
            ev)


def forced_pass(wsm, h, cd, nd, colors, counts, c, lab, it, paper_scan=False):
    """The GPU started from the oracle's state (fl32 centers, memberships),
    compared with the oracle's pass from that state."""
    K = c.shape[0]
    centers = dev(pad4(np.asarray(c).astype(np.float32)))
    labels = dev(lab.astype(np.int16 if h.wide else np.uint8))
    out = gpu_pass(wsm, h, cd, nd, len(colors), K, centers, labels)
    return check_pass(colors, counts, c, lab, *out, it, paper_scan)


def teacher_forced(wsm, h, img, K, seed, iters, paper_scan=False, exact=False):
    """Run `iters` oracle passes, each from the previous one's FP32-rounded
    centers and memberships; before each, start the GPU from the same state
    and compare one GPU pass with it.  Each GPU pass is the first pass of its
    launch, so it uses the candidate start unless paper_scan, which also
    checks the distance counts of Algorithm 2 where the arithmetic is exact.
    With exact, the state's centers are rounded to multiples of 1/8 instead:
    every distance is then exact on both sides and every membership (exact
    ties included) and distance count must agree.  Returns the number of
    differing memberships over all passes."""
    wsm.wsm_set_first_pass_start(h, not paper_scan)
    try:
        colors, counts = oracle.unique(img)
        cd, nd = dev(colors), dev(counts)
        c, lab = oracle.init(colors, K, seed)
        flips = 0
        for it in range(iters):
            if exact:
                assert all_exact(c)
            step, nflip = forced_pass(wsm, h, cd, nd, colors, counts, c, lab, it, paper_scan)
            flips += nflip
            c, lab = (np.round(step["centers"] * 8) / 8 if exact else fl32(step["centers"]),
                      step["labels"])
    finally:
        wsm.wsm_set_first_pass_start(h, True)
    return flips


def exact_ties(colors, c, lab):
    """Colors of an exact state (centers on the 1/8 grid) whose pass meets an
    exact tie: two centers at the same least distance (what the later-visit
    rule decides)."""
    best, second, _ = oracle.exhaustive(colors, c)
    return int(np.sum(second == best))


def compare_whole_path(wsm, h, img, K, seed, max_iter, eps, got=None, name="", index_of=None):
    """A whole GPU run (wsm.quantize on h, or the results `got` of another
    path: centers [K,4], iters, mse, index, n_unique, optionally colors,
    counts, labels, sse_trace) against oracle.quantize.

    The GPU run is replayed pass by pass from its own state next to the
    oracle's run: while memberships agree every pass must match as in
    teacher forcing.  At the first pass where they differ (only through
    rounding) the two runs may drift apart; the pass is recorded, and from
    there every remaining pass of the oracle's run is checked in teacher
    forcing (the GPU started from the oracle's state), and so are the final
    assignment, index image and MSE computed by the GPU from the oracle's
    final palette and memberships.  Without a divergence the run's own
    final centers, SSE trace, iteration count, MSE and index image must
    match the oracle's.  Returns (got, ref, divergence pass or None,
    relative MSE difference of the two free runs)."""
    if got is None:
        q = wsm.quantize(dev(img), K, seed=seed, max_iter=max_iter, eps=eps, handle=h)
        torch.cuda.synchronize()
        got = dict(centers=q.centers, iters=q.iters, mse=q.mse, index=q.index,
                   n_unique=q.n_unique, colors=q.colors, counts=q.counts, labels=q.labels,
                   sse_trace=list(q.sse_trace))
    ref = oracle.quantize(img, K, seed, max_iter, eps)
    colors, counts = ref["colors"], ref["counts"]
    assert got["n_unique"] == len(colors)
    if "colors" in got:
        assert np.array_equal(got["colors"].cpu().numpy(), colors)
        assert np.array_equal(got["counts"].cpu().numpy(), counts)
    cd, nd = dev(colors), dev(counts)
    ltype = torch.int16 if h.wide else torch.uint8
    centers = torch.empty((K, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(len(colors), dtype=ltype, device="cuda")
    wsm.wsm_init(h, cd, len(colors), K, seed, centers, labels)
    c, lab = oracle.init(colors, K, seed)
    assert np.array_equal(centers.cpu().numpy()[:, :3], c.astype(np.float32))
    diverged = None
    gpu_trace = []
    for it in range(got["iters"]):
        c_gpu = centers.cpu().numpy()[:, :3].astype(np.float64)
        out = gpu_pass(wsm, h, cd, nd, len(colors), K, centers, labels)
        gpu_trace.append(out[4])
        if diverged is None and it < ref["iters"]:
            step, nflip = check_pass(colors, counts, c, lab, *out, it, paper_scan=False,
                                     c_gpu=c_gpu)
            if nflip:
                diverged = it
                DIVERGENCES.append((name, it, nflip))
            c, lab = step["centers"], step["labels"]
    # the replay reproduces the run exactly
    if "sse_trace" in got:
        assert gpu_trace == list(got["sse_trace"])
    assert torch.equal(centers.cpu()[:, :3], got["centers"].cpu()[:, :3])
    keys = ((img[..., 0].astype(np.uint32) << 16) | (img[..., 1].astype(np.uint32) << 8)
            | img[..., 2]).ravel()
    gi = got["index"].cpu().numpy().ravel().astype(np.int64)
    # every pixel carries its color's final membership
    ukeys, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    assert np.array_equal(ukeys, colors)
    glab = gi[first]
    assert np.array_equal(gi, glab[inv])
    if "labels" in got:
        assert np.array_equal(got["labels"].cpu().numpy().astype(np.int64), glab)
    mse_rel = abs(got["mse"] - ref["mse"]) / ref["mse"] if ref["mse"] else abs(got["mse"])
    if diverged is None:
        assert got["iters"] == ref["iters"], (got["iters"], ref["iters"])
        tr = np.array(gpu_trace)
        assert np.all(np.abs(tr - ref["sse_trace"]) <= 1e-5 * ref["sse_trace"])
        gc = got["centers"].cpu().numpy()[:, :3]
        assert np.abs(gc - ref["centers"]).max() <= 1e-4
        assert mse_rel <= 1e-5, (got["mse"], ref["mse"])
        # the final assignment (from the last pass's memberships against the
        # final centers) differs only where rounding explains it, and the
        # index image is the oracle's wherever the memberships agree
        bad = unexplained_flips(colors, ref["centers"], fl32(ref["centers"]), lab, glab,
                                ref["labels"])
        assert bad.size == 0, bad[:5]
        clear = (glab == ref["labels"])[inv]
        assert np.array_equal(gi[clear], ref["index"][clear])
        RUNS.append((name, got["iters"], ref["iters"], None, mse_rel))
        return got, ref, None, mse_rel
    # after the divergence: every remaining pass of the oracle's run in
    # teacher forcing, from the oracle's own state
    for it in range(diverged + 1, ref["iters"]):
        step, _ = forced_pass(wsm, h, cd, nd, colors, counts, c, lab, it)
        c, lab = step["centers"], step["labels"]
    # the oracle's final palette (as FP32) and last memberships through the
    # GPU's final assignment, mapping and MSE
    pal = fl32(c)
    fin_lab, _, _ = oracle.assign(colors, pal, lab)
    glabels = dev(lab.astype(np.int16 if h.wide else np.uint8))
    index = torch.empty(img.shape[:2], dtype=ltype, device="cuda")
    pal_d = dev(pad4(pal.astype(np.float32)))
    wsm.wsm_map(h, dev(img), cd, len(colors), pal_d, K, glabels, index)
    gl = glabels.cpu().numpy().astype(np.int64)
    bad = unexplained_flips(colors, pal, pal, lab, gl, fin_lab)
    assert bad.size == 0, bad[:5]
    expect = oracle.map_pixels(img, colors, fin_lab)
    clear = (gl == fin_lab)[inv]
    assert np.array_equal(index.cpu().numpy().ravel().astype(np.int64)[clear], expect[clear])
    m = wsm.wsm_distortion(h, dev(img), pal_d, K, index)
    m_ref = oracle.mse(img, pal, expect)
    assert abs(m - m_ref) <= 1e-5 * m_ref, (m, m_ref)
    assert abs(m - ref["mse"]) <= 1e-5 * ref["mse"], (m, ref["mse"])
    RUNS.append((name, got["iters"], ref["iters"], diverged, mse_rel))
    return got, ref, diverged, mse_rel
