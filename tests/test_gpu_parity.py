"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars (Celebi, arXiv:1011.0093; tolerances of the FP32-vs-FP64 contract):
  - unique colors, counts, initial indices, integer cluster sums S_k / W_k,
    distance counts and the index image: bit-exact;
  - memberships: bit-exact except for colors whose best and second-best
    squared distances differ by at most 1e-3 in the oracle (a near-tie that
    FP32 may resolve the other way);
  - centers: the GPU stores fl32(S_k / W_k), so when the sums agree its
    centers equal the oracle's FP64 centers rounded to FP32 exactly, and
    always lie within 1e-4 of them;
  - SSE and MSE: within 1e-5 relative.
Near-ties are handled by teacher forcing: every iteration starts the GPU from
the oracle's centers and memberships, so one flipped tie cannot carry over.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GAP = 1e-3


@pytest.fixture(scope="module")
def wsm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1011_0093_gb300 import build as B
    B.build()
    import paper_1011_0093_gb300 as w
    return w


@pytest.fixture(scope="module")
def h(wsm):
    with wsm.Handle(256, 1 << 24, 1 << 24) as handle:
        yield handle


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_unique(wsm, h, img):
    n = img.shape[0] * img.shape[1] if img.ndim == 3 else 0
    colors = torch.empty(max(n, 1), dtype=torch.uint32, device="cuda")
    counts = torch.empty(max(n, 1), dtype=torch.uint32, device="cuda")
    nu = wsm.wsm_reduce(h, dev(img), colors, counts)
    return colors[:nu], counts[:nu], nu


def pad4(c):
    out = np.zeros((c.shape[0], 4), np.float32)
    out[:, :3] = c
    return out


def f32_centers(S, W, fallback):
    """fl32 of the exact quotient S/W (the oracle's FP64 quotient rounded)."""
    c = np.array(fallback, np.float64).copy()
    nz = W > 0
    c[nz] = S[nz].astype(np.float64) / W[nz, None].astype(np.float64)
    return c.astype(np.float32)


def gaps(colors, centers):
    best, second, _ = oracle.exhaustive(colors, centers)
    return second - best


# ---- unique colors and counts --------------------------------------------------

@pytest.mark.parametrize("case", ["plain256", "sweep0", "sweep3", "sweep7", "ragged", "stride4",
                                  "single_pixel", "one_color", "tiny_levels", "wide"])
def test_reduce_bit_exact(wsm, h, case):
    img = {
        "plain256": synth.plain_256,
        "sweep0": lambda: synth.sweep_512_one(0),
        "sweep3": lambda: synth.sweep_512_one(3),
        "sweep7": lambda: synth.sweep_512_one(7),
        "ragged": lambda: synth.image(257, 263, 9, 11),
        "stride4": lambda: np.concatenate([synth.image(131, 77, 4, 5),
                                           np.full((131, 77, 1), 200, np.uint8)], axis=-1),
        "single_pixel": lambda: np.array([[[1, 2, 3]]], np.uint8),
        "one_color": lambda: np.full((64, 48, 3), 77, np.uint8),
        "tiny_levels": lambda: synth.tiny(33, 31, 2, 4),
        "wide": lambda: synth.image(16, 2048, 12, 20),
    }[case]()
    c, n, nu = gpu_unique(wsm, h, img)
    rc, rn = oracle.unique(img)
    assert nu == len(rc)
    assert np.array_equal(c.cpu().numpy(), rc)
    assert np.array_equal(n.cpu().numpy(), rn)


def test_reduce_every_24bit_color_once(wsm, h):
    """Maximum size: a 4096x4096 image holding each of the 2^24 colors once."""
    keys = np.arange(1 << 24, dtype=np.uint32)
    img = np.stack([(keys >> 16) & 255, (keys >> 8) & 255, keys & 255], -1).astype(np.uint8)
    img = img.reshape(4096, 4096, 3)
    c, n, nu = gpu_unique(wsm, h, img)
    assert nu == 1 << 24
    assert np.array_equal(c.cpu().numpy(), keys)
    assert np.all(n.cpu().numpy() == 1)


def test_reduce_max_size_noisy_image(wsm, h):
    img = synth.image(4096, 4096, 77, 24)
    c, n, nu = gpu_unique(wsm, h, img)
    rc, rn = oracle.unique(img)
    assert nu == len(rc)
    assert np.array_equal(c.cpu().numpy(), rc) and np.array_equal(n.cpu().numpy(), rn)


def test_reduce_empty_image(wsm, h):
    colors = torch.empty(1, dtype=torch.uint32, device="cuda")
    assert wsm.wsm_reduce(h, torch.empty((0, 3), dtype=torch.uint8, device="cuda"), colors,
                          colors.clone()) == 0


def test_reduce_capacity_overflow_then_recovers(wsm, h):
    img = synth.sweep_512_one(5)
    colors = torch.empty(1000, dtype=torch.uint32, device="cuda")
    counts = torch.empty(1000, dtype=torch.uint32, device="cuda")
    with pytest.raises(wsm.WsmError, match="CAPACITY"):
        wsm.wsm_reduce(h, dev(img), colors, counts)
    rc, rn = oracle.unique(img)
    assert np.array_equal(colors.cpu().numpy(), rc[:1000])
    other = synth.image(200, 150, 3, 4)        # histogram was cleared despite the overflow
    c, n, nu = gpu_unique(wsm, h, other)
    oc, on = oracle.unique(other)
    assert np.array_equal(c.cpu().numpy(), oc) and np.array_equal(n.cpu().numpy(), on)


# ---- initial centers -------------------------------------------------------------

@pytest.mark.parametrize("K,seed", [(1, 0), (16, 0), (32, 5), (256, 123456789), (256, 2**64 - 1)])
def test_init_matches_oracle(wsm, h, K, seed):
    img = synth.plain_256()
    c, n, nu = gpu_unique(wsm, h, img)
    centers = torch.empty((K, 4), dtype=torch.float32, device="cuda")
    labels = torch.full((nu,), 9, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, c, nu, K, seed, centers, labels)
    rc, _ = oracle.unique(img)
    c0, lab0 = oracle.init(rc, K, seed)
    assert np.array_equal(centers.cpu().numpy()[:, :3], c0.astype(np.float32))
    assert int(labels.max()) == 0


def test_init_all_colors_and_too_many(wsm, h):
    img = synth.tiny(6, 5, 1, 3)
    c, n, nu = gpu_unique(wsm, h, img)
    centers = torch.empty((nu, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, c, nu, nu, 7, centers, labels)
    got = centers.cpu().numpy()[:, :3]
    assert np.array_equal(got, oracle.unpack(c.cpu().numpy()).astype(np.float32))
    with pytest.raises(wsm.WsmError, match="INVAL"):
        wsm.wsm_init(h, c, nu, nu + 1, 7, torch.empty((nu + 1, 4), dtype=torch.float32,
                                                      device="cuda"), labels)


# ---- the Sort-Means iterations, teacher-forced ----------------------------------

def check_pass(colors, counts, c, lab, got_labels, got_centers, got_S, got_W, got_sse,
               got_ev, it, paper_scan=True):
    """Compare one GPU pass with one oracle pass started from the same state
    (oracle centers c, memberships lab).  Returns the oracle's pass and the
    number of colors whose membership differs (each must be a near-tie)."""
    step = oracle.iteration(colors, counts, c, lab)
    g = gaps(colors, c)
    diff = got_labels != step["labels"]
    assert np.all(g[diff] <= GAP), (it, np.flatnonzero(diff)[:5], g[diff][:5])
    assert abs(got_sse - step["sse"]) <= 1e-5 * step["sse"], (it, got_sse, step["sse"])
    # clusters that no flipped color left or joined must match bit for bit
    touched = np.zeros(c.shape[0], bool)
    touched[got_labels[diff]] = True
    touched[step["labels"][diff]] = True
    ok = ~touched
    assert np.array_equal(got_S[ok], step["S"][ok]) and np.array_equal(got_W[ok], step["W"][ok])
    expect = f32_centers(step["S"], step["W"], c)
    assert np.array_equal(got_centers[ok], expect[ok]), it
    assert np.abs(got_centers[ok] - step["centers"][ok]).max(initial=0.0) <= 1e-4
    if paper_scan and it == 0 and not diff.any():   # integer centers: exact FP32 distances
        assert got_ev == step["evaluated"]
    return step, int(diff.sum())


def gpu_pass(wsm, h, cd, nd, nu, K, centers, labels):
    done, trace = wsm.wsm_iterate(h, cd, nd, nu, K, centers, labels, 1, 0.0)
    assert done == 1
    ev, S, W = wsm.wsm_iterate_stats(h, K)
    return (labels.cpu().numpy(), centers.cpu().numpy()[:, :3], S.numpy(), W.numpy(), trace[0],
            ev)


def teacher_forced(wsm, h, img, K, seed, iters, paper_scan=False):
    """Run `iters` oracle passes; before each, start the GPU from the
    oracle's centers and memberships and compare one GPU pass with it.  Each
    GPU pass is the first pass of its launch, so it uses the candidate start
    unless paper_scan, which also checks the distance counts of Algorithm 2."""
    wsm.wsm_set_first_pass_start(h, not paper_scan)
    colors, counts = oracle.unique(img)
    cd, nd = dev(colors), dev(counts)
    c, lab = oracle.init(colors, K, seed)
    flips = 0
    for it in range(iters):
        centers = dev(pad4(c.astype(np.float32)))
        labels = dev(lab.astype(np.int16 if h.wide else np.uint8))
        out = gpu_pass(wsm, h, cd, nd, len(colors), K, centers, labels)
        step, nflip = check_pass(colors, counts, c, lab, *out, it, paper_scan)
        flips += nflip
        c, lab = step["centers"], step["labels"]
    wsm.wsm_set_first_pass_start(h, True)
    return flips


def test_iterations_teacher_forced_plain256(wsm, h):
    flips = teacher_forced(wsm, h, synth.plain_256(), 16, 0, 40)
    assert flips <= 5


@pytest.mark.parametrize("s,K", [(0, 32), (2, 64), (5, 128), (7, 256), (3, 256)])
def test_iterations_teacher_forced_sweep512(wsm, h, s, K):
    teacher_forced(wsm, h, synth.sweep_512_one(s), K, 100 + s, 10)


@pytest.mark.parametrize("img_fn,K,passes", [(synth.plain_256, 16, 12),
                                             (lambda: synth.sweep_512_one(7), 256, 3)])
def test_visits_and_counts_follow_algorithm_2_without_the_candidate_start(wsm, h, img_fn, K,
                                                                          passes):
    teacher_forced(wsm, h, img_fn(), K, 3, passes, paper_scan=True)


def test_iterations_teacher_forced_ties(wsm, h):
    """Few levels per channel: exact distance ties everywhere, integer
    centers in the first pass, duplicate centers possible."""
    for seed in range(6):
        img = synth.tiny(40, 37, 50 + seed, 4)
        colors, _ = oracle.unique(img)
        teacher_forced(wsm, h, img, min(len(colors), 5 + 3 * seed), seed, 6)
        teacher_forced(wsm, h, img, min(len(colors), 5 + 3 * seed), seed, 6, paper_scan=True)


# ---- free-running: whole path vs the oracle's whole path --------------------------

def run_gpu(wsm, h, img, K, seed, max_iter, eps):
    q = wsm.quantize(dev(img), K, seed=seed, max_iter=max_iter, eps=eps, handle=h)
    torch.cuda.synchronize()
    return q


def compare_whole_path(wsm, h, img, K, seed, max_iter, eps):
    """One wsm.quantize call against oracle.quantize.  The GPU run is replayed
    pass by pass from its own state next to the oracle: while memberships
    agree, every pass must match as in teacher forcing; the first pass where
    they differ must differ only at near-ties, after which the two runs may
    legitimately drift apart and only the replay's agreement with the
    one-call run is checked.  Without such a divergence the final centers,
    SSE trace, MSE and index image must match the oracle's."""
    q = run_gpu(wsm, h, img, K, seed, max_iter, eps)
    ref = oracle.quantize(img, K, seed, max_iter, eps)
    colors, counts = ref["colors"], ref["counts"]
    assert q.n_unique == len(colors)
    assert np.array_equal(q.colors.cpu().numpy(), colors)
    assert np.array_equal(q.counts.cpu().numpy(), counts)
    # replay: the GPU one pass at a time from its own state
    cd, nd = dev(colors), dev(counts)
    centers = torch.empty((K, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(len(colors), dtype=torch.int16 if h.wide else torch.uint8, device="cuda")
    wsm.wsm_init(h, cd, len(colors), K, seed, centers, labels)
    c, lab = oracle.init(colors, K, seed)
    diverged = None
    gpu_trace = []
    for it in range(q.iters):
        out = gpu_pass(wsm, h, cd, nd, len(colors), K, centers, labels)
        gpu_trace.append(out[4])
        if diverged is None:
            step, nflip = check_pass(colors, counts, c, lab, *out, it, paper_scan=False)
            if nflip:
                diverged = it
            c, lab = step["centers"], step["labels"]
    # the replay reproduces the one-call run exactly
    assert gpu_trace == list(q.sse_trace)
    assert torch.equal(centers, q.centers)
    if diverged is not None:
        return q, ref, diverged
    assert q.iters == ref["iters"], (q.iters, ref["iters"])
    tr = np.array(q.sse_trace)
    assert np.all(np.abs(tr - ref["sse_trace"]) <= 1e-5 * ref["sse_trace"])
    gc = q.centers.cpu().numpy()[:, :3]
    assert np.abs(gc - ref["centers"]).max() <= 1e-4
    assert abs(q.mse - ref["mse"]) <= 1e-5 * ref["mse"]
    # index image: bit-exact except at pixels whose color is a near-tie for
    # the final centers
    g = gaps(colors, ref["centers"])
    glab = q.labels.cpu().numpy()
    diff = glab != ref["labels"]
    assert np.all(g[diff] <= GAP)
    keys = ((img[..., 0].astype(np.uint32) << 16) | (img[..., 1].astype(np.uint32) << 8)
            | img[..., 2]).ravel()
    clear = np.isin(keys, colors[~diff])
    assert np.array_equal(q.index.cpu().numpy().ravel()[clear], ref["index"][clear])
    return q, ref, None


def test_whole_path_plain256_convergent(wsm, h):
    q, ref, div = compare_whole_path(wsm, h, synth.plain_256(), 16, 0, 100, 1e-4)
    assert div is None and 2 <= q.iters < 100


@pytest.mark.parametrize("s", range(8))
def test_whole_path_sweep512_fixed10(wsm, h, s):
    img = synth.sweep_512_one(s)
    for K in (32, 64, 128, 256):
        compare_whole_path(wsm, h, img, K, 1000 * s + K, 10, 0.0)


# ---- palettes of more than 256 colors: 16-bit memberships ----------------------------

@pytest.fixture(scope="module")
def hw(wsm):
    with wsm.Handle(1024, 1 << 20, 1 << 20) as handle:
        assert handle.wide
        yield handle


@pytest.mark.parametrize("s,K", [(7, 512), (3, 1024)])
def test_wide_palette_iterations_teacher_forced(wsm, hw, s, K):
    teacher_forced(wsm, hw, synth.sweep_512_one(s), K, 300 + s, 4)


def test_wide_palette_visits_follow_algorithm_2(wsm, hw):
    teacher_forced(wsm, hw, synth.sweep_512_one(6), 640, 9, 2, paper_scan=True)


@pytest.mark.parametrize("s,K", [(5, 512), (1, 300)])
def test_wide_palette_whole_path(wsm, hw, s, K):
    """Init, iterations, final mapping and MSE with uint16 memberships and
    index image, against the oracle."""
    q, ref, div = compare_whole_path(wsm, hw, synth.sweep_512_one(s), K, 77 + s, 10, 0.0)
    assert q.index.dtype == torch.int16 and q.labels.dtype == torch.int16
    if div is None:
        assert int(q.index.max()) >= 256          # labels past one byte were written


def test_wide_palette_batch_equals_single(wsm, hw):
    """The batched graph path with a wide handle gives each image what the
    one-image path gives it."""
    imgs = [synth.sweep_512_one(s)[: 300 + 37 * s, : 256 + 51 * s] for s in (2, 4, 6)]
    Ks = [300, 1024, 513]
    seeds = [5, 6, 7]
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=6, handle=hw)
    plan.load([torch.from_numpy(np.ascontiguousarray(i)) for i in imgs])
    plan.capture()
    plan.replay()
    plan.sync()
    with wsm.Handle(1024, 1 << 20, 1 << 20) as h1:
        for q, img in enumerate(imgs):
            one = wsm.quantize(dev(img), Ks[q], seed=seeds[q], max_iter=6, handle=h1)
            r = plan.result(q)
            assert torch.equal(one.centers, r["centers"]) and torch.equal(one.index, r["index"])
            assert one.mse == r["mse"] and one.iters == r["iters"]


# ---- mapping and distortion -------------------------------------------------------

def test_map_and_distortion_given_labels(wsm, h):
    """wsm_map with its input memberships already final: the index image is the
    oracle's lookup of those memberships, bit for bit, and the MSE of Eq. 2
    matches the oracle on the same FP32 palette."""
    img = synth.image(300, 211, 8, 9)
    colors, counts = oracle.unique(img)
    K = 64
    c0, lab0 = oracle.init(colors, K, 4)
    r = oracle.run(colors, counts, c0, lab0, 15, 0.0)
    pal = r["centers"].astype(np.float32)
    lab, _, _ = oracle.assign(colors, pal.astype(np.float64), r["labels"])
    labels = dev(lab.astype(np.uint8))
    centers = dev(pad4(pal))
    index = torch.empty(img.shape[:2], dtype=torch.uint8, device="cuda")
    wsm.wsm_map(h, dev(img), dev(colors), len(colors), centers, K, labels, index)
    got_lab = labels.cpu().numpy()
    g = gaps(colors, pal.astype(np.float64))
    diff = got_lab != lab
    assert np.all(g[diff] <= GAP)
    expect = oracle.map_pixels(img, colors, got_lab.astype(np.int32))
    assert np.array_equal(index.cpu().numpy().ravel(), expect)
    m = wsm.wsm_distortion(h, dev(img), centers, K, index)
    ref = oracle.mse(img, pal.astype(np.float64), expect)
    assert abs(m - ref) <= 1e-6 * ref
    # stride-4 pixels give the same results
    img4 = np.concatenate([img, np.zeros(img.shape[:2] + (1,), np.uint8)], -1)
    index4 = torch.empty_like(index)
    wsm.wsm_map(h, dev(img4), dev(colors), len(colors), centers, K, labels, index4)
    assert torch.equal(index4, index)
    assert wsm.wsm_distortion(h, dev(img4), centers, K, index4) == m


def test_unaligned_buffers_take_the_byte_path(wsm, h):
    """Pixels and index images that do not start on a 16-byte boundary (the
    kernels then read one pixel at a time) give the same unique colors, index
    image and MSE as 16-byte-aligned copies; n % 16 != 0 covers the tail of
    the vector path too."""
    img = synth.image(173, 97, 21, 6)                     # 16781 pixels, 16781 % 16 == 13
    n = img.shape[0] * img.shape[1]
    K = 32
    c_al, w_al, nu = gpu_unique(wsm, h, img)
    for off in (1, 3, 8):
        buf = torch.zeros(3 * n + 16, dtype=torch.uint8, device="cuda")
        rgb = buf[off:off + 3 * n].view(img.shape)
        rgb.copy_(dev(img))
        assert rgb.data_ptr() % 16 == off % 16
        colors = torch.empty(n, dtype=torch.uint32, device="cuda")
        counts = torch.empty(n, dtype=torch.uint32, device="cuda")
        assert wsm.wsm_reduce(h, rgb, colors, counts) == nu
        assert torch.equal(colors[:nu], c_al) and torch.equal(counts[:nu], w_al)
    colors, counts = oracle.unique(img)
    c0, lab0 = oracle.init(colors, K, 5)
    r = oracle.run(colors, counts, c0, lab0, 5, 0.0)
    pal = dev(pad4(r["centers"].astype(np.float32)))
    labels = dev(r["labels"].astype(np.uint8))
    ref_index = torch.empty(img.shape[:2], dtype=torch.uint8, device="cuda")
    wsm.wsm_map(h, dev(img), dev(colors), len(colors), pal, K, labels, ref_index)
    ref_mse = wsm.wsm_distortion(h, dev(img), pal, K, ref_index)
    for off in (1, 5):
        buf = torch.zeros(3 * n + 16, dtype=torch.uint8, device="cuda")
        rgb = buf[off:off + 3 * n].view(img.shape)
        rgb.copy_(dev(img))
        ibuf = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
        index = ibuf[off:off + n].view(img.shape[:2])
        wsm.wsm_map(h, rgb, dev(colors), len(colors), pal, K, labels, index)
        assert torch.equal(index, ref_index)
        assert wsm.wsm_distortion(h, rgb, pal, K, index) == ref_mse


def test_round_palette_and_the_mse_of_the_8bit_palette(wsm, h):
    """The 8-bit palette is the oracle's rounding (ties to even, clamped) of
    the same FP32 centers, bit for bit, and the MSE with it equals the
    oracle's exactly (every squared distance is then an integer)."""
    rng = np.random.default_rng(77)
    K = 256
    c = (rng.random((K, 4)) * 270 - 5).astype(np.float32)
    c[:32, :3] = (rng.integers(0, 255, (32, 3)) + 0.5).astype(np.float32)   # exact ties
    pal8, rounded = wsm.wsm_round_palette(h, dev(c), K)
    expect = oracle.round_palette(c.astype(np.float64))
    assert np.array_equal(pal8.cpu().numpy()[:, :3], expect.astype(np.uint8))
    assert np.all(pal8.cpu().numpy()[:, 3] == 0)
    assert np.array_equal(rounded.cpu().numpy()[:, :3], expect.astype(np.float32))
    img = synth.image(211, 160, 31, 8)
    q = wsm.quantize(dev(img), 64, seed=5, max_iter=10, handle=h, palette8=True)
    pal = oracle.round_palette(q.centers.cpu().numpy().astype(np.float64))
    assert np.array_equal(q.palette8.cpu().numpy()[:, :3], pal.astype(np.uint8))
    ref = oracle.mse(img, pal, q.index.cpu().numpy())
    assert q.mse8 == ref
    assert q.mse8 >= 0.0 and abs(q.mse8 - q.mse) < 0.5 * 3 + 2 * (3 * q.mse) ** 0.5


# ---- edge cases -------------------------------------------------------------------

def test_k1_and_lossless(wsm, h):
    img = synth.image(50, 40, 6, 3)
    compare_whole_path(wsm, h, img, 1, 0, 5, 0.0)
    tiny = synth.tiny(8, 8, 2, 3)
    nu = len(oracle.unique(tiny)[0])
    q = run_gpu(wsm, h, tiny, nu, 5, 10, 1e-4)
    assert q.iters == 1 and q.mse == 0.0 and q.sse_trace[0] == 0.0


def test_single_color_image(wsm, h):
    img = np.full((17, 19, 3), (10, 200, 30), np.uint8)
    q = run_gpu(wsm, h, img, 1, 0, 10, 1e-4)
    assert q.n_unique == 1 and q.iters == 1 and q.mse == 0.0
    assert q.centers.cpu().numpy()[0, :3].tolist() == [10.0, 200.0, 30.0]


def test_max_iter_zero_keeps_centers(wsm, h):
    img = synth.image(64, 64, 2, 6)
    colors, counts, nu = gpu_unique(wsm, h, img)
    centers = torch.empty((8, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, colors, nu, 8, 1, centers, labels)
    before = centers.clone()
    done, trace = wsm.wsm_iterate(h, colors, counts, nu, 8, centers, labels, 0, 0.0)
    assert done == 0 and trace == [] and torch.equal(centers[:, :3], before[:, :3])


def test_bad_labels_and_indices_reported(wsm, h):
    img = synth.image(64, 64, 2, 6)
    colors, counts, nu = gpu_unique(wsm, h, img)
    centers = torch.empty((8, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, colors, nu, 8, 1, centers, labels)
    labels[nu // 2] = 200
    with pytest.raises(wsm.WsmError, match="INVAL"):
        wsm.wsm_iterate(h, colors, counts, nu, 8, centers, labels, 2, 0.0)
    index = torch.full((64, 64), 9, dtype=torch.uint8, device="cuda")
    with pytest.raises(wsm.WsmError, match="INVAL"):
        wsm.wsm_distortion(h, dev(img), centers, 8, index)
    compare_whole_path(wsm, h, img, 8, 1, 5, 0.0)        # handle still usable


def test_async_calls_then_status(wsm, h):
    img = synth.image(128, 96, 3, 7)
    colors, counts, nu = gpu_unique(wsm, h, img)
    centers = torch.empty((32, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, colors, nu, 32, 9, centers, labels)
    c2, l2 = centers.clone(), labels.clone()
    assert wsm.wsm_iterate(h, colors, counts, nu, 32, centers, labels, 10, 0.0, sync=False) is None
    wsm.wsm_sync_status(h)
    done, _ = wsm.wsm_iterate(h, colors, counts, nu, 32, c2, l2, 10, 0.0)
    assert done == 10 and torch.equal(centers, c2) and torch.equal(labels, l2)


def test_deterministic_repeat(wsm, h):
    img = synth.sweep_512_one(6)
    a = run_gpu(wsm, h, img, 256, 3, 10, 0.0)
    b = run_gpu(wsm, h, img, 256, 3, 10, 0.0)
    assert torch.equal(a.centers, b.centers) and torch.equal(a.index, b.index)
    assert a.sse_trace == b.sse_trace and a.mse == b.mse
