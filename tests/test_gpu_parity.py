"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The bars and the rule for memberships that may differ are those of
tests/parity.py (Celebi, arXiv:1011.0093, Algorithm 2): unique colors,
counts, initial centers, integer sums, the index image and, where the
arithmetic is exact, every membership (exact ties included) and Algorithm
2's distance count are bit-exact; a membership differs only where FP32
rounding can decide it; centers within 1e-4 (fl32(S/W) where the sums
agree), SSE and MSE within 1e-5 relative.  Teacher forcing starts every
compared GPU pass from the oracle's state, so one rounding decision cannot
carry over; whole runs are compared free-running until the first such
decision and in teacher forcing after it.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from parity import compare_whole_path, dev, exact_ties, pad4, teacher_forced, unexplained_flips

pytestmark = pytest.mark.gpu


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


def gpu_unique(wsm, h, img):
    n = img.shape[0] * img.shape[1] if img.ndim == 3 else 0
    colors = torch.empty(max(n, 1), dtype=torch.uint32, device="cuda")
    counts = torch.empty(max(n, 1), dtype=torch.uint32, device="cuda")
    nu = wsm.wsm_reduce(h, dev(img), colors, counts)
    return colors[:nu], counts[:nu], nu


# ---- unique colors and counts --------------------------------------------------

@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("case", ["plain256", "sweep0", "sweep3", "sweep7", "ragged", "stride4",
                                  "single_pixel", "one_color", "tiny_levels", "wide"])
def test_reduce_bit_exact(wsm, h, case, path):
    """Both ways of filling the histogram (direct atomics, bucketed), forced."""
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
    wsm.wsm_set_reduce_path(h, path)
    try:
        c, n, nu = gpu_unique(wsm, h, img)
    finally:
        wsm.wsm_set_reduce_path(h, 0)
    rc, rn = oracle.unique(img)
    assert nu == len(rc)
    assert np.array_equal(c.cpu().numpy(), rc)
    assert np.array_equal(n.cpu().numpy(), rn)


@pytest.mark.parametrize("path", [1, 2])
def test_reduce_large_flat_and_noisy_regions(wsm, h, path):
    """A 2048x2048 image whose left half is one color and right half noise:
    one bucket holds millions of pixels (split into many work items of the
    bucketed path) beside thousands of small buckets."""
    img = synth.image(2048, 2048, 33, 18)
    img[:, :1024] = (200, 40, 90)
    wsm.wsm_set_reduce_path(h, path)
    try:
        c, n, nu = gpu_unique(wsm, h, img)
    finally:
        wsm.wsm_set_reduce_path(h, 0)
    rc, rn = oracle.unique(img)
    assert nu == len(rc) and n.cpu().numpy().max() >= 2048 * 1024
    assert np.array_equal(c.cpu().numpy(), rc) and np.array_equal(n.cpu().numpy(), rn)


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


@pytest.mark.parametrize("paper_scan", [False, True])
@pytest.mark.parametrize("s,K", [(1, 256), (4, 64), (6, 32), (2, 200), (5, 100)])
def test_exact_arithmetic_every_membership_and_count(wsm, h, s, K, paper_scan):
    """Passes from centers on the 1/8 grid, where FP32 and FP64 compute every
    distance exactly: every membership, exact ties included, must be the one
    Algorithm 2's visit order gives (the later of equal distances), and with
    the paper's start the distance count must be Algorithm 2's.  Palettes of
    100 and 200 colors give rows of 65..128 and 129..200 kept entries, whose
    sort pads the keys to 128 and 256."""
    flips = teacher_forced(wsm, h, synth.sweep_512_one(s), K, 40 + s, 6, paper_scan=paper_scan,
                           exact=True)
    assert flips == 0


def test_iterations_teacher_forced_ties(wsm, h):
    """Few levels per channel: exact distance ties everywhere, duplicate
    centers possible.  From the FP32-rounded oracle state every difference
    must be explained by rounding; from centers on the 1/8 grid (exact
    arithmetic) there must be none, in both start modes, and the passes must
    meet exact ties."""
    met = 0
    for seed in range(6):
        img = synth.tiny(40, 37, 50 + seed, 4)
        colors, counts = oracle.unique(img)
        K = min(len(colors), 5 + 3 * seed)
        teacher_forced(wsm, h, img, K, seed, 6)
        teacher_forced(wsm, h, img, K, seed, 6, paper_scan=True)
        assert teacher_forced(wsm, h, img, K, seed, 6, exact=True) == 0
        assert teacher_forced(wsm, h, img, K, seed, 6, paper_scan=True, exact=True) == 0
        c, lab = oracle.init(colors, K, seed)
        met += exact_ties(colors, c, lab)
    assert met > 0


# ---- free-running: whole path vs the oracle's whole path --------------------------

def run_gpu(wsm, h, img, K, seed, max_iter, eps):
    q = wsm.quantize(dev(img), K, seed=seed, max_iter=max_iter, eps=eps, handle=h)
    torch.cuda.synchronize()
    return q


def test_whole_path_plain256_convergent(wsm, h):
    got, ref, div, _ = compare_whole_path(wsm, h, synth.plain_256(), 16, 0, 100, 1e-4,
                                          name="plain256 K=16 WSM-C")
    assert div is None and 2 <= got["iters"] < 100


@pytest.mark.parametrize("s", range(8))
def test_whole_path_sweep512_fixed10(wsm, h, s):
    """WSM (10 iterations) on every sweep image and K: the run itself while it
    agrees with the oracle's, teacher forcing after a rounding decision, and
    the final MSE from the oracle's palette within 1e-5; the free runs' MSEs
    must stay within 1e-4 of each other (relative) even after a divergence."""
    img = synth.sweep_512_one(s)
    for K in (32, 64, 128, 256):
        got, ref, div, mse_rel = compare_whole_path(wsm, h, img, K, 1000 * s + K, 10, 0.0,
                                                    name=f"sweep{s} K={K} WSM")
        assert mse_rel <= (1e-5 if div is None else 1e-4), (K, div, mse_rel)


@pytest.mark.parametrize("s", [1, 3, 5, 7])
def test_whole_path_sweep512_convergent(wsm, h, s):
    """WSM-C (Sec. 3.2 stop rule, eps = 1e-4, at most 100 iterations) on four
    sweep images at K = 32 and 256: the GPU's fixed-point SSE stop rule must
    stop at the oracle's iteration while the runs agree."""
    img = synth.sweep_512_one(s)
    for K in (32, 256):
        got, ref, div, mse_rel = compare_whole_path(wsm, h, img, K, 500 + s + K, 100, 1e-4,
                                                    name=f"sweep{s} K={K} WSM-C")
        if div is None:
            assert got["iters"] == ref["iters"]
        assert 2 <= ref["iters"] < 100


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
    got, ref, div, _ = compare_whole_path(wsm, hw, synth.sweep_512_one(s), K, 77 + s, 10, 0.0,
                                          name=f"sweep{s} K={K} wide")
    assert got["index"].dtype == torch.int16 and got["labels"].dtype == torch.int16
    assert int(got["index"].max()) >= 256          # labels past one byte were written


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
    p64 = pal.astype(np.float64)
    again, _, _ = oracle.assign(colors, p64, lab)           # the oracle from the same start
    assert unexplained_flips(colors, p64, p64, lab, got_lab, again).size == 0
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
    for off, path in ((1, 1), (3, 1), (8, 1), (1, 2), (5, 2)):
        buf = torch.zeros(3 * n + 16, dtype=torch.uint8, device="cuda")
        rgb = buf[off:off + 3 * n].view(img.shape)
        rgb.copy_(dev(img))
        assert rgb.data_ptr() % 16 == off % 16
        colors = torch.empty(n, dtype=torch.uint32, device="cuda")
        counts = torch.empty(n, dtype=torch.uint32, device="cuda")
        wsm.wsm_set_reduce_path(h, path)
        try:
            assert wsm.wsm_reduce(h, rgb, colors, counts) == nu
        finally:
            wsm.wsm_set_reduce_path(h, 0)
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
    compare_whole_path(wsm, h, img, 1, 0, 5, 0.0, name="50x40 K=1")
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


def test_empty_cluster_keeps_its_center_and_sse_is_taken_before_the_update(wsm, h):
    """The oracle's hand-worked pin (test_oracle_pins) through the C ABI: one
    pass from memberships 0, 0, 0 gives 0, 1, 1; nothing joins the third
    center, which keeps its place (reading R3); the second becomes the FP32
    rounding of 56/5; the pass's SSE is the assignment step's, 5/6 (reading
    R4; every distance is an integer here, so the fixed-point SSE is exact)."""
    colors = torch.tensor([0x000000, 0x0A0000, 0x0C0000], dtype=torch.uint32, device="cuda")
    counts = torch.tensor([1, 2, 3], dtype=torch.uint32, device="cuda")
    centers = torch.tensor([[0, 0, 0, 0], [11, 0, 0, 0], [200, 200, 200, 0]],
                           dtype=torch.float32, device="cuda")
    labels = torch.zeros(3, dtype=torch.uint8, device="cuda")
    for first_pass_start in (True, False):
        c, lab = centers.clone(), labels.clone()
        wsm.wsm_set_first_pass_start(h, first_pass_start)
        try:
            done, trace = wsm.wsm_iterate(h, colors, counts, 3, 3, c, lab, 1, 0.0)
        finally:
            wsm.wsm_set_first_pass_start(h, True)
        assert done == 1
        assert lab.cpu().tolist() == [0, 1, 1]
        assert c[:, :3].cpu().tolist() == [[0.0, 0.0, 0.0],
                                           [float(np.float32(56 / 5)), 0.0, 0.0],
                                           [200.0, 200.0, 200.0]]
        assert math.isclose(trace[0], 5 / 6, rel_tol=1e-15)


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
    compare_whole_path(wsm, h, img, 8, 1, 5, 0.0, name="64x64 K=8 after bad labels")


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
