"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: the autotuned launch shape and the path captured as three
CUDA graphs (unique colors + initialisation, the Sort-Means iterations, the
final assignment + mapping + MSE), replayed.

Workloads: the 8 seeded 512x512 images of the noise sweep (10k to 230k
unique colors) and the 64 seeded images of 256^2 to 2048^2 pixels (5k to 1M
unique colors), K = 256, WSM with 10 iterations.  At these sizes the oracle
checks, image by image, what holds at any size:
  - unique colors and counts: bit-exact (Sec. 2);
  - final memberships: each unique color's center is the nearest one, up to
    the FP32 rounding of the squared distances (Algorithm 2 is exact);
  - index image: every pixel carries its color's membership (Sec. 1);
  - MSE (Eq. 2): the oracle's FP64 MSE of the same palette and index image,
    within 1e-5 relative;
and, on sampled images, that the batch launch gives bit for bit what the
one-image calls give, and that its last pass is the oracle's Algorithm 2
pass from the same state (teacher forcing, as in the small-size tests).
The 8 sweep images of the benchmark's step are also compared with the
oracle's whole runs (tests/parity.py).
"""
import numpy as np
import pytest
import torch

import oracle
from parity import GAP, check_pass, compare_whole_path, gpu_pass

pytestmark = pytest.mark.gpu

K = 256
ITERS = 10


@pytest.fixture(scope="module")
def wsm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1011_0093_gb300 import build as B
    B.build()
    import paper_1011_0093_gb300 as w
    return w


@pytest.fixture(scope="module")
def workloads():
    import bench
    sweep = bench.workload(0)
    return dict(sweep=(sweep, [bench.image_seed(0, s) for s in range(len(sweep))]),
                batch=(bench.batch_workload(), [9000 + q for q in range(bench.BATCH_COUNT)]))


def run_as_benchmarked(wsm, images, seeds):
    plan = wsm.BatchPlan([im.shape for im in images], K, seeds, max_iter=ITERS)
    plan.load([torch.from_numpy(im) for im in images])
    plan.tune(repeats=1)
    plan.capture((wsm.STAGE_REDUCE | wsm.STAGE_INIT, wsm.STAGE_ITERATE,
                  wsm.STAGE_MAP | wsm.STAGE_INDEX | wsm.STAGE_DISTORTION))
    plan.replay()
    plan.sync()
    return plan


def check_image(img, res):
    colors, counts = oracle.unique(img)
    assert res["n_unique"] == len(colors)
    assert np.array_equal(res["colors"].cpu().numpy(), colors)
    assert np.array_equal(res["counts"].cpu().numpy(), counts)
    assert res["iters"] == ITERS
    C = res["centers"].cpu().numpy()[:, :3].astype(np.float64)
    lab = res["labels"].cpu().numpy().astype(np.int64)
    assert lab.min() >= 0 and lab.max() < K
    best, _, _ = oracle.exhaustive(colors, C)
    x = oracle.unpack(colors)
    mine = ((x - C[lab]) ** 2).sum(-1)
    # FP32 squared distances carry a relative error below 1e-6
    excess = mine - best
    assert np.all(excess <= GAP + 1e-6 * best), (excess.max(), int(np.argmax(excess)))
    keys = ((img[..., 0].astype(np.uint32) << 16) | (img[..., 1].astype(np.uint32) << 8)
            | img[..., 2]).ravel()
    expect = lab[np.searchsorted(colors, keys)]
    got = res["index"].cpu().numpy().ravel().astype(np.int64)
    assert np.array_equal(got, expect)
    ref = oracle.mse(img, C, got)
    assert abs(res["mse"] - ref) <= 1e-5 * ref + 2.0 ** -20, (res["mse"], ref)
    return colors, counts


def test_sweep_512_as_benchmarked(wsm, workloads):
    """The benchmark's own step (the 8 sweep images at the benchmark's seeds,
    autotuned shape, three captured graphs): each image's results against the
    oracle's whole run (tests/parity.py: the run while it agrees with the
    oracle's, teacher forcing after a rounding decision, the final MSE from
    the oracle's palette within 1e-5)."""
    images, seeds = workloads["sweep"]
    plan = run_as_benchmarked(wsm, images, seeds)
    with wsm.Handle(K, 1 << 18, 1 << 18) as h:
        for q, img in enumerate(images):
            res = plan.result(q)
            check_image(img, res)
            _, _, div, mse_rel = compare_whole_path(wsm, h, img, K, seeds[q], ITERS, 0.0,
                                                    got=res, name=f"bench sweep{q} K={K}")
            assert mse_rel <= (1e-5 if div is None else 1e-4), (q, div, mse_rel)


def test_uneven_batch_to_2048_as_benchmarked(wsm, workloads):
    images, seeds = workloads["batch"]
    plan = run_as_benchmarked(wsm, images, seeds)
    nus = [plan.result(q)["n_unique"] for q in range(len(images))]
    big, small = int(np.argmax(nus)), int(np.argmin(nus))
    sample = sorted({big, small, len(images) // 2, 7})
    assert max(nus) > 500_000
    for q in sample:
        check_image(images[q], plan.result(q))
    # the largest image: the one-image calls give the batch's results bit for
    # bit, and its last pass, rerun from the state after 9 passes, is the
    # oracle's pass from that state
    img, got = images[big], plan.result(big)
    n = img.shape[0] * img.shape[1]
    with wsm.Handle(K, n, n) as h:
        rgb = torch.from_numpy(img).cuda()
        colors = torch.empty(n, dtype=torch.uint32, device="cuda")
        counts = torch.empty(n, dtype=torch.uint32, device="cuda")
        nu = wsm.wsm_reduce(h, rgb, colors, counts)
        colors, counts = colors[:nu], counts[:nu]
        centers = torch.empty((K, 4), dtype=torch.float32, device="cuda")
        labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
        wsm.wsm_init(h, colors, nu, K, seeds[big], centers, labels)
        done, _ = wsm.wsm_iterate(h, colors, counts, nu, K, centers, labels, ITERS, 0.0)
        assert done == ITERS
        index = torch.empty(img.shape[:2], dtype=torch.uint8, device="cuda")
        wsm.wsm_map(h, rgb, colors, nu, centers, K, labels, index)
        assert torch.equal(centers, got["centers"])
        assert torch.equal(labels, got["labels"])
        assert torch.equal(index, got["index"])
        assert wsm.wsm_distortion(h, rgb, centers, K, index) == got["mse"]
        wsm.wsm_init(h, colors, nu, K, seeds[big], centers, labels)
        done, _ = wsm.wsm_iterate(h, colors, counts, nu, K, centers, labels, ITERS - 1, 0.0)
        assert done == ITERS - 1
        c9 = centers.cpu().numpy()[:, :3].astype(np.float64)
        l9 = labels.cpu().numpy().astype(np.int32)
        out = gpu_pass(wsm, h, colors, counts, nu, K, centers, labels)
    check_pass(colors.cpu().numpy(), counts.cpu().numpy(), c9, l9, *out, ITERS - 1,
               paper_scan=False)


def test_max_size_4096_image_whole_path(wsm):
    """The largest image a handle takes (2^24 pixels), with about 2M unique
    colors of nearly equal weight (every channel even, uniform), through the
    same captured path."""
    rng = np.random.default_rng(4096)
    img = (rng.integers(0, 128, (4096, 4096, 3), dtype=np.uint8) * 2).astype(np.uint8)
    plan = run_as_benchmarked(wsm, [img], [77])
    got = plan.result(0)
    assert got["n_unique"] > 2_000_000
    check_image(img, got)
