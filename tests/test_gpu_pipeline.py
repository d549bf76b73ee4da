"""wsm_quantize_batch (the whole path with N' kept on the device), its launch
shapes, the autotuner and CUDA-graph capture, against the one-image calls.

The contract is equality, bit for bit: the device-side initialisation draws
the same Floyd sample as the host one, the device-side block split changes
only which blocks do the work, and every reduction is exact, so each image's
N', centers, memberships, index image, iteration count and MSE equal those
of wsm_reduce -> wsm_init -> wsm_iterate -> wsm_map -> wsm_distortion.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wsm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1011_0093_gb300 import build as B
    B.build()
    import paper_1011_0093_gb300 as w
    return w


def single(wsm, h, img, K, seed, max_iter, eps):
    """The one-image calls, as the reference for an image of the batch."""
    rgb = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    n = img.shape[0] * img.shape[1]
    colors = torch.empty(n, dtype=torch.uint32, device="cuda")
    counts = torch.empty(n, dtype=torch.uint32, device="cuda")
    nu = wsm.wsm_reduce(h, rgb, colors, counts)
    centers = torch.empty((K, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, colors[:nu], nu, K, seed, centers, labels)
    init = centers.clone()
    it, _ = wsm.wsm_iterate(h, colors[:nu], counts[:nu], nu, K, centers, labels, max_iter, eps)
    index = torch.empty(img.shape[:2], dtype=torch.uint8, device="cuda")
    wsm.wsm_map(h, rgb, colors[:nu], nu, centers, K, labels, index)
    mse = wsm.wsm_distortion(h, rgb, centers, K, index)
    return dict(n_unique=nu, colors=colors[:nu], counts=counts[:nu], init=init, centers=centers,
                labels=labels, index=index, iters=it, mse=mse)


def uneven_batch(count, seed0=500):
    rng = np.random.default_rng(seed0)
    imgs, Ks = [], []
    for q in range(count):
        side = int(round(2 ** rng.uniform(5, 9)))              # 32 .. 512
        hh, ww = side, max(8, int(side * rng.uniform(0.5, 1.5)))
        img = synth.image(hh, ww, seed0 + q, int(rng.integers(0, 25)))
        if q % 5 == 3:
            img = np.concatenate([img, np.full((hh, ww, 1), 9, np.uint8)], -1)   # 4-byte pixels
        imgs.append(img)
        n_unique = len(np.unique(img[..., :3].reshape(-1, 3), axis=0))
        Ks.append(min(int(rng.choice([4, 16, 64, 256])), n_unique))
    return imgs, Ks


def check_against_single(wsm, plan, imgs, Ks, seeds, max_iter, eps):
    with wsm.Handle(256, max(i.shape[0] * i.shape[1] for i in imgs)) as h:
        for q, (img, K, s) in enumerate(zip(imgs, Ks, seeds)):
            ref = single(wsm, h, img, K, s, max_iter, eps)
            got = plan.result(q)
            assert got["n_unique"] == ref["n_unique"], q
            assert torch.equal(got["colors"], ref["colors"])
            assert torch.equal(got["counts"], ref["counts"])
            assert got["iters"] == ref["iters"], q
            assert torch.equal(got["centers"], ref["centers"]), q
            assert torch.equal(got["labels"], ref["labels"]), q
            assert torch.equal(got["index"], ref["index"]), q
            assert got["mse"] == ref["mse"], q


@pytest.mark.parametrize("max_iter,eps", [(10, 0.0), (60, 1e-4)])
def test_pipeline_equals_the_one_image_calls(wsm, max_iter, eps):
    imgs, Ks = uneven_batch(21)
    seeds = [77 + 3 * q for q in range(len(imgs))]
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=max_iter, eps=eps)
    plan.load([torch.from_numpy(i) for i in imgs])
    plan.run()
    plan.sync()
    check_against_single(wsm, plan, imgs, Ks, seeds, max_iter, eps)


def test_device_initialisation_equals_the_host_one(wsm):
    imgs, Ks = uneven_batch(10, seed0=900)
    seeds = [2**63 + 12345 * q for q in range(len(imgs))]
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=0)
    plan.load([torch.from_numpy(i) for i in imgs])
    plan.run()
    plan.sync()
    with wsm.Handle(256, 512 * 768) as h:
        for q, (img, K, s) in enumerate(zip(imgs, Ks, seeds)):
            ref = single(wsm, h, img, K, s, 0, 0.0)
            got = plan.result(q)
            assert got["iters"] == 0
            assert torch.equal(got["centers"], ref["init"]), q
            assert torch.equal(got["labels"], ref["labels"]), q   # the mapping's assignment


def test_every_launch_shape_gives_the_same_results(wsm):
    imgs, Ks = uneven_batch(9, seed0=1300)
    seeds = list(range(len(imgs)))
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=10)
    plan.load([torch.from_numpy(i) for i in imgs])
    outs = []
    for shape in range(5):
        _, threads, bps, resident = wsm.wsm_launch_shape(plan.handle, shape)
        assert threads in (256, 512, 1024) and bps >= 1
        if not resident:
            continue
        wsm.wsm_set_launch_shape(plan.handle, shape)
        assert wsm.wsm_launch_shape(plan.handle)[0] == shape
        plan.run()
        plan.sync()
        outs.append([(plan.result(q)["centers"].clone(), plan.result(q)["index"].clone())
                     for q in range(len(imgs))])
    assert len(outs) >= 3
    for other in outs[1:]:
        for (c0, i0), (c1, i1) in zip(outs[0], other):
            assert torch.equal(c0, c1) and torch.equal(i0, i1)


def test_autotune_then_graph_replay_on_new_pixels(wsm):
    imgs, Ks = uneven_batch(12, seed0=1700)
    seeds = [5 * q + 1 for q in range(len(imgs))]
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=10)
    plan.load([torch.from_numpy(i) for i in imgs])
    best, times = plan.tune(repeats=1)
    assert 0 <= best < 5 and times[best] > 0
    assert times[best] == min(t for t in times if t >= 0)
    plan.capture()
    # new pixels into the same buffers, then replay the captured graph
    imgs2 = [synth.image(i.shape[0], i.shape[1], 4000 + q, 11) if i.shape[2] == 3 else
             np.concatenate([synth.image(i.shape[0], i.shape[1], 4000 + q, 11),
                             np.zeros(i.shape[:2] + (1,), np.uint8)], -1)
             for q, i in enumerate(imgs)]
    plan.load([torch.from_numpy(i) for i in imgs2])
    plan.replay()
    plan.sync()
    check_against_single(wsm, plan, imgs2, Ks, seeds, 10, 0.0)
    plan.load([torch.from_numpy(i) for i in imgs])
    plan.replay()
    plan.replay()
    plan.sync()
    check_against_single(wsm, plan, imgs, Ks, seeds, 10, 0.0)


def test_more_than_one_launch_of_each_kernel(wsm):
    """70 images: five reduction launches (16 per launch) and two persistent
    launches (64 per launch) per step."""
    imgs = [synth.image(40 + (q % 6) * 8, 48 + (q % 4) * 8, 6000 + q, q % 13) for q in range(70)]
    Ks = [min(4 + (q % 3) * 6, len(np.unique(i.reshape(-1, 3), axis=0)))
          for q, i in enumerate(imgs)]
    seeds = [q * 31 for q in range(70)]
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=8)
    plan.load([torch.from_numpy(i) for i in imgs])
    plan.run()
    plan.sync()
    check_against_single(wsm, plan, imgs, Ks, seeds, 8, 0.0)


def test_an_image_with_fewer_colors_than_K_is_reported_and_skipped(wsm):
    imgs = [synth.image(64, 64, 1, 6), np.full((16, 16, 3), 3, np.uint8), synth.image(48, 40, 2, 9)]
    Ks = [16, 4, 16]
    seeds = [1, 2, 3]
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=10)
    plan.load([torch.from_numpy(i) for i in imgs])
    plan.run()
    with pytest.raises(wsm.WsmError, match="fewer unique colors than K"):
        plan.sync()
    wsm.wsm_sync_status(plan.handle)          # the report is cleared once read
    with wsm.Handle(16, 64 * 64) as h:
        for q in (0, 2):
            ref = single(wsm, h, imgs[q], Ks[q], seeds[q], 10, 0.0)
            got = plan.result(q)
            assert torch.equal(got["centers"], ref["centers"])
            assert torch.equal(got["index"], ref["index"])
    assert plan.result(1)["n_unique"] == 1


def test_stages_in_separate_calls_and_graphs_equal_one_call(wsm):
    imgs, Ks = uneven_batch(7, seed0=2500)
    seeds = [3 * q + 7 for q in range(len(imgs))]
    whole = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=10)
    whole.load([torch.from_numpy(i) for i in imgs])
    whole.run()
    whole.sync()
    parts = (wsm.STAGE_REDUCE | wsm.STAGE_INIT, wsm.STAGE_ITERATE,
             wsm.STAGE_MAP | wsm.STAGE_INDEX | wsm.STAGE_DISTORTION)
    split = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=10)
    split.load([torch.from_numpy(i) for i in imgs])
    # every stage in a call of its own, the MSE last
    for stages in (wsm.STAGE_REDUCE, wsm.STAGE_INIT, wsm.STAGE_ITERATE, wsm.STAGE_MAP,
                   wsm.STAGE_INDEX, wsm.STAGE_DISTORTION):
        split.run(stages)
    split.sync()
    # the MSE of the pipeline (from the final assignment) is the per-pixel
    # MSE of the index images, bit for bit
    per_pixel = wsm.wsm_distortion_batch(split.handle, split.images)
    for q in range(len(imgs)):
        assert per_pixel[q] == split.result(q)["mse"], q
    graphs = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=10)
    graphs.load([torch.from_numpy(i) for i in imgs])
    graphs.capture(parts)
    for q in range(3):
        graphs.replay(q)
    graphs.sync()
    for q in range(len(imgs)):
        a, b, c = whole.result(q), split.result(q), graphs.result(q)
        for r in (b, c):
            assert r["n_unique"] == a["n_unique"] and r["iters"] == a["iters"]
            assert r["mse"] == a["mse"]
            assert torch.equal(r["centers"], a["centers"]) and torch.equal(r["index"], a["index"])


def test_a_barrier_that_can_never_complete_times_out_and_the_handle_stays_usable(wsm):
    """Failure detection without a fault: the device barrier's bounded wait
    runs out, the status word says so, and the next call works."""
    from paper_1011_0093_gb300 import _native as N
    img = synth.image(64, 64, 3, 9)
    with wsm.Handle(16, 64 * 64) as h:
        rc = N.lib().wsm_selftest_barrier_timeout(h.ptr, 50, None)
        assert rc == -4                                          # WSM_E_TIMEOUT
        assert b"timed out" in N.lib().wsm_last_error()
        wsm.wsm_sync_status(h)                                   # the report was consumed
        q = wsm.quantize(torch.from_numpy(img).cuda(), 16, 1, max_iter=5, handle=h)
        ref = wsm.quantize(torch.from_numpy(img).cuda(), 16, 1, max_iter=5)
        assert torch.equal(q.centers, ref.centers) and torch.equal(q.index, ref.index)


def test_packed_load_and_fetch_equal_per_image_copies(wsm):
    """pack() + load() move all images' pixels in one copy and fetch() brings
    every index image, palette and MSE back in one copy per field; the parts
    sit at index_offset(i) / palette_offset(i) and equal the per-image
    results."""
    imgs, Ks = uneven_batch(6, seed0=3100)
    seeds = [11 * q + 1 for q in range(len(imgs))]
    a = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=6)
    a.load([torch.from_numpy(i) for i in imgs])
    a.run()
    a.sync()
    b = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=6)
    packed = b.pack(imgs)
    b.load(packed)
    b.run()
    out = b.host_outputs()
    b.fetch(out)
    b.sync()
    for q, img in enumerate(imgs):
        ra = a.result(q)
        h, w = img.shape[:2]
        K = Ks[q]
        i0, p0 = b.index_offset(q), b.palette_offset(q)
        assert i0 % 256 == 0 and (4 * p0) % 256 == 0
        idx = out["index"][i0:i0 + h * w].view(h, w)
        pal = out["centers"][p0:p0 + 4 * K].view(K, 4)
        assert torch.equal(idx, ra["index"].cpu())
        assert torch.equal(pal, ra["centers"].cpu())
        assert float(out["mse"][q]) == ra["mse"]
        assert torch.equal(b.images[q]["rgb"].cpu(), torch.from_numpy(img))


def test_weighing_the_images_changes_no_result(wsm):
    """wsm_weigh_batch (the image weights of the autotuner, for a fixed launch
    shape) moves blocks between the images of a launch; every image's
    results stay the same bit for bit."""
    imgs = [synth.image(64 + 40 * q, 80 + 24 * q, 700 + q, 3 * q) for q in range(6)]
    Ks = [16, 64, 32, 128, 48, 256]
    seeds = [5 + q for q in range(6)]
    plan = wsm.BatchPlan([i.shape for i in imgs], Ks, seeds, max_iter=8)
    plan.load([torch.from_numpy(i) for i in imgs])
    plan.run()
    plan.sync()
    before = [{k: (v.clone() if torch.is_tensor(v) else v) for k, v in plan.result(q).items()}
              for q in range(len(imgs))]
    wsm.wsm_set_launch_shape(plan.handle, 0)
    plan.weigh()
    plan.run()
    plan.sync()
    for q in range(len(imgs)):
        r = plan.result(q)
        assert torch.equal(r["centers"], before[q]["centers"])
        assert torch.equal(r["index"], before[q]["index"])
        assert r["mse"] == before[q]["mse"] and r["iters"] == before[q]["iters"]
