"""The batched persistent launch (wsm_iterate_batch, wsm_map_batch) gives, for
every image of a batch, exactly what the single-image calls give: the same
centers, memberships, iteration counts and index images, bit for bit (the
per-image computation is identical and every reduction is exact), for images
of uneven sizes, palettes and convergence lengths."""
import numpy as np
import pytest
import torch

import oracle
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


def prepare(wsm, h, img, K, seed):
    n = img.shape[0] * img.shape[1]
    rgb = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    colors = torch.empty(n, dtype=torch.uint32, device="cuda")
    counts = torch.empty(n, dtype=torch.uint32, device="cuda")
    nu = wsm.wsm_reduce(h, rgb, colors, counts)
    colors, counts = colors[:nu], counts[:nu]
    centers = torch.empty((K, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, colors, nu, K, seed, centers, labels)
    index = torch.empty(img.shape[:2], dtype=torch.uint8, device="cuda")
    return dict(rgb=rgb, colors=colors, counts=counts, n_unique=nu, K=K, centers=centers,
                labels=labels, index=index)


def clone(im):
    out = dict(im)
    for k in ("centers", "labels", "index"):
        out[k] = im[k].clone()
    return out


BATCH = [((512, 512), 7, 24, 256), ((256, 256), 0, 6, 16), ((96, 80), 5, 6, 16),
         ((300, 211), 8, 9, 64), ((512, 512), 2, 7, 128), ((64, 64), 2, 6, 8),
         ((700, 300), 11, 15, 32), ((40, 37), 50, 0, 5)]


@pytest.mark.parametrize("max_iter,eps", [(10, 0.0), (100, 1e-4)])
def test_batch_equals_single_calls(wsm, max_iter, eps):
    imgs = [synth.image(hw[0], hw[1], seed, noise) if noise else synth.tiny(hw[0], hw[1], seed, 4)
            for hw, seed, noise, _ in BATCH]
    with wsm.Handle(256, 512 * 512) as h:
        wsm.wsm_reserve_batch(h, len(BATCH))
        items = [prepare(wsm, h, img, K, 100 + q) for q, (img, (_, _, _, K)) in
                 enumerate(zip(imgs, BATCH))]
        single = [clone(im) for im in items]
        iters_single = []
        for im in single:
            done, _ = wsm.wsm_iterate(h, im["colors"], im["counts"], im["n_unique"], im["K"],
                                      im["centers"], im["labels"], max_iter, eps)
            iters_single.append(done)
            wsm.wsm_map(h, im["rgb"], im["colors"], im["n_unique"], im["centers"], im["K"],
                        im["labels"], im["index"])
        batch = [clone(im) for im in items]
        iters_batch = wsm.wsm_iterate_batch(h, batch, max_iter, eps)
        wsm.wsm_map_batch(h, batch)
        wsm.wsm_sync_status(h)
    assert iters_batch == iters_single
    if eps > 0:
        assert len(set(iters_single)) > 1          # uneven convergence lengths in one launch
    for a, b in zip(single, batch):
        assert torch.equal(a["centers"], b["centers"])
        assert torch.equal(a["labels"], b["labels"])
        assert torch.equal(a["index"], b["index"])


def test_batch_matches_oracle_and_more_than_one_launch(wsm):
    """A batch of 70 small images spans two launches (64 per launch); each
    image's index image matches the oracle's wherever no near-tie decides."""
    specs = [(48 + (q % 7) * 8, 40 + (q % 5) * 8, 200 + q, q % 9, 4 + (q % 13)) for q in range(70)]
    imgs = [synth.image(hh, ww, seed, noise) for hh, ww, seed, noise, _ in specs]
    with wsm.Handle(64, 112 * 72) as h:
        wsm.wsm_reserve_batch(h, len(specs))
        items = [prepare(wsm, h, img, K, 7 + q) for q, (img, (*_, K)) in
                 enumerate(zip(imgs, specs))]
        iters = wsm.wsm_iterate_batch(h, items, 10, 0.0)
        wsm.wsm_map_batch(h, items)
        wsm.wsm_sync_status(h)
    assert iters == [10] * len(specs)
    for img, im, (*_, K), q in zip(imgs, items, specs, range(len(specs))):
        ref = oracle.quantize(img, K, 7 + q, 10, 0.0)
        gc = im["centers"].cpu().numpy()[:, :3]
        best, second, _ = oracle.exhaustive(ref["colors"], ref["centers"])
        if np.all(second - best > 1e-3):
            assert np.abs(gc - ref["centers"]).max() <= 1e-4
            assert np.array_equal(im["index"].cpu().numpy().ravel(), ref["index"])


def test_batch_rejects_more_items_than_slots(wsm):
    img = synth.image(32, 32, 1, 3)
    with wsm.Handle(16, 32 * 32) as h:
        items = [prepare(wsm, h, img, 4, q) for q in range(2)]
        with pytest.raises(wsm.WsmError, match="slots"):
            wsm.wsm_iterate_batch(h, items, 5, 0.0)


def test_reduce_init_distortion_batch_equal_single_calls(wsm):
    """wsm_reduce_batch, wsm_init_batch and wsm_distortion_batch give each
    image what wsm_reduce, wsm_init and wsm_distortion give it, bit for bit,
    over 21 images (two reduction launches of at most 16), 3- and 4-byte
    pixels, and images with one color or every pixel distinct."""
    imgs = [synth.image(hh, ww, 300 + q, q % 11) for q, (hh, ww) in
            enumerate([(512, 512), (256, 256), (96, 80), (300, 211), (64, 64), (700, 300),
                       (40, 37), (128, 96), (17, 3), (200, 200), (33, 65), (256, 128),
                       (90, 90), (48, 160), (120, 77), (64, 256), (31, 31), (150, 100)])]
    imgs.append(np.full((20, 30, 3), 77, np.uint8))                        # one color
    ramp = np.arange(64 * 64, dtype=np.uint32) * 4099
    imgs.append(np.stack([ramp >> 16, (ramp >> 8) & 255, ramp & 255], -1)
                .astype(np.uint8).reshape(64, 64, 3))                      # all distinct
    rgba = np.concatenate([synth.image(100, 90, 9, 9), np.full((100, 90, 1), 255, np.uint8)], -1)
    imgs.append(rgba)                                                      # 4-byte pixels
    seeds = [1000 + 17 * q for q in range(len(imgs))]
    with wsm.Handle(256, 512 * 512) as h:
        wsm.wsm_reserve_batch(h, len(imgs))
        batch = []
        for img in imgs:
            n = img.shape[0] * img.shape[1]
            batch.append(dict(rgb=torch.from_numpy(np.ascontiguousarray(img)).cuda(),
                              colors=torch.empty(n, dtype=torch.uint32, device="cuda"),
                              counts=torch.empty(n, dtype=torch.uint32, device="cuda"),
                              labels=torch.empty(n, dtype=torch.uint8, device="cuda"),
                              index=torch.empty(img.shape[:2], dtype=torch.uint8,
                                                device="cuda")))
        nus = wsm.wsm_reduce_batch(h, batch)
        assert nus[-3] == 1 and nus[-2] == 64 * 64
        Ks = [min(256, 4 + 13 * q, nu) for q, nu in enumerate(nus)]
        for im, K in zip(batch, Ks):
            im["K"] = K
            im["centers"] = torch.empty((K, 4), dtype=torch.float32, device="cuda")
        wsm.wsm_init_batch(h, batch, seeds)
        init_c = [im["centers"].clone() for im in batch]
        init_l = [im["labels"][:nu].clone() for im, nu in zip(batch, nus)]
        wsm.wsm_iterate_batch(h, batch, 3, 0.0)
        wsm.wsm_map_batch(h, batch)
        mse_b = wsm.wsm_distortion_batch(h, batch)
        d_mse = torch.zeros(len(batch), dtype=torch.float64, device="cuda")
        wsm.wsm_distortion_batch(h, batch, d_mse=d_mse, sync=False)
        wsm.wsm_sync_status(h)
        for q, (im, nu) in enumerate(zip(batch, nus)):
            n = im["colors"].numel()
            colors = torch.empty(n, dtype=torch.uint32, device="cuda")
            counts = torch.empty(n, dtype=torch.uint32, device="cuda")
            assert wsm.wsm_reduce(h, im["rgb"], colors, counts) == nu
            assert torch.equal(colors[:nu], im["colors"][:nu])
            assert torch.equal(counts[:nu], im["counts"][:nu])
            centers = torch.empty_like(im["centers"])
            labels = torch.full((nu,), 9, dtype=torch.uint8, device="cuda")
            wsm.wsm_init(h, colors[:nu], nu, Ks[q], seeds[q], centers, labels)
            assert torch.equal(centers, init_c[q])
            assert torch.equal(labels, init_l[q])
            m = wsm.wsm_distortion(h, im["rgb"], im["centers"], Ks[q], im["index"])
            assert m == mse_b[q] == float(d_mse[q])
    for q in (0, len(imgs) - 1):
        ref_colors, ref_counts = oracle.unique(imgs[q])
        assert np.array_equal(batch[q]["colors"][:nus[q]].cpu().numpy(), ref_colors)
        assert np.array_equal(batch[q]["counts"][:nus[q]].cpu().numpy(), ref_counts)


@pytest.mark.parametrize("path", [1, 2])
def test_reduce_batch_both_paths_match_the_oracle(wsm, path):
    """A reduction launch of 5 images of uneven sizes (one empty-ish in colors,
    one 4-byte, one unaligned size) through either way of filling the
    histograms, image by image against the oracle."""
    imgs = [synth.image(1024, 768, 71, 20), synth.image(333, 517, 72, 3),
            np.full((64, 64, 3), 9, np.uint8), synth.image(1500, 1100, 73, 11),
            np.concatenate([synth.image(257, 263, 74, 7), np.full((257, 263, 1), 1, np.uint8)],
                           -1)]
    with wsm.Handle(256, 1500 * 1100) as h:
        wsm.wsm_reserve_batch(h, len(imgs))
        wsm.wsm_set_reduce_path(h, path)
        batch = []
        for img in imgs:
            n = img.shape[0] * img.shape[1]
            batch.append(dict(rgb=torch.from_numpy(np.ascontiguousarray(img)).cuda(),
                              colors=torch.empty(n, dtype=torch.uint32, device="cuda"),
                              counts=torch.empty(n, dtype=torch.uint32, device="cuda"),
                              labels=torch.empty(n, dtype=torch.uint8, device="cuda"),
                              index=torch.empty(img.shape[:2], dtype=torch.uint8,
                                                device="cuda")))
        for _ in range(2):                  # the second launch reuses the cleared scratch
            nus = wsm.wsm_reduce_batch(h, batch)
            for q, img in enumerate(imgs):
                rc, rn = oracle.unique(img)
                assert nus[q] == len(rc)
                assert np.array_equal(batch[q]["colors"][:nus[q]].cpu().numpy(), rc)
                assert np.array_equal(batch[q]["counts"][:nus[q]].cpu().numpy(), rn)


def test_quantize_batch_equals_quantize(wsm):
    imgs = [synth.image(hh, ww, 40 + q, 3 + 4 * q) for q, (hh, ww) in
            enumerate([(256, 256), (120, 200), (64, 48)])]
    seeds = [5, 6, 7]
    outs = wsm.quantize_batch([torch.from_numpy(i).cuda() for i in imgs], 32, seeds,
                              max_iter=100, eps=1e-4)
    for img, s, qb in zip(imgs, seeds, outs):
        q1 = wsm.quantize(torch.from_numpy(img).cuda(), 32, s, max_iter=100, eps=1e-4)
        assert q1.n_unique == qb.n_unique and q1.iters == qb.iters
        assert torch.equal(q1.centers, qb.centers)
        assert torch.equal(q1.index, qb.index)
        assert torch.equal(q1.labels, qb.labels)
        assert q1.mse == qb.mse
