"""The native serving loop (wsm_server_*): continuous batching over lanes,
admission by device-memory footprint, and results that are the same for a
request alone and in a mix of other requests -- bit for bit, and equal to
the one-image path (quantize) -- and that match the oracle's whole run
(Celebi, arXiv:1011.0093, Algorithm 2 per request) under the rules of
tests/parity.py."""
import threading

import numpy as np
import pytest
import torch

import synth
from parity import compare_whole_path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wsm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1011_0093_gb300 import build as B
    B.build()
    import paper_1011_0093_gb300 as w
    return w


def pinned(img):
    return torch.from_numpy(np.ascontiguousarray(img)).pin_memory()


def one_image_path(wsm, img, K, seed, max_iter=10, eps=0.0):
    q = wsm.quantize(torch.from_numpy(np.ascontiguousarray(img)).cuda(), K, seed,
                     max_iter=max_iter, eps=eps)
    return q.centers.cpu(), q.index.cpu(), q.mse, q.n_unique, q.iters


def same(res, ref):
    c, idx, mse, nu, it = ref
    return (torch.equal(res["palette"], c) and torch.equal(res["index"], idx)
            and res["mse"] == mse and res["n_unique"] == nu and res["iters"] == it)


def mix(count, seed0):
    rng = np.random.default_rng(seed0)
    out = []
    for q in range(count):
        hh, ww = (int(round(2 ** rng.uniform(5, 9.5))) for _ in range(2))
        out.append((synth.image(max(hh, 8), max(ww, 8), seed0 + q, int(rng.integers(0, 25))),
                    int(rng.choice([16, 64, 256])), int(rng.integers(0, 1 << 30))))
    return out


def test_a_request_gives_the_same_result_alone_and_in_a_mix(wsm):
    probe = synth.image(300, 260, 77, 9)
    K, seed = 64, 4242
    ref = one_image_path(wsm, probe, K, seed)
    others = mix(40, 100)
    with wsm.Server(lanes=2, slots_per_lane=8, arena_bytes=1 << 30) as srv:
        alone = srv.wait(srv.submit(pinned(probe), K, seed))
        assert same(alone, ref)
        pend = []
        for q, (img, k, s) in enumerate(others):
            pend.append((srv.submit(pinned(img), k, s), (img, k, s)))
            if q in (7, 19, 33):
                pend.append((srv.submit(pinned(probe), K, seed), None))
        results = [(srv.wait(p), meta) for p, meta in pend]
        st = srv.stats()
    assert st["completed"] == st["submitted"] == len(others) + 4 and st["failed"] == 0
    assert st["batches"] > 2 and st["max_in_flight"] > 1
    for res, meta in results:
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
        if meta is None:
            assert same(res, ref)
    for res, (img, k, s) in [(r, m) for r, m in results if m is not None][::7]:
        assert same(res, one_image_path(wsm, img, k, s))


def test_admission_respects_the_arena(wsm):
    imgs = [synth.image(256, 256, 300 + q, 12) for q in range(24)]
    per_request = 256 * 256 * 14 + 4096
    arena = 4 * per_request + (1 << 20)          # room for about four requests at a time
    with wsm.Server(lanes=2, slots_per_lane=16, arena_bytes=arena) as srv:
        pend = [srv.submit(pinned(im), 16, q) for q, im in enumerate(imgs)]
        res = [srv.wait(p) for p in pend]
        st = srv.stats()
        with pytest.raises(wsm.WsmError, match="more device memory than the arena"):
            srv.submit(pinned(synth.image(1024, 1024, 1, 3)), 16, 0)
    assert st["arena_peak"] <= st["arena_bytes"]
    assert st["max_in_flight"] <= 5
    for im, q, r in zip(imgs, range(len(imgs)), res):
        if q % 6 == 0:
            assert same(r, one_image_path(wsm, im, 16, q))


def test_settings_failures_and_concurrent_submitters(wsm):
    jobs = [(synth.image(120, 90, 500 + q, 7), 16, q, 10 if q % 3 else 50, 0.0 if q % 3 else 1e-4)
            for q in range(18)]
    few = np.full((20, 20, 3), 5, np.uint8)
    out = {}
    with wsm.Server(lanes=3, slots_per_lane=4, arena_bytes=256 << 20) as srv:
        def submitter(part):
            for q in part:
                img, K, s, it, eps = jobs[q]
                out[q] = srv.submit(pinned(img), K, s, max_iter=it, eps=eps)
        threads = [threading.Thread(target=submitter, args=(range(t, len(jobs), 3),))
                   for t in range(3)]
        bad = srv.submit(pinned(few), 4, 1)
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        with pytest.raises(wsm.WsmError, match="fewer unique colors than K"):
            srv.wait(bad)
        res = {q: srv.wait(p) for q, p in out.items()}
    for q, (img, K, s, it, eps) in enumerate(jobs):
        assert same(res[q], one_image_path(wsm, img, K, s, it, eps)), q


def test_served_results_match_the_oracle(wsm):
    """Requests of each palette size the server is driven with (K = 16, 64,
    256), one of them of the largest size the server admits (4096 x 4096),
    submitted in a mix with other requests, each compared with the oracle's
    whole run of its image, K and seed: N', the palette and iteration count
    while the runs agree, every pixel's index (its color's membership), the
    index image and the MSE (tests/parity.py)."""
    checks = [(synth.image(4096, 4096, 91, 8), 256, 17),
              (synth.image(300, 260, 92, 9), 16, 5),
              (synth.image(512, 384, 93, 14), 64, 6),
              (synth.sweep_512_one(4), 256, 7)]
    others = mix(24, 300)
    with wsm.Server(lanes=2, slots_per_lane=8, arena_bytes=2 << 30) as srv:
        pend = []
        for q, (img, k, s) in enumerate(others):
            pend.append((srv.submit(pinned(img), k, s), None))
            if q % 6 == 2:
                img_c, k_c, s_c = checks[q // 6]
                pend.append((srv.submit(pinned(img_c), k_c, s_c), q // 6))
        results = [(srv.wait(p), m) for p, m in pend]
        st = srv.stats()
    assert st["failed"] == 0 and st["max_in_flight"] > 1
    seen = set()
    with wsm.Handle(256, 1 << 24, 1 << 24) as h:
        for res, m in results:
            if m is None:
                continue
            img, K, seed = checks[m]
            got = dict(centers=res["palette"], iters=res["iters"], mse=res["mse"],
                       index=res["index"], n_unique=res["n_unique"])
            compare_whole_path(wsm, h, img, K, seed, 10, 0.0, got=got,
                               name=f"served {img.shape[0]}x{img.shape[1]} K={K}")
            seen.add(m)
    assert seen == set(range(len(checks)))
