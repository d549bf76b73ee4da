"""The seeded synthetic inputs: the generator's random stream is splitmix64
as published, images are deterministic in their seed, and the workloads have
the sizes and unique-color statistics the benchmark and the parity tests are
described with (so that a change to the generator cannot pass unnoticed)."""
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64.txt")


def unique_counts(img):
    keys = ((img[..., 0].astype(np.uint32) << 16) | (img[..., 1].astype(np.uint32) << 8)
            | img[..., 2]).ravel()
    return np.unique(keys, return_counts=True)[1]


def test_stream_zero_is_the_published_splitmix64_sequence():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    want = [int(v, 16) for s, _, v in rows if int(s) == 0]
    got = [int(v) for v in synth.stream_u64(0, 0, len(want))]
    assert got == want


def test_images_are_deterministic_in_their_seed():
    a, b = synth.image(64, 48, 5, 9), synth.image(64, 48, 5, 9)
    assert a.dtype == np.uint8 and a.shape == (64, 48, 3) and np.array_equal(a, b)
    assert not np.array_equal(a, synth.image(64, 48, 6, 9))
    assert not np.array_equal(a, synth.image(64, 48, 5, 10))


def test_workload_unique_color_statistics():
    assert len(unique_counts(synth.plain_256())) == 47158
    want = [18049, 90475, 166487, 139669, 201197, 187190, 206792, 229024]
    for s, n_unique in enumerate(want):
        counts = unique_counts(synth.sweep_512_one(s))
        assert len(counts) == n_unique, s
        assert counts.sum() == 512 * 512
        assert 0.06 <= n_unique / counts.sum() <= 0.88    # 7% .. 87% unique
        # heavy-tailed frequencies: the most frequent 1% of the colors cover
        # at least 4x their share of the pixels (5% to 29% here) ...
        top = np.sort(counts)[::-1][:n_unique // 100]
        assert top.sum() >= 0.04 * counts.sum(), s
        # ... and with noise most colors occur once
        if s >= 2:
            assert (counts == 1).mean() > 0.7, s


def test_batch_sizes_are_log_uniform_within_bounds():
    sizes = synth.batch_sizes(3, 64, 256, 2048)
    sides = np.array(sizes).ravel()
    assert len(sizes) == 64 and sides.min() >= 256 and sides.max() <= 2048
    assert sides.min() < 400 and sides.max() > 1500     # spans the range
    assert sizes == synth.batch_sizes(3, 64, 256, 2048)


def test_tiny_images_take_few_levels():
    img = synth.tiny(40, 37, 50, 4)
    assert set(np.unique(img)) <= {0, 85, 170, 255}
    assert len(unique_counts(img)) <= 64
