"""wsm_iterate_noalloc, the entry point for callers that cannot allocate
device memory (a plugin whose host program owns every device byte, a process
whose memory is already reserved by another allocator, a loop that cannot
take an allocation's implicit synchronisation).

It is called through the C ABI and must give what wsm_iterate gives on the
same inputs, within the tolerances of the parity tests (centers within 1e-4,
SSE within 1e-5 relative, memberships equal), on two calls in a row: the
second call runs on the scratch the first one left behind.  This file is
collected last so that a stop at the first failure has run everything else.
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


def prepared(wsm, h, img, K, seed):
    """Unique colors and initial state from the existing entry points."""
    n = img.shape[0] * img.shape[1]
    colors = torch.empty(n, dtype=torch.uint32, device="cuda")
    counts = torch.empty(n, dtype=torch.uint32, device="cuda")
    nu = wsm.wsm_reduce(h, torch.from_numpy(img).cuda(), colors, counts)
    colors, counts = colors[:nu], counts[:nu]
    centers = torch.empty((K, 4), dtype=torch.float32, device="cuda")
    labels = torch.empty(nu, dtype=torch.uint8, device="cuda")
    wsm.wsm_init(h, colors, nu, K, seed, centers, labels)
    torch.cuda.synchronize()
    return colors, counts, nu, centers, labels


def assert_close(ref, got):
    (it_r, tr_r, c_r, l_r), (it_g, tr_g, c_g, l_g) = ref, got
    assert it_g == it_r
    assert np.all(np.abs(np.array(tr_g) - np.array(tr_r)) <= 1e-5 * np.array(tr_r))
    assert float((c_g[:, :3] - c_r[:, :3]).abs().max()) <= 1e-4
    assert torch.equal(l_g, l_r)


@pytest.mark.parametrize("img_fn,K,max_iter,eps", [
    (lambda: synth.sweep_512_one(7), 256, 10, 0.0),
    (synth.plain_256, 16, 100, 1e-4),
])
def test_noalloc_matches_wsm_iterate_twice(wsm, img_fn, K, max_iter, eps):
    img = img_fn()
    with wsm.Handle(256, img.shape[0] * img.shape[1]) as h:
        colors, counts, nu, c0, l0 = prepared(wsm, h, img, K, 11)
        c_ref, l_ref = c0.clone(), l0.clone()
        it_ref, tr_ref = wsm.wsm_iterate(h, colors, counts, nu, K, c_ref, l_ref, max_iter, eps)
        ref = (it_ref, tr_ref, c_ref, l_ref)
    for _ in range(2):
        c, l = c0.clone(), l0.clone()
        it, tr = wsm.wsm_iterate_noalloc(colors, counts, nu, K, c, l, max_iter, eps)
        assert_close(ref, (it, tr, c, l))


def test_noalloc_rejects_sizes_beyond_its_scratch(wsm):
    colors = torch.zeros(4, dtype=torch.uint32, device="cuda")
    counts = torch.ones(4, dtype=torch.uint32, device="cuda")
    centers = torch.zeros((257, 4), dtype=torch.float32, device="cuda")
    labels = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(wsm.WsmError, match="K must be in"):
        wsm.wsm_iterate_noalloc(colors, counts, 4, 257, centers, labels, 1, 0.0)
    with pytest.raises(wsm.WsmError, match="max_iter"):
        wsm.wsm_iterate_noalloc(colors, counts, 4, 4, centers, labels, 5000, 0.0)
