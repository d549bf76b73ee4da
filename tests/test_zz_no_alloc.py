"""wsm_iterate_noalloc, the entry point for callers that cannot allocate
device memory (a plugin whose host program owns every device byte, a process
whose memory is already reserved by another allocator, a loop that cannot
take an allocation's implicit synchronisation).

It is called through the C ABI and must give what wsm_iterate gives on the
same inputs, within the tolerances of the parity tests (centers within 1e-4,
SSE within 1e-5 relative, memberships equal), on two calls in a row: the
second call runs on the scratch the first one left behind.  It also checks
that a call allocates nothing (free device memory unchanged), that handles of
other palette sizes do not disturb it, and that a failure found by a call
that did not synchronise is reported by the next one.  This file is
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


def test_noalloc_allocates_nothing(wsm):
    """After the first call on the device (which looks up the array's device
    address), a further call changes neither the driver's free device memory
    nor the caching allocator's reserved bytes."""
    img = synth.sweep_512_one(3)
    K = 64
    with wsm.Handle(256, img.shape[0] * img.shape[1]) as h:
        colors, counts, nu, c0, l0 = prepared(wsm, h, img, K, 4)
        c1, l1, c2, l2 = c0.clone(), l0.clone(), c0.clone(), l0.clone()
        wsm.wsm_iterate_noalloc(colors, counts, nu, K, c1, l1, 10, 0.0)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        it, _ = wsm.wsm_iterate_noalloc(colors, counts, nu, K, c2, l2, 10, 0.0)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert it == 10
        assert free1 == free0
        assert torch.cuda.memory_reserved() == reserved0
        assert torch.equal(c1, c2) and torch.equal(l1, l2)


def test_noalloc_unaffected_by_handles_of_other_palette_sizes(wsm):
    """A handle created for a small palette between two calls neither breaks
    the next call nor an earlier handle sized for K = 256."""
    img = synth.sweep_512_one(2)
    n = img.shape[0] * img.shape[1]
    with wsm.Handle(256, n) as big:
        colors, counts, nu, c0, l0 = prepared(wsm, big, img, 256, 8)
        c_ref, l_ref = c0.clone(), l0.clone()
        it_ref, tr_ref = wsm.wsm_iterate(big, colors, counts, nu, 256, c_ref, l_ref, 10, 0.0)
        ref = (it_ref, tr_ref, c_ref, l_ref)
        c, l = c0.clone(), l0.clone()
        assert_close(ref, (*wsm.wsm_iterate_noalloc(colors, counts, nu, 256, c, l, 10, 0.0),
                           c, l))
        with wsm.Handle(16, n) as small:
            s_col, s_cnt, s_nu, s_cen, s_lab = prepared(wsm, small, img, 16, 3)
            it, _ = wsm.wsm_iterate(small, s_col, s_cnt, s_nu, 16, s_cen, s_lab, 5, 0.0)
            assert it == 5
            c, l = c0.clone(), l0.clone()
            assert_close(ref, (*wsm.wsm_iterate_noalloc(colors, counts, nu, 256, c, l, 10, 0.0),
                               c, l))
        c, l = c0.clone(), l0.clone()
        it, tr = wsm.wsm_iterate(big, colors, counts, nu, 256, c, l, 10, 0.0)
        assert_close(ref, (it, tr, c, l))


def test_noalloc_reports_a_failure_of_an_unsynchronised_call_later(wsm):
    """A membership >= K found by a call that did not synchronise is reported
    by the next call that asks for results, once; the call after that, on
    valid inputs, succeeds."""
    img = synth.image(96, 80, 5, 6)
    K = 8
    with wsm.Handle(256, img.shape[0] * img.shape[1]) as h:
        colors, counts, nu, c0, l0 = prepared(wsm, h, img, K, 2)
        bad = l0.clone()
        bad[nu // 2] = 200
        assert wsm.wsm_iterate_noalloc(colors, counts, nu, K, c0.clone(), bad, 2, 0.0,
                                       sync=False) is None
        torch.cuda.synchronize()
        with pytest.raises(wsm.WsmError, match="INVAL"):
            wsm.wsm_iterate_noalloc(colors, counts, nu, K, c0.clone(), l0.clone(), 2, 0.0)
        it, _ = wsm.wsm_iterate_noalloc(colors, counts, nu, K, c0.clone(), l0.clone(), 2, 0.0)
        assert it == 2


def test_noalloc_rejects_sizes_beyond_its_scratch(wsm):
    colors = torch.zeros(4, dtype=torch.uint32, device="cuda")
    counts = torch.ones(4, dtype=torch.uint32, device="cuda")
    centers = torch.zeros((257, 4), dtype=torch.float32, device="cuda")
    labels = torch.zeros(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(wsm.WsmError, match="K must be in"):
        wsm.wsm_iterate_noalloc(colors, counts, 4, 257, centers, labels, 1, 0.0)
    with pytest.raises(wsm.WsmError, match="max_iter"):
        wsm.wsm_iterate_noalloc(colors, counts, 4, 4, centers, labels, 5000, 0.0)
