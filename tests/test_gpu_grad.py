"""The differentiable weighted distortion (wsm_distortion_fwd / _bwd and the
torch.autograd.Function above them) against the oracle's FP64 D(C, X) and
its analytic gradient, and against FP64 central differences (h = 1e-3) of
the oracle's D on the coordinates whose perturbation changes no assignment.

Workload: a 512x512 image of the benchmark's generator, K = 64, the palette
of 10 GPU WSM iterations; pixels as float points with w_i = 1/N (then D is
the MSE of Eq. 2), and seeded random weights and 4-float strides.
Tolerances: D within 1e-5 relative; dD/dC within 1e-5 + 1e-4 |ref| (FP32
sums of small residuals in a fixed order); dD/dX within 1e-6 relative
(one FP32 product of a difference).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

K = 64


@pytest.fixture(scope="module")
def wsm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1011_0093_gb300 import build as B
    B.build()
    import paper_1011_0093_gb300 as w
    return w


@pytest.fixture(scope="module")
def problem(wsm):
    img = synth.image(512, 512, 41, 6)
    q = wsm.quantize(torch.from_numpy(img).cuda(), K, 5, max_iter=10, eps=0.0)
    C = q.centers[:, :3].contiguous()
    X = torch.from_numpy(img.reshape(-1, 3).astype(np.float32)).cuda()
    return img, X, C


def oracle_grad(X, w, C):
    return oracle.distortion_grad(X.cpu().numpy().astype(np.float64),
                                  w.cpu().numpy().astype(np.float64),
                                  C.cpu().numpy().astype(np.float64))


def run(wsm, X, C, w=None, assign=None, warm=False):
    Xg = X.clone().requires_grad_(True)
    Cg = C.clone().requires_grad_(True)
    D = wsm.weighted_distortion(Xg, Cg, w, assign=assign, warm_start=warm)
    D.backward()
    torch.cuda.synchronize()
    return float(D.detach()), Cg.grad.clone(), Xg.grad.clone()


def gaps(X, C):
    d = ((X.double()[:, None, :] - C.double()[None, :, :]) ** 2).sum(-1)
    s = torch.sort(d, dim=1).values
    return (s[:, 1] - s[:, 0]).cpu().numpy()


def test_forward_and_gradients_match_the_oracle(wsm, problem):
    _, X, C = problem
    n = X.shape[0]
    w = torch.full((n,), 1.0 / n, dtype=torch.float32, device="cuda")
    assign = torch.empty(n, dtype=torch.uint8, device="cuda")
    D, gC, gX = run(wsm, X, C, None, assign)
    Dr, dC, dX, a = oracle_grad(X, w, C)
    assert abs(D - Dr) <= 1e-5 * Dr
    clear = gaps(X, C) > 1e-3
    assert clear.mean() > 0.99
    assert np.array_equal(assign.cpu().numpy()[clear], a[clear])
    assert np.all(np.abs(gC.cpu().numpy() - dC) <= 1e-5 + 1e-4 * np.abs(dC))
    assert np.all(np.abs(gX.cpu().numpy() - dX)[clear] <= 1e-6 * np.abs(dX[clear]) + 1e-12)


def test_distortion_equals_the_plain_path_mse(wsm, problem):
    """With w_i = 1/N, D at the final palette is the MSE of Eq. 2 that the
    plain path (final assignment, mapping, wsm_distortion) reports."""
    img, X, _ = problem
    q = wsm.quantize(torch.from_numpy(img).cuda(), K, 5, max_iter=10, eps=0.0)
    D = float(wsm.weighted_distortion(X, q.centers[:, :3].contiguous()))
    assert abs(D - q.mse) <= 1e-5 * q.mse


def test_gradient_matches_fp64_central_differences(wsm, problem):
    _, X, C = problem
    n = X.shape[0]
    w = torch.full((n,), 1.0 / n, dtype=torch.float32, device="cuda")
    _, gC, gX = run(wsm, X, C)
    Xd, wd, Cd = (X.cpu().numpy().astype(np.float64), w.cpu().numpy().astype(np.float64),
                  C.cpu().numpy().astype(np.float64))
    _, _, _, a = oracle.distortion_grad(Xd, wd, Cd)
    h = 1e-3
    checked = 0
    for k in range(K):
        for c in range(3):
            Cp, Cm = Cd.copy(), Cd.copy()
            Cp[k, c] += h
            Cm[k, c] -= h
            Dp, _, _, ap = oracle.distortion_grad(Xd, wd, Cp)
            Dm, _, _, am = oracle.distortion_grad(Xd, wd, Cm)
            if not (np.array_equal(ap, a) and np.array_equal(am, a)):
                continue                     # a tie is crossed: not differentiable here
            fd = (Dp - Dm) / (2 * h)
            assert abs(float(gC[k, c]) - fd) <= 1e-5 + 1e-4 * abs(fd), (k, c)
            checked += 1
    assert checked >= 96
    rng = np.random.default_rng(3)
    checked = 0
    for i in rng.choice(n, 40, replace=False):
        for c in range(3):
            Xp, Xm = Xd[i:i + 1].copy(), Xd[i:i + 1].copy()
            Xp[0, c] += h
            Xm[0, c] -= h
            Dp, _, _, ap = oracle.distortion_grad(Xp, wd[i:i + 1], Cd)
            Dm, _, _, am = oracle.distortion_grad(Xm, wd[i:i + 1], Cd)
            if ap[0] != a[i] or am[0] != a[i]:
                continue
            fd = (Dp - Dm) / (2 * h)
            assert abs(float(gX[i, c]) - fd) <= 1e-6 * abs(fd) + 1e-12
            checked += 1
    assert checked >= 100


def test_weights_strides_and_warm_start(wsm, problem):
    _, X, C = problem
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(9)
    w = (torch.rand(n, generator=g) * 2.0 / n).cuda()
    X4 = torch.cat([X, torch.full((n, 1), 7.0, device="cuda")], 1).contiguous()
    C4 = torch.cat([C, torch.full((K, 1), -3.0, device="cuda")], 1).contiguous()
    D3, gC3, gX3 = run(wsm, X, C, w)
    D4, gC4, gX4 = run(wsm, X4, C4, w)
    Dr, dC, dX, _ = oracle_grad(X, w, C)
    assert abs(D3 - Dr) <= 1e-5 * Dr
    assert D4 == D3
    assert torch.equal(gC4[:, :3], gC3) and torch.all(gC4[:, 3] == 0)
    assert torch.equal(gX4[:, :3], gX3) and torch.all(gX4[:, 3] == 0)
    assert np.all(np.abs(gC3.cpu().numpy() - dC) <= 1e-5 + 1e-4 * np.abs(dC))
    # warm start from a stale assignment: the same minima, hence the same D
    # (up to the order-dependent FP32 sums where a tie picks another center)
    assign = torch.randint(0, K, (n,), dtype=torch.uint8, device="cuda")
    Dw, gCw, _ = run(wsm, X, C, w, assign=assign, warm=True)
    assert abs(Dw - D3) <= 1e-6 * D3
    clear = gaps(X, C) > 1e-3
    assign_cold = torch.empty(n, dtype=torch.uint8, device="cuda")
    run(wsm, X, C, w, assign=assign_cold)
    assert torch.equal(assign[torch.from_numpy(clear).cuda()],
                       assign_cold[torch.from_numpy(clear).cuda()])
    # run to run: identical bits
    D3b, gC3b, gX3b = run(wsm, X, C, w)
    assert D3b == D3 and torch.equal(gC3b, gC3) and torch.equal(gX3b, gX3)


def test_gradient_vanishes_at_a_lloyd_fixed_point(wsm):
    img = synth.image(256, 256, 0, 6)
    q = wsm.quantize(torch.from_numpy(img).cuda(), 16, 0, max_iter=300, eps=0.0)
    C = q.centers[:, :3].contiguous()
    X = torch.from_numpy(img.reshape(-1, 3).astype(np.float32)).cuda()
    _, gC, _ = run(wsm, X, C)
    n = X.shape[0]
    _, dC, _, _ = oracle_grad(X, torch.full((n,), 1.0 / n, device="cuda"), C)
    # at the fixed point c_k = fl32(mean of cluster k): |dD/dc_k| <= 2 W_k |c_k - mean_k|
    assert np.abs(dC).max() <= 2 * 2.0 ** -24 * 256
    assert float(gC.abs().max()) <= 2 * 2.0 ** -24 * 256 + 1e-5


def test_adam_refines_the_wsm_palette(wsm, problem):
    """200 Adam steps (lr 0.1) on the palette from 10 WSM iterations, with
    the assignment carried from step to step as the warm start."""
    _, X, C = problem
    n = X.shape[0]
    Cp = C.clone().requires_grad_(True)
    opt = torch.optim.Adam([Cp], lr=0.1)
    assign = torch.empty(n, dtype=torch.uint8, device="cuda")
    D0 = None
    for step in range(200):
        opt.zero_grad()
        D = wsm.weighted_distortion(X, Cp, assign=assign, warm_start=step > 0)
        D.backward()
        if D0 is None:
            D0 = float(D.detach())
        opt.step()
    D_end = float(wsm.weighted_distortion(X, Cp.detach(), assign=assign, warm_start=True))
    n64 = torch.full((n,), 1.0 / n, device="cuda")
    Dr_end, _, _, _ = oracle_grad(X, n64, Cp.detach())
    assert abs(D_end - Dr_end) <= 1e-5 * Dr_end
    assert D_end <= D0 * (1 + 1e-6)
    assert D_end < 0.99 * D0                # 10 WSM iterations leave room to improve


def test_graph_captured_adam_matches_the_eager_loop(wsm, problem):
    """The refinement step captured into a CUDA graph (forward, backward, a
    capturable Adam step) and replayed 50 times ends where 50 eager steps end."""
    import bench
    _, X, C = problem
    n = X.shape[0]
    h = wsm.Handle(K, 1, 1)
    assign = torch.empty(n, dtype=torch.uint8, device="cuda")
    wsm.weighted_distortion(X, C, assign=assign, handle=h)
    Cp = C.clone().requires_grad_(True)
    opt = torch.optim.Adam([Cp], lr=0.1)
    a_eager = assign.clone()
    for _ in range(50):
        opt.zero_grad()
        wsm.weighted_distortion(X, Cp, assign=a_eager, warm_start=True, handle=h).backward()
        opt.step()
    Cg, graph, a_graph = bench.adam_graph(wsm, X, C, assign, h)
    for _ in range(50):
        graph.replay()
    torch.cuda.synchronize()
    assert float((Cg.detach() - Cp.detach()).abs().max()) <= 1e-3
    d_eager = float(wsm.weighted_distortion(X, Cp.detach(), handle=h))
    d_graph = float(wsm.weighted_distortion(X, Cg.detach(), handle=h))
    assert abs(d_graph - d_eager) <= 1e-5 * d_eager
    h.close()


def test_empty_input_and_errors(wsm):
    C = torch.rand(8, 3, device="cuda") * 255
    X = torch.empty(0, 3, device="cuda")
    D = wsm.weighted_distortion(X, C)
    assert float(D) == 0.0
    with pytest.raises(wsm.WsmError, match="K out of"):
        wsm.weighted_distortion(torch.rand(4, 3, device="cuda"), torch.rand(300, 3, device="cuda"))
    with pytest.raises(ValueError):
        wsm.weighted_distortion(torch.rand(4, 5, device="cuda"), C)
