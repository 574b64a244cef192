"""Learned warm start: tensor-core GEMM, N-grid transforms, features, the network's forward
and backward against the float64 CPU reference (oracle/fno.py), training, and the gain of
the warm start in CG iterations with bounds unchanged."""
import numpy as np
import pytest

import microstructures as ms
from oracle import fno

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hb():
    import paper_1404_3614_gb300 as hb
    return hb


@pytest.fixture(scope="module")
def ctx(hb):
    c = hb.hom_create(0)
    yield c
    hb.hom_destroy(c)


def bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


@pytest.mark.parametrize("M,N,K,ta,tb", [(64, 64, 32, 0, 0), (37, 53, 71, 0, 0), (100, 9, 300, 1, 0),
                                         (5, 130, 17, 0, 1), (77, 33, 5000, 1, 1), (1, 1, 1, 0, 0)])
def test_gemm_bf16_matches_reference(hb, ctx, M, N, K, ta, tb):
    g = torch.Generator().manual_seed(M * 1000 + N)
    A = torch.randn((K, M) if ta else (M, K), generator=g, dtype=torch.float64)
    B = torch.randn((N, K) if tb else (K, N), generator=g, dtype=torch.float64)
    C0 = torch.randn((M, N), generator=g, dtype=torch.float64)
    ref = 1.5 * (bf16(A).T if ta else bf16(A)) @ (bf16(B).T if tb else bf16(B)) - 0.5 * C0
    dA, dB, dC = A.float().cuda(), B.float().cuda(), C0.float().cuda()
    hb.binding.hom_gemm_bf16(ctx, M, N, K, dA.data_ptr(), A.shape[1], ta, dB.data_ptr(), B.shape[1], tb,
                             dC.data_ptr(), N, 1.5, -0.5)
    torch.cuda.synchronize()
    got = dC.cpu().double()
    assert (got - ref).abs().max() <= 1e-5 * max(1.0, ref.abs().max()) * np.sqrt(K)


def test_grid_half_transforms(hb, ctx):
    N, B, ch = 15, 3, 4
    rng = np.random.default_rng(0)
    grid = rng.normal(size=(B, N, N, ch))
    dgrid = torch.from_numpy(grid).float().cuda()
    half = torch.empty((B, ch, N, (N + 1) // 2), dtype=torch.complex128, device="cuda")
    hb.binding.hom_grid_to_half(ctx, N, B, ch, dgrid.data_ptr(), half.data_ptr(), hb.HOM_FP64)
    torch.cuda.synchronize()
    ref = np.fft.fft2(np.moveaxis(grid, -1, 1), axes=(2, 3)) / N ** 2       # [B, ch, y, x] -> [ky, kx]
    assert np.abs(half.cpu().numpy() - ref[..., :(N + 1) // 2]).max() < 2e-6
    back = torch.empty_like(dgrid)
    hb.binding.hom_half_to_grid(ctx, N, B, ch, half.data_ptr(), back.data_ptr(), hb.HOM_FP64)
    torch.cuda.synchronize()
    assert np.abs(back.cpu().numpy() - grid).max() < 2e-5


def test_features_match_geometry(hb, ctx):
    probs = [ms.random_rectangles_2d(s, N=15) for s in range(4)]
    feat = torch.empty((4, 15, 15, 1), dtype=torch.float32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    hb.binding.hom_net_features(ctx, probs, feat.data_ptr(), ws.data_ptr(), ws.numel())
    f = feat.cpu().numpy()[..., 0]
    for i, p in enumerate(probs):
        a = p.inclusions[0].A[0, 0]
        j = np.arange(15)
        X, Y = np.meshgrid(j / 15.0, j / 15.0, indexing="xy")     # [y, x]
        inside = np.zeros_like(X, dtype=bool)
        for inc in p.inclusions:
            dx = X - inc.center[0]
            dy = Y - inc.center[1]
            dx -= np.round(dx)
            dy -= np.round(dy)
            inside |= (np.abs(dx) < inc.size[0] / 2) & (np.abs(dy) < inc.size[1] / 2)
        ref = np.where(inside, np.log10(a), 0.0)
        # points exactly on an interface may fall either way in float32
        assert np.mean(np.abs(f[i] - ref) > 1e-5) < 0.02


CFG = dict(N=15, cin=1, width=8, modes=3, layers=2, proj=16, cout=8)


def _net(hb, cfg, batch):
    c = hb.binding.net_config(**cfg)
    ctx = hb.hom_create(0)
    npar, wsb = hb.binding.hom_net_sizes(ctx, c, batch)
    return ctx, c, npar, wsb


def test_forward_and_gradient_match_cpu_reference(hb):
    batch = 3
    ctx, c, npar, wsb = _net(hb, CFG, batch)
    try:
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        hb.binding.hom_net_init(ctx, c, 7, params.data_ptr())
        g = torch.Generator().manual_seed(3)
        x = torch.randn((batch, 15, 15, 1), generator=g, dtype=torch.float64)
        t = torch.randn((batch, 15, 15, 8), generator=g, dtype=torch.float64) * 0.1
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        out = torch.empty((batch, 15, 15, 8), dtype=torch.float32, device="cuda")
        hb.binding.hom_net_forward(ctx, c, params.data_ptr(), batch, x.float().cuda().data_ptr(), out.data_ptr(),
                                   ws.data_ptr(), wsb)
        grad = torch.empty_like(params)
        dx, dt = x.float().cuda(), t.float().cuda()
        loss = hb.binding.hom_net_gradient(ctx, c, params.data_ptr(), batch, dx.data_ptr(), dt.data_ptr(),
                                           grad.data_ptr(), ws.data_ptr(), wsb)
        p64 = params.cpu().double()
        rloss, rgrad, rout = fno.loss_and_grad(CFG, p64, x, t)
        o = out.cpu().double()
        assert (o - rout).abs().max() <= 2e-2 * rout.abs().max()
        assert abs(loss - rloss) <= 2e-2 * rloss
        offs = fno.offsets(**CFG)
        G = grad.cpu().double()
        for name, val in offs.items():
            if name == "total":
                continue
            s, n = val
            a, b = G[s:s + n], rgrad[s:s + n]
            scale = max(b.abs().max().item(), 1e-12)
            assert (a - b).abs().max().item() <= 5e-2 * scale, (name, (a - b).abs().max().item(), scale)
    finally:
        hb.hom_destroy(ctx)


def test_training_reduces_loss(hb):
    batch = 8
    ctx, c, npar, wsb = _net(hb, CFG, batch)
    try:
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        hb.binding.hom_net_init(ctx, c, 11, params.data_ptr())
        m = torch.zeros_like(params)
        v = torch.zeros_like(params)
        grad = torch.zeros_like(params)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        g = torch.Generator(device="cuda").manual_seed(1)
        x = torch.randn((batch, 15, 15, 1), generator=g, device="cuda")
        t = torch.tanh(x.repeat(1, 1, 1, 8)) * 0.5
        loss = torch.zeros(1, device="cuda")
        losses = []
        for step in range(1, 201):
            hb.binding.hom_net_train_step(ctx, c, params.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(),
                                          step, 3e-3, batch, x.data_ptr(), t.data_ptr(), loss.data_ptr(),
                                          ws.data_ptr(), wsb)
            if step in (1, 200):
                losses.append(loss.item())
        assert losses[1] < 0.2 * losses[0], losses
    finally:
        hb.hom_destroy(ctx)


def test_warm_start_gain_and_bounds(hb):
    """Train on method-generated fields (N = 23 cells), then start CG from the network's
    projected, Rayleigh-Ritz-scaled prediction on held-out cells. Measured: the CG
    iterations with and without the network (the start never raises the energy error
    above that of x0 = 0), and the bounds, which stay the guaranteed ones."""
    from paper_1404_3614_gb300 import warmstart
    res = warmstart.train_and_evaluate(N=23, n_train=768, n_test=64, epochs=20, batch=32, width=16, modes=6,
                                       layers=4, proj=64, seed_train=1000, seed_test=100000, tol=1e-4,
                                       precision="mixed")
    print("warm-start gain:", res["iters_zero_mean"], "->", res["iters_warm_mean"], "iterations per cell")
    assert res["loss_last_epoch"] < 0.5 * res["loss_first_epoch"], res
    assert res["iters_warm_mean"] <= 1.02 * res["iters_zero_mean"], res
    assert res["max_rel_bound_diff"] < 2e-5, res
    assert res["ordering_ok"]
    assert res["net_only_gap_ratio_median"] >= 1.0 - 1e-6      # the network-only field is a looser valid bound
