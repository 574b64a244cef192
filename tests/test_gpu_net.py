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
    hb.binding.hom_grid_to_half(ctx, 2, N, B, ch, dgrid.data_ptr(), half.data_ptr(), hb.HOM_FP64)
    torch.cuda.synchronize()
    ref = np.fft.fft2(np.moveaxis(grid, -1, 1), axes=(2, 3)) / N ** 2       # [B, ch, y, x] -> [ky, kx]
    assert np.abs(half.cpu().numpy() - ref[..., :(N + 1) // 2]).max() < 2e-6
    back = torch.empty_like(dgrid)
    hb.binding.hom_half_to_grid(ctx, 2, N, B, ch, half.data_ptr(), back.data_ptr(), hb.HOM_FP64)
    torch.cuda.synchronize()
    assert np.abs(back.cpu().numpy() - grid).max() < 2e-5


@pytest.mark.parametrize("N,prec", [(9, "fp64"), (15, "fp32"), (41, "fp64")])
def test_grid_half_transforms_3d(hb, ctx, N, prec):
    B, ch = 2, 3
    rng = np.random.default_rng(N)
    grid = rng.normal(size=(B, N, N, N, ch))
    dgrid = torch.from_numpy(grid).float().cuda()
    Nh = (N + 1) // 2
    cdt, p = (torch.complex128, hb.HOM_FP64) if prec == "fp64" else (torch.complex64, hb.HOM_FP32)
    half = torch.empty((B, ch, N, N, Nh), dtype=cdt, device="cuda")
    hb.binding.hom_grid_to_half(ctx, 3, N, B, ch, dgrid.data_ptr(), half.data_ptr(), p)
    torch.cuda.synchronize()
    ref = np.fft.fftn(np.moveaxis(grid, -1, 1), axes=(2, 3, 4)) / N ** 3   # [B, ch, kz, ky, kx]
    scale = np.abs(ref).max()
    assert np.abs(half.cpu().numpy() - ref[..., :Nh]).max() < 2e-6 * N * scale
    nws = hb.binding.hom_half_to_grid_workspace_size(ctx, 3, N, B, ch)
    assert nws == B * ch * N * N * Nh * 8
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    back = torch.empty_like(dgrid)
    hb.binding.hom_half_to_grid(ctx, 3, N, B, ch, half.data_ptr(), back.data_ptr(), p, ws.data_ptr(), nws)
    torch.cuda.synchronize()
    assert np.abs(back.cpu().numpy() - grid).max() < 1e-5 * N
    with pytest.raises(hb.HombError):
        hb.binding.hom_half_to_grid(ctx, 3, N, B, ch, half.data_ptr(), back.data_ptr(), p, ws.data_ptr(), nws - 8)


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
        ref = np.where(inside, np.log10(a), 0.0) / 3.0          # log10(a) / 3
        # points exactly on an interface may fall either way in float32
        assert np.mean(np.abs(f[i] - ref) > 1e-5) < 0.02


def test_features_3d_match_geometry(hb, ctx):
    N = 13
    probs = [ms.random_spheres_3d(s, N=N, n_balls=6, phi=0.25, contrast=30.0) for s in range(3)]
    feat = torch.empty((3, N, N, N, 1), dtype=torch.float32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    hb.binding.hom_net_features(ctx, probs, feat.data_ptr(), ws.data_ptr(), ws.numel())
    f = feat.cpu().numpy()[..., 0]
    j = np.arange(N) / N
    Z, Y, X = np.meshgrid(j, j, j, indexing="ij")      # [z, y, x]
    for i, p in enumerate(probs):
        ref = np.full(X.shape, np.log10(np.trace(p.A0) / 3) / 3.0)
        for inc in p.inclusions:
            r2 = np.zeros_like(X)
            for a, C_ in enumerate((X, Y, Z)):
                dd = C_ - inc.center[a]
                r2 += (dd - np.round(dd)) ** 2
            ref = np.where(r2 < inc.size[0] ** 2, np.log10(np.trace(inc.A) / 3) / 3.0, ref)
        # points exactly on an interface may fall either way in float32
        assert np.mean(np.abs(f[i] - ref) > 1e-5) < 0.01


CFG = dict(N=15, cin=1, width=8, modes=3, layers=2, proj=16, cout=8)
CFG3 = dict(N=9, cin=1, width=6, modes=2, layers=2, proj=20, cout=18, d=3)


def _net(hb, cfg, batch):
    c = hb.binding.net_config(**cfg)
    ctx = hb.hom_create(0)
    npar, wsb = hb.binding.hom_net_sizes(ctx, c, batch)
    return ctx, c, npar, wsb


@pytest.mark.parametrize("cfg", [CFG, CFG3], ids=["2d", "3d"])
def test_forward_and_gradient_match_cpu_reference(hb, cfg):
    batch = 3
    CFG = cfg
    ctx, c, npar, wsb = _net(hb, CFG, batch)
    grid = (CFG["N"],) * CFG.get("d", 2)
    try:
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        assert npar == fno.offsets(**CFG)["total"]
        hb.binding.hom_net_init(ctx, c, 7, params.data_ptr())
        g = torch.Generator().manual_seed(3)
        x = torch.randn((batch,) + grid + (1,), generator=g, dtype=torch.float64)
        t = torch.randn((batch,) + grid + (CFG["cout"],), generator=g, dtype=torch.float64) * 0.1
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        out = torch.empty((batch,) + grid + (CFG["cout"],), dtype=torch.float32, device="cuda")
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


def test_forward_3d_large_batch_matches_single(hb):
    """B * N^2 = 67240 rows of x transforms (above the 65535 grid limit, chunked): each
    sample's output equals the output of the same sample run alone."""
    cfg = dict(N=41, cin=1, width=4, modes=3, layers=1, proj=8, cout=2, d=3)
    B, N = 40, 41
    ctx, c, npar, wsb = _net(hb, cfg, B)
    try:
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        hb.binding.hom_net_init(ctx, c, 5, params.data_ptr())
        x = torch.randn((B, N, N, N, 1), generator=torch.Generator(device="cuda").manual_seed(2), device="cuda")
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        out = torch.empty((B, N, N, N, 2), dtype=torch.float32, device="cuda")
        hb.binding.hom_net_forward(ctx, c, params.data_ptr(), B, x.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb)
        one = torch.empty((1, N, N, N, 2), dtype=torch.float32, device="cuda")
        for i in (0, 23, 39):
            xi = x[i:i + 1].contiguous()
            hb.binding.hom_net_forward(ctx, c, params.data_ptr(), 1, xi.data_ptr(), one.data_ptr(), ws.data_ptr(), wsb)
            torch.cuda.synchronize()
            assert (one[0] - out[i]).abs().max().item() <= 1e-5 * out[i].abs().max().item(), i
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


def test_warm_start_3d_small(hb):
    """The 3D warm start end to end on small grids: fields from hom_bounds_io at N = 15,
    training, then starts on held-out N = 15 cells and on an N = 23 cell (the network runs
    on a grid it was not trained on). Whatever the prediction, the bounds stay guaranteed:
    each run's upper bound dominates every run's lower bound, the network-only field gives
    a valid, looser bound."""
    from paper_1404_3614_gb300 import warmstart
    res = warmstart.train_and_evaluate_3d(N_train=15, N_eval=23, n_train=48, n_test=3, eval_seeds=(5,), epochs=6,
                                          batch=4, width=8, modes=3, layers=2, proj=24, tol=1e-4, chunk=8)
    print("3D warm start:", res["test_iters_zero_mean"], "->", res["test_iters_warm_mean"], "eval", res["eval"])
    assert res["loss_last_epoch"] < res["loss_first_epoch"], res
    assert res["test_ordering_ok"], res
    assert res["test_max_rel_bound_diff"] < 1e-2, res
    for r in res["eval"]:
        assert r["net_only_gap_ratio"] >= 1.0 - 1e-6, r
    assert res["test_net_only_gap_ratio_median"] >= 1.0 - 1e-6, res


def _resample_ref(x, d, nf, nt):
    """out(k) = in(k) for k held by grid nf (no Nyquist rows), else 0; numpy loops."""
    def sf(i, n):
        return i if i <= (n - 1) // 2 else i - n

    def holds(k, n):
        return -((n - 1) // 2) <= k <= (n - 1) // 2
    count = x.shape[0]
    tz = nt[2] if d == 3 else 1
    fz = nf[2] if d == 3 else 1
    out = np.zeros((count, tz, nt[1], (nt[0] + 1) // 2), dtype=x.dtype)
    xi = x.reshape(count, fz, nf[1], (nf[0] + 1) // 2)
    for iz in range(tz):
        kz = sf(iz, tz) if d == 3 else 0
        for iy in range(nt[1]):
            ky = sf(iy, nt[1])
            for kx in range((nt[0] + 1) // 2):
                nyq = (nt[1] % 2 == 0 and ky == -nt[1] // 2) or (d == 3 and tz % 2 == 0 and kz == -tz // 2)
                if kx < (nf[0] + 1) // 2 and holds(ky, nf[1]) and (d != 3 or holds(kz, fz)) and not nyq:
                    out[:, iz, iy, kx] = xi[:, kz % fz, ky % nf[1], kx]
    return out


@pytest.mark.parametrize("d,nf,nt,prec", [(3, (9, 9, 9), (15, 13, 11), "fp64"), (3, (15, 13, 11), (9, 9, 9), "fp32"),
                                          (2, (8, 8), (11, 11), "fp64"), (2, (11, 9), (6, 10), "fp64")])
def test_resample_fields(hb, ctx, d, nf, nt, prec):
    rng = np.random.default_rng(sum(nf) + sum(nt))
    count = 4
    shape_f = (count,) + ((nf[2],) if d == 3 else ()) + (nf[1], (nf[0] + 1) // 2)
    x = rng.normal(size=shape_f) + 1j * rng.normal(size=shape_f)
    cdt, p = (torch.complex128, hb.HOM_FP64) if prec == "fp64" else (torch.complex64, hb.HOM_FP32)
    dx = torch.from_numpy(x).to(cdt).cuda()
    shape_t = (count,) + ((nt[2],) if d == 3 else ()) + (nt[1], (nt[0] + 1) // 2)
    out = torch.full(shape_t, 7.0, dtype=cdt, device="cuda")
    hb.binding.hom_resample_fields(ctx, d, nf, nt, count, p, dx.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    ref = _resample_ref(dx.cpu().numpy(), d, nf, nt)
    assert np.array_equal(out.cpu().numpy().reshape(ref.shape), ref)
    with pytest.raises(hb.HombError):
        hb.binding.hom_resample_fields(ctx, d, nf, nt, count, p, dx.data_ptr(), dx.data_ptr())


# ----------------------------------------------------------------------------------
# the learned start inside the library: network files, hom_opts.warm_start, energy bounds
# ----------------------------------------------------------------------------------
def _python_start(hb, ctx, cfg, params, p):
    """The learned start chained call by call: features, forward on the cell's grid, half
    spectra (FP64) -- what hom_bounds does itself with warm_start = 1."""
    d = p.d
    N = int(p.N[0])
    feat = torch.empty((1,) + (N,) * d + (1,), dtype=torch.float32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    hb.binding.hom_net_features(ctx, [p], feat.data_ptr(), ws.data_ptr(), ws.numel())
    c = hb.binding.net_config(N, 1, cfg.width, cfg.modes, cfg.layers, cfg.proj, cfg.cout, d)
    _, nws = hb.binding.hom_net_sizes(ctx, c, 1)
    nw = torch.empty(nws, dtype=torch.uint8, device="cuda")
    pred = torch.empty((1,) + (N,) * d + (cfg.cout,), dtype=torch.float32, device="cuda")
    hb.binding.hom_net_forward(ctx, c, params.data_ptr(), 1, feat.data_ptr(), pred.data_ptr(), nw.data_ptr(), nws)
    half = torch.empty((2, d, d) + (N,) * (d - 1) + ((N + 1) // 2,), dtype=torch.complex128, device="cuda")
    hb.binding.hom_grid_to_half(ctx, d, N, 1, cfg.cout, pred.data_ptr(), half.data_ptr(), hb.HOM_FP64)
    return half


@pytest.mark.parametrize("d,N,train_N", [(2, 23, 15), (3, 13, 9)])
def test_learned_start_inside_hom_bounds(hb, tmp_path, d, N, train_N):
    """A network saved to a file and loaded back gives, through hom_opts.warm_start, the same
    bounds and iterations (1e-12) as the same start chained call by call; its grid need not be
    the one in the file's config."""
    solver = hb.Bounds(0)
    ctx = solver.ctx
    net = None
    try:
        cfg = hb.binding.net_config(train_N, 1, 8, 3, 2, 24, 2 * d * d, d)
        npar, _ = hb.binding.hom_net_sizes(ctx, cfg, 1)
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        hb.binding.hom_net_init(ctx, cfg, 11, params.data_ptr())
        path = str(tmp_path / "net.bin")
        hb.binding.hom_net_save(ctx, cfg, params.data_ptr(), path)
        net = hb.binding.hom_net_load(ctx, path)
        got_cfg, got_n = hb.binding.hom_net_info(net)
        assert got_n == npar and (got_cfg.N, got_cfg.width, got_cfg.cout, got_cfg.d) == (train_N, 8, 2 * d * d, d)
        p = ms.random_rectangles_2d(21, N=N) if d == 2 else ms.random_spheres_3d(4, N=N, n_balls=5, phi=0.25,
                                                                                contrast=100.0)
        for prec in (hb.HOM_FP64, hb.HOM_MIXED):
            x0 = _python_start(hb, ctx, cfg, params, p)
            ref = solver(p, precision=prec, tol=1e-8, x0=x0)
            for rep in range(2):        # the second call finds the parameters resident
                out = solver(p, precision=prec, tol=1e-8, net=net)
                for key in ("upper", "lower"):
                    assert np.abs(out[key] - ref[key]).max() <= 1e-12 * np.abs(ref[key]).max(), (prec, key)
                assert out["report"]["iters"] == ref["report"]["iters"]
        # a different problem in between on the same workspace: the parameters are uploaded again
        solver(ms.cube_inclusion_3d(N=11) if d == 2 else ms.square_inclusion_2d(N=31), precision=hb.HOM_FP64)
        out = solver(p, precision=hb.HOM_FP64, tol=1e-8, net=net)
        ref = solver(p, precision=hb.HOM_FP64, tol=1e-8, x0=_python_start(hb, ctx, cfg, params, p))
        assert np.abs(out["upper"] - ref["upper"]).max() <= 1e-12 * np.abs(ref["upper"]).max()
    finally:
        if net:
            hb.binding.hom_net_free(net)
        solver.close()


def _python_batch_start(hb, ctx, cfg, params, probs, prec, chunk):
    """The learned start of a batch chained call by call, the network run on chunks of
    `chunk` cells: what hom_bounds_batched does itself with warm_start = 1."""
    n, N = len(probs), int(probs[0].N[0])
    feat = torch.empty((n, N, N, 1), dtype=torch.float32, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    hb.binding.hom_net_features(ctx, probs, feat.data_ptr(), ws.data_ptr(), ws.numel())
    c = hb.binding.net_config(N, 1, cfg.width, cfg.modes, cfg.layers, cfg.proj, cfg.cout, 2)
    _, nws = hb.binding.hom_net_sizes(ctx, c, chunk)
    nw = torch.empty(nws, dtype=torch.uint8, device="cuda")
    pred = torch.empty((chunk, N, N, cfg.cout), dtype=torch.float32, device="cuda")
    f32 = prec == hb.HOM_MIXED
    half = torch.empty((n, 2, 2, 2, N, (N + 1) // 2), dtype=torch.complex64 if f32 else torch.complex128,
                       device="cuda")
    for c0 in range(0, n, chunk):
        nb = min(chunk, n - c0)
        fc = feat[c0:c0 + nb].contiguous()
        hb.binding.hom_net_forward(ctx, c, params.data_ptr(), nb, fc.data_ptr(), pred.data_ptr(), nw.data_ptr(), nws)
        hb.binding.hom_grid_to_half(ctx, 2, N, nb, cfg.cout, pred.data_ptr(), half[c0:c0 + nb].data_ptr(),
                                    hb.HOM_FP32 if f32 else hb.HOM_FP64)
    return half


def test_learned_start_inside_hom_bounds_batched(hb, tmp_path):
    """hom_bounds_batched with warm_start = 1 gives the same bounds (1e-12) and iterations as
    the same start chained call by call and passed as starting fields, in both precisions,
    with the network run on the whole batch or on chunks of 3 cells (a ragged last chunk);
    cells of different N in one batch, or starting fields together with the network, are
    refused."""
    solver = hb.Bounds(0)
    ctx = solver.ctx
    net = None
    try:
        cfg = hb.binding.net_config(15, 1, 8, 3, 2, 24, 8, 2)
        npar, _ = hb.binding.hom_net_sizes(ctx, cfg, 1)
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        hb.binding.hom_net_init(ctx, cfg, 13, params.data_ptr())
        path = str(tmp_path / "net.bin")
        hb.binding.hom_net_save(ctx, cfg, params.data_ptr(), path)
        net = hb.binding.hom_net_load(ctx, path)
        probs = [ms.random_rectangles_2d(40 + i, N=23) for i in range(7)]
        for chunk in (0, 3):
            hb.binding.hom_set_net_chunk(ctx, chunk)
            for prec, tol in ((hb.HOM_FP64, 1e-8), (hb.HOM_MIXED, 1e-5)):
                x0 = _python_batch_start(hb, ctx, cfg, params, probs, prec, chunk or len(probs))
                ref = solver.batched(probs, precision=prec, tol=tol, x0=x0)
                out = solver.batched(probs, precision=prec, tol=tol, net=net)
                for key in ("upper", "lower"):
                    assert np.abs(out[key] - ref[key]).max() <= 1e-12 * np.abs(ref[key]).max(), (chunk, prec, key)
                assert np.array_equal(out["iters"], ref["iters"]), (chunk, prec)
                zero = solver.batched(probs, precision=prec, tol=tol)
                assert not np.array_equal(out["iters"], zero["iters"])
        hb.binding.hom_set_net_chunk(ctx, 0)
        mixed = probs[:2] + [ms.random_rectangles_2d(3, N=25)]
        with pytest.raises(hb.HombError) as e:
            solver.batched(mixed, precision=hb.HOM_FP64, net=net)
        assert e.value.status == hb.binding.HOM_ERR_INVALID_ARG
        x0 = torch.zeros((7, 2, 2, 2, 23, 12), dtype=torch.complex128, device="cuda")
        with pytest.raises(hb.HombError):
            solver.batched(probs, precision=hb.HOM_FP64, x0=x0, net=net)
    finally:
        if net:
            hb.binding.hom_net_free(net)
        solver.close()


def test_network_file_is_checked(hb, tmp_path):
    ctx = hb.hom_create(0)
    try:
        cfg = hb.binding.net_config(9, 1, 4, 2, 1, 8, 8, 2)
        npar, _ = hb.binding.hom_net_sizes(ctx, cfg, 1)
        params = torch.empty(npar, dtype=torch.float32, device="cuda")
        hb.binding.hom_net_init(ctx, cfg, 2, params.data_ptr())
        path = tmp_path / "net.bin"
        hb.binding.hom_net_save(ctx, cfg, params.data_ptr(), str(path))
        raw = bytearray(path.read_bytes())
        raw[60] ^= 0x40                            # one parameter bit: the checksum fails
        bad = tmp_path / "bad.bin"
        bad.write_bytes(bytes(raw))
        for f in (bad, tmp_path / "missing.bin"):
            with pytest.raises(hb.HombError) as e:
                hb.binding.hom_net_load(ctx, str(f))
            assert e.value.status == hb.binding.HOM_ERR_INVALID_ARG
    finally:
        hb.hom_destroy(ctx)


def test_learned_start_needs_a_fitting_network(hb, tmp_path):
    solver = hb.Bounds(0)
    net = None
    try:
        cfg = hb.binding.net_config(9, 1, 4, 2, 1, 8, 8, 2)      # a 2D network
        npar, _ = hb.binding.hom_net_sizes(solver.ctx, cfg, 1)
        params = torch.zeros(npar, dtype=torch.float32, device="cuda")
        path = str(tmp_path / "net.bin")
        hb.binding.hom_net_save(solver.ctx, cfg, params.data_ptr(), path)
        net = hb.binding.hom_net_load(solver.ctx, path)
        for p, kw in ((ms.cube_inclusion_3d(N=9), {}), (ms.square_inclusion_2d(N=9), {"discretization": 1}),
                      (ms.make_problem(2, (9, 11), 1.0, 1.0, []), {})):
            with pytest.raises(hb.HombError) as e:
                solver(p, precision=hb.HOM_FP64, net=net, **kw)
            assert e.value.status == hb.binding.HOM_ERR_INVALID_ARG
        # an all-zero network predicts zero: the start is x0 = 0, the plain solve
        p = ms.square_inclusion_2d(N=9)
        a = solver(p, precision=hb.HOM_FP64, tol=1e-10, net=net)
        b = solver(p, precision=hb.HOM_FP64, tol=1e-10)
        assert np.abs(a["upper"] - b["upper"]).max() <= 1e-12
    finally:
        if net:
            hb.binding.hom_net_free(net)
        solver.close()


def test_energy_bounds(hb):
    import oracle
    solver = hb.Bounds(0)
    try:
        p = ms.random_anisotropic_2d(5, N=11)
        ref = oracle.dense_bounds(p)
        opts = hb.make_opts(hb.HOM_FP64, 1e-12)
        nws = hb.hom_workspace_size(solver.ctx, p, opts)
        ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
        for E in ([1.0, 0.0], [0.3, -0.7], [2.0, 1.0]):
            up, lo = hb.binding.hom_energy_bounds(solver.ctx, p, opts, ws.data_ptr(), nws, E)
            Ev = np.asarray(E)
            assert abs(up - Ev @ ref["upper"] @ Ev) <= 1e-10 * abs(Ev @ ref["upper"] @ Ev)
            assert abs(lo - Ev @ ref["lower"] @ Ev) <= 1e-10 * abs(Ev @ ref["lower"] @ Ev)
            assert lo <= up
    finally:
        solver.close()
